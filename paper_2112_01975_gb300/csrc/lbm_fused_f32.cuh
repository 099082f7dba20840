// Fused single-pass step, D3Q27 tiles of 32 x 8 nodes (namespace lbmf; the
// D2Q9 tile is a 128-wide row in every build). The code is in
// lbm_fused_f32_body.cuh.
#pragma once

#define LBMF_NS lbmf
#define LBMF_ROWS 8
#include "lbm_fused_f32_body.cuh"
#undef LBMF_NS
#undef LBMF_ROWS
