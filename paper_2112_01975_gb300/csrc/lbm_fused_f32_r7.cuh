// Fused single-pass step, D3Q27 tiles of 32 x 7 nodes (namespace lbmf7):
// 224 threads per CTA. At 128^3 its 4 x 19 x 4 tiles fill the 304 slots of
// two CTAs per SM in one wave, where 32 x 8 tiles leave 48 SMs with one
// CTA; `lbm_autotune` picks the tile height per lattice. The code is in
// lbm_fused_f32_body.cuh.
#pragma once

#define LBMF_NS lbmf7
#define LBMF_ROWS 7
#include "lbm_fused_f32_body.cuh"
#undef LBMF_NS
#undef LBMF_ROWS
