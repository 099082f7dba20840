// Launcher of the TMA-staged fused FP32 step (k_step_f32_wstma), compiled in
// its own translation unit (lbm_step_tma.cu): one kernel per equation of
// state and solid-node mode, 2 x 6 instantiations, built in parallel with
// the rest of the library. Internal to the library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_fused_f32.cuh"

namespace lbmtma {

// One step of the D3Q27 FP32 lattice g from src to dst on stream s: grid
// (ceil(nx/32), ceil(ny/8), ceil(nz/chunk)), 512 threads, sizeof(SharedWT<1>)
// bytes of dynamic shared memory; maps describe src. mask (device, one byte
// per node) is read only when `solid`. The equation of state is p.eos.
void launch(const lbmf::GeoF &g, const lbmf::PhysF &p, const uint8_t *mask, const lbmf::BoxMaps &maps,
            const float *src, float *dst, int *status, bool solid, cudaStream_t s);

// The same for shifted 16-bit storage (ST __half or __nv_bfloat16): src/dst
// the stored values, rho_src/rho_dst their source densities; the equation
// of state is taken from p.eos at run time.
template <typename ST>
void launch_shifted(const lbmf::GeoF &g, const lbmf::PhysF &p, const uint8_t *mask, const lbmf::BoxMaps &maps,
                    const ST *src, ST *dst, const float *rho_src, float *rho_dst, int *status, bool solid,
                    cudaStream_t s);

// The one-thread-group Tensor Memory form of the shifted step with TMA-staged
// planes (k_step_shifted_tmtma): the same arguments; 256 threads and
// sizeof(SharedSB<1, ST>) bytes of shared memory per block, two per SM.
template <typename ST>
void launch_shifted_tm(const lbmf::GeoF &g, const lbmf::PhysF &p, const uint8_t *mask, const lbmf::BoxMaps &maps,
                       const ST *src, ST *dst, const float *rho_src, float *rho_dst, int *status, bool solid,
                       cudaStream_t s);

}  // namespace lbmtma
