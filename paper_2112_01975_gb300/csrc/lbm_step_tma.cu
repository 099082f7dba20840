// The TMA-staged fused FP32 step's instantiations and launcher (see
// lbm_step_tma.h; the kernel itself is in lbm_fused_f32_body.cuh).
#include "lbm_step_tma.h"

#include <atomic>

namespace lbmtma {
namespace {

template <bool MASK, int EOSK>
void launch_k(const lbmf::GeoF &g, const lbmf::PhysF &p, const uint8_t *mask, const lbmf::BoxMaps &maps,
              const float *src, float *dst, int *status, cudaStream_t s)
{
    static std::atomic<unsigned long long> done{0};   // devices whose kernel is opted in
    using L = lbmf::LatF<1>;
    const int bytes = (int)sizeof(lbmf::SharedWT<1>);
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {   // more than 48 KB of dynamic shared memory
        cudaFuncSetAttribute(lbmf::k_step_f32_wstma<1, MASK, EOSK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
        done.fetch_or(bit);
    }
    const dim3 grid((g.nx + L::TX - 1) / L::TX, (g.ny + L::TY - 1) / L::TY, (g.nz + g.chunk - 1) / g.chunk);
    lbmf::k_step_f32_wstma<1, MASK, EOSK><<<grid, 2 * L::TX * L::TY, bytes, s>>>(g, p, mask, maps, src, dst,
                                                                                 status);
}

template <bool MASK>
void launch_m(const lbmf::GeoF &g, const lbmf::PhysF &p, const uint8_t *mask, const lbmf::BoxMaps &maps,
              const float *src, float *dst, int *status, cudaStream_t s)
{
    switch (p.eos) {
    case 0: launch_k<MASK, 0>(g, p, mask, maps, src, dst, status, s); break;
    case 1: launch_k<MASK, 1>(g, p, mask, maps, src, dst, status, s); break;
    case 2: launch_k<MASK, 2>(g, p, mask, maps, src, dst, status, s); break;
    case 4: launch_k<MASK, 4>(g, p, mask, maps, src, dst, status, s); break;
    case 5: launch_k<MASK, 5>(g, p, mask, maps, src, dst, status, s); break;
    default: launch_k<MASK, 3>(g, p, mask, maps, src, dst, status, s); break;   // CS
    }
}

template <typename ST, bool MASK>
void launch_s(const lbmf::GeoF &g, const lbmf::PhysF &p, const uint8_t *mask, const lbmf::BoxMaps &maps,
              const ST *src, ST *dst, const float *rho_src, float *rho_dst, int *status, cudaStream_t s)
{
    static std::atomic<unsigned long long> done{0};   // devices whose kernel is opted in
    using L = lbmf::LatF<1>;
    const int bytes = (int)sizeof(lbmf::SharedSWT<1, ST>);
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
        cudaFuncSetAttribute(lbmf::k_step_shifted_wstma<1, ST, MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
        done.fetch_or(bit);
    }
    const dim3 grid((g.nx + L::TX - 1) / L::TX, (g.ny + L::TY - 1) / L::TY, (g.nz + g.chunk - 1) / g.chunk);
    lbmf::k_step_shifted_wstma<1, ST, MASK><<<grid, 2 * L::TX * L::TY, bytes, s>>>(g, p, mask, maps, src, dst,
                                                                                   rho_src, rho_dst, status);
}

template <typename ST, bool MASK>
void launch_t(const lbmf::GeoF &g, const lbmf::PhysF &p, const uint8_t *mask, const lbmf::BoxMaps &maps,
              const ST *src, ST *dst, const float *rho_src, float *rho_dst, int *status, cudaStream_t s)
{
    static std::atomic<unsigned long long> done{0};   // devices whose kernel is opted in
    using L = lbmf::LatF<1>;
    const int bytes = (int)sizeof(lbmf::SharedSB<1, ST>);
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
        cudaFuncSetAttribute(lbmf::k_step_shifted_tmtma<1, ST, MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
        done.fetch_or(bit);
    }
    const dim3 grid((g.nx + L::TX - 1) / L::TX, (g.ny + L::TY - 1) / L::TY, (g.nz + g.chunk - 1) / g.chunk);
    lbmf::k_step_shifted_tmtma<1, ST, MASK><<<grid, L::TX * L::TY, bytes, s>>>(g, p, mask, maps, src, dst,
                                                                              rho_src, rho_dst, status);
}

}  // namespace

template <typename ST>
void launch_shifted_tm(const lbmf::GeoF &g, const lbmf::PhysF &p, const uint8_t *mask, const lbmf::BoxMaps &maps,
                       const ST *src, ST *dst, const float *rho_src, float *rho_dst, int *status, bool solid,
                       cudaStream_t s)
{
    if (solid) launch_t<ST, true>(g, p, mask, maps, src, dst, rho_src, rho_dst, status, s);
    else       launch_t<ST, false>(g, p, mask, maps, src, dst, rho_src, rho_dst, status, s);
}

template void launch_shifted_tm<__half>(const lbmf::GeoF &, const lbmf::PhysF &, const uint8_t *,
                                        const lbmf::BoxMaps &, const __half *, __half *, const float *, float *,
                                        int *, bool, cudaStream_t);
template void launch_shifted_tm<__nv_bfloat16>(const lbmf::GeoF &, const lbmf::PhysF &, const uint8_t *,
                                               const lbmf::BoxMaps &, const __nv_bfloat16 *, __nv_bfloat16 *,
                                               const float *, float *, int *, bool, cudaStream_t);

template <typename ST>
void launch_shifted(const lbmf::GeoF &g, const lbmf::PhysF &p, const uint8_t *mask, const lbmf::BoxMaps &maps,
                    const ST *src, ST *dst, const float *rho_src, float *rho_dst, int *status, bool solid,
                    cudaStream_t s)
{
    if (solid) launch_s<ST, true>(g, p, mask, maps, src, dst, rho_src, rho_dst, status, s);
    else       launch_s<ST, false>(g, p, mask, maps, src, dst, rho_src, rho_dst, status, s);
}

template void launch_shifted<__half>(const lbmf::GeoF &, const lbmf::PhysF &, const uint8_t *,
                                     const lbmf::BoxMaps &, const __half *, __half *, const float *, float *,
                                     int *, bool, cudaStream_t);
template void launch_shifted<__nv_bfloat16>(const lbmf::GeoF &, const lbmf::PhysF &, const uint8_t *,
                                            const lbmf::BoxMaps &, const __nv_bfloat16 *, __nv_bfloat16 *,
                                            const float *, float *, int *, bool, cudaStream_t);

void launch(const lbmf::GeoF &g, const lbmf::PhysF &p, const uint8_t *mask, const lbmf::BoxMaps &maps,
            const float *src, float *dst, int *status, bool solid, cudaStream_t s)
{
    if (solid) launch_m<true>(g, p, mask, maps, src, dst, status, s);
    else       launch_m<false>(g, p, mask, maps, src, dst, status, s);
}

}  // namespace lbmtma
