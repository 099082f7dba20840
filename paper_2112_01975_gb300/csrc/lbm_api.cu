// C ABI of the two-phase lattice Boltzmann library (declared in include/lbm.h).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "lbm.h"
#include "lbm_fused_f32.cuh"
#include "lbm_fused_f32_r7.cuh"
#include "lbm_kernels.cuh"
#include "lbm_step_tma.h"

using lbmk::Geo;
using lbmk::Phys;
using lbmf::GeoF;
using lbmf::PhysF;

struct lbm_ctx {
    int lattice, D, Q;
    Geo geo;
    Phys phys;
    GeoF geof;     // FP32 fused step: 3D frame (D2Q9: ny = 1, nz = 2D y extent)
    PhysF physf;
    int tile_rows = 8;   // D3Q27 FP32 step: 32 x 8 (lbmf) or 32 x 7 (lbmf7) tiles
    int variant = LBM_FUSED_PLAIN;   // FP32 step: plain, warp-specialised or Tensor Memory form
    bool e64 = false;    // reduced storage: EOS, psi and force sums in FP64 (LBM_FLAG_EOS_F64)
    int storage, flags;
    double t_over_tc, tau;
    std::vector<uint8_t> mask_host, zsolid_host;
    bool any_solid = false;
    int device;
    cudaStream_t own_stream = nullptr, stream = nullptr, cap_stream = nullptr;
    // device memory
    void *base = nullptr;
    bool owns_base = false;
    size_t bytes = 0;
    void *fv[2] = {nullptr, nullptr};   // population buffers (double, float or 16-bit)
    float *rs[2] = {nullptr, nullptr};  // shifted storage: source densities of buffer k
    double2 *rp = nullptr;
    double *u = nullptr, *gflux = nullptr, *partial = nullptr, *sums = nullptr;
    uint8_t *mask = nullptr;
    int *status = nullptr;
    int cur = 0;
    bool initialised = false, bad = false;
    cudaGraphExec_t graph = nullptr;
    int64_t launches = 0;
    // status polling of long lbm_step calls: a pinned copy of the status word
    // and the event that marks its arrival
    int *poll_host = nullptr;
    cudaEvent_t poll_ev = nullptr;
    bool poll_pending = false;
    // D3Q27, FP32 with nx % 4 == 0 or shifted 16-bit with nx % 8 == 0: the
    // two population buffers as 4D tensors (x, y, z, i) for the TMA-staged
    // form (LBM_FUSED_WS_TMA)
    lbmf::BoxMaps tmaps[2];
    bool tmap_ready = false;
    // interpolated bounce-back: boundary nodes, their active links, wall distances
    int nb = 0;
    unsigned *bn = nullptr, *bmask = nullptr;
    double *bq = nullptr;
    char err[512] = {0};
};

namespace {

// Opt a kernel in to more than 48 KB of dynamic shared memory, once per
// device (the attribute belongs to the device the call runs on).
template <typename Kern>
void smem_opt_in(Kern kernel, int bytes, std::atomic<unsigned long long> &done)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done.fetch_or(bit);
}

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t f0, f1, rs0, rs1, rp, u, g, mask, zs, partial, sums, status, total;
};

bool shifted(int storage) { return storage == LBM_F16S || storage == LBM_BF16S; }

size_t pop_bytes(int storage)
{
    return storage == LBM_F64 ? sizeof(double) : storage == LBM_F32 ? sizeof(float) : 2;
}

// planes: the fused step's march-axis extent (nz; ny for D2Q9).
Layout layout_for(int D, int Q, size_t N, int storage, size_t planes)
{
    Layout L;
    size_t o = 0;
    const size_t pb = pop_bytes(storage);
    // Either buffer, when it is the dead one between steps, also stages host
    // I/O: (1 + 2D) doubles per node (more than 9 floats on D2Q9).
    const size_t fb = pb * Q * N > sizeof(double) * (1 + 2 * D) * N ? pb * Q * N
                                                                   : sizeof(double) * (1 + 2 * D) * N;
    L.f0 = o; o = align_up(o + fb);
    L.f1 = o; o = align_up(o + fb);
    const size_t rsb = (storage == LBM_F16S || storage == LBM_BF16S) ? sizeof(float) * N : 0;
    L.rs0 = o; o = align_up(o + rsb);
    L.rs1 = o; o = align_up(o + rsb);
    L.rp = o; o = align_up(o + sizeof(double2) * N);
    L.u = o; o = align_up(o + sizeof(double) * D * N);
    L.g = o; o = align_up(o + sizeof(double) * D * N);
    L.mask = o; o = align_up(o + N);
    L.zs = o; o = align_up(o + planes);   // per-plane solid flags
    L.partial = o; o = align_up(o + sizeof(double) * 4 * lbmk::RED_BLOCKS);
    L.sums = o; o = align_up(o + sizeof(double) * 4);
    L.status = o; o = align_up(o + sizeof(int) * 4);
    L.total = o;
    return L;
}

bool valid_shape(int lattice, int nx, int ny, int nz)
{
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q27) return false;
    if (nx < 5 || ny < 5) return false;
    if (lattice == LBM_D2Q9 && nz != 1) return false;
    if (lattice == LBM_D3Q27 && nz < 5) return false;
    // 32-bit node indices in the kernels
    if ((double)nx * ny * nz * 27.0 > 4.0e9) return false;
    return true;
}

int fail(lbm_ctx *h, int code, const char *fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CU(h, call)                                                                      \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail((h), LBM_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                             \
    } while (0)

double eos_rtc(int eos, double a, double b)
{
    switch (eos) {
    case LBM_EOS_VDW: return 8.0 * a / (27.0 * b);
    case LBM_EOS_PR: return (0.0778 / 0.45724) * a / b;
    case LBM_EOS_RKS: return (0.08664 / 0.42748) * a / b;
    case LBM_EOS_CS: return (0.18727 / 0.4963) * a / b;
    case LBM_EOS_SC1: return -4.0;          // critical coupling G_c (Appendix G)
    case LBM_EOS_SC2: return -std::exp(2.0);
    }
    return NAN;
}

// The EOS's temperature parameter at T/Tc: R T for the cubic equations, the
// coupling G = G_c / (T/Tc) for Shan-Chen (kept in the RT slot).
double eos_temperature(int eos, double a, double b, double tr)
{
    const double c = eos_rtc(eos, a, b);
    return eos >= LBM_EOS_SC1 ? c / tr : tr * c;
}

double eos_alpha(int eos, double acentric, double tr)
{
    double m;
    if (eos == LBM_EOS_PR) m = 0.37464 + 1.54226 * acentric - 0.26992 * acentric * acentric;
    else if (eos == LBM_EOS_RKS) m = 0.480 + 1.574 * acentric - 0.176 * acentric * acentric;
    else return 1.0;
    const double s = 1.0 + m * (1.0 - std::sqrt(tr));
    return s * s;
}

// P - rho/3 in FP64 on the host (the EOS of the solid nodes' virtual density
// for the FP64-EOS form of the reduced-precision steps).
double excess_pressure_host(int eos, double a, double b, double RT, double aalpha, double r)
{
    const double br = b * r, rt = r * RT;
    double P;
    switch (eos) {
    case LBM_EOS_VDW: P = rt / (1.0 - br) - a * r * r; break;
    case LBM_EOS_PR: P = (rt * (1.0 + br * (2.0 - br)) - aalpha * r * r * (1.0 - br)) /
                         ((1.0 - br) * (1.0 + br * (2.0 - br))); break;
    case LBM_EOS_RKS: P = (rt * (1.0 + br) - aalpha * r * r * (1.0 - br)) / ((1.0 - br) * (1.0 + br)); break;
    case LBM_EOS_SC1: { const double q = 1.0 - std::exp(-r); P = r / 3.0 + RT / 6.0 * q * q; break; }
    case LBM_EOS_SC2: { const double q = std::exp(-1.0 / r); P = r / 3.0 + RT / 6.0 * q * q; break; }
    default: {
        const double e = 0.25 * br, om = 1.0 - e;
        P = rt * (1.0 + e + e * e - e * e * e) / (om * om * om) - a * r * r;
    }
    }
    return P - r / 3.0;
}

dim3 node_block(const Geo &g)
{
    int bx = g.nx >= 128 ? 128 : ((g.nx + 31) / 32) * 32;
    return dim3(bx, 1, 1);
}

dim3 node_grid(const Geo &g)
{
    dim3 b = node_block(g);
    return dim3((g.nx + b.x - 1) / b.x, g.ny, g.nz);
}

void make_tensor_maps(lbm_ctx *h);

int ensure_memory(lbm_ctx *h)
{
    if (h->fv[0]) return LBM_OK;
    Layout L = layout_for(h->D, h->Q, h->geo.N, h->storage, h->geof.nz);
    if (!h->base) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, LBM_ENOMEM, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e));
        }
        h->base = p;
        h->owns_base = true;
        h->bytes = L.total;
    }
    char *b = static_cast<char *>(h->base);
    h->fv[0] = b + L.f0;
    h->fv[1] = b + L.f1;
    if (shifted(h->storage)) {
        h->rs[0] = reinterpret_cast<float *>(b + L.rs0);
        h->rs[1] = reinterpret_cast<float *>(b + L.rs1);
    }
    h->rp = reinterpret_cast<double2 *>(b + L.rp);
    h->u = reinterpret_cast<double *>(b + L.u);
    h->gflux = reinterpret_cast<double *>(b + L.g);
    h->mask = reinterpret_cast<uint8_t *>(b + L.mask);
    h->geof.zsolid = reinterpret_cast<const uint8_t *>(b + L.zs);
    h->partial = reinterpret_cast<double *>(b + L.partial);
    h->sums = reinterpret_cast<double *>(b + L.sums);
    h->status = reinterpret_cast<int *>(b + L.status);
    CU(h, cudaMemcpyAsync(h->mask, h->mask_host.data(), h->geo.N, cudaMemcpyHostToDevice, h->stream));
    {   // planes of the fused step's march axis (z; the 2D y axis for D2Q9) that hold a solid
        const size_t plane = (size_t)h->geof.nx * h->geof.ny;
        h->zsolid_host.assign(h->geof.nz, 0);
        for (size_t n = 0; n < h->geo.N; ++n)
            if (h->mask_host[n]) h->zsolid_host[n / plane] = 1;
        CU(h, cudaMemcpyAsync(const_cast<uint8_t *>(h->geof.zsolid), h->zsolid_host.data(), h->geof.nz,
                              cudaMemcpyHostToDevice, h->stream));
    }
    CU(h, cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    make_tensor_maps(h);
    if (h->variant == LBM_FUSED_WS_TMA && !h->tmap_ready) h->variant = LBM_FUSED_WS_TMEM;
    if (h->variant == LBM_FUSED_TM_TMA && !h->tmap_ready) h->variant = LBM_FUSED_TMEM;
    return LBM_OK;
}

bool has_solid(const lbm_ctx *h) { return h->any_solid; }

// Row alignment the TMA-staged form needs: nx a multiple of 4 (FP32) or 8
// (16-bit shifted storage), so that rows start on 16 bytes.
int tma_nx_multiple(int storage) { return storage == LBM_F32 ? 4 : shifted(storage) ? 8 : 0; }

// The two population buffers of a D3Q27 FP32 or shifted-storage handle as
// 4D tensors (x, y, z, i) of the stored type, each with the five box shapes
// of the TMA-staged forms (32 x 8, 32 x 2, W x 8, W x 2 and the one-copy
// (32 + 2 W) x 12 nodes of one plane, all 27 populations; W = 16 bytes of
// the type). Needs nx a multiple
// of tma_nx_multiple (16-byte row strides) and the CUDA driver's tensor-map
// encoder, found through the runtime's entry-point query; leaves tmap_ready
// false when either is missing.
void make_tensor_maps(lbm_ctx *h)
{
    h->tmap_ready = false;
    const int mult = tma_nx_multiple(h->storage);
    if (h->lattice != LBM_D3Q27 || !mult || h->geo.nx % mult || !h->fv[0]) return;
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                CUtensorMapFloatOOBfill);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return;
    }
    const Geo &g = h->geo;
    const cuuint64_t es = pop_bytes(h->storage);
    const CUtensorMapDataType dt = h->storage == LBM_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : h->storage == LBM_F16S ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint32_t w = (cuuint32_t)(16 / es);
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 27};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * es, (cuuint64_t)g.nx * g.ny * es, (cuuint64_t)g.N * es};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int k = 0; k < 2; ++k) {
        CUtensorMap *m[5] = {&h->tmaps[k].mc, &h->tmaps[k].tc, &h->tmaps[k].ml, &h->tmaps[k].tl,
                             &h->tmaps[k].wide};
        const cuuint32_t wx[5] = {32, 32, w, w, 32 + 2 * w}, wy[5] = {8, 2, 8, 2, 12};
        for (int j = 0; j < 5; ++j) {
            const cuuint32_t box[4] = {wx[j], wy[j], 1, 27};
            if (reinterpret_cast<Encode>(fn)(m[j], dt, 4, h->fv[k], dims, strides, box, estr,
                                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return;
        }
    }
    h->tmap_ready = true;
}

double *f64(lbm_ctx *h, int k) { return static_cast<double *>(h->fv[k]); }
float *f32(lbm_ctx *h, int k) { return static_cast<float *>(h->fv[k]); }

template <int LAT>
dim3 fused_grid(const GeoF &g, int rows = lbmf::LatF<LAT>::TY)
{
    using L = lbmf::LatF<LAT>;
    const int ty = LAT == 1 ? rows : L::TY;
    return dim3((g.nx + L::TX - 1) / L::TX, (g.ny + ty - 1) / ty, (g.nz + g.chunk - 1) / g.chunk);
}

// The same parameters as the 7-row build's types (one source, one layout).
template <typename T, typename U>
T as_layout(const U &u)
{
    static_assert(sizeof(T) == sizeof(U), "same source, same layout");
    T t;
    memcpy(&t, &u, sizeof t);
    return t;
}

template <bool MASK>
void launch_fused_r7(lbm_ctx *h, cudaStream_t s, const float *src, float *dst)
{
    using L = lbmf7::LatF<1>;
    if (h->variant == LBM_FUSED_TMEM) {
        static std::atomic<unsigned long long> done{0};   // devices already opted in
        const int bytes = (int)sizeof(lbmf7::SharedF<1>);
        smem_opt_in(lbmf7::k_step_f32_tm<1, MASK>, bytes, done);
        lbmf7::k_step_f32_tm<1, MASK><<<fused_grid<1>(h->geof, L::TY), L::TX * L::TY, bytes, s>>>(
            as_layout<lbmf7::GeoF>(h->geof), as_layout<lbmf7::PhysF>(h->physf), h->mask, src, dst,
            h->status);
        return;
    }
    if (h->variant == LBM_FUSED_WARP_SPECIALISED) {
        static std::atomic<unsigned long long> done{0};   // devices already opted in
        const int bytes = (int)sizeof(lbmf7::SharedWS<1>);
        smem_opt_in(lbmf7::k_step_f32_ws<1, MASK>, bytes, done);
        lbmf7::k_step_f32_ws<1, MASK><<<fused_grid<1>(h->geof, L::TY), 2 * L::TX * L::TY, bytes, s>>>(
            as_layout<lbmf7::GeoF>(h->geof), as_layout<lbmf7::PhysF>(h->physf), h->mask, src, dst,
            h->status);
        return;
    }
    static std::atomic<unsigned long long> done{0};   // devices already opted in
    const int bytes = (int)sizeof(lbmf7::SharedF<1>);
    smem_opt_in(lbmf7::k_step_f32<1, MASK>, bytes, done);
    lbmf7::k_step_f32<1, MASK><<<fused_grid<1>(h->geof, L::TY), L::TX * L::TY, bytes, s>>>(
        as_layout<lbmf7::GeoF>(h->geof), as_layout<lbmf7::PhysF>(h->physf), h->mask, src, dst,
        h->status);
}

template <int LAT, bool MASK>
void launch_fused_tm(lbm_ctx *h, cudaStream_t s, const float *src, float *dst)
{
    static std::atomic<unsigned long long> done{0};   // devices already opted in
    using L = lbmf::LatF<LAT>;
    const int bytes = (int)sizeof(lbmf::SharedF<LAT>);
    smem_opt_in(lbmf::k_step_f32_tm<LAT, MASK>, bytes, done);
    lbmf::k_step_f32_tm<LAT, MASK><<<fused_grid<LAT>(h->geof), L::TX * L::TY, bytes, s>>>(
        h->geof, h->physf, h->mask, src, dst, h->status);
}

template <bool MASK>
void launch_fused_wstm(lbm_ctx *h, cudaStream_t s, const float *src, float *dst)
{
    static std::atomic<unsigned long long> done{0};   // devices already opted in
    using L = lbmf::LatF<1>;
    const int bytes = (int)sizeof(lbmf::SharedWS<1>);
    smem_opt_in(lbmf::k_step_f32_wstm<1, MASK>, bytes, done);
    lbmf::k_step_f32_wstm<1, MASK><<<fused_grid<1>(h->geof), 2 * L::TX * L::TY, bytes, s>>>(
        h->geof, h->physf, h->mask, src, dst, h->status);
}

template <int LAT, bool MASK>
void launch_fused_ws(lbm_ctx *h, cudaStream_t s, const float *src, float *dst)
{
    static std::atomic<unsigned long long> done{0};   // devices already opted in
    using L = lbmf::LatF<LAT>;
    const int bytes = (int)sizeof(lbmf::SharedWS<LAT>);
    smem_opt_in(lbmf::k_step_f32_ws<LAT, MASK>, bytes, done);
    lbmf::k_step_f32_ws<LAT, MASK><<<fused_grid<LAT>(h->geof), 2 * L::TX * L::TY, bytes, s>>>(
        h->geof, h->physf, h->mask, src, dst, h->status);
}

template <int LAT, bool MASK>
void launch_fused_e64(lbm_ctx *h, cudaStream_t s, const float *src, float *dst)
{
    static std::atomic<unsigned long long> done{0};   // devices already opted in
    using L = lbmf::LatF<LAT>;
    const int bytes = (int)sizeof(lbmf::SharedF<LAT>);
    smem_opt_in(lbmf::k_step_f32<LAT, MASK, true>, bytes, done);
    lbmf::k_step_f32<LAT, MASK, true><<<fused_grid<LAT>(h->geof), L::TX * L::TY, bytes, s>>>(
        h->geof, h->physf, h->mask, src, dst, h->status);
}

template <int LAT>
void launch_fused(lbm_ctx *h, cudaStream_t s, const float *src, float *dst)
{
    if (h->e64) {   // the plain 32 x 8 form only
        if (has_solid(h)) launch_fused_e64<LAT, true>(h, s, src, dst);
        else              launch_fused_e64<LAT, false>(h, s, src, dst);
        return;
    }
    if (LAT == 1 && h->tile_rows == 7) {
        if (has_solid(h)) launch_fused_r7<true>(h, s, src, dst);
        else              launch_fused_r7<false>(h, s, src, dst);
        return;
    }
    if (h->variant == LBM_FUSED_WARP_SPECIALISED) {
        if (has_solid(h)) launch_fused_ws<LAT, true>(h, s, src, dst);
        else              launch_fused_ws<LAT, false>(h, s, src, dst);
        return;
    }
    if (h->variant == LBM_FUSED_TMEM) {
        if (has_solid(h)) launch_fused_tm<LAT, true>(h, s, src, dst);
        else              launch_fused_tm<LAT, false>(h, s, src, dst);
        return;
    }
    if (LAT == 1 && h->variant == LBM_FUSED_WS_TMA) {   // D3Q27, 32 x 8 tiles, tensor maps made
        lbmtma::launch(h->geof, h->physf, h->mask, h->tmaps[src == h->fv[0] ? 0 : 1], src, dst, h->status,
                       has_solid(h), s);
        return;
    }
    if (LAT == 1 && h->variant == LBM_FUSED_WS_TMEM) {   // D3Q27, 32 x 8 tiles
        if (has_solid(h)) launch_fused_wstm<true>(h, s, src, dst);
        else              launch_fused_wstm<false>(h, s, src, dst);
        return;
    }
    static std::atomic<unsigned long long> done_m{0}, done_f{0};   // devices already opted in
    using L = lbmf::LatF<LAT>;
    const int bytes = (int)sizeof(lbmf::SharedF<LAT>);
    const dim3 gr = fused_grid<LAT>(h->geof);
    if (has_solid(h)) {
        smem_opt_in(lbmf::k_step_f32<LAT, true>, bytes, done_m);
        lbmf::k_step_f32<LAT, true><<<gr, L::TX * L::TY, bytes, s>>>(h->geof, h->physf, h->mask, src,
                                                                    dst, h->status);
    } else {
        smem_opt_in(lbmf::k_step_f32<LAT, false>, bytes, done_f);
        lbmf::k_step_f32<LAT, false><<<gr, L::TX * L::TY, bytes, s>>>(h->geof, h->physf, h->mask, src,
                                                                     dst, h->status);
    }
}

template <int LAT, typename ST, bool E64, bool MASK>
void launch_shifted_e(lbm_ctx *h, cudaStream_t s, int k)
{
    static std::atomic<unsigned long long> done{0};   // devices already opted in
    const int bytes = (int)sizeof(lbmf::SharedS<LAT>);
    smem_opt_in(lbmf::k_step_shifted<LAT, ST, E64, MASK>, bytes, done);
    using L = lbmf::LatF<LAT>;
    lbmf::k_step_shifted<LAT, ST, E64, MASK><<<fused_grid<LAT>(h->geof), L::TX * L::TY, bytes, s>>>(
        h->geof, h->physf, h->mask, static_cast<const ST *>(h->fv[k]), static_cast<ST *>(h->fv[k ^ 1]),
        h->rs[k], h->rs[k ^ 1], h->status);
}

template <int LAT, typename ST, bool MASK>
void launch_shifted_tm(lbm_ctx *h, cudaStream_t s, int k)
{
    static std::atomic<unsigned long long> done{0};   // devices already opted in
    const int bytes = (int)sizeof(lbmf::SharedS<LAT>);
    smem_opt_in(lbmf::k_step_shifted_tm<LAT, ST, MASK>, bytes, done);
    using L = lbmf::LatF<LAT>;
    lbmf::k_step_shifted_tm<LAT, ST, MASK><<<fused_grid<LAT>(h->geof), L::TX * L::TY, bytes, s>>>(
        h->geof, h->physf, h->mask, static_cast<const ST *>(h->fv[k]), static_cast<ST *>(h->fv[k ^ 1]),
        h->rs[k], h->rs[k ^ 1], h->status);
}

template <typename ST, bool MASK>
void launch_shifted_wstm(lbm_ctx *h, cudaStream_t s, int k)
{
    static std::atomic<unsigned long long> done{0};   // devices already opted in
    const int bytes = (int)sizeof(lbmf::SharedSWS<1>);
    smem_opt_in(lbmf::k_step_shifted_wstm<1, ST, MASK>, bytes, done);
    using L = lbmf::LatF<1>;
    lbmf::k_step_shifted_wstm<1, ST, MASK><<<fused_grid<1>(h->geof), 2 * L::TX * L::TY, bytes, s>>>(
        h->geof, h->physf, h->mask, static_cast<const ST *>(h->fv[k]), static_cast<ST *>(h->fv[k ^ 1]),
        h->rs[k], h->rs[k ^ 1], h->status);
}

template <int LAT, typename ST, bool MASK>
void launch_shifted_m(lbm_ctx *h, cudaStream_t s, int k)
{
    if (LAT == 1 && !h->e64 && h->variant == LBM_FUSED_WS_TMA) {   // tensor maps made
        lbmtma::launch_shifted(h->geof, h->physf, h->mask, h->tmaps[k], static_cast<const ST *>(h->fv[k]),
                               static_cast<ST *>(h->fv[k ^ 1]), h->rs[k], h->rs[k ^ 1], h->status, MASK, s);
        return;
    }
    if (LAT == 1 && !h->e64 && h->variant == LBM_FUSED_TM_TMA) {   // tensor maps made
        lbmtma::launch_shifted_tm(h->geof, h->physf, h->mask, h->tmaps[k], static_cast<const ST *>(h->fv[k]),
                                  static_cast<ST *>(h->fv[k ^ 1]), h->rs[k], h->rs[k ^ 1], h->status, MASK,
                                  s);
        return;
    }
    if (h->e64) launch_shifted_e<LAT, ST, true, MASK>(h, s, k);
    else if (h->variant == LBM_FUSED_TMEM) launch_shifted_tm<LAT, ST, MASK>(h, s, k);
    else if (LAT == 1 && h->variant == LBM_FUSED_WS_TMEM) launch_shifted_wstm<ST, MASK>(h, s, k);
    else launch_shifted_e<LAT, ST, false, MASK>(h, s, k);
}

template <int LAT, typename ST>
void launch_shifted_t(lbm_ctx *h, cudaStream_t s, int k)
{
    if (has_solid(h)) launch_shifted_m<LAT, ST, true>(h, s, k);
    else              launch_shifted_m<LAT, ST, false>(h, s, k);
}

template <int LAT>
void launch_shifted(lbm_ctx *h, cudaStream_t s, int k)
{
    if (h->storage == LBM_F16S) launch_shifted_t<LAT, __half>(h, s, k);
    else                        launch_shifted_t<LAT, __nv_bfloat16>(h, s, k);
}

// One time step; returns the number of kernels launched (0 on error).
template <int LAT>
int launch_step(lbm_ctx *h, cudaStream_t s, int *nk)
{
    if (shifted(h->storage)) {
        launch_shifted<LAT>(h, s, h->cur);
        *nk = 1;
    } else if (h->storage == LBM_F32) {
        launch_fused<LAT>(h, s, f32(h, h->cur), f32(h, h->cur ^ 1));
        *nk = 1;
    } else {
        const dim3 gr = node_grid(h->geo), bl = node_block(h->geo);
        const double *src = f64(h, h->cur);
        double *dst = f64(h, h->cur ^ 1);
        lbmk::k_macro<LAT><<<gr, bl, 0, s>>>(h->geo, h->phys, h->mask, src, h->rp, h->u,
                                             h->gflux, h->status);
        lbmk::k_collide<LAT><<<gr, bl, 0, s>>>(h->geo, h->phys, h->mask, src, dst, h->rp, h->u,
                                               h->gflux);
        *nk = 2;
    }
    if (h->nb > 0) {   // interpolated bounce-back on the new state
        const int th = 128, bl = (h->nb + th - 1) / th;
        if (h->storage == LBM_F32)
            lbmk::k_interp_bounce_back<LAT, float><<<bl, th, 0, s>>>(h->geo, h->bn, h->bmask, h->bq,
                                                                     h->nb, f32(h, h->cur ^ 1));
        else
            lbmk::k_interp_bounce_back<LAT, double><<<bl, th, 0, s>>>(h->geo, h->bn, h->bmask, h->bq,
                                                                      h->nb, f64(h, h->cur ^ 1));
        *nk += 1;
    }
    CU(h, cudaGetLastError());
    h->cur ^= 1;
    return LBM_OK;
}

int step_plain(lbm_ctx *h, cudaStream_t s, int *nk_out = nullptr)
{
    int nk = 0;
    int rc = h->lattice == LBM_D2Q9 ? launch_step<0>(h, s, &nk) : launch_step<1>(h, s, &nk);
    if (rc == LBM_OK) h->launches += nk;
    if (nk_out) *nk_out = nk;
    return rc;
}

int kernels_per_step(const lbm_ctx *h) { return (h->storage == LBM_F64 ? 2 : 1) + (h->nb > 0); }

// Shifted storage I/O goes through a temporary FP64 copy of the populations.
struct TempF64 {
    double *p = nullptr;
    ~TempF64() { if (p) cudaFree(p); }
};

template <int LAT>
int decode_to(lbm_ctx *h, int k, double *out)
{
    const dim3 gr = node_grid(h->geo), bl = node_block(h->geo);
    if (h->storage == LBM_F16S)
        lbmk::k_decode_shifted<LAT, __half><<<gr, bl, 0, h->stream>>>(
            h->geo, static_cast<const __half *>(h->fv[k]), h->rs[k], out);
    else
        lbmk::k_decode_shifted<LAT, __nv_bfloat16><<<gr, bl, 0, h->stream>>>(
            h->geo, static_cast<const __nv_bfloat16 *>(h->fv[k]), h->rs[k], out);
    CU(h, cudaGetLastError());
    h->launches += 1;
    return LBM_OK;
}

template <int LAT>
int encode_from(lbm_ctx *h, const double *f)
{
    const dim3 gr = node_grid(h->geo), bl = node_block(h->geo);
    // both buffers' source densities: -1 at solid nodes stays for good
    lbmk::k_density<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->mask, f, h->rs[0]);
    lbmk::k_density<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->mask, f, h->rs[1]);
    if (h->storage == LBM_F16S)
        lbmk::k_encode_shifted<LAT, __half><<<gr, bl, 0, h->stream>>>(
            h->geo, f, h->rs[0], static_cast<__half *>(h->fv[0]));
    else
        lbmk::k_encode_shifted<LAT, __nv_bfloat16><<<gr, bl, 0, h->stream>>>(
            h->geo, f, h->rs[0], static_cast<__nv_bfloat16 *>(h->fv[0]));
    CU(h, cudaGetLastError());
    h->launches += 3;
    h->cur = 0;
    return LBM_OK;
}

int temp_alloc(lbm_ctx *h, TempF64 &t)
{
    const size_t bytes = sizeof(double) * (size_t)h->Q * h->geo.N;
    if (cudaMalloc(&t.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        t.p = nullptr;
        return fail(h, LBM_ENOMEM, "no room for the FP64 copy of shifted populations");
    }
    return LBM_OK;
}

// Two steps (state buffer 0 -> 1 -> 0) captured once on the library's own
// stream; replayed on the handle's stream.
int ensure_graph(lbm_ctx *h)
{
    if (h->graph) return LBM_OK;
    if (!h->cap_stream) CU(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CU(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int saved = h->cur;
    int rc = step_plain(h, h->cap_stream);
    if (rc == LBM_OK) rc = step_plain(h, h->cap_stream);
    h->launches -= 2 * kernels_per_step(h);  // captured, not launched
    h->cur = saved;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return fail(h, LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

int read_status(lbm_ctx *h)
{
    int st = 0;
    CU(h, cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    if (st) {
        h->bad = true;
        if (st & 8)
            return fail(h, LBM_ECUDA, "the TMA-staged step found its shared memory not 128-byte aligned");
        if (st & 2)
            return fail(h, LBM_ETIMEOUT, "a wait between the fused step's thread groups timed out");
        return fail(h, LBM_ENONFINITE, "a density became non-finite or non-positive");
    }
    return LBM_OK;
}

int check_ready(lbm_ctx *h)
{
    if (!h) return LBM_EINVAL;
    if (!h->initialised) return fail(h, LBM_ESTATE, "handle not initialised (call lbm_init)");
    return LBM_OK;
}

template <int LAT>
int launch_macro_and_out(lbm_ctx *h, double *rho, double *u, double *U)
{
    const dim3 gr = node_grid(h->geo), bl = node_block(h->geo);
    if (shifted(h->storage)) {
        TempF64 t;
        int rc = temp_alloc(h, t);
        if (!rc) rc = decode_to<LAT>(h, h->cur, t.p);
        if (rc) return rc;
        lbmk::k_macro<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, t.p, h->rp, h->u,
                                                     h->gflux, h->status);
        CU(h, cudaStreamSynchronize(h->stream));   // before the temporary is freed
    } else if (h->storage == LBM_F32)
        lbmk::k_macro<LAT, float><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask,
                                                            f32(h, h->cur), h->rp, h->u,
                                                            h->gflux, h->status);
    else
        lbmk::k_macro<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, f64(h, h->cur),
                                                     h->rp, h->u, h->gflux, h->status);
    lbmk::k_moments_out<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, h->rp, h->u,
                                                       rho, u, U);
    CU(h, cudaGetLastError());
    h->launches += 2;
    return LBM_OK;
}

template <int LAT>
int launch_pressure(lbm_ctx *h, double *out)
{
    const dim3 gr = node_grid(h->geo), bl = node_block(h->geo);
    if (shifted(h->storage)) {
        TempF64 t;
        int rc = temp_alloc(h, t);
        if (!rc) rc = decode_to<LAT>(h, h->cur, t.p);
        if (rc) return rc;
        lbmk::k_macro<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, t.p, h->rp, h->u,
                                                     h->gflux, h->status);
        lbmk::k_pressure_tensor<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, t.p, h->rp, out);
        CU(h, cudaGetLastError());
        CU(h, cudaStreamSynchronize(h->stream));   // before the temporary is freed
    } else if (h->storage == LBM_F32) {
        lbmk::k_macro<LAT, float><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, f32(h, h->cur),
                                                            h->rp, h->u, h->gflux, h->status);
        lbmk::k_pressure_tensor<LAT, float><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask,
                                                                      f32(h, h->cur), h->rp, out);
    } else {
        lbmk::k_macro<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, f64(h, h->cur), h->rp,
                                                     h->u, h->gflux, h->status);
        lbmk::k_pressure_tensor<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask,
                                                               f64(h, h->cur), h->rp, out);
    }
    CU(h, cudaGetLastError());
    h->launches += 2;
    return LBM_OK;
}

template <int LAT>
int launch_init(lbm_ctx *h, const double *rho0, const double *u0)
{
    const dim3 gr = node_grid(h->geo), bl = node_block(h->geo);
    // side fields first: the initial force needs rho and s psi of every node
    lbmk::k_fill_solid<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, h->rp, h->u,
                                                      h->gflux);
    lbmk::k_init_density<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, rho0, h->rp);
    h->launches += 3;
    if (shifted(h->storage)) {
        TempF64 t;
        int rc = temp_alloc(h, t);
        if (rc) return rc;
        lbmk::k_init<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, h->rp, u0, t.p);
        rc = encode_from<LAT>(h, t.p);
        if (rc) return rc;
        CU(h, cudaGetLastError());
        CU(h, cudaStreamSynchronize(h->stream));   // before the temporary is freed
        return LBM_OK;
    }
    if (h->storage == LBM_F32)
        lbmk::k_init<LAT, float><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, h->rp, u0,
                                                           f32(h, h->cur));
    else
        lbmk::k_init<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, h->rp, u0,
                                                    f64(h, h->cur));
    CU(h, cudaGetLastError());
    return LBM_OK;
}

template <int LAT>
int launch_fill_solid(lbm_ctx *h)
{
    const dim3 gr = node_grid(h->geo), bl = node_block(h->geo);
    lbmk::k_fill_solid<LAT><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, h->rp, h->u,
                                                      h->gflux);
    CU(h, cudaGetLastError());
    h->launches += 1;
    return LBM_OK;
}

template <int LAT>
int launch_reduce(lbm_ctx *h)
{
    if (shifted(h->storage)) {
        TempF64 t;
        int rc = temp_alloc(h, t);
        if (!rc) rc = decode_to<LAT>(h, h->cur, t.p);
        if (rc) return rc;
        lbmk::k_reduce_partial<LAT><<<lbmk::RED_BLOCKS, lbmk::RED_THREADS, 0, h->stream>>>(
            h->geo, h->mask, t.p, h->partial);
        lbmk::k_reduce_final<<<1, lbmk::RED_BLOCKS, 0, h->stream>>>(h->partial, h->sums);
        CU(h, cudaGetLastError());
        CU(h, cudaStreamSynchronize(h->stream));
        h->launches += 2;
        return LBM_OK;
    }
    if (h->storage == LBM_F32)
        lbmk::k_reduce_partial<LAT, float><<<lbmk::RED_BLOCKS, lbmk::RED_THREADS, 0, h->stream>>>(
            h->geo, h->mask, f32(h, h->cur), h->partial);
    else
        lbmk::k_reduce_partial<LAT><<<lbmk::RED_BLOCKS, lbmk::RED_THREADS, 0, h->stream>>>(
            h->geo, h->mask, f64(h, h->cur), h->partial);
    lbmk::k_reduce_final<<<1, lbmk::RED_BLOCKS, 0, h->stream>>>(h->partial, h->sums);
    CU(h, cudaGetLastError());
    h->launches += 2;
    return LBM_OK;
}

// Status polling of long step sequences: every kPollReplays graph replays
// (2 steps each) the status word is copied to pinned host memory behind an
// event; before the next copy is queued the previous one is awaited, so the
// host runs at most one polling interval ahead of the device and a diverged
// lattice stops within two intervals.
constexpr int64_t kPollReplays = 32;

int ensure_poll(lbm_ctx *h)
{
    if (h->poll_host) return LBM_OK;
    CU(h, cudaHostAlloc(reinterpret_cast<void **>(&h->poll_host), sizeof(int), cudaHostAllocDefault));
    *h->poll_host = 0;
    CU(h, cudaEventCreateWithFlags(&h->poll_ev, cudaEventDisableTiming));
    return LBM_OK;
}

// Wait for the last queued status copy and act on it; queue the next one.
int poll_status(lbm_ctx *h)
{
    if (h->poll_pending) {
        CU(h, cudaEventSynchronize(h->poll_ev));
        h->poll_pending = false;
        if (*h->poll_host) {
            h->bad = true;
            return fail(h, LBM_ENONFINITE, "a density became non-finite or non-positive");
        }
    }
    CU(h, cudaMemcpyAsync(h->poll_host, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaEventRecord(h->poll_ev, h->stream));
    h->poll_pending = true;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_default_params(int eos, lbm_params *p)
{
    if (!p) return LBM_EINVAL;
    switch (eos) {
    case LBM_EOS_VDW: p->a = 9.0 / 49.0; p->b = 2.0 / 21.0; break;
    case LBM_EOS_PR:
    case LBM_EOS_RKS: p->a = 2.0 / 49.0; p->b = 2.0 / 21.0; break;
    case LBM_EOS_CS: p->a = 1.0; p->b = 4.0; break;
    case LBM_EOS_SC1:
    case LBM_EOS_SC2: p->a = 1.0; p->b = 1.0; break;   // not used by Shan-Chen
    default: return LBM_EINVAL;
    }
    p->acentric = 0.344;
    p->rho_w = 1.0;
    p->g[0] = p->g[1] = p->g[2] = 0.0;
    p->tau_v = 0.0;
    p->visc_rho[0] = 0.0;
    p->visc_rho[1] = 1.0;
    p->storage = LBM_F64;
    p->flags = 0;
    return LBM_OK;
}

size_t lbm_required_bytes(int lattice, int nx, int ny, int nz, int storage)
{
    if (!valid_shape(lattice, nx, ny, nz) || storage < LBM_F64 || storage > LBM_BF16S) return 0;
    const int D = lattice == LBM_D2Q9 ? 2 : 3, Q = lattice == LBM_D2Q9 ? 9 : 27;
    return layout_for(D, Q, (size_t)nx * ny * nz, storage, lattice == LBM_D2Q9 ? ny : nz).total;
}

int lbm_create(lbm_handle *out, int lattice, int nx, int ny, int nz, int eos, double t_over_tc,
               double kappa, double tau, const uint8_t *solid_mask, const lbm_params *p)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!valid_shape(lattice, nx, ny, nz)) return LBM_EINVAL;
    if (eos < LBM_EOS_VDW || eos > LBM_EOS_SC2) return LBM_EINVAL;
    if (!(t_over_tc > 0.0 && t_over_tc < 1.0) || !(kappa >= 0.0) || !(tau > 0.5)) return LBM_EINVAL;
    lbm_params prm;
    if (p) prm = *p;
    else lbm_default_params(eos, &prm);
    if (prm.storage < LBM_F64 || prm.storage > LBM_BF16S) return LBM_EINVAL;
    if (!(prm.a > 0.0) || !(prm.b > 0.0) || !(prm.rho_w > 0.0)) return LBM_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(prm.g[a])) return LBM_EINVAL;
    if (prm.tau_v != 0.0 && !(prm.tau_v > 0.5 && prm.visc_rho[0] > 0.0 &&
                              prm.visc_rho[1] > prm.visc_rho[0] && std::isfinite(prm.tau_v)))
        return LBM_EINVAL;
    lbm_ctx *h = new (std::nothrow) lbm_ctx();
    if (!h) return LBM_ENOMEM;
    h->lattice = lattice;
    h->D = lattice == LBM_D2Q9 ? 2 : 3;
    h->Q = lattice == LBM_D2Q9 ? 9 : 27;
    h->geo.nx = nx; h->geo.ny = ny; h->geo.nz = nz;
    h->geo.N = (unsigned)((size_t)nx * ny * nz);
    h->storage = prm.storage;
    h->flags = prm.flags;
    h->t_over_tc = t_over_tc;
    h->tau = tau;
    Phys &ph = h->phys;
    ph.eos = eos;
    ph.a = prm.a;
    ph.b = prm.b;
    ph.RT = eos_temperature(eos, prm.a, prm.b, t_over_tc);
    ph.alpha = eos_alpha(eos, prm.acentric, t_over_tc);
    ph.kappa = kappa;
    ph.omega = 1.0 / tau;
    ph.phi_pref = (prm.flags & LBM_FLAG_PHI_OFF) ? 0.0 : -(1.0 - 0.5 * ph.omega);
    ph.rho_w = prm.rho_w;
    for (int a = 0; a < 3; ++a) ph.g[a] = (a < (lattice == LBM_D2Q9 ? 2 : 3)) ? prm.g[a] : 0.0;
    ph.var_visc = prm.tau_v > 0.0 ? 1 : 0;
    ph.nu_l = (tau - 0.5) / 3.0;
    ph.nu_v = ph.var_visc ? (prm.tau_v - 0.5) / 3.0 : ph.nu_l;
    ph.visc_rv = prm.visc_rho[0];
    ph.visc_rl = prm.visc_rho[1];
    ph.phi_sign = (prm.flags & LBM_FLAG_PHI_OFF) ? 0.0 : -1.0;
    // FP32 fused step: D2Q9 runs in the 3D frame with one y row.
    h->geof.nx = nx;
    h->geof.ny = lattice == LBM_D2Q9 ? 1 : ny;
    h->geof.nz = lattice == LBM_D2Q9 ? ny : nz;
    h->geof.N = h->geo.N;
    h->geof.chunk = lattice == LBM_D2Q9 ? 64 : 16;
    PhysF &pf = h->physf;
    pf.eos = eos;
    pf.a = (float)ph.a;
    pf.b = (float)ph.b;
    pf.RT = (float)ph.RT;
    pf.aalpha = (float)(ph.a * ph.alpha);
    pf.kappa = (float)kappa;
    pf.omega = (float)ph.omega;
    pf.omw = (float)(1.0 - ph.omega);
    pf.phi_pref = (float)ph.phi_pref;
    pf.rho_w = (float)prm.rho_w;
    pf.g[0] = (float)ph.g[0];
    pf.g[1] = lattice == LBM_D2Q9 ? 0.0f : (float)ph.g[1];
    pf.g[2] = lattice == LBM_D2Q9 ? (float)ph.g[1] : (float)ph.g[2];
    pf.var_visc = ph.var_visc;
    pf.nu_l = (float)ph.nu_l;
    pf.nu_v = (float)ph.nu_v;
    pf.visc_rl = (float)ph.visc_rl;
    pf.inv_drho = ph.var_visc ? (float)(1.0 / (ph.visc_rl - ph.visc_rv)) : 0.0f;
    pf.phi_sign = (float)ph.phi_sign;
    pf.da = ph.a;
    pf.db = ph.b;
    pf.dRT = ph.RT;
    pf.daalpha = ph.a * ph.alpha;
    pf.dkappa = kappa;
    h->e64 = (prm.flags & LBM_FLAG_EOS_F64) != 0;
    {
        // P - P0 of the solid density, in FP32
        const float r = pf.rho_w;
        float P;
        const float rep = r * pf.RT / (1.0f - pf.b * r);
        switch (eos) {
        case LBM_EOS_VDW: P = rep - pf.a * r * r; break;
        case LBM_EOS_PR: P = rep - pf.aalpha * r * r / (1.0f + 2.0f * pf.b * r - pf.b * pf.b * r * r); break;
        case LBM_EOS_RKS: P = rep - pf.aalpha * r * r / (1.0f + pf.b * r); break;
        case LBM_EOS_SC1: {
            const float q = 1.0f - std::exp(-r);
            P = r * (1.0f / 3.0f) + pf.RT / 6.0f * q * q;
            break;
        }
        case LBM_EOS_SC2: {
            const float q = std::exp(-1.0f / r);
            P = r * (1.0f / 3.0f) + pf.RT / 6.0f * q * q;
            break;
        }
        default: {
            const float e = 0.25f * pf.b * r, om = 1.0f - e;
            P = r * pf.RT * (1.0f + e + e * e - e * e * e) / (om * om * om) - pf.a * r * r;
        }
        }
        const float d = P - r * (1.0f / 3.0f);
        pf.spsi_w = d;
        if (h->e64) pf.spsi_w = (float)excess_pressure_host(eos, ph.a, ph.b, ph.RT, ph.a * ph.alpha, prm.rho_w);
    }
    h->mask_host.assign(h->geo.N, 0);
    if (solid_mask)
        for (size_t n = 0; n < h->geo.N; ++n) {
            h->mask_host[n] = solid_mask[n] ? 1 : 0;
            h->any_solid = h->any_solid || solid_mask[n];
        }
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return LBM_ECUDA;
    }
    h->stream = h->own_stream;
    *out = h;
    return LBM_OK;
}

int lbm_bind_device_memory(lbm_handle h, void *dev, size_t bytes)
{
    if (!h || !dev) return LBM_EINVAL;
    if (h->fv[0]) return fail(h, LBM_ESTATE, "device memory already in use");
    if (reinterpret_cast<uintptr_t>(dev) % kAlign) return fail(h, LBM_EINVAL, "memory not 256-byte aligned");
    const size_t need = layout_for(h->D, h->Q, h->geo.N, h->storage, h->geof.nz).total;
    if (bytes < need) return fail(h, LBM_ENOMEM, "bound memory %zu < required %zu", bytes, need);
    h->base = dev;
    h->owns_base = false;
    h->bytes = bytes;
    return LBM_OK;
}

int lbm_set_stream(lbm_handle h, void *stream)
{
    if (!h) return LBM_EINVAL;
    h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own_stream;
    return LBM_OK;
}

int lbm_init(lbm_handle h, const double *rho0, const double *u0, int on_device)
{
    if (!h || !rho0) return LBM_EINVAL;
    int rc = ensure_memory(h);
    if (rc) return rc;
    const size_t N = h->geo.N;
    h->cur = 0;
    const double *r = rho0, *v = u0;
    if (!on_device) {
        // stage through the second population buffer, dead between steps
        double *st = static_cast<double *>(h->fv[1]);
        CU(h, cudaMemcpyAsync(st, rho0, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
        r = st;
        if (u0) {
            CU(h, cudaMemcpyAsync(st + N, u0, sizeof(double) * h->D * N, cudaMemcpyHostToDevice,
                                  h->stream));
            v = st + N;
        }
    }
    CU(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    rc = h->lattice == LBM_D2Q9 ? launch_init<0>(h, r, v) : launch_init<1>(h, r, v);
    if (rc) return rc;
    CU(h, cudaStreamSynchronize(h->stream));
    h->initialised = true;
    h->bad = false;
    return LBM_OK;
}

int lbm_step(lbm_handle h, int64_t n)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (n < 0) return fail(h, LBM_EINVAL, "negative step count");
    if (h->bad) return fail(h, LBM_ESTATE, "state holds a non-finite density; re-initialise");
    if (n >= 4) {
        if (h->cur != 0) {
            if ((rc = step_plain(h, h->stream))) return rc;
            --n;
        }
        if ((rc = ensure_graph(h))) return rc;
        const int64_t reps = n / 2;
        if (reps > kPollReplays && (rc = ensure_poll(h))) return rc;
        h->poll_pending = false;
        for (int64_t k = 0; k < reps; ++k) {
            if (k > 0 && k % kPollReplays == 0 && (rc = poll_status(h))) return rc;
            CU(h, cudaGraphLaunch(h->graph, h->stream));
            h->launches += 2 * kernels_per_step(h);
        }
        n %= 2;
    }
    for (int64_t k = 0; k < n; ++k)
        if ((rc = step_plain(h, h->stream))) return rc;
    return LBM_OK;
}

int lbm_moments(lbm_handle h, double *rho, double *u, double *U, int on_device)
{
    int rc = check_ready(h);
    if (rc) return rc;
    const size_t N = h->geo.N, D = h->D;
    double *dr = rho, *du = u, *dU = U;
    if (!on_device) {
        double *st = static_cast<double *>(h->fv[h->cur ^ 1]);  // dead between steps
        dr = rho ? st : nullptr;
        du = u ? st + N : nullptr;
        dU = U ? st + N + D * N : nullptr;
    }
    rc = h->lattice == LBM_D2Q9 ? launch_macro_and_out<0>(h, dr, du, dU)
                                : launch_macro_and_out<1>(h, dr, du, dU);
    if (rc) return rc;
    if (!on_device) {
        if (rho) CU(h, cudaMemcpyAsync(rho, dr, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
        if (u) CU(h, cudaMemcpyAsync(u, du, sizeof(double) * D * N, cudaMemcpyDeviceToHost, h->stream));
        if (U) CU(h, cudaMemcpyAsync(U, dU, sizeof(double) * D * N, cudaMemcpyDeviceToHost, h->stream));
    }
    return read_status(h);
}

int lbm_set_wall_distances(lbm_handle h, const double *q)
{
    if (!h) return LBM_EINVAL;
    const size_t N = h->geo.N;
    const int Q = h->Q, D = h->D;
    const Geo &g = h->geo;
    std::vector<unsigned> bn, bm;
    std::vector<double> bq;
    if (q) {
        for (size_t n = 0; n < N; ++n) {
            if (h->mask_host[n]) continue;
            const int x = n % g.nx, y = (n / g.nx) % g.ny, z = n / ((size_t)g.nx * g.ny);
            unsigned m = 0;
            double qq[27] = {0.0};
            for (int i = 0; i < Q; ++i) {
                const int c[3] = {i % 3 - 1, (i / 3) % 3 - 1, D == 3 ? i / 9 - 1 : 0};
                const size_t nd = (size_t)((x + c[0] + g.nx) % g.nx) +
                                  (size_t)g.nx * (((y + c[1] + g.ny) % g.ny) +
                                                  (size_t)g.ny * ((z + c[2] + g.nz) % g.nz));
                const size_t nm = (size_t)((x - c[0] + g.nx) % g.nx) +
                                  (size_t)g.nx * (((y - c[1] + g.ny) % g.ny) +
                                                  (size_t)g.ny * ((z - c[2] + g.nz) % g.nz));
                const double qi = q[(size_t)i * N + n];
                if (!h->mask_host[nd] || !(qi > 0.0)) continue;
                if (!(qi <= 1.0)) return fail(h, LBM_EINVAL, "wall distance q > 1 at node %zu", n);
                if (h->mask_host[nm]) continue;   // no fluid node behind: stays halfway
                m |= 1u << i;
                qq[i] = qi;
            }
            if (m) {
                bn.push_back((unsigned)n);
                bm.push_back(m);
                bq.insert(bq.end(), qq, qq + Q);
            }
        }
    }
    if (h->stream) CU(h, cudaStreamSynchronize(h->stream));
    if (h->bn) cudaFree(h->bn);
    if (h->bmask) cudaFree(h->bmask);
    if (h->bq) cudaFree(h->bq);
    h->bn = h->bmask = nullptr;
    h->bq = nullptr;
    h->nb = 0;
    if (h->graph) {   // the captured steps change
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (bn.empty()) return LBM_OK;
    CU(h, cudaMalloc(&h->bn, sizeof(unsigned) * bn.size()));
    CU(h, cudaMalloc(&h->bmask, sizeof(unsigned) * bm.size()));
    CU(h, cudaMalloc(&h->bq, sizeof(double) * bq.size()));
    CU(h, cudaMemcpy(h->bn, bn.data(), sizeof(unsigned) * bn.size(), cudaMemcpyHostToDevice));
    CU(h, cudaMemcpy(h->bmask, bm.data(), sizeof(unsigned) * bm.size(), cudaMemcpyHostToDevice));
    CU(h, cudaMemcpy(h->bq, bq.data(), sizeof(double) * bq.size(), cudaMemcpyHostToDevice));
    h->nb = (int)bn.size();
    return LBM_OK;
}

int lbm_pressure_tensor(lbm_handle h, double *P, int on_device)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!P) return fail(h, LBM_EINVAL, "null output");
    const size_t N = h->geo.N, na = h->D == 3 ? 6 : 3;
    // the dead population buffer holds (1 + 2D) N >= na N doubles
    double *out = on_device ? P : static_cast<double *>(h->fv[h->cur ^ 1]);
    rc = h->lattice == LBM_D2Q9 ? launch_pressure<0>(h, out) : launch_pressure<1>(h, out);
    if (rc) return rc;
    if (!on_device)
        CU(h, cudaMemcpyAsync(P, out, sizeof(double) * na * N, cudaMemcpyDeviceToHost, h->stream));
    return read_status(h);
}

int lbm_reduce(lbm_handle h, double *mass, double *momentum)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!mass && !momentum) return LBM_EINVAL;
    rc = h->lattice == LBM_D2Q9 ? launch_reduce<0>(h) : launch_reduce<1>(h);
    if (rc) return rc;
    double s[4];
    CU(h, cudaMemcpyAsync(s, h->sums, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
    rc = read_status(h);  // synchronises
    if (mass) *mass = s[0];
    if (momentum)
        for (int a = 0; a < h->D; ++a) momentum[a] = s[1 + a];
    return rc;
}

int lbm_get_populations(lbm_handle h, double *f, int on_device)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (!f) return LBM_EINVAL;
    const size_t N = h->geo.N, QN = (size_t)h->Q * N;
    if (shifted(h->storage)) {
        TempF64 t;
        rc = temp_alloc(h, t);
        if (!rc) rc = h->lattice == LBM_D2Q9 ? decode_to<0>(h, h->cur, t.p) : decode_to<1>(h, h->cur, t.p);
        if (rc) return rc;
        CU(h, cudaMemcpyAsync(f, t.p, sizeof(double) * QN,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
        CU(h, cudaStreamSynchronize(h->stream));
    } else if (h->storage == LBM_F32) {
        if (on_device) {
            lbmk::k_convert<float, double><<<1024, 256, 0, h->stream>>>(QN, f32(h, h->cur), f);
            CU(h, cudaGetLastError());
            h->launches += 1;
        } else {
            std::vector<float> tmp(QN);
            CU(h, cudaMemcpyAsync(tmp.data(), f32(h, h->cur), sizeof(float) * QN,
                                  cudaMemcpyDeviceToHost, h->stream));
            CU(h, cudaStreamSynchronize(h->stream));
            for (size_t k = 0; k < QN; ++k) f[k] = tmp[k];
        }
    } else {
        CU(h, cudaMemcpyAsync(f, f64(h, h->cur), sizeof(double) * QN,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              h->stream));
    }
    rc = read_status(h);
    if (!on_device)
        for (size_t n = 0; n < N; ++n)
            if (h->mask_host[n])
                for (int i = 0; i < h->Q; ++i) f[(size_t)i * N + n] = 0.0;
    return rc;
}

int lbm_set_populations(lbm_handle h, const double *f, int on_device)
{
    if (!h || !f) return LBM_EINVAL;
    int rc = ensure_memory(h);
    if (rc) return rc;
    const size_t QN = (size_t)h->Q * h->geo.N;
    h->cur = 0;
    if (shifted(h->storage)) {
        TempF64 t;
        rc = temp_alloc(h, t);
        if (rc) return rc;
        CU(h, cudaMemcpyAsync(t.p, f, sizeof(double) * QN,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        rc = h->lattice == LBM_D2Q9 ? encode_from<0>(h, t.p) : encode_from<1>(h, t.p);
        if (rc) return rc;
        CU(h, cudaStreamSynchronize(h->stream));
    } else if (h->storage == LBM_F32) {
        if (on_device) {
            lbmk::k_convert<double, float><<<1024, 256, 0, h->stream>>>(QN, f, f32(h, 0));
            CU(h, cudaGetLastError());
            h->launches += 1;
        } else {
            std::vector<float> tmp(QN);
            for (size_t k = 0; k < QN; ++k) tmp[k] = (float)f[k];
            CU(h, cudaMemcpyAsync(f32(h, 0), tmp.data(), sizeof(float) * QN,
                                  cudaMemcpyHostToDevice, h->stream));
            CU(h, cudaStreamSynchronize(h->stream));
        }
    } else {
        CU(h, cudaMemcpyAsync(f64(h, 0), f, sizeof(double) * QN,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              h->stream));
    }
    CU(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    rc = h->lattice == LBM_D2Q9 ? launch_fill_solid<0>(h) : launch_fill_solid<1>(h);
    if (rc) return rc;
    CU(h, cudaStreamSynchronize(h->stream));
    h->initialised = true;
    h->bad = false;
    return LBM_OK;
}

int lbm_sync(lbm_handle h, int timeout_ms)
{
    if (!h) return LBM_EINVAL;
    if (!h->initialised) return LBM_OK;
    if (timeout_ms >= 0) {
        cudaEvent_t ev;
        CU(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, h->stream);
        if (e != cudaSuccess) {
            cudaEventDestroy(ev);
            return fail(h, LBM_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
        }
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            e = cudaEventQuery(ev);
            if (e != cudaErrorNotReady) break;
            if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms)) {
                cudaEventDestroy(ev);
                return fail(h, LBM_ETIMEOUT, "work still running after %d ms", timeout_ms);
            }
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        cudaEventDestroy(ev);
        if (e != cudaSuccess) return fail(h, LBM_ECUDA, "stream error: %s", cudaGetErrorString(e));
    }
    return read_status(h);
}

int64_t lbm_launch_count(lbm_handle h) { return h ? h->launches : -1; }

int lbm_selftest_wait_timeout(long long limit_cycles, int *status_bits, double *ms)
{
    if (!status_bits || !ms || limit_cycles < 1 || limit_cycles > 2000000000ll) return LBM_EINVAL;
    int *st = nullptr;
    if (cudaMalloc(&st, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBM_OK, host = 0;
    float t = 0.0f;
    if (cudaMemset(st, 0, sizeof(int)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = LBM_ECUDA;
    if (rc == LBM_OK) {
        cudaEventRecord(e0, 0);
        lbmf::k_wait_selftest<<<1, 64>>>(st, limit_cycles);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
            cudaMemcpy(&host, st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = LBM_ECUDA;
    }
    if (rc != LBM_OK) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(st);
    if (rc == LBM_OK) {
        *status_bits = host;
        *ms = t;
    }
    return rc;
}

int lbm_probe_fp64_tflops(double *tflops)
{
    if (!tflops) return LBM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    const int threads = 256, blocks = 8 * sms, iters = 4096;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * threads * blocks) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBM_OK;
    double best = 0.0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = LBM_ECUDA;
    for (int rep = 0; rep < 4 && rc == LBM_OK; ++rep) {   // the first launch warms up
        cudaEventRecord(e0, 0);
        lbmk::k_fp64_fma_probe<<<blocks, threads>>>(out, iters);
        cudaEventRecord(e1, 0);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = LBM_ECUDA;
            break;
        }
        const double tf = 2.0 * 8.0 * iters * (double)threads * blocks / (ms * 1e-3) / 1e12;
        if (rep > 0 && tf > best) best = tf;
    }
    if (rc != LBM_OK) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc == LBM_OK) *tflops = best;
    return rc;
}

}  // extern "C"

struct lbm_batch_ctx {
    std::vector<lbm_ctx *> members;
    std::vector<int> cur0;   // each member's buffer index when the batch was made
    std::vector<cudaStream_t> prev;   // each member's stream before the batch
    int lattice = 0, storage = LBM_F32;
    cudaStream_t stream = nullptr;
    lbmf::MemberF *d_members[2] = {nullptr, nullptr};   // step parity 0 and 1
    lbmf::WorkItem *d_items = nullptr;
    int n_items = 0, grid = 0, parity = 0;
    cudaGraphExec_t graph = nullptr;
    int64_t launches = 0;
};

namespace {

template <int LAT, typename ST>
void launch_batch_shifted(lbm_batch_ctx *b, int parity, cudaStream_t s)
{
    static std::atomic<unsigned long long> done{0};   // devices already opted in
    const int bytes = (int)sizeof(lbmf::SharedS<LAT>);
    smem_opt_in(lbmf::k_step_shifted_batch<LAT, ST>, bytes, done);
    lbmf::k_step_shifted_batch<LAT, ST>
        <<<b->grid, lbmf::LatF<LAT>::TX * lbmf::LatF<LAT>::TY, bytes, s>>>(
            b->d_members[parity], b->d_items, b->n_items);
}

template <int LAT>
void launch_batch(lbm_batch_ctx *b, int parity, cudaStream_t s)
{
    if (b->storage == LBM_F16S) launch_batch_shifted<LAT, __half>(b, parity, s);
    else if (b->storage == LBM_BF16S) launch_batch_shifted<LAT, __nv_bfloat16>(b, parity, s);
    else {
        static std::atomic<unsigned long long> done{0};   // devices already opted in
        const int bytes = (int)sizeof(lbmf::SharedF<LAT>);
        smem_opt_in(lbmf::k_step_f32_batch<LAT>, bytes, done);
        lbmf::k_step_f32_batch<LAT><<<b->grid, lbmf::LatF<LAT>::TX * lbmf::LatF<LAT>::TY, bytes, s>>>(
            b->d_members[parity], b->d_items, b->n_items);
    }
}

void batch_launch(lbm_batch_ctx *b, int parity, cudaStream_t s)
{
    if (b->lattice == LBM_D2Q9) launch_batch<0>(b, parity, s);
    else launch_batch<1>(b, parity, s);
}

void batch_free(lbm_batch_ctx *b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (auto *m : b->d_members) if (m) cudaFree(m);
    if (b->d_items) cudaFree(b->d_items);
    for (size_t k = 0; k < b->prev.size(); ++k) b->members[k]->stream = b->prev[k];
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_batch *out, const lbm_handle *members, int count)
{
    if (!out || !members || count < 1) return LBM_EINVAL;
    *out = nullptr;
    const int lattice = members[0] ? members[0]->lattice : -1;
    const int storage = members[0] ? members[0]->storage : -1;
    if (storage == LBM_F64) return LBM_EINVAL;
    for (int k = 0; k < count; ++k) {
        lbm_ctx *h = members[k];
        if (!h || !h->initialised || h->bad || h->storage != storage || h->lattice != lattice ||
            h->nb > 0 ||   // interpolated bounce-back is not part of the batched step
            h->e64)        // nor the FP64-EOS form
            return LBM_EINVAL;
        for (int j = 0; j < k; ++j)
            if (members[j] == h) return LBM_EINVAL;   // a lattice at most once
    }
    lbm_batch_ctx *b = new (std::nothrow) lbm_batch_ctx();
    if (!b) return LBM_ENOMEM;
    b->lattice = lattice;
    b->storage = storage;
    b->members.assign(members, members + count);
    for (lbm_ctx *h : b->members) {
        b->cur0.push_back(h->cur);
        b->prev.push_back(h->stream);
    }
    for (lbm_ctx *h : b->members) cudaStreamSynchronize(h->stream);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        batch_free(b);
        return LBM_ECUDA;
    }
    std::vector<lbmf::MemberF> desc[2];
    std::vector<lbmf::WorkItem> items;
    for (int k = 0; k < count; ++k) {
        lbm_ctx *h = b->members[k];
        const int TX = lattice == LBM_D2Q9 ? lbmf::LatF<0>::TX : lbmf::LatF<1>::TX;
        const int TY = lattice == LBM_D2Q9 ? lbmf::LatF<0>::TY : lbmf::LatF<1>::TY;
        const int tx = (h->geof.nx + TX - 1) / TX, ty = (h->geof.ny + TY - 1) / TY;
        const int tz = (h->geof.nz + h->geof.chunk - 1) / h->geof.chunk;
        for (int par = 0; par < 2; ++par) {
            lbmf::MemberF m;
            m.g = h->geof;
            m.p = h->physf;
            m.mask = h->any_solid ? h->mask : nullptr;
            m.src = h->fv[h->cur ^ par];
            m.dst = h->fv[h->cur ^ par ^ 1];
            m.rho_src = h->rs[h->cur ^ par];
            m.rho_dst = h->rs[h->cur ^ par ^ 1];
            m.status = h->status;
            m.tiles_x = tx;
            m.tiles_y = ty;
            desc[par].push_back(m);
        }
        for (int bz = 0; bz < tz; ++bz)
            for (int by = 0; by < ty; ++by)
                for (int bx = 0; bx < tx; ++bx) items.push_back({k, bx, by, bz});
        h->stream = b->stream;   // members' later work is ordered after the batch
    }
    b->n_items = (int)items.size();
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = std::min(b->n_items, 2 * std::max(sms, 1));
    const size_t db = sizeof(lbmf::MemberF) * count, ib = sizeof(lbmf::WorkItem) * items.size();
    if (cudaMalloc(&b->d_members[0], db) != cudaSuccess || cudaMalloc(&b->d_members[1], db) != cudaSuccess ||
        cudaMalloc(&b->d_items, ib) != cudaSuccess) {
        batch_free(b);
        return LBM_ENOMEM;
    }
    if (cudaMemcpy(b->d_members[0], desc[0].data(), db, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_members[1], desc[1].data(), db, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_items, items.data(), ib, cudaMemcpyHostToDevice) != cudaSuccess) {
        batch_free(b);
        return LBM_ECUDA;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch b, int64_t n)
{
    if (!b || n < 0) return LBM_EINVAL;
    for (lbm_ctx *h : b->members)
        if (h->bad) return LBM_ESTATE;
    if (n >= 4) {
        if (b->parity != 0) {
            batch_launch(b, b->parity, b->stream);
            b->parity ^= 1;
            ++b->launches;
            --n;
        }
        if (!b->graph) {
            cudaStream_t cap = nullptr;
            if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return LBM_ECUDA;
            cudaGraph_t gr = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                batch_launch(b, 0, cap);
                batch_launch(b, 1, cap);
                e = cudaStreamEndCapture(cap, &gr);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, gr, 0);
            if (gr) cudaGraphDestroy(gr);
            cudaStreamDestroy(cap);
            if (e != cudaSuccess) {
                b->graph = nullptr;
                cudaGetLastError();
                return LBM_ECUDA;
            }
        }
        for (int64_t k = 0; k < n / 2; ++k)
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return LBM_ECUDA;
        b->launches += 2 * (n / 2);
        n %= 2;
    }
    for (int64_t k = 0; k < n; ++k) {
        batch_launch(b, b->parity, b->stream);
        b->parity ^= 1;
        ++b->launches;
    }
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}

int lbm_batch_sync(lbm_batch b)
{
    if (!b) return LBM_EINVAL;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LBM_ECUDA;
    // members' state buffers follow the batch parity; their moments, reductions
    // and population reads are valid between lbm_batch_sync and the next step
    int bad = LBM_OK;
    for (size_t k = 0; k < b->members.size(); ++k) {
        lbm_ctx *h = b->members[k];
        h->cur = b->cur0[k] ^ b->parity;
        int rc = read_status(h);
        if (rc && !bad) bad = rc;
    }
    return bad;
}

int64_t lbm_batch_launch_count(lbm_batch b) { return b ? b->launches : -1; }

void lbm_batch_destroy(lbm_batch b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (size_t k = 0; k < b->members.size(); ++k) b->members[k]->cur = b->cur0[k] ^ b->parity;
    batch_free(b);
}

int lbm_time_kernels(lbm_handle h, int64_t n, double *ms)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (n < 1 || !ms) return fail(h, LBM_EINVAL, "need n >= 1 and an output array");
    if (h->bad) return fail(h, LBM_ESTATE, "state holds a non-finite density; re-initialise");
    std::vector<cudaEvent_t> ev(3 * n);
    for (auto &e : ev) CU(h, cudaEventCreate(&e));
    const dim3 gr = node_grid(h->geo), bl = node_block(h->geo);
    const bool fused = h->storage != LBM_F64;
    for (int64_t k = 0; k < n; ++k) {
        CU(h, cudaEventRecord(ev[3 * k], h->stream));
        if (fused) {
            CU(h, cudaEventRecord(ev[3 * k + 1], h->stream));
            if (shifted(h->storage)) {
                if (h->lattice == LBM_D2Q9) launch_shifted<0>(h, h->stream, h->cur);
                else launch_shifted<1>(h, h->stream, h->cur);
            } else if (h->lattice == LBM_D2Q9) {
                launch_fused<0>(h, h->stream, f32(h, h->cur), f32(h, h->cur ^ 1));
            } else {
                launch_fused<1>(h, h->stream, f32(h, h->cur), f32(h, h->cur ^ 1));
            }
            h->launches += 1;
        } else {
            const double *src = f64(h, h->cur);
            double *dst = f64(h, h->cur ^ 1);
            if (h->lattice == LBM_D2Q9)
                lbmk::k_macro<0><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, src, h->rp,
                                                           h->u, h->gflux, h->status);
            else
                lbmk::k_macro<1><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, src, h->rp,
                                                           h->u, h->gflux, h->status);
            CU(h, cudaEventRecord(ev[3 * k + 1], h->stream));
            if (h->lattice == LBM_D2Q9)
                lbmk::k_collide<0><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, src, dst,
                                                             h->rp, h->u, h->gflux);
            else
                lbmk::k_collide<1><<<gr, bl, 0, h->stream>>>(h->geo, h->phys, h->mask, src, dst,
                                                             h->rp, h->u, h->gflux);
            h->launches += 2;
        }
        CU(h, cudaEventRecord(ev[3 * k + 2], h->stream));
        CU(h, cudaGetLastError());
        h->cur ^= 1;
    }
    CU(h, cudaStreamSynchronize(h->stream));
    double t0 = 0.0, t1 = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        float a = 0.f, b = 0.f;
        CU(h, cudaEventElapsedTime(&a, ev[3 * k], ev[3 * k + 1]));
        CU(h, cudaEventElapsedTime(&b, ev[3 * k + 1], ev[3 * k + 2]));
        t0 += a;
        t1 += b;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    ms[0] = t0 / n;
    ms[1] = t1 / n;
    return read_status(h);
}

int lbm_autotune(lbm_handle h, int *chunk_out)
{
    int rc = check_ready(h);
    if (rc) return rc;
    if (h->storage == LBM_F64) {
        if (chunk_out) *chunk_out = 0;
        return LBM_OK;   // the FP64 step has no tile parameters
    }
    if (h->bad) return fail(h, LBM_ESTATE, "state holds a non-finite density; re-initialise");
    const size_t bytes = pop_bytes(h->storage) * (size_t)h->Q * h->geo.N;
    const size_t rbytes = shifted(h->storage) ? sizeof(float) * h->geo.N : 0;
    void *save = nullptr;
    if (cudaMalloc(&save, bytes + rbytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, LBM_ENOMEM, "autotune: no room to save the state");
    }
    CU(h, cudaMemcpyAsync(save, h->fv[h->cur], bytes, cudaMemcpyDeviceToDevice, h->stream));
    if (rbytes)
        CU(h, cudaMemcpyAsync(static_cast<char *>(save) + bytes, h->rs[h->cur], rbytes,
                              cudaMemcpyDeviceToDevice, h->stream));
    const int nz = h->geof.nz;
    // plane chunks per CTA; on a march axis longer than 128 planes also 10/16
    // .. 16/16 of it: one long chunk per column and a short one after it,
    // whose blocks (launched after all long ones) fill the last wave
    std::vector<int> cands = {4, 6, 8, 11, 13, 16, 22, 26, 32, 43, 64, 128};
    if (nz > 128)
        for (int k = 10; k <= 16; ++k) cands.push_back(std::max(129, nz * k / 16));
    const int chunk0 = h->geof.chunk, rows0 = h->tile_rows;   // restored on failure
    // FP32: the plain, warp-specialised and Tensor Memory kernels; D3Q27 FP32
    // also 32 x 8 and 32 x 7 tiles (the shifted and batched steps use plain
    // 32 x 8)
    const bool fp32 = h->storage == LBM_F32 && !h->e64;   // the FP64-EOS form is plain 32 x 8
    const bool two_heights = h->lattice == LBM_D3Q27 && fp32;
    const int variant0 = h->variant;
    int best = h->geof.chunk, best_rows = h->tile_rows, best_variant = h->variant;
    double best_ms = 1e30;
    for (int var = 0; var <= LBM_FUSED_TM_TMA && rc == LBM_OK; ++var) {
        // shifted storage: plain, Tensor Memory and (D3Q27) the two warp-specialised Tensor Memory forms
        if (var > 0 && (h->e64 || (!fp32 && var == LBM_FUSED_WARP_SPECIALISED))) continue;
        if (var >= LBM_FUSED_WS_TMEM && h->lattice != LBM_D3Q27) continue;
        if ((var == LBM_FUSED_WS_TMA || var == LBM_FUSED_TM_TMA) && !h->tmap_ready) continue;
        if (var == LBM_FUSED_TM_TMA && !shifted(h->storage)) continue;   // a form of shifted storage
        h->variant = var;
        for (int rows : {8, 7}) {
            if (rows == 7 && (!two_heights || var >= LBM_FUSED_WS_TMEM)) continue;
            h->tile_rows = rows;
            for (size_t j = 0; j < cands.size(); ++j) {
                const int c = cands[j];
                if ((c > nz && j != 0) || (j > 0 && c == cands[j - 1])) continue;
                h->geof.chunk = c;
                double ms[2];
                rc = lbm_time_kernels(h, 1, ms);                  // warm-up
                if (rc == LBM_OK) rc = lbm_time_kernels(h, 6, ms);
                if (rc != LBM_OK) break;
                if (ms[1] < best_ms) { best_ms = ms[1]; best = c; best_rows = rows; best_variant = var; }
            }
            if (rc != LBM_OK) break;
        }
    }
    // the best candidate, or on failure the kernel, chunk and tile the handle
    // had; a graph captured before the search may hold either, so it is dropped
    h->tile_rows = rc == LBM_OK ? best_rows : rows0;
    h->geof.chunk = rc == LBM_OK ? best : chunk0;
    h->variant = rc == LBM_OK ? best_variant : variant0;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaError_t e = cudaMemcpyAsync(h->fv[0], save, bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && rbytes)
        e = cudaMemcpyAsync(h->rs[0], static_cast<char *>(save) + bytes, rbytes,
                            cudaMemcpyDeviceToDevice, h->stream);
    cudaStreamSynchronize(h->stream);
    cudaFree(save);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "autotune restore: %s", cudaGetErrorString(e));
    h->cur = 0;
    if (rc != LBM_OK) return rc;
    if (chunk_out) *chunk_out = best;
    return LBM_OK;
}

int lbm_get_tile(lbm_handle h, int *tile_x, int *tile_y)
{
    if (!h) return LBM_EINVAL;
    int tx = 0, ty = 0;
    if (h->storage != LBM_F64) {
        tx = h->lattice == LBM_D2Q9 ? lbmf::LatF<0>::TX : lbmf::LatF<1>::TX;
        ty = h->lattice == LBM_D2Q9 ? lbmf::LatF<0>::TY
             : (h->tile_rows == 7 && h->storage == LBM_F32) ? 7 : lbmf::LatF<1>::TY;
    }
    if (tile_x) *tile_x = tx;
    if (tile_y) *tile_y = ty;
    return LBM_OK;
}

int lbm_set_tile(lbm_handle h, int tile_y)
{
    if (!h) return LBM_EINVAL;
    if (h->lattice != LBM_D3Q27 || h->storage != LBM_F32)
        return fail(h, LBM_EINVAL, "the tile height is a parameter of the D3Q27 FP32 step only");
    if (tile_y != 7 && tile_y != 8) return fail(h, LBM_EINVAL, "tile height must be 7 or 8");
    if (tile_y == 7 && h->e64) return fail(h, LBM_EINVAL, "the FP64-EOS step runs 8-row tiles");
    if (tile_y == 7 && h->variant >= LBM_FUSED_WS_TMEM)
        return fail(h, LBM_EINVAL, "the warp-specialised Tensor Memory forms run 8-row tiles");
    if (h->tile_rows != tile_y && h->graph) {   // the captured graph holds the other kernel
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->tile_rows = tile_y;
    return LBM_OK;
}

int lbm_set_fused_variant(lbm_handle h, int variant)
{
    if (!h) return LBM_EINVAL;
    if (variant < LBM_FUSED_PLAIN || variant > LBM_FUSED_TM_TMA)
        return fail(h, LBM_EINVAL, "unknown fused-step variant %d", variant);
    if (variant == LBM_FUSED_TM_TMA && !shifted(h->storage))
        return fail(h, LBM_EINVAL, "the one-group TMA-staged form is a form of shifted storage");
    if (variant >= LBM_FUSED_WS_TMEM && (h->lattice != LBM_D3Q27 || h->tile_rows != 8))
        return fail(h, LBM_EINVAL, "the warp-specialised Tensor Memory forms run D3Q27 32 x 8 tiles");
    if ((variant == LBM_FUSED_WS_TMA || variant == LBM_FUSED_TM_TMA) &&
        (!tma_nx_multiple(h->storage) || h->geo.nx % tma_nx_multiple(h->storage) ||
         (h->fv[0] && !h->tmap_ready)))
        return fail(h, LBM_EINVAL, "the TMA-staged form needs FP32 storage with nx a multiple of 4 or shifted "
                                   "storage with nx a multiple of 8, and the CUDA driver's tensor-map encoder");
    if (h->storage == LBM_F64 && variant != LBM_FUSED_PLAIN)
        return fail(h, LBM_EINVAL, "the FP64 step has one form");
    if (h->e64 && variant != LBM_FUSED_PLAIN)
        return fail(h, LBM_EINVAL, "the FP64-EOS step has one form");
    if (shifted(h->storage) && variant == LBM_FUSED_WARP_SPECIALISED)
        return fail(h, LBM_EINVAL, "shifted storage has the plain and the Tensor Memory forms");
    if (h->variant != variant && h->graph) {   // the captured graph holds the other kernel
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->variant = variant;
    return LBM_OK;
}

int lbm_get_fused_variant(lbm_handle h, int *variant)
{
    if (!h || !variant) return LBM_EINVAL;
    *variant = h->variant;
    return LBM_OK;
}

int lbm_set_chunk(lbm_handle h, int chunk)
{
    if (!h) return LBM_EINVAL;
    if (chunk < 1) return fail(h, LBM_EINVAL, "chunk must be >= 1");
    if (h->geof.chunk != chunk && h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->geof.chunk = chunk;
    return LBM_OK;
}

const char *lbm_last_error(lbm_handle h) { return h ? h->err : "null handle"; }

void lbm_destroy(lbm_handle h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->owns_base && h->base) cudaFree(h->base);
    if (h->bn) cudaFree(h->bn);
    if (h->bmask) cudaFree(h->bmask);
    if (h->bq) cudaFree(h->bq);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    if (h->poll_ev) cudaEventDestroy(h->poll_ev);
    if (h->poll_host) cudaFreeHost(h->poll_host);
    cudaGetLastError();
    delete h;
}

}  // extern "C"
