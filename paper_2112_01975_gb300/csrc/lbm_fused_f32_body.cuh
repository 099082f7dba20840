// Fused single-pass step for FP32 populations with FP32 arithmetic.
//
// One CTA owns a TX x TY column tile of the x-y plane and marches along z
// through a chunk of planes (D2Q9 runs as a 3D lattice with one y row and
// the 2D y axis as the march axis). For each plane that enters, it reads the
// 27 populations of every node of the tile plus a 2-node halo, forms
// (rho, s psi) there and rho u_a^3 on the 1-node halo, and keeps them in
// shared-memory rings. Two planes behind, it collides the tile: the 2-ring
// force stencils and the Phi differences read only shared memory, the
// node's bare velocity and 1/rho come from its phase-A moments through a
// ring, its populations are read again (an L2 hit), and the post-collision
// populations are pushed to the neighbours with halfway bounce-back. HBM
// sees each population read about once and written once; the halo and the
// second read of a node are served from L2.
//
// This file is the body of the fused tile: it is included once per tile
// height by a header that defines LBMF_NS (the namespace) and LBMF_ROWS (the
// D3Q27 tile height TY), `lbm_fused_f32.cuh` (lbmf, 8 rows) and
// `lbm_fused_f32_r7.cuh` (lbmf7, 7 rows); it has no include guard of its own.
#if !defined(LBMF_NS) || !defined(LBMF_ROWS)
#error "include lbm_fused_f32.cuh or lbm_fused_f32_r7.cuh"
#endif

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace LBMF_NS {

// Storage of populations: float (FP32), or 16-bit values of the relative
// shift h_i = f_i / rho(src) - w_i, with rho(src) the FP32 density of the node
// that pushed the population (the node itself after a bounce-back). Relative
// to the source density, h stays O(1e-3) in a vapour of any density, where
// the absolute shift f_i - w_i rho would fall below FP16's normal range.
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename ST> __device__ __forceinline__ ST from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}
template <typename ST> struct IsShifted { static constexpr bool value = true; };
template <> struct IsShifted<float> { static constexpr bool value = false; };

struct GeoF {
    int nx, ny, nz;   // as stored; D2Q9: ny = 1 and nz = the 2D y extent
    unsigned N;
    int chunk;        // planes per CTA along z
    const uint8_t *zsolid;   // per plane along z: 1 if it holds a solid node (masked lattices)
};

// Masked lattices: whether plane z (wrapped) holds a solid node, and
// whether any of the planes z-1, z, z+1 do (the planes a collision at z
// pushes into). Planes without solids run the unmasked code.
__device__ __forceinline__ bool plane_solid(const GeoF &g, int z)
{
    return g.zsolid[z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z)] != 0;
}
__device__ __forceinline__ bool planes_solid3(const GeoF &g, int z)
{
    return plane_solid(g, z - 1) || plane_solid(g, z) || plane_solid(g, z + 1);
}

struct PhysF {
    int eos;
    float a, b, RT, aalpha;
    float kappa, omega, omw, phi_pref;  // omw = 1 - omega
    float rho_w, spsi_w;                // virtual solid density and its P - P0
    float g[3];                         // body acceleration in the kernel frame (D2Q9: gx, 0, gy)
    int var_visc;                       // density-dependent relaxation (nu linear in rho)
    float nu_l, nu_v, visc_rl, inv_drho, phi_sign;   // inv_drho = 1 / (rho_l - rho_v)
    // FP64 constants of the EOS and the capillary term, for the kernels that
    // evaluate the EOS and the force in FP64 (lbm_params.flags & LBM_FLAG_EOS_F64)
    double da, db, dRT, daalpha, dkappa;
};

// Relaxation rate at density rho: nu from nu_l at rho_l to nu_v at rho_v,
// linear in rho and constant beyond (used only when var_visc).
__device__ __forceinline__ float omega_var_f(const PhysF &p, float rho)
{
    const float t = fminf(fmaxf((p.visc_rl - rho) * p.inv_drho, 0.0f), 1.0f);
    return __frcp_rn(3.0f * fmaf(p.nu_v - p.nu_l, t, p.nu_l) + 0.5f);
}

// Lattice description in the 3D frame: D2Q9 uses (cx, 0, cy).
template <int LAT> struct LatF;
template <> struct LatF<0> {
    static constexpr int Q = 9, TX = 128, TY = 1, HY = 0;
    __device__ static constexpr int cx(int i) { return i % 3 - 1; }
    __device__ static constexpr int cy(int) { return 0; }
    __device__ static constexpr int cz(int i) { return i / 3 - 1; }
};
template <> struct LatF<1> {
    static constexpr int Q = 27, TX = 32, TY = LBMF_ROWS, HY = 2;
    __device__ static constexpr int cx(int i) { return i % 3 - 1; }
    __device__ static constexpr int cy(int i) { return (i / 3) % 3 - 1; }
    __device__ static constexpr int cz(int i) { return i / 9 - 1; }
};

// Lattice weight w_i = prod of 1D weights 2/3 (c = 0), 1/6 (c = +-1) (Eq. wi).
template <int LAT> __device__ __forceinline__ constexpr float weight_f(int i)
{
    using L = LatF<LAT>;
    return (L::cx(i) ? 1.0f / 6.0f : 2.0f / 3.0f) * (LAT == 1 ? (L::cy(i) ? 1.0f / 6.0f : 2.0f / 3.0f) : 1.0f) *
           (L::cz(i) ? 1.0f / 6.0f : 2.0f / 3.0f);
}

// P - rho/3 in FP32, one reciprocal per EOS (Sec. 3.1 and Appendix G equations of state).
// Every operation is an explicitly rounded intrinsic, so each inlined call
// site rounds the same way (no call-site-dependent contraction). EOSK >= 0
// fixes the equation of state at compile time (the same operations as its
// case below); EOSK < 0 takes it from p.eos.
template <int EOSK = -1>
__device__ __forceinline__ float excess_pressure_ft(const PhysF &p, float rho)
{
    const float br = __fmul_rn(p.b, rho), rr = __fmul_rn(rho, rho);
    const float nr3 = __fmul_rn(rho, -1.0f / 3.0f);
    const float rt = __fmul_rn(rho, p.RT);
    switch (EOSK >= 0 ? EOSK : p.eos) {
    case 0:   // rho RT / (1 - b rho) - a rho^2 - rho/3
        return __fmaf_rn(-p.a, rr, __fmaf_rn(rt, __frcp_rn(__fsub_rn(1.0f, br)), nr3));
    case 1: {   // PR: d1 = 1 - b rho, d2 = 1 + 2 b rho - (b rho)^2
        const float d1 = __fsub_rn(1.0f, br), d2 = __fmaf_rn(br, __fsub_rn(2.0f, br), 1.0f);
        const float num = __fmaf_rn(rt, d2, -__fmul_rn(__fmul_rn(p.aalpha, rr), d1));
        return __fmaf_rn(num, __frcp_rn(__fmul_rn(d1, d2)), nr3);
    }
    case 2: {   // RKS: d1 = 1 - b rho, d2 = 1 + b rho
        const float d1 = __fsub_rn(1.0f, br), d2 = __fadd_rn(1.0f, br);
        const float num = __fmaf_rn(rt, d2, -__fmul_rn(__fmul_rn(p.aalpha, rr), d1));
        return __fmaf_rn(num, __frcp_rn(__fmul_rn(d1, d2)), nr3);
    }
    case 4: {   // Shan-Chen, psi_SC = 1 - exp(-rho): P - rho/3 = (G/6) psi_SC^2, G in RT
        const float q = __fsub_rn(1.0f, expf(-rho));
        return __fmul_rn(__fmul_rn(q, q), __fmul_rn(p.RT, 1.0f / 6.0f));
    }
    case 5: {   // Shan-Chen, psi_SC = exp(-1/rho)
        const float q = expf(-__frcp_rn(rho));
        return __fmul_rn(__fmul_rn(q, q), __fmul_rn(p.RT, 1.0f / 6.0f));
    }
    default: {   // CS with e = b rho / 4
        const float e = __fmul_rn(0.25f, br), om = __fsub_rn(1.0f, e);
        const float poly = __fmaf_rn(__fmul_rn(e, e), __fsub_rn(1.0f, e), __fadd_rn(1.0f, e));
        const float den = __fmul_rn(__fmul_rn(om, om), om);
        return __fmaf_rn(-p.a, rr, __fmaf_rn(__fmul_rn(rt, poly), __frcp_rn(den), nr3));
    }
    }
}

__device__ __forceinline__ float excess_pressure_f(const PhysF &p, float rho)
{
    return excess_pressure_ft<-1>(p, rho);
}

// P - rho/3 in FP64: the same equations of state, for the FP64-EOS form of
// the reduced-precision steps (Sec. 3.1 and Appendix G).
__device__ __forceinline__ double excess_pressure_d(const PhysF &p, double rho)
{
    const double br = p.db * rho, rr = rho * rho, rt = rho * p.dRT;
    switch (p.eos) {
    case 0:
        return rt / (1.0 - br) - p.da * rr - rho * (1.0 / 3.0);
    case 1: {
        const double d1 = 1.0 - br, d2 = 1.0 + br * (2.0 - br);
        return (rt * d2 - p.daalpha * rr * d1) / (d1 * d2) - rho * (1.0 / 3.0);
    }
    case 2: {
        const double d1 = 1.0 - br, d2 = 1.0 + br;
        return (rt * d2 - p.daalpha * rr * d1) / (d1 * d2) - rho * (1.0 / 3.0);
    }
    case 4: {
        const double q = 1.0 - exp(-rho);
        return p.dRT * (1.0 / 6.0) * q * q;
    }
    case 5: {
        const double q = exp(-1.0 / rho);
        return p.dRT * (1.0 / 6.0) * q * q;
    }
    default: {
        const double e = 0.25 * br, om = 1.0 - e;
        return rt * (1.0 + e + e * e - e * e * e) / (om * om * om) - p.da * rr - rho * (1.0 / 3.0);
    }
    }
}

// Sum of v[0..n-1] as a balanced tree of additions.
template <int N>
__device__ __forceinline__ float pairwise_sum(const float *v)
{
    if constexpr (N == 1) {
        return v[0];
    } else {
        constexpr int H = N / 2;
        return pairwise_sum<H>(v) + pairwise_sum<N - H>(v + H);
    }
}

__device__ __forceinline__ int wrapf(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Shared-memory rings of one CTA (size fixed per lattice type; the kernels
// take it as dynamic shared memory, 63,856 bytes for 32 x 8 D3Q27 tiles).
template <int LAT> struct SharedF {
    using L = LatF<LAT>;
    static constexpr int TX = L::TX, TY = L::TY, HY = L::HY;
    static constexpr int AX = TX + 4, AY = TY + 2 * HY;               // (rho, |psi|) halo tile
    static constexpr int GX = TX + 2, GY = LAT == 1 ? TY + 2 : 1;     // rho u^3 halo tile
    static constexpr int RS = 6, GS = 5;                               // ring slots
    float2 rp[RS][AY][AX];   // (rho, |psi|)
    float sg[RS][TY][TX];    // sign of P - P0, interior nodes
    float g[GS][3][GY][GX];  // rho u_a^3
    int xw[AX], yw[AY];      // wrapped halo coordinates
    float4 uv[4][TY][TX];    // (u_x, u_y, u_z, 1/rho) of the interior nodes, from phase A (forms
                             // without Tensor Memory staging)
    unsigned tmem;           // Tensor Memory base address (k_step_f32_tm)
};

// Shifted 16-bit storage also keeps the source densities of the planes in
// flight on a 3-node halo (the sources of the 2-halo's populations).
template <int LAT> struct SharedS : SharedF<LAT> {
    static constexpr int RX = SharedF<LAT>::AX + 2, RY = LAT == 1 ? SharedF<LAT>::AY + 2 : 1;
    static constexpr int QS = 8;   // ring slots (planes pl-4 .. pl+2 live)
    float rs[QS][RY][RX];
    int rxw[RX], ryw[RY];
};

// Population i of the node at halo coordinates (r, c) of ring plane q:
// stored value plus w_i times the density of its source node. With solid
// nodes (MASK), a population whose source r - c_i is solid was bounced back
// by the node itself and stored relative to the node's own density: solid
// nodes hold -1 in the source-density field, which selects the node's own.
template <int LAT, bool MASK = false, typename ST, typename SM>
__device__ __forceinline__ float decode_pop(ST hv, int i, int r, int c, int q, const SM &sm)
{
    if constexpr (IsShifted<ST>::value) {
        using L = LatF<LAT>;
        const int rr = r + (LAT == 1 ? 1 : 0) - L::cy(i), cc = c + 1 - L::cx(i);
        float src = sm.rs[(q - L::cz(i) + SM::QS) & (SM::QS - 1)][rr][cc];
        if (MASK && src < 0.0f) src = sm.rs[(q + SM::QS) & (SM::QS - 1)][r + (LAT == 1 ? 1 : 0)][c + 1];
        return (weight_f<LAT>(i) + to_f(hv)) * src;
    } else {
        return to_f(hv);
    }
}

// Source densities of one plane (ring index q) on the 3-halo into the ring.
template <int LAT, typename SM>
__device__ __forceinline__ void load_rho_plane(SM &sm, const GeoF &g, const float *__restrict__ rho_src,
                                               int z0, int q, int t, int nt)
{
    constexpr int RX = SM::RX, RY = SM::RY, QS = SM::QS;
    const int zq = ((z0 - 2 + q) % g.nz + g.nz) % g.nz;
    const unsigned plane = (unsigned)g.nx * (unsigned)g.ny;
    for (int k = t; k < RX * RY; k += nt) {
        const int r = k / RX, c = k - r * RX;
        sm.rs[(q + QS) & (QS - 1)][r][c] =
            __ldg(rho_src + ((unsigned)sm.rxw[c] + (unsigned)g.nx * (unsigned)sm.ryw[r] + plane * (unsigned)zq));
    }
}

// Shared-memory address of a generic pointer into shared memory.
__device__ __forceinline__ unsigned smem_u32(const void *ptr)
{
    return (unsigned)__cvta_generic_to_shared(ptr);
}

// ---- Tensor Memory staging of a node's populations --------------------
// Phase A loads every interior node's populations (its thread's first halo
// node) and phase B, two planes later, needs them again. Instead of a
// second read through L2, the thread keeps them in its own lane of the
// SM's Tensor Memory (tcgen05.st / tcgen05.ld, 32 x 32-bit per lane and
// column), four plane slots deep. Warp w reaches lanes 32 (w % 4) ..
// 32 (w % 4) + 31, so warps w and w + 4 share lanes and take separate
// column ranges. The block allocates TmemF::COLS columns (256 for D3Q27
// tiles, two blocks per SM fill the 512) and frees them before it exits.
template <int LAT> struct TmemF {
    static constexpr int Q = LatF<LAT>::Q;
    static constexpr int CPS = Q <= 16 ? 16 : 32;          // columns per plane slot
    static constexpr int SLOTS = 4;   // planes pl - 2 .. pl + 1 (the warp-specialised form needs 4)
    static constexpr int WARPS = LatF<LAT>::TX * LatF<LAT>::TY / 32;
    static constexpr int NEED = (WARPS + 3) / 4 * SLOTS * CPS;
    static constexpr int COLS = NEED <= 32 ? 32 : NEED <= 64 ? 64 : NEED <= 128 ? 128 : NEED <= 256 ? 256 : 512;
};

// Tensor Memory address of this thread's lane, plane slot `slot`.
template <int LAT>
__device__ __forceinline__ unsigned tmem_slot(unsigned base, int slot)
{
    using T = TmemF<LAT>;
    const int w = threadIdx.x >> 5;   // warps w and w + 8 (a producer and its consumer) share a lane range
    return base + ((unsigned)(32 * (w & 3)) << 16) +
           (unsigned)(((w & 7) >> 2) * T::SLOTS * T::CPS + slot * T::CPS);
}

__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Allocate ncols columns (one warp, all lanes); the base address lands in *dst.
__device__ __forceinline__ void tmem_alloc(unsigned *dst, unsigned ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n\t"
                 "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;"
                 ::"r"(smem_u32(dst)), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_dealloc(unsigned base, unsigned ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// Store the Q populations f and, in the columns after them, the kTmemExtra
// values x (when given) into this thread's lane at taddr (whole warp), and
// wait for the store to complete.
constexpr int kTmemExtra = 5;   // (u_x, u_y, u_z, 1/rho, sign of P - P0)

template <int Q>
__device__ __forceinline__ void tmem_store_pop(unsigned taddr, const float *f, const float *x = nullptr)
{
    constexpr int N = Q <= 16 ? 16 : 32;
    static_assert(Q + kTmemExtra <= N, "the extra values fit the plane slot");
    unsigned v[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
        v[i] = __float_as_uint(i < Q ? f[i] : (x && i - Q < kTmemExtra) ? x[i - Q] : f[0]);
    if constexpr (N == 32)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n\ttcgen05.wait::st.sync.aligned;" ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31]) : "memory");
    else
        asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n\ttcgen05.wait::st.sync.aligned;" ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]) : "memory");
}

// Load the Q populations of this thread's lane at taddr into f and, when x
// is given, the kTmemExtra values after them into x (whole warp).
template <int Q>
__device__ __forceinline__ void tmem_load_pop(unsigned taddr, float *f, float *x = nullptr)
{
    constexpr int N = Q <= 16 ? 16 : 32;
    unsigned v[N];
    if constexpr (N == 32)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\ttcgen05.wait::ld.sync.aligned;" : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]) : "r"(taddr) : "memory");
    else
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\ttcgen05.wait::ld.sync.aligned;" : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]) : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = __uint_as_float(v[i]);
    if (x)
#pragma unroll
        for (int k = 0; k < kTmemExtra; ++k) x[k] = __uint_as_float(v[Q + k]);
}

// Halo node k of a tile, interior nodes first: k < NT is the interior node
// (k / TX, k % TX), so a thread's first halo node is the node it collides in
// phase B; then the 2-node border: the HY top rows, the HY bottom rows, and
// two columns on either side of each interior row.
template <int LAT>
__device__ __forceinline__ void halo_rc(int k, int &r, int &c)
{
    using L = LatF<LAT>;
    constexpr int TX = L::TX, TY = L::TY, HY = L::HY, NT = TX * TY;
    constexpr int AX = SharedF<LAT>::AX, AY = SharedF<LAT>::AY;
    if (k < NT) {
        r = k / TX + HY;
        c = k % TX + 2;
        return;
    }
    int m = k - NT;
    if (m < HY * AX) {
        r = m / AX;
        c = m - r * AX;
        return;
    }
    m -= HY * AX;
    if (m < HY * AX) {
        const int q = m / AX;
        r = AY - HY + q;
        c = m - q * AX;
        return;
    }
    m -= HY * AX;
    const int e = m & 3;
    r = HY + (m >> 2);
    c = e < 2 ? e : AX - 4 + e;
}

// Per-tile constants of one CTA's work: the column tile at (x0, y0) over the
// planes z0 .. z1-1; planes z0-2 .. z1+1 enter the rings one per iteration,
// plane z0-2+pl with ring index pl, np iterations.
struct TileF {
    int x0, y0, z0, z1, np;
};

// Wrapped halo coordinates of the tile (bx, by, bz) and, for shifted
// storage, the source densities of its first planes; threads t = 0..nt-1 of
// the CTA share the work. The caller synchronises before the rings are used.
template <int LAT, typename ST, typename SM>
__device__ __forceinline__ TileF tile_setup(const GeoF &g, int bx, int by, int bz, SM &sm, int t,
                                            int nt, const float *__restrict__ rho_src)
{
    using L = LatF<LAT>;
    constexpr bool THREE = LAT == 1;
    constexpr int AX = SharedF<LAT>::AX, AY = SharedF<LAT>::AY, HY = L::HY;
    TileF T;
    T.x0 = bx * L::TX;
    T.y0 = by * L::TY;
    T.z0 = bz * g.chunk;
    T.z1 = min(T.z0 + g.chunk, g.nz);
    T.np = (T.z1 - T.z0) + 4;
    for (int c = t; c < AX; c += nt) sm.xw[c] = ((T.x0 - 2 + c) % g.nx + g.nx) % g.nx;
    for (int r = t; r < AY; r += nt) sm.yw[r] = THREE ? ((T.y0 - HY + r) % g.ny + g.ny) % g.ny : 0;
    if constexpr (IsShifted<ST>::value) {
        for (int c = t; c < SM::RX; c += nt) sm.rxw[c] = ((T.x0 - 3 + c) % g.nx + g.nx) % g.nx;
        for (int r = t; r < SM::RY; r += nt)
            sm.ryw[r] = THREE ? ((T.y0 - HY - 1 + r) % g.ny + g.ny) % g.ny : 0;
        __syncthreads();
        load_rho_plane<LAT>(sm, g, rho_src, T.z0, -1, t, nt);
        load_rho_plane<LAT>(sm, g, rho_src, T.z0, 0, t, nt);
        load_rho_plane<LAT>(sm, g, rho_src, T.z0, 1, t, nt);
    }
    return T;
}

// Phase A of iteration pl: plane z0 - 2 + pl enters the rings (ring index
// pl): (rho, |psi|) on the 2-node halo, rho u_a^3 on the 1-node halo, the sign
// of P - P0 and (u, 1/rho) of the interior nodes (in shared memory, or with
// the node's populations in Tensor Memory: TMX, the warp-specialised Tensor
// Memory forms); thread tid of NT. Each
// thread owns up to KA halo nodes and issues all their loads before any
// arithmetic, for memory-level parallelism.
// With BOXED (the TMA-staged form, D3Q27 32 x 8 tiles) the plane's
// populations on the halo tile are already in shared memory (`box`), and
// the halo nodes are taken in the order of halo_rc_boxed; a node whose
// coordinates the box does not hold (a ragged tile's wrapped nodes: the box
// holds the fill value there) is read from global memory as before.
//
// The box of one plane in nine dense TMA boxes (D3Q27 32 x 8 tiles): rows
// top (y0 - 2, y0 - 1), middle (y0 .. y0 + 7), bottom (y0 + 8, y0 + 9) by
// columns left (x0 - W .. x0 - 1), centre (x0 .. x0 + 31), right (x0 + 32 ..
// x0 + 31 + W), each [i][row][column] of the stored type ST and fetched from
// its own wrapped origin, so that a tile on the lattice's edge finds its
// periodic halo there too. Left and right boxes are W = 16 bytes wide (4
// FP32 or 8 16-bit columns), the narrowest a box with 16-byte aligned rows
// can be (halo columns x0 - 2, x0 - 1 and x0 + 32, x0 + 33 are its last two
// and first two). A tiled bulk tensor copy writes shared memory from a
// 128-byte aligned address, so each box starts on one (FP32 corners of 864
// bytes are padded to 896).
template <typename ST> struct BoxT {
    static constexpr int Q = 27, W = 16 / (int)sizeof(ST);
    alignas(128) ST mc[Q][8][32];
    alignas(128) ST tc[Q][2][32];
    alignas(128) ST bc[Q][2][32];
    alignas(128) ST ml[Q][8][W];
    alignas(128) ST mr[Q][8][W];
    alignas(128) ST tl[Q][2][W];
    alignas(128) ST tr[Q][2][W];
    alignas(128) ST bl[Q][2][W];
    alignas(128) ST br[Q][2][W];
    // bytes the nine copies of one plane deliver (without the padding)
    static constexpr unsigned BYTES = Q * sizeof(ST) * (8 * 32 + 2 * 2 * 32 + 2 * 8 * W + 4 * 2 * W);
    // A tile whose halo neither wraps nor leaves the lattice can take the
    // plane in one copy instead: [i][row][column], 12 rows of WX = 32 + 2 W
    // columns from (x0 - W, y0 - 2), in the same space.
    static constexpr int WX = 32 + 2 * W;
    static constexpr unsigned WIDE_BYTES = Q * 12 * WX * sizeof(ST);
    __device__ const ST *wide() const { return &mc[0][0][0]; }
};
using BoxS = BoxT<float>;
static_assert(BoxT<float>::WIDE_BYTES <= sizeof(BoxT<float>) && BoxT<__half>::WIDE_BYTES <= sizeof(BoxT<__half>),
              "the one-copy layout fits the nine boxes' space");
template <typename B>
constexpr bool boxes_aligned()
{
    return offsetof(B, tc) % 128 == 0 && offsetof(B, bc) % 128 == 0 && offsetof(B, ml) % 128 == 0 &&
           offsetof(B, mr) % 128 == 0 && offsetof(B, tl) % 128 == 0 && offsetof(B, tr) % 128 == 0 &&
           offsetof(B, bl) % 128 == 0 && offsetof(B, br) % 128 == 0 && sizeof(B) % 128 == 0;
}
static_assert(boxes_aligned<BoxT<float>>() && boxes_aligned<BoxT<__half>>() &&
                  boxes_aligned<BoxT<__nv_bfloat16>>(),
              "every box starts on a 128-byte boundary");

// Halo node k of a 32 x 8 tile in the TMA-staged order: interior nodes first
// (as halo_rc), then the centre columns of the two top and two bottom rows
// (four warps), the four side columns of the middle rows (one warp) and the
// four 2 x 2 corners (half a warp), so that each warp reads one kind of box.
__device__ __forceinline__ void halo_rc_boxed(int k, int &r, int &c)
{
    if (k < 256) {
        r = (k >> 5) + 2;
        c = (k & 31) + 2;
        return;
    }
    const int m = k - 256;
    if (m < 128) {   // rows 0, 1 (m < 64) and 10, 11, centre columns
        const int q = m >> 5;
        r = q < 2 ? q : q + 8;
        c = (m & 31) + 2;
    } else if (m < 160) {   // middle rows, columns 0, 1, 34, 35
        const int e = m & 3;
        r = 2 + ((m - 128) >> 2);
        c = e < 2 ? e : e + 32;
    } else {   // corners: rows 0, 1, 10, 11 by columns 0, 1, 34, 35
        const int e = m & 3, q = (m - 160) >> 2;
        r = q < 2 ? q : q + 8;
        c = e < 2 ? e : e + 32;
    }
}

// The 27 populations of halo node (r, c) of ring plane pl from the one-copy
// layout into v, decoded (shifted storage) as decode_pop does.
template <int LAT, bool MASK, typename ST, typename SM, typename V>
__device__ __forceinline__ void load_from_wide(const BoxT<ST> &b, int r, int c, int pl, const SM &sm, V &v)
{
    using B = BoxT<ST>;
    const ST *q = b.wide() + r * B::WX + c - 2 + B::W;
#pragma unroll
    for (int i = 0; i < 27; ++i) v[i] = decode_pop<LAT, MASK>(q[i * 12 * B::WX], i, r, c, pl, sm);
}

// The 27 populations of halo node (r, c) of ring plane pl from the box into
// v, decoded (shifted storage) as decode_pop does.
template <int LAT, bool MASK, typename ST, typename SM, typename V>
__device__ __forceinline__ void load_from_box(const BoxT<ST> &b, int r, int c, int pl, const SM &sm, V &v)
{
    constexpr int W = BoxT<ST>::W;
    const int rc = r < 2 ? 0 : r < 10 ? 1 : 2;   // top, middle, bottom
    const int cc = c < 2 ? 0 : c < 34 ? 1 : 2;   // left, centre, right
    const int rr = rc == 0 ? r : rc == 1 ? r - 2 : r - 10;
    const int xx = cc == 0 ? c + W - 2 : cc == 1 ? c - 2 : c - 34;
    if (rc == 1 && cc == 1) {
#pragma unroll
        for (int i = 0; i < 27; ++i) v[i] = decode_pop<LAT, MASK>(b.mc[i][rr][xx], i, r, c, pl, sm);
    } else if (cc == 1) {
        const ST *q = rc == 0 ? &b.tc[0][rr][xx] : &b.bc[0][rr][xx];
#pragma unroll
        for (int i = 0; i < 27; ++i) v[i] = decode_pop<LAT, MASK>(q[i * 64], i, r, c, pl, sm);
    } else if (rc == 1) {
        const ST *q = cc == 0 ? &b.ml[0][rr][xx] : &b.mr[0][rr][xx];
#pragma unroll
        for (int i = 0; i < 27; ++i) v[i] = decode_pop<LAT, MASK>(q[i * 8 * W], i, r, c, pl, sm);
    } else {
        const ST *q = rc == 0 ? (cc == 0 ? &b.tl[0][rr][xx] : &b.tr[0][rr][xx])
                              : (cc == 0 ? &b.bl[0][rr][xx] : &b.br[0][rr][xx]);
#pragma unroll
        for (int i = 0; i < 27; ++i) v[i] = decode_pop<LAT, MASK>(q[i * 2 * W], i, r, c, pl, sm);
    }
}

template <int LAT, bool MASK, bool TM = false, bool E64 = false, bool TMX = false, bool BOXED = false,
          int EOSK = -1, typename ST, typename SM>
__device__ __forceinline__ void phase_a(const GeoF &g, const PhysF &p,
                                        const uint8_t *__restrict__ mask,
                                        const ST *__restrict__ f, SM &sm, const TileF &T,
                                        int pl, int tid, const float *__restrict__ rho_src,
                                        unsigned tbase = 0, const BoxT<ST> *box = nullptr,
                                        bool wide_box = false)
{
    constexpr bool SHIFT = IsShifted<ST>::value;
    using L = LatF<LAT>;
    constexpr int Q = L::Q, TX = L::TX, TY = L::TY, HY = L::HY;
    constexpr bool THREE = LAT == 1;
    constexpr int NT = TX * TY;
    constexpr int AX = SharedF<LAT>::AX, AY = SharedF<LAT>::AY;
    constexpr int RS = SharedF<LAT>::RS, GS = SharedF<LAT>::GS;
    auto &s_rp = sm.rp;
    auto &s_sg = sm.sg;
    auto &s_g = sm.g;
    auto &s_xw = sm.xw;
    auto &s_yw = sm.yw;
    const int z0 = T.z0;
    const unsigned N = g.N;
    const unsigned plane = (unsigned)g.nx * (unsigned)g.ny;
    constexpr int KA = (AX * AY + NT - 1) / NT;
    const int zl = wrapf(z0 - 2 + pl, g.nz);
    const int rs = pl % RS, gs = pl % GS;
    const bool msk = MASK && g.zsolid[zl];   // the plane holds a solid node
    // Solid halo nodes: handled inline, or (BOXED) by a pass after the
    // fluid computation that overwrites what it wrote for them, so that the
    // main path is the one of a lattice without solids
    constexpr bool SOLID_INLINE = MASK && !BOXED;
    float fi[KA][Q];
    float ex[kTmemExtra] = {};   // TMX: (u, 1/rho, sign) of the interior node, kept in Tensor Memory
    unsigned nk[KA];
    bool live[KA], solid[KA];
    if constexpr (SHIFT) load_rho_plane<LAT>(sm, g, rho_src, z0, pl + 2, tid, NT);   // for the next iteration
#pragma unroll
    for (int u = 0; u < KA; ++u) {
        const int k = tid + u * NT;
        live[u] = k < AX * AY;
        int r, c;
        if constexpr (BOXED) halo_rc_boxed(live[u] ? k : 0, r, c);
        else                 halo_rc<LAT>(live[u] ? k : 0, r, c);
        nk[u] = (unsigned)s_xw[c] + (unsigned)g.nx * (unsigned)s_yw[r] + plane * (unsigned)zl;
        solid[u] = SOLID_INLINE && live[u] && msk && mask[nk[u]];
        if (live[u] && !solid[u]) {
            bool in_box = false;
            if constexpr (BOXED) in_box = sm.xok[c] && sm.yok[r];
            if (in_box) {
                if constexpr (BOXED) {
                    if (wide_box) load_from_wide<LAT, MASK>(*box, r, c, pl, sm, fi[u]);
                    else          load_from_box<LAT, MASK>(*box, r, c, pl, sm, fi[u]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) fi[u][i] = decode_pop<LAT, MASK>(__ldg(f + (i * N + nk[u])), i, r, c, pl, sm);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < KA; ++u) {
        if (!live[u]) continue;
        int r, c;
        if constexpr (BOXED) halo_rc_boxed(tid + u * NT, r, c);
        else                 halo_rc<LAT>(tid + u * NT, r, c);
        const bool ring1 = c >= 1 && c < AX - 1 && (!THREE || (r >= 1 && r < AY - 1));
        float rho, d, psi64 = 0.0f, gx = 0.0f, gy = 0.0f, gz = 0.0f;
        float4 uvk = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (solid[u]) {
            rho = p.rho_w;
            d = p.spsi_w;
        } else {
            // x-row sums for each (cy, cz), then the moments from them, each
            // summed pairwise (short dependency chains)
            constexpr int R = Q / 3;
            float row[R], dx[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                row[q] = (fi[u][3 * q] + fi[u][3 * q + 1]) + fi[u][3 * q + 2];
                dx[q] = fi[u][3 * q + 2] - fi[u][3 * q];
            }
            rho = pairwise_sum<R>(row);
            const float jx = pairwise_sum<R>(dx);
            if (ring1) {
                // D3Q27 rows q = (cy + 1) + 3 (cz + 1); D2Q9 rows q = cz + 1
                const float jy = THREE ? ((row[2] + row[5]) + row[8]) - ((row[0] + row[3]) + row[6]) : 0.0f;
                const float jz = THREE ? ((row[6] + row[7]) + row[8]) - ((row[0] + row[1]) + row[2])
                                       : row[R - 1] - row[0];
                const float inv = __frcp_rn(rho);
                const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
                gx = rho * ux * ux * ux;
                gy = rho * uy * uy * uy;
                gz = rho * uz * uz * uz;
                uvk = make_float4(ux, uy, uz, inv);
            }
            if constexpr (E64) {
                const double dd = excess_pressure_d(p, (double)rho);
                d = (float)dd;
                psi64 = (float)sqrt(fabs(dd));
            } else {
                d = excess_pressure_ft<EOSK>(p, rho);
            }
        }
        s_rp[rs][r][c] = f2(rho, E64 && !solid[u] ? psi64 : sqrtf(fabsf(d)));
        if (ring1) {
            const int gr = THREE ? r - 1 : 0;
            s_g[gs][0][gr][c - 1] = gx;
            s_g[gs][1][gr][c - 1] = gy;
            s_g[gs][2][gr][c - 1] = gz;
        }
        if constexpr (TMX) {
            if (u == 0) {   // the interior node (halo node tid < NT)
                ex[0] = uvk.x;
                ex[1] = uvk.y;
                ex[2] = uvk.z;
                ex[3] = uvk.w;
                ex[4] = d > 0.0f ? 1.0f : -1.0f;
            }
        } else {
            const int ir = r - HY, ic = c - 2;
            if (ir >= 0 && ir < TY && ic >= 0 && ic < TX) {
                s_sg[rs][ir][ic] = d > 0.0f ? 1.0f : -1.0f;
                sm.uv[pl & 3][ir][ic] = uvk;
            }
        }
    }
    if constexpr (MASK && BOXED) {
        // the solid nodes of the plane: the wall's (rho_w, |psi_w|), no rho u^3
        // (phase B skips solid nodes, so their other values go unread)
        if (msk) {
#pragma unroll
            for (int u = 0; u < KA; ++u) {
                if (!live[u]) continue;
                int r, c;
                halo_rc_boxed(tid + u * NT, r, c);
                if (!mask[(unsigned)s_xw[c] + (unsigned)g.nx * (unsigned)s_yw[r] + plane * (unsigned)zl]) continue;
                s_rp[rs][r][c] = f2(p.rho_w, sqrtf(fabsf(p.spsi_w)));
                if (c >= 1 && c < AX - 1 && r >= 1 && r < AY - 1) {
                    s_g[gs][0][r - 1][c - 1] = 0.0f;
                    s_g[gs][1][r - 1][c - 1] = 0.0f;
                    s_g[gs][2][r - 1][c - 1] = 0.0f;
                }
            }
        }
    }
    // the thread's interior node (its halo node tid), for phase B two planes
    // on: populations, bare velocity, 1/rho and the sign of P - P0
    if constexpr (TM) {
        __syncwarp();   // tcgen05.st is warp-collective: reconverge after the loops
        tmem_store_pop<Q>(tmem_slot<LAT>(tbase, pl & 3), fi[0], TMX ? ex : nullptr);
    }
}

// Phase B of iteration pl >= 4: the tile's nodes on plane zc = z0 + pl - 4
// (ring index pl - 2) collide with all stencil reads from the rings and push
// their post-collision populations with halfway bounce-back; thread tid of
// NT owns node (tid % TX, tid / TX), which the caller has checked to lie in
// the lattice (a ragged tile's last columns or rows may not).
template <int LAT, bool MASK, bool TM = false, bool E64 = false, bool TMX = false, typename ST, typename SM>
__device__ __forceinline__ void phase_b(const GeoF &g, const PhysF &p,
                                        const uint8_t *__restrict__ mask,
                                        const ST *__restrict__ f, ST *__restrict__ fout,
                                        int *__restrict__ status, SM &sm, const TileF &T, int pl,
                                        int tid, float *__restrict__ rho_dst, unsigned tbase = 0,
                                        bool inside = true)
{
    constexpr bool SHIFT = IsShifted<ST>::value;
    using L = LatF<LAT>;
    constexpr int Q = L::Q, TX = L::TX, HY = L::HY;
    constexpr bool THREE = LAT == 1;
    constexpr int RS = SharedF<LAT>::RS, GS = SharedF<LAT>::GS;
    auto &s_rp = sm.rp;
    auto &s_sg = sm.sg;
    auto &s_g = sm.g;
    const int z0 = T.z0;
    const int tx = tid % TX, ty = tid / TX;
    const int xi = T.x0 + tx, yi = T.y0 + ty;
    const unsigned N = g.N;
    const unsigned plane = (unsigned)g.nx * (unsigned)g.ny;
    const int pc = pl - 2;             // ring index of the collided plane
    const int zc = z0 + pl - 4;
    const unsigned n = (unsigned)xi + (unsigned)g.nx * (unsigned)yi + plane * (unsigned)zc;
    // the node's own populations: from Tensor Memory, where phase A left them
    // (all lanes of the warp take part), or read again (an L2 hit), first
    float fi[Q];
    float ex[kTmemExtra] = {};   // TMX: (u, 1/rho, sign) from phase A, through Tensor Memory
    if constexpr (TM) {
        __syncwarp();   // tcgen05.ld is warp-collective
        tmem_load_pop<Q>(tmem_slot<LAT>(tbase, pc & 3), fi, TMX ? ex : nullptr);
        if (!inside) return;
    }
    if (!(MASK && g.zsolid[zc] && mask[n])) {
        if constexpr (!TM) {
#pragma unroll
            for (int i = 0; i < Q; ++i) fi[i] = decode_pop<LAT, MASK>(__ldg(f + (i * N + n)), i, ty + HY, tx + 2, pc, sm);
        }
        const int cr = ty + HY, cc = tx + 2;
        const float2 c0 = s_rp[pc % RS][cr][cc];
        const float rho = c0.x;
        const float spsi = (TMX ? ex[4] : s_sg[pc % RS][ty][tx]) * c0.y;
        if (!(rho > 0.0f) || !isfinite(rho)) atomicOr(status, 1);
        if constexpr (SHIFT) rho_dst[n] = rho;   // source density of what this node pushes
        // Korteweg force (Eq. Kforce_final, sign as the force on the fluid).
        // Per ring s, the pairs (|psi|, rho) of neighbours with c_a = +1 and
        // c_a = -1 are summed by weight class (centre, edge, corner).
        int slot[5];
#pragma unroll
        for (int dz = 0; dz < 5; ++dz) slot[dz] = (pc - 2 + dz) % RS;
        float F[3];
        if constexpr (E64) {
            // the same sums in FP64: neighbours widened, sums and force in FP64
            double Sp[3] = {0.0, 0.0, 0.0}, Sr[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int s = 1; s <= 2; ++s) {
                double Pp[3][3], Pr[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int k = 0; k < 3; ++k) Pp[a][k] = Pr[a][k] = 0.0;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
                    if (c[0] == 0 && c[1] == 0 && c[2] == 0) continue;
                    const float2 r2 = s_rp[slot[2 + s * c[2]]][cr + s * c[1]][cc + s * c[0]];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (c[a] == 0) continue;
                        const int k = (a != 0 && c[0] != 0) + (a != 1 && c[1] != 0) +
                                      (a != 2 && c[2] != 0);
                        Pp[a][k] += c[a] * (double)r2.y;
                        Pr[a][k] += c[a] * (double)r2.x;
                    }
                }
                const double gp = s == 1 ? 4.0 / 3.0 : -1.0 / 6.0, gr = s == 1 ? 2.0 : -1.0;
                const double w0 = THREE ? 2.0 / 9.0 : 1.0 / 3.0, w1 = THREE ? 1.0 / 18.0 : 1.0 / 12.0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (!THREE && a == 1) continue;
                    Sp[a] += gp * (w0 * Pp[a][0] + w1 * Pp[a][1] + (THREE ? Pp[a][2] / 72.0 : 0.0));
                    Sr[a] += gr * (w0 * Pr[a][0] + w1 * Pr[a][1] + (THREE ? Pr[a][2] / 72.0 : 0.0));
                }
            }
            const double rd = rho, sd = (double)s_sg[pc % RS][ty][tx] * (double)c0.y;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                F[a] = (float)(rd * (double)p.g[a] - 2.0 * sd * Sp[a] - p.dkappa * rd * Sr[a]);
        } else {
        float2 S[3] = {f2(0.0f, 0.0f), f2(0.0f, 0.0f), f2(0.0f, 0.0f)};   // (S_psi, S_rho)
        const float2 neg1 = f2(-1.0f, -1.0f);
#pragma unroll
        for (int s = 1; s <= 2; ++s) {
            float2 P[3][3], M[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int k = 0; k < 3; ++k) { P[a][k] = f2(0.0f, 0.0f); M[a][k] = f2(0.0f, 0.0f); }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
                if (c[0] == 0 && c[1] == 0 && c[2] == 0) continue;
                const float2 r2 = s_rp[slot[2 + s * c[2]]][cr + s * c[1]][cc + s * c[0]];
                const float2 v = f2(r2.y, r2.x);   // (|psi|, rho)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (c[a] == 0) continue;
                    const int k = (a != 0 && c[0] != 0) + (a != 1 && c[1] != 0) +
                                  (a != 2 && c[2] != 0);
                    if (c[a] > 0) P[a][k] = __fadd2_rn(P[a][k], v);
                    else          M[a][k] = __fadd2_rn(M[a][k], v);
                }
            }
            // weights w_i/cs2 c_a = 1/2 W(c_b) W(c_c): D3Q27 2/9, 1/18, 1/72;
            // D2Q9 1/3, 1/12; ring coefficients (4/3, 2) and (-1/6, -1)
            const float2 gsr = s == 1 ? f2(4.0f / 3.0f, 2.0f) : f2(-1.0f / 6.0f, -1.0f);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (!THREE && a == 1) continue;
                const float2 D0 = __ffma2_rn(M[a][0], neg1, P[a][0]);
                const float2 D1 = __ffma2_rn(M[a][1], neg1, P[a][1]);
                float2 Dw;
                if (THREE) {
                    const float2 D2 = __ffma2_rn(M[a][2], neg1, P[a][2]);
                    Dw = __fmul2_rn(D0, f2(2.0f / 9.0f, 2.0f / 9.0f));
                    Dw = __ffma2_rn(D1, f2(1.0f / 18.0f, 1.0f / 18.0f), Dw);
                    Dw = __ffma2_rn(D2, f2(1.0f / 72.0f, 1.0f / 72.0f), Dw);
                } else {
                    Dw = __fmul2_rn(D0, f2(1.0f / 3.0f, 1.0f / 3.0f));
                    Dw = __ffma2_rn(D1, f2(1.0f / 12.0f, 1.0f / 12.0f), Dw);
                }
                S[a] = __ffma2_rn(Dw, gsr, S[a]);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)   // Korteweg force plus the body force rho g
            F[a] = __fmaf_rn(rho, p.g[a], -2.0f * spsi * S[a].x - p.kappa * rho * S[a].y);
        }
        // Phi_aa = -(1 - omega/2) (g_a(r + e_a) - g_a(r - e_a)) / 2, the node's omega
        const float om = p.var_visc ? omega_var_f(p, rho) : p.omega;
        const float pref = p.var_visc ? p.phi_sign * (1.0f - 0.5f * om) : p.phi_pref;
        const float omw = p.var_visc ? 1.0f - om : p.omw;
        const int gr0 = THREE ? ty + 1 : 0, gc0 = tx + 1;
        float Phi[3];
        Phi[0] = pref * 0.5f * (s_g[pc % GS][0][gr0][gc0 + 1] - s_g[pc % GS][0][gr0][gc0 - 1]);
        Phi[1] = THREE ? pref * 0.5f *
                             (s_g[pc % GS][1][gr0 + 1][gc0] - s_g[pc % GS][1][gr0 - 1][gc0])
                       : 0.0f;
        Phi[2] = pref * 0.5f *
                 (s_g[(pc + 1) % GS][2][gr0][gc0] - s_g[(pc - 1) % GS][2][gr0][gc0]);
        // bare velocity and 1/rho of the node, formed by phase A from the same populations
        const float4 uvn = TMX ? make_float4(ex[0], ex[1], ex[2], ex[3]) : sm.uv[pc & 3][ty][tx];
        const float inv = uvn.w;
        const float un[3] = {uvn.x, uvn.y, uvn.z};
        // product-form factors, paired (equilibrium, extended)
        float2 ES[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!THREE && a == 1) {
                ES[1][0] = ES[1][1] = ES[1][2] = f2(1.0f, 1.0f);
                continue;
            }
            const float ua = un[a];
            const float ze = 1.0f / 3.0f + ua * ua;
            const float xs = ua + F[a] * inv;
            const float zs = 1.0f / 3.0f + xs * xs + Phi[a] * inv;
            ES[a][0] = f2(0.5f * (ze - ua), 0.5f * (zs - xs));
            ES[a][1] = f2(1.0f - ze, 1.0f - zs);
            ES[a][2] = f2(0.5f * (ze + ua), 0.5f * (zs + xs));
        }
        float2 A[3][3];
        const float2 rr = f2(rho, rho);
#pragma unroll
        for (int cx = 0; cx < 3; ++cx) {
            const float2 rx = __fmul2_rn(rr, ES[0][cx]);
#pragma unroll
            for (int cy = 0; cy < 3; ++cy) A[cx][cy] = __fmul2_rn(rx, ES[1][cy]);
        }
        // post = f* + (1 - omega)(f - feq), pushed to r + c_i
        const int X[3] = {wrapf(xi - 1, g.nx), xi, wrapf(xi + 1, g.nx)};
        const int Y[3] = {THREE ? wrapf(yi - 1, g.ny) : 0, yi, THREE ? wrapf(yi + 1, g.ny) : 0};
        const int Z[3] = {wrapf(zc - 1, g.nz), zc, wrapf(zc + 1, g.nz)};
        // Solids among the destinations are looked up only where one of the
        // planes zc - 1 .. zc + 1 holds a solid node.
        if (MASK && planes_solid3(g, zc)) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
                const float2 es = __fmul2_rn(A[cx + 1][cy + 1], ES[2][cz + 1]);   // (feq, f*)
                const float post = SHIFT ? fmaf(fmaf(omw, fi[i] - es.x, es.y), inv, -weight_f<LAT>(i))
                                         : fmaf(omw, fi[i] - es.x, es.y);
                const unsigned dst = (unsigned)X[cx + 1] + (unsigned)g.nx * (unsigned)Y[cy + 1] +
                                     plane * (unsigned)Z[cz + 1];
                if (mask[dst]) fout[(Q - 1 - i) * N + n] = from_f<ST>(post);
                else           fout[i * N + dst] = from_f<ST>(post);
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
                const float2 es = __fmul2_rn(A[cx + 1][cy + 1], ES[2][cz + 1]);   // (feq, f*)
                const float post = SHIFT ? fmaf(fmaf(omw, fi[i] - es.x, es.y), inv, -weight_f<LAT>(i))
                                         : fmaf(omw, fi[i] - es.x, es.y);
                const unsigned dst = (unsigned)X[cx + 1] + (unsigned)g.nx * (unsigned)Y[cy + 1] +
                                     plane * (unsigned)Z[cz + 1];
                fout[i * N + dst] = from_f<ST>(post);
            }
        }
    }
}

// One CTA's work: the column tile (bx, by) over the plane chunk bz. Six
// (rho, |psi|) slots and five rho u^3 slots let the next plane enter while
// slower warps still collide: one barrier per plane.
template <int LAT, bool MASK, typename ST = float, typename SM = SharedF<LAT>, bool TM = false,
          bool E64 = false>
__device__ __forceinline__ void fused_tile(const GeoF &g, const PhysF &p,
                                           const uint8_t *__restrict__ mask,
                                           const ST *__restrict__ f, ST *__restrict__ fout,
                                           int *__restrict__ status, int bx, int by, int bz,
                                           SM &sm, const float *__restrict__ rho_src = nullptr,
                                           float *__restrict__ rho_dst = nullptr,
                                           unsigned tbase = 0)
{
    constexpr int TX = LatF<LAT>::TX, NT = TX * LatF<LAT>::TY;
    const int tid = threadIdx.x;
    const TileF T = tile_setup<LAT, ST>(g, bx, by, bz, sm, tid, NT, rho_src);
    const bool inside = T.x0 + tid % TX < g.nx && T.y0 + tid / TX < g.ny;
    __syncthreads();
    for (int pl = 0; pl < T.np; ++pl) {
        phase_a<LAT, MASK, TM, E64>(g, p, mask, f, sm, T, pl, tid, rho_src, tbase);
        __syncthreads();
        if (TM ? pl >= 4 : pl >= 4 && inside)
            phase_b<LAT, MASK, TM, E64>(g, p, mask, f, fout, status, sm, T, pl, tid, rho_dst, tbase, inside);
    }
}

// ---- warp-specialised form --------------------------------------------
// The same tile with two thread groups of NT: producers run phase A, and
// consumers run phase B, handing planes over through mbarriers instead of a
// CTA-wide barrier per plane, so the loads and moments of the next planes
// overlap the collision of the current one.
//   full[pl % 6] completes when the producers have written ring index pl;
//     the consumers wait for it before iteration pl (which reads ring
//     indices up to pl).
//   empty[j % 6] completes when the consumers have finished iteration j >= 4;
//     producer iteration pl >= 6 waits for iteration pl - 2, the last reader
//     of every ring slot that pl overwrites ((rho, |psi|) slot pl % 6 held
//     pl - 6, read up to iteration pl - 2; rho u^3 slot pl % 5 held pl - 5,
//     read up to iteration pl - 2; (u, 1/rho) slot pl % 4 held pl - 4, read in
//     iteration pl - 2).
// Each barrier completes once per use of its slot, and neither side can get
// a full cycle ahead of the other, so waiting on the phase parity is exact.
// Every wait gives up after about a second (kWaitCycles), sets bit 2 of the
// status word and returns: the step then reports an error instead of hanging.
constexpr long long kWaitCycles = 2000000000ll;

template <int LAT> struct SharedWS : SharedF<LAT> {
    unsigned long long full[6], empty[6];
};

// The same with the source-density ring of shifted 16-bit storage, and two
// producer-only barriers (pbar[pl % 2] completes when every producer has
// finished iteration pl, its source-density plane included).
template <int LAT> struct SharedSWS : SharedS<LAT> {
    unsigned long long full[6], empty[6], pbar[2];
};

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Arrive with release semantics: this thread's shared-memory writes are
// visible to a thread whose wait observes the phase completion.
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

// Wait (acquire) for the completion of the phase of the given parity;
// false after `limit` clock cycles without it.
__device__ __forceinline__ bool mbar_wait_for(unsigned long long *bar, unsigned parity, long long limit)
{
    const long long t0 = clock64();
    for (;;) {
        unsigned done;
        asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, q;\n\t}"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    return mbar_wait_for(bar, parity, kWaitCycles);
}

// Self-test of the bounded waits: each warp of one block waits, through the
// wait the fused kernels use, for a barrier phase that nothing completes
// (no thread arrives), gives up after `limit` cycles, records it as the
// kernels do (bit 2 of the status word) and returns. A template so that
// only the build that launches it instantiates it.
template <int N = 1>
__global__ void k_wait_selftest(int *__restrict__ status, long long limit)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) mbar_init(&bar, N);
    __syncthreads();
    if (!mbar_wait_for(&bar, 0, limit) && (threadIdx.x & 31) == 0) atomicOr(status, 2);
}

// Shifted storage (ST 16-bit, SM = SharedSWS): the producers also keep the
// source-density ring, which only they read (the consumers take the decoded
// populations from Tensor Memory: TM), and wait for one another once per
// plane (pbar, bounded like the other waits) so that the plane one producer
// loads is in place before another decodes with it. Producer iteration pl
// waits for pbar[(pl - 1) % 2]'s completion of iteration pl - 1; the next
// arrival on that barrier (iteration pl + 1) comes from a producer that has
// seen iteration pl complete, so after every producer's wait: parity exact.
template <int LAT, bool MASK, bool TM = false, typename ST = float, typename SM = SharedWS<LAT>>
__device__ __forceinline__ void fused_tile_ws(const GeoF &g, const PhysF &p,
                                              const uint8_t *__restrict__ mask,
                                              const ST *__restrict__ f, ST *__restrict__ fout,
                                              int *__restrict__ status, int bx, int by, int bz,
                                              SM &sm, unsigned tbase = 0,
                                              const float *__restrict__ rho_src = nullptr,
                                              float *__restrict__ rho_dst = nullptr)
{
    constexpr bool SHIFT = IsShifted<ST>::value;
    constexpr int TX = LatF<LAT>::TX, NT = TX * LatF<LAT>::TY;
    static_assert(!TM || NT % 256 == 0, "a consumer warp shares its producer's Tensor Memory lanes");
    static_assert(!SHIFT || TM, "shifted storage hands the decoded populations over in Tensor Memory");
    const int tid = threadIdx.x;
    const TileF T = tile_setup<LAT, ST>(g, bx, by, bz, sm, tid, 2 * NT, rho_src);
    if (tid == 0) {
        for (int k = 0; k < 6; ++k) {
            mbar_init(&sm.full[k], NT);
            mbar_init(&sm.empty[k], NT);
        }
        if constexpr (SHIFT)
            for (int k = 0; k < 2; ++k) mbar_init(&sm.pbar[k], NT);
    }
    __syncthreads();
    // A wait that runs out sets bit 2 of the status and ends this group's
    // loop; the other group's next wait then runs out too, so every thread
    // reaches the end of the tile (where the caller may free Tensor Memory).
    if (tid < NT) {
        for (int pl = 0; pl < T.np; ++pl) {
            if (pl >= 6 && !mbar_wait(&sm.empty[(pl - 2) % 6], ((pl - 6) / 6) & 1)) {
                atomicOr(status, 2);
                break;
            }
            if constexpr (SHIFT) {   // the source densities loaded in iteration pl - 1 are in place
                if (pl > 0 && !mbar_wait(&sm.pbar[(pl - 1) & 1], ((pl - 1) >> 1) & 1)) {
                    atomicOr(status, 2);
                    break;
                }
            }
            if constexpr (TM) tmem_fence_after();
            phase_a<LAT, MASK, TM, false, TM>(g, p, mask, f, sm, T, pl, tid, rho_src, tbase);
            if constexpr (TM) tmem_fence_before();
            if constexpr (SHIFT) mbar_arrive(&sm.pbar[pl & 1]);
            mbar_arrive(&sm.full[pl % 6]);
        }
    } else {
        const int t = tid - NT;
        const bool inside = T.x0 + t % TX < g.nx && T.y0 + t / TX < g.ny;
        for (int pl = 0; pl < T.np; ++pl) {
            if (!mbar_wait(&sm.full[pl % 6], (pl / 6) & 1)) {
                atomicOr(status, 2);
                break;
            }
            if (pl >= 4) {
                if constexpr (TM) {
                    tmem_fence_after();
                    phase_b<LAT, MASK, true, false, true>(g, p, mask, f, fout, status, sm, T, pl, t, rho_dst,
                                                          tbase, inside);
                    tmem_fence_before();
                } else if (inside) {
                    phase_b<LAT, MASK>(g, p, mask, f, fout, status, sm, T, pl, t, nullptr);
                }
                mbar_arrive(&sm.empty[pl % 6]);
            }
        }
    }
}

// FP32 populations, warp-specialised; 2 TX TY threads, dynamic shared memory
// of sizeof(SharedWS<LAT>).
template <int LAT, bool MASK>
__global__ void __launch_bounds__(2 * LatF<LAT>::TX * LatF<LAT>::TY, 1)
k_step_f32_ws(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const float *__restrict__ f,
              float *__restrict__ fout, int *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedWS<LAT> &sm = *reinterpret_cast<SharedWS<LAT> *>(smem_raw);
    fused_tile_ws<LAT, MASK>(g, p, mask, f, fout, status, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

// Warp-specialised with Tensor Memory staging: the producer that loads an
// interior node leaves its populations in the Tensor Memory lane of the
// consumer that collides it (warps w and w + 8 share lanes; 32 x 8 tiles
// only); the full/empty barriers also order the Tensor Memory accesses.
template <int LAT, bool MASK>
__global__ void __launch_bounds__(2 * LatF<LAT>::TX * LatF<LAT>::TY, 1)
k_step_f32_wstm(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const float *__restrict__ f,
                float *__restrict__ fout, int *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedWS<LAT> &sm = *reinterpret_cast<SharedWS<LAT> *>(smem_raw);
    constexpr unsigned COLS = TmemF<LAT>::COLS;
    if (threadIdx.x < 32) tmem_alloc(&sm.tmem, COLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned tbase = sm.tmem;
    fused_tile_ws<LAT, MASK, true>(g, p, mask, f, fout, status, blockIdx.x, blockIdx.y, blockIdx.z, sm,
                                   tbase);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tbase, COLS);
}

// ---- TMA staging of the entering planes -------------------------------
// The warp-specialised producers above spend most of a plane waiting for
// their own loads (27 per halo node, issued before any arithmetic, then a
// full memory round trip per plane). Here nine bulk tensor copies per plane
// (BoxS) move the plane's populations on the tile's halo into shared memory,
// the populations viewed as a 4D tensor (x, y, z, i), and one producer warp
// requests each plane's boxes kBoxAhead planes before the producers need
// them, so phase A reads shared memory. Box stage (pl + kBoxAhead) %
// kBoxStages held ring index pl - 1: the requesting warp asks for the boxes
// of pl + kBoxAhead once full[(pl - 1) % 6] shows every producer past
// pl - 1. Issuing nine copies takes that warp over a thousand cycles per
// plane, so it is the last producer warp, whose halo share is empty (its
// threads form only their interior nodes): the wait and the issue fall in
// time it would otherwise spend waiting for the consumers.
constexpr int kBoxWarp = 7;
constexpr int kBoxStages = 3, kBoxAhead = kBoxStages - 1;

// The box shapes as tensor maps of one population buffer: 32 x 8, 32 x 2,
// W x 8, W x 2 and the one-copy WX x 12 (x by y), one plane, all 27
// populations.
struct BoxMaps {
    CUtensorMap mc, tc, ml, tl, wide;   // wide: the one-copy box, WX x 12
};

// Shared memory of the TMA-staged tile: that of the warp-specialised tile
// (BASE: SharedWS, or SharedSWS for shifted storage) and the box stages.
template <int LAT, typename ST, typename BASE> struct SharedWTT : BASE {
    alignas(128) BoxT<ST> box[kBoxStages];
    unsigned long long bfull[kBoxStages];
    // the box holds halo column c / row r (its source coordinate is the
    // node's wrapped one; false only on ragged tiles)
    unsigned char xok[SharedF<LAT>::AX], yok[SharedF<LAT>::AY];
};
template <int LAT> using SharedWT = SharedWTT<LAT, float, SharedWS<LAT>>;
template <int LAT, typename ST> using SharedSWT = SharedWTT<LAT, ST, SharedSWS<LAT>>;

// Arm bar for `bytes` more bytes (one arrival).
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\t"
                 "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Copy the box whose first element is (x, y, z, 0) into dst, completing on
// bar. x must be a multiple of 4 (16-byte aligned rows).
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, unsigned long long *bar, int x,
                                            int y, int z)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];"
                 ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(0), "r"(smem_u32(bar))
                 : "memory");
}

// Shifted storage (ST 16-bit, SM = SharedSWT): the producers also keep the
// source-density ring and wait for one another once per plane (pbar), as
// in fused_tile_ws; the boxes hold the stored 16-bit values, which phase A
// decodes.
template <int LAT, bool MASK, int EOSK, typename ST = float, typename SM = SharedWT<LAT>>
__device__ __forceinline__ void fused_tile_wstma(const GeoF &g, const PhysF &p,
                                                 const uint8_t *__restrict__ mask,
                                                 const ST *__restrict__ f, ST *__restrict__ fout,
                                                 int *__restrict__ status, int bx, int by, int bz,
                                                 SM &sm, unsigned tbase, const BoxMaps *maps,
                                                 const float *__restrict__ rho_src = nullptr,
                                                 float *__restrict__ rho_dst = nullptr)
{
    constexpr bool SHIFT = IsShifted<ST>::value;
    constexpr int TX = LatF<LAT>::TX, NT = TX * LatF<LAT>::TY;
    constexpr int AX = SharedF<LAT>::AX, AY = SharedF<LAT>::AY;
    constexpr int W = BoxT<ST>::W;
    static_assert(LAT == 1 && TX == 32 && LatF<LAT>::TY == 8, "the box layout is that of D3Q27 32 x 8 tiles");
    const int tid = threadIdx.x;
    const TileF T = tile_setup<LAT, ST>(g, bx, by, bz, sm, tid, 2 * NT, rho_src);
    // box origins: columns x0 - W, x0, x0 + 32 and rows y0 - 2, y0, y0 + 8, wrapped
    const int xl = ((T.x0 - W) % g.nx + g.nx) % g.nx, xr = (T.x0 + 32) % g.nx;
    const int yt = ((T.y0 - 2) % g.ny + g.ny) % g.ny, yb = (T.y0 + 8) % g.ny;
    if (tid < AX) {   // (the wrapped coordinates formed here, not read from tile_setup's)
        const int c = tid;
        const int xs = c < 2 ? xl + c + W - 2 : c < 34 ? T.x0 + c - 2 : xr + c - 34;
        sm.xok[c] = xs < g.nx && xs == ((T.x0 - 2 + c) % g.nx + g.nx) % g.nx;
    } else if (tid < AX + AY) {
        const int r = tid - AX;
        const int ys = r < 2 ? yt + r : r < 10 ? T.y0 + r - 2 : yb + r - 10;
        sm.yok[r] = ys < g.ny && ys == ((T.y0 - 2 + r) % g.ny + g.ny) % g.ny;
    }
    if (tid == 0) {
        for (int k = 0; k < 6; ++k) {
            mbar_init(&sm.full[k], NT);
            mbar_init(&sm.empty[k], NT);
        }
        for (int k = 0; k < kBoxStages; ++k) mbar_init(&sm.bfull[k], 1);
        if constexpr (SHIFT)
            for (int k = 0; k < 2; ++k) mbar_init(&sm.pbar[k], NT);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // The boxes' 128-byte alignment rests on that of the dynamic shared
    // memory's base: a block that finds it otherwise sets bit 3 of the
    // status and copies nothing (the same for all its threads).
    if (smem_u32(&sm.box[0]) % 128u) {
        if (tid == 0) atomicOr(status, 8);
        return;
    }
    // the nine boxes of ring index r (plane z0 - 2 + r) into stage r % kBoxStages
    auto request = [&](int r) {
        const int st = r % kBoxStages;
        BoxT<ST> &b = sm.box[st];
        unsigned long long *bar = &sm.bfull[st];
        const int z = wrapf(T.z0 - 2 + r, g.nz);
        mbar_expect_tx(bar, BoxT<ST>::BYTES);
        tma_load_4d(&b.mc[0][0][0], &maps->mc, bar, T.x0, T.y0, z);
        tma_load_4d(&b.tc[0][0][0], &maps->tc, bar, T.x0, yt, z);
        tma_load_4d(&b.bc[0][0][0], &maps->tc, bar, T.x0, yb, z);
        tma_load_4d(&b.ml[0][0][0], &maps->ml, bar, xl, T.y0, z);
        tma_load_4d(&b.mr[0][0][0], &maps->ml, bar, xr, T.y0, z);
        tma_load_4d(&b.tl[0][0][0], &maps->tl, bar, xl, yt, z);
        tma_load_4d(&b.tr[0][0][0], &maps->tl, bar, xr, yt, z);
        tma_load_4d(&b.bl[0][0][0], &maps->tl, bar, xl, yb, z);
        tma_load_4d(&b.br[0][0][0], &maps->tl, bar, xr, yb, z);
    };
    static_assert(kBoxWarp * 32 >= (SharedF<LAT>::AX * SharedF<LAT>::AY - NT) && kBoxWarp * 32 < NT,
                  "the requesting warp has no halo node beyond its interior one");
    const bool boxer = tid >> 5 == kBoxWarp, boxer0 = tid == kBoxWarp * 32;
    if (tid < NT) {
        int issued = 0;   // ring indices whose boxes have been requested (lane 0 of kBoxWarp's count)
        if (boxer0)
            for (; issued < kBoxStages && issued < T.np; ++issued) request(issued);
        int pl = 0;
        for (; pl < T.np; ++pl) {
            if (boxer && pl >= 1 && pl + kBoxAhead < T.np) {
                const int old = pl - 1;
                if (!mbar_wait(&sm.full[old % 6], (old / 6) & 1)) {
                    atomicOr(status, 2);
                    break;
                }
                if (boxer0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    request(pl + kBoxAhead);
                    issued = pl + kBoxAhead + 1;
                }
                __syncwarp();
            }
            if (pl >= 6 && !mbar_wait(&sm.empty[(pl - 2) % 6], ((pl - 6) / 6) & 1)) {
                atomicOr(status, 2);
                break;
            }
            if (!mbar_wait(&sm.bfull[pl % kBoxStages], (pl / kBoxStages) & 1)) {
                atomicOr(status, 2);
                break;
            }
            if constexpr (SHIFT) {   // the source densities loaded in iteration pl - 1 are in place
                if (pl > 0 && !mbar_wait(&sm.pbar[(pl - 1) & 1], ((pl - 1) >> 1) & 1)) {
                    atomicOr(status, 2);
                    break;
                }
            }
            tmem_fence_after();
            phase_a<LAT, MASK, true, false, true, true, EOSK>(g, p, mask, f, sm, T, pl, tid, rho_src, tbase,
                                                              &sm.box[pl % kBoxStages]);
            tmem_fence_before();
            if constexpr (SHIFT) mbar_arrive(&sm.pbar[pl & 1]);
            mbar_arrive(&sm.full[pl % 6]);
        }
        // After a wait ran out, the boxes requested but not yet seen to land
        // (ring indices pl .. issued - 1, distinct stages) land, each wait
        // bounded, before the block exits and its shared memory is reused.
        if (boxer0)
            for (int r = pl; r < issued; ++r)
                if (!mbar_wait(&sm.bfull[r % kBoxStages], (r / kBoxStages) & 1)) break;
    } else {
        const int t = tid - NT;
        const bool inside = T.x0 + t % TX < g.nx && T.y0 + t / TX < g.ny;
        for (int pl = 0; pl < T.np; ++pl) {
            if (!mbar_wait(&sm.full[pl % 6], (pl / 6) & 1)) {
                atomicOr(status, 2);
                break;
            }
            if (pl >= 4) {
                tmem_fence_after();
                // the solid-node code only where a node or one of its
                // neighbours can be solid (planes zc - 1 .. zc + 1)
                if (MASK && planes_solid3(g, T.z0 + pl - 4))
                    phase_b<LAT, true, true, false, true>(g, p, mask, f, fout, status, sm, T, pl, t, rho_dst,
                                                          tbase, inside);
                else
                    phase_b<LAT, false, true, false, true>(g, p, mask, f, fout, status, sm, T, pl, t, rho_dst,
                                                           tbase, inside);
                tmem_fence_before();
                mbar_arrive(&sm.empty[pl % 6]);
            }
        }
    }
}

// Warp-specialised with Tensor Memory staging and TMA staging of each
// entering plane's halo (D3Q27 FP32 32 x 8 tiles; nx a multiple of 4, so
// the tensor's rows are 16-byte aligned); maps are the source population
// buffer f as a 4D tensor (x, y, z, i) with the four box shapes; EOSK the
// equation of state (p.eos) fixed at compile time; dynamic shared memory
// of sizeof(SharedWT<LAT>).
template <int LAT, bool MASK, int EOSK>
__global__ void __launch_bounds__(2 * LatF<LAT>::TX * LatF<LAT>::TY, 1)
k_step_f32_wstma(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const __grid_constant__ BoxMaps maps,
                 const float *__restrict__ f, float *__restrict__ fout, int *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw128[];
    SharedWT<LAT> &sm = *reinterpret_cast<SharedWT<LAT> *>(smem_raw128);
    constexpr unsigned COLS = TmemF<LAT>::COLS;
    if (threadIdx.x < 32) tmem_alloc(&sm.tmem, COLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned tbase = sm.tmem;
    fused_tile_wstma<LAT, MASK, EOSK>(g, p, mask, f, fout, status, blockIdx.x, blockIdx.y, blockIdx.z, sm,
                                      tbase, &maps);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tbase, COLS);
}

// Shifted 16-bit storage, TMA-staged (D3Q27 32 x 8 tiles; nx a multiple of 8,
// so the 16-bit tensor's rows are 16-byte aligned): the boxes carry the
// stored values, the source densities come through the producers' ring;
// dynamic shared memory of sizeof(SharedSWT<LAT, ST>).
template <int LAT, typename ST, bool MASK>
__global__ void __launch_bounds__(2 * LatF<LAT>::TX * LatF<LAT>::TY, 1)
k_step_shifted_wstma(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const __grid_constant__ BoxMaps maps,
                     const ST *__restrict__ f, ST *__restrict__ fout, const float *__restrict__ rho_src,
                     float *__restrict__ rho_dst, int *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw128[];
    SharedSWT<LAT, ST> &sm = *reinterpret_cast<SharedSWT<LAT, ST> *>(smem_raw128);
    constexpr unsigned COLS = TmemF<LAT>::COLS;
    if (threadIdx.x < 32) tmem_alloc(&sm.tmem, COLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned tbase = sm.tmem;
    fused_tile_wstma<LAT, MASK, -1, ST, SharedSWT<LAT, ST>>(g, p, mask, f, fout, status, blockIdx.x, blockIdx.y,
                                                            blockIdx.z, sm, tbase, &maps, rho_src, rho_dst);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tbase, COLS);
}

// FP32 populations; dynamic shared memory of sizeof(SharedF<LAT>).
// E64: the EOS, pseudo-potential and force sums in FP64 (LBM_FLAG_EOS_F64).
template <int LAT, bool MASK, bool E64 = false>
__global__ void __launch_bounds__(LatF<LAT>::TX * LatF<LAT>::TY, 2)
k_step_f32(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const float *__restrict__ f,
           float *__restrict__ fout, int *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedF<LAT> &sm = *reinterpret_cast<SharedF<LAT> *>(smem_raw);
    fused_tile<LAT, MASK, float, SharedF<LAT>, false, E64>(g, p, mask, f, fout, status, blockIdx.x,
                                                           blockIdx.y, blockIdx.z, sm);
}

// FP32 populations with the interior nodes' populations kept in Tensor
// Memory between the phases (TmemF::COLS columns per block, allocated by
// warp 0 and freed before the block exits); dynamic shared memory of
// sizeof(SharedF<LAT>).
template <int LAT, bool MASK>
__global__ void __launch_bounds__(LatF<LAT>::TX * LatF<LAT>::TY, 2)
k_step_f32_tm(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const float *__restrict__ f,
              float *__restrict__ fout, int *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedF<LAT> &sm = *reinterpret_cast<SharedF<LAT> *>(smem_raw);
    constexpr unsigned COLS = TmemF<LAT>::COLS;
    if (threadIdx.x < 32) tmem_alloc(&sm.tmem, COLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned tbase = sm.tmem;
    fused_tile<LAT, MASK, float, SharedF<LAT>, true>(g, p, mask, f, fout, status, blockIdx.x, blockIdx.y,
                                                     blockIdx.z, sm, nullptr, nullptr, tbase);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tbase, COLS);
}

// Shifted 16-bit storage (ST = __half or __nv_bfloat16): populations h_i
// with the source densities rho_src read and rho_dst written; dynamic shared
// memory of sizeof(SharedS<LAT>).
template <int LAT, typename ST, bool E64 = false, bool MASK = false>
__global__ void __launch_bounds__(LatF<LAT>::TX * LatF<LAT>::TY, 2)
k_step_shifted(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const ST *__restrict__ f,
               ST *__restrict__ fout, const float *__restrict__ rho_src, float *__restrict__ rho_dst,
               int *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedS<LAT> &sm = *reinterpret_cast<SharedS<LAT> *>(smem_raw);
    fused_tile<LAT, MASK, ST, SharedS<LAT>, false, E64>(g, p, mask, f, fout, status, blockIdx.x,
                                                        blockIdx.y, blockIdx.z, sm, rho_src, rho_dst);
}

// Shifted 16-bit storage with the interior nodes' decoded populations kept in
// Tensor Memory between the phases (as k_step_f32_tm).
template <int LAT, typename ST, bool MASK = false>
__global__ void __launch_bounds__(LatF<LAT>::TX * LatF<LAT>::TY, 2)
k_step_shifted_tm(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const ST *__restrict__ f,
                  ST *__restrict__ fout, const float *__restrict__ rho_src, float *__restrict__ rho_dst,
                  int *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedS<LAT> &sm = *reinterpret_cast<SharedS<LAT> *>(smem_raw);
    constexpr unsigned COLS = TmemF<LAT>::COLS;
    if (threadIdx.x < 32) tmem_alloc(&sm.tmem, COLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned tbase = sm.tmem;
    fused_tile<LAT, MASK, ST, SharedS<LAT>, true>(g, p, mask, f, fout, status, blockIdx.x,
                                                  blockIdx.y, blockIdx.z, sm, rho_src, rho_dst, tbase);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tbase, COLS);
}

// Shifted 16-bit storage, warp-specialised with the decoded populations
// handed from producer to consumer in Tensor Memory (D3Q27 32 x 8 tiles, as
// k_step_f32_wstm); dynamic shared memory of sizeof(SharedSWS<LAT>).
template <int LAT, typename ST, bool MASK>
__global__ void __launch_bounds__(2 * LatF<LAT>::TX * LatF<LAT>::TY, 1)
k_step_shifted_wstm(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const ST *__restrict__ f,
                    ST *__restrict__ fout, const float *__restrict__ rho_src, float *__restrict__ rho_dst,
                    int *__restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedSWS<LAT> &sm = *reinterpret_cast<SharedSWS<LAT> *>(smem_raw);
    constexpr unsigned COLS = TmemF<LAT>::COLS;
    if (threadIdx.x < 32) tmem_alloc(&sm.tmem, COLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned tbase = sm.tmem;
    fused_tile_ws<LAT, MASK, true, ST, SharedSWS<LAT>>(g, p, mask, f, fout, status, blockIdx.x, blockIdx.y,
                                                       blockIdx.z, sm, tbase, rho_src, rho_dst);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tbase, COLS);
}

// ---- Tensor Memory form with TMA-staged planes, one thread group ---------
// The Tensor Memory form of the shifted step (one group of 256 threads, a
// block barrier per plane, two blocks per SM) with each entering plane's
// 16-bit values copied into shared memory in one stage: the copy of plane
// pl + 1 is requested once the block barrier after phase A of pl shows every
// thread past the stage, and lands during phase B of pl. Tiles whose halo
// stays inside the lattice take one copy per plane (BoxT::wide), the others
// the nine boxes; one thread of warp 7 (whose phase A holds no halo node
// beyond its interior one) issues them. A wait that runs out sets bit 2 of
// the status and the block carries on with what shared memory holds (no
// thread leaves the loop, so no block barrier is left waiting): the step
// then reports LBM_ETIMEOUT.
template <int LAT, typename ST> struct SharedSB : SharedS<LAT> {
    alignas(128) BoxT<ST> box;
    unsigned long long bfull;
    unsigned char xok[SharedF<LAT>::AX], yok[SharedF<LAT>::AY];
};

template <int LAT, bool MASK, typename ST>
__device__ __forceinline__ void fused_tile_tmb(const GeoF &g, const PhysF &p, const uint8_t *__restrict__ mask,
                                               const ST *__restrict__ f, ST *__restrict__ fout,
                                               int *__restrict__ status, int bx, int by, int bz,
                                               SharedSB<LAT, ST> &sm, unsigned tbase, const BoxMaps *maps,
                                               const float *__restrict__ rho_src, float *__restrict__ rho_dst)
{
    constexpr int TX = LatF<LAT>::TX, NT = TX * LatF<LAT>::TY;
    constexpr int AX = SharedF<LAT>::AX, AY = SharedF<LAT>::AY;
    constexpr int W = BoxT<ST>::W;
    static_assert(LAT == 1 && TX == 32 && LatF<LAT>::TY == 8, "the box layout is that of D3Q27 32 x 8 tiles");
    constexpr int kIssuer = 7 * 32;   // lane 0 of warp 7
    const int tid = threadIdx.x;
    const TileF T = tile_setup<LAT, ST>(g, bx, by, bz, sm, tid, NT, rho_src);
    const bool inside = T.x0 + tid % TX < g.nx && T.y0 + tid / TX < g.ny;
    const int xl = ((T.x0 - W) % g.nx + g.nx) % g.nx, xr = (T.x0 + 32) % g.nx;
    const int yt = ((T.y0 - 2) % g.ny + g.ny) % g.ny, yb = (T.y0 + 8) % g.ny;
    const bool wide = T.x0 - W >= 0 && T.x0 + 32 + W <= g.nx && T.y0 - 2 >= 0 && T.y0 + 10 <= g.ny;
    if (tid < AX) {
        const int c = tid;
        const int xs = c < 2 ? xl + c + W - 2 : c < 34 ? T.x0 + c - 2 : xr + c - 34;
        sm.xok[c] = xs < g.nx && xs == ((T.x0 - 2 + c) % g.nx + g.nx) % g.nx;
    } else if (tid < AX + AY) {
        const int r = tid - AX;
        const int ys = r < 2 ? yt + r : r < 10 ? T.y0 + r - 2 : yb + r - 10;
        sm.yok[r] = ys < g.ny && ys == ((T.y0 - 2 + r) % g.ny + g.ny) % g.ny;
    }
    if (tid == kIssuer) {
        mbar_init(&sm.bfull, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (smem_u32(&sm.box) % 128u) {   // the boxes' 128-byte alignment rests on the base's
        if (tid == 0) atomicOr(status, 8);
        return;
    }
    // the copies of ring index r (plane z0 - 2 + r) into the stage
    auto request = [&](int r) {
        BoxT<ST> &b = sm.box;
        unsigned long long *bar = &sm.bfull;
        const int z = wrapf(T.z0 - 2 + r, g.nz);
        if (wide) {
            mbar_expect_tx(bar, BoxT<ST>::WIDE_BYTES);
            tma_load_4d(&b.mc[0][0][0], &maps->wide, bar, T.x0 - W, T.y0 - 2, z);
            return;
        }
        mbar_expect_tx(bar, BoxT<ST>::BYTES);
        tma_load_4d(&b.mc[0][0][0], &maps->mc, bar, T.x0, T.y0, z);
        tma_load_4d(&b.tc[0][0][0], &maps->tc, bar, T.x0, yt, z);
        tma_load_4d(&b.bc[0][0][0], &maps->tc, bar, T.x0, yb, z);
        tma_load_4d(&b.ml[0][0][0], &maps->ml, bar, xl, T.y0, z);
        tma_load_4d(&b.mr[0][0][0], &maps->ml, bar, xr, T.y0, z);
        tma_load_4d(&b.tl[0][0][0], &maps->tl, bar, xl, yt, z);
        tma_load_4d(&b.tr[0][0][0], &maps->tl, bar, xr, yt, z);
        tma_load_4d(&b.bl[0][0][0], &maps->tl, bar, xl, yb, z);
        tma_load_4d(&b.br[0][0][0], &maps->tl, bar, xr, yb, z);
    };
    if (tid == kIssuer) request(0);
    bool copies = true;   // no wait has run out (after one has, the copies stop)
    for (int pl = 0; pl < T.np; ++pl) {
        if (copies && !mbar_wait(&sm.bfull, pl & 1)) {
            atomicOr(status, 2);
            copies = false;
        }
        phase_a<LAT, MASK, true, false, false, true>(g, p, mask, f, sm, T, pl, tid, rho_src, tbase, &sm.box,
                                                     wide);
        __syncthreads();
        if (tid == kIssuer && copies && pl + 1 < T.np) {   // every thread is past the stage
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            request(pl + 1);
        }
        if (pl >= 4) phase_b<LAT, MASK, true>(g, p, mask, f, fout, status, sm, T, pl, tid, rho_dst, tbase, inside);
    }
}

// Shifted 16-bit storage: Tensor Memory form with TMA-staged planes (D3Q27
// 32 x 8 tiles, nx a multiple of 8), TmemF::COLS columns of Tensor Memory and
// sizeof(SharedSB<LAT, ST>) bytes of dynamic shared memory per block.
template <int LAT, typename ST, bool MASK>
__global__ void __launch_bounds__(LatF<LAT>::TX * LatF<LAT>::TY, 2)
k_step_shifted_tmtma(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const __grid_constant__ BoxMaps maps,
                     const ST *__restrict__ f, ST *__restrict__ fout, const float *__restrict__ rho_src,
                     float *__restrict__ rho_dst, int *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw128[];
    SharedSB<LAT, ST> &sm = *reinterpret_cast<SharedSB<LAT, ST> *>(smem_raw128);
    constexpr unsigned COLS = TmemF<LAT>::COLS;
    if (threadIdx.x < 32) tmem_alloc(&sm.tmem, COLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned tbase = sm.tmem;
    fused_tile_tmb<LAT, MASK, ST>(g, p, mask, f, fout, status, blockIdx.x, blockIdx.y, blockIdx.z, sm, tbase,
                                  &maps, rho_src, rho_dst);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tbase, COLS);
}

// Many lattices of one type and one storage in one launch: descriptor of one
// member for the current step parity, and the (member, tile) work items.
struct MemberF {
    GeoF g;
    PhysF p;
    const uint8_t *mask;   // nullptr when the member has no solid node
    const void *src;       // float, or 16-bit shifted populations
    void *dst;
    const float *rho_src;  // shifted storage: densities of src and dst
    float *rho_dst;
    int *status;
    int tiles_x, tiles_y;
};

struct WorkItem {
    int member, bx, by, bz;
};

// Persistent: CTA b takes items b, b + gridDim.x, ... (a fixed assignment,
// so each member's result does not depend on what else is in the batch);
// dynamic shared memory of sizeof(SharedF<LAT>).
template <int LAT>
__global__ void __launch_bounds__(LatF<LAT>::TX * LatF<LAT>::TY, 2)
k_step_f32_batch(const MemberF *__restrict__ members, const WorkItem *__restrict__ items,
                 int n_items)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedF<LAT> &sm = *reinterpret_cast<SharedF<LAT> *>(smem_raw);
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const MemberF &m = members[w.member];
        const float *src = static_cast<const float *>(m.src);
        float *dst = static_cast<float *>(m.dst);
        if (m.mask)
            fused_tile<LAT, true>(m.g, m.p, m.mask, src, dst, m.status, w.bx, w.by, w.bz, sm);
        else
            fused_tile<LAT, false>(m.g, m.p, m.mask, src, dst, m.status, w.bx, w.by, w.bz, sm);
        __syncthreads();   // the rings are reused by the next item
    }
}

// The same over members with 16-bit shifted storage;
// dynamic shared memory of sizeof(SharedS<LAT>).
template <int LAT, typename ST>
__global__ void __launch_bounds__(LatF<LAT>::TX * LatF<LAT>::TY, 2)
k_step_shifted_batch(const MemberF *__restrict__ members, const WorkItem *__restrict__ items,
                     int n_items)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedS<LAT> &sm = *reinterpret_cast<SharedS<LAT> *>(smem_raw);
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const MemberF &m = members[w.member];
        if (m.mask)
            fused_tile<LAT, true, ST, SharedS<LAT>>(m.g, m.p, m.mask, static_cast<const ST *>(m.src),
                                                   static_cast<ST *>(m.dst), m.status, w.bx, w.by,
                                                   w.bz, sm, m.rho_src, m.rho_dst);
        else
            fused_tile<LAT, false, ST, SharedS<LAT>>(m.g, m.p, nullptr, static_cast<const ST *>(m.src),
                                                    static_cast<ST *>(m.dst), m.status, w.bx, w.by,
                                                    w.bz, sm, m.rho_src, m.rho_dst);
        __syncthreads();
    }
}

}  // namespace LBMF_NS
