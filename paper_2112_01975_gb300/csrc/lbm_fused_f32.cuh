// Fused single-pass step for FP32 populations with FP32 arithmetic.
//
// One CTA owns a TX x TY column tile of the x-y plane and marches along z
// through a chunk of planes (D2Q9 runs as a 3D lattice with one y row and
// the 2D y axis as the march axis). For each plane that enters, it reads the
// 27 populations of every node of the tile plus a 2-node halo, forms
// (rho, s psi) there and rho u_a^3 on the 1-node halo, and keeps them in
// shared-memory rings. Two planes behind, it collides the tile: the 2-ring
// force stencils and the Phi differences read only shared memory, the
// node's own populations are read again (an L2 hit), and the post-collision
// populations are pushed to the neighbours with halfway bounce-back. HBM
// sees each population read about once and written once; the halo and the
// second read of a node are served from L2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmf {

struct GeoF {
    int nx, ny, nz;   // as stored; D2Q9: ny = 1 and nz = the 2D y extent
    unsigned N;
    int chunk;        // planes per CTA along z
};

struct PhysF {
    int eos;
    float a, b, RT, aalpha;
    float kappa, omega, omw, phi_pref;  // omw = 1 - omega
    float rho_w, spsi_w;                // virtual solid density and its s psi
};

// Lattice description in the 3D frame: D2Q9 uses (cx, 0, cy).
template <int LAT> struct LatF;
template <> struct LatF<0> {
    static constexpr int Q = 9, TX = 128, TY = 1, HY = 0;
    __device__ static constexpr int cx(int i) { return i % 3 - 1; }
    __device__ static constexpr int cy(int) { return 0; }
    __device__ static constexpr int cz(int i) { return i / 3 - 1; }
};
template <> struct LatF<1> {
    static constexpr int Q = 27, TX = 32, TY = 8, HY = 2;
    __device__ static constexpr int cx(int i) { return i % 3 - 1; }
    __device__ static constexpr int cy(int i) { return (i / 3) % 3 - 1; }
    __device__ static constexpr int cz(int i) { return i / 9 - 1; }
};

__device__ __forceinline__ float eos_pressure_f(const PhysF &p, float rho)
{
    const float rep = rho * p.RT / (1.0f - p.b * rho);
    switch (p.eos) {
    case 0: return rep - p.a * rho * rho;
    case 1: return rep - p.aalpha * rho * rho / (1.0f + 2.0f * p.b * rho - p.b * p.b * rho * rho);
    case 2: return rep - p.aalpha * rho * rho / (1.0f + p.b * rho);
    default: {
        const float e = 0.25f * p.b * rho, om = 1.0f - e;
        return rho * p.RT * (1.0f + e + e * e - e * e * e) / (om * om * om) - p.a * rho * rho;
    }
    }
}

__device__ __forceinline__ float signed_psi_f(const PhysF &p, float rho)
{
    const float d = eos_pressure_f(p, rho) - rho * (1.0f / 3.0f);
    return d > 0.0f ? sqrtf(d) : -sqrtf(-d);
}

__device__ __forceinline__ int wrapf(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <int LAT, bool MASK>
__global__ void __launch_bounds__(LatF<LAT>::TX * LatF<LAT>::TY, 2)
k_step_f32(GeoF g, PhysF p, const uint8_t *__restrict__ mask, const float *__restrict__ f,
           float *__restrict__ fout, int *__restrict__ status)
{
    using L = LatF<LAT>;
    constexpr int Q = L::Q, TX = L::TX, TY = L::TY, HY = L::HY;
    constexpr bool THREE = LAT == 1;
    constexpr int NT = TX * TY;
    constexpr int AX = TX + 4, AY = TY + 2 * HY;          // (rho, s psi) halo tile
    constexpr int GX = TX + 2, GY = THREE ? TY + 2 : 1;   // rho u^3 halo tile
    constexpr int RS = 6, GS = 5;                          // ring slots
    __shared__ float2 s_rp[RS][AY][AX];
    __shared__ float s_g[GS][3][GY][GX];
    __shared__ int s_xw[AX], s_yw[AY];   // wrapped halo coordinates (any size >= 5)

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * g.chunk;
    const int z1 = min(z0 + g.chunk, g.nz);
    const int tx = tid % TX, ty = tid / TX;
    const int xi = x0 + tx, yi = y0 + ty;
    const bool inside = xi < g.nx && yi < g.ny;
    const size_t N = g.N;
    for (int c = tid; c < AX; c += NT) s_xw[c] = ((x0 - 2 + c) % g.nx + g.nx) % g.nx;
    for (int r = tid; r < AY; r += NT) s_yw[r] = THREE ? ((y0 - HY + r) % g.ny + g.ny) % g.ny : 0;
    __syncthreads();

    // Planes z0-2 .. z1+1 enter the rings one per iteration; plane z0-2+pl
    // has ring index pl. Six (rho, s psi) slots and five rho u^3 slots let
    // the next plane enter while slower warps still collide: one barrier
    // per plane.
    const int np = (z1 - z0) + 4;
    for (int pl = 0; pl < np; ++pl) {
        // ---- phase A: plane z0 - 2 + pl enters the rings -------------------
        {
            const int zl = wrapf(z0 - 2 + pl, g.nz);
            const int rs = pl % RS, gs = pl % GS;
            for (int k = tid; k < AX * AY; k += NT) {
                const int r = k / AX, c = k - r * AX;
                const int x = s_xw[c];
                const int y = s_yw[r];
                const unsigned n = x + g.nx * (y + g.ny * zl);
                const bool ring1 = c >= 1 && c < AX - 1 && (!THREE || (r >= 1 && r < AY - 1));
                float rho, sp, gx = 0.0f, gy = 0.0f, gz = 0.0f;
                if (MASK && mask[n]) {
                    rho = p.rho_w;
                    sp = p.spsi_w;
                } else {
                    float fi[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) fi[i] = __ldg(f + i * N + n);
                    float sx[3] = {0.0f, 0.0f, 0.0f};   // sums over cx = -1, 0, +1
                    float jy = 0.0f, jz = 0.0f;
#pragma unroll
                    for (int i = 0; i < Q; ++i) sx[L::cx(i) + 1] += fi[i];
                    rho = sx[0] + sx[1] + sx[2];
                    if (ring1) {
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            if (L::cy(i) > 0) jy += fi[i];
                            if (L::cy(i) < 0) jy -= fi[i];
                            if (L::cz(i) > 0) jz += fi[i];
                            if (L::cz(i) < 0) jz -= fi[i];
                        }
                        const float inv = 1.0f / rho;
                        const float ux = (sx[2] - sx[0]) * inv, uy = jy * inv, uz = jz * inv;
                        gx = rho * ux * ux * ux;
                        gy = rho * uy * uy * uy;
                        gz = rho * uz * uz * uz;
                    }
                    sp = signed_psi_f(p, rho);
                }
                s_rp[rs][r][c] = make_float2(rho, sp);
                if (ring1) {
                    const int gr = THREE ? r - 1 : 0;
                    s_g[gs][0][gr][c - 1] = gx;
                    s_g[gs][1][gr][c - 1] = gy;
                    s_g[gs][2][gr][c - 1] = gz;
                }
            }
        }
        __syncthreads();
        // ---- phase B: collide plane zc = z0 + pl - 4 --------------------------
        if (pl >= 4 && inside) {
            const int pc = pl - 2;             // ring index of the collided plane
            const int zc = z0 + pl - 4;
            const unsigned n = xi + g.nx * (yi + g.ny * zc);
            if (!(MASK && mask[n])) {
                const int cr = ty + HY, cc = tx + 2;
                const float2 c0 = s_rp[pc % RS][cr][cc];
                const float rho = c0.x;
                if (!(rho > 0.0f) || !isfinite(rho)) atomicOr(status, 1);
                // Korteweg force (Eq. Kforce_final, sign as the force on the fluid)
                float Sp[3] = {0.0f, 0.0f, 0.0f}, Sr[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int s = 1; s <= 2; ++s) {
                    float ap[3][3], ar[3][3];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int k = 0; k < 3; ++k) { ap[a][k] = 0.0f; ar[a][k] = 0.0f; }
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
                        if (c[0] == 0 && c[1] == 0 && c[2] == 0) continue;
                        const float2 v = s_rp[(pc + s * c[2] + RS) % RS][cr + s * c[1]][cc + s * c[0]];
                        const float ps = fabsf(v.y);
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            if (c[a] == 0) continue;
                            const int k = (a != 0 && c[0] != 0) + (a != 1 && c[1] != 0) +
                                          (a != 2 && c[2] != 0);
                            if (c[a] > 0) { ap[a][k] += ps; ar[a][k] += v.x; }
                            else          { ap[a][k] -= ps; ar[a][k] -= v.x; }
                        }
                    }
                    const float gp = s == 1 ? 4.0f / 3.0f : -1.0f / 6.0f;
                    const float gr = s == 1 ? 2.0f : -1.0f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (!THREE && a == 1) continue;
                        float dp, dr;
                        if (THREE) {
                            dp = (2.0f / 9.0f) * ap[a][0] + (1.0f / 18.0f) * ap[a][1] + (1.0f / 72.0f) * ap[a][2];
                            dr = (2.0f / 9.0f) * ar[a][0] + (1.0f / 18.0f) * ar[a][1] + (1.0f / 72.0f) * ar[a][2];
                        } else {
                            dp = (1.0f / 3.0f) * ap[a][0] + (1.0f / 12.0f) * ap[a][1];
                            dr = (1.0f / 3.0f) * ar[a][0] + (1.0f / 12.0f) * ar[a][1];
                        }
                        Sp[a] += gp * dp;
                        Sr[a] += gr * dr;
                    }
                }
                float F[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) F[a] = -2.0f * c0.y * Sp[a] - p.kappa * rho * Sr[a];
                // Phi_aa = -(1 - omega/2) (g_a(r + e_a) - g_a(r - e_a)) / 2
                const int gr0 = THREE ? ty + 1 : 0, gc0 = tx + 1;
                float Phi[3];
                Phi[0] = p.phi_pref * 0.5f * (s_g[pc % GS][0][gr0][gc0 + 1] - s_g[pc % GS][0][gr0][gc0 - 1]);
                Phi[1] = THREE ? p.phi_pref * 0.5f *
                                     (s_g[pc % GS][1][gr0 + 1][gc0] - s_g[pc % GS][1][gr0 - 1][gc0])
                               : 0.0f;
                Phi[2] = p.phi_pref * 0.5f *
                         (s_g[(pc + 1) % GS][2][gr0][gc0] - s_g[(pc - 1) % GS][2][gr0][gc0]);
                // the node's populations (second read, from L2) and its velocity
                float fi[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) fi[i] = __ldg(f + i * N + n);
                float j[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if (L::cx(i) > 0) j[0] += fi[i];
                    if (L::cx(i) < 0) j[0] -= fi[i];
                    if (L::cy(i) > 0) j[1] += fi[i];
                    if (L::cy(i) < 0) j[1] -= fi[i];
                    if (L::cz(i) > 0) j[2] += fi[i];
                    if (L::cz(i) < 0) j[2] -= fi[i];
                }
                const float inv = 1.0f / rho;
                float E[3][3], S[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (!THREE && a == 1) {   // no y factor on D2Q9
                        E[1][0] = E[1][1] = E[1][2] = 1.0f;
                        S[1][0] = S[1][1] = S[1][2] = 1.0f;
                        continue;
                    }
                    const float ua = j[a] * inv;
                    const float ze = 1.0f / 3.0f + ua * ua;
                    E[a][0] = 0.5f * (ze - ua);
                    E[a][1] = 1.0f - ze;
                    E[a][2] = 0.5f * (ze + ua);
                    const float xs = ua + F[a] * inv;
                    const float zs = 1.0f / 3.0f + xs * xs + Phi[a] * inv;
                    S[a][0] = 0.5f * (zs - xs);
                    S[a][1] = 1.0f - zs;
                    S[a][2] = 0.5f * (zs + xs);
                }
                // post = f* + (1 - omega)(f - feq), pushed to r + c_i
                const int X[3] = {wrapf(xi - 1, g.nx), xi, wrapf(xi + 1, g.nx)};
                const int Y[3] = {THREE ? wrapf(yi - 1, g.ny) : 0, yi, THREE ? wrapf(yi + 1, g.ny) : 0};
                const int Z[3] = {wrapf(zc - 1, g.nz), zc, wrapf(zc + 1, g.nz)};
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
                    const float eq = rho * E[0][cx + 1] * E[1][cy + 1] * E[2][cz + 1];
                    const float st = rho * S[0][cx + 1] * S[1][cy + 1] * S[2][cz + 1];
                    const float post = fmaf(p.omw, fi[i] - eq, st);
                    const unsigned dst = X[cx + 1] + g.nx * (Y[cy + 1] + g.ny * Z[cz + 1]);
                    if (MASK && mask[dst]) fout[(Q - 1 - i) * N + n] = post;
                    else                   fout[i * N + dst] = post;
                }
            }
        }
    }
}

}  // namespace lbmf
