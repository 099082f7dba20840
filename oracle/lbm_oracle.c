/*
 * Plain single-threaded FP64 CPU oracle of the two-phase lattice Boltzmann
 * update of Hosseini, Dorschner & Karlin (arXiv 2112.01975).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU baseline leg of
 * the benchmark use it. It shares no code with the CUDA library.
 *
 * It follows the paper's steps in the paper's order, with naive loops over
 * all Q directions and no blocking, fusion or reordering:
 *   moments            Sec. 2.3.3, rho = sum f_i, rho u = sum c_i f_i
 *   equation of state  Sec. 3.1, Eqs. vdWEoS, PREoS, RKSEoS, CSEos; Appendix G,
 *                      Eqs. SCeos, SC1, SC2 (Shan-Chen)
 *   pseudo-potential   Sec. 2.3.4, psi = sqrt|P - P0|, P0 = rho/3 (end of Sec. 2.3.5)
 *   Korteweg force     Eq. Kforce_final with w_i of Eq. wi, plus an optional
 *                      body force rho g (the generic F of Eq. LBGK; Sec. 4.1)
 *   correction Phi     Eq. correction, central difference along alpha
 *   collision          Eqs. LBMeq, LBGK, xistar, zetastar, LBMstar
 *   streaming          left side of Eq. LBGK, halfway bounce-back at solids
 *
 * Readings of the paper taken here (each switchable where noted):
 *  - Force sign. The printed Kforce_final is Korteweg's force in the form it
 *    takes on the left-hand side of the momentum balance (Eq. Kforce minus
 *    grad P0). The velocity shift xi* = u + F/rho needs the force acting on
 *    the fluid, which is its negative:
 *      F = -s 2 psi S_psi - kappa rho S_rho,
 *    S_psi = sum_i (w_i/cs2) c_i [4/3 psi(r+c_i) - 1/6 psi(r+2c_i)],
 *    S_rho = sum_i (w_i/cs2) c_i [2 rho(r+c_i) - rho(r+2c_i)],
 *    s = +1 where P > P0, else -1. With it, F -> -grad(P - P0) + kappa rho
 *    grad lap rho, which gives the Maxwell coexistence densities; the printed
 *    sign gives none (tested).
 *  - zeta*. Printed with u_alpha^2; the remark after Eq. LBMstar and the
 *    moments of f* in Appendix D (sum c c f*(2) = F F / rho, diagonal
 *    included) need (u_alpha + F_alpha/rho)^2. Default: the shifted form;
 *    flag ORACLE_ZETA_LITERAL selects the printed one.
 *  - Phi. With P0 = rho/3 the last two terms of Eq. correction cancel and
 *    Phi_aa = -(1 - omega/2) d_a(rho u_a^3), by the 2nd-order central
 *    difference on bare u. The sign is opposite to the printed one: the
 *    third moment of the D3Q27 equilibrium falls short of the Maxwellian by
 *    rho u_a^3, and cancelling that deficit in the Chapman-Enskog expansion
 *    needs the minus sign. The paper's own criterion decides it (Sec. 4.2):
 *    with this sign the normal-mode decay rate is independent of the frame
 *    velocity, with the printed sign the dependence doubles (tested).
 *    Flags: ORACLE_PHI_PRINTED_SIGN, ORACLE_PHI_OFF.
 *  - psi sign at P == P0 is -1 (the P <= P0 branch); neighbours enter by
 *    magnitude, the sign comes from the centre node.
 *  - Solid nodes carry the virtual density rho_w (Sec. 4.5) in both
 *    stencils, u = 0, and are never collided or streamed.
 *  - Initial populations (the paper gives none): the equilibrium at the bare
 *    velocity u = U0 - F(rho0)/(2 rho0), so that the flow starts with the
 *    requested physical velocity U0 (oracle_init).
 *
 * The node loops carry OpenMP pragmas: every iteration writes its own
 * entries, so a build with -fopenmp (the all-cores CPU baseline) gives the
 * same results bit for bit; the plain build ignores them. Reductions stay
 * serial.
 *
 * Lattice units: dr = dt = 1, cs2 = 1/3, R = 1.
 * Direction index i = (cx+1) + 3(cy+1) [+ 9(cz+1)], opposite = Q-1-i.
 * Populations f[i*N + n], node n = x + nx*(y + ny*z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_ZETA_LITERAL 1
#define ORACLE_PHI_OFF 2
#define ORACLE_FORCE_PRINTED_SIGN 4
#define ORACLE_PHI_PRINTED_SIGN 8

typedef struct {
    int lattice, D, Q;
    int nx, ny, nz;
    long N;
    int c[27][3];
    double w[27];
    int eos;
    double a, b, acentric, RTc, RT, alpha;
    double kappa, omega, rho_w;
    double g[3];      /* body acceleration: force rho g added to F (Sec. 4.1) */
    double tau_v, visc_rv, visc_rl;   /* density-dependent relaxation (tau_v > 0) */
    int flags;
    unsigned char *mask;
    double *qw;       /* wall distance of each link into a solid, [i][n]; NULL: halfway */
    double *f, *fnew;
    double *rho, *u, *psi, *F, *Phi;
    int *sgn;
} oracle_ctx;

/* ---- Product form, Eqs. phi0, phiPlus, phis and prod -------------------- */
static double Psi(int c, double xi, double zeta)
{
    if (c == 0) return 1.0 - zeta;
    if (c == 1) return 0.5 * (xi + zeta);
    return 0.5 * (-xi + zeta);
}

/* ---- Equations of state, Sec. 3.1 (R = 1) ------------------------------- */
double oracle_eos_pressure(int eos, double a, double b, double RT, double alpha, double rho)
{
    switch (eos) {
    case 0: /* van der Waals, Eq. vdWEoS */
        return rho * RT / (1.0 - b * rho) - a * rho * rho;
    case 1: /* Peng-Robinson, Eq. PREoS */
        return rho * RT / (1.0 - b * rho)
               - a * alpha * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
    case 2: /* Redlich-Kwong-Soave, Eq. RKSEoS */
        return rho * RT / (1.0 - b * rho) - a * alpha * rho * rho / (1.0 + b * rho);
    case 3: { /* Carnahan-Starling, Eq. CSEos */
        double e = b * rho / 4.0;
        return rho * RT * (1.0 + e + e * e - e * e * e) / ((1.0 - e) * (1.0 - e) * (1.0 - e))
               - a * rho * rho;
    }
    case 4: { /* Shan-Chen, Eqs. SCeos and SC1; RT holds the coupling G */
        double psi = 1.0 - exp(-rho);
        return rho / 3.0 + RT / 6.0 * psi * psi;
    }
    case 5: { /* Shan-Chen, Eqs. SCeos and SC2; RT holds the coupling G */
        double psi = exp(-1.0 / rho);
        return rho / 3.0 + RT / 6.0 * psi * psi;
    }
    }
    return NAN;
}

/* R Tc from (a, b): the relations printed under each EOS in Sec. 3.1. */
double oracle_eos_RTc(int eos, double a, double b)
{
    switch (eos) {
    case 0: return 8.0 * a / (27.0 * b);            /* a = 27/64 R2Tc2/Pc, b = 1/8 RTc/Pc */
    case 1: return (0.0778 / 0.45724) * a / b;
    case 2: return (0.08664 / 0.42748) * a / b;
    case 3: return (0.18727 / 0.4963) * a / b;
    case 4: return -4.0;              /* critical coupling G_c of Eq. SC1 (Appendix G) */
    case 5: return -exp(2.0);         /* critical coupling G_c of Eq. SC2 */
    }
    return NAN;
}

/* The temperature parameter of each EOS at T/Tc: R T = (T/Tc) R Tc for the
 * cubic equations; for Shan-Chen the coupling G = G_c / (T/Tc) (G plays the
 * role of an inverse temperature: |G| > |G_c| separates phases). */
double oracle_eos_temperature(int eos, double a, double b, double t_over_tc)
{
    double c = oracle_eos_RTc(eos, a, b);
    return eos >= 4 ? c / t_over_tc : t_over_tc * c;
}

/* alpha(T) of PR and RKS, Sec. 3.1; 1 for vdW and CS. */
double oracle_eos_alpha(int eos, double acentric, double t_over_tc)
{
    double m;
    if (eos == 1) m = 0.37464 + 1.54226 * acentric - 0.26992 * acentric * acentric;
    else if (eos == 2) m = 0.480 + 1.574 * acentric - 0.176 * acentric * acentric;
    else return 1.0;
    double s = 1.0 + m * (1.0 - sqrt(t_over_tc));
    return s * s;
}

static long wrap(long v, long n) { return ((v % n) + n) % n; }

static long node_at(const oracle_ctx *o, long x, long y, long z)
{
    return wrap(x, o->nx) + o->nx * (wrap(y, o->ny) + o->ny * wrap(z, o->nz));
}

/* Relaxation rate at density rho. One tau for all nodes unless tau_v > 0:
 * then the kinematic viscosity nu = (tau - 1/2)/3 goes linearly in rho from
 * its liquid value at rho_l (the tau of oracle_create) to its vapour value
 * at rho_v (tau_v), held constant beyond them (the paper sets a vapour to
 * liquid viscosity ratio, Sec. 5.2, without stating the interpolation). */
static double omega_at(const oracle_ctx *o, double rho)
{
    if (!(o->tau_v > 0.0)) return o->omega;
    double nl = (1.0 / o->omega - 0.5) / 3.0, nv = (o->tau_v - 0.5) / 3.0;
    double t = (o->visc_rl - rho) / (o->visc_rl - o->visc_rv);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    return 1.0 / (3.0 * (nl + (nv - nl) * t) + 0.5);
}

oracle_ctx *oracle_create(int lattice, int nx, int ny, int nz, int eos, double t_over_tc,
                          double kappa, double tau, const unsigned char *mask,
                          double a, double b, double acentric, double rho_w, int flags,
                          double gx, double gy, double gz)
{
    if (lattice != 0 && lattice != 1) return NULL;
    if (lattice == 0 && nz != 1) return NULL;
    if (nx < 5 || ny < 5 || (lattice == 1 && nz < 5)) return NULL;
    oracle_ctx *o = (oracle_ctx *)calloc(1, sizeof(oracle_ctx));
    o->lattice = lattice;
    o->D = lattice == 0 ? 2 : 3;
    o->Q = lattice == 0 ? 9 : 27;
    o->nx = nx; o->ny = ny; o->nz = nz;
    o->N = (long)nx * ny * nz;
    for (int i = 0; i < o->Q; ++i) {
        o->c[i][0] = i % 3 - 1;
        o->c[i][1] = (i / 3) % 3 - 1;
        o->c[i][2] = o->D == 3 ? i / 9 - 1 : 0;
        /* Eq. wi: product form at xi = 0, zeta = cs2 = 1/3 */
        double wi = 1.0;
        for (int al = 0; al < o->D; ++al) wi *= Psi(o->c[i][al], 0.0, 1.0 / 3.0);
        o->w[i] = wi;
    }
    o->eos = eos;
    o->a = a; o->b = b; o->acentric = acentric;
    o->RTc = oracle_eos_RTc(eos, a, b);
    o->RT = oracle_eos_temperature(eos, a, b, t_over_tc);
    o->alpha = oracle_eos_alpha(eos, acentric, t_over_tc);
    o->kappa = kappa;
    o->omega = 1.0 / tau;
    o->rho_w = rho_w;
    o->flags = flags;
    o->g[0] = gx;
    o->g[1] = gy;
    o->g[2] = lattice == 1 ? gz : 0.0;
    long N = o->N;
    o->mask = (unsigned char *)calloc(N, 1);
    if (mask) memcpy(o->mask, mask, N);
    o->f = (double *)calloc((size_t)o->Q * N, sizeof(double));
    o->fnew = (double *)calloc((size_t)o->Q * N, sizeof(double));
    o->rho = (double *)calloc(N, sizeof(double));
    o->u = (double *)calloc((size_t)3 * N, sizeof(double));
    o->psi = (double *)calloc(N, sizeof(double));
    o->F = (double *)calloc((size_t)3 * N, sizeof(double));
    o->Phi = (double *)calloc((size_t)3 * N, sizeof(double));
    o->sgn = (int *)calloc(N, sizeof(int));
    return o;
}

void oracle_destroy(oracle_ctx *o)
{
    if (!o) return;
    free(o->mask); free(o->f); free(o->fnew); free(o->rho); free(o->u);
    free(o->psi); free(o->F); free(o->Phi); free(o->sgn); free(o->qw); free(o);
}

double oracle_rt(const oracle_ctx *o) { return o->RT; }
double oracle_alpha(const oracle_ctx *o) { return o->alpha; }

/* Product-form population: rho * prod_alpha Psi_{c_i alpha}(xi_alpha, zeta_alpha). */
static double product_form(const oracle_ctx *o, int i, double rho, const double *xi, const double *zeta)
{
    double p = rho;
    for (int al = 0; al < o->D; ++al) p *= Psi(o->c[i][al], xi[al], zeta[al]);
    return p;
}

/* Equilibrium of Eq. LBMeq with P0 = rho/3: xi = u, zeta = 1/3 + u^2. */
void oracle_feq(const oracle_ctx *o, double rho, const double *u, double *out)
{
    double zeta[3];
    for (int al = 0; al < o->D; ++al) zeta[al] = 1.0 / 3.0 + u[al] * u[al];
    for (int i = 0; i < o->Q; ++i) out[i] = product_form(o, i, rho, u, zeta);
}

/* Extended equilibrium of Eq. LBMstar (zeta* reading in the header). */
void oracle_fstar(const oracle_ctx *o, double rho, const double *u, const double *F,
                  const double *Phi, double *out)
{
    double xi[3], zeta[3];
    for (int al = 0; al < o->D; ++al) {
        xi[al] = u[al] + F[al] / rho;                         /* Eq. xistar */
        double v = (o->flags & ORACLE_ZETA_LITERAL) ? u[al] : xi[al];
        zeta[al] = 1.0 / 3.0 + v * v + Phi[al] / rho;         /* Eq. zetastar */
    }
    for (int i = 0; i < o->Q; ++i) out[i] = product_form(o, i, rho, xi, zeta);
}

/* Lattice stencil of Eqs. PP_discrete and capillary_discrete:
 * out_alpha(r) = sum_i (w_i / cs2) c_i alpha [g1 g(r + c_i) + g2 g(r + 2 c_i)],
 * periodic wrap. out holds D planes of N. */
void oracle_stencil(const oracle_ctx *o, const double *g, double g1, double g2, double *out)
{
    #pragma omp parallel for collapse(2)
    for (long z = 0; z < o->nz; ++z)
        for (long y = 0; y < o->ny; ++y)
            for (long x = 0; x < o->nx; ++x) {
                long n = node_at(o, x, y, z);
                double acc[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < o->Q; ++i) {
                    const int *c = o->c[i];
                    double v = g1 * g[node_at(o, x + c[0], y + c[1], z + c[2])]
                             + g2 * g[node_at(o, x + 2 * c[0], y + 2 * c[1], z + 2 * c[2])];
                    for (int al = 0; al < o->D; ++al)
                        acc[al] += (o->w[i] * 3.0) * c[al] * v;
                }
                for (int al = 0; al < o->D; ++al) out[al * o->N + n] = acc[al];
            }
}

/* Steps 2-3 on the density field o->rho (rho_w at solid nodes): P, psi, s, F. */
static void force_from_density(oracle_ctx *o)
{
    long N = o->N;
    int D = o->D;
    /* equation of state and pseudo-potential, Sec. 2.3.4 with P0 = rho/3 */
    #pragma omp parallel for
    for (long n = 0; n < N; ++n) {
        double rho = o->rho[n];
        double P = oracle_eos_pressure(o->eos, o->a, o->b, o->RT, o->alpha, rho);
        double P0 = rho / 3.0;
        o->psi[n] = P > P0 ? sqrt(P - P0) : sqrt(P0 - P);
        o->sgn[n] = P > P0 ? 1 : -1;
    }
    /* Korteweg force, Eq. Kforce_final (sign reading in the header) */
    double *Spsi = (double *)malloc(sizeof(double) * 3 * N);
    double *Srho = (double *)malloc(sizeof(double) * 3 * N);
    oracle_stencil(o, o->psi, 4.0 / 3.0, -1.0 / 6.0, Spsi);
    oracle_stencil(o, o->rho, 2.0, -1.0, Srho);
    double fs = (o->flags & ORACLE_FORCE_PRINTED_SIGN) ? 1.0 : -1.0;
    #pragma omp parallel for
    for (long n = 0; n < N; ++n)
        for (int al = 0; al < 3; ++al) {
            long k = al * N + n;
            if (o->mask[n] || al >= D) { o->F[k] = 0.0; continue; }
            o->F[k] = fs * (o->sgn[n] * 2.0 * o->psi[n] * Spsi[k] + o->kappa * o->rho[n] * Srho[k])
                      + o->rho[n] * o->g[al];
        }
    free(Spsi);
    free(Srho);
}

/* Steps 1-4 of the update on the current populations: rho, u, P, psi, s, F, Phi. */
static void macroscopic(oracle_ctx *o)
{
    long N = o->N;
    int Q = o->Q, D = o->D;
    /* moments, Sec. 2.3.3 */
    #pragma omp parallel for
    for (long n = 0; n < N; ++n) {
        if (o->mask[n]) {
            o->rho[n] = o->rho_w;
            for (int al = 0; al < 3; ++al) o->u[al * N + n] = 0.0;
            continue;
        }
        double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            double fi = o->f[(long)i * N + n];
            rho += fi;
            for (int al = 0; al < D; ++al) j[al] += o->c[i][al] * fi;
        }
        o->rho[n] = rho;
        for (int al = 0; al < 3; ++al) o->u[al * N + n] = al < D ? j[al] / rho : 0.0;
    }
    force_from_density(o);
    /* correction term, Eq. correction with P0 = rho/3 (sign reading in the header);
     * the omega of (1 - omega/2) is the node's own */
    double psg = (o->flags & ORACLE_PHI_OFF) ? 0.0 : ((o->flags & ORACLE_PHI_PRINTED_SIGN) ? 1.0 : -1.0);
    #pragma omp parallel for collapse(2)
    for (long z = 0; z < o->nz; ++z)
        for (long y = 0; y < o->ny; ++y)
            for (long x = 0; x < o->nx; ++x) {
                long n = node_at(o, x, y, z);
                for (int al = 0; al < 3; ++al) {
                    long k = al * N + n;
                    if (o->mask[n] || al >= D) { o->Phi[k] = 0.0; continue; }
                    long e[3] = {0, 0, 0};
                    e[al] = 1;
                    long np = node_at(o, x + e[0], y + e[1], z + e[2]);
                    long nm = node_at(o, x - e[0], y - e[1], z - e[2]);
                    double up = o->u[al * N + np], um = o->u[al * N + nm];
                    double gp = o->rho[np] * up * up * up;
                    double gm = o->rho[nm] * um * um * um;
                    double pref = psg * (1.0 - 0.5 * omega_at(o, o->rho[n]));
                    o->Phi[k] = pref * 0.5 * (gp - gm);
                }
            }
}

/* Interpolated bounce-back (Bouzidi, Firdaouss and Lallemand, linear form;
 * the paper uses it for curved solids, Sec. 4.5): for a link from fluid x
 * along c_i into a solid, with the wall at the fraction q of the link,
 *   q < 1/2:  f_ib(x) = 2q f_i*(x) + (1 - 2q) f_i*(x - c_i)
 *   q >= 1/2: f_ib(x) = f_i*(x) / (2q) + (2q - 1)/(2q) f_ib*(x)
 * (f* post-collision, ib the opposite of i). After the push step with
 * halfway bounce-back, f_ib(x) holds f_i*(x), f_i(x) holds f_i*(x - c_i)
 * and f_ib(x - c_i) holds f_ib*(x), so each link is updated from the new
 * buffer. Links with q <= 0, or whose x - c_i is solid, stay halfway;
 * q = 1/2 is halfway exactly. Reading: the interpolation does not conserve
 * mass, and with the non-ideal force and a virtual wall density that
 * defect grows exponentially at walls (tested), so each node returns the
 * sum of its links' changes through its rest population, which makes the
 * boundary mass-conserving. */
static void interpolated_bounce_back(oracle_ctx *o)
{
    const long N = o->N;
    const int Q = o->Q, D = o->D;
    for (long z = 0; z < o->nz; ++z)
        for (long y = 0; y < o->ny; ++y)
            for (long x = 0; x < o->nx; ++x) {
                long n = node_at(o, x, y, z);
                if (o->mask[n]) continue;
                double excess = 0.0;
                for (int i = 0; i < Q; ++i) {
                    const int *c = o->c[i];
                    long nd = node_at(o, x + c[0], y + c[1], z + (D == 3 ? c[2] : 0));
                    double q = o->qw[(long)i * N + n];
                    if (!o->mask[nd] || !(q > 0.0)) continue;
                    long nm = node_at(o, x - c[0], y - c[1], z - (D == 3 ? c[2] : 0));
                    if (o->mask[nm]) continue;
                    int ib = Q - 1 - i;
                    double a = o->fnew[(long)ib * N + n];
                    double v;
                    if (q < 0.5) v = 2.0 * q * a + (1.0 - 2.0 * q) * o->fnew[(long)i * N + n];
                    else v = a / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * o->fnew[(long)ib * N + nm];
                    o->fnew[(long)ib * N + n] = v;
                    excess += v - a;
                }
                o->fnew[(long)(Q / 2) * N + n] -= excess;   /* mass-conserving */
            }
}

/* One time step: Eq. LBGK with push streaming, f_i(r + c_i, t+1) = post_i(r, t);
 * halfway bounce-back: a population headed into a solid node returns to
 * its origin in the opposite direction. */
static void step_once(oracle_ctx *o)
{
    long N = o->N;
    int Q = o->Q, D = o->D;
    macroscopic(o);
    double feq[27], fst[27];
    #pragma omp parallel for collapse(2) private(feq, fst)
    for (long z = 0; z < o->nz; ++z)
        for (long y = 0; y < o->ny; ++y)
            for (long x = 0; x < o->nx; ++x) {
                long n = node_at(o, x, y, z);
                if (o->mask[n]) continue;
                double u[3], F[3], Phi[3];
                for (int al = 0; al < 3; ++al) {
                    u[al] = o->u[al * N + n];
                    F[al] = o->F[al * N + n];
                    Phi[al] = o->Phi[al * N + n];
                }
                oracle_feq(o, o->rho[n], u, feq);
                oracle_fstar(o, o->rho[n], u, F, Phi, fst);
                const double om = omega_at(o, o->rho[n]);
                for (int i = 0; i < Q; ++i) {
                    double fi = o->f[(long)i * N + n];
                    double post = fi + om * (feq[i] - fi) + (fst[i] - feq[i]);
                    const int *c = o->c[i];
                    long dst = node_at(o, x + c[0], y + c[1], z + (D == 3 ? c[2] : 0));
                    if (o->mask[dst]) o->fnew[(long)(Q - 1 - i) * N + n] = post;
                    else o->fnew[(long)i * N + dst] = post;
                }
            }
    if (o->qw) interpolated_bounce_back(o);
    double *t = o->f; o->f = o->fnew; o->fnew = t;
}

/* Populations at rest in the physical velocity: f = f_eq(rho0, U0 - F/(2 rho0))
 * at fluid nodes, with F the force of the density field rho0 (Eq. Kforce_final),
 * so that U = u + F/(2 rho) (Sec. 2.3.5) equals U0 at t = 0; 0 at solid nodes.
 * The paper does not state its initial populations; f_eq(rho0, U0) would start
 * every interface with U = F/(2 rho) != 0, an impulse that at large density
 * ratios sends a pressure wave into the liquid. u0 NULL means U0 = 0. */
void oracle_init(oracle_ctx *o, const double *rho0, const double *u0)
{
    long N = o->N;
    double feq[27];
    memset(o->fnew, 0, sizeof(double) * o->Q * N);
    for (long n = 0; n < N; ++n) o->rho[n] = o->mask[n] ? o->rho_w : rho0[n];
    force_from_density(o);
    for (long n = 0; n < N; ++n) {
        if (o->mask[n]) {
            for (int i = 0; i < o->Q; ++i) o->f[(long)i * N + n] = 0.0;
            continue;
        }
        double u[3] = {0.0, 0.0, 0.0};
        for (int al = 0; al < o->D; ++al)
            u[al] = (u0 ? u0[al * N + n] : 0.0) - o->F[al * N + n] / (2.0 * rho0[n]);
        oracle_feq(o, rho0[n], u, feq);
        for (int i = 0; i < o->Q; ++i) o->f[(long)i * N + n] = feq[i];
    }
}

/* Density-dependent relaxation: vapour relaxation time tau_v (> 0; 0 turns
 * it off) and the densities rho_v < rho_l between which nu is interpolated. */
void oracle_set_viscosity(oracle_ctx *o, double tau_v, double rho_v, double rho_l)
{
    o->tau_v = tau_v;
    o->visc_rv = rho_v;
    o->visc_rl = rho_l;
}

/* Wall distances q[i * N + n] of the links from node n along c_i into a
 * solid (ignored elsewhere; q <= 0: halfway bounce-back). NULL clears. */
void oracle_set_wall_distances(oracle_ctx *o, const double *q)
{
    free(o->qw);
    o->qw = NULL;
    if (!q) return;
    o->qw = (double *)malloc(sizeof(double) * o->Q * o->N);
    memcpy(o->qw, q, sizeof(double) * o->Q * o->N);
}

void oracle_step(oracle_ctx *o, long nsteps)
{
    for (long s = 0; s < nsteps; ++s) step_once(o);
}

/* rho, bare u (D planes), physical U = u + F/(2 rho) (Sec. 2.3.5), force F. */
void oracle_moments(oracle_ctx *o, double *rho, double *u, double *U, double *F)
{
    long N = o->N;
    macroscopic(o);
    for (long n = 0; n < N; ++n) {
        if (rho) rho[n] = o->rho[n];
        for (int al = 0; al < o->D; ++al) {
            long k = al * N + n;
            if (u) u[k] = o->u[k];
            if (U) U[k] = o->mask[n] ? 0.0 : o->u[k] + o->F[k] / (2.0 * o->rho[n]);
            if (F) F[k] = o->F[k];
        }
    }
}

/* Mass and momentum over fluid nodes: M = sum rho, J = sum rho u = sum c_i f_i. */
void oracle_reduce(oracle_ctx *o, double *mass, double *mom)
{
    long N = o->N;
    double M = 0.0, J[3] = {0.0, 0.0, 0.0};
    for (long n = 0; n < N; ++n) {
        if (o->mask[n]) continue;
        for (int i = 0; i < o->Q; ++i) {
            double fi = o->f[(long)i * N + n];
            M += fi;
            for (int al = 0; al < o->D; ++al) J[al] += o->c[i][al] * fi;
        }
    }
    *mass = M;
    for (int al = 0; al < o->D; ++al) mom[al] = J[al];
}

void oracle_get_populations(const oracle_ctx *o, double *out)
{
    memcpy(out, o->f, sizeof(double) * o->Q * o->N);
}

void oracle_set_populations(oracle_ctx *o, const double *in)
{
    memcpy(o->f, in, sizeof(double) * o->Q * o->N);
}

void oracle_weights(const oracle_ctx *o, double *w, int *c)
{
    for (int i = 0; i < o->Q; ++i) {
        w[i] = o->w[i];
        for (int al = 0; al < 3; ++al) c[3 * i + al] = o->c[i][al];
    }
}

/* Vectorised EOS for host-side tools (Maxwell construction, widths). */
void oracle_eos_pressure_array(int eos, double a, double b, double RT, double alpha,
                               const double *rho, long n, double *out)
{
    for (long k = 0; k < n; ++k) out[k] = oracle_eos_pressure(eos, a, b, RT, alpha, rho[k]);
}

/* Discrete pressure tensor (Appendix E) of the current state, at fluid nodes:
 *   P_ab = sum_i c_ia c_ib f_i  +  P^A + P^B + P^C + P^D,
 * the populations' momentum flux plus the non-local contributions of the
 * four ring terms of the force. With the force on the fluid being the
 * negative of the printed Kforce_final (sign reading in the header), the
 * non-local part is the negative of the printed one:
 *   P^A =  s 4/3 psi sum_i (w_i/cs2) c_ia c_ib psi(r+c_i)
 *   P^B = -s 1/6 [psi sum_i (w_i/cs2) c c psi(r+2c_i) + sum_i (w_i/cs2) c c psi(r-c_i) psi(r+c_i)]
 *   P^C =  kappa rho sum_i (w_i/cs2) c c rho(r+c_i)
 *   P^D = -kappa/2 [rho sum_i (w_i/cs2) c c rho(r+2c_i) + sum_i (w_i/cs2) c c rho(r-c_i) rho(r+c_i)]
 * with s the sign of P - P0 at r. For a uniform state at rest it reduces to
 * P(rho) I. Out: components xx, yy[, zz], xy[, xz, yz], each an N-plane
 * (0 at solid nodes). Reading of the kinetic part: the paper does not state
 * it; the populations' second moment makes P_xx uniform across a resting
 * flat interface, rho/3 alone does not (tested). */
void oracle_pressure_tensor(oracle_ctx *o, double *out)
{
    const long N = o->N;
    const int Q = o->Q, D = o->D;
    const int na = D == 3 ? 6 : 3;
    const int A_[6] = {0, 1, 2, 0, 0, 1}, B_[6] = {0, 1, 2, 1, 2, 2};
    const int A2[3] = {0, 1, 0}, B2[3] = {0, 1, 1};
    macroscopic(o);
    #pragma omp parallel for collapse(2)
    for (long z = 0; z < o->nz; ++z)
        for (long y = 0; y < o->ny; ++y)
            for (long x = 0; x < o->nx; ++x) {
                long n = node_at(o, x, y, z);
                for (int k = 0; k < na; ++k) {
                    int al = D == 3 ? A_[k] : A2[k], be = D == 3 ? B_[k] : B2[k];
                    if (o->mask[n]) { out[(long)k * N + n] = 0.0; continue; }
                    double kin = 0.0, pa = 0.0, pb1 = 0.0, pb2 = 0.0, pc = 0.0, pd1 = 0.0, pd2 = 0.0;
                    for (int i = 0; i < Q; ++i) {
                        const int *c = o->c[i];
                        double cc = (double)(c[al] * c[be]);
                        kin += cc * o->f[(long)i * N + n];
                        if (cc == 0.0) continue;
                        double wc = o->w[i] * 3.0 * cc;
                        long n1 = node_at(o, x + c[0], y + c[1], z + (D == 3 ? c[2] : 0));
                        long n2 = node_at(o, x + 2 * c[0], y + 2 * c[1], z + (D == 3 ? 2 * c[2] : 0));
                        long nm = node_at(o, x - c[0], y - c[1], z - (D == 3 ? c[2] : 0));
                        pa += wc * o->psi[n1];
                        pb1 += wc * o->psi[n2];
                        pb2 += wc * o->psi[nm] * o->psi[n1];
                        pc += wc * o->rho[n1];
                        pd1 += wc * o->rho[n2];
                        pd2 += wc * o->rho[nm] * o->rho[n1];
                    }
                    double sg = (double)o->sgn[n], ps = o->psi[n], r = o->rho[n];
                    out[(long)k * N + n] = kin + sg * (4.0 / 3.0) * ps * pa
                                           - sg * (1.0 / 6.0) * (ps * pb1 + pb2)
                                           + o->kappa * r * pc - 0.5 * o->kappa * (r * pd1 + pd2);
                }
            }
}

/* One node's post-collision populations from its local neighbourhood, for
 * checking large lattices at sampled nodes. block[((dz*5 + dy)*5 + dx)*Q + i]
 * holds the populations of the node at offset (dx-2, dy-2, dz-2) (dz = 2 only
 * for D2Q9), mblock the matching solid flags. The same steps as a full step
 * (moments, EOS and pseudo-potential, Eq. Kforce_final stencils, Eq.
 * correction, product-form collision) restricted to what the centre needs.
 * out[i] = post-collision population i of the centre node. */
void oracle_post_local(const oracle_ctx *o, const double *block, const unsigned char *mblock,
                       double *out)
{
    const int Q = o->Q, D = o->D;
    const int nz5 = D == 3 ? 5 : 1;
    double rho[125], u[3][125], psi[125];
    int sgn[125];
    for (int k = 0; k < 125; ++k) { rho[k] = 0.0; psi[k] = 0.0; sgn[k] = -1; u[0][k] = u[1][k] = u[2][k] = 0.0; }
#define LIDX(dx, dy, dz) ((((D == 3 ? (dz) + 2 : 0) * 5 + (dy) + 2) * 5) + (dx) + 2)
    for (int bz = 0; bz < nz5; ++bz)
        for (int by = 0; by < 5; ++by)
            for (int bx = 0; bx < 5; ++bx) {
                int k = (bz * 5 + by) * 5 + bx;
                if (mblock[k]) {
                    rho[k] = o->rho_w;
                } else {
                    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
                    for (int i = 0; i < Q; ++i) {
                        double fi = block[(long)k * Q + i];
                        r += fi;
                        for (int al = 0; al < D; ++al) j[al] += o->c[i][al] * fi;
                    }
                    rho[k] = r;
                    for (int al = 0; al < D; ++al) u[al][k] = j[al] / r;
                }
                double P = oracle_eos_pressure(o->eos, o->a, o->b, o->RT, o->alpha, rho[k]);
                double P0 = rho[k] / 3.0;
                psi[k] = P > P0 ? sqrt(P - P0) : sqrt(P0 - P);
                sgn[k] = P > P0 ? 1 : -1;
            }
    const int c0 = LIDX(0, 0, 0);
    /* force at the centre: the two stencils of Eq. Kforce_final, force on the fluid */
    double Spsi[3] = {0.0, 0.0, 0.0}, Srho[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        const int *c = o->c[i];
        int k1 = LIDX(c[0], c[1], c[2]), k2 = LIDX(2 * c[0], 2 * c[1], 2 * c[2]);
        double vp = (4.0 / 3.0) * psi[k1] + (-1.0 / 6.0) * psi[k2];
        double vr = 2.0 * rho[k1] + (-1.0) * rho[k2];
        for (int al = 0; al < D; ++al) {
            Spsi[al] += (o->w[i] * 3.0) * c[al] * vp;
            Srho[al] += (o->w[i] * 3.0) * c[al] * vr;
        }
    }
    double fs = (o->flags & ORACLE_FORCE_PRINTED_SIGN) ? 1.0 : -1.0;
    double F[3] = {0.0, 0.0, 0.0}, Phi[3] = {0.0, 0.0, 0.0}, uc[3] = {0.0, 0.0, 0.0};
    const double om = omega_at(o, rho[c0]);
    double pref = (o->flags & ORACLE_PHI_OFF) ? 0.0 : -(1.0 - 0.5 * om);
    if (o->flags & ORACLE_PHI_PRINTED_SIGN) pref = -pref;
    for (int al = 0; al < D; ++al) {
        F[al] = fs * (sgn[c0] * 2.0 * psi[c0] * Spsi[al] + o->kappa * rho[c0] * Srho[al])
                + rho[c0] * o->g[al];
        int e[3] = {0, 0, 0};
        e[al] = 1;
        int kp = LIDX(e[0], e[1], e[2]), km = LIDX(-e[0], -e[1], -e[2]);
        double gp = rho[kp] * u[al][kp] * u[al][kp] * u[al][kp];
        double gm = rho[km] * u[al][km] * u[al][km] * u[al][km];
        Phi[al] = pref * 0.5 * (gp - gm);
        uc[al] = u[al][c0];
    }
    double feq[27], fst[27];
    oracle_feq(o, rho[c0], uc, feq);
    oracle_fstar(o, rho[c0], uc, F, Phi, fst);
    for (int i = 0; i < Q; ++i) {
        double fi = block[(long)c0 * Q + i];
        out[i] = fi + om * (feq[i] - fi) + (fst[i] - feq[i]);
    }
#undef LIDX
}
