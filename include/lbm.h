/*
 * lbm.h - C ABI of the GB300 two-phase lattice Boltzmann library (liblbm.so).
 *
 * The library advances the kinetic model of Hosseini, Dorschner & Karlin,
 * "Towards a consistent lattice Boltzmann model for two-phase fluids"
 * (arXiv 2112.01975), on the D2Q9 and D3Q27 lattices, one GPU per handle.
 * One time step (Sec. 2.3) is:
 *   moments            rho = sum_i f_i, rho u = sum_i c_i f_i           (Sec. 2.3.3)
 *   equation of state  P(rho) of vdW, PR, RKS or CS                    (Sec. 3.1)
 *   pseudo-potential   psi = sqrt|P - P0|, P0 = rho/3                   (Sec. 2.3.4, 2.3.5)
 *   Korteweg force     2-ring isotropic stencils of psi and rho         (Eq. Kforce_final)
 *   correction Phi     diagonal third-moment correction                 (Eq. correction)
 *   collision          f + omega (feq - f) + (f* - feq), product form   (Eqs. LBMeq, LBGK, LBMstar)
 *   streaming          f_i(r + c_i, t + 1) = post_i(r, t); a population
 *                      headed into a solid node is bounced back halfway
 *                      into the opposite direction at its origin.
 * The force enters xi* = u + F/rho as the force acting on the fluid,
 * F = -s 2 psi S_psi - kappa rho S_rho (the printed Kforce_final is the
 * momentum-balance term, of opposite sign); zeta* = 1/3 + xi*^2 + Phi/rho;
 * Phi_aa = -(1 - omega/2) d_a(rho u_a^3) by a central difference.
 *
 * Units are lattice units: dr = dt = 1, cs^2 = 1/3, gas constant R = 1.
 *
 * Layouts (all arrays row-major with x fastest):
 *   node index        n = x + nx * (y + ny * z), N = nx * ny * nz nodes
 *   scalar field      double[N]
 *   vector field      double[D * N], component a at [a * N + n] (D = 2 or 3)
 *   populations       double[Q * N], direction i at [i * N + n],
 *                     i = (cx+1) + 3 (cy+1) [+ 9 (cz+1)], opposite = Q-1-i
 *   solid mask        uint8_t[N], 1 = solid, 0 = fluid
 *
 * Ownership: the library copies every host input and keeps no caller
 * pointer, except memory passed to lbm_bind_device_memory, which the caller
 * keeps alive until lbm_destroy. A handle is not thread-safe; all its work
 * is ordered on one CUDA stream (lbm_set_stream). Device pointers passed
 * with on_device = 1 must be readable/writable on the handle's device and
 * stream.
 *
 * Errors: every call returns an lbm_status; nothing is thrown across the
 * ABI. lbm_last_error() gives a message for the last failure of a handle.
 * A step that produced a non-finite or non-positive density is reported as
 * LBM_ENONFINITE by the next synchronising call (lbm_sync, lbm_moments,
 * lbm_reduce, lbm_get_populations); the handle then refuses lbm_step with
 * LBM_ESTATE until lbm_init or lbm_set_populations.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx *lbm_handle;

enum lbm_lattice { LBM_D2Q9 = 0, LBM_D3Q27 = 1 };

/* Equations of state of Sec. 3.1: van der Waals (Eq. vdWEoS), Peng-Robinson
 * (Eq. PREoS), Redlich-Kwong-Soave (Eq. RKSEoS), Carnahan-Starling (Eq. CSEos);
 * and the two Shan-Chen forms of Appendix G, P = rho/3 + (G/6) psi_SC^2 with
 * psi_SC = 1 - exp(-rho) (Eq. SC1, critical coupling G_c = -4) or
 * exp(-1/rho) (Eq. SC2, G_c = -e^2). For these T/Tc sets the coupling
 * G = G_c / (T/Tc), and the a, b of lbm_params are not used (b must still
 * be positive). */
enum lbm_eos {
    LBM_EOS_VDW = 0, LBM_EOS_PR = 1, LBM_EOS_RKS = 2, LBM_EOS_CS = 3,
    LBM_EOS_SC1 = 4, LBM_EOS_SC2 = 5
};

/* Population storage. LBM_F64 stores and computes in FP64 (two kernels per
 * step). LBM_F32 stores populations in FP32 and runs the step as one fused
 * FP32 kernel. LBM_F16S / LBM_BF16S store each population as the 16-bit
 * (FP16 / BF16) relative deviation h_i = f_i / rho(src) - w_i from the
 * weight, rho(src) the FP32 density of the node that pushed it (the node
 * itself after a bounce-back), with an FP32 density field beside each
 * buffer (-1 at solid nodes, whose fluid neighbours' bounced populations
 * are stored relative to those neighbours' own densities); the fused step
 * computes in FP32. Moments, reductions and population I/O are FP64 at the
 * ABI for every storage. */
enum lbm_storage { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2, LBM_BF16S = 3 };

enum lbm_status {
    LBM_OK = 0,
    LBM_EINVAL = 1,      /* bad argument; nothing changed */
    LBM_ENOMEM = 2,      /* device allocation failed or bound memory too small */
    LBM_ECUDA = 3,       /* a CUDA call failed; see lbm_last_error */
    LBM_ENONFINITE = 4,  /* a density became non-finite or <= 0 */
    LBM_ETIMEOUT = 5,    /* lbm_sync deadline passed; work still in flight */
    LBM_ESTATE = 6,      /* call not valid in the handle's state */
    LBM_ETOOBIG = 7      /* size beyond a fixed maximum of the library */
};

/* Flags of lbm_params.flags. */
enum {
    LBM_FLAG_PHI_OFF = 1,  /* drop the correction Phi (Eq. correction) */
    /* Reduced storage (LBM_F32, LBM_F16S, LBM_BF16S): evaluate the EOS, the
     * pseudo-potential psi = sqrt|P - P0| and the force's stencil sums and
     * combination in FP64 inside the fused step (populations, moments and
     * the collision stay FP32). Meant for deep-subcritical states, where P
     * and rho/3 nearly cancel in the vapour and 1 - b rho is small in the
     * liquid. Runs the plain 32 x 8 form only (no other variant or tile, no
     * batches: LBM_EINVAL), at the GPU's FP64 rate. No effect on LBM_F64. */
    LBM_FLAG_EOS_F64 = 2
};

/* EOS constants and options. a, b: EOS attraction and co-volume (lattice
 * units, R = 1); acentric: acentric factor of PR/RKS (Sec. 3.1); rho_w:
 * virtual density of solid nodes seen by both force stencils (Sec. 4.5). */
typedef struct {
    double a, b, acentric, rho_w;
    int storage;   /* enum lbm_storage */
    int flags;     /* LBM_FLAG_* */
    double g[3];   /* body acceleration (gx, gy, gz; D2Q9 uses gx, gy): the force
                      rho g joins the Korteweg force in xi* and in U (the generic
                      force F of Eq. LBGK; Sec. 4.1 drives layered Poiseuille
                      flow with it). Must be finite; default 0. */
    double tau_v;        /* > 0: density-dependent relaxation. The kinematic
                            viscosity nu = (tau - 1/2)/3 goes linearly in rho
                            from the liquid value (the tau of lbm_create) at
                            visc_rho[1] to the vapour value (tau_v) at
                            visc_rho[0], constant beyond; omega, and the
                            (1 - omega/2) of Eq. correction, per node. The
                            paper sets a vapour to liquid viscosity ratio
                            (Sec. 5.2) without the interpolation. 0 (default):
                            one tau everywhere. Else must exceed 1/2, and
                            0 < visc_rho[0] < visc_rho[1]. */
    double visc_rho[2];  /* rho_v, rho_l of the interpolation */
} lbm_params;

/* Fill p with the defaults of an EOS: vdW a = 9/49, b = 2/21; PR and RKS
 * a = 2/49, b = 2/21; CS a = 1, b = 4; Shan-Chen a = b = 1 (unused);
 * acentric 0.344; rho_w = 1; LBM_F64; no flags; g = 0; tau_v = 0 (one
 * relaxation time). Returns LBM_EINVAL for an unknown eos. */
int lbm_default_params(int eos, lbm_params *p);

/* Create a handle for one lattice. lattice: enum lbm_lattice. nx, ny, nz:
 * lattice size, each >= 5 (the 2-ring stencils must not alias under the
 * periodic wrap); nz must be 1 for D2Q9; at most 4e9 / 27 nodes (about
 * 148 million, e.g. 529^3: the kernels index populations with 32-bit
 * integers), else LBM_EINVAL. eos: enum lbm_eos. t_over_tc:
 * reduced temperature, 0 < T/Tc < 1 (T = (T/Tc) Tc, Tc from a and b by the
 * relations printed under each EOS). kappa: capillary coefficient kappa~ of
 * Eq. capillary_discrete, >= 0. tau: relaxation time, omega = 1/tau, > 1/2
 * (kinematic viscosity (tau - 1/2)/3). solid_mask: host uint8_t[N] or NULL
 * (all fluid); copied. p: NULL for lbm_default_params(eos). Allocates no
 * device memory; uses the current CUDA device. */
int lbm_create(lbm_handle *out, int lattice, int nx, int ny, int nz, int eos,
               double t_over_tc, double kappa, double tau, const uint8_t *solid_mask,
               const lbm_params *p);

/* Device bytes a handle of this shape and storage needs (populations,
 * side fields, mask, reduction partials), or 0 for invalid arguments. */
size_t lbm_required_bytes(int lattice, int nx, int ny, int nz, int storage);

/* Use caller-owned device memory (e.g. a torch tensor) of at least
 * lbm_required_bytes bytes, 256-byte aligned, instead of allocating.
 * Must be called before lbm_init. */
int lbm_bind_device_memory(lbm_handle h, void *dev, size_t bytes);

/* Order all later work of the handle on this cudaStream_t (NULL: the
 * handle's own stream, created by lbm_create). */
int lbm_set_stream(lbm_handle h, void *stream);

/* Set the initial populations at fluid nodes to the equilibrium of Eq. LBMeq
 * at density rho0 and bare velocity u = U0 - F/(2 rho0), where F is the
 * Korteweg force of the density field rho0 (Eq. Kforce_final, solid nodes at
 * rho_w), so that the physical velocity U = u + F/(2 rho) of Sec. 2.3.5 (the
 * U of lbm_moments) equals U0 at t = 0. The paper gives no initial
 * populations; starting from f_eq(rho0, U0) instead would give every
 * interface an initial velocity F/(2 rho). Solid nodes get zero populations.
 * rho0: double[N] (> 0 at fluid nodes); u0: double[D*N], component-major
 * (U0_x of all nodes, then U0_y[, U0_z]), or NULL for U0 = 0.
 * on_device: 0 if the pointers are host memory, 1 if device.
 * Allocates the device memory on first use unless bound. */
int lbm_init(lbm_handle h, const double *rho0, const double *u0, int on_device);

/* Advance n >= 0 time steps. Asynchronous on the handle's stream; steps
 * after the first are replayed from a CUDA graph of two steps. For n > 64
 * the device's status word is polled every 64 steps: each poll copies it to
 * pinned host memory behind an event and first waits for the previous copy,
 * so the call returns when at most one polling interval is still queued,
 * and a density that became non-finite or non-positive stops the launches
 * within 128 steps of appearing: LBM_ENONFINITE, after which the handle is
 * in LBM_ESTATE until lbm_init or lbm_set_populations. Divergence in the
 * last interval (or in calls with n <= 64) is reported by the next
 * synchronising call (lbm_sync, lbm_moments, lbm_reduce). The first long
 * call allocates the pinned word and the event (freed by lbm_destroy). */
int lbm_step(lbm_handle h, int64_t n);

/* Macroscopic fields of the current state: rho (double[N]), bare velocity
 * u = sum c_i f_i / rho (double[D*N]) and the physical velocity
 * U = u + F/(2 rho) of Sec. 2.3.5 (double[D*N]); any may be NULL. Solid
 * nodes report rho_w and zero velocities. Synchronises the stream. */
int lbm_moments(lbm_handle h, double *rho, double *u, double *U, int on_device);

/* Interpolated bounce-back for curved or off-grid walls (the linear scheme of
 * Bouzidi, Firdaouss and Lallemand that the paper uses for curved solids,
 * Sec. 4.5). q: host double[Q * N], component-major (q[i * N + n]): for a
 * link from fluid node n along c_i into a solid node, the wall sits at the
 * fraction q in (0, 1] of the link; entries <= 0, entries of other links,
 * and links whose node n - c_i is solid keep halfway bounce-back (q = 1/2
 * is halfway exactly). Each step then rewrites the populations bounced at
 * such links by interpolation and returns each boundary node's net change
 * through its rest population, so the walls conserve mass (without that
 * the interpolation's mass defect grows at walls under the non-ideal force).
 * NULL clears. Copies what it needs to device memory it allocates (freed by
 * lbm_destroy); synchronises. LBM_EINVAL for q > 1. Lattices with such walls
 * cannot join a batch. */
int lbm_set_wall_distances(lbm_handle h, const double *q);

/* Discrete pressure tensor of the current state (Appendix E): at each fluid
 * node the populations' momentum flux sum_i c_ia c_ib f_i plus the non-local
 * contributions of the four ring terms of the force (Eq. Kforce_final), with
 * the force on the fluid's sign. A uniform state at rest gives P(rho) I; a
 * resting flat interface gives a uniform normal component, and the tension
 * sigma = integral of (P_nn - P_tt) across it (Sec. 3.2). P: double[k * N],
 * components k = xx, yy, xy (D2Q9) or xx, yy, zz, xy, xz, yz (D3Q27), each
 * a node plane; 0 at solid nodes. on_device: P is device memory. Synchronises;
 * LBM_ENONFINITE if the state holds a bad density. */
int lbm_pressure_tensor(lbm_handle h, double *P, int on_device);

/* Mass sum rho and momentum sum rho u over fluid nodes (host outputs;
 * momentum has D entries), summed in a fixed order on the device.
 * Synchronises the stream. */
int lbm_reduce(lbm_handle h, double *mass, double *momentum);

/* Copy the populations (double[Q*N]) out or in. Solid-node entries read as
 * 0 and are ignored on input. Synchronising. */
int lbm_get_populations(lbm_handle h, double *f, int on_device);
int lbm_set_populations(lbm_handle h, const double *f, int on_device);

/* Wait for the handle's stream at most timeout_ms milliseconds (< 0: no
 * limit); LBM_ETIMEOUT if work is still running, LBM_ENONFINITE if a step
 * saw a bad density. */
int lbm_sync(lbm_handle h, int timeout_ms);

/* Number of kernel launches the handle has issued (graph replays count
 * each kernel in the graph). */
int64_t lbm_launch_count(lbm_handle h);

/* Measured FP64 rate of the current device: a grid of 8 blocks of 256
 * threads per SM runs eight independent FP64 fused multiply-add chains per
 * thread; *tflops = the best of three launches' 2 x FMAs / duration (CUDA
 * events), in TFLOP/s. The denominator for the FP64 step's ALU roofline,
 * measured on the machine that runs it. Allocates and frees a small device
 * buffer; synchronising. LBM_EINVAL for a null pointer, LBM_ECUDA (or
 * LBM_ENOMEM) if a CUDA call fails. */
int lbm_probe_fp64_tflops(double *tflops);

/* Self-test of the fused kernels' bounded waits on the current device: one
 * block of 64 threads waits, through the same wait function, for an
 * mbarrier phase that no thread ever completes; each warp gives up after
 * limit_cycles (1 .. 2e9) SM clock cycles and sets bit 2 of a status word,
 * as a timed-out wait in a step does. *status_bits = that word (2 when the
 * waits ran out and returned), *ms = the launch's duration. No fault, trap
 * or hang is involved: the kernel returns by itself and the context stays
 * usable. LBM_EINVAL for null pointers or a limit out of range, LBM_ECUDA
 * (or LBM_ENOMEM) if a CUDA call fails; synchronising. */
int lbm_selftest_wait_timeout(long long limit_cycles, int *status_bits, double *ms);

/* Advance n >= 1 steps with plain launches, timing each kernel with CUDA
 * events on the handle's stream. ms[0] receives the mean duration of the
 * moments kernel, ms[1] of the collide-and-stream kernel (milliseconds);
 * with LBM_F32 storage the step is one fused kernel, ms[0] = 0 and ms[1]
 * is its duration. Synchronising. */
int lbm_time_kernels(lbm_handle h, int64_t n, double *ms);

/* Planes per CTA along the march axis (z; the 2D y axis for D2Q9) of the
 * fused FP32 step, >= 1 (default 16 for D3Q27, 64 for D2Q9). A tuning knob:
 * results do not depend on it. */
int lbm_set_chunk(lbm_handle h, int chunk);

/* Pick the chunk of the fused FP32 step by timing candidates (4 to 128
 * planes and, on a longer march axis, 10/16 to 16/16 of it) on the
 * handle's own state (saved to a temporary device buffer and restored
 * afterwards, so the state is unchanged). Sets and returns it in
 * *chunk_out (0 for FP64 storage, which has no tile parameter). With
 * LBM_F32 storage it also picks the form of the step
 * (lbm_set_fused_variant), and for D3Q27 the tile height, 8 or 7
 * rows of 32 nodes (7 rows fill every SM with two CTAs in one wave where 8
 * rows leave some SMs with one, e.g. at 128^3); the shifted storages and
 * batches keep the plain form with 8 rows. Forms, tiles and chunks
 * change the work split only: results are bitwise the same. Synchronising;
 * allocates and frees one state-sized buffer; on failure the handle keeps
 * the form, tile and chunk it had. */
int lbm_autotune(lbm_handle h, int *chunk_out);

/* The tile of the fused step in use, in nodes: *tile_x = 32, *tile_y = 8 or
 * 7 (D3Q27; 7 only after lbm_autotune chose it), or 128 x 1 for D2Q9 rows;
 * 0 x 0 for LBM_F64 storage, which runs one thread per node. Either pointer
 * may be NULL. */
int lbm_get_tile(lbm_handle h, int *tile_x, int *tile_y);

/* Set the tile height of the D3Q27 LBM_F32 fused step: 8 (the default) or 7
 * rows of 32 nodes. Results are bitwise the same; only the work split and
 * the speed change. LBM_EINVAL for another height, another lattice or
 * storage. */
int lbm_set_tile(lbm_handle h, int tile_y);

/* Forms of the fused step of the reduced storages (LBM_F32 all but
 * LBM_FUSED_TM_TMA; LBM_F16S and LBM_BF16S all but
 * LBM_FUSED_WARP_SPECIALISED); the same arithmetic in the same order, so
 * results are bitwise the same whichever runs.
 *   LBM_FUSED_PLAIN (default): one thread group per tile; each entering
 *     plane's densities, pseudo-potentials and velocities are formed, the
 *     block synchronises, and the plane two behind collides and streams,
 *     reading its node's populations again (an L2 hit).
 *   LBM_FUSED_WARP_SPECIALISED: two thread groups per tile, one forming the
 *     entering planes and one colliding, handing planes over through
 *     shared-memory barriers instead of a barrier of the whole block per
 *     plane. A wait between the groups that does not end within about a
 *     second (a fault, never normal operation) makes the next synchronising
 *     call return LBM_ETIMEOUT.
 *   LBM_FUSED_TMEM: the plain form, with each node's populations kept in the
 *     SM's Tensor Memory from the plane's entry to its collision instead of
 *     being read twice; each block holds 256 columns (D3Q27; 64 for D2Q9) of
 *     Tensor Memory while it runs. */
enum {
    LBM_FUSED_PLAIN = 0,
    LBM_FUSED_WARP_SPECIALISED = 1,
    LBM_FUSED_TMEM = 2,
    LBM_FUSED_WS_TMEM = 3,
    LBM_FUSED_WS_TMA = 4,
    LBM_FUSED_TM_TMA = 5
};

/*   LBM_FUSED_WS_TMEM (D3Q27, 32 x 8 tiles; FP32 or shifted storage): the
 *     warp-specialised form with the Tensor Memory staging, the producer that
 *     loads a node leaving its populations in the lane of the consumer that
 *     collides it.
 *   LBM_FUSED_WS_TMA (D3Q27, 32 x 8 tiles; FP32 with nx a multiple of 4, or
 *     shifted storage with nx a multiple of 8): the LBM_FUSED_WS_TMEM form
 *     with each entering plane's populations on the tile's halo copied into
 *     shared memory by the tensor-memory-access unit (nine bulk tensor
 *     copies per plane, requested two planes ahead) instead of loaded by the
 *     producers; 215 KB (FP32) or 175 KB of shared memory per block. The
 *     tensor maps are made when the handle's device memory is laid out; if
 *     the CUDA driver offers no tensor-map encoder, a handle set to this
 *     form runs LBM_FUSED_WS_TMEM (lbm_get_fused_variant says which).
 *   LBM_FUSED_TM_TMA (shifted storage only; D3Q27, 32 x 8 tiles, nx a
 *     multiple of 8): the LBM_FUSED_TMEM form (one thread group, two blocks
 *     per SM) with each entering plane copied into shared memory by the
 *     tensor-memory-access unit in one stage, requested a phase ahead (one
 *     copy per plane where the tile's halo stays inside the lattice, nine
 *     elsewhere); without a tensor-map encoder it runs LBM_FUSED_TMEM.
 * Select a form of the fused step (lbm_autotune times the forms the
 * storage has). LBM_EINVAL for an unknown form, a form other than
 * LBM_FUSED_PLAIN with LBM_F64 storage or LBM_FLAG_EOS_F64, or
 * LBM_FUSED_WARP_SPECIALISED with shifted storage, LBM_FUSED_TM_TMA with
 * LBM_F32, or LBM_FUSED_WS_TMEM, LBM_FUSED_WS_TMA or LBM_FUSED_TM_TMA with
 * D2Q9 or 7-row tiles, or the TMA-staged forms with nx not a multiple of 4
 * (FP32) or 8 (shifted) or, after the memory is laid out, without tensor
 * maps. */
int lbm_set_fused_variant(lbm_handle h, int variant);

/* *variant = the form of the fused step in use. */
int lbm_get_fused_variant(lbm_handle h, int *variant);

/* ---- Batches: many lattices advanced by one persistent launch ----------
 * A batch holds count >= 1 distinct, initialised handles with the same
 * storage (LBM_F32, LBM_F16S or LBM_BF16S, not LBM_F64) and the same lattice
 * type, of any sizes and parameters; otherwise LBM_EINVAL. Each
 * lbm_batch_step launch gives every member one time step (the fused step of
 * that storage over all members' tiles, spread over a persistent grid of two
 * CTAs per SM); steps after the first replay a CUDA graph of two launches. Each
 * member's result is bitwise the same as stepping it alone. While the batch
 * exists the members' work is ordered on the batch's stream (members must
 * not be stepped, initialised or written individually); lbm_batch_destroy
 * hands them back, with their state advanced. Host-side arrays (descriptors, work items) are
 * copied to device memory allocated by lbm_batch_create. */
typedef struct lbm_batch_ctx *lbm_batch;

int lbm_batch_create(lbm_batch *out, const lbm_handle *members, int count);

/* Advance every member n >= 0 steps; asynchronous. */
int lbm_batch_step(lbm_batch b, int64_t n);

/* Wait for the batch; LBM_ENONFINITE if a member saw a bad density. After
 * it returns, and until the next lbm_batch_step, members may be read
 * (lbm_moments, lbm_reduce, lbm_get_populations). */
int lbm_batch_sync(lbm_batch b);

/* Launches issued by the batch (one per step). */
int64_t lbm_batch_launch_count(lbm_batch b);

void lbm_batch_destroy(lbm_batch b);

const char *lbm_last_error(lbm_handle h);

/* Largest node count lbm_reduce_noalloc accepts (8192 x 8192 nodes). */
#define LBM_REDUCE_NOALLOC_MAX_NODES 67108864

/* Mass sum_i f_i and momentum sum_i c_i f_i over the fluid nodes of a
 * caller-owned population array, computed without allocating anything.
 * The paper has no counterpart: this is for callers that cannot allocate
 * device memory (a process whose memory pool is reserved or frozen, or code
 * that only borrows device pointers from another framework). It does what
 * lbm_reduce does, but on arrays the caller passes and without a handle.
 *
 * lattice, nx, ny, nz: as lbm_create (nz = 1 for D2Q9), each >= 1 and at
 * most LBM_REDUCE_NOALLOC_MAX_NODES nodes in total, else LBM_ETOOBIG.
 * f_dev: device double[Q*N], layout of lbm_get_populations. mask_dev:
 * device uint8_t[N] (1 = solid, skipped) or NULL for all fluid. sums_dev:
 * device double[4] receiving (mass, jx, jy, jz); jz = 0 for D2Q9. stream: a
 * cudaStream_t or NULL (legacy default stream); the call is asynchronous on
 * it.
 *
 * Scratch: the per-block partial sums live in a 256 KiB array of static
 * device memory inside the library, present on every GPU that loads it
 * until the process exits. The first call on a device looks the array up
 * on that device (make it before any stream capture). Every call shares
 * the array and overwrites the partials it reads, so nothing needs
 * clearing, but calls whose kernels overlap on the GPU race: order them on
 * one stream. Returns LBM_EINVAL for bad arguments, LBM_ECUDA on a failed
 * launch. Calls no cudaMalloc, cudaFree or allocating library routine. */
int lbm_reduce_noalloc(int lattice, int nx, int ny, int nz, const double *f_dev,
                       const uint8_t *mask_dev, double *sums_dev, void *stream);

void lbm_destroy(lbm_handle h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
