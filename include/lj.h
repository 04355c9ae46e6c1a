/*
 * lj.h -- C ABI of liblj.so, a GB300 (sm_103a) implementation of the
 * short-ranged molecular-dynamics hot path of van Meel, Arnold, Frenkel,
 * Portegies Zwart and Belleman, "Harvesting graphics power for MD
 * simulations" (arXiv:0709.3225):
 *
 *   - periodic Lennard-Jones forces over cell lists with cutoff rc and the
 *     minimum image (Section 2, Eq. n2_force and the truncated/shifted LJ
 *     force; Section 3, cell lists over the centre cell and its 26
 *     neighbours);
 *   - the cell lists rebuilt at every step by a counting sort (Section 3.1
 *     places particles physically together per cell; here: count, scan and
 *     scatter into one sorted array);
 *   - velocity-Verlet integration (Section 2, last paragraph), run entirely
 *     on the GPU (Section 1).
 *
 * Conventions shared by every entry point:
 *   - Reduced units.  Positions x and velocities v are row-major (n, 3)
 *     IEEE double arrays.  Forces f are (n, 4): float x, y, z, e for
 *     LJ_PREC_MIXED, double x, y, z, e for LJ_PREC_FP64, where e is the
 *     particle's share (half of each pair energy) of the potential energy
 *     when energies were requested and 0 otherwise.
 *   - Unless the name ends in _host, array arguments are DEVICE pointers on
 *     the context's device, owned by the caller, 16-byte aligned (any
 *     cudaMalloc / torch allocation is), and must stay valid until the work
 *     queued on the context's stream has finished.
 *   - Work is queued asynchronously on the stream given to lj_create.  Calls
 *     that return host scalars (e_pot, virial, lj_energy, lj_check,
 *     lj_read_timing, lj_step_host) synchronize that stream first.
 *   - Every call returns an lj_status; nothing crosses the ABI as an
 *     exception.  Errors found inside kernels (non-finite coordinates, a
 *     wait that timed out) are latched on the device and returned by the
 *     next synchronizing call.
 *   - A context is not thread-safe: use one context per host thread.
 */
#ifndef LJ_H
#define LJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LJ_ABI_VERSION 1

typedef enum lj_status {
    LJ_OK = 0,
    LJ_EINVAL = 1,      /* bad argument (NULL, size, mode, misaligned pointer) */
    LJ_EBOX = 2,        /* box too small: fewer than 2k+1 cells per side */
    LJ_ECUDA = 3,       /* a CUDA runtime call failed */
    LJ_ENONFINITE = 4,  /* a position was NaN or infinite */
    LJ_ETIMEOUT = 5,    /* a bounded device wait expired */
    LJ_EOVERFLOW = 6,   /* an index would not fit in 32 bits */
    LJ_ENOMEM = 7       /* device or host allocation failed */
} lj_status;

typedef enum lj_shift {
    LJ_SHIFT_NONE = 0,   /* plain truncation at rc */
    LJ_SHIFT_ENERGY = 1, /* U - U(rc) for r < rc: energy continuous at rc */
    LJ_SHIFT_FORCE = 2   /* F - F(rc) (the paper's Section 2 form) and the
                            matching energy U - U(rc) + (r - rc) F(rc) */
} lj_shift;

typedef enum lj_precision {
    LJ_PREC_MIXED = 0,   /* FP32 pair arithmetic and per-particle sums,
                            FP64 positions, integrator, energy and virial */
    LJ_PREC_FP64 = 1     /* FP64 throughout */
} lj_precision;

/* Simulation parameters (Section 2 and 3: N, box, eps, sigma, rc, dt). */
typedef struct lj_params {
    int64_t n;           /* number of particles, 0 <= n < 2^31 */
    double box;          /* cubic periodic box side L > 0 */
    double eps;          /* LJ well depth, >= 0 */
    double sigma;        /* LJ diameter, > 0 */
    double rc;           /* cutoff radius, > 0 (the paper uses 2.5 sigma) */
    double dt;           /* time step for lj_step */
    double mass;         /* particle mass, > 0 */
    int32_t shift_mode;  /* lj_shift */
    int32_t precision;   /* lj_precision */
    int32_t cell_subdiv; /* cells per rc along each axis, k: 1 (cell side
                            >= rc, 27-cell stencil, Section 3), 2 (side >= rc/2,
                            125-cell stencil; FP32-mixed and flags 0 only) or
                            0 for the default (1).  n = floor(k L / rc) cells
                            per axis, n >= 2k + 1 required (LJ_EBOX). */
    int32_t flags;       /* 0, LJ_FLAG_RUN_STAGED or LJ_FLAG_RUN_DIRECT */
} lj_params;

/* lj_params.flags select the force kernel (same results; for comparison).
 * Default (0): the warp-per-cell kernels that take each pair once over the
 * half stencil (lj_set_tuning kernel 7; kernel 3, the 27-cell stencil, for
 * cell_subdiv 2), staged in shared memory relative to the cell centre: in
 * FP32-mixed contexts the FP32-mixed kernel, in FP64 contexts the FP64 warp
 * kernel in its pair-once form.
 * LJ_FLAG_RUN_STAGED: the run kernel (a CTA per run of cells along x) with its
 *   9 neighbour-row windows staged by bulk asynchronous copies.
 * LJ_FLAG_RUN_DIRECT: the run kernel reading neighbour cells from global
 *   memory. */
#define LJ_FLAG_RUN_STAGED 1
#define LJ_FLAG_RUN_DIRECT 2

typedef struct lj_ctx lj_ctx;

/* Library ABI version (LJ_ABI_VERSION). Host only. */
int lj_version(void);

/* Human-readable name of a status code. Host only; never NULL. */
const char *lj_strerror(int code);

/* Cells per box side for these parameters, n_x = int[k L / rc]
 * (Section 3.2, worked example L = 11 sigma, rc = 2.5 sigma -> 4), and
 * validation of p.  Host only, needs no GPU.  Returns LJ_EBOX when
 * n_x < 2k + 1 (Section 3.2 requires at least 3 cells per dimension),
 * LJ_EINVAL for bad parameters. */
int lj_grid(const lj_params *p, int32_t *nc_out);

/* Create a context on the current CUDA device for the simulation of
 * Sections 2 and 3: p gives N, the box, eps, sigma, rc, dt and the cell grid
 * (validated as by lj_grid: at least 2k + 1 cells per side, the Section 3.2
 * lower limit of three cells per dimension for k = 1).  Allocates all device
 * scratch (cell arrays, sorted positions, partial sums) once; no later call
 * allocates on the device except lj_step_host, lj_energy and
 * lj_observables, which allocate their staging buffers on first use.
 * stream is a cudaStream_t (NULL = the legacy default stream).  On error
 * *out is NULL. */
int lj_create(lj_ctx **out, const lj_params *p, void *stream);

/* Free a context (synchronizes its stream).  NULL is ignored. */
void lj_destroy(lj_ctx *ctx);

/* Bin x into cells (counting sort; Section 3.1 keeps each cell's particles
 * together in memory, here as one array sorted by cell, in CSR form with
 * per-cell counts and starts; the paper leaves the binning rule unstated,
 * read here as follows).  For each particle the wrapped position
 * w = x - L floor(x / L) (w >= L folds to w - L), the cell coordinate
 * c = trunc(w * (n_x / L)) clamped to [0, n_x - 1] per axis, the linear id
 * c_x + n_x (c_y + n_x c_z); per-cell counts and exclusive starts; the
 * sorted order.  x: device (n, 3) double, not modified. */
int lj_bin(lj_ctx *ctx, const double *x);

/* Copy the result of the last binning (the Section 3.1 cell lists) to
 * caller-owned DEVICE arrays (any may be NULL; 4-byte aligned, else
 * LJ_EINVAL): cell_of[n], count[n_x^3], start[n_x^3 + 1], perm[n], where
 * perm[start[c] .. start[c+1]) lists the particles of cell c (their order
 * within a cell is unspecified). */
int lj_get_cells(lj_ctx *ctx, int32_t *cell_of, int32_t *count, int32_t *start, int32_t *perm);

/* Bin x, then f_i = sum_{j != i, r_ij < rc} F(r_ij) (x_i - x_j)/r_ij over
 * the 27 surrounding cells at the minimum image (Eq. n2_force restricted to
 * the cutoff, Section 3).  f: device (n, 4) float or double per the
 * precision.  If e_pot or virial is non-NULL the potential energy
 * sum_{i<j} U(r_ij) and the virial sum_{i<j} r_ij F(r_ij) (FP64) are written
 * to those HOST addresses (synchronizes), and f[:, 3] holds per-particle
 * energies. */
int lj_forces(lj_ctx *ctx, const double *x, void *f, double *e_pot, double *virial);

/* ---- rand48 random numbers (Section 4) ---------------------------------
 * The series x_{n+1} = (a x_n + c) mod 2^48, a = 0x5DEECE66D, c = 0xB (Eq.
 * lrand48; the POSIX rand48 constants), generated by S parallel streams with
 * the leap-frog rule x_{n+S} = (A x_n + C) mod 2^48 (Eq. lrand48m).
 * `state` is a caller-owned device array of S uint64 (one 48-bit value per
 * stream).  Stream i holds the series element it outputs next; output round
 * r writes element r S + i of the call's range, so a call's output is the
 * serial series in order and consecutive calls continue it.  Calls on one
 * state array must not overlap.  Errors: LJ_EINVAL (negative sizes, host or
 * misaligned pointers), LJ_EOVERFLOW (S R >= 2^40), LJ_ECUDA. */

/* x_0 of srand48(seed): (low 32 bits of seed) << 16 | 0x330E.  Host. */
uint64_t lj_srand48_state(int64_t seed);

/* Jump constants A = a^m, C = c (1 + a + ... + a^{m-1}) mod 2^48 (Eq. AC,
 * with m terms in the sum).  Host; LJ_EINVAL for m < 0 or NULL outputs. */
int lj_rand48_jump(int64_t m, uint64_t *A, uint64_t *C);

/* state[i] = x_{i+1} for i < S: the first S elements after x0.  Async. */
int lj_rand48_seed(uint64_t *state, int64_t S, uint64_t x0, void *stream);

/* R rounds: out[r S + i] = x >> 17 (lrand48, 31 bits) of stream i's
 * element, then the stream jumps by S.  out: device int32[R S].  Async. */
int lj_rand48_lrand(uint64_t *state, int64_t S, int64_t R, int32_t *out, void *stream);

/* As lj_rand48_lrand with out[r S + i] = x 2^-48 (drand48, [0, 1)): device
 * double[R S]. */
int lj_rand48_drand(uint64_t *state, int64_t S, int64_t R, double *out, void *stream);

/* ---- Langevin thermostat ------------------------------------------------
 * The stochastic thermostat Section 1 names (single precision suffices for
 * systems held in equilibrium by one); the paper gives no scheme, read here
 * as BAOAB: v += (dt/2m) f; x += (dt/2) v; v = c1 v + c2 sqrt(kT/m) xi with
 * c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2); x += (dt/2) v, wrap, rebin;
 * f = F(x); v += (dt/2m) f.  xi: Box-Muller normals from the context's
 * rand48 series, one stream per particle: step s of particle i uses series
 * elements (4 s + k) n + i + 1, k = 0..3 (xi_x, xi_y from k = 0, 1; xi_z
 * from k = 2, 3).  In FP32-mixed the normals are formed in FP32.
 * lj_langevin_seed starts the series at srand48(seed) (allocates n uint64
 * on first use); lj_langevin_step runs nsteps steps (x, v, f as lj_step;
 * gamma, kT >= 0); it returns LJ_EINVAL before the first seed.  Async. */
int lj_langevin_seed(lj_ctx *ctx, int64_t seed);
int lj_langevin_step(lj_ctx *ctx, double *x, double *v, void *f, int32_t nsteps, double gamma, double kT);

/* Checkpoint / resume of the thermostat's random series (the paper has no
 * checkpointing; the rest of a run's state -- x, v, f -- is caller-owned).
 * lj_get_rng_state copies the context's n stream states (uint64, each the
 * 48-bit series element that stream outputs next) to the caller's device
 * array `state`; LJ_EINVAL before lj_langevin_seed or lj_set_rng_state.
 * lj_set_rng_state copies n states from `state` into the context
 * (allocating n uint64 on first use, as lj_langevin_seed); the values must
 * be below 2^48, as lj_get_rng_state returns them (larger ones cause no
 * fault but are no rand48 series).  A context given the state, x, v and f that
 * another context of the same parameters held between two calls continues
 * the run as that context would have: bitwise with lj_set_deterministic on
 * (the in-cell order then does not depend on the binning atomics) and no
 * skin (a skin's cell lists are rebuilt on the first step of a context).
 * Both: device pointers, 8-byte aligned (LJ_EINVAL otherwise); async on the
 * context's stream; n = 0 is a no-op. */
int lj_get_rng_state(lj_ctx *ctx, uint64_t *state);
int lj_set_rng_state(lj_ctx *ctx, const uint64_t *state);

/* All-pairs forces (Section 2, Eq. n2_force with the cutoff): the same
 * forces as lj_forces computed without cells, every pair at the minimum
 * image, O(n^2) work.  For small systems, as a GPU brute-force cross-check,
 * and for the all-pairs versus cell-list break-even study.  Arguments,
 * layout, precision, energy semantics and error behaviour as lj_forces.
 * Positions are taken relative to the box centre (absolute coordinates,
 * as the paper's N^2 code), so in FP32-mixed the pair vectors carry
 * rounding of order 2^-24 L rather than 2^-24 rc.  The cell arrays are not
 * touched.  Scratch of n x 16 B (32 B in FP64) times (1 + j-splits) is
 * allocated on the first call and kept. */
int lj_forces_n2(lj_ctx *ctx, const double *x, void *f, double *e_pot, double *virial);

/* nsteps velocity-Verlet steps (Section 2): v += dt/(2m) f; x += dt v;
 * x wrapped into [0, L); cells rebuilt; f = F(x); v += dt/(2m) f.
 * x, v: device (n, 3) double, updated in place.  f: device (n, 4), must hold
 * F(x) on entry (from lj_forces or a previous lj_step) and holds F at the
 * final positions on return. */
int lj_step(lj_ctx *ctx, double *x, double *v, void *f, int32_t nsteps);

/* As lj_step on HOST arrays (pageable or pinned): copies x, v, f to the
 * device, steps, copies them back, synchronizes.  The copies in arrive in
 * four parts on a second stream, and each part is kicked, drifted and
 * binned as soon as it is there (velocity Verlet without a skin or a fused
 * update); the copy of x back runs while the last force evaluation does.
 * Allocates staging buffers for x, v, f on first use. */
int lj_step_host(lj_ctx *ctx, double *x, double *v, void *f, int32_t nsteps);

/* Energies of the state (x, v): out[0] = kinetic energy (1/2) m sum v^2,
 * out[1] = potential energy sum_{i<j} U(r_ij) at x (the Section 2 pair
 * potential, truncated/shifted per shift_mode), out[2] = their sum, the
 * quantity whose conservation Section 5 names as the test of
 * single-precision runs; FP64; out is a HOST array of 3.  x, v: device.
 * Allocates a force buffer on first use.  Synchronizes. */
int lj_energy(lj_ctx *ctx, const double *x, const double *v, double *out);

/* Thermodynamic observables of the state (x, v), FP64, into the HOST array
 * out[6] (synchronizes):
 *   out[0] = E_kin = (1/2) m sum v^2,  out[1] = E_pot = sum_{i<j} U(r_ij),
 *   out[2] = E_kin + E_pot (the conserved energy whose drift Section 5 names
 *            as the test of single-precision runs),
 *   out[3] = W = sum_{i<j} r_ij F(r_ij), the virial of lj_forces,
 *   out[4] = T = 2 E_kin / (3n - 3) (k_B = 1; velocity Verlet conserves the
 *            total momentum, leaving 3n - 3 degrees of freedom; 0 for n < 2;
 *            the temperature a thermostat holds, Section 1),
 *   out[5] = P = (2 E_kin + W) / (3 L^3), the virial pressure.
 * E_pot and W come from the force kernels (Section 2 pair terms over the
 * Section 3 cells); T and P are formed on the device from the FP64 sums.
 * x, v: device (n, 3) double.  Errors as lj_energy. */
int lj_observables(lj_ctx *ctx, const double *x, const double *v, double *out);

/* Synchronize the stream and return (and clear) any error latched by a
 * kernel since the last check. */
int lj_check(lj_ctx *ctx);

/* Change eps and sigma of an existing context (rc, the box and the cell grid
 * stay).  Later launches on the context's stream use the new values.
 * LJ_EINVAL unless sigma > 0 and eps >= 0, both finite. */
int lj_set_params(lj_ctx *ctx, double eps, double sigma);

/* Vector-Jacobian product of the forces (the derivative of Eq. n2_force with
 * the Section 2 pair force, rc held fixed; the paper has no adjoint).  With
 * g = dL/dF (device (n, 3) double) at positions x (device (n, 3) double):
 *   dx     += scale * dL/dx,  dL/dx_i = sum_j J_ij (g_i - g_j),
 *             J = phi I + (phi'(r)/r) d d^T, phi = F(r)/r  (a Hessian-vector
 *             product of the potential energy; device (n, 3) double);
 *   dparam += scale * (dL/deps, dL/dsigma)  (device double[2]).
 * The cell list is piecewise constant in x and contributes nothing.  Pair
 * arithmetic in the context's precision; parameter sums in FP64 (FP32-mixed:
 * FP32 partial sums over a cell or a group of 32 candidates, then FP64).
 * Contexts on lj_set_tuning kernel 7 (the default for cell_subdiv 1, FP32-
 * mixed and FP64) evaluate each pair once (the contribution to j is the
 * negative of i's, J being even in d), adding by atomics, so their last bits
 * can differ between calls too.  Each call bins x again, so with the atomic
 * in-cell order FP32 results can differ in their last bits between calls
 * (lj_set_deterministic makes them repeat, with the 27-cell form).
 * Allocates an (n)-element cotangent buffer on first use, and for the
 * pair-once FP32-mixed form an (n)-element float4 accumulator.
 * Asynchronous. */
int lj_forces_vjp(lj_ctx *ctx, const double *x, const double *g, double scale, double *dx, double *dparam);

/* One step of the adjoint of lj_step's velocity Verlet (Section 2), from the
 * positions before (x_n) and after (x_n1) the step (device (n, 3) double).
 * With h = dt / 2m, in place on the device (n, 3) adjoints:
 *   lam_x += h VJP(x_n1, lam_v);  lam_v += dt lam_x;  lam_x += h VJP(x_n, lam_v),
 * and dparam += the matching parameter parts.  Running it for steps
 * n = N-1 .. 0 with lam = (dL/dx_N, dL/dv_N) leaves (dL/dx_0, dL/dv_0) in
 * lam and adds dL/d(eps, sigma) to dparam.  Asynchronous. */
int lj_vv_adjoint_step(lj_ctx *ctx, const double *x_n, const double *x_n1, double *lam_x, double *lam_v,
                       double *dparam);

/* Cell lists with a skin (Section 3.1: cells wider than the interaction
 * range plus a skin lambda stay valid while particles move, so they need not
 * be rebuilt every step; the paper's one-step-lagged update is the case of a
 * skin covering one step's motion, and it notes that a larger skin with
 * rebuilds every few steps is common practice).  skin = lambda >= 0:
 * cells of side >= (rc + skin) / k, i.e. n = int[k L / (rc + skin)] per
 * axis (LJ_EBOX if n < 2k + 1); skin = 0 restores rebuilding every step.
 * With skin > 0, lj_step rebuilds the cell lists only when some particle
 * has moved more than skin/2 since the last rebuild -- then two particles
 * within rc may have drifted out of each other's stencil -- or every
 * max_interval steps if max_interval > 0.  The decision is made on the
 * device from FP32 displacement sums, without host synchronization;
 * between rebuilds the sorted positions are refreshed from x in the old
 * cell order.  Forces are those of the exact cell list.  lj_forces,
 * lj_energy and the adjoint always rebuild.  Reallocates the cell arrays
 * when n changes; LJ_EINVAL with the fused update (lj_set_tuning kernel 0)
 * or skin < 0.  Synchronizes. */
int lj_set_skin(lj_ctx *ctx, double skin, int32_t max_interval);

/* Failure-detection self test.  Runs one device-side wait that cannot be
 * satisfied -- an mbarrier phase expecting 16 bytes that no copy delivers --
 * with the same bound as every bulk-copy wait of the force kernels: after
 * about 2^31 SM cycles (~1 s) it gives up, latches the timeout and the
 * kernel returns.  Returns what lj_check then reports: LJ_ETIMEOUT when the
 * bound works.  The context stays usable.  Synchronizes. */
int lj_wait_selftest(lj_ctx *ctx);

/* Deterministic cell order (enable 1; 0, the default, leaves the order in
 * which the binning atomics placed the particles).  With it on, every
 * binning sorts each cell's particles by index -- the order of a serial
 * counting sort -- so lj_get_cells returns exactly that permutation and
 * the forces are bitwise reproducible from run to run (energies summed
 * with dynamic work pulls still differ in the last bits; cells_per_grab 0
 * makes them reproducible too).  Costs one pass over the sorted positions
 * per binning and a second sorted-position buffer.  Synchronous only
 * through the allocation on first use. */
int lj_set_deterministic(lj_ctx *ctx, int32_t enable);

/* Graph replay for lj_step (enable 1, 0 = direct launches, the default).
 * With it on, a call of nsteps >= 3 launches its first and last steps
 * directly and replays one captured CUDA graph of a middle step for the
 * others (one launch per step instead of four or five).  The graph is
 * captured on the first such call and again whenever x, v or f point
 * elsewhere or lj_set_tuning, lj_set_skin, lj_set_params or
 * lj_set_deterministic changed the context; it is not used while
 * lj_set_timing is on.  Same results as direct launches. */
int lj_set_graph(lj_ctx *ctx, int32_t enable);

/* Rebuilds and steps counted in skin mode since lj_set_skin (a full
 * rebuild by lj_forces is not counted).  Host pointers; synchronizes. */
int lj_skin_stats(lj_ctx *ctx, int64_t *rebuilds, int64_t *steps);

/* Choose the force kernel of a context (same results; for autotuning):
 * kernel 0 = warp-per-cell kernel (FP32-mixed only) with the velocity-Verlet
 * update of lj_step fused into it, 1 = run kernel with bulk-copy staging,
 * 2 = run kernel reading global memory, 3 = warp-per-cell kernel over the
 * 27-cell stencil with the update in a separate kernel (in FP64 contexts
 * the FP64 warp kernel that compacts the in-range pairs before any FP64
 * arithmetic), 7 = warp-per-cell kernel that evaluates each pair once
 * (Newton's third law: Eq. n2_force is antisymmetric, so the pair force is
 * added to i and subtracted from j; the home cell with itself and with the
 * 13 neighbours of positive offset; the default for cell_subdiv 1, in
 * FP32-mixed and FP64 contexts; the contributions are added with atomics,
 * into f zeroed first (FP32-mixed) or into a context buffer in cell order
 * then copied to f (FP64), so the sums are not bitwise reproducible between
 * runs, and contexts with lj_set_deterministic on take kernel 3 instead), 4 = the paper's
 * fixed-capacity cell arrays (Section 3.1: 32 placeholders per cell, empty
 * ones computed as virtual particles; FP32-mixed; a cell with more than 32
 * particles latches LJ_EOVERFLOW, reported by lj_check), 5 = the warp
 * kernel with each cell's stencil bulk-copied into shared memory while the
 * previous cell computes (FP32-mixed), 6 = kernel 3 for forces, with
 * lj_step's steps run as one cooperative persistent launch each (the
 * batched kernel below with one replica, given this call's group_width
 * and cells_per_grab (0 taken as 1): no gaps between the phases of a step,
 * for small systems; FP32-mixed; steps with a skin or the deterministic
 * in-cell order take the regular path); kernels 1, 2, 4, 5, 6
 * and 7 need cell_subdiv 1.  group_width: the warp kernel takes a cell's particles
 * in chunks of this many lanes, the other 32 / group_width lane groups
 * splitting the candidates; 0 = the compiled-in default (16 for
 * cell_subdiv 1, 4 for 2), -1 = chosen per cell to minimise idle lanes, or
 * 2, 4, 8, 16, 32.  cells_per_grab: 0 = the warp kernel's warps take cells
 * by static striding, 1..1024 = they pull that many cells at a time from an
 * atomic work counter (a new context uses 4).  LJ_EINVAL for other values. */
int lj_set_tuning(lj_ctx *ctx, int32_t kernel, int32_t group_width, int32_t cells_per_grab);

/* ---------------------------------------------------------------------- */
/* Batched ensembles.  nrep independent periodic systems ("replicas") of
 * possibly different N and box, each the method above (Sections 2 and 3),
 * stored back to back: replica r owns particles [o_r, o_r + n[r]) of the
 * concatenated (sum n, 3) / (sum n, 4) arrays, o_r = n[0] + ... + n[r-1].
 * One velocity-Verlet step of every replica is ONE cooperative persistent
 * kernel launch (binning, scan, scatter and forces separated by bounded grid
 * barriers), captured once in a CUDA graph and replayed.  FP32-mixed only.
 * Batching is not in the paper; it serves many small systems at once.    */

typedef struct lj_batch lj_batch;

/* Create a batch: n[r] particles in a cubic box of side box[r] for
 * r < nrep; common supplies eps, sigma, rc, dt, mass, shift_mode, flags and
 * precision (must be LJ_PREC_MIXED); common->n and common->box are ignored.
 * Each replica is validated as by lj_grid.  common->cell_subdiv (0 or 1:
 * cells of side >= rc and the 27-cell stencil; 2: side >= rc / 2 and the
 * 125-cell stencil) applies to every replica, which then needs at least
 * 2k + 1 cells per side; other values give LJ_EINVAL.  stream: cudaStream_t
 * (NULL = legacy default stream; graph capture then uses a private
 * stream). */
int lj_batch_create(lj_batch **out, int32_t nrep, const int64_t *n, const double *box, const lj_params *common,
                    void *stream);
void lj_batch_destroy(lj_batch *b);

/* Totals and launch geometry: particles, cells, cooperative grid size and
 * staging capacity per warp.  Host only. */
int lj_batch_info(const lj_batch *b, int64_t *ntot, int64_t *ncell, int32_t *grid, int32_t *cap);

/* Tuning: cells a warp takes per pull from the work counter (1..1024),
 * whether steps are graph-replayed (1) or launched directly (0), and the
 * lane-group width of the warp kernel (0 or -1 = per cell, 2, 4, 8, 16, 32;
 * as in lj_set_tuning). */
int lj_batch_set_tuning(lj_batch *b, int32_t cells_per_grab, int32_t use_graph, int32_t group_width);

/* Force kernel of the batch's step launch: 3 = the 27-cell warp-per-cell
 * code (the default, and the only choice for cell subdivision 2), 7 = each
 * pair once over the half stencil (the pair-once device code of
 * lj_set_tuning kernel 7, with f zeroed in the scatter phase and the
 * reactions added with atomics; FP32 sums not bitwise reproducible between
 * runs; its 128 registers leave fewer resident warps for the other phases
 * of the launch).  LJ_EINVAL for other values, or 7 with subdivision 2.
 * Host only; a captured step graph is captured again. */
int lj_batch_set_kernel(lj_batch *b, int32_t kernel);

/* Forces of every replica at x into f (device arrays as above); with
 * energy != 0, f[:, 3] holds per-particle energies.  Asynchronous. */
int lj_batch_forces(lj_batch *b, const double *x, void *f, int32_t energy);

/* nsteps velocity-Verlet steps of every replica (as lj_step: f must hold
 * F(x) on entry and holds F at the final positions on return). */
int lj_batch_step(lj_batch *b, double *x, double *v, void *f, int32_t nsteps);

/* Per-replica energies into the HOST array out[3 * nrep]: (kinetic,
 * potential, total) of replica r at out[3r .. 3r+2]; f is overwritten with
 * forces and per-particle energies.  Synchronizes. */
int lj_batch_energy(lj_batch *b, const double *x, const double *v, void *f, double *out);

/* nsteps capped steepest-descent moves x += alpha F (the move of a particle
 * scaled down to length max_disp when longer), then wrapped; f holds F at
 * the final positions.  For relaxing random starting configurations. */
int lj_batch_relax(lj_batch *b, double *x, void *f, int32_t nsteps, double alpha, double max_disp);

/* Synchronize and return latched kernel errors (as lj_check). */
int lj_batch_check(lj_batch *b);

/* Kernel launches issued so far and whether steps are graph-replayed. */
int lj_batch_launches(const lj_batch *b, int64_t *launches, int32_t *graph);

/* Limits of lj_forces_static's fixed scratch buffer. */
#define LJ_STATIC_MAX_N 32768      /* particles */
#define LJ_STATIC_MAX_CELLS 32768  /* n_x^3, i.e. n_x <= 32 */

/* Forces without any device allocation.  The paper has no counterpart: this
 * is lj_forces for callers that cannot call cudaMalloc -- code that runs on
 * a fixed device-memory budget, inside another runtime's memory pool, or at
 * points where allocating (and the synchronization it can imply) is not
 * allowed.  It computes what lj_create + lj_forces(x, f, NULL, NULL) +
 * lj_destroy compute (same kernels, same precision modes), but needs no
 * context: the cell arrays and sorted positions live in one fixed buffer of
 * about 1.8 MB inside liblj.so, which every GPU that loads the library holds
 * until the process exits.  x (n, 3) double and f (n, 4) float or double are
 * caller-owned DEVICE arrays; p is validated as by lj_grid, and p->flags
 * must be 0 (the warp kernels; LJ_EINVAL otherwise).
 * Limits: p->n <= LJ_STATIC_MAX_N and n_x^3 <= LJ_STATIC_MAX_CELLS; larger
 * sizes return LJ_EOVERFLOW before any work is queued.
 * Set-up: every call looks up the buffer's device address on the current
 * device (a host-side lookup; it is not kept, so a cudaDeviceReset between
 * calls is safe).  The first call on a device, and the first after a reset,
 * loads the library's device code: make it before any stream capture.
 * All calls share the one buffer, which keeps the previous call's contents
 * (the call clears what must start at zero).  Calls whose work overlaps on
 * the GPU -- two streams, two host threads -- race on it: serialize them.
 * Work is queued on `stream` (a cudaStream_t, NULL = legacy default stream)
 * and not synchronized.  Errors the kernels find are not reported here:
 * a particle with a non-finite coordinate gets no force written, and the
 * binning's consistency check goes unread. */
int lj_forces_static(const lj_params *p, const double *x, void *f, void *stream);

/* Measured floating-point peak of the current device at its current clocks
 * (Section 1 compares the GPU's peak floating-point rate with a CPU's; the
 * roofline fractions divide by this measurement, not a datasheet figure).
 * kind 0: FP32 fused multiply-adds (fmaf), 1: FP32 packed pairs
 * (__ffma2_rn, two FMAs per instruction), 2: FP64 (fma).  Runs chains of
 * FMAs on every SM (8 CTAs of 256 threads per SM, 8 independent chains per
 * thread) on a private stream, lengthened until one launch takes >= 20 ms,
 * and returns the fastest of three timed launches: flop/s (an FMA counts 2)
 * in *flops_per_s, that launch's milliseconds in *ms and the SM count in
 * *sms (both optional).  Host pointers; synchronizes; allocates nothing on
 * the device.  LJ_EINVAL for another kind or a NULL flops_per_s. */
int lj_measure_peak(int32_t kind, double *flops_per_s, double *ms, int32_t *sms);

/* Enable (1) or disable (0) CUDA-event timing of the force kernel on the
 * context's stream; enabling resets the counters. */
int lj_set_timing(lj_ctx *ctx, int32_t enable);

/* Synchronize and read: total milliseconds spent in force-kernel launches
 * timed since timing was enabled, their number, and the number of kernels
 * this context has launched since creation.  Any pointer may be NULL. */
int lj_read_timing(lj_ctx *ctx, double *force_ms, int64_t *force_launches, int64_t *kernel_launches);

#ifdef __cplusplus
}
#endif

#endif /* LJ_H */
