// Internal declarations shared by the liblj.so translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lj.h"

// Particles with a non-finite coordinate are binned into one extra cell
// with id ncell, after the grid: no stencil visits it, so they cannot pile
// into a real cell and make its force work quadratic.  count[] and start[]
// hold ncell + 1 and ncell + 2 entries.
//
// Error bits latched in device memory by kernels, mapped to lj_status by
// lj_check.
enum : int32_t {
    LJ_ERRBIT_NONFINITE = 1,
    LJ_ERRBIT_TIMEOUT = 2,
    LJ_ERRBIT_SCAN = 4,
    LJ_ERRBIT_OVERFLOW = 8,   // a cell held more particles than the AOP capacity
};

// Force-kernel geometry: a work item is a run of up to kRunMax consecutive
// cells along x in one (y, z) row of cells; one consumer warp per home cell.
constexpr int kRunMax = 8;
constexpr int kWinMax = kRunMax + 2;           // window cells per row
constexpr int kTabMax = 9 * kWinMax;           // 9 neighbour rows
constexpr int kConsumerWarps = kRunMax;
constexpr int kForceThreads = (kConsumerWarps + 1) * 32;  // + 1 producer warp

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kReduceThreads = 256;

constexpr int kWarpForceThreads = 256;         // warp-per-cell force kernel

struct lj_ctx {
    lj_params p;
    int nc;              // cells per side
    int64_t ncell;       // nc^3
    double inv_cw;       // s = nc / L (cell index scale)
    float inv_nc_f;      // 1 / nc for lj_cell_decode (0 for grids of 2^24 cells or more)
    double cw;           // cell side L / nc
    cudaStream_t stream;
    int device;
    int nsm;

    // device scratch
    int32_t *cell_of, *rank, *count, *start, *perm;
    void *pos;           // float4 or double4_16a [n], sorted, cell-centred coordinates
    double *centre;      // [nc] cell-centre coordinate (k + 1/2) L / nc
    long long *thb;      // [nc + 1] bits of the cell thresholds (lj_cell_from_guess)
    double wrap_hi, wrap_lo;  // lj_wrap_fast bounds
    int32_t *tile_sum;
    int ntiles;
    // single-pass scan: per-tile status words and [ticket, done, epoch]
    // (NULL: the two-launch scan, as for contexts without them)
    unsigned long long *scan_status;
    unsigned *scan_ctl;
    double *partial;     // force-kernel per-block (energy, virial) partials
    double *ekin_partial;
    double *scalars;     // 8 doubles: [0] = E_pot, [1] = virial, [2] = E_kin, [3] = E_tot, [4] = T, [5] = P
    int32_t *err;
    double *host_scalars;   // pinned, 8 doubles
    int32_t *host_err;      // pinned

    // force kernel configuration: run-staged kernel (lj_force.cu) ...
    int run_len, runs, nitems, cap, force_grid, force_smem, use_tma, use_run_kernel;
    // ... and warp-per-cell kernel (lj_force_warp.cu, FP32-mixed)
    int wcap, wforce_smem, wforce_grid;
    int gw;              // tuning: lane-group width of the warp kernel (0 compiled default, -1 per cell)
    // pipelined warp kernel (lj_force_pipe.cu): slice capacities, launch shape
    int pcap, praw, pipe_smem, pipe_grid;
    int pipe;            // tuning: 1 = warp kernel with bulk-copied stencils (kernel 5)
    // Newton's-third-law kernels (tuning kernel 7; FP32-mixed: lj_force_n3.cu,
    // the default for cell subdivision 1; FP64: the pair-once form of
    // lj_force_w64.cu, whose sums go to f_sorted in cell order, n x 32 B):
    // slice capacity, launch shape
    int n3, n3cap, n3_smem, n3_grid;
    void *f_sorted;
    int fuse_update;     // warp kernel applies the velocity-Verlet update (lj_step)
    int grab;            // tuning: cells per work pull in the warp kernel (0 = static)
    int w64_lcap;        // FP64 warp kernel: list entries per warp
    int use_pers;        // tuning kernel 6: lj_step through a one-replica persistent batch
    lj_batch *pers;      // created by the first such step
    int pers_gen;        // tuning generation last applied to it
    unsigned *work;      // work counter of the warp kernel, zeroed by k_scan_tiles
    int npartial;        // partials written by the last energy launch
    int npartial_cap;    // capacity of `partial` in (energy, virial) pairs
    void *g4;            // sorted cotangents for the adjoint (lazily allocated)
    void *n2_scratch;    // all-pairs kernel scratch (lazily allocated)
    void *aop;           // fixed-capacity cell arrays of the AOP kernel (lazily allocated)
    size_t aop_bytes;
    int use_aop;         // tuning: force kernel 4 (AOP layout)
    uint64_t *r48_state; // Langevin thermostat: one rand48 stream per particle (lazily allocated)
    // cell lists with a skin (lj_set_skin): 0 = rebuilt every step
    double skin;
    int skin_max_interval;
    float4 *disp;        // displacement of each particle since the last rebuild (FP32)
    int32_t *skin_flags; // [0] max |disp|^2 (float bits), [1] rebuild now, [2] steps since rebuild
    long long *skin_counts;  // [0] rebuilds, [1] steps (skin mode)
    int skin_dirty;      // the grid changed: the next step rebuilds unconditionally
    // deterministic order inside the cells (lj_set_deterministic): a sorted
    // copy goes to the spare buffers, which then swap with pos / perm
    int deterministic;
    void *pos_alt;
    int32_t *perm_alt;
    // lj_step_host: the copy of x back overlaps the last force evaluation;
    // the copies in arrive in 4 parts, each kicked, drifted and binned as
    // soon as it is there (kdb_done: step 0's update is done)
    cudaStream_t copy_stream;
    cudaEvent_t ev_xfinal, ev_entry;
    cudaEvent_t ev_chunk[4];
    int kdb_done;
    // lj_step: the zeroing of f that the pair-once kernel needs runs on
    // zero_stream, concurrently with the scan and the scatter (f is dead
    // once the update has read it); f_prezeroed tells launch_force_n3 that
    // it is done
    cudaStream_t zero_stream;
    cudaEvent_t ev_zfork, ev_zjoin;
    int f_prezeroed;
    // graph replay of the middle steps of lj_step (lj_set_graph)
    int use_graph;
    cudaGraphExec_t gexec;   // one captured middle step
    const void *gx, *gv, *gf;
    int gen, ggen;       // configuration generation; the one captured
    int64_t glaunches;   // kernel launches in one captured step
    size_t n2_bytes;
    int ekin_grid;

    // lazily allocated staging for lj_step_host / lj_energy
    double *xs, *vs;
    void *fs;

    // timing
    int timing;
    cudaEvent_t *ev;
    int nev, ev_used;
    double force_ms;
    int64_t force_launches;
    int64_t kernel_launches;
};

// ---------------------------------------------------------------- device --

// Wrap one coordinate into [0, L): w = x - L floor(x / L), then w >= L folds
// to w - L.  Every operation is separately rounded (no contraction) so that
// the cell assignment is reproducible bit for bit.
__device__ __forceinline__ double lj_wrap(double x, double L)
{
    double q = floor(__ddiv_rn(x, L));
    double w = __dsub_rn(x, __dmul_rn(L, q));
    if (w >= L) w = __dsub_rn(w, L);
    return w;
}

// lj_wrap without the division in the common cases: for x in [0, L - L/2^50)
// the quotient floor(x / L) is exactly 0, in [L + L/2^50, 2L - L/2^49) it is
// exactly 1 and in (-L + L/2^50, -L/2^50] exactly -1, so the result is bit
// for bit that of lj_wrap; other inputs take lj_wrap itself.  The first test
// runs on the integer pipe (non-negative doubles order like their bits).
// hi = L (1 - 2^-50), lo = L 2^-50.
__device__ __forceinline__ double lj_wrap_fast(double x, double L, double hi, double lo)
{
    const long long b = __double_as_longlong(x);
    if (b >= 0 && b < __double_as_longlong(hi)) return x;
    double q;
    if (x >= L + lo && x < 2.0 * L - 2.0 * lo) q = 1.0;
    else if (x <= -lo && x > -hi) q = -1.0;
    else return lj_wrap(x, L);
    double w = __dsub_rn(x, __dmul_rn(L, q));
    if (w >= L) w = __dsub_rn(w, L);
    return w;
}

// Cell coordinate trunc(w * s), clamped to [0, nc - 1].
__device__ __forceinline__ int lj_cell1(double w, double s, int nc)
{
    int c = __double2int_rz(__dmul_rn(w, s));
    c = c < nc ? c : nc - 1;
    c = c > 0 ? c : 0;
    return c;
}

// Cell coordinates (c mod n, (c / n) mod n, c / n^2) of a linear cell id.
// For grids of fewer than 2^24 cells inv_n = 1/n in FP32 gives the quotient
// of c < 2^24 to within one (relative error < 2^-22), fixed by one
// comparison; inv_n = 0 selects integer division.
__device__ __forceinline__ int lj_div_small(int c, int n, float inv_n, int &r)
{
    int q = __float2int_rz((float)c * inv_n);
    r = c - q * n;
    if (r < 0) {
        q -= 1;
        r += n;
    } else if (r >= n) {
        q += 1;
        r -= n;
    }
    return q;
}

__device__ __forceinline__ void lj_cell_decode(int c, int nc, float inv_nc, int &cx, int &cy, int &cz)
{
    if (inv_nc > 0.0f) {
        const int q = lj_div_small(c, nc, inv_nc, cx);
        cz = lj_div_small(q, nc, inv_nc, cy);
    } else {
        cx = c % nc;
        cy = (c / nc) % nc;
        cz = c / (nc * nc);
    }
}

// Rank of a particle within its cell by one atomicAdd per distinct cell in
// the warp: lanes holding the same cell id are grouped with match.any, the
// lowest lane adds the group size, and ranks follow lane order inside the
// group.  All 32 lanes must call it (valid = false lanes get no rank).
__device__ __forceinline__ int lj_warp_rank(int32_t *count, int c, bool valid)
{
    const unsigned key = valid ? (unsigned)c : 0xffffffffu;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(count + c, __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

// Stencil of radius R (cell subdivision k = R, Section 3): W^3 cells with
// W = 2R + 1.  Entry 0 is the home cell, entries 1 .. NS-1 the neighbours in
// x-fastest order with the centre skipped.
template <int R>
struct Stencil {
    static constexpr int W = 2 * R + 1;
    static constexpr int NS = W * W * W;
    static constexpr int P2 = NS <= 32 ? 32 : (NS <= 64 ? 64 : 128);   // power of two >= NS
};

template <int R>
__device__ __forceinline__ void stencil_delta(int k, int &dx, int &dy, int &dz)
{
    constexpr int W = Stencil<R>::W, C = Stencil<R>::NS / 2;
    const int idx = k == 0 ? C : (k <= C ? k - 1 : k);
    dx = idx % W - R;
    dy = (idx / W) % W - R;
    dz = idx / (W * W) - R;
}

// Exact cell coordinate of a wrapped w from a guess g: thb[k] holds the bits
// of the smallest double t with trunc(t * s) >= k (thb[0] = 0, thb[nc] =
// INT64_MAX), so the cell is the largest k with w >= t_k -- the same value
// lj_cell1 returns.  Checks g - 1, g, g + 1 with integer compares and falls
// back to lj_cell1 when the guess is further off.
__device__ __forceinline__ int lj_cell_from_guess(double w, int g, const long long *__restrict__ thb, double s,
                                                  int nc)
{
    long long b = __double_as_longlong(w);
    b = b < 0 ? 0 : b;                  // -0 and negative values bin like 0
    g = g < 0 ? 0 : (g >= nc ? nc - 1 : g);
    if (b < __ldg(thb + g)) {
        g -= 1;
        if (g < 0 || b < __ldg(thb + g)) return lj_cell1(w, s, nc);
    } else if (b >= __ldg(thb + g + 1)) {
        g += 1;
        if (g >= nc || b >= __ldg(thb + g + 1)) return lj_cell1(w, s, nc);
    }
    return g;
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_16a; };

// ------------------------------------------------------------------ host --

// Kernel launchers (each returns cudaGetLastError()).
// gated: skin mode, run only when the device-side rebuild flag is set
cudaError_t launch_bin_count(lj_ctx *c, const double *x, bool gated = false);
cudaError_t launch_scan(lj_ctx *c, bool gated = false);
cudaError_t launch_scatter(lj_ctx *c, const double *x, bool wrap);
cudaError_t launch_force(lj_ctx *c, void *f, bool energy);
cudaError_t launch_energy_reduce(lj_ctx *c);
// Particles [i_begin, i_end) (i_end < 0: to n).
cudaError_t launch_kick_drift_bin(lj_ctx *c, double *x, double *v, const void *f, int nkick, int64_t i_begin = 0,
                                  int64_t i_end = -1);
cudaError_t launch_kick(lj_ctx *c, double *v, const void *f);
// Skin mode: kick + drift + displacement tracking, then the rebuild decision.
cudaError_t launch_kick_drift_skin(lj_ctx *c, double *x, double *v, const void *f, int nkick);
cudaError_t launch_ekin(lj_ctx *c, const double *v);
// Temperature and virial pressure from scalars[0..2] into scalars[3..5].
cudaError_t launch_observables(lj_ctx *c);
cudaError_t launch_counts_from_start(lj_ctx *c, int32_t *count);
cudaError_t force_configure(lj_ctx *c);
// Allow kernel `kern` at least `bytes` of dynamic shared memory.  The limit
// is a property of the function, shared by every context in the process, so
// it is only ever raised: a context configured later with smaller slices
// must not lower it under one configured earlier.
inline cudaError_t raise_dyn_smem(const void *kern, int bytes)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kern);
    if (e != cudaSuccess) return e;
    if (a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// LJ_OK if ptr is device (or managed) memory aligned to `align` bytes, else
// LJ_EINVAL (lj_api.cu).
int check_dev_ptr(const void *ptr, size_t align);

cudaError_t warp_force_configure(lj_ctx *c);
// Staged-candidate capacity per warp of the warp kernels (lj_force_warp.cu).
int warp_stencil_cap(double mean_occupancy, int subdiv, int threads, int static_bytes);
cudaError_t launch_vjp(lj_ctx *c, const double *g, double scale, double *dx, double *dparam);
cudaError_t launch_axpy(lj_ctx *c, double *y, const double *x, double a);
cudaError_t launch_force_warp(lj_ctx *c, void *f, bool energy);
// FP64 warp kernel with compacted pair lists (lj_force_w64.cu); it uses the
// warp kernel's slice capacity, shared memory and grid fields.
cudaError_t w64_force_configure(lj_ctx *c);
cudaError_t launch_force_w64(lj_ctx *c, void *f, bool energy);
// Its VJP form (FP64 contexts): dx += scale J g over the sorted cotangents
// c->g4; per-CTA parameter sums into c->partial, *grid_out of them.
// a1, b1, fc1, dfc1: the eps = 1 coefficients of the VJP (lj_adjoint.cu).
cudaError_t launch_vjp_w64(lj_ctx *c, double scale, double *dx, double a1, double b1, double fc1, double dfc1,
                           int *grid_out);
// Pipelined warp kernel (lj_force_pipe.cu): configuration and launch.
cudaError_t pipe_force_configure(lj_ctx *c);
cudaError_t launch_force_pipe(lj_ctx *c, void *f, bool energy);
// rand48 streams and the Langevin update (lj_rand48.cu).
cudaError_t launch_r48_seed(uint64_t *state, int64_t S, uint64_t x0, cudaStream_t stream);
cudaError_t launch_langevin_bin(lj_ctx *c, double *x, double *v, const void *f, int nkick, double gamma, double kT);

// One bounded mbarrier wait that cannot complete (lj_force.cu).
cudaError_t launch_wait_selftest(lj_ctx *c);

// Forces with the paper's fixed-capacity cell arrays (lj_force_aop.cu).
cudaError_t launch_force_aop(lj_ctx *c, void *f, bool energy);

// All-pairs forces (lj_n2.cu); energies into c->scalars[0..1] when energy.
cudaError_t launch_forces_n2(lj_ctx *c, const double *x, void *f, bool energy);
cudaError_t launch_force_warp_fused(lj_ctx *c, void *f, double *x, double *v, bool last);
// Newton's-third-law warp kernel (lj_force_n3.cu): configuration, and a
// launch that zeroes f and adds every pair's force to both particles.
cudaError_t n3_force_configure(lj_ctx *c);
bool uses_force_n3(const lj_ctx *c);   // launch_force dispatches to the pair-once kernel
// The pair-once FP32-mixed VJP (lj_vjp_n3.cu), used where the pair-once
// force kernel is: coef = (rc^2, 48 sigma^12, 24 sigma^6, F(rc) rc at
// eps = 1, its sigma-derivative, eps, 1 / sigma); sums into acc (float4
// [n], zeroed there), parameter partials into c->partial (*grid_out).
bool uses_vjp_n3(const lj_ctx *c);
cudaError_t launch_vjp_n3(lj_ctx *c, const double *coef, double scale, double *dx, float4 *acc, int *grid_out);
cudaError_t launch_force_n3(lj_ctx *c, void *f, bool energy);
