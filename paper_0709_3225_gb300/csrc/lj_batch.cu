// Batched ensembles: many independent periodic LJ systems (replicas) of
// uneven size advanced together.  Each replica is the method of the paper
// (Section 3 cell lists, Section 2 force and velocity Verlet); the batch
// concatenates their particles and cells so that one persistent launch per
// step covers all of them.
//
// One step is one cooperative launch of k_batch_step (captured once in a
// CUDA graph and replayed), whose phases are separated by grid barriers:
//   1. kick, drift, wrap, cell id and rank   (every particle)
//   2. scan of the per-cell counts            (tiles of 4096 cells)
//   3. scatter to cell-sorted, cell-centred FP32 positions
//   4. forces: warps pull chunks of cells from an atomic work counter and
//      run the warp-per-cell code of lj_force_cell.cuh with each replica's
//      own grid (n_x, cell side, cell offset).
// Barriers are counted with bounded waits: a wait that exceeds ~2 s of SM
// clock latches LJ_ETIMEOUT and the block leaves the kernel, so a fault in
// the bookkeeping ends the launch instead of hanging the GPU.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "lj_force_cell.cuh"
#include "lj_force_n3.cuh"

namespace {

constexpr int kBatchThreads = kWarpForceThreads;

struct BatchDev {
    int64_t ntot, ncell;
    int nrep, ntiles, cells_per_grab;
    double h, dt, mass;
    const int32_t *poff, *coff, *ncs, *thoff, *ceoff, *rep_of, *rep_of_cell;
    const double *L, *s, *cw, *whi, *wlo, *centre;
    const long long *thb;
    int32_t *cell_of, *rank, *count, *start, *tile_sum, *err;
    float4 *pos;
    unsigned *bar_count, *bar_gen, *work;
    unsigned char *first;
};

// Grid barrier for a cooperative launch.  Thread 0 of each block reads the
// generation, publishes its block's writes, arrives; the last arrival resets
// the counter and bumps the generation; the others wait for the bump with a
// bound on the wait.  Returns false (error latched) if the wait timed out.
__device__ __forceinline__ bool grid_barrier(const BatchDev &b)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *gen = b.bar_gen;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(b.bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(b.bar_count, 0u);
            __threadfence();
            atomicAdd(b.bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > (1ll << 32)) {
                    atomicOr(b.err, LJ_ERRBIT_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ void decode_cell(int local, int nc, int &cx, int &cy, int &cz)
{
    cx = local % nc;
    cy = (local / nc) % nc;
    cz = local / (nc * nc);
}

// Phase 1.  op 0: velocity-Verlet kick + drift from the previous step's
// forces, then bin; op 1: bin the given positions (general wrap).
__device__ void phase_bin(const BatchDev &b, int op, double *__restrict__ x, double *__restrict__ v,
                          const float4 *__restrict__ f)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double hk = (b.first[0] ? 1.0 : 2.0) * b.h;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < b.ntot; base += stride) {
        const int64_t i = base + lane;
        const bool valid = i < b.ntot;
        int gc = 0;
        if (valid) {
            const int r = b.rep_of[i];
            const double L = b.L[r], whi = b.whi[r], wlo = b.wlo[r], s = b.s[r];
            const int nc = b.ncs[r];
            double px, py, pz;
            int cx, cy, cz;
            if (op == 0) {
                const float4 q = f[i];
                const double vx = __fma_rn(hk, (double)q.x, v[3 * i]);
                const double vy = __fma_rn(hk, (double)q.y, v[3 * i + 1]);
                const double vz = __fma_rn(hk, (double)q.z, v[3 * i + 2]);
                px = lj_wrap_fast(__fma_rn(b.dt, vx, x[3 * i]), L, whi, wlo);
                py = lj_wrap_fast(__fma_rn(b.dt, vy, x[3 * i + 1]), L, whi, wlo);
                pz = lj_wrap_fast(__fma_rn(b.dt, vz, x[3 * i + 2]), L, whi, wlo);
                v[3 * i] = vx;
                v[3 * i + 1] = vy;
                v[3 * i + 2] = vz;
                x[3 * i] = px;
                x[3 * i + 1] = py;
                x[3 * i + 2] = pz;
                const long long *thb = b.thb + b.thoff[r];
                int ox, oy, oz;
                decode_cell(b.cell_of[i] - b.coff[r], nc, ox, oy, oz);
                cx = lj_cell_from_guess(px, ox, thb, s, nc);
                cy = lj_cell_from_guess(py, oy, thb, s, nc);
                cz = lj_cell_from_guess(pz, oz, thb, s, nc);
            } else {
                px = lj_wrap_fast(x[3 * i], L, whi, wlo);
                py = lj_wrap_fast(x[3 * i + 1], L, whi, wlo);
                pz = lj_wrap_fast(x[3 * i + 2], L, whi, wlo);
                cx = lj_cell1(px, s, nc);
                cy = lj_cell1(py, s, nc);
                cz = lj_cell1(pz, s, nc);
            }
            if (isfinite(px) && isfinite(py) && isfinite(pz)) {
                gc = b.coff[r] + cx + nc * (cy + nc * cz);
            } else {   // the extra cell after all replicas' grids
                atomicOr(b.err, LJ_ERRBIT_NONFINITE);
                gc = (int)b.ncell;
            }
        }
        const int rk = lj_warp_rank(b.count, gc, valid);
        if (valid) {
            b.cell_of[i] = gc;
            b.rank[i] = rk;
        }
    }
}

// Phase 2a: sum of each tile of counts.
__device__ void phase_tiles(const BatchDev &b)
{
    __shared__ int32_t wsum[kBatchThreads / 32];
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        int32_t acc = 0;
        for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
            const int64_t e = (int64_t)t * kScanTile + k;
            if (e <= b.ncell) acc += b.count[e];
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t s = 0;
            for (int w = 0; w < kBatchThreads / 32; w++) s += wsum[w];
            b.tile_sum[t] = s;
        }
        __syncthreads();
    }
}

// Phase 2b: exclusive scan of each tile with the sum of the earlier tiles;
// counts are reset; the last tile writes start[ncell].
__device__ void phase_scan(const BatchDev &b)
{
    constexpr int items = kScanTile / kBatchThreads;
    __shared__ int32_t wtot[kBatchThreads / 32];
    __shared__ int32_t sp;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
        int32_t pre = 0;
        for (int q = threadIdx.x; q < t; q += blockDim.x) pre += b.tile_sum[q];
        for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
        if (lane == 0) wtot[wid] = pre;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t s = 0;
            for (int w = 0; w < kBatchThreads / 32; w++) s += wtot[w];
            sp = s;
        }
        __syncthreads();
        const int32_t tile_pre = sp;
        const int64_t base = (int64_t)t * kScanTile + (int64_t)threadIdx.x * items;
        int32_t vals[items];
        int32_t local = 0;
#pragma unroll
        for (int k = 0; k < items; k++) {
            const int64_t e = base + k;
            vals[k] = e <= b.ncell ? b.count[e] : 0;
            local += vals[k];
        }
        int32_t incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __syncthreads();
        if (lane == 31) wtot[wid] = incl;
        __syncthreads();
        int32_t wpre = 0;
        for (int w = 0; w < wid; w++) wpre += wtot[w];
        int32_t run = tile_pre + wpre + incl - local;
#pragma unroll
        for (int k = 0; k < items; k++) {
            const int64_t e = base + k;
            if (e <= b.ncell) {
                b.start[e] = run;
                b.count[e] = 0;
            }
            run += vals[k];
        }
        if (t == b.ntiles - 1 && threadIdx.x == blockDim.x - 1) {
            b.start[b.ncell + 1] = run;
            if ((int64_t)run != b.ntot) atomicOr(b.err, LJ_ERRBIT_SCAN);
        }
        __syncthreads();
    }
}

// Phase 3: sorted, cell-centred FP32 positions (w = particle index).  With
// fz (the pair-once force phase, which adds into f) f is zeroed too; the
// first phase has read it already.  Two particles per thread, their loads
// issued before either is stored: the launch runs at the force phase's
// occupancy, so this memory phase needs the extra loads in flight.
__device__ __forceinline__ void scatter_one(const BatchDev &b, int op, int64_t i, int r, int c, int rk, double px,
                                            double py, double pz)
{
    if (c >= b.ncell) {   // non-finite particle in the extra cell
        b.pos[b.start[c] + rk] = make_float4((float)px, (float)px, (float)px, __int_as_float((int)i));
        return;
    }
    const int nc = b.ncs[r];
    int cx, cy, cz;
    decode_cell(c - b.coff[r], nc, cx, cy, cz);
    if (op != 0) {
        const double L = b.L[r], whi = b.whi[r], wlo = b.wlo[r];
        px = lj_wrap_fast(px, L, whi, wlo);
        py = lj_wrap_fast(py, L, whi, wlo);
        pz = lj_wrap_fast(pz, L, whi, wlo);
    }
    const double *ce = b.centre + b.ceoff[r];
    b.pos[b.start[c] + rk] =
        make_float4((float)(px - ce[cx]), (float)(py - ce[cy]), (float)(pz - ce[cz]), __int_as_float((int)i));
}

__device__ void phase_scatter(const BatchDev &b, int op, const double *__restrict__ x, float4 *__restrict__ fz)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < b.ntot; i0 += 2 * stride) {
        const int64_t i1 = i0 + stride;
        const bool two = i1 < b.ntot;
        const int r0 = b.rep_of[i0], c0 = b.cell_of[i0], k0 = b.rank[i0];
        const double x0 = x[3 * i0], y0 = x[3 * i0 + 1], z0 = x[3 * i0 + 2];
        int r1 = 0, c1 = 0, k1 = 0;
        double x1 = 0.0, y1 = 0.0, z1 = 0.0;
        if (two) {
            r1 = b.rep_of[i1];
            c1 = b.cell_of[i1];
            k1 = b.rank[i1];
            x1 = x[3 * i1];
            y1 = x[3 * i1 + 1];
            z1 = x[3 * i1 + 2];
        }
        if (fz) {
            fz[i0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (two) fz[i1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        scatter_one(b, op, i0, r0, c0, k0, x0, y0, z0);
        if (two) scatter_one(b, op, i1, r1, c1, k1, x1, y1, z1);
    }
}

// Phase 4: forces, cells pulled in chunks from the work counter.  R: the
// stencil radius, the cell subdivision k of every replica's grid (1: the
// 27-cell stencil of cells >= rc; 2: 125 cells of side >= rc / 2).
template <int R, int MODE, bool ENERGY, int GFIX>
__device__ void phase_force(const BatchDev &b, const WarpParams &k, float4 *__restrict__ f)
{
    extern __shared__ __align__(16) float bsmem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *slice = bsmem + (size_t)warp * warp_slice_words(k.cap, R);
    double eacc = 0.0, wacc = 0.0;
    for (;;) {
        unsigned c0 = 0;
        if (lane == 0) c0 = atomicAdd(b.work, (unsigned)b.cells_per_grab);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if ((int64_t)c0 >= b.ncell) break;
        const int64_t c1 = min((int64_t)c0 + b.cells_per_grab, b.ncell);
        for (int64_t c = c0; c < c1; c++) {
            const int r = b.rep_of_cell[c];
            const int nc = b.ncs[r];
            int cx, cy, cz;
            decode_cell((int)(c - b.coff[r]), nc, cx, cy, cz);
            const StoreForce<MODE, ENERGY> out{f, k.n};
            process_home_cell<R, MODE, ENERGY, false, GFIX>(k, b.pos, b.start, out, slice, cx, cy, cz, nc, b.coff[r],
                                                      (float)b.cw[r], eacc, wacc);
        }
    }
}

// GFIX as in k_force_warp: the default width compiled in (group width 0:
// 16 for the 27-cell stencil, 4 for the 125-cell one), 0 general.
template <int R, int MODE, bool ENERGY, int GFIX>
__global__ void __launch_bounds__(kBatchThreads, 4) k_batch_step(BatchDev b, WarpParams k, int op, double *x,
                                                                  double *v, float4 *f)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *b.work = 0u;
    phase_bin(b, op, x, v, f);
    if (!grid_barrier(b)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) b.first[0] = 0;
    phase_tiles(b);
    if (!grid_barrier(b)) return;
    phase_scan(b);
    if (!grid_barrier(b)) return;
    phase_scatter(b, op, x, nullptr);
    if (!grid_barrier(b)) return;
    phase_force<R, MODE, ENERGY, GFIX>(b, k, f);
}

// Phase 4 with each pair once: the single-system pair-once kernel's device
// code (lj_force_n3.cuh, coherent loads: the positions and starts were
// written by earlier phases of this launch) on each replica's grid.
template <int MODE, bool ENERGY>
__device__ void phase_force_n3(const BatchDev &b, const WarpParams &k, float4 *__restrict__ f)
{
    extern __shared__ __align__(16) float bsmem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float4 *S = reinterpret_cast<float4 *>(bsmem + (size_t)warp * n3_slice_words(k.cap));
    float4 *stab = S + k.cap;
    int *spre = reinterpret_cast<int *>(stab + kN3Half);
    float4 *H = reinterpret_cast<float4 *>(spre + 16);
    double eacc = 0.0, wacc = 0.0;
    auto load = [&](int c) {
        const int r = b.rep_of_cell[c];
        const int nc = b.ncs[r];
        return half_load<false>(b.start, c - b.coff[r], nc, 1.0f / (float)nc, b.coff[r]);
    };
    // pulls of cells_per_grab cells, single cells over the last stretch (as
    // k_force_n3)
    const int64_t tail = 2 * (int64_t)b.cells_per_grab * gridDim.x * (kBatchThreads / 32);
    unsigned last = 0;
    for (;;) {
        const unsigned gr = (int64_t)last + tail >= b.ncell ? 1u : (unsigned)b.cells_per_grab;
        unsigned c0 = 0;
        if (lane == 0) c0 = atomicAdd(b.work, gr);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if ((int64_t)c0 >= b.ncell) break;
        last = c0;
        const int c1 = (int)min((int64_t)c0 + gr, b.ncell);
        HalfLoad nxt = load((int)c0);   // the next cell's table loads before this cell's work
        for (int c = (int)c0; c < c1; c++) {
            const HalfLoad cur = nxt;
            if (c + 1 < c1) nxt = load(c + 1);
            n3_cell<MODE, ENERGY, false>(k, b.pos, f, cur, (float)b.cw[b.rep_of_cell[c]], S, stab, spre, H, eacc,
                                         wacc);
        }
    }
}

// One step with the pair-once force phase (cell subdivision 1): the force
// phase reads the home positions from shared memory, which keeps the
// kernel at 80 registers, so 3 blocks of 256 threads per SM (24 warps).
template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kBatchThreads, 3) k_batch_step_n3(BatchDev b, WarpParams k, int op, double *x,
                                                                     double *v, float4 *f)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *b.work = 0u;
    phase_bin(b, op, x, v, f);
    if (!grid_barrier(b)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) b.first[0] = 0;
    phase_tiles(b);
    if (!grid_barrier(b)) return;
    phase_scan(b);
    if (!grid_barrier(b)) return;
    phase_scatter(b, op, x, f);
    if (!grid_barrier(b)) return;
    phase_force_n3<MODE, ENERGY>(b, k, f);
}

// Closing half kick of the last step: v += h f.
__global__ void k_batch_kick(double *__restrict__ v, const float4 *__restrict__ f, int64_t n, double h)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 q = f[i];
    v[3 * i] = __fma_rn(h, (double)q.x, v[3 * i]);
    v[3 * i + 1] = __fma_rn(h, (double)q.y, v[3 * i + 1]);
    v[3 * i + 2] = __fma_rn(h, (double)q.z, v[3 * i + 2]);
}

// Capped steepest-descent move: d = alpha f, scaled down to |d| <= dmax,
// then wrapped into the replica's box.
__global__ void k_batch_sd(double *__restrict__ x, const float4 *__restrict__ f, int64_t n,
                           const int32_t *__restrict__ rep_of, const double *__restrict__ Ls,
                           const double *__restrict__ whis, const double *__restrict__ wlos, double alpha,
                           double dmax)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 q = f[i];
    double dx = alpha * q.x, dy = alpha * q.y, dz = alpha * q.z;
    const double d = sqrt(dx * dx + dy * dy + dz * dz);
    if (d > dmax) {
        const double sc = dmax / d;
        dx *= sc;
        dy *= sc;
        dz *= sc;
    }
    const int r = rep_of[i];
    const double L = Ls[r], whi = whis[r], wlo = wlos[r];
    x[3 * i] = lj_wrap_fast(x[3 * i] + dx, L, whi, wlo);
    x[3 * i + 1] = lj_wrap_fast(x[3 * i + 1] + dy, L, whi, wlo);
    x[3 * i + 2] = lj_wrap_fast(x[3 * i + 2] + dz, L, whi, wlo);
}

// Per-replica (kinetic, potential, total) energy: block r sums its range.
__global__ void __launch_bounds__(kReduceThreads) k_batch_energy(const double *__restrict__ v,
                                                                 const float4 *__restrict__ f,
                                                                 const int32_t *__restrict__ poff, double mass,
                                                                 double *__restrict__ out)
{
    __shared__ double sk[kReduceThreads], su[kReduceThreads];
    const int r = blockIdx.x;
    double ek = 0.0, eu = 0.0;
    for (int64_t i = poff[r] + threadIdx.x; i < poff[r + 1]; i += kReduceThreads) {
        ek += v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
        eu += (double)f[i].w;
    }
    sk[threadIdx.x] = ek;
    su[threadIdx.x] = eu;
    __syncthreads();
    for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sk[threadIdx.x] += sk[threadIdx.x + w];
            su[threadIdx.x] += su[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[3 * r] = 0.5 * mass * sk[0];
        out[3 * r + 1] = su[0];
        out[3 * r + 2] = out[3 * r] + su[0];
    }
}

template <int R, int G>
void *batch_kernel_g(int mode, bool energy)
{
    switch (mode * 2 + (energy ? 1 : 0)) {
        case 0: return (void *)k_batch_step<R, 0, false, G>;
        case 1: return (void *)k_batch_step<R, 0, true, G>;
        case 2: return (void *)k_batch_step<R, 1, false, G>;
        case 3: return (void *)k_batch_step<R, 1, true, G>;
        case 4: return (void *)k_batch_step<R, 2, false, G>;
        default: return (void *)k_batch_step<R, 2, true, G>;
    }
}

void *batch_kernel_n3(int mode, bool energy)
{
    switch (mode * 2 + (energy ? 1 : 0)) {
        case 0: return (void *)k_batch_step_n3<0, false>;
        case 1: return (void *)k_batch_step_n3<0, true>;
        case 2: return (void *)k_batch_step_n3<1, false>;
        case 3: return (void *)k_batch_step_n3<1, true>;
        case 4: return (void *)k_batch_step_n3<2, false>;
        default: return (void *)k_batch_step_n3<2, true>;
    }
}

void *batch_kernel(int subdiv, int mode, bool energy, int gw)
{
    if (subdiv == 2)
        return gw == 0 ? batch_kernel_g<2, DefaultGroup<2>::value>(mode, energy) : batch_kernel_g<2, 0>(mode, energy);
    return gw == 0 ? batch_kernel_g<1, DefaultGroup<1>::value>(mode, energy) : batch_kernel_g<1, 0>(mode, energy);
}

// Same threshold construction as lj_create (smallest t with t * s >= k).
double threshold(int k, double s)
{
    double t = (double)k / s;
    while (t > 0.0 && nextafter(t, 0.0) * s >= (double)k) t = nextafter(t, 0.0);
    while (!(t * s >= (double)k)) t = nextafter(t, INFINITY);
    return t;
}

int map_err(cudaError_t e) { return e == cudaErrorMemoryAllocation ? LJ_ENOMEM : LJ_ECUDA; }

int check_ptr(const void *ptr, size_t align)
{
    if (!ptr || ((uintptr_t)ptr) % align != 0) return LJ_EINVAL;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return LJ_EINVAL;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? LJ_OK : LJ_EINVAL;
}

}  // namespace

struct lj_batch {
    lj_params p;
    int nrep;
    int64_t ntot, ncell;
    cudaStream_t stream;
    int device, nsm;
    std::vector<void *> allocs;
    BatchDev d;
    WarpParams k;
    int grid, smem, use_graph;
    // the pair-once step kernel (cell subdivision 1): its parameters (k with
    // its own staging capacity), grid and shared memory; n3: it is selected
    WarpParams kn3;
    int grid_n3, smem_n3, n3;
    double max_mean_occ;
    double *rep_out, *host_out;
    int32_t *host_err;
    cudaGraphExec_t gexec;
    const void *gx, *gv, *gf;
    int64_t launches;
};

namespace {

template <typename T>
cudaError_t balloc(lj_batch *b, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e == cudaSuccess) b->allocs.push_back(q);
    *p = (T *)q;
    return e;
}

void batch_free(lj_batch *b)
{
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (void *q : b->allocs) cudaFree(q);
    if (b->host_out) cudaFreeHost(b->host_out);
    if (b->host_err) cudaFreeHost(b->host_err);
    delete b;
}

cudaError_t configure(lj_batch *b)
{
    // Staging capacity from the mean occupancy over all replicas (cells of
    // denser replicas that overflow take the plain path); static shared
    // memory of the scan phases: at most 2 KB.
    const double mean_occ = b->ncell > 0 ? (double)b->ntot / (double)b->ncell : 0.0;
    const int R = b->p.cell_subdiv;
    const int cap = warp_stencil_cap(mean_occ, R, kBatchThreads, 2048);
    b->k.cap = cap;
    b->smem = (kBatchThreads / 32) * warp_slice_words(cap, R) * (int)sizeof(float);
    int minblk = 1 << 30;
    for (int mode = 0; mode < 3; mode++)
        for (int en = 0; en < 4; en++) {
            void *kern = batch_kernel(R, mode, en % 2 != 0, en < 2 ? 0 : -1);
            cudaError_t e = raise_dyn_smem(kern, b->smem);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kBatchThreads, b->smem);
            if (e != cudaSuccess) return e;
            if (nb < minblk) minblk = nb;
        }
    if (minblk < 1) return cudaErrorInvalidConfiguration;
    b->grid = minblk * b->nsm;   // all blocks co-resident (cooperative launch)
    b->grid_n3 = 0;
    if (R != 1) return cudaSuccess;
    // the pair-once kernel: staging capacity as for single systems, from the
    // mean occupancy (the raw half stencil m = 14 n_cell plus a Poisson
    // spread and the padding, at least kN3Home * 32, a multiple of 32)
    const double m = kN3Half * mean_occ;
    int cap3 = (int)(m + 4.0 * sqrt(m)) + 64;
    cap3 = cap3 < kN3Home * 32 ? kN3Home * 32 : ((cap3 + 31) & ~31);   // S also holds the home forces' transpose
    // (3 blocks per SM: up to 75 KB of shared memory each, 2 KB of it static)
    const int max3 = ((75 * 1024 - 2048) / (4 * (kBatchThreads / 32)) - kN3FixedWords) / 4 & ~31;
    if (cap3 > max3) cap3 = max3;
    b->kn3 = b->k;
    b->kn3.cap = cap3;
    b->smem_n3 = (kBatchThreads / 32) * n3_slice_words(cap3) * (int)sizeof(float);
    int minblk3 = 1 << 30;
    for (int mode = 0; mode < 3; mode++)
        for (int en = 0; en < 2; en++) {
            void *kern = batch_kernel_n3(mode, en != 0);
            cudaError_t e = raise_dyn_smem(kern, b->smem_n3);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kBatchThreads, b->smem_n3);
            if (e != cudaSuccess) return e;
            if (nb < minblk3) minblk3 = nb;
        }
    b->grid_n3 = minblk3 >= 1 ? minblk3 * b->nsm : 0;
    return cudaSuccess;
}

cudaError_t launch_step_kernel(lj_batch *b, bool energy, int op, double *x, double *v, float4 *f)
{
    b->launches++;
    if (b->n3) {
        void *kern = batch_kernel_n3(b->p.shift_mode, energy);
        void *args[] = {&b->d, &b->kn3, &op, &x, &v, &f};
        return cudaLaunchCooperativeKernel(kern, dim3(b->grid_n3), dim3(kBatchThreads), args, b->smem_n3, b->stream);
    }
    void *kern = batch_kernel(b->p.cell_subdiv, b->p.shift_mode, energy, b->k.gw);
    void *args[] = {&b->d, &b->k, &op, &x, &v, &f};
    return cudaLaunchCooperativeKernel(kern, dim3(b->grid), dim3(kBatchThreads), args, b->smem, b->stream);
}

int sync_check(lj_batch *b)
{
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->host_err, b->d.err, sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return map_err(e);
    const int32_t bits = *b->host_err;
    if (bits) {
        cudaMemsetAsync(b->d.err, 0, sizeof(int32_t), b->stream);
        if (bits & LJ_ERRBIT_TIMEOUT) {   // a launch left its barrier early: restart the counter
            cudaMemsetAsync(b->d.bar_count, 0, sizeof(unsigned), b->stream);
            cudaMemsetAsync(b->d.bar_gen, 0, sizeof(unsigned), b->stream);
        }
        cudaStreamSynchronize(b->stream);
    }
    if (bits & LJ_ERRBIT_NONFINITE) return LJ_ENONFINITE;
    if (bits & LJ_ERRBIT_TIMEOUT) return LJ_ETIMEOUT;
    if (bits & LJ_ERRBIT_SCAN) return LJ_ECUDA;
    return LJ_OK;
}

}  // namespace

extern "C" int lj_batch_create(lj_batch **out, int32_t nrep, const int64_t *n, const double *box,
                               const lj_params *common, void *stream)
{
    if (!out) return LJ_EINVAL;
    *out = nullptr;
    if (nrep < 1 || !n || !box || !common) return LJ_EINVAL;
    if (common->precision != LJ_PREC_MIXED) return LJ_EINVAL;
    // cell subdivision k of every replica: 1 (the default, also for 0) or 2
    if (common->cell_subdiv < 0 || common->cell_subdiv > 2) return LJ_EINVAL;
    std::vector<int32_t> ncs(nrep), poff(nrep + 1), coff(nrep + 1), thoff(nrep + 1), ceoff(nrep + 1);
    int64_t ntot = 0, ncell = 0, nth = 0, nce = 0;
    double max_occ = 0.0;
    for (int r = 0; r < nrep; r++) {
        lj_params q = *common;
        q.n = n[r];
        q.box = box[r];
        int32_t nc = 0;
        int st = lj_grid(&q, &nc);
        if (st != LJ_OK) return st;
        ncs[r] = nc;
        poff[r] = (int32_t)ntot;
        coff[r] = (int32_t)ncell;
        thoff[r] = (int32_t)nth;
        ceoff[r] = (int32_t)nce;
        ntot += n[r];
        ncell += (int64_t)nc * nc * nc;
        nth += nc + 1;
        nce += nc;
        const double occ = (double)n[r] / ((double)nc * nc * nc);
        if (occ > max_occ) max_occ = occ;
        if (ntot >= INT32_MAX || ncell >= INT32_MAX) return LJ_EOVERFLOW;
    }
    poff[nrep] = (int32_t)ntot;
    coff[nrep] = (int32_t)ncell;
    thoff[nrep] = (int32_t)nth;
    ceoff[nrep] = (int32_t)nce;

    lj_batch *b = new lj_batch();
    b->p = *common;
    if (b->p.cell_subdiv == 0) b->p.cell_subdiv = 1;
    b->p.n = ntot;
    b->nrep = nrep;
    b->ntot = ntot;
    b->ncell = ncell;
    b->stream = (cudaStream_t)stream;
    b->use_graph = 1;
    b->max_mean_occ = max_occ;
#define LJ_BCK(call)                 \
    do {                             \
        cudaError_t e_ = (call);     \
        if (e_ != cudaSuccess) {     \
            batch_free(b);           \
            return map_err(e_);      \
        }                            \
    } while (0)
    LJ_BCK(cudaGetDevice(&b->device));
    LJ_BCK(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device));
    int coop = 0;
    LJ_BCK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device));
    if (!coop) {
        batch_free(b);
        return LJ_ECUDA;
    }

    // host tables
    std::vector<double> L(nrep), s(nrep), cw(nrep), whi(nrep), wlo(nrep), centre(nce > 0 ? nce : 1);
    std::vector<long long> thb(nth);
    std::vector<int32_t> rep_of(ntot > 0 ? ntot : 1), rep_of_cell(ncell);
    for (int r = 0; r < nrep; r++) {
        const int nc = ncs[r];
        L[r] = box[r];
        s[r] = (double)nc / box[r];
        cw[r] = box[r] / (double)nc;
        whi[r] = box[r] * (1.0 - ldexp(1.0, -50));
        wlo[r] = box[r] * ldexp(1.0, -50);
        for (int q = 0; q < nc; q++) centre[ceoff[r] + q] = ((double)q + 0.5) * cw[r];
        thb[thoff[r]] = 0;
        for (int q = 1; q < nc; q++) {
            const double t = threshold(q, s[r]);
            memcpy(&thb[thoff[r] + q], &t, sizeof(double));
        }
        thb[thoff[r] + nc] = INT64_MAX;
        for (int64_t i = poff[r]; i < poff[r + 1]; i++) rep_of[i] = r;
        for (int64_t c = coff[r]; c < coff[r + 1]; c++) rep_of_cell[c] = r;
    }

    BatchDev &d = b->d;
    d.ntot = ntot;
    d.ncell = ncell;
    d.nrep = nrep;
    d.ntiles = (int)((ncell + 1 + kScanTile - 1) / kScanTile);   // grid cells + the extra cell
    d.cells_per_grab = 4;
    d.h = 0.5 * common->dt / common->mass;
    d.dt = common->dt;
    d.mass = common->mass;
    int32_t *poff_d, *coff_d, *ncs_d, *thoff_d, *ceoff_d, *rep_of_d, *rep_of_cell_d;
    double *L_d, *s_d, *cw_d, *whi_d, *wlo_d, *centre_d;
    long long *thb_d;
    const size_t n1 = (size_t)(ntot > 0 ? ntot : 1);
    LJ_BCK(balloc(b, &poff_d, nrep + 1));
    LJ_BCK(balloc(b, &coff_d, nrep + 1));
    LJ_BCK(balloc(b, &ncs_d, nrep));
    LJ_BCK(balloc(b, &thoff_d, nrep + 1));
    LJ_BCK(balloc(b, &ceoff_d, nrep + 1));
    LJ_BCK(balloc(b, &rep_of_d, n1));
    LJ_BCK(balloc(b, &rep_of_cell_d, (size_t)ncell));
    LJ_BCK(balloc(b, &L_d, nrep));
    LJ_BCK(balloc(b, &s_d, nrep));
    LJ_BCK(balloc(b, &cw_d, nrep));
    LJ_BCK(balloc(b, &whi_d, nrep));
    LJ_BCK(balloc(b, &wlo_d, nrep));
    LJ_BCK(balloc(b, &centre_d, centre.size()));
    LJ_BCK(balloc(b, &thb_d, thb.size()));
    LJ_BCK(cudaMemcpy(poff_d, poff.data(), sizeof(int32_t) * (nrep + 1), cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(coff_d, coff.data(), sizeof(int32_t) * (nrep + 1), cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(ncs_d, ncs.data(), sizeof(int32_t) * nrep, cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(thoff_d, thoff.data(), sizeof(int32_t) * (nrep + 1), cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(ceoff_d, ceoff.data(), sizeof(int32_t) * (nrep + 1), cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(rep_of_d, rep_of.data(), sizeof(int32_t) * rep_of.size(), cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(rep_of_cell_d, rep_of_cell.data(), sizeof(int32_t) * (size_t)ncell, cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(L_d, L.data(), sizeof(double) * nrep, cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(s_d, s.data(), sizeof(double) * nrep, cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(cw_d, cw.data(), sizeof(double) * nrep, cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(whi_d, whi.data(), sizeof(double) * nrep, cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(wlo_d, wlo.data(), sizeof(double) * nrep, cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(centre_d, centre.data(), sizeof(double) * centre.size(), cudaMemcpyHostToDevice));
    LJ_BCK(cudaMemcpy(thb_d, thb.data(), sizeof(long long) * thb.size(), cudaMemcpyHostToDevice));
    d.poff = poff_d;
    d.coff = coff_d;
    d.ncs = ncs_d;
    d.thoff = thoff_d;
    d.ceoff = ceoff_d;
    d.rep_of = rep_of_d;
    d.rep_of_cell = rep_of_cell_d;
    d.L = L_d;
    d.s = s_d;
    d.cw = cw_d;
    d.whi = whi_d;
    d.wlo = wlo_d;
    d.centre = centre_d;
    d.thb = thb_d;
    LJ_BCK(balloc(b, &d.cell_of, n1));
    LJ_BCK(balloc(b, &d.rank, n1));
    LJ_BCK(balloc(b, &d.count, (size_t)ncell + 1));
    LJ_BCK(balloc(b, &d.start, (size_t)ncell + 2));
    LJ_BCK(balloc(b, &d.tile_sum, (size_t)d.ntiles));
    LJ_BCK(balloc(b, &d.err, 1));
    LJ_BCK(balloc(b, &d.pos, n1));
    LJ_BCK(balloc(b, &d.bar_count, 1));
    LJ_BCK(balloc(b, &d.bar_gen, 1));
    LJ_BCK(balloc(b, &d.work, 1));
    LJ_BCK(balloc(b, &d.first, 16));
    LJ_BCK(balloc(b, &b->rep_out, 3 * (size_t)nrep));
    LJ_BCK(cudaMallocHost(&b->host_out, sizeof(double) * 3 * (size_t)nrep));
    LJ_BCK(cudaMallocHost(&b->host_err, sizeof(int32_t)));
    LJ_BCK(cudaMemset(d.count, 0, sizeof(int32_t) * ((size_t)ncell + 1)));
    LJ_BCK(cudaMemset(d.cell_of, 0, sizeof(int32_t) * n1));
    LJ_BCK(cudaMemset(d.err, 0, sizeof(int32_t)));
    LJ_BCK(cudaMemset(d.bar_count, 0, sizeof(unsigned)));
    LJ_BCK(cudaMemset(d.bar_gen, 0, sizeof(unsigned)));
    LJ_BCK(cudaMemset(d.first, 1, 1));

    WarpParams &k = b->k;
    k.gw = 0;
    k.n = (int)ntot;
    k.nc = 0;
    k.ncell = ncell;
    k.cw = 0.f;
    const double eps = common->eps, sg = common->sigma, rc = common->rc;
    const double s6 = sg * sg * sg * sg * sg * sg, s12 = s6 * s6;
    const double rci2 = 1.0 / (rc * rc), rci6 = rci2 * rci2 * rci2;
    k.rc2 = (float)(rc * rc);
    k.rc = (float)rc;
    k.a12 = (float)(48.0 * eps * s12);
    k.b6 = (float)(24.0 * eps * s6);
    k.c12 = (float)(4.0 * eps * s12);
    k.c6 = (float)(4.0 * eps * s6);
    k.uc = (float)(rci6 * (4.0 * eps * s12 * rci6 - 4.0 * eps * s6));
    k.fc = (float)(rc * rci2 * rci6 * (48.0 * eps * s12 * rci6 - 24.0 * eps * s6));
    LJ_BCK(configure(b));
    // the 27-cell code by default: the pair-once step measured slower on the
    // 256-replica ensemble (2.12 against 1.70 ms per step), its 128
    // registers leaving 16 warps per SM for every phase of the launch
    b->n3 = 0;
#undef LJ_BCK
    *out = b;
    return LJ_OK;
}

extern "C" void lj_batch_destroy(lj_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
}

extern "C" int lj_batch_info(const lj_batch *b, int64_t *ntot, int64_t *ncell, int32_t *grid, int32_t *cap)
{
    if (!b) return LJ_EINVAL;
    if (ntot) *ntot = b->ntot;
    if (ncell) *ncell = b->ncell;
    if (grid) *grid = b->n3 ? b->grid_n3 : b->grid;
    if (cap) *cap = b->n3 ? b->kn3.cap : b->k.cap;
    return LJ_OK;
}

extern "C" int lj_batch_set_tuning(lj_batch *b, int32_t cells_per_grab, int32_t use_graph, int32_t group_width)
{
    if (!b || cells_per_grab < 1 || cells_per_grab > 1024) return LJ_EINVAL;
    if (group_width != 0 && group_width != -1 && group_width != 2 && group_width != 4 && group_width != 8 &&
        group_width != 16 && group_width != 32)
        return LJ_EINVAL;
    b->d.cells_per_grab = cells_per_grab;
    b->k.gw = group_width;
    b->kn3.gw = group_width;
    b->use_graph = use_graph ? 1 : 0;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return LJ_OK;
}

extern "C" int lj_batch_set_kernel(lj_batch *b, int32_t kernel)
{
    if (!b || (kernel != 3 && kernel != 7)) return LJ_EINVAL;
    if (kernel == 7 && b->grid_n3 == 0) return LJ_EINVAL;   // cell subdivision 2
    b->n3 = kernel == 7 ? 1 : 0;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return LJ_OK;
}

extern "C" int lj_batch_forces(lj_batch *b, const double *x, void *f, int32_t energy)
{
    if (!b) return LJ_EINVAL;
    if (b->ntot == 0) return LJ_OK;
    int r;
    if ((r = check_ptr(x, 8)) != LJ_OK) return r;
    if ((r = check_ptr(f, 16)) != LJ_OK) return r;
    cudaError_t e = launch_step_kernel(b, energy != 0, 1, (double *)x, nullptr, (float4 *)f);
    return e == cudaSuccess ? LJ_OK : map_err(e);
}

extern "C" int lj_batch_step(lj_batch *b, double *x, double *v, void *f, int32_t nsteps)
{
    if (!b || nsteps < 0) return LJ_EINVAL;
    if (b->ntot == 0 || nsteps == 0) return LJ_OK;
    int r;
    if ((r = check_ptr(x, 8)) != LJ_OK) return r;
    if ((r = check_ptr(v, 8)) != LJ_OK) return r;
    if ((r = check_ptr(f, 16)) != LJ_OK) return r;
    cudaError_t e = cudaMemsetAsync(b->d.first, 1, 1, b->stream);
    if (e != cudaSuccess) return map_err(e);
    bool graph = b->use_graph != 0;
    if (graph && (!b->gexec || b->gx != x || b->gv != v || b->gf != f)) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaStream_t cs = b->stream;
        bool own = false;
        if (!cs) {  // the legacy stream cannot be captured
            if (cudaStreamCreate(&cs) != cudaSuccess) return LJ_ECUDA;
            own = true;
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaStream_t keep = b->stream;
            b->stream = cs;
            cudaError_t el = launch_step_kernel(b, false, 0, x, v, (float4 *)f);
            b->launches--;
            b->stream = keep;
            e = cudaStreamEndCapture(cs, &g);
            if (el != cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (own) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->gexec = nullptr;
            b->use_graph = 0;   // capture unsupported here: launch directly
            graph = false;
        } else {
            b->gx = x;
            b->gv = v;
            b->gf = f;
        }
    }
    for (int s = 0; s < nsteps; s++) {
        if (graph) {
            e = cudaGraphLaunch(b->gexec, b->stream);
            b->launches++;
        } else {
            e = launch_step_kernel(b, false, 0, x, v, (float4 *)f);
        }
        if (e != cudaSuccess) return map_err(e);
    }
    k_batch_kick<<<(unsigned)((b->ntot + 255) / 256), 256, 0, b->stream>>>(v, (const float4 *)f, b->ntot, b->d.h);
    b->launches++;
    e = cudaGetLastError();
    return e == cudaSuccess ? LJ_OK : map_err(e);
}

extern "C" int lj_batch_energy(lj_batch *b, const double *x, const double *v, void *f, double *out)
{
    if (!b || !out) return LJ_EINVAL;
    int r;
    if (b->ntot > 0) {
        if ((r = check_ptr(x, 8)) != LJ_OK) return r;
        if ((r = check_ptr(v, 8)) != LJ_OK) return r;
        if ((r = check_ptr(f, 16)) != LJ_OK) return r;
        cudaError_t e = launch_step_kernel(b, true, 1, (double *)x, nullptr, (float4 *)f);
        if (e != cudaSuccess) return map_err(e);
    }
    k_batch_energy<<<b->nrep, kReduceThreads, 0, b->stream>>>(v, (const float4 *)f, b->d.poff, b->p.mass,
                                                              b->rep_out);
    b->launches++;
    cudaError_t e = cudaMemcpyAsync(b->host_out, b->rep_out, sizeof(double) * 3 * (size_t)b->nrep,
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return map_err(e);
    r = sync_check(b);
    if (r != LJ_OK) return r;
    memcpy(out, b->host_out, sizeof(double) * 3 * (size_t)b->nrep);
    return LJ_OK;
}

extern "C" int lj_batch_relax(lj_batch *b, double *x, void *f, int32_t nsteps, double alpha, double max_disp)
{
    if (!b || nsteps < 0 || !(alpha >= 0.0) || !(max_disp >= 0.0)) return LJ_EINVAL;
    if (b->ntot == 0) return LJ_OK;
    int r;
    if ((r = check_ptr(x, 8)) != LJ_OK) return r;
    if ((r = check_ptr(f, 16)) != LJ_OK) return r;
    for (int s = 0; s < nsteps; s++) {
        cudaError_t e = launch_step_kernel(b, false, 1, x, nullptr, (float4 *)f);
        if (e != cudaSuccess) return map_err(e);
        k_batch_sd<<<(unsigned)((b->ntot + 255) / 256), 256, 0, b->stream>>>(
            x, (const float4 *)f, b->ntot, b->d.rep_of, b->d.L, b->d.whi, b->d.wlo, alpha, max_disp);
        b->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return map_err(e);
    }
    // leave f = F(x) at the relaxed positions
    cudaError_t e = launch_step_kernel(b, false, 1, x, nullptr, (float4 *)f);
    return e == cudaSuccess ? LJ_OK : map_err(e);
}

extern "C" int lj_batch_check(lj_batch *b)
{
    if (!b) return LJ_EINVAL;
    return sync_check(b);
}

extern "C" int lj_batch_launches(const lj_batch *b, int64_t *launches, int32_t *graph)
{
    if (!b) return LJ_EINVAL;
    if (launches) *launches = b->launches;
    if (graph) *graph = b->use_graph && b->gexec ? 1 : 0;
    return LJ_OK;
}
