// Cell binning as a counting sort: count (atomics), exclusive scan, scatter.
// This rebuilds the cell lists of Section 3 from scratch at every call; the
// sorted positions play the role of the paper's per-cell arrays of
// placeholders (Section 3.1: particles of a cell physically together in
// memory) without a fixed capacity.
#include "lj_internal.cuh"

namespace {

// Per particle: wrapped position, cell id, rank within the cell (one
// atomic per distinct cell per warp).  Launched with whole warps.  With a
// gate (cell lists with a skin), nothing happens unless *gate is set, and
// then the particle's displacement accumulator is cleared too.
__global__ void k_bin_count(const double *__restrict__ x, int n, double L, double whi, double wlo, double s, int nc,
                            int32_t *__restrict__ cell_of, int32_t *__restrict__ rank,
                            int32_t *__restrict__ count, int32_t *__restrict__ err, const int32_t *gate,
                            float4 *__restrict__ disp)
{
    if (gate && !*gate) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (disp && i < n) disp[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool valid = i < n;
    int c = 0;
    if (valid) {
        double px = x[3 * (int64_t)i + 0], py = x[3 * (int64_t)i + 1], pz = x[3 * (int64_t)i + 2];
        if (isfinite(px) && isfinite(py) && isfinite(pz)) {
            int cx = lj_cell1(lj_wrap_fast(px, L, whi, wlo), s, nc);
            int cy = lj_cell1(lj_wrap_fast(py, L, whi, wlo), s, nc);
            int cz = lj_cell1(lj_wrap_fast(pz, L, whi, wlo), s, nc);
            c = cx + nc * (cy + nc * cz);
        } else {
            atomicOr(err, LJ_ERRBIT_NONFINITE);
            c = nc * nc * nc;   // the extra cell
        }
    }
    const int r = lj_warp_rank(count, c, valid);
    if (valid) {
        cell_of[i] = c;
        rank[i] = r;
    }
}

// Scan phase 1: sum of each tile of kScanTile counts.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int32_t *__restrict__ count, int64_t ncell,
                                                             int32_t *__restrict__ tile_sum, unsigned *work,
                                                             const int32_t *gate)
{
    if (work && blockIdx.x == 0 && threadIdx.x == 0) *work = 0u;   // the force kernel's work counter
    if (gate && !*gate) return;
    __shared__ int32_t warp_sum[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int32_t acc = 0;
    for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
        int64_t e = base + k;
        if (e < ncell) acc += count[e];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; w++) t += warp_sum[w];
        tile_sum[blockIdx.x] = t;
    }
}

// Scan phase 2: each tile adds the sum of all earlier tiles and scans its
// own counts into start[].  Counts are reset to zero for the next binning.
// The last tile writes start[ncell] and checks it against n.
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int32_t *__restrict__ count, int64_t ncell,
                                                             const int32_t *__restrict__ tile_sum,
                                                             int32_t *__restrict__ start, int n,
                                                             int32_t *__restrict__ err, const int32_t *gate)
{
    if (gate && !*gate) return;
    __shared__ int32_t warp_tot[kScanThreads / 32];
    __shared__ int32_t s_prefix;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    // prefix of earlier tiles
    int32_t pre = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += kScanThreads) pre += tile_sum[t];
    for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, o);
    if (lane == 0) warp_tot[wid] = pre;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; w++) t += warp_tot[w];
        s_prefix = t;
    }
    __syncthreads();
    const int32_t tile_prefix = s_prefix;

    // thread-local run of kScanItems consecutive counts
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int64_t e = base + k;
        v[k] = e < ncell ? count[e] : 0;
        local += v[k];
    }
    // block exclusive scan of the per-thread totals
    int32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    int32_t warp_pre = 0;
    for (int w = 0; w < wid; w++) warp_pre += warp_tot[w];
    int32_t run = tile_prefix + warp_pre + incl - local;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int64_t e = base + k;
        if (e < ncell) {
            start[e] = run;
            count[e] = 0;
        }
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) {
        start[ncell] = run;
        if (run != n) atomicOr(err, LJ_ERRBIT_SCAN);
    }
}

// Single-pass exclusive scan of the cell counts into start[] (ordered tiles
// with look-back).  A block takes the next tile from a ticket, so a tile
// only ever waits on tiles whose blocks started earlier and are running or
// done: progress does not depend on how blocks are scheduled.  Each tile
// publishes its total, then (after looking back over its predecessors) its
// inclusive prefix, as 64-bit status words [epoch:30 | kind:2 | value:32]
// (kind 1 = total only, 2 = inclusive prefix).  The epoch (ctl[2]) changes
// at every launch, so the status words need no clearing.  Waits are
// bounded: after ~1 s a wait latches LJ_ERRBIT_TIMEOUT and goes on (wrong
// starts, reported by lj_check) instead of hanging.  The last block to
// finish resets the ticket and the done count and advances the epoch.
// Counts are reset to zero for the next binning; the last tile writes
// start[ncell] and checks it against n.  ctl: [ticket, done, epoch].
__device__ __forceinline__ unsigned long long scan_word(unsigned epoch, unsigned kind, int32_t value)
{
    return ((unsigned long long)(epoch & 0x3fffffffu) << 34) | ((unsigned long long)kind << 32) | (unsigned)value;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_onepass(int32_t *__restrict__ count, int64_t ncell,
                                                               int32_t *__restrict__ start, int n,
                                                               unsigned long long *status, unsigned *ctl,
                                                               int32_t *__restrict__ err, unsigned *work,
                                                               const int32_t *gate)
{
    if (work && blockIdx.x == 0 && threadIdx.x == 0) *work = 0u;   // the force kernel's work counter
    if (gate && !*gate) return;
    __shared__ int32_t warp_tot[kScanThreads / 32];
    __shared__ int32_t s_prefix;
    __shared__ unsigned s_tile, s_epoch;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(ctl, 1u);
        s_epoch = *(volatile unsigned *)(ctl + 2);
    }
    __syncthreads();
    const int tile = (int)s_tile;
    const unsigned epoch = s_epoch & 0x3fffffffu;

    // this tile's counts, kScanItems consecutive ones per thread
    const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t e = base + k;
        v[k] = e < ncell ? count[e] : 0;
        local += v[k];
    }
    int32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    int32_t warp_pre = 0, total = 0;
    for (int w = 0; w < kScanThreads / 32; w++) {
        warp_pre += w < wid ? warp_tot[w] : 0;
        total += warp_tot[w];
    }
    volatile unsigned long long *vst = status;
    if (wid == 0) {
        if (tile == 0) {
            if (lane == 0) {
                vst[0] = scan_word(epoch, 2u, total);
                s_prefix = 0;
            }
        } else {
            if (lane == 0) vst[tile] = scan_word(epoch, 1u, total);
            // look back over windows of 32 predecessors, nearest first
            int32_t excl = 0;
            int p = tile - 1;
            unsigned spins = 0;
            const long long t0 = clock64();
            for (;;) {
                const int q = p - lane;
                unsigned kind = 0;
                int32_t val = 0;
                if (q >= 0) {
                    const unsigned long long w = vst[q];
                    if ((unsigned)(w >> 34) == epoch) {
                        kind = (unsigned)(w >> 32) & 3u;
                        val = (int32_t)(unsigned)w;
                    }
                }
                if (!__all_sync(0xffffffffu, q < 0 || kind != 0)) {
                    if ((++spins & 63u) == 0 && clock64() - t0 > (1ll << 31)) {
                        if (lane == 0) atomicOr(err, LJ_ERRBIT_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);
                    continue;
                }
                const unsigned inc = __ballot_sync(0xffffffffu, q >= 0 && kind == 2u);
                const int upto = inc ? __ffs(inc) - 1 : 31;   // nearest inclusive prefix, or the whole window
                int32_t part = lane <= upto && q >= 0 ? val : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                excl += part;
                if (inc || p - 32 < 0) break;   // tile 0 is inclusive, so a window reaching it ends too
                p -= 32;
            }
            if (lane == 0) {
                vst[tile] = scan_word(epoch, 2u, excl + total);
                s_prefix = excl;
            }
        }
    }
    __syncthreads();
    int32_t run = s_prefix + warp_pre + incl - local;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t e = base + k;
        if (e < ncell) {
            start[e] = run;
            count[e] = 0;
        }
        run += v[k];
    }
    if (tile == (int)gridDim.x - 1 && threadIdx.x == kScanThreads - 1) {
        start[ncell] = run;
        if (run != n) atomicOr(err, LJ_ERRBIT_SCAN);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(ctl + 1, 1u) == gridDim.x - 1) {
            ctl[0] = 0u;
            ctl[1] = 0u;
            atomicAdd(ctl + 2, 1u);
        }
    }
}

// Scatter each particle to its sorted slot: perm[slot] = i and the position
// relative to the centre of its cell (FP32 or FP64), with the particle index
// carried in .w.  centre[k] = (k + 1/2) L / nc, one FP64 subtraction per
// coordinate.  One particle per thread (kScatterPer; two measured slower,
// 66 against 49 us at 4M).
constexpr int kScatterPer = 1;

template <typename T>
__global__ void __launch_bounds__(256) k_scatter(const double *__restrict__ x, int n, double L, double whi,
                                                 double wlo, const double *__restrict__ centre, int nc,
                                                 float inv_nc, bool wrap, const int32_t *__restrict__ cell_of,
                                                 const int32_t *__restrict__ rank, const int32_t *__restrict__ start,
                                                 int32_t *__restrict__ perm, typename Vec4<T>::type *__restrict__ pos)
{
    const int i0 = blockIdx.x * (kScatterPer * blockDim.x) + threadIdx.x;
    int cr[kScatterPer], rr[kScatterPer];
    double xr[kScatterPer][3];
#pragma unroll
    for (int u = 0; u < kScatterPer; u++) {
        const int i = i0 + u * blockDim.x;
        if (i < n) {
            cr[u] = cell_of[i];
            rr[u] = rank[i];
            xr[u][0] = x[3 * (int64_t)i + 0];
            xr[u][1] = x[3 * (int64_t)i + 1];
            xr[u][2] = x[3 * (int64_t)i + 2];
        }
    }
#pragma unroll
    for (int u = 0; u < kScatterPer; u++) {
        const int i = i0 + u * blockDim.x;
        if (i >= n) continue;
        const int c = cr[u];
        const int slot = __ldg(start + c) + rr[u];
        double px = xr[u][0], py = xr[u][1], pz = xr[u][2];
        if (wrap) {
            px = lj_wrap_fast(px, L, whi, wlo);
            py = lj_wrap_fast(py, L, whi, wlo);
            pz = lj_wrap_fast(pz, L, whi, wlo);
        }
        typename Vec4<T>::type q;
        if (c < nc * nc * nc) {
            int cx, cy, cz;
            lj_cell_decode(c, nc, inv_nc, cx, cy, cz);
            q.x = (T)(px - __ldg(centre + cx));
            q.y = (T)(py - __ldg(centre + cy));
            q.z = (T)(pz - __ldg(centre + cz));
        } else {   // the extra cell of non-finite particles (never read as a neighbour)
            q.x = q.y = q.z = (T)px;
        }
        if constexpr (sizeof(T) == 4) {
            q.w = __int_as_float(i);
        } else {
            q.w = (double)i;
        }
        perm[slot] = i;
        pos[slot] = q;
    }
}

// Deterministic order inside the cells: particle p of cell c moves to slot
// start[c] + (number of particles of c with a smaller index), i.e. the cells
// are sorted by particle index -- the order a serial counting sort gives.
// One warp per cell; the cell's indices are read as warp-uniform loads.
// Writes the sorted copy to (pos_out, perm_out) and the new ranks.
template <typename T>
__global__ void k_cell_sort(const int32_t *__restrict__ start, int64_t ncell,
                            const typename Vec4<T>::type *__restrict__ pos, const int32_t *__restrict__ perm,
                            typename Vec4<T>::type *__restrict__ pos_out, int32_t *__restrict__ perm_out,
                            int32_t *__restrict__ rank)   // rank: nullptr = not needed afterwards
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c <= ncell; c += nwarps) {
        const int s = start[c], n = start[c + 1] - s;
        if (n <= 32) {
            // the cell's indices sit in the lanes: compare by shuffles
            const int my = lane < n ? perm[s + lane] : 0x7fffffff;
            int below = 0;
            for (int j = 0; j < n; j++) below += __shfl_sync(0xffffffffu, my, j) < my ? 1 : 0;
            if (lane < n) {
                pos_out[s + below] = pos[s + lane];
                perm_out[s + below] = my;
                if (rank) rank[my] = below;
            }
            continue;
        }
        for (int p0 = 0; p0 < n; p0 += 32) {
            const int p = p0 + lane;
            const int my = p < n ? perm[s + p] : 0x7fffffff;
            int below = 0;
            for (int j = 0; j < n; j++) below += perm[s + j] < my ? 1 : 0;
            if (p < n) {
                pos_out[s + below] = pos[s + p];
                perm_out[s + below] = my;
                if (rank) rank[my] = below;
            }
        }
    }
}

__global__ void k_counts_from_start(const int32_t *__restrict__ start, int64_t ncell, int32_t *__restrict__ count)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) count[c] = start[c + 1] - start[c];
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_bin_count(lj_ctx *c, const double *x, bool gated)
{
    int n = (int)c->p.n;
    if (n > 0) {
        // an ungated binning in skin mode also restarts the displacement count
        float4 *disp = c->skin > 0.0 ? c->disp : nullptr;
        k_bin_count<<<blocks_for(n, 256), 256, 0, c->stream>>>(x, n, c->p.box, c->wrap_hi, c->wrap_lo, c->inv_cw, c->nc, c->cell_of,
                                                                c->rank, c->count, c->err,
                                                                gated ? c->skin_flags + 1 : nullptr, disp);
        c->kernel_launches++;
    }
    return cudaGetLastError();
}

cudaError_t launch_scan(lj_ctx *c, bool gated)
{
    // ncell + 1 cells: the grid and the extra cell of non-finite particles
    const int32_t *gate = gated ? c->skin_flags + 1 : nullptr;
    if (c->scan_status) {
        k_scan_onepass<<<c->ntiles, kScanThreads, 0, c->stream>>>(c->count, c->ncell + 1, c->start, (int)c->p.n,
                                                                   c->scan_status, c->scan_ctl, c->err, c->work, gate);
        c->kernel_launches++;
        return cudaGetLastError();
    }
    k_scan_tiles<<<c->ntiles, kScanThreads, 0, c->stream>>>(c->count, c->ncell + 1, c->tile_sum, c->work, gate);
    k_scan_apply<<<c->ntiles, kScanThreads, 0, c->stream>>>(c->count, c->ncell + 1, c->tile_sum, c->start,
                                                             (int)c->p.n, c->err, gate);
    c->kernel_launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_scatter(lj_ctx *c, const double *x, bool wrap)
{
    int n = (int)c->p.n;
    if (n > 0) {
        const unsigned grid = blocks_for(n, kScatterPer * 256);
        // inv_nc_f is 0 in contexts that do not set it (integer division)
        if (c->p.precision == LJ_PREC_FP64)
            k_scatter<double><<<grid, 256, 0, c->stream>>>(x, n, c->p.box, c->wrap_hi, c->wrap_lo, c->centre, c->nc,
                                                            c->inv_nc_f, wrap, c->cell_of, c->rank, c->start, c->perm,
                                                            (double4_16a *)c->pos);
        else
            k_scatter<float><<<grid, 256, 0, c->stream>>>(x, n, c->p.box, c->wrap_hi, c->wrap_lo, c->centre, c->nc,
                                                           c->inv_nc_f, wrap, c->cell_of, c->rank, c->start, c->perm,
                                                           (float4 *)c->pos);
        c->kernel_launches++;
    }
    if (n > 0 && c->deterministic) {
        // sorted copy into the spare buffers, which then become the current
        // ones; the ranks are rewritten only where a later refresh reuses
        // them (cells with a skin)
        int32_t *rk = c->skin > 0.0 ? c->rank : nullptr;
        const unsigned grid = (unsigned)((c->ncell + 1 + 7) / 8);
        if (c->p.precision == LJ_PREC_FP64)
            k_cell_sort<double><<<grid, 256, 0, c->stream>>>(c->start, c->ncell, (const double4_16a *)c->pos, c->perm,
                                                              (double4_16a *)c->pos_alt, c->perm_alt, rk);
        else
            k_cell_sort<float><<<grid, 256, 0, c->stream>>>(c->start, c->ncell, (const float4 *)c->pos, c->perm,
                                                             (float4 *)c->pos_alt, c->perm_alt, rk);
        c->kernel_launches++;
        void *tp = c->pos;
        c->pos = c->pos_alt;
        c->pos_alt = tp;
        int32_t *tq = c->perm;
        c->perm = c->perm_alt;
        c->perm_alt = tq;
    }
    return cudaGetLastError();
}

cudaError_t launch_counts_from_start(lj_ctx *c, int32_t *count)
{
    k_counts_from_start<<<blocks_for(c->ncell, 256), 256, 0, c->stream>>>(c->start, c->ncell, count);
    c->kernel_launches++;
    return cudaGetLastError();
}
