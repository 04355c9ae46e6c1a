// Warp-per-cell force kernel with the stencil loads pipelined through the
// copy engine (FP32-mixed, 27-cell stencil, forces stored).
//
// Same method and arithmetic as lj_force_warp.cu (Section 3 cell list,
// Section 2 pair force); only the way a cell's stencil reaches shared
// memory differs.  The direct kernel loads the ~360 stencil particles of a
// cell with per-lane global loads, each round an L2 round trip, and its
// profile shows that staging as latency.  Here, while a warp computes cell
// c, the 27 stencil cells of its next cell are already in flight:
//  * the warp writes the next cell's stencil table (start, count, shift)
//    and lanes 0..26 each issue one cp.async.bulk of their cell's contiguous
//    float4 range into the warp's raw buffer, completing on the warp's
//    mbarrier (bounded waits, LJ_ETIMEOUT);
//  * when the warp reaches that cell it waits on the mbarrier, converts the
//    raw particles to the home-cell frame and prunes them against the home
//    particles' bounding box from shared memory (lane k walks stencil cell
//    k), then issues the copies for the cell after, and only then computes.
// One raw buffer suffices: the conversion has consumed it before the next
// copies are issued.  Cells whose stencil exceeds the raw buffer, with more
// than 32 particles, or whose pruned list overflows the slice take the plain
// path of lj_force_cell.cuh.
#include <math.h>
#include <string.h>

#include "lj_force_cell.cuh"
#include "lj_pair.cuh"

namespace {

constexpr int kPipeThreads = 64;   // 2 warps per CTA: shared memory, not threads, sets residency

// Words of one warp's slice: raw float4[raw_cap], X, Y, Z float[cap],
// stencil table float4[27] and prefix int[28], mbarrier (8 B) + padding.
__host__ __device__ constexpr int pipe_slice_words(int cap, int raw_cap)
{
    return 4 * raw_cap + 3 * cap + 4 * 27 + 28 + 4;
}

struct PipeCell {
    int64_t c;       // cell id, -1 for none
    int n_home, Ttot;
    int bulk;        // 1: copies issued into raw; 0: plain path
};

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kPipeThreads, 9) k_force_pipe(WarpParams k, int raw_cap, const float4 *__restrict__ pos,
                                                            const int32_t *__restrict__ start,
                                                            float4 *__restrict__ fout, double *__restrict__ partial,
                                                            int32_t *__restrict__ err)
{
    extern __shared__ __align__(16) float psmem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *slice = psmem + (size_t)warp * pipe_slice_words(k.cap, raw_cap);
    float4 *raw = reinterpret_cast<float4 *>(slice);
    float *X = slice + 4 * raw_cap;
    float *Y = X + k.cap;
    float *Z = Y + k.cap;
    float4 *stab = reinterpret_cast<float4 *>(Z + k.cap);
    int *spre = reinterpret_cast<int *>(stab + 27);
    uint64_t *bar = reinterpret_cast<uint64_t *>(spre + 28);
    const int nc = k.nc;
    const StoreForce<MODE, ENERGY> out{fout, k.n};
    double eacc = 0.0, wacc = 0.0;
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity = 0;

    // the warp's cells: chunks of k.grab consecutive cells pulled from the
    // work counter
    int64_t chunk_end = 0;
    auto pull = [&]() -> int64_t {
        unsigned c0 = 0;
        if (lane == 0) c0 = atomicAdd(k.work, (unsigned)k.grab);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        chunk_end = min((int64_t)c0 + k.grab, k.ncell);
        return (int64_t)c0 < k.ncell ? (int64_t)c0 : -1;
    };

    // Stencil table of cell c; issue its copies when they fit.
    auto prepare = [&](int64_t c) -> PipeCell {
        PipeCell pc;
        pc.c = c;
        pc.n_home = 0;
        pc.Ttot = 0;
        pc.bulk = 0;
        if (c < 0) return pc;
        __syncwarp();   // every lane is done with the previous table and raw data
        const int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        int s = 0, nn = 0;
        if (lane < 27) {
            int dx, dy, dz;
            stencil_delta<1>(lane, dx, dy, dz);
            int ux = cx + dx, uy = cy + dy, uz = cz + dz;
            ux += ux < 0 ? nc : 0;
            ux -= ux >= nc ? nc : 0;
            uy += uy < 0 ? nc : 0;
            uy -= uy >= nc ? nc : 0;
            uz += uz < 0 ? nc : 0;
            uz -= uz >= nc ? nc : 0;
            const int64_t cn = ux + (int64_t)nc * (uy + (int64_t)nc * uz);
            s = start[cn];
            nn = start[cn + 1] - s;
            stab[lane] = make_float4((float)dx * k.cw, (float)dy * k.cw, (float)dz * k.cw, __int_as_float(s));
        }
        int P = nn;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, P, o);
            if (lane >= o) P += y;
        }
        const int excl = P - nn;
        if (lane < 27) spre[lane] = excl;
        pc.Ttot = __shfl_sync(0xffffffffu, P, 31);
        if (lane == 0) spre[27] = pc.Ttot;
        pc.n_home = __shfl_sync(0xffffffffu, nn, 0);
        pc.bulk = (pc.n_home > 0 && pc.n_home <= 32 && pc.Ttot <= raw_cap) ? 1 : 0;
        if (pc.bulk) {
            fence_proxy_async_smem();   // the raw buffer's earlier reads before the copies' writes
            if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)pc.Ttot * 16u);
            __syncwarp();
            if (lane < 27 && nn > 0) bulk_g2s(raw + excl, pos + s, (uint32_t)nn * 16u, bar);
        }
        __syncwarp();
        return pc;
    };

    int64_t c = pull();
    PipeCell cur = prepare(c);
    while (cur.c >= 0) {
        // the cell after this one
        int64_t nxt = cur.c + 1 < chunk_end ? cur.c + 1 : pull();
        if (cur.n_home == 0) {
            cur = prepare(nxt);
            continue;
        }
        bool staged = false;
        int T = 0, hid = 0;
        if (cur.bulk) {
            if (!mbar_wait_bounded(bar, parity, err)) {
                // give the copies a second bounded wait before the buffer is
                // abandoned, then stop (forces of the remaining cells unset)
                mbar_wait_bounded(bar, parity, err);
                break;
            }
            parity ^= 1u;
            __syncwarp();   // the previous cell's compute is done with X, Y, Z
            // home particles (entry 0, raw[0 .. n_home)) and their box
            const int n_home = cur.n_home;
            float4 ph = make_float4(0.f, 0.f, 0.f, 0.f);
            float bxl = 3.4e38f, byl = 3.4e38f, bzl = 3.4e38f, bxh = -3.4e38f, byh = -3.4e38f, bzh = -3.4e38f;
            if (lane < n_home) {
                ph = raw[lane];
                hid = __float_as_int(ph.w);
                X[lane] = ph.x;
                Y[lane] = ph.y;
                Z[lane] = ph.z;
                bxl = bxh = ph.x;
                byl = byh = ph.y;
                bzl = bzh = ph.z;
            }
            box_reduce(bxl, byl, bzl, bxh, byh, bzh);
            // lane k (1..26) converts and prunes stencil cell k from raw
            const float rcut2 = k.rc2 * 1.0001f;
            const unsigned lt = (1u << lane) - 1u;
            float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
            int my_n = 0, my_off = 0;
            if (lane >= 1 && lane < 27) {
                sh = stab[lane];
                my_off = spre[lane];
                my_n = spre[lane + 1] - my_off;
            }
            T = n_home;
            bool full = false;
            for (int e = 0; __any_sync(0xffffffffu, e < my_n); e++) {
                if (T + 64 > k.cap) {
                    full = true;
                    break;
                }
                bool keep = false;
                float cx = 0.f, cy = 0.f, cz = 0.f;
                if (e < my_n) {
                    const float4 q = raw[my_off + e];
                    cx = q.x + sh.x;
                    cy = q.y + sh.y;
                    cz = q.z + sh.z;
                    const float dx = fmaxf(fmaxf(bxl - cx, cx - bxh), 0.f);
                    const float dy = fmaxf(fmaxf(byl - cy, cy - byh), 0.f);
                    const float dz = fmaxf(fmaxf(bzl - cz, cz - bzh), 0.f);
                    keep = dx * dx + dy * dy + dz * dz < rcut2;
                }
                const unsigned kept = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int sl = T + __popc(kept & lt);
                    X[sl] = cx;
                    Y[sl] = cy;
                    Z[sl] = cz;
                }
                T += __popc(kept);
            }
            staged = !full;
            if (staged) {
                X[T + lane] = kFar;
                Y[T + lane] = kFar;
                Z[T + lane] = kFar;
            }
        }
        if (!staged) {
            // the table of this cell is still in place
            __syncwarp();
            const int s_home = __float_as_int(stab[0].w);
            cell_plain<1, MODE, ENERGY, true>(k, pos, out, stab, spre, s_home, cur.n_home, eacc, wacc);
            cur = prepare(nxt);
            continue;
        }
        // copies of the next cell go out before this one is computed
        const PipeCell next = prepare(nxt);
        const int s_home = 0;   // home particles are all in lanes (n_home <= 32)
        switch (choose_group(cur.n_home, T, k.gw)) {
            case 2: compute_chunks<2, MODE, ENERGY, true>(k, pos, out, X, Y, Z, T, s_home, cur.n_home, hid, eacc, wacc); break;
            case 4: compute_chunks<4, MODE, ENERGY, true>(k, pos, out, X, Y, Z, T, s_home, cur.n_home, hid, eacc, wacc); break;
            case 8: compute_chunks<8, MODE, ENERGY, true>(k, pos, out, X, Y, Z, T, s_home, cur.n_home, hid, eacc, wacc); break;
            case 16: compute_chunks<16, MODE, ENERGY, true>(k, pos, out, X, Y, Z, T, s_home, cur.n_home, hid, eacc, wacc); break;
            default: compute_chunks<32, MODE, ENERGY, true>(k, pos, out, X, Y, Z, T, s_home, cur.n_home, hid, eacc, wacc); break;
        }
        cur = next;
    }
    if constexpr (ENERGY) {
        __shared__ double red[2 * (kPipeThreads / 32)];
        for (int o = 16; o > 0; o >>= 1) {
            eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
            wacc += __shfl_xor_sync(0xffffffffu, wacc, o);
        }
        if (lane == 0) {
            red[2 * warp] = eacc;
            red[2 * warp + 1] = wacc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double es = 0.0, ws = 0.0;
            for (int q = 0; q < kPipeThreads / 32; q++) {
                es += red[2 * q];
                ws += red[2 * q + 1];
            }
            partial[2 * blockIdx.x] = es;
            partial[2 * blockIdx.x + 1] = ws;
        }
    }
}

void *pipe_kernel(int mode, bool energy)
{
    switch (mode * 2 + (energy ? 1 : 0)) {
        case 0: return (void *)k_force_pipe<0, false>;
        case 1: return (void *)k_force_pipe<0, true>;
        case 2: return (void *)k_force_pipe<1, false>;
        case 3: return (void *)k_force_pipe<1, true>;
        case 4: return (void *)k_force_pipe<2, false>;
        default: return (void *)k_force_pipe<2, true>;
    }
}

}  // namespace

cudaError_t pipe_force_configure(lj_ctx *c)
{
    // raw buffer: the mean stencil population m plus 3.5 sqrt(m); pruned list:
    // 3/4 of that (the bounding-box test keeps ~2/3 at cell side ~rc) plus the
    // 32-entry padding and one round's margin.
    const double mean = c->ncell > 0 ? (double)c->p.n / (double)c->ncell : 0.0;
    const double m = 27.0 * mean;
    int raw_cap = ((int)(m + 3.5 * sqrt(m)) + 8 + 7) & ~7;
    if (raw_cap < 64) raw_cap = 64;
    int cap = ((int)(0.75 * raw_cap) + 64 + 7) & ~7;
    c->pcap = cap;
    c->praw = raw_cap;
    c->pipe_smem = (kPipeThreads / 32) * pipe_slice_words(cap, raw_cap) * (int)sizeof(float);
    if (c->pipe_smem > 227 * 1024) return cudaErrorInvalidValue;
    int minblk = 1 << 30;
    for (int mode = 0; mode < 3; mode++)
        for (int en = 0; en < 2; en++) {
            void *kern = pipe_kernel(mode, en == 1);
            cudaError_t e = raise_dyn_smem(kern, c->pipe_smem);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kPipeThreads, c->pipe_smem);
            if (e != cudaSuccess) return e;
            if (nb < minblk) minblk = nb;
        }
    if (minblk < 1) minblk = 1;
    int64_t need = (c->ncell + kPipeThreads / 32 - 1) / (kPipeThreads / 32);
    int64_t grid = (int64_t)minblk * c->nsm;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    c->pipe_grid = (int)grid;
    return cudaSuccess;
}

cudaError_t launch_force_pipe(lj_ctx *c, void *f, bool energy)
{
    if (c->pipe_grid == 0) {
        cudaError_t e = pipe_force_configure(c);
        if (e != cudaSuccess) return e;
    }
    WarpParams k = warp_params_of(c);
    k.cap = c->pcap;
    if (k.grab <= 0) k.grab = 4;   // the pipeline follows pulled runs of cells
    int raw_cap = c->praw;
    const float4 *pos = (const float4 *)c->pos;
    const int32_t *start = c->start;
    double *partial = c->partial;
    int32_t *err = c->err;
    if (c->pipe_grid > c->npartial_cap) return cudaErrorInvalidValue;
    c->npartial = c->pipe_grid;
    void *args[] = {&k, &raw_cap, (void *)&pos, (void *)&start, &f, &partial, &err};
    if (c->timing && c->ev_used + 2 <= c->nev) cudaEventRecord(c->ev[c->ev_used], c->stream);
    cudaError_t e = cudaLaunchKernel(pipe_kernel(c->p.shift_mode, energy), dim3(c->pipe_grid), dim3(kPipeThreads),
                                     args, c->pipe_smem, c->stream);
    if (c->timing && c->ev_used + 2 <= c->nev) {
        cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
        c->ev_used += 2;
    }
    c->kernel_launches++;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
