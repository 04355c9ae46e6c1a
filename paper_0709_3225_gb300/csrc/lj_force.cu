// Lennard-Jones forces over cell lists (Section 3 of van Meel et al.): every
// particle interacts with the particles of its own cell and of the 26
// neighbouring cells; pair force per Section 2 (Eq. n2_force with the
// truncated / shifted LJ force).
//
// Design (GB300):
//  * Particles are sorted by cell, so a row of cells along x is one
//    contiguous range.  A work item is a run of up to 8 consecutive home
//    cells of one (y, z) row; its stencil is 9 neighbour rows, each a window
//    of run+2 consecutive cells -- at most 2 contiguous ranges per row.
//  * A persistent CTA = 1 producer warp + 8 consumer warps.  The producer
//    reads the cell starts of the next item and stages its 9 row windows into
//    shared memory with bulk asynchronous copies (cp.async.bulk, completion
//    on an mbarrier), double-buffered, while the consumers work on the
//    current item.  If a window does not fit in shared memory the consumers
//    read it from global memory instead (correct, slower).
//  * One consumer warp per home cell.  Lanes form S = 32/G groups of G lanes
//    (G = 8, 16 or 32 by the cell's occupancy); lane g of a group owns home
//    particle g, groups split the candidates, and a butterfly of shuffles
//    joins the groups' partial forces.  All lanes of a group read the same
//    candidate (shared-memory broadcast).
//  * Positions are stored relative to their cell centre, so FP32 pair
//    arithmetic keeps ~1e-7 absolute resolution at any box size; the cell
//    offset (dx, dy, dz) * cw is applied once per neighbour cell.
//  * The cutoff and self-pair test is a select, not a branch.
//  * Energies and virials: per-particle FP32 (mixed) sums, accumulated into
//    FP64 per CTA, reduced by a second small kernel in a fixed order.
#include "lj_pair.cuh"

namespace {

struct ForceParams {
    int n, nc, run_len, runs, nitems, cap;
    double cw;
    double rc2, rc, a12, b6, c12, c6, uc, fc;  // see pair_coeffs()
};

// Candidate loaders: explicit ld.shared for the staged path, read-only
// global loads otherwise.
template <typename V, bool STAGED> struct Loader;

template <> struct Loader<float4, true> {
    uint32_t base;
    __device__ __forceinline__ explicit Loader(const float4 *p) : base(smem_addr(p)) {}
    __device__ __forceinline__ float4 operator()(int j) const
    {
        float4 v;
        asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "r"(base + 16u * (uint32_t)j));
        return v;
    }
};

template <> struct Loader<double4_16a, true> {
    uint32_t base;
    __device__ __forceinline__ explicit Loader(const double4_16a *p) : base(smem_addr(p)) {}
    __device__ __forceinline__ double4_16a operator()(int j) const
    {
        double4_16a v;
        asm("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(base + 32u * (uint32_t)j));
        asm("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.z), "=d"(v.w) : "r"(base + 32u * (uint32_t)j + 16u));
        return v;
    }
};

template <typename V> struct Loader<V, false> {
    const V *p;
    __device__ __forceinline__ explicit Loader(const V *q) : p(q) {}
    __device__ __forceinline__ V operator()(int j) const { return p[j]; }
};

struct ItemGeom {
    int cy, cz, cx0, rlen, W;
};

__device__ __forceinline__ ItemGeom item_geom(int item, const ForceParams &p)
{
    ItemGeom g;
    int row = item / p.runs;
    int run = item - row * p.runs;
    g.cy = row % p.nc;
    g.cz = row / p.nc;
    g.cx0 = run * p.run_len;
    g.rlen = min(p.run_len, p.nc - g.cx0);
    g.W = g.rlen + 2;
    return g;
}

// Shared-memory bookkeeping of one staged item.
struct ItemTable {
    int2 seg[kTabMax];       // (base, count) per (row, window cell): base indexes
                             // the staged buffer, or pos[] when staged_global
    int staged_global;
};

// Producer warp: build the table of item `item` and start its copies.
template <typename V>
__device__ void produce(int item, const ForceParams &p, const int32_t *__restrict__ start,
                        const V *__restrict__ pos, V *buf, ItemTable *tab, uint64_t *bar, int *scratch_xx,
                        int *scratch_off, int *scratch_g, bool use_tma)
{
    const int lane = threadIdx.x & 31;
    const ItemGeom g = item_geom(item, p);
    const int KW = 9 * g.W;
    const int nc = p.nc;
    int carry = 0;
    for (int r = 0; r < (kTabMax + 31) / 32; r++) {
        int k = r * 32 + lane;
        int len = 0, s0 = 0, xx = 0;
        if (k < KW) {
            int r9 = k / g.W;
            int ui = k - r9 * g.W;
            int dy = r9 % 3 - 1, dz = r9 / 3 - 1;
            int yy = g.cy + dy, zz = g.cz + dz;
            yy += (yy < 0) ? nc : 0;
            yy -= (yy >= nc) ? nc : 0;
            zz += (zz < 0) ? nc : 0;
            zz -= (zz >= nc) ? nc : 0;
            int u = g.cx0 - 1 + ui;
            xx = u % nc;
            xx += (xx < 0) ? nc : 0;
            int c = xx + nc * (yy + nc * zz);
            s0 = start[c];
            len = start[c + 1] - s0;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int off = carry + incl - len;
        carry += __shfl_sync(0xffffffffu, incl, 31);
        if (k < KW) {
            scratch_xx[k] = xx;
            scratch_off[k] = off;
            scratch_g[k] = s0;
            tab->seg[k] = make_int2(off, len);
        }
    }
    const int total = carry;
    const bool global = (total > p.cap) || !use_tma;
    __syncwarp();
    if (global) {
        for (int k = lane; k < KW; k += 32) tab->seg[k].x = scratch_g[k];
    }
    if (lane == 0) tab->staged_global = global ? 1 : 0;
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, global ? 0u : (uint32_t)(total * sizeof(V)));
    }
    __syncwarp();
    if (!global) {
        for (int k = lane; k < KW; k += 32) {
            int ui = k % g.W;
            if (ui != 0 && scratch_xx[k] != 0) continue;   // not the first cell of a contiguous run
            int kend = k + 1;
            int row_end = (k / g.W + 1) * g.W;
            while (kend < row_end && scratch_xx[kend] != 0) kend++;
            int first = scratch_off[k];
            int last = (kend < KW) ? scratch_off[kend] : total;
            // scratch_off of the next row's first cell == end of this run only
            // when the run reaches the row end; otherwise kend is a wrap
            // point inside the row and scratch_off[kend] is also the run end.
            int cnt = last - first;
            if (cnt > 0) bulk_g2s(buf + first, pos + scratch_g[k], (uint32_t)(cnt * sizeof(V)), bar);
        }
    }
}

// One consumer warp on its home cell of the current item.
template <typename T, int MODE, bool ENERGY, bool STAGED>
__device__ __forceinline__ void consume_cell(const ForceParams &p, const Coef<T> &k, const ItemGeom &g,
                                             const ItemTable *tab, const typename Vec4<T>::type *src, int w,
                                             typename Vec4<T>::type *__restrict__ fout, double &eacc,
                                             double &wacc)
{
    using V = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31;
    const T cw = (T)p.cw;
    const int W = g.W;
    const int2 home = tab->seg[4 * W + w + 1];
    const int hn = home.y;
    const int G = hn <= 8 ? 8 : (hn <= 16 ? 16 : 32);
    const int S = 32 / G;
    const int gl = lane & (G - 1);
    const int sg = lane / G;
    const Loader<V, STAGED> ld(src);
    for (int p0 = 0; p0 < hn; p0 += G) {
        const int i = p0 + gl;
        const bool vi = i < hn;
        V pi = ld(home.x + (vi ? i : 0));
        T fx = 0, fy = 0, fz = 0, e = 0, vir = 0;
#pragma unroll 1
        for (int r9 = 0; r9 < 9; r9++) {
            const T ys = pi.y - (T)(r9 % 3 - 1) * cw;
            const T zs = pi.z - (T)(r9 / 3 - 1) * cw;
#pragma unroll
            for (int dxc = -1; dxc <= 1; dxc++) {
                const int2 sgm = tab->seg[r9 * W + w + 1 + dxc];
                const T xs = pi.x - (T)dxc * cw;
#pragma unroll 4
                for (int j = sg; j < sgm.y; j += S) {
                    V pj = ld(sgm.x + j);
                    pair_accum<T, MODE, ENERGY>(xs - pj.x, ys - pj.y, zs - pj.z, k, fx, fy, fz, e, vir);
                }
            }
        }
        for (int o = G; o < 32; o <<= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
            if constexpr (ENERGY) {
                e += __shfl_xor_sync(0xffffffffu, e, o);
                vir += __shfl_xor_sync(0xffffffffu, vir, o);
            }
        }
        int idx;
        if constexpr (sizeof(T) == 4) {
            idx = __float_as_int(pi.w);
        } else {
            idx = (int)pi.w;
        }
        if (sg == 0 && vi && (unsigned)idx < (unsigned)p.n) {
            V out;
            out.x = fx;
            out.y = fy;
            out.z = fz;
            out.w = ENERGY ? (T)0.5 * e : (T)0;
            fout[idx] = out;
            if constexpr (ENERGY) {
                eacc += 0.5 * (double)e;
                wacc += 0.5 * (double)vir;
            }
        }
    }
}

template <typename T, int MODE, bool ENERGY>
__global__ void __launch_bounds__(kForceThreads) k_force(ForceParams p, const typename Vec4<T>::type *__restrict__ pos,
                                                         const int32_t *__restrict__ start,
                                                         typename Vec4<T>::type *__restrict__ fout,
                                                         double *__restrict__ partial, int32_t *__restrict__ err,
                                                         int use_tma)
{
    using V = typename Vec4<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V *buf0 = reinterpret_cast<V *>(smem_raw);
    V *buf1 = buf0 + p.cap;
    ItemTable *tabs = reinterpret_cast<ItemTable *>(buf1 + p.cap);
    uint64_t *bars = reinterpret_cast<uint64_t *>(tabs + 2);
    int *pscratch = reinterpret_cast<int *>(bars + 2);   // 3 * kTabMax ints, producer only
    double *red = reinterpret_cast<double *>(pscratch + 3 * kTabMax + 1 /* keep 8-byte alignment */ + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const bool producer = (warp == kConsumerWarps);

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const int stride = gridDim.x;
    const int first = blockIdx.x;
    if (producer) {
        if (first < p.nitems)
            produce<V>(first, p, start, pos, buf0, &tabs[0], &bars[0], pscratch, pscratch + kTabMax,
                       pscratch + 2 * kTabMax, use_tma != 0);
        if (first + stride < p.nitems)
            produce<V>(first + stride, p, start, pos, buf1, &tabs[1], &bars[1], pscratch, pscratch + kTabMax,
                       pscratch + 2 * kTabMax, use_tma != 0);
    }

    const Coef<T> kc(p);
    double eacc = 0.0, wacc = 0.0;
    int t = 0;
    for (int item = first; item < p.nitems; item += stride, t++) {
        const int b = t & 1;
        if (!producer) {
            // A wait that timed out skips the item (its buffer may be partial).
            const bool ready = mbar_wait_bounded(&bars[b], (uint32_t)((t >> 1) & 1), err);
            const ItemGeom g = item_geom(item, p);
            const ItemTable *tab = &tabs[b];
            if (ready && warp < g.rlen) {
                if (tab->staged_global)
                    consume_cell<T, MODE, ENERGY, false>(p, kc, g, tab, pos, warp, fout, eacc, wacc);
                else
                    consume_cell<T, MODE, ENERGY, true>(p, kc, g, tab, b ? buf1 : buf0, warp, fout, eacc,
                                                         wacc);
            }
        }
        __syncthreads();   // everyone is done with buffer b
        if (producer) {
            const int nxt = item + 2 * stride;
            if (nxt < p.nitems)
                produce<V>(nxt, p, start, pos, b ? buf1 : buf0, &tabs[b], &bars[b], pscratch,
                           pscratch + kTabMax, pscratch + 2 * kTabMax, use_tma != 0);
        }
    }

    if constexpr (ENERGY) {
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
            for (int q = 0; q < kConsumerWarps + 1; q++) {
                es += red[2 * q];
                ws += red[2 * q + 1];
            }
            partial[2 * blockIdx.x] = es;
            partial[2 * blockIdx.x + 1] = ws;
        }
    }
}

// Failure-detection self test: one bounded wait on an mbarrier phase that
// cannot complete (it expects 16 bytes that no copy delivers).  The wait
// gives up after its bound (~2^31 SM cycles, about a second), latches
// LJ_ERRBIT_TIMEOUT and the kernel returns: the path every bulk-copy wait of
// the force kernels takes when a copy never lands.
__global__ void k_wait_selftest(int32_t *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16u);
    __syncwarp();
    mbar_wait_bounded(&bar, 0u, err);
}

// Sum the per-CTA (energy, virial) partials in a fixed order.
__global__ void k_reduce_pairs(const double *__restrict__ partial, int n, double *__restrict__ out)
{
    __shared__ double se[kReduceThreads], sw[kReduceThreads];
    double e = 0.0, w = 0.0;
    for (int k = threadIdx.x; k < n; k += kReduceThreads) {
        e += partial[2 * k];
        w += partial[2 * k + 1];
    }
    se[threadIdx.x] = e;
    sw[threadIdx.x] = w;
    __syncthreads();
    for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            se[threadIdx.x] += se[threadIdx.x + s];
            sw[threadIdx.x] += sw[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = se[0];
        out[1] = sw[0];
    }
}

template <typename T, int MODE, bool ENERGY>
void *force_kernel_ptr()
{
    return (void *)k_force<T, MODE, ENERGY>;
}

template <typename T>
void *pick_kernel(int mode, bool energy)
{
    switch (mode * 2 + (energy ? 1 : 0)) {
        case 0: return force_kernel_ptr<T, 0, false>();
        case 1: return force_kernel_ptr<T, 0, true>();
        case 2: return force_kernel_ptr<T, 1, false>();
        case 3: return force_kernel_ptr<T, 1, true>();
        case 4: return force_kernel_ptr<T, 2, false>();
        default: return force_kernel_ptr<T, 2, true>();
    }
}

size_t force_smem_bytes(int cap, size_t vsize)
{
    size_t b = 2 * (size_t)cap * vsize;
    b += 2 * sizeof(ItemTable);
    b += 2 * sizeof(uint64_t);
    b += (3 * kTabMax + 2) * sizeof(int);
    b += 2 * (kConsumerWarps + 1) * sizeof(double) + 16;
    return b;
}

ForceParams make_params(const lj_ctx *c)
{
    ForceParams fp;
    fp.n = (int)c->p.n;
    fp.nc = c->nc;
    fp.run_len = c->run_len;
    fp.runs = c->runs;
    fp.nitems = c->nitems;
    fp.cap = c->cap;
    fp.cw = c->cw;
    const double eps = c->p.eps, sg = c->p.sigma, rc = c->p.rc;
    const double s6 = sg * sg * sg * sg * sg * sg;
    const double s12 = s6 * s6;
    fp.rc2 = rc * rc;
    fp.rc = rc;
    fp.a12 = 48.0 * eps * s12;
    fp.b6 = 24.0 * eps * s6;
    fp.c12 = 4.0 * eps * s12;
    fp.c6 = 4.0 * eps * s6;
    const double rci2 = 1.0 / (rc * rc);
    const double rci6 = rci2 * rci2 * rci2;
    fp.uc = rci6 * (fp.c12 * rci6 - fp.c6);               // U_LJ(rc)
    fp.fc = rc * rci2 * rci6 * (fp.a12 * rci6 - fp.b6);   // F_LJ(rc) = rc * (F/r)(rc)
    return fp;
}

}  // namespace

cudaError_t force_configure(lj_ctx *c)
{
    const size_t vsize = c->p.precision == LJ_PREC_FP64 ? sizeof(double4_16a) : sizeof(float4);
    c->run_len = c->nc < kRunMax ? c->nc : kRunMax;
    c->runs = (c->nc + c->run_len - 1) / c->run_len;
    int64_t nitems = (int64_t)c->nc * c->nc * c->runs;
    if (nitems > INT32_MAX) return cudaErrorInvalidValue;
    c->nitems = (int)nitems;
    // Staging capacity: twice the mean window population, at least 512.
    double mean = c->ncell > 0 ? (double)c->p.n / (double)c->ncell : 0.0;
    double want = 2.0 * 9.0 * (c->run_len + 2) * mean + 64.0;
    int cap = (int)want;
    cap = cap < 512 ? 512 : cap;
    size_t budget = (vsize == sizeof(float4)) ? 96 * 1024 : 160 * 1024;
    int cap_max = (int)((budget - force_smem_bytes(0, vsize)) / (2 * vsize));
    cap = cap > cap_max ? cap_max : cap;
    cap = (cap + 31) & ~31;
    c->cap = cap;
    c->force_smem = (int)force_smem_bytes(cap, vsize);
    int maxblk = 1 << 30;
    for (int mode = 0; mode < 3; mode++)
        for (int en = 0; en < 2; en++) {
            void *kern = vsize == sizeof(float4) ? pick_kernel<float>(mode, en != 0)
                                                 : pick_kernel<double>(mode, en != 0);
            cudaError_t e = raise_dyn_smem(kern, c->force_smem);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kForceThreads, c->force_smem);
            if (e != cudaSuccess) return e;
            if (nb < maxblk) maxblk = nb;
        }
    if (maxblk < 1) maxblk = 1;
    int64_t grid = (int64_t)maxblk * c->nsm;
    if (grid > c->nitems) grid = c->nitems;
    if (grid < 1) grid = 1;
    c->force_grid = (int)grid;
    return cudaSuccess;
}

cudaError_t launch_force(lj_ctx *c, void *f, bool energy)
{
    if (c->p.n == 0) return cudaSuccess;
    if (c->use_aop) return launch_force_aop(c, f, energy);   // sets npartial
    if (!c->use_run_kernel) {
        c->npartial = c->wforce_grid;
        return launch_force_warp(c, f, energy);
    }
    c->npartial = c->force_grid;
    ForceParams fp = make_params(c);
    const bool fp64 = c->p.precision == LJ_PREC_FP64;
    void *kern = fp64 ? pick_kernel<double>(c->p.shift_mode, energy) : pick_kernel<float>(c->p.shift_mode, energy);
    const void *pos = c->pos;
    const int32_t *start = c->start;
    double *partial = c->partial;
    int32_t *err = c->err;
    int use_tma = c->use_tma;
    void *args[] = {&fp, (void *)&pos, (void *)&start, &f, &partial, &err, &use_tma};
    if (c->timing && c->ev_used + 2 <= c->nev) cudaEventRecord(c->ev[c->ev_used], c->stream);
    cudaError_t e = cudaLaunchKernel(kern, dim3(c->force_grid), dim3(kForceThreads), args, c->force_smem, c->stream);
    if (c->timing && c->ev_used + 2 <= c->nev) {
        cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
        c->ev_used += 2;
    }
    c->kernel_launches++;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_energy_reduce(lj_ctx *c)
{
    k_reduce_pairs<<<1, kReduceThreads, 0, c->stream>>>(c->partial, c->npartial, c->scalars);
    c->kernel_launches++;
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(lj_ctx *c)
{
    k_wait_selftest<<<1, 32, 0, c->stream>>>(c->err);
    c->kernel_launches++;
    return cudaGetLastError();
}
