// All-pairs forces (Section 2, Eq. n2_force): every particle against every
// other at the minimum image, with the cutoff and the shift of the context.
// This is the paper's first GPU algorithm, kept as the GPU brute-force
// cross-check of the cell list and for the N^2-versus-cells break-even study.
//
// Organisation on GB300:
//  * A CTA of kN2Threads threads; thread t owns particle
//    i = blockIdx.x * kN2Threads + t.
//  * The j particles stream through shared memory in tiles of kN2Tile,
//    copied by cp.async.bulk (issued by thread 0, completing on an mbarrier,
//    two buffers, bounded waits).  This is the paper's "load a block of
//    particles into shared memory, synchronise, compute", with the copy
//    engine doing the loads while the threads compute on the other buffer.
//  * The grid is i-blocks x j-splits: split s takes tiles s, s + nsplit, ...,
//    so that small systems still fill the SMs.  The per-split partial forces
//    are summed in split order by k_n2_sum (deterministic).
//  * Coordinates are the wrapped positions minus L/2 (|x| <= L/2) in the
//    context's precision: absolute coordinates, as in the paper's N^2 code.
//    The minimum image is d -= L rint(d / L).
#include "lj_pair.cuh"

namespace {

constexpr int kN2Threads = 128;
constexpr int kN2Tile = 512;   // j particles per shared-memory tile

struct N2Params {
    int n, ntiles;
    double L, invL;
    double rc2, rc, a12, b6, c12, c6, uc, fc;
};

// pos[i] = (wrap(x_i) - L/2, i); non-finite coordinates latch LJ_ENONFINITE.
template <typename T>
__global__ void k_n2_prep(const double *__restrict__ x, int n, double L, double whi, double wlo,
                          typename Vec4<T>::type *__restrict__ pos, int32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double px = x[3 * (int64_t)i], py = x[3 * (int64_t)i + 1], pz = x[3 * (int64_t)i + 2];
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) atomicOr(err, LJ_ERRBIT_NONFINITE);
    const double h = 0.5 * L;
    typename Vec4<T>::type q;
    q.x = (T)(lj_wrap_fast(px, L, whi, wlo) - h);
    q.y = (T)(lj_wrap_fast(py, L, whi, wlo) - h);
    q.z = (T)(lj_wrap_fast(pz, L, whi, wlo) - h);
    if constexpr (sizeof(T) == 4) {
        q.w = __int_as_float(i);
    } else {
        q.w = (double)i;
    }
    pos[i] = q;
}

template <typename V>
__device__ __forceinline__ V load_shared(const V *p)
{
    return *p;
}

template <typename T>
__device__ __forceinline__ T rint_t(T v)
{
    if constexpr (sizeof(T) == 4) {
        return rintf(v);
    } else {
        return rint(v);
    }
}

// part[split * n + i] = (sum over this split's j of the pair force on i,
// half the pair energies of i); epart[cta] = (sum of half energies, half
// virials) of this CTA's particles, FP64.
template <typename T, int MODE, bool ENERGY>
__global__ void __launch_bounds__(kN2Threads) k_n2_force(N2Params p, const typename Vec4<T>::type *__restrict__ pos,
                                                         typename Vec4<T>::type *__restrict__ part,
                                                         double *__restrict__ epart, int32_t *err)
{
    using V = typename Vec4<T>::type;
    extern __shared__ __align__(128) unsigned char n2_smem[];
    V *buf0 = reinterpret_cast<V *>(n2_smem);
    V *buf1 = buf0 + kN2Tile;
    uint64_t *bars = reinterpret_cast<uint64_t *>(buf1 + kN2Tile);
    __shared__ int s_abort;
    __shared__ double red[2 * (kN2Threads / 32)];

    const int i = blockIdx.x * kN2Threads + threadIdx.x;
    const bool vi = i < p.n;
    V pi;
    if (vi) {
        pi = pos[i];
    } else {
        pi.x = pi.y = pi.z = (T)0;
        pi.w = (T)0;
    }
    const int split = blockIdx.y, nsplit = gridDim.y;
    const int mine = p.ntiles > split ? (p.ntiles - split + nsplit - 1) / nsplit : 0;
    auto issue = [&](int k, V *dst, uint64_t *bar) {
        const int t = split + k * nsplit;
        const int cnt = min(kN2Tile, p.n - t * kN2Tile);
        mbar_arrive_expect_tx(bar, (uint32_t)(cnt * sizeof(V)));
        bulk_g2s(dst, pos + (size_t)t * kN2Tile, (uint32_t)(cnt * sizeof(V)), bar);
    };
    if (threadIdx.x == 0) {
        s_abort = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (mine > 0) issue(0, buf0, &bars[0]);
        if (mine > 1) issue(1, buf1, &bars[1]);
    }
    const Coef<T> kc(p);
    const T L = (T)p.L, invL = (T)p.invL;
    T fx = 0, fy = 0, fz = 0, e = 0, w = 0;
    int k = 0;
    for (; k < mine; k++) {
        const int b = k & 1;
        V *buf = b ? buf1 : buf0;
        const int t = split + k * nsplit;
        const int cnt = min(kN2Tile, p.n - t * kN2Tile);
        if (!mbar_wait_bounded(&bars[b], (uint32_t)((k >> 1) & 1), err)) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        for (int j = 0; j < cnt; j++) {
            const V q = load_shared(buf + j);
            T dx = pi.x - q.x, dy = pi.y - q.y, dz = pi.z - q.z;
            dx -= L * rint_t(dx * invL);
            dy -= L * rint_t(dy * invL);
            dz -= L * rint_t(dz * invL);
            pair_accum<T, MODE, ENERGY>(dx, dy, dz, kc, fx, fy, fz, e, w);
        }
        __syncthreads();   // everyone is done with buffer b
        if (threadIdx.x == 0 && k + 2 < mine) {
            fence_proxy_async_smem();
            issue(k + 2, buf, &bars[b]);
        }
    }
    if (s_abort && threadIdx.x == 0) {
        // a wait gave up: wait once more (bounded) for the copies that may
        // still be in flight, tile k and tile k + 1, before the CTA's shared
        // memory goes away
        mbar_wait_bounded(&bars[k & 1], (uint32_t)((k >> 1) & 1), err);
        if (k + 1 < mine) mbar_wait_bounded(&bars[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1), err);
    }
    if (vi) {
        V o;
        o.x = fx;
        o.y = fy;
        o.z = fz;
        o.w = ENERGY ? (T)0.5 * e : (T)0;
        part[(size_t)split * p.n + i] = o;
    }
    if constexpr (ENERGY) {
        double de = vi ? 0.5 * (double)e : 0.0, dw = vi ? 0.5 * (double)w : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            de += __shfl_xor_sync(0xffffffffu, de, o);
            dw += __shfl_xor_sync(0xffffffffu, dw, o);
        }
        const int warp = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            red[2 * warp] = de;
            red[2 * warp + 1] = dw;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double es = 0.0, ws = 0.0;
            for (int q = 0; q < kN2Threads / 32; q++) {
                es += red[2 * q];
                ws += red[2 * q + 1];
            }
            const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
            epart[2 * cta] = es;
            epart[2 * cta + 1] = ws;
        }
    }
}

// f[i] = sum over splits s = 0 .. nsplit-1 (in order) of part[s * n + i].
template <typename T>
__global__ void k_n2_sum(const typename Vec4<T>::type *__restrict__ part, int nsplit, int n,
                         typename Vec4<T>::type *__restrict__ f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    typename Vec4<T>::type a = part[i];
    for (int s = 1; s < nsplit; s++) {
        const typename Vec4<T>::type b = part[(size_t)s * n + i];
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
    }
    f[i] = a;
}

// scalars[0..1] = sums of the (energy, virial) pairs of epart, fixed order.
__global__ void k_n2_energy(const double *__restrict__ epart, int m, double *__restrict__ scalars)
{
    __shared__ double se[256], sw[256];
    double e = 0.0, w = 0.0;
    for (int k = threadIdx.x; k < m; k += 256) {
        e += epart[2 * k];
        w += epart[2 * k + 1];
    }
    se[threadIdx.x] = e;
    sw[threadIdx.x] = w;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            se[threadIdx.x] += se[threadIdx.x + s];
            sw[threadIdx.x] += sw[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scalars[0] = se[0];
        scalars[1] = sw[0];
    }
}

template <typename T>
void *n2_kernel(int mode, bool energy)
{
    switch (mode * 2 + (energy ? 1 : 0)) {
        case 0: return (void *)k_n2_force<T, 0, false>;
        case 1: return (void *)k_n2_force<T, 0, true>;
        case 2: return (void *)k_n2_force<T, 1, false>;
        case 3: return (void *)k_n2_force<T, 1, true>;
        case 4: return (void *)k_n2_force<T, 2, false>;
        default: return (void *)k_n2_force<T, 2, true>;
    }
}

template <typename T>
cudaError_t run_n2(lj_ctx *c, const double *x, void *f, bool energy)
{
    using V = typename Vec4<T>::type;
    const int n = (int)c->p.n;
    const int iblocks = (n + kN2Threads - 1) / kN2Threads;
    const int ntiles = (n + kN2Tile - 1) / kN2Tile;
    int nsplit = (2 * c->nsm + iblocks - 1) / iblocks;
    nsplit = nsplit < 1 ? 1 : (nsplit > ntiles ? ntiles : nsplit);
    nsplit = nsplit > 64 ? 64 : nsplit;
    // scratch: sorted-free positions, per-split partials, per-CTA energy pairs
    const size_t need = (size_t)n * sizeof(V) * (size_t)(1 + nsplit) + 2 * sizeof(double) * (size_t)iblocks * nsplit;
    if (need > c->n2_bytes) {
        cudaFree(c->n2_scratch);
        c->n2_scratch = nullptr;
        c->n2_bytes = 0;
        cudaError_t e = cudaMalloc(&c->n2_scratch, need);
        if (e != cudaSuccess) return e;
        c->n2_bytes = need;
    }
    V *pos = reinterpret_cast<V *>(c->n2_scratch);
    V *part = pos + n;
    double *epart = reinterpret_cast<double *>(part + (size_t)n * nsplit);
    V *fo = reinterpret_cast<V *>(f);
    k_n2_prep<T><<<(n + 255) / 256, 256, 0, c->stream>>>(x, n, c->p.box, c->wrap_hi, c->wrap_lo, pos, c->err);
    N2Params p;
    p.n = n;
    p.ntiles = ntiles;
    p.L = c->p.box;
    p.invL = 1.0 / c->p.box;
    const double eps = c->p.eps, sg = c->p.sigma, rc = c->p.rc;
    const double s6 = sg * sg * sg * sg * sg * sg, s12 = s6 * s6;
    const double rci2 = 1.0 / (rc * rc), rci6 = rci2 * rci2 * rci2;
    p.rc2 = rc * rc;
    p.rc = rc;
    p.a12 = 48.0 * eps * s12;
    p.b6 = 24.0 * eps * s6;
    p.c12 = 4.0 * eps * s12;
    p.c6 = 4.0 * eps * s6;
    p.uc = rci6 * (p.c12 * rci6 - p.c6);
    p.fc = rc * rci2 * rci6 * (p.a12 * rci6 - p.b6);
    void *kern = n2_kernel<T>(c->p.shift_mode, energy);
    const int smem = 2 * kN2Tile * (int)sizeof(V) + 2 * (int)sizeof(uint64_t);
    cudaError_t e = raise_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    V *dst = nsplit == 1 ? fo : part;
    int32_t *err = c->err;
    void *args[] = {&p, (void *)&pos, (void *)&dst, (void *)&epart, (void *)&err};
    e = cudaLaunchKernel(kern, dim3(iblocks, nsplit), dim3(kN2Threads), args, smem, c->stream);
    if (e != cudaSuccess) return e;
    c->kernel_launches += 2;
    if (nsplit > 1) {
        k_n2_sum<T><<<(n + 255) / 256, 256, 0, c->stream>>>(part, nsplit, n, fo);
        c->kernel_launches++;
    }
    if (energy) {
        k_n2_energy<<<1, 256, 0, c->stream>>>(epart, iblocks * nsplit, c->scalars);
        c->kernel_launches++;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_forces_n2(lj_ctx *c, const double *x, void *f, bool energy)
{
    if (c->p.n == 0) return cudaSuccess;
    if (c->p.precision == LJ_PREC_FP64) return run_n2<double>(c, x, f, energy);
    return run_n2<float>(c, x, f, energy);
}
