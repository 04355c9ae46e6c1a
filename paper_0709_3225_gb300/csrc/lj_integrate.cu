// Velocity-Verlet integration (Section 2, last paragraph: the paper cites
// the standard scheme without printing it; read here as kick-drift-kick)
// fused with the first binning pass of the next force evaluation, and the
// kinetic-energy reduction.  All arithmetic on x and v is FP64; the force is
// read in the context's precision and promoted.
#include "lj_internal.cuh"

namespace {

template <typename F4>
__device__ __forceinline__ void load_f(const F4 *__restrict__ f, int i, double &fx, double &fy, double &fz)
{
    F4 q = f[i];
    fx = (double)q.x;
    fy = (double)q.y;
    fz = (double)q.z;
}

// nkick half kicks v += h f (1 on the first step of a call, 2 when the
// closing half kick of the previous step is fused in, applied as one FP64
// FMA with nkick*h), drift x += dt v (FP64 FMA), wrap into [0, L), cell id
// (exact, from the previous cell as a guess) and rank of the new position
// (one atomic per distinct cell per warp).  No FP64 division or multiply
// in the common path: this GPU's FP64 rate is a small fraction of FP32.
// One particle per thread (kKdbPer): two per thread, with all loads issued
// first, measured slower (114 against 101 us at 4M): each thread then runs
// two dependent chains of table lookups and atomics.
constexpr int kKdbPer = 1;

template <typename F4>
__global__ void __launch_bounds__(256) k_kick_drift_bin(double *__restrict__ x, double *__restrict__ v,
                                                        const F4 *__restrict__ f, int n, double hk, double dt,
                                                        double L, double whi, double wlo, double s, int nc,
                                                        float inv_nc, const long long *__restrict__ thb,
                                                        int32_t *__restrict__ cell_of, int32_t *__restrict__ rank,
                                                        int32_t *__restrict__ count, int32_t *__restrict__ err,
                                                        int i_begin)
{
    // particles i_begin .. n-1 (a chunk when the host copies arrive in parts)
    const int i0 = i_begin + blockIdx.x * (kKdbPer * blockDim.x) + threadIdx.x;
    double xr[kKdbPer][3], vr[kKdbPer][3], fr[kKdbPer][3];
    int old[kKdbPer];
#pragma unroll
    for (int u = 0; u < kKdbPer; u++) {
        const int i = i0 + u * blockDim.x;
        if (i < n) {
            const int64_t b = 3 * (int64_t)i;
            load_f(f, i, fr[u][0], fr[u][1], fr[u][2]);
            vr[u][0] = v[b];
            vr[u][1] = v[b + 1];
            vr[u][2] = v[b + 2];
            xr[u][0] = x[b];
            xr[u][1] = x[b + 1];
            xr[u][2] = x[b + 2];
            old[u] = cell_of[i];
        }
    }
#pragma unroll
    for (int u = 0; u < kKdbPer; u++) {
        const int i = i0 + u * blockDim.x;
        const bool valid = i < n;
        int c = 0;
        if (valid) {
            const int64_t b = 3 * (int64_t)i;
            const double vx = __fma_rn(hk, fr[u][0], vr[u][0]);
            const double vy = __fma_rn(hk, fr[u][1], vr[u][1]);
            const double vz = __fma_rn(hk, fr[u][2], vr[u][2]);
            const double px = lj_wrap_fast(__fma_rn(dt, vx, xr[u][0]), L, whi, wlo);
            const double py = lj_wrap_fast(__fma_rn(dt, vy, xr[u][1]), L, whi, wlo);
            const double pz = lj_wrap_fast(__fma_rn(dt, vz, xr[u][2]), L, whi, wlo);
            v[b] = vx;
            v[b + 1] = vy;
            v[b + 2] = vz;
            x[b] = px;
            x[b + 1] = py;
            x[b + 2] = pz;
            if (isfinite(px) && isfinite(py) && isfinite(pz)) {
                int ox, oy, oz;
                lj_cell_decode(old[u], nc, inv_nc, ox, oy, oz);
                c = lj_cell_from_guess(px, ox, thb, s, nc) +
                    nc * (lj_cell_from_guess(py, oy, thb, s, nc) + nc * lj_cell_from_guess(pz, oz, thb, s, nc));
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
}

// Skin mode (cell lists rebuilt only when needed): kick and drift as
// k_kick_drift_bin without binning; each particle's displacement since the
// last rebuild accumulates in FP32, and the largest |displacement|^2 goes
// to *maxd2 (float bits: non-negative floats order as their bit patterns).
template <typename F4>
__global__ void k_kick_drift_skin(double *__restrict__ x, double *__restrict__ v, const F4 *__restrict__ f, int n,
                                  double hk, double dt, double L, double whi, double wlo,
                                  float4 *__restrict__ disp, int32_t *maxd2, int32_t *__restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.f;
    if (i < n) {
        const int64_t b = 3 * (int64_t)i;
        double fx, fy, fz;
        load_f(f, i, fx, fy, fz);
        const double vx = __fma_rn(hk, fx, v[b]);
        const double vy = __fma_rn(hk, fy, v[b + 1]);
        const double vz = __fma_rn(hk, fz, v[b + 2]);
        const double px = lj_wrap_fast(__fma_rn(dt, vx, x[b]), L, whi, wlo);
        const double py = lj_wrap_fast(__fma_rn(dt, vy, x[b + 1]), L, whi, wlo);
        const double pz = lj_wrap_fast(__fma_rn(dt, vz, x[b + 2]), L, whi, wlo);
        v[b] = vx;
        v[b + 1] = vy;
        v[b + 2] = vz;
        x[b] = px;
        x[b + 1] = py;
        x[b + 2] = pz;
        if (!(isfinite(px) && isfinite(py) && isfinite(pz))) atomicOr(err, LJ_ERRBIT_NONFINITE);
        float4 d = disp[i];
        d.x += (float)(dt * vx);
        d.y += (float)(dt * vy);
        d.z += (float)(dt * vz);
        disp[i] = d;
        d2 = d.x * d.x + d.y * d.y + d.z * d.z;
        if (!(d2 <= 3.0e38f)) d2 = 3.0e38f;   // non-finite: force a rebuild
    }
    for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0 && d2 > 0.f) atomicMax(maxd2, __float_as_int(d2));
}

// One thread: decide whether this step rebuilds the cell lists (largest
// displacement past thr2, or max_interval steps since the last rebuild) and
// count.  flags: [0] max |disp|^2 bits, [1] rebuild, [2] steps since.
__global__ void k_skin_decide(int32_t *flags, long long *counts, float thr2, int max_interval)
{
    const int since = flags[2] + 1;
    const bool rebuild = __int_as_float(flags[0]) > thr2 || (max_interval > 0 && since >= max_interval);
    flags[1] = rebuild ? 1 : 0;
    if (rebuild) {
        flags[0] = 0;
        flags[2] = 0;
        counts[0] += 1;
    } else {
        flags[2] = since;
    }
    counts[1] += 1;
}

template <typename F4>
__global__ void k_kick(double *__restrict__ v, const F4 *__restrict__ f, int n, double h)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = 3 * (int64_t)i;
    double fx, fy, fz;
    load_f(f, i, fx, fy, fz);
    v[b] = __fma_rn(h, fx, v[b]);
    v[b + 1] = __fma_rn(h, fy, v[b + 1]);
    v[b + 2] = __fma_rn(h, fz, v[b + 2]);
}

// Per-block partial sums of v.v (grid-stride, fixed grid), then one block
// adds the partials in order: out = (1/2) m sum v^2.
__global__ void __launch_bounds__(kReduceThreads) k_vsq_partial(const double *__restrict__ v, int64_t m,
                                                                double *__restrict__ partial)
{
    __shared__ double s[kReduceThreads];
    double acc = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * kReduceThreads + threadIdx.x; q < m;
         q += (int64_t)gridDim.x * kReduceThreads)
        acc += v[q] * v[q];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(kReduceThreads) k_sum_scaled(const double *__restrict__ partial, int np,
                                                               double scale, double *__restrict__ out)
{
    __shared__ double s[kReduceThreads];
    double acc = 0.0;
    for (int q = threadIdx.x; q < np; q += kReduceThreads) acc += partial[q];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = scale * s[0];
}

// Observables from the FP64 sums (one thread): E_tot = E_kin + E_pot,
// T = 2 E_kin / (3n - 3) (k_B = 1; the total momentum is conserved, so
// 3n - 3 degrees of freedom; 0 for n < 2) and the virial pressure
// P = (2 E_kin + W) / (3V), inv3v = 1 / (3 L^3).
__global__ void k_observables(double *__restrict__ s, int64_t n, double inv3v)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double ep = s[0], w = s[1], ek = s[2];
        s[3] = ek + ep;
        s[4] = n >= 2 ? 2.0 * ek / (double)(3 * n - 3) : 0.0;
        s[5] = (2.0 * ek + w) * inv3v;
    }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_kick_drift_bin(lj_ctx *c, double *x, double *v, const void *f, int nkick, int64_t i_begin,
                                  int64_t i_end)
{
    const int n = (int)(i_end < 0 ? c->p.n : i_end);
    const int b0 = (int)i_begin;
    if (n <= b0) return cudaSuccess;
    const double hk = nkick * (0.5 * c->p.dt / c->p.mass);
    const unsigned grid = blocks_for(n - b0, kKdbPer * 256);
    if (c->p.precision == LJ_PREC_FP64)
        k_kick_drift_bin<double4_16a><<<grid, 256, 0, c->stream>>>(
            x, v, (const double4_16a *)f, n, hk, c->p.dt, c->p.box, c->wrap_hi, c->wrap_lo, c->inv_cw, c->nc,
            c->inv_nc_f, c->thb, c->cell_of, c->rank, c->count, c->err, b0);
    else
        k_kick_drift_bin<float4><<<grid, 256, 0, c->stream>>>(
            x, v, (const float4 *)f, n, hk, c->p.dt, c->p.box, c->wrap_hi, c->wrap_lo, c->inv_cw, c->nc,
            c->inv_nc_f, c->thb, c->cell_of, c->rank, c->count, c->err, b0);
    c->kernel_launches++;
    return cudaGetLastError();
}

cudaError_t launch_kick_drift_skin(lj_ctx *c, double *x, double *v, const void *f, int nkick)
{
    int n = (int)c->p.n;
    if (n == 0) return cudaSuccess;
    const double hk = nkick * (0.5 * c->p.dt / c->p.mass);
    if (c->p.precision == LJ_PREC_FP64)
        k_kick_drift_skin<double4_16a><<<blocks_for(n, 256), 256, 0, c->stream>>>(
            x, v, (const double4_16a *)f, n, hk, c->p.dt, c->p.box, c->wrap_hi, c->wrap_lo, c->disp,
            c->skin_flags, c->err);
    else
        k_kick_drift_skin<float4><<<blocks_for(n, 256), 256, 0, c->stream>>>(
            x, v, (const float4 *)f, n, hk, c->p.dt, c->p.box, c->wrap_hi, c->wrap_lo, c->disp, c->skin_flags,
            c->err);
    // rebuild once some particle has moved half the skin (slightly less, for
    // the FP32 displacement sums): then no pair within rc can have left the
    // stencil, whose cells are at least rc + skin wide
    const float thr = (float)(0.5 * c->skin * 0.999);
    k_skin_decide<<<1, 1, 0, c->stream>>>(c->skin_flags, c->skin_counts, thr * thr, c->skin_max_interval);
    c->kernel_launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_kick(lj_ctx *c, double *v, const void *f)
{
    int n = (int)c->p.n;
    if (n == 0) return cudaSuccess;
    const double h = 0.5 * c->p.dt / c->p.mass;
    if (c->p.precision == LJ_PREC_FP64)
        k_kick<double4_16a><<<blocks_for(n, 256), 256, 0, c->stream>>>(v, (const double4_16a *)f, n, h);
    else
        k_kick<float4><<<blocks_for(n, 256), 256, 0, c->stream>>>(v, (const float4 *)f, n, h);
    c->kernel_launches++;
    return cudaGetLastError();
}

cudaError_t launch_ekin(lj_ctx *c, const double *v)
{
    k_vsq_partial<<<c->ekin_grid, kReduceThreads, 0, c->stream>>>(v, 3 * c->p.n, c->ekin_partial);
    k_sum_scaled<<<1, kReduceThreads, 0, c->stream>>>(c->ekin_partial, c->ekin_grid, 0.5 * c->p.mass,
                                                      c->scalars + 2);
    c->kernel_launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_observables(lj_ctx *c)
{
    const double L = c->p.box;
    k_observables<<<1, 32, 0, c->stream>>>(c->scalars, c->p.n, 1.0 / (3.0 * L * L * L));
    c->kernel_launches++;
    return cudaGetLastError();
}
