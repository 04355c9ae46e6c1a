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
// closing half kick of the previous step is fused in), drift x += dt v, wrap
// into [0, L), cell id and rank (atomic count) of the new position.
template <typename F4>
__global__ void k_kick_drift_bin(double *__restrict__ x, double *__restrict__ v, const F4 *__restrict__ f, int n,
                                 double h, double dt, int nkick, double L, double s, int nc,
                                 int32_t *__restrict__ cell_of, int32_t *__restrict__ rank,
                                 int32_t *__restrict__ count, int32_t *__restrict__ err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = 3 * (int64_t)i;
    double fx, fy, fz;
    load_f(f, i, fx, fy, fz);
    double vx = v[b], vy = v[b + 1], vz = v[b + 2];
    for (int k = 0; k < nkick; k++) {
        vx = __dadd_rn(vx, __dmul_rn(h, fx));
        vy = __dadd_rn(vy, __dmul_rn(h, fy));
        vz = __dadd_rn(vz, __dmul_rn(h, fz));
    }
    double px = lj_wrap(__dadd_rn(x[b], __dmul_rn(dt, vx)), L);
    double py = lj_wrap(__dadd_rn(x[b + 1], __dmul_rn(dt, vy)), L);
    double pz = lj_wrap(__dadd_rn(x[b + 2], __dmul_rn(dt, vz)), L);
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) atomicOr(err, LJ_ERRBIT_NONFINITE);
    v[b] = vx;
    v[b + 1] = vy;
    v[b + 2] = vz;
    x[b] = px;
    x[b + 1] = py;
    x[b + 2] = pz;
    int c = lj_cell1(px, s, nc) + nc * (lj_cell1(py, s, nc) + nc * lj_cell1(pz, s, nc));
    cell_of[i] = c;
    rank[i] = atomicAdd(count + c, 1);
}

template <typename F4>
__global__ void k_kick(double *__restrict__ v, const F4 *__restrict__ f, int n, double h)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = 3 * (int64_t)i;
    double fx, fy, fz;
    load_f(f, i, fx, fy, fz);
    v[b] = __dadd_rn(v[b], __dmul_rn(h, fx));
    v[b + 1] = __dadd_rn(v[b + 1], __dmul_rn(h, fy));
    v[b + 2] = __dadd_rn(v[b + 2], __dmul_rn(h, fz));
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

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_kick_drift_bin(lj_ctx *c, double *x, double *v, const void *f, int nkick)
{
    int n = (int)c->p.n;
    if (n == 0) return cudaSuccess;
    const double h = 0.5 * c->p.dt / c->p.mass;
    if (c->p.precision == LJ_PREC_FP64)
        k_kick_drift_bin<double4_16a><<<blocks_for(n, 256), 256, 0, c->stream>>>(
            x, v, (const double4_16a *)f, n, h, c->p.dt, nkick, c->p.box, c->inv_cw, c->nc, c->cell_of, c->rank,
            c->count, c->err);
    else
        k_kick_drift_bin<float4><<<blocks_for(n, 256), 256, 0, c->stream>>>(
            x, v, (const float4 *)f, n, h, c->p.dt, nkick, c->p.box, c->inv_cw, c->nc, c->cell_of, c->rank,
            c->count, c->err);
    c->kernel_launches++;
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
