// Adjoint of the cell-list forces and of a velocity-Verlet step, for
// gradients with respect to positions and to the LJ parameters (eps, sigma).
// The paper has no adjoint; this is the derivative of its force (Eq.
// n2_force with the Section 2 pair force, rc held fixed):
//   F_i = sum_j phi(r_ij) d_ij,  phi = F(r)/r,  d_ij = x_i - x_j,
//   dL/dx_i   = sum_j J_ij (g_i - g_j),  J = phi I + (phi'(r)/r) d d^T,
//   dL/deps   = sum_i g_i . dF_i/deps   (F is linear in eps),
//   dL/dsigma = sum_i g_i . dF_i/dsigma,
// with g_i = dL/dF_i.  With q = r^2, phi = A q^-7 - B q^-4 (A = 48 eps
// sigma^12, B = 24 eps sigma^6), so phi'(r)/r = 2 dphi/dq = q^-5 (8B - 14A
// q^-3) and dphi/dsigma = (12 A q^-7 - 6 B q^-4) / sigma; the force shift
// (mode 2) adds -Fc / r, whose terms are +Fc / r^3 and -(dFc/dsigma) / r.
//
// Layout: one warp per home cell (persistent grid over cells), lanes own
// home particles (passes of 32), neighbour cells read from the sorted
// positions and sorted cotangents with the cell offset applied to the home
// particle.  Pair arithmetic in the context's precision; per-particle sums
// in that precision; parameter gradients reduced in FP64.
#include "lj_internal.cuh"

namespace {

constexpr int kVjpThreads = 256;

struct VjpCoef {
    double rc2, a1, b1, fc1, dfc1, eps, inv_sigma;
};

template <typename T>
__device__ __forceinline__ T rcp_t(T x)
{
    return (T)1 / x;
}

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x)
{
    return (T)1 / sqrt(x);
}

// Sorted cotangents: g4[slot] = g[perm[slot]] (w unused).
template <typename V>
__global__ void k_gather_cotangent(const double *__restrict__ g, const int32_t *__restrict__ perm, int n,
                                   V *__restrict__ g4)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm[s];
    V q;
    q.x = g[3 * i];
    q.y = g[3 * i + 1];
    q.z = g[3 * i + 2];
    q.w = 0;
    g4[s] = q;
}

template <typename T, int MODE, int R>
__global__ void __launch_bounds__(kVjpThreads) k_vjp(int n, int nc, int64_t ncell, double cw_d, VjpCoef kd,
                                                     const typename Vec4<T>::type *__restrict__ pos,
                                                     const typename Vec4<T>::type *__restrict__ g4,
                                                     const int32_t *__restrict__ start, double scale,
                                                     double *__restrict__ dx, double *__restrict__ partial)
{
    using V = typename Vec4<T>::type;
    constexpr int NS = Stencil<R>::NS;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const T cw = (T)cw_d, rc2 = (T)kd.rc2, a1 = (T)kd.a1, b1 = (T)kd.b1, fc1 = (T)kd.fc1, dfc1 = (T)kd.dfc1;
    const T eps = (T)kd.eps, isg = (T)kd.inv_sigma;
    double acc_e = 0.0, acc_s = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * (kVjpThreads / 32);
    // stencil entry kk of home cell (cx, cy, cz): first particle, count, shift
    auto entry = [&](int kk, int cx, int cy, int cz, int &s, int &nn, T &shx, T &shy, T &shz) {
        int ddx, ddy, ddz;
        stencil_delta<R>(kk, ddx, ddy, ddz);
        int ux = cx + ddx, uy = cy + ddy, uz = cz + ddz;
        ux += ux < 0 ? nc : 0;
        ux -= ux >= nc ? nc : 0;
        uy += uy < 0 ? nc : 0;
        uy -= uy >= nc ? nc : 0;
        uz += uz < 0 ? nc : 0;
        uz -= uz >= nc ? nc : 0;
        const int64_t cn = ux + (int64_t)nc * (uy + (int64_t)nc * uz);
        s = start[cn];
        nn = start[cn + 1] - s;
        shx = (T)ddx * cw;
        shy = (T)ddy * cw;
        shz = (T)ddz * cw;
    };
    for (int64_t c = (int64_t)blockIdx.x * (kVjpThreads / 32) + warp; c < ncell; c += nwarps) {
        const int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        int s_home, n_home;
        T h0, h1, h2;
        entry(0, cx, cy, cz, s_home, n_home, h0, h1, h2);
        for (int p0 = 0; p0 < n_home; p0 += 32) {
            const int i = p0 + lane;
            const bool vi = i < n_home;
            const V pi = pos[s_home + (vi ? i : 0)];
            const V gi = g4[s_home + (vi ? i : 0)];
            T ax = 0, ay = 0, az = 0;
            // Parameter sums over pairs: per stencil cell in the working
            // precision (a few dozen terms), then in FP64 across cells and
            // particles (the totals cancel).  One FP64 addition per stencil
            // cell, not per candidate: FP64 is rationed on this GPU.
            double ae = 0.0, as = 0.0;
            for (int kk = 0; kk < NS; kk++) {
                int s, nn;
                T shx, shy, shz;
                entry(kk, cx, cy, cz, s, nn, shx, shy, shz);
                const T xs = pi.x - shx;
                const T ys = pi.y - shy;
                const T zs = pi.z - shz;
                T ae_c = 0, as_c = 0;
                for (int j = 0; j < nn; j++) {
                    const V qj = pos[s + j];
                    const V gj = g4[s + j];
                    const T dx_ = xs - qj.x, dy_ = ys - qj.y, dz_ = zs - qj.z;
                    const T r2 = dx_ * dx_ + dy_ * dy_ + dz_ * dz_;
                    const bool in = (r2 < rc2) && (r2 > (T)0);
                    T ri, rinv = 0;
                    if constexpr (MODE == 2) {
                        rinv = in ? rsqrt_t<T>(r2) : (T)0;
                        ri = rinv * rinv;
                    } else {
                        ri = in ? rcp_t<T>(r2) : (T)0;
                    }
                    const T r6 = ri * ri * ri;
                    const T r8 = ri * r6;              // q^-4
                    T phi1 = r8 * (a1 * r6 - b1);      // phi with eps = 1
                    T dphi1 = r8 * ri * ((T)8 * b1 - (T)14 * a1 * r6);
                    T dsig1 = r8 * ((T)12 * a1 * r6 - (T)6 * b1) * isg;
                    if constexpr (MODE == 2) {
                        phi1 -= fc1 * rinv;
                        dphi1 += fc1 * rinv * rinv * rinv;
                        dsig1 -= dfc1 * rinv;
                    }
                    const T phi = eps * phi1, dphi = eps * dphi1;
                    const T gx = gi.x - gj.x, gy = gi.y - gj.y, gz = gi.z - gj.z;
                    const T dot = dx_ * gx + dy_ * gy + dz_ * gz;
                    const T gid = dx_ * gi.x + dy_ * gi.y + dz_ * gi.z;
                    ax += phi * gx + dphi * dot * dx_;
                    ay += phi * gy + dphi * dot * dy_;
                    az += phi * gz + dphi * dot * dz_;
                    ae_c += phi1 * gid;
                    as_c += eps * dsig1 * gid;
                }
                ae += (double)ae_c;
                as += (double)as_c;
            }
            if (vi) {
                int idx;
                if constexpr (sizeof(T) == 4) {
                    idx = __float_as_int(pi.w);
                } else {
                    idx = (int)pi.w;
                }
                if ((unsigned)idx < (unsigned)n) {
                    dx[3 * (int64_t)idx] += scale * (double)ax;
                    dx[3 * (int64_t)idx + 1] += scale * (double)ay;
                    dx[3 * (int64_t)idx + 2] += scale * (double)az;
                    acc_e += ae;
                    acc_s += as;
                }
            }
        }
    }
    __shared__ double red[2 * (kVjpThreads / 32)];
    for (int o = 16; o > 0; o >>= 1) {
        acc_e += __shfl_xor_sync(0xffffffffu, acc_e, o);
        acc_s += __shfl_xor_sync(0xffffffffu, acc_s, o);
    }
    if (lane == 0) {
        red[2 * warp] = acc_e;
        red[2 * warp + 1] = acc_s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0, s = 0.0;
        for (int q = 0; q < kVjpThreads / 32; q++) {
            e += red[2 * q];
            s += red[2 * q + 1];
        }
        partial[2 * blockIdx.x] = e;
        partial[2 * blockIdx.x + 1] = s;
    }
}

// dparam[k] += scale * sum of the partials (fixed order).
__global__ void k_accum_params(const double *__restrict__ partial, int np, double scale, double *__restrict__ dparam)
{
    __shared__ double se[kReduceThreads], ss[kReduceThreads];
    double e = 0.0, s = 0.0;
    for (int k = threadIdx.x; k < np; k += kReduceThreads) {
        e += partial[2 * k];
        s += partial[2 * k + 1];
    }
    se[threadIdx.x] = e;
    ss[threadIdx.x] = s;
    __syncthreads();
    for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            se[threadIdx.x] += se[threadIdx.x + w];
            ss[threadIdx.x] += ss[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dparam[0] += scale * se[0];
        dparam[1] += scale * ss[0];
    }
}

// y += a x over 3n doubles.
__global__ void k_axpy(double *__restrict__ y, const double *__restrict__ x, double a, int64_t m)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < m) y[q] = __fma_rn(a, x[q], y[q]);
}

template <typename T>
void *vjp_kernel(int mode, int subdiv)
{
    // modes 0 and 1 have the same force
    if (subdiv == 2) return mode == 2 ? (void *)k_vjp<T, 2, 2> : (void *)k_vjp<T, 0, 2>;
    return mode == 2 ? (void *)k_vjp<T, 2, 1> : (void *)k_vjp<T, 0, 1>;
}

}  // namespace

int vjp_grid(lj_ctx *c)
{
    int nb = 0;
    void *kern = c->p.precision == LJ_PREC_FP64 ? vjp_kernel<double>(c->p.shift_mode, c->p.cell_subdiv)
                                                : vjp_kernel<float>(c->p.shift_mode, c->p.cell_subdiv);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kVjpThreads, 0) != cudaSuccess || nb < 1) nb = 1;
    int64_t need = (c->ncell + kVjpThreads / 32 - 1) / (kVjpThreads / 32);
    int64_t grid = (int64_t)nb * c->nsm;
    if (grid > need) grid = need;
    return (int)(grid < 1 ? 1 : grid);
}

cudaError_t launch_vjp(lj_ctx *c, const double *g, double scale, double *dx, double *dparam)
{
    const int n = (int)c->p.n;
    if (n == 0) return cudaSuccess;
    const bool fp64 = c->p.precision == LJ_PREC_FP64;
    const unsigned gb = (unsigned)((n + 255) / 256);
    if (fp64)
        k_gather_cotangent<double4_16a><<<gb, 256, 0, c->stream>>>(g, c->perm, n, (double4_16a *)c->g4);
    else
        k_gather_cotangent<float4><<<gb, 256, 0, c->stream>>>(g, c->perm, n, (float4 *)c->g4);
    c->kernel_launches++;
    VjpCoef k;
    const double sg = c->p.sigma, rc = c->p.rc;
    const double s6 = sg * sg * sg * sg * sg * sg, s12 = s6 * s6;
    k.rc2 = rc * rc;
    k.a1 = 48.0 * s12;
    k.b1 = 24.0 * s6;
    k.fc1 = rc * (k.a1 * pow(rc, -14.0) - k.b1 * pow(rc, -8.0));
    k.dfc1 = rc * (12.0 * k.a1 * pow(rc, -14.0) - 6.0 * k.b1 * pow(rc, -8.0)) / sg;
    k.eps = c->p.eps;
    k.inv_sigma = 1.0 / sg;
    const int grid = vjp_grid(c);
    if (grid > c->npartial_cap) return cudaErrorInvalidValue;
    void *kern = fp64 ? vjp_kernel<double>(c->p.shift_mode, c->p.cell_subdiv)
                      : vjp_kernel<float>(c->p.shift_mode, c->p.cell_subdiv);
    int nc = c->nc;
    int64_t ncell = c->ncell;
    double cw = c->cw;
    const void *pos = c->pos;
    const void *g4 = c->g4;
    const int32_t *start = c->start;
    double *partial = c->partial;
    void *args[] = {(void *)&n, &nc, &ncell, &cw, &k, (void *)&pos, (void *)&g4, (void *)&start, &scale, &dx, &partial};
    cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(kVjpThreads), args, 0, c->stream);
    if (e != cudaSuccess) return e;
    k_accum_params<<<1, kReduceThreads, 0, c->stream>>>(c->partial, grid, scale, dparam);
    c->kernel_launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_axpy(lj_ctx *c, double *y, const double *x, double a)
{
    const int64_t m = 3 * c->p.n;
    if (m == 0) return cudaSuccess;
    k_axpy<<<(unsigned)((m + 255) / 256), 256, 0, c->stream>>>(y, x, a, m);
    c->kernel_launches++;
    return cudaGetLastError();
}
