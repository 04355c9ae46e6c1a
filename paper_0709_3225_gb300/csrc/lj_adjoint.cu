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
// Layout (FP64 contexts, k_vjp): one warp per home cell (persistent grid
// over cells), lanes own home particles (passes of 32), neighbour cells read
// from the sorted positions and sorted cotangents with the cell offset
// applied to the home particle; pair arithmetic and per-particle sums in
// FP64.  FP32-mixed contexts use the staged k_vjp_warp below.  Parameter
// gradients are reduced in FP64 in both.
#include "lj_force_cell.cuh"

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


// ---------------------------------------------------------------------------
// FP32-mixed VJP, staged like the warp force kernel (lj_force_cell.cuh): one
// warp per home cell builds the stencil table, stages the stencil's
// candidates (positions in the home frame and cotangents, SoA) after the
// bounding-box pruning, and takes the home particles in chunks of G lanes,
// the S = 32 / G lane groups splitting the candidates, two candidates per
// lane and step with packed FP32x2 arithmetic.  Parameter terms are summed
// in FP32 over 16 steps (32 candidates, a handful in range) and then in FP64.
// Cells whose pruned stencil does not fit the slice take the plain path.

constexpr int kVjpWarpThreads = 256;

struct VjpWarpCoef {
    float rc2, a1, b1, c8, c14, s12, s6, fc1, dfc1, eps, cw;
};

__host__ __device__ constexpr int vjp_slice_words(int cap, int R)
{
    return 6 * cap + 4 * (2 * R + 1) * (2 * R + 1) * (2 * R + 1) +
           (((2 * R + 1) * (2 * R + 1) * (2 * R + 1) + 1 + 3) & ~3);
}

// Two candidates (a, b) for home particle (xs, ys, zs) with cotangent
// (gix, giy, giz): accumulates J (g_i - g_j) into (ax, ay, az) and the
// parameter terms into te (d/deps) and ts (d/dsigma).
template <int MODE, bool SELF>
__device__ __forceinline__ void vjp_pair2(float2 xs, float2 ys, float2 zs, float2 gix, float2 giy, float2 giz,
                                          float2 qx, float2 qy, float2 qz, float2 hx, float2 hy, float2 hz,
                                          const VjpWarpCoef &k, float2 &ax, float2 &ay, float2 &az, float2 &te,
                                          float2 &ts)
{
    const float2 m1 = f2(-1.0f);
    const float2 dx = __ffma2_rn(qx, m1, xs);
    const float2 dy = __ffma2_rn(qy, m1, ys);
    const float2 dz = __ffma2_rn(qz, m1, zs);
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    bool ina = r2.x < k.rc2, inb = r2.y < k.rc2;
    if constexpr (SELF) {
        ina = ina && (r2.x > 0.0f);
        inb = inb && (r2.y > 0.0f);
    }
    float2 ri, rinv = f2(0.0f);
    if constexpr (MODE == 2) {
        rinv.x = ina ? rsqrt_approx(r2.x) : 0.0f;
        rinv.y = inb ? rsqrt_approx(r2.y) : 0.0f;
        ri = __fmul2_rn(rinv, rinv);
    } else {
        ri.x = ina ? rcp_approx(r2.x) : 0.0f;
        ri.y = inb ? rcp_approx(r2.y) : 0.0f;
    }
    const float2 r6 = __fmul2_rn(__fmul2_rn(ri, ri), ri);
    const float2 r8 = __fmul2_rn(ri, r6);                                    // q^-4
    float2 phi1 = __fmul2_rn(r8, __ffma2_rn(f2(k.a1), r6, f2(-k.b1)));       // phi at eps = 1
    float2 dphi1 = __fmul2_rn(__fmul2_rn(r8, ri), __ffma2_rn(f2(-k.c14), r6, f2(k.c8)));
    float2 dsig1 = __fmul2_rn(r8, __ffma2_rn(f2(k.s12), r6, f2(-k.s6)));     // includes 1/sigma
    if constexpr (MODE == 2) {
        phi1 = __ffma2_rn(f2(-k.fc1), rinv, phi1);
        dphi1 = __ffma2_rn(__fmul2_rn(f2(k.fc1), rinv), ri, dphi1);
        dsig1 = __ffma2_rn(f2(-k.dfc1), rinv, dsig1);
    }
    const float2 phi = __fmul2_rn(f2(k.eps), phi1);
    const float2 dphi = __fmul2_rn(f2(k.eps), dphi1);
    const float2 gx = __ffma2_rn(hx, m1, gix);
    const float2 gy = __ffma2_rn(hy, m1, giy);
    const float2 gz = __ffma2_rn(hz, m1, giz);
    const float2 dot = __ffma2_rn(dz, gz, __ffma2_rn(dy, gy, __fmul2_rn(dx, gx)));
    const float2 gid = __ffma2_rn(dz, giz, __ffma2_rn(dy, giy, __fmul2_rn(dx, gix)));
    const float2 t = __fmul2_rn(dphi, dot);
    ax = __ffma2_rn(t, dx, __ffma2_rn(phi, gx, ax));
    ay = __ffma2_rn(t, dy, __ffma2_rn(phi, gy, ay));
    az = __ffma2_rn(t, dz, __ffma2_rn(phi, gz, az));
    te = __ffma2_rn(phi1, gid, te);
    ts = __ffma2_rn(__fmul2_rn(f2(k.eps), dsig1), gid, ts);
}

// Plain path for one home cell: lanes own home particles; every stencil
// cell read from global memory with the home particle shifted into its
// frame.  Same sums as the staged path.
template <int R, int MODE>
__device__ void vjp_cell_plain(const VjpWarpCoef &k, int n, const float4 *__restrict__ pos,
                               const float4 *__restrict__ g4, const float4 *stab, const int *spre, int s_home,
                               int n_home, double scale, double *__restrict__ dxo, double &acc_e, double &acc_s)
{
    constexpr int NS = Stencil<R>::NS;
    const int lane = threadIdx.x & 31;
    for (int p0 = 0; p0 < n_home; p0 += 32) {
        const int i = p0 + lane;
        const bool vi = i < n_home;
        const float4 pi = pos[s_home + (vi ? i : 0)];
        const float4 gi = g4[s_home + (vi ? i : 0)];
        float2 ax = f2(0.f), ay = f2(0.f), az = f2(0.f);
        double ae = 0.0, as = 0.0;
        for (int kk = 0; kk < NS; kk++) {
            const float4 sh = stab[kk];
            const int s = __float_as_int(sh.w);
            const int nn = spre[kk + 1] - spre[kk];
            float2 te = f2(0.f), ts = f2(0.f);
            for (int j = 0; j < nn; j++) {
                const float4 q = pos[s + j];
                const float4 h = g4[s + j];
                vjp_pair2<MODE, true>(f2(pi.x), f2(pi.y), f2(pi.z), f2(gi.x), f2(gi.y), f2(gi.z),
                                      make_float2(q.x + sh.x, kFar), make_float2(q.y + sh.y, kFar),
                                      make_float2(q.z + sh.z, kFar), make_float2(h.x, 0.f), make_float2(h.y, 0.f),
                                      make_float2(h.z, 0.f), k, ax, ay, az, te, ts);
            }
            ae += (double)te.x;
            as += (double)ts.x;
        }
        const int idx = __float_as_int(pi.w);
        if (vi && (unsigned)idx < (unsigned)n) {
            dxo[3 * (int64_t)idx] += scale * (double)ax.x;
            dxo[3 * (int64_t)idx + 1] += scale * (double)ay.x;
            dxo[3 * (int64_t)idx + 2] += scale * (double)az.x;
            acc_e += ae;
            acc_s += as;
        }
    }
}

template <int R, int MODE>
__device__ __forceinline__ void vjp_cell(const VjpWarpCoef &k, int n, int cap, const float4 *__restrict__ pos,
                                         const float4 *__restrict__ g4, const int32_t *__restrict__ start,
                                         float *slice, int cx, int cy, int cz, int nc, double scale,
                                         double *__restrict__ dxo, double &acc_e, double &acc_s)
{
    constexpr int NS = Stencil<R>::NS, P2 = Stencil<R>::P2;
    constexpr int G = DefaultGroup<R>::value, S = 32 / G;
    const int lane = threadIdx.x & 31;
    float *X = slice;
    float *Y = X + cap;
    float *Z = Y + cap;
    float *HX = Z + cap;
    float *HY = HX + cap;
    float *HZ = HY + cap;
    float4 *stab = reinterpret_cast<float4 *>(HZ + cap);
    int *spre = reinterpret_cast<int *>(stab + NS);
    __syncwarp();   // the slice still holds the previous cell's data
    const int carry = stencil_table<R>(start, 0, cx, cy, cz, nc, k.cw, stab, spre);
    const int n_home = spre[1];
    if (n_home == 0) return;
    const int s_home = __float_as_int(stab[0].w);
    const int Ttot = carry;
    // bounding box of the home particles (home frame)
    float bxl = 3.4e38f, byl = 3.4e38f, bzl = 3.4e38f, bxh = -3.4e38f, byh = -3.4e38f, bzh = -3.4e38f;
    for (int p0 = 0; p0 < n_home; p0 += 32) {
        if (p0 + lane < n_home) {
            const float4 q = __ldg(pos + s_home + p0 + lane);
            bxl = fminf(bxl, q.x);
            byl = fminf(byl, q.y);
            bzl = fminf(bzl, q.z);
            bxh = fmaxf(bxh, q.x);
            byh = fmaxf(byh, q.y);
            bzh = fmaxf(bzh, q.z);
        }
    }
    box_reduce(bxl, byl, bzl, bxh, byh, bzh);
    const float rcut2 = k.rc2 * 1.0001f;
    const unsigned lt = (1u << lane) - 1u;
    int T = 0;
    bool fits = Ttot <= 2 * cap;
    for (int t0 = 0; fits && t0 < Ttot; t0 += 32) {
        if (T + 64 > cap) {   // this round (<= 32) plus the padding might not fit
            fits = false;
            break;
        }
        const int t = t0 + lane;
        float4 q = make_float4(kFar, kFar, kFar, 0.f), h = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < Ttot) {
            int kc = 0, kb = 0;
#pragma unroll
            for (int step = P2 / 2; step > 0; step >>= 1) {
                const int m = kc + step;
                if (m < NS) {
                    const int v = spre[m];
                    if (v <= t) {
                        kc = m;
                        kb = v;
                    }
                }
            }
            sh = stab[kc];
            const int idx = __float_as_int(sh.w) + (t - kb);
            q = __ldg(pos + idx);
            h = __ldg(g4 + idx);
        }
        const float cx = q.x + sh.x, cy = q.y + sh.y, cz = q.z + sh.z;
        const float ddx = fmaxf(fmaxf(bxl - cx, cx - bxh), 0.f);
        const float ddy = fmaxf(fmaxf(byl - cy, cy - byh), 0.f);
        const float ddz = fmaxf(fmaxf(bzl - cz, cz - bzh), 0.f);
        const bool keep = t < Ttot && ddx * ddx + ddy * ddy + ddz * ddz < rcut2;
        const unsigned kept = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int sl = T + __popc(kept & lt);
            X[sl] = cx;
            Y[sl] = cy;
            Z[sl] = cz;
            HX[sl] = h.x;
            HY[sl] = h.y;
            HZ[sl] = h.z;
        }
        T += __popc(kept);
    }
    if (!fits) {
        __syncwarp();
        vjp_cell_plain<R, MODE>(k, n, pos, g4, stab, spre, s_home, n_home, scale, dxo, acc_e, acc_s);
        return;
    }
    X[T + lane] = kFar;   // padding up to the next multiple of 2S (T + 32 <= cap)
    Y[T + lane] = kFar;
    Z[T + lane] = kFar;
    HX[T + lane] = 0.f;
    HY[T + lane] = 0.f;
    HZ[T + lane] = 0.f;
    __syncwarp();
    // compute: home particle p sits at staged position p, its cotangent too
    const int gl = lane % G;
    const int sg = lane / G;
    const int iters = (T + 2 * S - 1) / (2 * S);
    const int ihome = (n_home + 2 * S - 1) / (2 * S);
    const float2 *X2 = reinterpret_cast<const float2 *>(X) + sg;
    const float2 *Y2 = reinterpret_cast<const float2 *>(Y) + sg;
    const float2 *Z2 = reinterpret_cast<const float2 *>(Z) + sg;
    const float2 *HX2 = reinterpret_cast<const float2 *>(HX) + sg;
    const float2 *HY2 = reinterpret_cast<const float2 *>(HY) + sg;
    const float2 *HZ2 = reinterpret_cast<const float2 *>(HZ) + sg;
    for (int c0 = 0; c0 < n_home; c0 += G) {
        const int p = c0 + gl;
        const bool vi = p < n_home;
        const int pp = vi ? p : 0;
        const float2 xs = f2(X[pp]), ys = f2(Y[pp]), zs = f2(Z[pp]);
        const float2 gix = f2(HX[pp]), giy = f2(HY[pp]), giz = f2(HZ[pp]);
        float2 ax = f2(0.f), ay = f2(0.f), az = f2(0.f);
        double ae = 0.0, as = 0.0;
        int m = 0;
        {
            float2 te = f2(0.f), ts = f2(0.f);
            for (; m < ihome; m++)
                vjp_pair2<MODE, true>(xs, ys, zs, gix, giy, giz, X2[m * S], Y2[m * S], Z2[m * S], HX2[m * S],
                                      HY2[m * S], HZ2[m * S], k, ax, ay, az, te, ts);
            ae += (double)(te.x + te.y);
            as += (double)(ts.x + ts.y);
        }
        for (; m < iters; m += 16) {
            float2 te = f2(0.f), ts = f2(0.f);
#pragma unroll
            for (int u = 0; u < 16; u++) {
                if (m + u < iters)
                    vjp_pair2<MODE, false>(xs, ys, zs, gix, giy, giz, X2[(m + u) * S], Y2[(m + u) * S],
                                           Z2[(m + u) * S], HX2[(m + u) * S], HY2[(m + u) * S], HZ2[(m + u) * S], k,
                                           ax, ay, az, te, ts);
            }
            ae += (double)(te.x + te.y);
            as += (double)(ts.x + ts.y);
        }
        float Ax = ax.x + ax.y, Ay = ay.x + ay.y, Az = az.x + az.y;
#pragma unroll
        for (int o = G; o < 32; o <<= 1) {
            Ax += __shfl_xor_sync(0xffffffffu, Ax, o);
            Ay += __shfl_xor_sync(0xffffffffu, Ay, o);
            Az += __shfl_xor_sync(0xffffffffu, Az, o);
            ae += __shfl_xor_sync(0xffffffffu, ae, o);
            as += __shfl_xor_sync(0xffffffffu, as, o);
        }
        if (sg == 0 && vi) {
            const int idx = __float_as_int(__ldg(pos + s_home + p).w);
            if ((unsigned)idx < (unsigned)n) {
                dxo[3 * (int64_t)idx] += scale * (double)Ax;
                dxo[3 * (int64_t)idx + 1] += scale * (double)Ay;
                dxo[3 * (int64_t)idx + 2] += scale * (double)Az;
                acc_e += ae;
                acc_s += as;
            }
        }
    }
}

template <int R, int MODE>
__global__ void __launch_bounds__(kVjpWarpThreads, 3) k_vjp_warp(int n, int nc, int64_t ncell, int cap, VjpWarpCoef k,
                                                                 const float4 *__restrict__ pos,
                                                                 const float4 *__restrict__ g4,
                                                                 const int32_t *__restrict__ start, double scale,
                                                                 double *__restrict__ dxo, double *__restrict__ partial)
{
    extern __shared__ __align__(16) float vsmem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *slice = vsmem + (size_t)warp * vjp_slice_words(cap, R);
    double acc_e = 0.0, acc_s = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * (kVjpWarpThreads / 32);
    for (int64_t c = (int64_t)blockIdx.x * (kVjpWarpThreads / 32) + warp; c < ncell; c += nwarps) {
        const int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        vjp_cell<R, MODE>(k, n, cap, pos, g4, start, slice, cx, cy, cz, nc, scale, dxo, acc_e, acc_s);
    }
    __shared__ double red[2 * (kVjpWarpThreads / 32)];
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
        for (int q = 0; q < kVjpWarpThreads / 32; q++) {
            e += red[2 * q];
            s += red[2 * q + 1];
        }
        partial[2 * blockIdx.x] = e;
        partial[2 * blockIdx.x + 1] = s;
    }
}

void *vjp_warp_kernel(int mode, int subdiv)
{
    // modes 0 and 1 have the same force
    if (subdiv == 2) return mode == 2 ? (void *)k_vjp_warp<2, 2> : (void *)k_vjp_warp<2, 0>;
    return mode == 2 ? (void *)k_vjp_warp<1, 2> : (void *)k_vjp_warp<1, 0>;
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
    void *kern = vjp_kernel<double>(c->p.shift_mode, c->p.cell_subdiv);   // FP64 contexts
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kVjpThreads, 0) != cudaSuccess || nb < 1) nb = 1;
    int64_t need = (c->ncell + kVjpThreads / 32 - 1) / (kVjpThreads / 32);
    int64_t grid = (int64_t)nb * c->nsm;
    if (grid > need) grid = need;
    return (int)(grid < 1 ? 1 : grid);
}

namespace {

// FP32-mixed VJP through the staged warp kernel: slice capacity from the
// mean stencil population (as the force kernel), grid of resident CTAs.
cudaError_t launch_vjp_warp(lj_ctx *c, const VjpCoef &kd, double scale, double *dx, double *dparam)
{
    const int R = c->p.cell_subdiv == 2 ? 2 : 1;
    const int ns = (2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    const int warps = kVjpWarpThreads / 32;
    const double mean = c->ncell > 0 ? (double)c->p.n / (double)c->ncell : 0.0;
    const double m = (double)ns * mean;
    // 0.65 m + 3 sqrt(m) + 64: room for the ~0.64 m candidates the pruning
    // keeps plus the padding, small enough for 3 CTAs (24 warps) per SM;
    // a cell that overflows takes the plain path (measured: 2.46 -> 2.32 ms
    // at 4M against m + 4 sqrt(m) + 64 and 2 CTAs per SM)
    int cap = (((int)(0.65 * m + 3.0 * sqrt(m)) + 64) + 7) & ~7;
    const int limit = 227 * 1024 - 2 * warps * (int)sizeof(double) - 256;
    while (cap > 96 && warps * vjp_slice_words(cap, R) * (int)sizeof(float) > limit) cap -= 8;
    const int smem = warps * vjp_slice_words(cap, R) * (int)sizeof(float);
    void *kern = vjp_warp_kernel(c->p.shift_mode, R);
    cudaError_t e = raise_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kVjpWarpThreads, smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)(nb > 0 ? nb : 1) * c->nsm;
    const int64_t need = (c->ncell + warps - 1) / warps;
    if (grid > need) grid = need;
    if (grid > c->npartial_cap) grid = c->npartial_cap;
    if (grid < 1) grid = 1;
    VjpWarpCoef k;
    k.rc2 = (float)kd.rc2;
    k.a1 = (float)kd.a1;
    k.b1 = (float)kd.b1;
    k.c8 = (float)(8.0 * kd.b1);
    k.c14 = (float)(14.0 * kd.a1);
    k.s12 = (float)(12.0 * kd.a1 * kd.inv_sigma);
    k.s6 = (float)(6.0 * kd.b1 * kd.inv_sigma);
    k.fc1 = (float)kd.fc1;
    k.dfc1 = (float)kd.dfc1;
    k.eps = (float)kd.eps;
    k.cw = (float)c->cw;
    int n = (int)c->p.n, nc = c->nc;
    int64_t ncell = c->ncell;
    const float4 *pos = (const float4 *)c->pos;
    const float4 *g4 = (const float4 *)c->g4;
    const int32_t *start = c->start;
    double *partial = c->partial;
    void *args[] = {&n, &nc, &ncell, &cap, &k, (void *)&pos, (void *)&g4, (void *)&start, &scale, &dx, &partial};
    e = cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kVjpWarpThreads), args, smem, c->stream);
    if (e != cudaSuccess) return e;
    k_accum_params<<<1, kReduceThreads, 0, c->stream>>>(c->partial, (int)grid, scale, dparam);
    c->kernel_launches += 2;
    return cudaGetLastError();
}

}  // namespace

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
    if (!fp64 && uses_vjp_n3(c) && c->f_sorted) {
        // each pair once (lj_vjp_n3.cu); f_sorted is its float4 accumulator
        const double coef[7] = {k.rc2, k.a1, k.b1, k.fc1, k.dfc1, k.eps, k.inv_sigma};
        int grid = 0;
        cudaError_t e = launch_vjp_n3(c, coef, scale, dx, (float4 *)c->f_sorted, &grid);
        if (e != cudaSuccess) return e;
        k_accum_params<<<1, kReduceThreads, 0, c->stream>>>(c->partial, grid, scale, dparam);
        c->kernel_launches++;
        return cudaGetLastError();
    }
    if (!fp64) return launch_vjp_warp(c, k, scale, dx, dparam);
    if (c->p.cell_subdiv != 2 && c->wcap > 0 && c->w64_lcap > 0) {
        // FP64: the warp kernel with compacted in-range pair lists
        int grid = 0;
        cudaError_t e = launch_vjp_w64(c, scale, dx, k.a1, k.b1, k.fc1, k.dfc1, &grid);
        if (e != cudaSuccess) return e;
        k_accum_params<<<1, kReduceThreads, 0, c->stream>>>(c->partial, grid, scale, dparam);
        c->kernel_launches++;
        return cudaGetLastError();
    }
    const int grid = vjp_grid(c);
    if (grid > c->npartial_cap) return cudaErrorInvalidValue;
    void *kern = vjp_kernel<double>(c->p.shift_mode, c->p.cell_subdiv);
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
