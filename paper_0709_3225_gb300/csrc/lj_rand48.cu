// rand48 random numbers on the GPU (Section 4) and the Langevin thermostat
// step that consumes them.
//
// Generator (Section 4, Eq. lrand48): x_{n+1} = (a x_n + c) mod 2^48 with
// the rand48 constants a = 0x5DEECE66D, c = 0xB.  Parallel rule (Eq.
// lrand48m): x_{n+m} = (A x_n + C) mod 2^48, A = a^m, C = c (1 + a + ...
// + a^{m-1}).  S streams: stream i holds the series element x_{k+i+1}
// that it outputs next, and steps by m = S, so that round r of all streams
// writes elements r S + i -- the serial series in order, coalesced.  On
// GB300 one 64-bit integer holds the 48-bit state (the paper's 24 + 24-bit
// split was a workaround for 32-bit integer hardware); the jump constants
// for any m come from squaring the affine map, O(log m).
//
// Langevin step (the stochastic thermostat named in Section 1; scheme
// BAOAB): B v += (dt/2m) f, A x += (dt/2) v, O v = c1 v + c2 sqrt(kT/m) xi,
// A x += (dt/2) v, wrap, bin; after the force the closing B.  xi from
// Box-Muller on four uniforms per particle and step: stream i is particle
// i, S = n, and step s uses series elements (4 s + k) n + i + 1, k = 0..3.
#include "lj_internal.cuh"

namespace {

constexpr uint64_t kA48 = 0x5DEECE66DULL;
constexpr uint64_t kC48 = 0xBULL;
constexpr uint64_t kMask48 = (1ULL << 48) - 1ULL;

// (A, C) of m steps: the affine map x -> a x + c composed m times, by
// binary powering (compose(p, q) applies q first: (Ap Aq, Ap Cq + Cp)).
__host__ __device__ inline void r48_jump(uint64_t m, uint64_t &A, uint64_t &C)
{
    uint64_t ra = 1, rc = 0;            // result
    uint64_t pa = kA48, pc = kC48;      // map^(2^bit)
    while (m) {
        if (m & 1ULL) {
            rc = (pa * rc + pc) & kMask48;
            ra = (pa * ra) & kMask48;
        }
        pc = (pa * pc + pc) & kMask48;
        pa = (pa * pa) & kMask48;
        m >>= 1;
    }
    A = ra;
    C = rc;
}

__device__ __forceinline__ uint64_t r48_next(uint64_t x, uint64_t A, uint64_t C)
{
    return (A * x + C) & kMask48;
}

// x 2^-48 exactly, assembled from the bits with integer operations (this
// GPU's FP64 conversion and multiply run at a small fraction of its integer
// rate): highest set bit e gives the exponent e - 48, the bits below it the
// mantissa.
__device__ __forceinline__ double r48_to_double(uint64_t x)
{
    if (x == 0) return 0.0;
    const int e = 63 - __clzll((long long)x);   // 0 .. 47
    const uint64_t mant = (x << (52 - e)) & ((1ULL << 52) - 1ULL);
    return __longlong_as_double((long long)((((uint64_t)(e - 48 + 1023)) << 52) | mant));
}

// state[i] = x_{i+1} of the series from x0 (i < S).
__global__ void k_r48_seed(uint64_t *__restrict__ state, int64_t S, uint64_t x0)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    uint64_t A, C;
    r48_jump((uint64_t)i + 1ULL, A, C);
    state[i] = r48_next(x0 & kMask48, A, C);
}

// out[r S + i] = Y(state_i), state_i -> state_i jumped by S, for r < R.
// DOUBLE: Y = x 2^-48 (drand48); else Y = x >> 17 (lrand48).
template <bool DOUBLE>
__global__ void k_r48_gen(uint64_t *__restrict__ state, int64_t S, int64_t R, uint64_t A, uint64_t C, void *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    uint64_t x = state[i];
    for (int64_t r = 0; r < R; r++) {
        if constexpr (DOUBLE) {
            reinterpret_cast<double *>(out)[r * S + i] = r48_to_double(x);
        } else {
            reinterpret_cast<int32_t *>(out)[r * S + i] = (int32_t)(x >> 17);
        }
        x = r48_next(x, A, C);
    }
    state[i] = x;
}

// Standard normals from pairs of uniforms in [0, 1) (Box-Muller), in T.
template <typename T>
__device__ __forceinline__ void box_muller(uint64_t a, uint64_t b, T &z0, T &z1)
{
    if constexpr (sizeof(T) == 4) {
        // 1 - u0 = y 2^-48 with y = 2^48 - a, formed from y's two 24-bit
        // halves (32-bit conversions, one FMA), so it keeps FP32 relative
        // precision down to 2^-48 (the logarithm's steep end); the angle
        // takes the 24 leading bits of b.
        const uint64_t y = (1ULL << 48) - a;
        const float w0 = fmaf((float)(uint32_t)(y & 0xFFFFFFu), 0x1p-24f, (float)(uint32_t)(y >> 24)) * 0x1p-24f;
        const float u1 = (float)(uint32_t)(b >> 24) * 0x1p-24f;
        const float r = sqrtf(-2.0f * logf(w0));
        float sn, cs;
        sincospif(2.0f * u1, &sn, &cs);
        z0 = r * cs;
        z1 = r * sn;
    } else {
        const double u0 = (double)a * 0x1p-48, u1 = (double)b * 0x1p-48;
        const double r = sqrt(-2.0 * log(1.0 - u0));
        double sn, cs;
        sincospi(2.0 * u1, &sn, &cs);
        z0 = r * cs;
        z1 = r * sn;
    }
}

template <typename F4, typename T>
__global__ void k_langevin_bin(double *__restrict__ x, double *__restrict__ v, const F4 *__restrict__ f, int n,
                               double hk, double hdt, double c1, double c2s, double L, double whi, double wlo,
                               double s, int nc, const long long *__restrict__ thb, uint64_t *__restrict__ state,
                               uint64_t A, uint64_t C, int32_t *__restrict__ cell_of, int32_t *__restrict__ rank,
                               int32_t *__restrict__ count, int32_t *__restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    int c = 0;
    if (valid) {
        // four series elements of this particle for this step
        const uint64_t u0 = state[i];
        const uint64_t u1 = r48_next(u0, A, C);
        const uint64_t u2 = r48_next(u1, A, C);
        const uint64_t u3 = r48_next(u2, A, C);
        state[i] = r48_next(u3, A, C);
        T z0, z1, z2, z3;
        box_muller<T>(u0, u1, z0, z1);
        box_muller<T>(u2, u3, z2, z3);
        (void)z3;
        const double xi[3] = {(double)z0, (double)z1, (double)z2};
        const int64_t b = 3 * (int64_t)i;
        const F4 q = f[i];
        const double fq[3] = {(double)q.x, (double)q.y, (double)q.z};
        double p[3];
        for (int d = 0; d < 3; d++) {
            double vv = __fma_rn(hk, fq[d], v[b + d]);
            double xx = __fma_rn(hdt, vv, x[b + d]);
            vv = __fma_rn(c2s, xi[d], c1 * vv);
            xx = __fma_rn(hdt, vv, xx);
            p[d] = lj_wrap_fast(xx, L, whi, wlo);
            v[b + d] = vv;
            x[b + d] = p[d];
        }
        if (isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2])) {
            const int old = cell_of[i];
            const int ox = old % nc, oy = (old / nc) % nc, oz = old / (nc * nc);
            c = lj_cell_from_guess(p[0], ox, thb, s, nc) +
                nc * (lj_cell_from_guess(p[1], oy, thb, s, nc) + nc * lj_cell_from_guess(p[2], oz, thb, s, nc));
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

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_langevin_bin(lj_ctx *c, double *x, double *v, const void *f, int nkick, double gamma, double kT)
{
    const int n = (int)c->p.n;
    if (n == 0) return cudaSuccess;
    const double dt = c->p.dt, m = c->p.mass;
    const double hk = nkick * (0.5 * dt / m);
    const double c1 = exp(-gamma * dt);
    const double c2s = sqrt(1.0 - c1 * c1) * sqrt(kT / m);
    uint64_t A, C;
    r48_jump((uint64_t)n, A, C);
    if (c->p.precision == LJ_PREC_FP64)
        k_langevin_bin<double4_16a, double><<<grid_for(n, 256), 256, 0, c->stream>>>(
            x, v, (const double4_16a *)f, n, hk, 0.5 * dt, c1, c2s, c->p.box, c->wrap_hi, c->wrap_lo, c->inv_cw,
            c->nc, c->thb, c->r48_state, A, C, c->cell_of, c->rank, c->count, c->err);
    else
        k_langevin_bin<float4, float><<<grid_for(n, 256), 256, 0, c->stream>>>(
            x, v, (const float4 *)f, n, hk, 0.5 * dt, c1, c2s, c->p.box, c->wrap_hi, c->wrap_lo, c->inv_cw, c->nc,
            c->thb, c->r48_state, A, C, c->cell_of, c->rank, c->count, c->err);
    c->kernel_launches++;
    return cudaGetLastError();
}

cudaError_t launch_r48_seed(uint64_t *state, int64_t S, uint64_t x0, cudaStream_t stream)
{
    if (S <= 0) return cudaSuccess;
    k_r48_seed<<<grid_for(S, 256), 256, 0, stream>>>(state, S, x0);
    return cudaGetLastError();
}

extern "C" int lj_rand48_jump(int64_t m, uint64_t *A, uint64_t *C)
{
    if (m < 0 || !A || !C) return LJ_EINVAL;
    r48_jump((uint64_t)m, *A, *C);
    return LJ_OK;
}

extern "C" uint64_t lj_srand48_state(int64_t seed)
{
    return ((((uint64_t)seed) & 0xFFFFFFFFULL) << 16) | 0x330EULL;
}

extern "C" int lj_rand48_seed(uint64_t *state, int64_t S, uint64_t x0, void *stream)
{
    if (S < 0) return LJ_EINVAL;
    if (S == 0) return LJ_OK;
    int r = check_dev_ptr(state, 8);
    if (r) return r;
    return launch_r48_seed(state, S, x0, (cudaStream_t)stream) == cudaSuccess ? LJ_OK : LJ_ECUDA;
}

namespace {

int r48_generate(uint64_t *state, int64_t S, int64_t R, void *out, bool dbl, void *stream)
{
    if (S < 0 || R < 0) return LJ_EINVAL;
    if (S == 0 || R == 0) return LJ_OK;
    if (S > ((int64_t)1 << 40) / (R > 0 ? R : 1)) return LJ_EOVERFLOW;
    int r = check_dev_ptr(state, 8);
    if (r) return r;
    r = check_dev_ptr(out, dbl ? 8 : 4);
    if (r) return r;
    uint64_t A, C;
    r48_jump((uint64_t)S, A, C);
    if (dbl)
        k_r48_gen<true><<<grid_for(S, 256), 256, 0, (cudaStream_t)stream>>>(state, S, R, A, C, out);
    else
        k_r48_gen<false><<<grid_for(S, 256), 256, 0, (cudaStream_t)stream>>>(state, S, R, A, C, out);
    return cudaGetLastError() == cudaSuccess ? LJ_OK : LJ_ECUDA;
}

}  // namespace

extern "C" int lj_rand48_lrand(uint64_t *state, int64_t S, int64_t R, int32_t *out, void *stream)
{
    return r48_generate(state, S, R, out, false, stream);
}

extern "C" int lj_rand48_drand(uint64_t *state, int64_t S, int64_t R, double *out, void *stream)
{
    return r48_generate(state, S, R, out, true, stream);
}
