// Device code shared by the single-system and batched warp-per-cell force
// kernels (see lj_force_warp.cu for the design): the packed pair math, the
// staging of one home cell's stencil and the plain fallback path.
#pragma once

#include "lj_internal.cuh"

namespace {

constexpr float kFar = 1.0e4f;   // padding candidate: r^2 ~ 1e8 > rc^2

struct WarpParams {
    int n, nc, cap;              // cap: staged candidates per warp (multiple of 8)
    int gmin;                    // smallest lane-group width to use (0, 8, 16 or 32)
    int grab;                    // cells per pull from *work (0 = static striding)
    unsigned *work;              // work counter, zero at launch
    int64_t ncell;
    float cw;
    float rc2, rc, a12, b6, c12, c6, uc, fc;
};

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Position loads: read-only path (NC) when the sorted positions are not
// written during the launch, plain coherent loads otherwise (the batched
// persistent kernel writes them in an earlier phase of the same launch).
template <bool NC>
__device__ __forceinline__ float4 load_pos(const float4 *p)
{
    if constexpr (NC) {
        return __ldg(p);
    } else {
        return *p;
    }
}

// Two candidate pairs at once: d = x_i - x_j for j = a, b; see lj_force.cu
// for the scalar form.  SELF adds the r^2 > 0 test that drops i == j.
template <int MODE, bool ENERGY, bool SELF>
__device__ __forceinline__ void pair2(float2 xs, float2 ys, float2 zs, float2 qx, float2 qy, float2 qz,
                                      const WarpParams &k, float2 &fx, float2 &fy, float2 &fz, float2 &e,
                                      float2 &w)
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
    const float2 t = __ffma2_rn(f2(k.a12), r6, f2(-k.b6));
    float2 ff = __fmul2_rn(__fmul2_rn(ri, r6), t);
    if constexpr (MODE == 2) ff = __ffma2_rn(f2(-k.fc), rinv, ff);
    fx = __ffma2_rn(ff, dx, fx);
    fy = __ffma2_rn(ff, dy, fy);
    fz = __ffma2_rn(ff, dz, fz);
    if constexpr (ENERGY) {
        float2 u = __fmul2_rn(r6, __ffma2_rn(f2(k.c12), r6, f2(-k.c6)));
        if constexpr (MODE >= 1) u = __fadd2_rn(u, f2(-k.uc));
        if constexpr (MODE == 2) u = __ffma2_rn(__ffma2_rn(r2, rinv, f2(-k.rc)), f2(k.fc), u);
        u.x = ina ? u.x : 0.0f;
        u.y = inb ? u.y : 0.0f;
        e = __fadd2_rn(e, u);
        w = __ffma2_rn(ff, r2, w);
    }
}

// Scalar pair for the plain path (per stencil cell, shifted home particle).
template <int MODE, bool ENERGY>
__device__ __forceinline__ void pair1(float dx, float dy, float dz, const WarpParams &k, float &fx, float &fy,
                                      float &fz, float &e, float &w)
{
    const float r2 = dx * dx + dy * dy + dz * dz;
    const bool in = (r2 < k.rc2) && (r2 > 0.0f);
    float ri, rinv = 0.0f;
    if constexpr (MODE == 2) {
        rinv = in ? rsqrt_approx(r2) : 0.0f;
        ri = rinv * rinv;
    } else {
        ri = in ? rcp_approx(r2) : 0.0f;
    }
    const float r6 = ri * ri * ri;
    float ff = ri * r6 * (k.a12 * r6 - k.b6);
    if constexpr (MODE == 2) ff -= k.fc * rinv;
    fx += ff * dx;
    fy += ff * dy;
    fz += ff * dz;
    if constexpr (ENERGY) {
        float u = r6 * (k.c12 * r6 - k.c6);
        if constexpr (MODE >= 1) u -= k.uc;
        if constexpr (MODE == 2) u += (r2 * rinv - k.rc) * k.fc;
        e += in ? u : 0.0f;
        w += ff * r2;
    }
}

// Stencil slot k = 0 is the home cell, k = 1..26 the neighbours.
__device__ __forceinline__ void stencil_offset(int k, int &dx, int &dy, int &dz)
{
    const int idx = k == 0 ? 13 : (k <= 13 ? k - 1 : k);
    dx = idx % 3 - 1;
    dy = (idx / 3) % 3 - 1;
    dz = idx / 9 - 1;
}

// Position of flat candidate j in the interleaved SoA layout for S streams.
template <int S>
__device__ __forceinline__ int slot_of(int j)
{
    const int m = j / (2 * S);
    const int r = j - m * 2 * S;
    const int s = r % S;
    const int h = r / S;
    return 2 * (m * S + s) + h;
}

// Output of one home particle's result, called by all 32 lanes of the warp
// (valid = this lane holds a particle's final sums).  StoreForce writes the
// force (and its energy share); KickDriftBin applies the velocity-Verlet
// update of that particle instead (see k_force_warp).
template <int MODE, bool ENERGY>
struct StoreForce {
    float4 *fout;
    int n;
    __device__ __forceinline__ void set_home(int, int, int) {}
    __device__ __forceinline__ void operator()(int idx, bool valid, float fx, float fy, float fz, float e, float w,
                                               double &eacc, double &wacc) const
    {
        if (valid && (unsigned)idx < (unsigned)n) {
            fout[idx] = make_float4(fx, fy, fz, ENERGY ? 0.5f * e : 0.0f);
            if constexpr (ENERGY) {
                eacc += 0.5 * (double)e;
                wacc += 0.5 * (double)w;
            }
        }
    }
};

// Velocity-Verlet update fused behind the force (FP64 state):
//   last == 0: v += hk f (the closing half kick of this step and the opening
//              half kick of the next, hk = dt/m), x += dt v, wrap, new cell
//              (the home cell is the guess) and rank for the next binning;
//   last != 0: v += hk f (hk = dt/2m) and f is stored (the end of lj_step).
struct KickDriftBin {
    float4 *fout;
    int n;
    double *x, *v;
    double hk, dt, L, whi, wlo, s;
    int nc, last;
    const long long *thb;
    int32_t *cell_of, *rank, *count, *err;
    int hx, hy, hz;
    __device__ __forceinline__ void set_home(int cx, int cy, int cz)
    {
        hx = cx;
        hy = cy;
        hz = cz;
    }
    __device__ __forceinline__ void operator()(int idx, bool valid, float fx, float fy, float fz, float, float,
                                               double &, double &) const
    {
        valid = valid && (unsigned)idx < (unsigned)n;
        int c = 0;
        if (valid) {
            const int64_t b = 3 * (int64_t)idx;
            const double vx = __fma_rn(hk, (double)fx, v[b]);
            const double vy = __fma_rn(hk, (double)fy, v[b + 1]);
            const double vz = __fma_rn(hk, (double)fz, v[b + 2]);
            v[b] = vx;
            v[b + 1] = vy;
            v[b + 2] = vz;
            if (last) {
                fout[idx] = make_float4(fx, fy, fz, 0.0f);
            } else {
                const double px = lj_wrap_fast(__fma_rn(dt, vx, x[b]), L, whi, wlo);
                const double py = lj_wrap_fast(__fma_rn(dt, vy, x[b + 1]), L, whi, wlo);
                const double pz = lj_wrap_fast(__fma_rn(dt, vz, x[b + 2]), L, whi, wlo);
                x[b] = px;
                x[b + 1] = py;
                x[b + 2] = pz;
                if (isfinite(px) && isfinite(py) && isfinite(pz)) {
                    c = lj_cell_from_guess(px, hx, thb, s, nc) +
                        nc * (lj_cell_from_guess(py, hy, thb, s, nc) + nc * lj_cell_from_guess(pz, hz, thb, s, nc));
                } else {
                    atomicOr(err, LJ_ERRBIT_NONFINITE);
                    c = nc * nc * nc;   // the extra cell
                }
            }
        }
        if (!last) {
            const int r = lj_warp_rank(count, c, valid);
            if (valid) {
                cell_of[idx] = c;
                rank[idx] = r;
            }
        }
    }
};

// Fast path: staged flat list, G lanes per group, S = 32 / G groups.
template <int G, int MODE, bool ENERGY, bool NC, class Out>
__device__ __forceinline__ void cell_staged(const WarpParams &k, const float4 *__restrict__ pos, const Out &out,
                                            float *X, float *Y, float *Z, int s_k,
                                            int n_k, float sx, float sy, float sz, int s_home, int n_home,
                                            double &eacc, double &wacc)
{
    constexpr int S = 32 / G;
    const int lane = threadIdx.x & 31;
    // Home particles (lane e holds home particle e) and their bounding box in
    // the home-centre frame.  Stencil candidates farther than rc from the box
    // cannot interact with any home particle and are not staged (the margin
    // covers FP32 rounding of the box test).
    const bool hl = lane < n_home;
    const float4 ph = load_pos<NC>(pos + s_home + (hl ? lane : 0));
    float bxl = hl ? ph.x : 3.4e38f, byl = hl ? ph.y : 3.4e38f, bzl = hl ? ph.z : 3.4e38f;
    float bxh = hl ? ph.x : -3.4e38f, byh = hl ? ph.y : -3.4e38f, bzh = hl ? ph.z : -3.4e38f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bxl = fminf(bxl, __shfl_xor_sync(0xffffffffu, bxl, o));
        byl = fminf(byl, __shfl_xor_sync(0xffffffffu, byl, o));
        bzl = fminf(bzl, __shfl_xor_sync(0xffffffffu, bzl, o));
        bxh = fmaxf(bxh, __shfl_xor_sync(0xffffffffu, bxh, o));
        byh = fmaxf(byh, __shfl_xor_sync(0xffffffffu, byh, o));
        bzh = fmaxf(bzh, __shfl_xor_sync(0xffffffffu, bzh, o));
    }
    // stage the home cell first (candidates 0 .. n_home-1, all kept)
    if (hl) {
        const int sl = slot_of<S>(lane);
        X[sl] = ph.x;
        Y[sl] = ph.y;
        Z[sl] = ph.z;
    }
    // then lane k = 1..26 walks stencil cell k; kept candidates are appended
    // in ballot order
    const float rcut2 = k.rc2 * 1.0001f;
    const int my_n = (lane >= 1 && lane < 27) ? n_k : 0;
    const unsigned lt = (1u << lane) - 1u;
    int T = n_home;
    for (int e = 0; __any_sync(0xffffffffu, e < my_n); e++) {
        bool keep = false;
        float cx = 0.f, cy = 0.f, cz = 0.f;
        if (e < my_n) {
            const float4 q = load_pos<NC>(pos + s_k + e);
            cx = q.x + sx;
            cy = q.y + sy;
            cz = q.z + sz;
            const float dx = fmaxf(fmaxf(bxl - cx, cx - bxh), 0.f);
            const float dy = fmaxf(fmaxf(byl - cy, cy - byh), 0.f);
            const float dz = fmaxf(fmaxf(bzl - cz, cz - bzh), 0.f);
            keep = dx * dx + dy * dy + dz * dz < rcut2;
        }
        const unsigned kept = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int sl = slot_of<S>(T + __popc(kept & lt));
            X[sl] = cx;
            Y[sl] = cy;
            Z[sl] = cz;
        }
        T += __popc(kept);
    }
    const int Tpad = (T + 2 * S - 1) / (2 * S) * (2 * S);
    if (lane < Tpad - T) {
        const int sl = slot_of<S>(T + lane);
        X[sl] = kFar;
        Y[sl] = kFar;
        Z[sl] = kFar;
    }
    __syncwarp();

    const int gl = lane % G;
    const int sg = lane / G;
    const bool vi = gl < n_home;
    const float4 pi = make_float4(__shfl_sync(0xffffffffu, ph.x, gl), __shfl_sync(0xffffffffu, ph.y, gl),
                                  __shfl_sync(0xffffffffu, ph.z, gl), __shfl_sync(0xffffffffu, ph.w, gl));
    const float2 xs = f2(pi.x), ys = f2(pi.y), zs = f2(pi.z);
    float2 fx = f2(0.f), fy = f2(0.f), fz = f2(0.f), e = f2(0.f), w = f2(0.f);
    const int iters = Tpad / (2 * S);
    const int ihome = (n_home + 2 * S - 1) / (2 * S);   // iterations that may hold i itself
    const float2 *X2 = reinterpret_cast<const float2 *>(X) + sg;
    const float2 *Y2 = reinterpret_cast<const float2 *>(Y) + sg;
    const float2 *Z2 = reinterpret_cast<const float2 *>(Z) + sg;
    int m = 0;
    for (; m < ihome; m++)
        pair2<MODE, ENERGY, true>(xs, ys, zs, X2[m * S], Y2[m * S], Z2[m * S], k, fx, fy, fz, e, w);
#pragma unroll 4
    for (; m < iters; m++)
        pair2<MODE, ENERGY, false>(xs, ys, zs, X2[m * S], Y2[m * S], Z2[m * S], k, fx, fy, fz, e, w);
    float Fx = fx.x + fx.y, Fy = fy.x + fy.y, Fz = fz.x + fz.y, E = e.x + e.y, Wv = w.x + w.y;
#pragma unroll
    for (int o = G; o < 32; o <<= 1) {
        Fx += __shfl_xor_sync(0xffffffffu, Fx, o);
        Fy += __shfl_xor_sync(0xffffffffu, Fy, o);
        Fz += __shfl_xor_sync(0xffffffffu, Fz, o);
        if constexpr (ENERGY) {
            E += __shfl_xor_sync(0xffffffffu, E, o);
            Wv += __shfl_xor_sync(0xffffffffu, Wv, o);
        }
    }
    out(__float_as_int(pi.w), sg == 0 && vi, Fx, Fy, Fz, E, Wv, eacc, wacc);
    __syncwarp();   // the slice is reused by the next cell
}

// Plain path: any occupancy; each stencil cell read from global memory with
// the home particle shifted into that cell's frame.
template <int MODE, bool ENERGY, bool NC, class Out>
__device__ void cell_plain(const WarpParams &k, const float4 *__restrict__ pos, const Out &out, int s_k,
                           int n_k, float sx, float sy, float sz, int s_home, int n_home, double &eacc, double &wacc)
{
    const int lane = threadIdx.x & 31;
    for (int p0 = 0; p0 < n_home; p0 += 32) {
        const int i = p0 + lane;
        const bool vi = i < n_home;
        const float4 pi = load_pos<NC>(pos + s_home + (vi ? i : 0));
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f, w = 0.f;
        for (int kk = 0; kk < 27; kk++) {
            const int s = __shfl_sync(0xffffffffu, s_k, kk);
            const int nn = __shfl_sync(0xffffffffu, n_k, kk);
            const float xs = pi.x - __shfl_sync(0xffffffffu, sx, kk);
            const float ys = pi.y - __shfl_sync(0xffffffffu, sy, kk);
            const float zs = pi.z - __shfl_sync(0xffffffffu, sz, kk);
            for (int j = 0; j < nn; j++) {
                const float4 q = load_pos<NC>(pos + s + j);
                pair1<MODE, ENERGY>(xs - q.x, ys - q.y, zs - q.z, k, fx, fy, fz, e, w);
            }
        }
        out(__float_as_int(pi.w), vi, fx, fy, fz, e, w, eacc, wacc);
    }
}

// One home cell at cell coordinates (cx, cy, cz) of a grid of nc^3 cells
// whose linear ids start at cell_base in start[] (0 for a single system),
// cell side cw.  Builds the 27-cell stencil table in lanes 0..26 and runs
// the staged or the plain path.
template <int MODE, bool ENERGY, bool NC, class Out>
__device__ __forceinline__ void process_home_cell(const WarpParams &k, const float4 *__restrict__ pos,
                                                  const int32_t *__restrict__ start, const Out &out_in,
                                                  float *X, float *Y, float *Z, int cx, int cy, int cz, int nc,
                                                  int64_t cell_base, float cw, double &eacc, double &wacc)
{
    Out out = out_in;
    out.set_home(cx, cy, cz);
    const int lane = threadIdx.x & 31;
    int s_k = 0, n_k = 0;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    if (lane < 27) {
        int dx, dy, dz;
        stencil_offset(lane, dx, dy, dz);
        int ux = cx + dx, uy = cy + dy, uz = cz + dz;
        ux += ux < 0 ? nc : 0;
        ux -= ux >= nc ? nc : 0;
        uy += uy < 0 ? nc : 0;
        uy -= uy >= nc ? nc : 0;
        uz += uz < 0 ? nc : 0;
        uz -= uz >= nc ? nc : 0;
        const int64_t cn = cell_base + ux + (int64_t)nc * (uy + (int64_t)nc * uz);
        s_k = start[cn];
        n_k = start[cn + 1] - s_k;
        sx = (float)dx * cw;
        sy = (float)dy * cw;
        sz = (float)dz * cw;
    }
    int P = n_k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, P, o);
        if (lane >= o) P += y;
    }
    const int T = __shfl_sync(0xffffffffu, P, 31);
    const int s_home = __shfl_sync(0xffffffffu, s_k, 0);
    const int n_home = __shfl_sync(0xffffffffu, n_k, 0);
    if (n_home == 0) return;
    if (n_home <= 32 && T + 8 <= k.cap) {
        const int need = n_home > k.gmin ? n_home : k.gmin;
        if (need <= 8)
            cell_staged<8, MODE, ENERGY, NC>(k, pos, out, X, Y, Z, s_k, n_k, sx, sy, sz, s_home, n_home, eacc, wacc);
        else if (need <= 16)
            cell_staged<16, MODE, ENERGY, NC>(k, pos, out, X, Y, Z, s_k, n_k, sx, sy, sz, s_home, n_home, eacc, wacc);
        else
            cell_staged<32, MODE, ENERGY, NC>(k, pos, out, X, Y, Z, s_k, n_k, sx, sy, sz, s_home, n_home, eacc, wacc);
    } else {
        cell_plain<MODE, ENERGY, NC>(k, pos, out, s_k, n_k, sx, sy, sz, s_home, n_home, eacc, wacc);
    }
}

}  // namespace
