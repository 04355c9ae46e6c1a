// Device code shared by the single-system and batched warp-per-cell force
// kernels (see lj_force_warp.cu for the design): the packed pair math, the
// stencil table, the staging of one home cell's stencil, the chunked
// compute phase and the plain fallback path.
#pragma once

#include "lj_internal.cuh"

namespace {

constexpr float kFar = 1.0e4f;   // padding candidate: r^2 ~ 1e8 > rc^2
constexpr int kStageBatch = 2;   // staging rounds whose loads are in flight together (measured: 2 > 4 > 1)

// Order-preserving map of a float's bits to a signed int (negative floats:
// magnitude bits flipped), so that the warp's integer min / max reductions
// (one instruction each) give the float min / max of a bounding box.
// An involution: f_unord undoes it.
__device__ __forceinline__ int f_ord(float f)
{
    const int i = __float_as_int(f);
    return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float f_unord(int i) { return __int_as_float(i ^ ((i >> 31) & 0x7fffffff)); }
__device__ __forceinline__ void box_reduce(float &bxl, float &byl, float &bzl, float &bxh, float &byh, float &bzh)
{
    bxl = f_unord(__reduce_min_sync(0xffffffffu, f_ord(bxl)));
    byl = f_unord(__reduce_min_sync(0xffffffffu, f_ord(byl)));
    bzl = f_unord(__reduce_min_sync(0xffffffffu, f_ord(bzl)));
    bxh = f_unord(__reduce_max_sync(0xffffffffu, f_ord(bxh)));
    byh = f_unord(__reduce_max_sync(0xffffffffu, f_ord(byh)));
    bzh = f_unord(__reduce_max_sync(0xffffffffu, f_ord(bzh)));
}

struct WarpParams {
    int n, nc, cap;              // cap: staged candidates per warp (multiple of 8, >= 40)
    int gw;                      // lane-group width: 0 compiled default, -1 per-cell choice, 2 .. 32 fixed
    int grab;                    // cells per pull from *work (0 = static striding)
    unsigned *work;              // work counter, zero at launch
    int64_t ncell;
    float cw;
    float rc2, rc, a12, b6, c12, c6, uc, fc;
    float inv_nc;                // 1 / nc (cell-id decoding of the pair-once kernel)
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

// 32-bit words of one warp's shared-memory slice: staged X, Y, Z (cap each),
// the stencil table (float4 per entry: shift xyz, start index) and the
// stencil prefix sums (NS + 1 ints, padded to 4).
__host__ __device__ constexpr int warp_slice_words(int cap, int R)
{
    return 3 * cap + 4 * (2 * R + 1) * (2 * R + 1) * (2 * R + 1) +
           (((2 * R + 1) * (2 * R + 1) * (2 * R + 1) + 1 + 3) & ~3);
}

// Compiled-in group width of the default kernels: 16 for the 27-cell
// stencil (~13 particles per cell), 4 for the 125-cell one (~1.7).
template <int R>
struct DefaultGroup {
    static constexpr int value = R == 1 ? 16 : 4;
};

// Lane-group width of the compute phase: the warp takes the home particles
// in chunks of G; lane g of a group owns particle g of the chunk and the
// S = 32 / G groups split the candidates (group s takes candidate pairs
// s, s + S, s + 2S, ...).  Automatic choice: the G in {2, 4, 8, 16} with the
// fewest candidate-pair iterations (a chunk's stream reduction and set-up
// count as about one iteration).
__device__ __forceinline__ int choose_group(int n_home, int T, int fixed)
{
    if (fixed > 0) return fixed;
    int best = 4, best_cost = 1 << 30;
#pragma unroll
    for (int lg = 1; lg <= 4; lg++) {
        const int G = 1 << lg;
        const int chunks = (n_home + G - 1) / G;
        const int cost = chunks * ((T * G + 63) / 64 + 1);
        if (cost < best_cost) {
            best_cost = cost;
            best = G;
        }
    }
    return best;
}

// Compute phase over the staged list: candidates 0 .. T-1 (home particles
// first, 0 .. n_home-1), padded with far points to a multiple of 2S.
// Home particle p sits at staged position p (coordinates in shared memory);
// its particle index is in lane p's hid for p < 32, else read from pos.
template <int G, int MODE, bool ENERGY, bool NC, class Out>
__device__ __forceinline__ void compute_chunks(const WarpParams &k, const float4 *__restrict__ pos, const Out &out,
                                               const float *X, const float *Y, const float *Z, int T, int s_home,
                                               int n_home, int hid, double &eacc, double &wacc)
{
    constexpr int S = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int sg = lane / G;
    const int iters = (T + 2 * S - 1) / (2 * S);
    const int ihome = (n_home + 2 * S - 1) / (2 * S);   // iterations that may hold i itself
    const float2 *X2 = reinterpret_cast<const float2 *>(X) + sg;
    const float2 *Y2 = reinterpret_cast<const float2 *>(Y) + sg;
    const float2 *Z2 = reinterpret_cast<const float2 *>(Z) + sg;
    for (int c0 = 0; c0 < n_home; c0 += G) {
        const int p = c0 + gl;
        const bool vi = p < n_home;
        const int pp = vi ? p : 0;
        const float2 xs = f2(X[pp]), ys = f2(Y[pp]), zs = f2(Z[pp]);
        int idx = __shfl_sync(0xffffffffu, hid, pp & 31);
        if (pp >= 32) idx = __float_as_int(load_pos<NC>(pos + s_home + pp).w);
        float2 fx = f2(0.f), fy = f2(0.f), fz = f2(0.f), e = f2(0.f), w = f2(0.f);
        int m = 0;
        for (; m < ihome; m++)
            pair2<MODE, ENERGY, true>(xs, ys, zs, X2[m * S], Y2[m * S], Z2[m * S], k, fx, fy, fz, e, w);
#pragma unroll 8
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
        out(idx, sg == 0 && vi, Fx, Fy, Fz, E, Wv, eacc, wacc);
    }
}

// Staged path.  The stencil's candidates are taken as one flat index space
// t = 0 .. Ttot-1 (lane l takes t = l, l + 32, ...; the stencil entry of t
// comes from warp votes for the 27-entry stencil and from a binary search of
// the prefix sums for the 125-entry one), converted to the home-cell
// frame and kept only if within rc of the home particles' bounding box (the
// margin covers FP32 rounding of the box test).  Kept candidates are
// appended in ballot order, so the home particles (entry 0, all inside the
// box) occupy 0 .. n_home-1.
// Returns false, having computed nothing, when the kept candidates would not
// fit the slice (then the caller takes the plain path).
template <int R, int MODE, bool ENERGY, bool NC, int GFIX, class Out>
__device__ __forceinline__ bool cell_staged(const WarpParams &k, const float4 *__restrict__ pos, const Out &out,
                                            float *X, float *Y, float *Z, const float4 *stab, const int *spre,
                                            int Ttot, int s_home, int n_home, double &eacc, double &wacc)
{
    constexpr int NS = Stencil<R>::NS, P2 = Stencil<R>::P2;
    const int lane = threadIdx.x & 31;
    float bxl = 3.4e38f, byl = 3.4e38f, bzl = 3.4e38f, bxh = -3.4e38f, byh = -3.4e38f, bzh = -3.4e38f;
    int hid = 0;   // particle index of home particle `lane`
    for (int p0 = 0; p0 < n_home; p0 += 32) {
        if (p0 + lane < n_home) {
            const float4 q = load_pos<NC>(pos + s_home + p0 + lane);
            if (p0 == 0) hid = __float_as_int(q.w);
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
    // Stencil entry of a candidate t.  With one entry per lane (NS <= 32) it
    // comes from warp votes instead of a search: lane e holds entry e's first
    // candidate s_e; the non-empty entries have distinct s_e, and the entry
    // of t is the last non-empty one with s_e <= t.  Per round of 32
    // candidates starting at tb, the non-empty entries with s_e <= tb are
    // counted (the last of them holds tb), and those starting inside the
    // round set bit s_e - tb of a mask, so lane l's entry is the
    // (count + set bits 1 .. l)-th non-empty entry; lane j holds the index
    // of the j-th non-empty entry (0 past their number), passed through the
    // X array before the staging fills it.
    [[maybe_unused]] int s_e = 0, j_entry = 0;
    [[maybe_unused]] bool ne = false;
    if constexpr (NS <= 32) {
        s_e = lane < NS ? spre[lane] : 0x7fffffff;
        ne = lane < NS && spre[lane + 1] > s_e;
        const unsigned nem = __ballot_sync(0xffffffffu, ne);
        if (ne) X[__popc(nem & lt)] = __int_as_float(lane);
        __syncwarp();
        j_entry = lane < __popc(nem) ? __float_as_int(X[lane]) : 0;
        __syncwarp();
    }
    const unsigned le = (2u << lane) - 1u;   // bits 0 .. lane
    int T = 0;
    // Batches of kStageBatch rounds: the stencil-entry lookups and the
    // position loads of a batch are issued before any of them is used,
    // so their latencies overlap.
    for (int t0 = 0; t0 < Ttot; t0 += 32 * kStageBatch) {
        float4 q[kStageBatch], sh[kStageBatch];
#pragma unroll
        for (int u = 0; u < kStageBatch; u++) {
            const int t = t0 + 32 * u + lane;
            int kc = 0, kb = 0;   // stencil entry of t and its prefix
            if constexpr (NS <= 32) {
                const int tb = t0 + 32 * u;
                const int o = s_e - tb;
                const unsigned inside = __reduce_or_sync(0xffffffffu, (ne && o >= 1 && o <= 31) ? (1u << o) : 0u);
                const int jc = __popc(__ballot_sync(0xffffffffu, ne && o <= 0)) - 1 + __popc(inside & le);
                kc = __shfl_sync(0xffffffffu, j_entry, jc & 31);
                kb = __shfl_sync(0xffffffffu, s_e, kc);
            }
            q[u] = make_float4(kFar, kFar, kFar, 0.f);
            sh[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (t < Ttot) {
                if constexpr (NS > 32) {
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
                }
                sh[u] = stab[kc];
                q[u] = load_pos<NC>(pos + __float_as_int(sh[u].w) + (t - kb));
            }
        }
        bool full = false;
#pragma unroll
        for (int u = 0; u < kStageBatch; u++) {
            if (T + 64 > k.cap) {   // this round (<= 32) plus the padding might not fit
                full = true;
                break;
            }
            const int t = t0 + 32 * u + lane;
            const float cx = q[u].x + sh[u].x;
            const float cy = q[u].y + sh[u].y;
            const float cz = q[u].z + sh[u].z;
            const float dx = fmaxf(fmaxf(bxl - cx, cx - bxh), 0.f);
            const float dy = fmaxf(fmaxf(byl - cy, cy - byh), 0.f);
            const float dz = fmaxf(fmaxf(bzl - cz, cz - bzh), 0.f);
            const bool keep = t < Ttot && dx * dx + dy * dy + dz * dz < rcut2;
            const unsigned kept = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int sl = T + __popc(kept & lt);
                X[sl] = cx;
                Y[sl] = cy;
                Z[sl] = cz;
            }
            T += __popc(kept);
        }
        if (full) {
            __syncwarp();   // the slice is rewritten by the next cell
            return false;
        }
    }
    X[T + lane] = kFar;   // padding up to the next multiple of 2S (T + 32 <= cap)
    Y[T + lane] = kFar;
    Z[T + lane] = kFar;
    __syncwarp();
    if constexpr (GFIX > 0) {
        // one compiled group width: a single compute path keeps the kernel
        // small and its registers unspilled (measured faster than choosing
        // per cell)
        compute_chunks<GFIX, MODE, ENERGY, NC>(k, pos, out, X, Y, Z, T, s_home, n_home, hid, eacc, wacc);
    } else {
        switch (choose_group(n_home, T, k.gw)) {
            case 2: compute_chunks<2, MODE, ENERGY, NC>(k, pos, out, X, Y, Z, T, s_home, n_home, hid, eacc, wacc); break;
            case 4: compute_chunks<4, MODE, ENERGY, NC>(k, pos, out, X, Y, Z, T, s_home, n_home, hid, eacc, wacc); break;
            case 8: compute_chunks<8, MODE, ENERGY, NC>(k, pos, out, X, Y, Z, T, s_home, n_home, hid, eacc, wacc); break;
            case 16: compute_chunks<16, MODE, ENERGY, NC>(k, pos, out, X, Y, Z, T, s_home, n_home, hid, eacc, wacc); break;
            default: compute_chunks<32, MODE, ENERGY, NC>(k, pos, out, X, Y, Z, T, s_home, n_home, hid, eacc, wacc); break;
        }
    }
    return true;
}

// Plain path: any occupancy; each stencil cell read from global memory with
// the home particle shifted into that cell's frame.
template <int R, int MODE, bool ENERGY, bool NC, class Out>
__device__ void cell_plain(const WarpParams &k, const float4 *__restrict__ pos, const Out &out, const float4 *stab,
                           const int *spre, int s_home, int n_home, double &eacc, double &wacc)
{
    constexpr int NS = Stencil<R>::NS;
    const int lane = threadIdx.x & 31;
    for (int p0 = 0; p0 < n_home; p0 += 32) {
        const int i = p0 + lane;
        const bool vi = i < n_home;
        const float4 pi = load_pos<NC>(pos + s_home + (vi ? i : 0));
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f, w = 0.f;
        for (int kk = 0; kk < NS; kk++) {
            const float4 sh = stab[kk];
            const int s = __float_as_int(sh.w);
            const int nn = spre[kk + 1] - spre[kk];
            const float xs = pi.x - sh.x;
            const float ys = pi.y - sh.y;
            const float zs = pi.z - sh.z;
            for (int j = 0; j < nn; j++) {
                const float4 q = load_pos<NC>(pos + s + j);
                pair1<MODE, ENERGY>(xs - q.x, ys - q.y, zs - q.z, k, fx, fy, fz, e, w);
            }
        }
        out(__float_as_int(pi.w), vi, fx, fy, fz, e, w, eacc, wacc);
    }
}

// Stencil table of home cell (cx, cy, cz) in a grid of nc^3 cells whose
// linear ids start at cell_base in start[] (0 for a single system), cell
// side cw: per stencil entry kk the shift to the home frame and the first
// particle, stab[kk] = (dx cw, dy cw, dz cw, start), and the exclusive
// prefix sums of the entries' counts, spre[0 .. NS].  With s64 it also
// writes the shifts in FP64, s64[kk], s64[NS + kk], s64[2 NS + kk] (cell
// side cw64).  Returns the stencil population spre[NS].  Called by all 32
// lanes; the table is visible to the warp on return.
template <int R>
__device__ __forceinline__ int stencil_table(const int32_t *__restrict__ start, int64_t cell_base, int cx, int cy,
                                             int cz, int nc, float cw, float4 *stab, int *spre,
                                             double *s64 = nullptr, double cw64 = 0.0)
{
    constexpr int NS = Stencil<R>::NS;
    const int lane = threadIdx.x & 31;
    int carry = 0;
#pragma unroll 1
    for (int b0 = 0; b0 < NS; b0 += 32) {
        const int kk = b0 + lane;
        int nn = 0;
        if (kk < NS) {
            int dx, dy, dz;
            stencil_delta<R>(kk, dx, dy, dz);
            int ux = cx + dx, uy = cy + dy, uz = cz + dz;
            ux += ux < 0 ? nc : 0;
            ux -= ux >= nc ? nc : 0;
            uy += uy < 0 ? nc : 0;
            uy -= uy >= nc ? nc : 0;
            uz += uz < 0 ? nc : 0;
            uz -= uz >= nc ? nc : 0;
            const int64_t cn = cell_base + ux + (int64_t)nc * (uy + (int64_t)nc * uz);
            const int s = start[cn];
            nn = start[cn + 1] - s;
            stab[kk] = make_float4((float)dx * cw, (float)dy * cw, (float)dz * cw, __int_as_float(s));
            if (s64) {
                s64[kk] = (double)dx * cw64;
                s64[NS + kk] = (double)dy * cw64;
                s64[2 * NS + kk] = (double)dz * cw64;
            }
        }
        int P = nn;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, P, o);
            if (lane >= o) P += y;
        }
        if (kk < NS) spre[kk] = carry + P - nn;
        carry += __shfl_sync(0xffffffffu, P, 31);
    }
    if (lane == 0) spre[NS] = carry;
    __syncwarp();
    return carry;
}

// One home cell at cell coordinates (cx, cy, cz) of a grid of nc^3 cells
// whose linear ids start at cell_base in start[] (0 for a single system),
// cell side cw.  Builds the stencil table in the warp's slice and runs the
// staged path, or the plain path when the stencil does not fit the slice.
template <int R, int MODE, bool ENERGY, bool NC, int GFIX, class Out>
__device__ __forceinline__ void process_home_cell(const WarpParams &k, const float4 *__restrict__ pos,
                                                  const int32_t *__restrict__ start, const Out &out_in,
                                                  float *slice, int cx, int cy, int cz, int nc, int64_t cell_base,
                                                  float cw, double &eacc, double &wacc)
{
    constexpr int NS = Stencil<R>::NS;
    Out out = out_in;
    out.set_home(cx, cy, cz);
    float *X = slice;
    float *Y = X + k.cap;
    float *Z = Y + k.cap;
    float4 *stab = reinterpret_cast<float4 *>(Z + k.cap);
    int *spre = reinterpret_cast<int *>(stab + NS);
    __syncwarp();   // the slice still holds the previous cell's data
    const int carry = stencil_table<R>(start, cell_base, cx, cy, cz, nc, cw, stab, spre);
    const int n_home = spre[1];
    if (n_home == 0) return;
    const int s_home = __float_as_int(stab[0].w);
    // Staged unless even the pruned stencil clearly cannot fit; the staging
    // itself gives up (and the plain path runs) if the kept candidates do not.
    if (carry <= 2 * k.cap &&
        cell_staged<R, MODE, ENERGY, NC, GFIX>(k, pos, out, X, Y, Z, stab, spre, carry, s_home, n_home, eacc, wacc))
        return;
    cell_plain<R, MODE, ENERGY, NC>(k, pos, out, stab, spre, s_home, n_home, eacc, wacc);
}

// Kernel parameters of a context: geometry, tuning and the pair coefficients
// in FP32 (U = c12 r^-12 - c6 r^-6, F/r = r^-2 (a12 r^-12 - b6 r^-6)).
inline WarpParams warp_params_of(const lj_ctx *c)
{
    WarpParams k;
    k.gw = c->gw;
    k.grab = c->grab;
    k.work = c->work;
    k.n = (int)c->p.n;
    k.nc = c->nc;
    k.cap = c->wcap;
    k.ncell = c->ncell;
    k.cw = (float)c->cw;
    const double eps = c->p.eps, sg = c->p.sigma, rc = c->p.rc;
    const double s6 = sg * sg * sg * sg * sg * sg, s12 = s6 * s6;
    const double rci2 = 1.0 / (rc * rc), rci6 = rci2 * rci2 * rci2;
    k.rc2 = (float)(rc * rc);
    k.rc = (float)rc;
    k.a12 = (float)(48.0 * eps * s12);
    k.b6 = (float)(24.0 * eps * s6);
    k.c12 = (float)(4.0 * eps * s12);
    k.c6 = (float)(4.0 * eps * s6);
    k.uc = (float)(rci6 * (4.0 * eps * s12 * rci6 - 4.0 * eps * s6));
    k.fc = (float)(rc * rci2 * rci6 * (48.0 * eps * s12 * rci6 - 24.0 * eps * s6));
    return k;
}

}  // namespace
