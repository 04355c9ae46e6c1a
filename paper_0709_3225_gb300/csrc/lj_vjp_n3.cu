// Vector-Jacobian product of the forces with each pair once (FP32-mixed).
//
// For cotangents g = dL/dF the VJP is, per particle, dL/dx_i = sum_j J_ij
// (g_i - g_j) with J_ij = phi I + (phi'/r) d d^T, phi = F(r)/r and d = x_i -
// x_j (the derivative of Eq. n2_force with the Section 2 pair force, rc
// held fixed), plus the parameter terms dL/deps = sum_pairs phi|eps=1 d.(g_i
// - g_j) and dL/dsigma = sum_pairs eps dphi/dsigma d.(g_i - g_j).  J_ij is
// even in d, so particle j receives the negative of particle i's term: as
// in the pair-once force kernel (lj_force_n3.cuh), a home cell is paired
// with itself (pairs i < j) and its 13 forward neighbours, every pair is
// evaluated once, and the term is added to i and subtracted from j.
//
// Organisation (the force kernel's, with cotangents):
//  * staging: the half stencil's candidates, pruned against the home box,
//    into S (x, y, z in the home frame, particle index) and SG (the
//    candidates' cotangents, from the cell-ordered copy g4);
//  * compute: lane (a, b) of A groups of B lanes takes candidate b of each
//    block against the home particles u A + a in FP32x2 pairs, whose
//    positions and cotangents are read from a per-warp table at every
//    evaluation; the term accumulates for the home pair in registers and as
//    the candidate's reaction, which goes out by float4 atomic adds (one per
//    pair of lane groups) into a particle-order FP32 buffer; the home sums
//    follow through a transpose in S;
//  * the parameter terms are summed per lane in FP32 over a cell and then
//    in FP64;
//  * cells with more than 32 home particles or an overflowing pruned list
//    take a plain path over global memory.
// A last kernel adds scale times the buffer to dL/dx (FP64).  The sums of
// a particle are formed in an order set by the atomics (not bitwise
// reproducible; the deterministic in-cell mode keeps the 27-cell VJP).
#include <math.h>

#include "lj_force_n3.cuh"

namespace {

constexpr int kVn3Threads = 128;              // 4 warps per CTA
constexpr int kVn3HomeStride = 2 * (4 + 2) + 1;   // float4 per lane group in the home table

struct VjpN3Coef {
    float rc2, a1, b1, c8, c14, s12, s6, fc1, dfc1, eps, cw, inv_nc;
    int n, nc, cap, grab;
    int64_t ncell;
    unsigned *work;
};

// Words of a warp's slice: S and SG (cap float4 each), the half-stencil
// table (14 float4), its prefix sums (16 int), the home table (4 groups x
// kVn3HomeStride float4).
__host__ __device__ constexpr int vn3_slice_words(int cap) { return 8 * cap + 4 * kN3Half + 16 + 16 * kVn3HomeStride; }

// Staging as n3_stage (lj_force_n3.cuh) with the cotangents copied along,
// and the slice checked per round.  Returns false when the kept candidates
// would not fit.
__device__ __forceinline__ bool vn3_stage(const VjpN3Coef &k, const float4 *__restrict__ pos,
                                          const float4 *__restrict__ g4, float4 *S, float4 *SG, const float4 *stab,
                                          const int *spre, int Ttot, int n_home, int &T_out)
{
    const int lane = threadIdx.x & 31;
    float bxl = 3.4e38f, byl = 3.4e38f, bzl = 3.4e38f, bxh = -3.4e38f, byh = -3.4e38f, bzh = -3.4e38f;
    const float rcut2 = k.rc2 * 1.0001f;
    float bcx = 0.f, bcy = 0.f, bcz = 0.f, bhx = 0.f, bhy = 0.f, bhz = 0.f;
    const unsigned lt = (1u << lane) - 1u;
    int *tmp = reinterpret_cast<int *>(S);
    const int s_e = lane < kN3Half ? spre[lane] : 0x7fffffff;
    const bool ne = lane < kN3Half && spre[lane + 1] > s_e;
    const unsigned nem = __ballot_sync(0xffffffffu, ne);
    if (ne) tmp[__popc(nem & lt)] = lane;
    __syncwarp();
    const int j_entry = lane < __popc(nem) ? tmp[lane] : 0;
    __syncwarp();
    const unsigned le = (2u << lane) - 1u;
    const int last = k.n - 1;
    int T = 0;
    for (int t0 = 0; t0 < Ttot; t0 += 32 * kN3Batch) {
        float4 q[kN3Batch], qg[kN3Batch], sh[kN3Batch];
#pragma unroll
        for (int u = 0; u < kN3Batch; u++) {
            const int t = t0 + 32 * u + lane;
            const int tb = t0 + 32 * u;
            const int o = s_e - tb;
            const unsigned inside = __reduce_or_sync(0xffffffffu, (ne && o >= 1 && o <= 31) ? (1u << o) : 0u);
            const int jc = __popc(__ballot_sync(0xffffffffu, ne && o <= 0)) - 1 + __popc(inside & le);
            const int kc = __shfl_sync(0xffffffffu, j_entry, jc & 31);
            const int kb = __shfl_sync(0xffffffffu, s_e, kc);
            sh[u] = stab[kc];
            const int idx = min(__float_as_int(sh[u].w) + (t - kb), last);
            q[u] = __ldg(pos + idx);
            qg[u] = __ldg(g4 + idx);
        }
        if (t0 == 0) {   // the home particles are candidates 0 .. n_home-1 of the first round
            if (lane < n_home) {
                bxl = bxh = q[0].x;
                byl = byh = q[0].y;
                bzl = bzh = q[0].z;
            }
            box_reduce(bxl, byl, bzl, bxh, byh, bzh);
            bcx = 0.5f * (bxl + bxh);
            bcy = 0.5f * (byl + byh);
            bcz = 0.5f * (bzl + bzh);
            bhx = 0.5f * (bxh - bxl);
            bhy = 0.5f * (byh - byl);
            bhz = 0.5f * (bzh - bzl);
        }
#pragma unroll
        for (int u = 0; u < kN3Batch; u++) {
            const int t = t0 + 32 * u + lane;
            const float cx = q[u].x + sh[u].x;
            const float cy = q[u].y + sh[u].y;
            const float cz = q[u].z + sh[u].z;
            const float dx = fmaxf(fabsf(cx - bcx) - bhx, 0.f);
            const float dy = fmaxf(fabsf(cy - bcy) - bhy, 0.f);
            const float dz = fmaxf(fabsf(cz - bcz) - bhz, 0.f);
            const bool keep = t < Ttot && dx * dx + dy * dy + dz * dz < rcut2;
            const unsigned kept = __ballot_sync(0xffffffffu, keep);
            if (T + __popc(kept) + 32 > k.cap) {   // the padding must fit too
                __syncwarp();
                return false;
            }
            if (keep) {
                const int sl = T + __popc(kept & lt);
                S[sl] = make_float4(cx, cy, cz, q[u].w);
                SG[sl] = qg[u];
            }
            T += __popc(kept);
        }
    }
    S[T + lane] = make_float4(kFar, kFar, kFar, 0.0f);
    SG[T + lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    __syncwarp();
    T_out = T;
    return true;
}

// One (home pair, candidate) term: d = x_h - x_c for the two home particles
// of (hx, hy, hz) with cotangents (ux, uy, uz) against the broadcast
// candidate (cx, cy, cz) with cotangent (wx, wy, wz).  v = J (g_h - g_c) is
// added to the home sums (ax, ay, az) and to the candidate's reaction sums
// (rx, ry, rz), which the caller subtracts; the parameter terms go to te and
// ts.  SELF: a home-home pair counts only for s < j.
template <int MODE, bool SELF>
__device__ __forceinline__ void vn3_pair2(float2 hx, float2 hy, float2 hz, float2 ux, float2 uy, float2 uz, int s0,
                                          int s1, float2 cx, float2 cy, float2 cz, float2 wx, float2 wy, float2 wz,
                                          int j, const VjpN3Coef &k, float2 &ax, float2 &ay, float2 &az, float2 &rx,
                                          float2 &ry, float2 &rz, float2 &te, float2 &ts)
{
    const float2 m1 = f2(-1.0f);
    const float2 dx = __ffma2_rn(cx, m1, hx);
    const float2 dy = __ffma2_rn(cy, m1, hy);
    const float2 dz = __ffma2_rn(cz, m1, hz);
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    float2 ri, rinv = f2(0.0f);
    if constexpr (MODE != 2 && !SELF) {
        // the cutoff as a 0/1 factor, as in the force kernel (pair2_n3)
        float2 m;
        m.x = fma_sat(r2.x, -0x1p100f, k.rc2 * 0x1p100f);
        m.y = fma_sat(r2.y, -0x1p100f, k.rc2 * 0x1p100f);
        ri.x = rcp_approx(r2.x);
        ri.y = rcp_approx(r2.y);
        ri = __fmul2_rn(ri, m);
    } else {
        bool ina = r2.x < k.rc2, inb = r2.y < k.rc2;
        if constexpr (SELF) {
            ina = ina && (j > s0);
            inb = inb && (j > s1);
        }
        if constexpr (MODE == 2) {
            const float qa = rsqrt_approx(r2.x), qb = rsqrt_approx(r2.y);
            rinv.x = ina ? qa : 0.0f;
            rinv.y = inb ? qb : 0.0f;
            ri = __fmul2_rn(rinv, rinv);
        } else {
            const float qa = rcp_approx(r2.x), qb = rcp_approx(r2.y);
            ri.x = ina ? qa : 0.0f;
            ri.y = inb ? qb : 0.0f;
        }
    }
    const float2 r6 = __fmul2_rn(__fmul2_rn(ri, ri), ri);
    const float2 r8 = __fmul2_rn(ri, r6);                                    // r^-8
    float2 phi1 = __fmul2_rn(r8, __ffma2_rn(f2(k.a1), r6, f2(-k.b1)));       // phi at eps = 1
    float2 dphi1 = __fmul2_rn(__fmul2_rn(r8, ri), __ffma2_rn(f2(-k.c14), r6, f2(k.c8)));   // phi'/r at eps = 1
    float2 dsig1 = __fmul2_rn(r8, __ffma2_rn(f2(k.s12), r6, f2(-k.s6)));     // dphi/dsigma at eps = 1
    if constexpr (MODE == 2) {
        phi1 = __ffma2_rn(f2(-k.fc1), rinv, phi1);
        dphi1 = __ffma2_rn(__fmul2_rn(f2(k.fc1), rinv), ri, dphi1);
        dsig1 = __ffma2_rn(f2(-k.dfc1), rinv, dsig1);
    }
    const float2 phi = __fmul2_rn(f2(k.eps), phi1);
    const float2 gx = __ffma2_rn(wx, m1, ux);   // g_h - g_c
    const float2 gy = __ffma2_rn(wy, m1, uy);
    const float2 gz = __ffma2_rn(wz, m1, uz);
    const float2 dot = __ffma2_rn(dz, gz, __ffma2_rn(dy, gy, __fmul2_rn(dx, gx)));
    const float2 t = __fmul2_rn(__fmul2_rn(f2(k.eps), dphi1), dot);
    const float2 vx = __ffma2_rn(t, dx, __fmul2_rn(phi, gx));
    const float2 vy = __ffma2_rn(t, dy, __fmul2_rn(phi, gy));
    const float2 vz = __ffma2_rn(t, dz, __fmul2_rn(phi, gz));
    ax = __fadd2_rn(ax, vx);
    ay = __fadd2_rn(ay, vy);
    az = __fadd2_rn(az, vz);
    rx = __fadd2_rn(rx, vx);
    ry = __fadd2_rn(ry, vy);
    rz = __fadd2_rn(rz, vz);
    te = __ffma2_rn(phi1, dot, te);
    ts = __ffma2_rn(__fmul2_rn(f2(k.eps), dsig1), dot, ts);
}

// One candidate block: lane (a, b) takes candidate blk B + b against its NH
// home pairs.  Home table of group a: the (x0, x1, y0, y1) of pairs 0..3,
// the z of pairs (0, 1) and (2, 3), then the same for the cotangents, and a
// float4 of padding.
template <int NH, int LGB, int MODE, bool SELF>
__device__ __forceinline__ void vn3_block(const VjpN3Coef &k, float4 *__restrict__ acc, const float4 *S,
                                          const float4 *SG, int T, int blk, int a, int b, int A, const float4 *H,
                                          float2 *ax, float2 *ay, float2 *az, float2 &te, float2 &ts)
{
    constexpr int B = 1 << LGB;
    const int j = (blk << LGB) + b;
    const float4 c = S[j];
    const float4 cg = SG[j];
    const float2 cx = f2(c.x), cy = f2(c.y), cz = f2(c.z);
    const float2 wx = f2(cg.x), wy = f2(cg.y), wz = f2(cg.z);
    float2 rx = f2(0.0f), ry = f2(0.0f), rz = f2(0.0f);
    const float4 *Hg = H + kVn3HomeStride * a;
#pragma unroll
    for (int h = 0; h < NH; h += 2) {
        const float4 z2 = n3_ld4(Hg + 4 + (h >> 1));
        const float4 gz2 = n3_ld4(Hg + 10 + (h >> 1));
        const float4 q0 = n3_ld4(Hg + h);
        const float4 u0 = n3_ld4(Hg + 6 + h);
        vn3_pair2<MODE, SELF>(make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(z2.x, z2.y),
                              make_float2(u0.x, u0.y), make_float2(u0.z, u0.w), make_float2(gz2.x, gz2.y),
                              2 * h * A + a, (2 * h + 1) * A + a, cx, cy, cz, wx, wy, wz, j, k, ax[h], ay[h], az[h], rx,
                              ry, rz, te, ts);
        if (h + 1 < NH) {
            const float4 q1 = n3_ld4(Hg + h + 1);
            const float4 u1 = n3_ld4(Hg + 6 + h + 1);
            vn3_pair2<MODE, SELF>(make_float2(q1.x, q1.y), make_float2(q1.z, q1.w), make_float2(z2.z, z2.w),
                                  make_float2(u1.x, u1.y), make_float2(u1.z, u1.w), make_float2(gz2.z, gz2.w),
                                  2 * (h + 1) * A + a, (2 * (h + 1) + 1) * A + a, cx, cy, cz, wx, wy, wz, j, k,
                                  ax[h + 1], ay[h + 1], az[h + 1], rx, ry, rz, te, ts);
        }
    }
    float sx = rx.x + rx.y, sy = ry.x + ry.y, sz = rz.x + rz.y;
    if constexpr (LGB == 3) {   // four groups: one shuffle level, then two groups add
        sx += __shfl_xor_sync(0xffffffffu, sx, 8);
        sy += __shfl_xor_sync(0xffffffffu, sy, 8);
        sz += __shfl_xor_sync(0xffffffffu, sz, 8);
        if ((a & 1) == 0 && j < T) atomicAdd(acc + __float_as_int(c.w), make_float4(-sx, -sy, -sz, 0.0f));
    } else {
        if (j < T) atomicAdd(acc + __float_as_int(c.w), make_float4(-sx, -sy, -sz, 0.0f));
    }
}

template <int NH, int LGB, int MODE>
__device__ __forceinline__ void vn3_blocks(const VjpN3Coef &k, float4 *__restrict__ acc, const float4 *S,
                                           const float4 *SG, int T, int n_home, int a, int b, int A, const float4 *H,
                                           float2 *ax, float2 *ay, float2 *az, float2 &te, float2 &ts)
{
    constexpr int B = 1 << LGB;
    const int nblk = (T + B - 1) >> LGB;
    const int nself = min(nblk, (n_home + B - 1) >> LGB);
    int blk = 0;
    for (; blk < nself; blk++) vn3_block<NH, LGB, MODE, true>(k, acc, S, SG, T, blk, a, b, A, H, ax, ay, az, te, ts);
    for (; blk < nblk; blk++) vn3_block<NH, LGB, MODE, false>(k, acc, S, SG, T, blk, a, b, A, H, ax, ay, az, te, ts);
}

// Compute phase of a staged cell of n_home <= 32 home particles (S holds at
// least kN3Home * 32 slots, reused for the transpose of the home sums).
template <int MODE>
__device__ __forceinline__ void vn3_compute(const VjpN3Coef &k, float4 *__restrict__ acc, float4 *S,
                                            const float4 *SG, float4 *H, int T, int n_home, double &acc_e,
                                            double &acc_s)
{
    const int lane = threadIdx.x & 31;
    const int hp = n_home;
    const int lgB = hp > 16 ? 3 : 4;
    const int B = 1 << lgB, A = 32 >> lgB;
    const int a = lane >> lgB, b = lane & (B - 1);
    const int nu = (hp + A - 1) >> (5 - lgB);
    if (b < kN3Home / 2) {   // lane (a, b < 4) writes pair b of group a
        const int s0 = 2 * b * A + a, s1 = s0 + A;
        const bool v0 = s0 < hp, v1 = s1 < hp;
        const float4 q0 = S[v0 ? s0 : 0], q1 = S[v1 ? s1 : 0];
        const float4 g0 = SG[v0 ? s0 : 0], g1 = SG[v1 ? s1 : 0];
        float4 *p = H + kVn3HomeStride * a;
        p[b] = make_float4(v0 ? q0.x : -kFar, v1 ? q1.x : -kFar, v0 ? q0.y : -kFar, v1 ? q1.y : -kFar);
        float *z = reinterpret_cast<float *>(p + 4) + 2 * b;
        z[0] = v0 ? q0.z : -kFar;
        z[1] = v1 ? q1.z : -kFar;
        p[6 + b] = make_float4(v0 ? g0.x : 0.0f, v1 ? g1.x : 0.0f, v0 ? g0.y : 0.0f, v1 ? g1.y : 0.0f);
        float *gz = reinterpret_cast<float *>(p + 10) + 2 * b;
        gz[0] = v0 ? g0.z : 0.0f;
        gz[1] = v1 ? g1.z : 0.0f;
    }
    __syncwarp();
    float2 ax[kN3Home / 2], ay[kN3Home / 2], az[kN3Home / 2];
    float2 te = f2(0.0f), ts = f2(0.0f);
#pragma unroll
    for (int h = 0; h < kN3Home / 2; h++) ax[h] = ay[h] = az[h] = f2(0.0f);
    const int nh = (nu + 1) >> 1;
    if (lgB == 4) {
        if (nh >= 4) vn3_blocks<4, 4, MODE>(k, acc, S, SG, T, n_home, a, b, A, H, ax, ay, az, te, ts);
        else if (nh == 3) vn3_blocks<3, 4, MODE>(k, acc, S, SG, T, n_home, a, b, A, H, ax, ay, az, te, ts);
        else vn3_blocks<2, 4, MODE>(k, acc, S, SG, T, n_home, a, b, A, H, ax, ay, az, te, ts);
    } else {
        if (nh >= 4) vn3_blocks<4, 3, MODE>(k, acc, S, SG, T, n_home, a, b, A, H, ax, ay, az, te, ts);
        else if (nh == 3) vn3_blocks<3, 3, MODE>(k, acc, S, SG, T, n_home, a, b, A, H, ax, ay, az, te, ts);
        else vn3_blocks<2, 3, MODE>(k, acc, S, SG, T, n_home, a, b, A, H, ax, ay, az, te, ts);
    }
    acc_e += (double)(te.x + te.y);
    acc_s += (double)(ts.x + ts.y);
    const int p = A == 2 ? lane >> 1 : lane;
    const int bh = A == 2 ? (lane & 1) * 8 : 0;
    const int u = p >> (5 - lgB), g = p & (A - 1);
    const int hidx = p < hp ? __float_as_int(S[p].w) : 0;
    __syncwarp();   // every lane is done reading S
    float4 *part = S;
#pragma unroll
    for (int h = 0; h < kN3Home / 2; h++) {
        if (2 * h < nu) part[(2 * h) * 32 + lane] = make_float4(ax[h].x, ay[h].x, az[h].x, 0.0f);
        if (2 * h + 1 < nu) part[(2 * h + 1) * 32 + lane] = make_float4(ax[h].y, ay[h].y, az[h].y, 0.0f);
    }
    __syncwarp();
    float4 sum = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (p < hp) {
        const float4 *row = part + u * 32 + g * B + bh;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const float4 q = row[(i + lane) & 7];
            sum.x += q.x;
            sum.y += q.y;
            sum.z += q.z;
        }
    }
    if (A == 2) {
        sum.x += __shfl_xor_sync(0xffffffffu, sum.x, 1);
        sum.y += __shfl_xor_sync(0xffffffffu, sum.y, 1);
        sum.z += __shfl_xor_sync(0xffffffffu, sum.z, 1);
    }
    if (p < hp && bh == 0) atomicAdd(acc + hidx, sum);
    __syncwarp();
}

// Plain path: lane = home particle, the half stencil's candidates read
// from global memory (all lanes the same one), reactions summed over the
// warp.
template <int MODE>
__device__ void vn3_plain(const VjpN3Coef &k, const float4 *__restrict__ pos, const float4 *__restrict__ g4,
                          float4 *__restrict__ acc, const float4 *stab, const int *spre, int s_home, int n_home,
                          double &acc_e, double &acc_s)
{
    const int lane = threadIdx.x & 31;
    for (int p0 = 0; p0 < n_home; p0 += 32) {
        const int i = p0 + lane;
        const bool vi = i < n_home;
        const float4 pi = __ldg(pos + s_home + (vi ? i : 0));
        const float4 gi = __ldg(g4 + s_home + (vi ? i : 0));
        float2 ax = f2(0.f), ay = f2(0.f), az = f2(0.f), te = f2(0.f), ts = f2(0.f);
        for (int kk = 0; kk < kN3Half; kk++) {
            const float4 sh = stab[kk];
            const int s = __float_as_int(sh.w);
            const int nn = spre[kk + 1] - spre[kk];
            for (int j = (kk == 0 ? p0 + 1 : 0); j < nn; j++) {
                const float4 q = __ldg(pos + s + j);
                const float4 h = __ldg(g4 + s + j);
                float2 rx = f2(0.f), ry = f2(0.f), rz = f2(0.f);
                // slot y is a far dummy; home pairs count for j > i only
                vn3_pair2<MODE, true>(make_float2(pi.x, -kFar), make_float2(pi.y, -kFar), make_float2(pi.z, -kFar),
                                      make_float2(gi.x, 0.f), make_float2(gi.y, 0.f), make_float2(gi.z, 0.f),
                                      kk == 0 ? i : -1, 0x7fffffff, f2(q.x + sh.x), f2(q.y + sh.y), f2(q.z + sh.z),
                                      f2(h.x), f2(h.y), f2(h.z), vi ? j : -1, k, ax, ay, az, rx, ry, rz, te, ts);
                float sx = rx.x, sy = ry.x, sz = rz.x;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sx += __shfl_xor_sync(0xffffffffu, sx, o);
                    sy += __shfl_xor_sync(0xffffffffu, sy, o);
                    sz += __shfl_xor_sync(0xffffffffu, sz, o);
                }
                if (lane == 0) atomicAdd(acc + __float_as_int(q.w), make_float4(-sx, -sy, -sz, 0.0f));
            }
        }
        if (vi) {
            atomicAdd(acc + __float_as_int(pi.w), make_float4(ax.x, ay.x, az.x, 0.0f));
            acc_e += (double)te.x;
            acc_s += (double)ts.x;
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kVn3Threads, 4) k_vjp_n3(VjpN3Coef k, const float4 *__restrict__ pos,
                                                         const float4 *__restrict__ g4,
                                                         const int32_t *__restrict__ start, float4 *__restrict__ acc,
                                                         double *__restrict__ partial)
{
    extern __shared__ __align__(16) float vsm[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float4 *S = reinterpret_cast<float4 *>(vsm + (size_t)warp * vn3_slice_words(k.cap));
    float4 *SG = S + k.cap;
    float4 *stab = SG + k.cap;
    int *spre = reinterpret_cast<int *>(stab + kN3Half);
    float4 *H = reinterpret_cast<float4 *>(spre + 16);
    double acc_e = 0.0, acc_s = 0.0;
    // pulls of k.grab cells, single cells over the last stretch (as k_force_n3)
    const int64_t tail = 2 * (int64_t)k.grab * gridDim.x * (kVn3Threads / 32);
    unsigned last = 0;
    for (;;) {
        const unsigned gr = (int64_t)last + tail >= k.ncell ? 1u : (unsigned)k.grab;
        unsigned c0 = 0;
        if (lane == 0) c0 = atomicAdd(k.work, gr);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if ((int64_t)c0 >= k.ncell) break;
        last = c0;
        const int c1 = (int)min((int64_t)c0 + gr, k.ncell);
        HalfLoad nxt = half_load<true>(start, (int)c0, k.nc, k.inv_nc);
        for (int c = (int)c0; c < c1; c++) {
            const HalfLoad cur = nxt;
            if (c + 1 < c1) nxt = half_load<true>(start, c + 1, k.nc, k.inv_nc);
            __syncwarp();   // the slice still holds the previous cell's data
            const int tot = half_finish(cur, k.cw, stab, spre);
            const int n_home = spre[1];
            if (n_home == 0) continue;
            int T = 0;
            if (n_home <= 32 && tot <= 2 * k.cap && vn3_stage(k, pos, g4, S, SG, stab, spre, tot, n_home, T))
                vn3_compute<MODE>(k, acc, S, SG, H, T, n_home, acc_e, acc_s);
            else
                vn3_plain<MODE>(k, pos, g4, acc, stab, spre, __float_as_int(stab[0].w), n_home, acc_e, acc_s);
        }
    }
    __shared__ double red[2 * (kVn3Threads / 32)];
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
        for (int q = 0; q < kVn3Threads / 32; q++) {
            e += red[2 * q];
            s += red[2 * q + 1];
        }
        partial[2 * blockIdx.x] = e;
        partial[2 * blockIdx.x + 1] = s;
    }
}

// dx[i] += scale * acc[i] (FP64), particle order.
__global__ void k_add_scaled_acc(const float4 *__restrict__ acc, int n, double scale, double *__restrict__ dx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 q = acc[i];
    const int64_t b = 3 * (int64_t)i;
    dx[b] = __fma_rn(scale, (double)q.x, dx[b]);
    dx[b + 1] = __fma_rn(scale, (double)q.y, dx[b + 1]);
    dx[b + 2] = __fma_rn(scale, (double)q.z, dx[b + 2]);
}

void *vn3_kernel(int mode)
{
    // modes 0 and 1 have the same force
    return mode == 2 ? (void *)k_vjp_n3<2> : (void *)k_vjp_n3<0>;
}

}  // namespace

bool uses_vjp_n3(const lj_ctx *c) { return uses_force_n3(c); }

// The pair-once FP32-mixed VJP: the sums go to acc (float4 [n], particle
// order, zeroed here), the parameter partials to c->partial (*grid_out of
// them), and dx += scale acc.  The work counter must be zero (the scan of
// the binning before it zeroes it).
cudaError_t launch_vjp_n3(lj_ctx *c, const double *coef, double scale, double *dx, float4 *acc, int *grid_out)
{
    const double *q = coef;
    const double mean = c->ncell > 0 ? (double)c->p.n / (double)c->ncell : 0.0;
    const double m = kN3Half * mean;
    int cap = (int)(0.8 * m + 4.0 * sqrt(m)) + 32;
    cap = cap < kN3Home * 32 ? kN3Home * 32 : cap;   // S also holds the home sums' transpose
    cap = (cap + 31) & ~31;
    const int warps = kVn3Threads / 32;
    while (cap > kN3Home * 32 && warps * vn3_slice_words(cap) * (int)sizeof(float) > 227 * 1024 - 256) cap -= 32;
    const int smem = warps * vn3_slice_words(cap) * (int)sizeof(float);
    void *kern = vn3_kernel(c->p.shift_mode);
    cudaError_t e = raise_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kVn3Threads, smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)(nb > 0 ? nb : 1) * c->nsm;
    const int64_t need = (c->ncell + warps - 1) / warps;
    if (grid > need) grid = need;
    if (grid > c->npartial_cap) grid = c->npartial_cap;
    if (grid < 1) grid = 1;
    VjpN3Coef k;
    k.rc2 = (float)q[0];
    k.a1 = (float)q[1];
    k.b1 = (float)q[2];
    k.c8 = (float)(8.0 * q[2]);
    k.c14 = (float)(14.0 * q[1]);
    k.s12 = (float)(12.0 * q[1] * q[6]);
    k.s6 = (float)(6.0 * q[2] * q[6]);
    k.fc1 = (float)q[3];
    k.dfc1 = (float)q[4];
    k.eps = (float)q[5];
    k.cw = (float)c->cw;
    k.inv_nc = c->inv_nc_f;
    k.n = (int)c->p.n;
    k.nc = c->nc;
    k.cap = cap;
    k.grab = 4;
    k.ncell = c->ncell;
    k.work = c->work;
    const float4 *pos = (const float4 *)c->pos;
    const float4 *g4 = (const float4 *)c->g4;
    const int32_t *start = c->start;
    double *partial = c->partial;
    e = cudaMemsetAsync(acc, 0, (size_t)c->p.n * sizeof(float4), c->stream);
    if (e != cudaSuccess) return e;
    void *args[] = {&k, (void *)&pos, (void *)&g4, (void *)&start, &acc, &partial};
    e = cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kVn3Threads), args, smem, c->stream);
    if (e != cudaSuccess) return e;
    const int n = (int)c->p.n;
    k_add_scaled_acc<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(acc, n, scale, dx);
    c->kernel_launches += 2;
    *grid_out = (int)grid;
    return cudaGetLastError();
}
