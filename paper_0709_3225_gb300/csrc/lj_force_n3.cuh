// Lennard-Jones forces over cell lists with Newton's third law (FP32-mixed).
//
// The method is that of lj_force_warp.cu (Section 3: each particle
// interacts with the particles of its own cell and of the 26 neighbouring
// cells; Section 2 pair force), but every pair is evaluated ONCE: the pair
// force F(r) d / r is added to particle i and subtracted from particle j
// (Eq. n2_force is antisymmetric in i and j).  A home cell is paired with
// itself (pairs i < j) and with the 13 neighbours whose offset (dz, dy, dx)
// is lexicographically positive; the other 13 neighbours pair with it when
// they are the home cell.  For cell grids of n >= 3 per side no cell pair is
// visited twice: d and -d cannot both be positive, and no two offsets of
// the stencil coincide modulo n.
//
// Organisation for GB300 (one warp per home cell, persistent grid, dynamic
// pulls of consecutive cells, as the 27-cell kernel):
//  * Staging: the half stencil's candidates are taken as one flat index
//    space (warp-vote stencil lookup), converted to the home-cell-centre
//    frame, pruned against the home particles' bounding box (rc plus a
//    0.01 % margin; the box comes from the first staging round, where the
//    home particles are) and appended as float4 (x, y, z, particle index);
//    the home particles come first, in their sorted order.
//  * Compute: the warp is A groups of B = 32 / A lanes (A = 2, or 4 when
//    the cell holds more than 16 home particles).  Lane (a, b) takes
//    candidate b of each block of B against the home particles u A + a,
//    u = 0..7, as four FP32x2 pairs; one packed evaluation covers two home
//    particles against that candidate, whose reaction stays in registers
//    for the block.  The home pairs' positions are read from a per-warp
//    table in shared memory at every evaluation (broadcast loads), and only
//    their partial forces live in registers: that keeps the kernel at 79
//    registers, 24 resident warps per SM instead of 20, and the extra
//    loads cost less than the latency the extra warps hide.
//  * After a block each candidate's reaction goes to f[j] by float4 atomic
//    adds: one per lane group with two groups, one per pair of groups (after
//    a shuffle) with four, so two adds per candidate either way; the second
//    add costs less than the shuffles and additions that would merge the
//    two parts.  There is no test for zero (its four comparisons cost more
//    issue slots than the atomics it saves).  After the last block the home
//    partial forces are summed over the B lanes of their group through a
//    shared-memory transpose (in the staged list's space, which is free by
//    then) and added to f[i] (skipped when zero).  f is zeroed before the
//    launch.
//  * Energies: per-particle f.w gets half of each pair energy on both sides;
//    the FP64 totals take each pair once.
//  * A cell with more than 32 home particles, or whose pruned half stencil
//    does not fit the warp's slice, takes a plain path over global memory
//    (home particle per lane, reactions reduced over the warp).
// The FP32 sums of a particle's force are formed in an order set by the
// atomics, so forces are not bitwise reproducible between runs (their
// rounding error is that of any order); the deterministic mode uses the
// 27-cell kernel.
#pragma once

#include "lj_force_cell.cuh"
#include "lj_pair.cuh"

namespace {

constexpr int kN3Threads = 128;   // 4 warps per CTA
constexpr int kN3Home = 8;        // home particles per lane per pass
constexpr int kN3Half = 14;       // home cell + 13 forward neighbours
constexpr int kN3Batch = 3;       // staging rounds whose loads are in flight together (measured: 3 > 2 > 1)

// Offset of half-stencil entry e: e = 0 the home cell, e = 1 .. 13 the
// neighbours with (dz, dy, dx) > 0 lexicographically (x-fastest index
// 13 + e of the 3 x 3 x 3 block).
__device__ __forceinline__ void half_delta(int e, int &dx, int &dy, int &dz)
{
    const int idx = 13 + e;
    dx = idx % 3 - 1;
    dy = (idx / 3) % 3 - 1;
    dz = idx / 9 - 1;
}

// 32-bit words of one warp's slice: the staged candidates S (cap float4:
// x, y, z in the home frame and the particle index; cap >= kN3Home * 32,
// since S also holds the home forces' transpose), the half-stencil table
// (14 float4), its prefix sums (15 ints, padded to 16) and the home table H
// (4 groups x 7 float4, laid out as n3_block1 describes).
constexpr int kN3HomeStride = 4 + 2 + 1;   // float4 per lane group in H
constexpr int kN3FixedWords = 4 * kN3Half + 16 + 4 * 4 * kN3HomeStride;
__host__ __device__ constexpr int n3_slice_words(int cap) { return 4 * cap + kN3FixedWords; }

// Half-stencil table, in two parts so that a cell's loads can be issued one
// cell ahead: half_load reads, for lane e < 14, the first and end particle
// of entry e of cell c (cell id c < 2^31); half_finish writes stab[e] =
// (shift to the home frame, first particle) and spre[0 .. 14], the
// exclusive prefix sums of the counts, and returns the total.  Both are
// called by all 32 lanes.  c is the cell's id in its grid of nc^3 cells,
// whose ids start at cell_base in start[] (0 for a single system; the
// replica's first cell in a batch); inv_nc as lj_cell_decode.
struct HalfLoad {
    int s, e;
};

template <bool NC>
__device__ __forceinline__ HalfLoad half_load(const int32_t *__restrict__ start, int c, int nc, float inv_nc,
                                              int cell_base = 0)
{
    const int lane = threadIdx.x & 31;
    HalfLoad t{0, 0};
    if (lane < kN3Half) {
        int cx, cy, cz, dx, dy, dz;
        lj_cell_decode(c, nc, inv_nc, cx, cy, cz);
        half_delta(lane, dx, dy, dz);
        int ux = cx + dx, uy = cy + dy, uz = cz + dz;
        ux += ux < 0 ? nc : 0;
        ux -= ux >= nc ? nc : 0;
        uy += uy < 0 ? nc : 0;
        uy -= uy >= nc ? nc : 0;
        uz += uz < 0 ? nc : 0;
        uz -= uz >= nc ? nc : 0;
        const int cn = cell_base + ux + nc * (uy + nc * uz);   // < 2^31
        if constexpr (NC) {
            t.s = __ldg(start + cn);
            t.e = __ldg(start + cn + 1);
        } else {
            t.s = start[cn];
            t.e = start[cn + 1];
        }
    }
    return t;
}

__device__ __forceinline__ int half_finish(HalfLoad t, float cw, float4 *stab, int *spre)
{
    const int lane = threadIdx.x & 31;
    const int nn = t.e - t.s;
    if (lane < kN3Half) {
        int dx, dy, dz;
        half_delta(lane, dx, dy, dz);
        stab[lane] = make_float4((float)dx * cw, (float)dy * cw, (float)dz * cw, __int_as_float(t.s));
    }
    int P = nn;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, P, o);
        if (lane >= o) P += y;
    }
    if (lane < kN3Half) spre[lane] = P - nn;
    if (lane == kN3Half - 1) spre[kN3Half] = P;
    __syncwarp();
    return __shfl_sync(0xffffffffu, P, kN3Half - 1);
}

// a b + c rounded once, clamped to [0, 1] (NaN to 0)
__device__ __forceinline__ float fma_sat(float a, float b, float c)
{
    float d;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// One (home pair, candidate) evaluation: d = x_home - x_cand for the two
// home particles s0, s1 of (hx, hy, hz) and one candidate j broadcast in
// (cx, cy, cz).  The home particles' forces accumulate in (fx, fy, fz), the
// candidate's reaction, with the opposite sign and as two partial sums, in
// (rx, ry, rz).  SELF: the block holds home particles, and a home-home pair
// counts only for s < j.
template <int MODE, bool ENERGY, bool SELF>
__device__ __forceinline__ void pair2_n3(float2 hx, float2 hy, float2 hz, int s0, int s1, float2 cx, float2 cy,
                                         float2 cz, int j, const WarpParams &k, float2 &fx, float2 &fy, float2 &fz,
                                         float2 &fe, float2 &fw, float2 &rx, float2 &ry, float2 &rz, float2 &re)
{
    const float2 m1 = f2(-1.0f);
    const float2 dx = __ffma2_rn(cx, m1, hx);
    const float2 dy = __ffma2_rn(cy, m1, hy);
    const float2 dz = __ffma2_rn(cz, m1, hz);
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    if constexpr (MODE != 2 && !ENERGY && !SELF) {
        // the cutoff as a 0/1 factor from a saturated FMA on the FMA pipe
        // (instead of a compare and a select on the ALU pipe): 2^100 (rc^2 -
        // r^2) is formed exactly (2^100 rc^2 is exact and the FMA rounds
        // once), so it clamps to 1 for every r^2 < rc^2 (the gap is at least
        // one ulp of rc^2) and to 0 for r^2 >= rc^2 (or an overflow to -inf)
        float2 m;
        m.x = fma_sat(r2.x, -0x1p100f, k.rc2 * 0x1p100f);
        m.y = fma_sat(r2.y, -0x1p100f, k.rc2 * 0x1p100f);
        float2 ri;
        ri.x = rcp_approx(r2.x);
        ri.y = rcp_approx(r2.y);
        ri = __fmul2_rn(ri, m);
        const float2 r6 = __fmul2_rn(__fmul2_rn(ri, ri), ri);
        const float2 t = __ffma2_rn(f2(k.a12), r6, f2(-k.b6));
        const float2 ff = __fmul2_rn(__fmul2_rn(ri, r6), t);
        fx = __ffma2_rn(ff, dx, fx);
        fy = __ffma2_rn(ff, dy, fy);
        fz = __ffma2_rn(ff, dz, fz);
        rx = __ffma2_rn(ff, dx, rx);
        ry = __ffma2_rn(ff, dy, ry);
        rz = __ffma2_rn(ff, dz, rz);
        return;
    }
    bool ina = r2.x < k.rc2, inb = r2.y < k.rc2;
    if constexpr (SELF) {
        ina = ina && (j > s0);
        inb = inb && (j > s1);
    }
    // the reciprocal (square root) of every r^2, then a select: no branch
    // (r^2 = 0 of a pair outside the count gives inf, which is dropped)
    float2 ri, rinv = f2(0.0f);
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
    const float2 r6 = __fmul2_rn(__fmul2_rn(ri, ri), ri);
    const float2 t = __ffma2_rn(f2(k.a12), r6, f2(-k.b6));
    float2 ff = __fmul2_rn(__fmul2_rn(ri, r6), t);
    if constexpr (MODE == 2) ff = __ffma2_rn(f2(-k.fc), rinv, ff);
    fx = __ffma2_rn(ff, dx, fx);
    fy = __ffma2_rn(ff, dy, fy);
    fz = __ffma2_rn(ff, dz, fz);
    rx = __ffma2_rn(ff, dx, rx);
    ry = __ffma2_rn(ff, dy, ry);
    rz = __ffma2_rn(ff, dz, rz);
    if constexpr (ENERGY) {
        float2 u = __fmul2_rn(r6, __ffma2_rn(f2(k.c12), r6, f2(-k.c6)));
        if constexpr (MODE >= 1) u = __fadd2_rn(u, f2(-k.uc));
        if constexpr (MODE == 2) u = __ffma2_rn(__ffma2_rn(r2, rinv, f2(-k.rc)), f2(k.fc), u);
        u.x = ina ? u.x : 0.0f;
        u.y = inb ? u.y : 0.0f;
        fe = __fadd2_rn(fe, u);
        re = __fadd2_rn(re, u);
        fw = __ffma2_rn(ff, r2, fw);
    }
}

__device__ __forceinline__ void add_force(float4 *fout, int idx, float4 v)
{
    if (v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f) atomicAdd(fout + idx, v);
}

// A float4 of the home table, loaded at every use: the asm keeps the
// compiler from hoisting the loads out of the candidate loop, so the home
// positions do not occupy registers across it.
__device__ __forceinline__ float4 n3_ld4(const float4 *p)
{
    float4 q;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(q.x), "=f"(q.y), "=f"(q.z), "=f"(q.w) : "r"(smem_addr(p)));
    return q;
}

// One candidate block: lane (a, b) takes candidate blk B + b against its NH
// home pairs (pairs past its home particles sit far away and add nothing),
// then the candidate's reaction is added to f in two parts (see the file
// header).
// Group a's home table: the (x0, x1, y0, y1) of pairs 0..3, then the z of
// pairs (0, 1) and (2, 3), one float4 each, then a float4 of padding so
// that the groups' simultaneous reads fall in different banks.
template <int NH, int LGB, int MODE, bool ENERGY, bool SELF>
__device__ __forceinline__ void n3_block1(const WarpParams &k, float4 *__restrict__ fout, const float4 *S, int T, int blk,
                                          int a, int b, int A, const float4 *H, float2 *fx, float2 *fy, float2 *fz,
                                          float2 *fe, float2 &fw)
{
    constexpr int B = 1 << LGB;
    const int j = (blk << LGB) + b;
    const float4 c = S[j];
    const float2 cx = f2(c.x), cy = f2(c.y), cz = f2(c.z);
    float2 rx = f2(0.0f), ry = f2(0.0f), rz = f2(0.0f), re = f2(0.0f);
    const float4 *Hg = H + kN3HomeStride * a;
#pragma unroll
    for (int h = 0; h < NH; h += 2) {
        const float4 z2 = n3_ld4(Hg + 4 + (h >> 1));   // z of pairs h and h + 1
        const float4 q0 = n3_ld4(Hg + h);
        pair2_n3<MODE, ENERGY, SELF>(make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(z2.x, z2.y),
                                     2 * h * A + a, (2 * h + 1) * A + a, cx, cy, cz, j, k, fx[h], fy[h], fz[h], fe[h],
                                     fw, rx, ry, rz, re);
        if (h + 1 < NH) {
            const float4 q1 = n3_ld4(Hg + h + 1);
            pair2_n3<MODE, ENERGY, SELF>(make_float2(q1.x, q1.y), make_float2(q1.z, q1.w), make_float2(z2.z, z2.w),
                                         2 * (h + 1) * A + a, (2 * (h + 1) + 1) * A + a, cx, cy, cz, j, k, fx[h + 1],
                                         fy[h + 1], fz[h + 1], fe[h + 1], fw, rx, ry, rz, re);
        }
    }
    float sx = rx.x + rx.y, sy = ry.x + ry.y, sz = rz.x + rz.y, se = ENERGY ? re.x + re.y : 0.0f;
    if constexpr (LGB == 3) {   // four groups: one shuffle level, then two groups add
        sx += __shfl_xor_sync(0xffffffffu, sx, 8);
        sy += __shfl_xor_sync(0xffffffffu, sy, 8);
        sz += __shfl_xor_sync(0xffffffffu, sz, 8);
        if constexpr (ENERGY) se += __shfl_xor_sync(0xffffffffu, se, 8);
        if ((a & 1) == 0 && j < T) atomicAdd(fout + __float_as_int(c.w), make_float4(-sx, -sy, -sz, 0.5f * se));
    } else {   // every group adds its own part of the reaction
        if (j < T) atomicAdd(fout + __float_as_int(c.w), make_float4(-sx, -sy, -sz, 0.5f * se));
    }
}

template <int NH, int LGB, int MODE, bool ENERGY>
__device__ __forceinline__ void n3_blocks(const WarpParams &k, float4 *__restrict__ fout, const float4 *S, int T,
                                          int n_home, int a, int b, int A, const float4 *H, float2 *fx, float2 *fy,
                                          float2 *fz, float2 *fe, float2 &fw)
{
    constexpr int B = 1 << LGB;
    const int nblk = (T + B - 1) >> LGB;
    const int nself = min(nblk, (n_home + B - 1) >> LGB);   // blocks holding home particles
    int blk = 0;
    for (; blk < nself; blk++)
        n3_block1<NH, LGB, MODE, ENERGY, true>(k, fout, S, T, blk, a, b, A, H, fx, fy, fz, fe, fw);
    for (; blk < nblk; blk++)
        n3_block1<NH, LGB, MODE, ENERGY, false>(k, fout, S, T, blk, a, b, A, H, fx, fy, fz, fe, fw);
}

// Compute phase of a cell of n_home <= 32 home particles staged in S (home
// particles at 0 .. n_home-1, candidates after them, padded with far points
// to a multiple of 32).  The warp is A groups of B lanes (A = 2 for up to 16
// home particles, else 4); lane (a, b) takes candidate blk B + b of each
// block against the home particles u A + a, u = 0..7, in FP32x2 pairs read
// from the table H (kN3HomeStride float4 per group).  The home forces' transpose
// reuses S once the candidate blocks are done (S holds >= kN3Home * 32).
template <int MODE, bool ENERGY>
__device__ __forceinline__ void n3_compute(const WarpParams &k, float4 *__restrict__ fout, float4 *S, float4 *H,
                                           int T, int n_home, double &eacc, double &wacc)
{
    const int lane = threadIdx.x & 31;
    const int hp = n_home;
    const int lgB = hp > 16 ? 3 : 4;
    const int B = 1 << lgB, A = 32 >> lgB;
    const int a = lane >> lgB, b = lane & (B - 1);
    const int nu = (hp + A - 1) >> (5 - lgB);   // home particles per lane
    // the home table: lane (a, b < 4) writes pair h = b of group a
    if (b < kN3Home / 2) {
        const int s0 = 2 * b * A + a, s1 = s0 + A;
        const bool v0 = s0 < hp, v1 = s1 < hp;
        const float4 q0 = S[v0 ? s0 : 0];
        const float4 q1 = S[v1 ? s1 : 0];
        float4 *p = H + kN3HomeStride * a;
        p[b] = make_float4(v0 ? q0.x : -kFar, v1 ? q1.x : -kFar, v0 ? q0.y : -kFar, v1 ? q1.y : -kFar);
        float *z = reinterpret_cast<float *>(p + 4) + 2 * b;   // z of pair b at float 2b of the z block
        z[0] = v0 ? q0.z : -kFar;
        z[1] = v1 ? q1.z : -kFar;
    }
    __syncwarp();
    float2 fx[kN3Home / 2], fy[kN3Home / 2], fz[kN3Home / 2], fe[kN3Home / 2];
    float2 fw = f2(0.0f);
#pragma unroll
    for (int h = 0; h < kN3Home / 2; h++) fx[h] = fy[h] = fz[h] = fe[h] = f2(0.0f);
    const int nh = (nu + 1) >> 1;
    if (lgB == 4) {
        if (nh >= 4)
            n3_blocks<4, 4, MODE, ENERGY>(k, fout, S, T, n_home, a, b, A, H, fx, fy, fz, fe, fw);
        else if (nh == 3)
            n3_blocks<3, 4, MODE, ENERGY>(k, fout, S, T, n_home, a, b, A, H, fx, fy, fz, fe, fw);
        else
            n3_blocks<2, 4, MODE, ENERGY>(k, fout, S, T, n_home, a, b, A, H, fx, fy, fz, fe, fw);
    } else {
        if (nh >= 4)
            n3_blocks<4, 3, MODE, ENERGY>(k, fout, S, T, n_home, a, b, A, H, fx, fy, fz, fe, fw);
        else if (nh == 3)
            n3_blocks<3, 3, MODE, ENERGY>(k, fout, S, T, n_home, a, b, A, H, fx, fy, fz, fe, fw);
        else
            n3_blocks<2, 3, MODE, ENERGY>(k, fout, S, T, n_home, a, b, A, H, fx, fy, fz, fe, fw);
    }
    const int p = A == 2 ? lane >> 1 : lane;            // home particle of this lane
    const int bh = A == 2 ? (lane & 1) * 8 : 0;         // its half of the B columns
    const int u = p >> (5 - lgB), g = p & (A - 1);
    const int hidx = p < hp ? __float_as_int(S[p].w) : 0;
    __syncwarp();   // every lane is done reading S
    float4 *part = S;
#pragma unroll
    for (int h = 0; h < kN3Home / 2; h++) {
        if (2 * h < nu) part[(2 * h) * 32 + lane] = make_float4(fx[h].x, fy[h].x, fz[h].x, fe[h].x);
        if (2 * h + 1 < nu) part[(2 * h + 1) * 32 + lane] = make_float4(fx[h].y, fy[h].y, fz[h].y, fe[h].y);
        if constexpr (ENERGY) eacc += (double)(fe[h].x + fe[h].y);
    }
    if constexpr (ENERGY) wacc += (double)(fw.x + fw.y);
    __syncwarp();
    float4 sum = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (p < hp) {
        const float4 *row = part + u * 32 + g * B + bh;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const float4 q = row[(i + lane) & 7];   // rotated: no bank conflicts
            sum.x += q.x;
            sum.y += q.y;
            sum.z += q.z;
            sum.w += q.w;
        }
    }
    if (A == 2) {
        sum.x += __shfl_xor_sync(0xffffffffu, sum.x, 1);
        sum.y += __shfl_xor_sync(0xffffffffu, sum.y, 1);
        sum.z += __shfl_xor_sync(0xffffffffu, sum.z, 1);
        if constexpr (ENERGY) sum.w += __shfl_xor_sync(0xffffffffu, sum.w, 1);
    }
    if (p < hp && bh == 0) {
        sum.w *= 0.5f;
        add_force(fout, hidx, sum);
    }
    __syncwarp();
}

// Staging of the half stencil (see the file header) into S.  Returns false,
// having computed nothing, when the kept candidates would not fit the slice.
template <bool NC>
__device__ __forceinline__ bool n3_stage(const WarpParams &k, const float4 *__restrict__ pos, float4 *S,
                                         const float4 *stab, const int *spre, int Ttot, int s_home, int n_home,
                                         int &T_out)
{
    const int lane = threadIdx.x & 31;
    float bxl = 3.4e38f, byl = 3.4e38f, bzl = 3.4e38f, bxh = -3.4e38f, byh = -3.4e38f, bzh = -3.4e38f;
    if (n_home > 32) {   // bounding box from a pass of its own; else from the first staging round
        for (int p0 = 0; p0 < n_home; p0 += 32) {
            if (p0 + lane < n_home) {
                const float4 q = load_pos<NC>(pos + s_home + p0 + lane);
                bxl = fminf(bxl, q.x);
                byl = fminf(byl, q.y);
                bzl = fminf(bzl, q.z);
                bxh = fmaxf(bxh, q.x);
                byh = fmaxf(byh, q.y);
                bzh = fmaxf(bzh, q.z);
            }
        }
    }
    // the margin of the box test (0.01 % of rc^2) covers the FP32 rounding of
    // the centre and half extents (~1e-7 relative)
    const float rcut2 = k.rc2 * 1.0001f;
    float bcx = 0.f, bcy = 0.f, bcz = 0.f, bhx = 0.f, bhy = 0.f, bhz = 0.f;
    const unsigned lt = (1u << lane) - 1u;
    // warp-vote stencil lookup (as the 27-cell kernel): lane e holds entry
    // e's first candidate s_e; lane j the index of the j-th non-empty entry
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
        float4 q[kN3Batch], sh[kN3Batch];
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
            // past the stencil (t >= Ttot) the index is clamped into the array
            // and the candidate is not kept
            q[u] = load_pos<NC>(pos + min(__float_as_int(sh[u].w) + (t - kb), last));
        }
        if (t0 == 0 && n_home <= 32) {
            // the home particles are candidates 0 .. n_home-1 of the first round
            if (lane < n_home) {
                bxl = bxh = q[0].x;
                byl = byh = q[0].y;
                bzl = bzh = q[0].z;
            }
            box_reduce(bxl, byl, bzl, bxh, byh, bzh);
        } else if (t0 == 0) {
            box_reduce(bxl, byl, bzl, bxh, byh, bzh);
        }
        if (T + 32 * kN3Batch + 32 > k.cap) {   // this batch plus the padding might not fit
            __syncwarp();
            return false;
        }
        if (t0 == 0) {   // the box as centre and half extents
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
            if (keep) S[T + __popc(kept & lt)] = make_float4(cx, cy, cz, q[u].w);
            T += __popc(kept);
        }
    }
    S[T + lane] = make_float4(kFar, kFar, kFar, 0.0f);   // padding to the next multiple of 32 (T + 32 <= cap)
    __syncwarp();
    T_out = T;
    return true;
}

// Plain path for a cell whose pruned half stencil overflows the slice: lane
// = home particle, candidates read from global memory (all lanes the same
// one), reactions summed over the warp.
template <int MODE, bool ENERGY, bool NC>
__device__ void n3_plain(const WarpParams &k, const float4 *__restrict__ pos, float4 *__restrict__ fout,
                         const float4 *stab, const int *spre, int s_home, int n_home, double &eacc, double &wacc)
{
    const int lane = threadIdx.x & 31;
    for (int p0 = 0; p0 < n_home; p0 += 32) {
        const int i = p0 + lane;
        const bool vi = i < n_home;
        const float4 pi = load_pos<NC>(pos + s_home + (vi ? i : 0));
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f, w = 0.f;
        for (int kk = 0; kk < kN3Half; kk++) {
            const float4 sh = stab[kk];
            const int s = __float_as_int(sh.w);
            const int nn = spre[kk + 1] - spre[kk];
            const float xs = pi.x - sh.x, ys = pi.y - sh.y, zs = pi.z - sh.z;
            for (int j = (kk == 0 ? p0 + 1 : 0); j < nn; j++) {
                const float4 q = load_pos<NC>(pos + s + j);
                const float dx = xs - q.x, dy = ys - q.y, dz = zs - q.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                const bool in = vi && r2 < k.rc2 && (kk != 0 || j > i);
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
                float u = 0.0f;
                if constexpr (ENERGY) {
                    u = r6 * (k.c12 * r6 - k.c6);
                    if constexpr (MODE >= 1) u -= k.uc;
                    if constexpr (MODE == 2) u += (r2 * rinv - k.rc) * k.fc;
                    u = in ? u : 0.0f;
                    e += u;
                    w += ff * r2;
                }
                fx += ff * dx;
                fy += ff * dy;
                fz += ff * dz;
                float rx = ff * dx, ry = ff * dy, rz = ff * dz, ru = u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    rx += __shfl_xor_sync(0xffffffffu, rx, o);
                    ry += __shfl_xor_sync(0xffffffffu, ry, o);
                    rz += __shfl_xor_sync(0xffffffffu, rz, o);
                    if constexpr (ENERGY) ru += __shfl_xor_sync(0xffffffffu, ru, o);
                }
                if (lane == 0) add_force(fout, __float_as_int(q.w), make_float4(-rx, -ry, -rz, 0.5f * ru));
            }
        }
        if (vi) {
            add_force(fout, __float_as_int(pi.w), make_float4(fx, fy, fz, 0.5f * e));
            if constexpr (ENERGY) {
                eacc += (double)e;
                wacc += (double)w;
            }
        }
    }
}

// One home cell whose table loads are tl (half_load): table, staging, and
// the compute phase, or the plain path for a cell of more than 32 home
// particles or whose pruned half stencil does not fit the slice (S, stab,
// spre, H: the warp's slice).  cw: the
// cell side of the cell's grid.  NC: read-only loads of the sorted
// positions (not when an earlier phase of the same launch writes them).
template <int MODE, bool ENERGY, bool NC>
__device__ __forceinline__ void n3_cell(const WarpParams &k, const float4 *__restrict__ pos, float4 *__restrict__ fout,
                                        HalfLoad tl, float cw, float4 *S, float4 *stab, int *spre, float4 *H,
                                        double &eacc, double &wacc)
{
    __syncwarp();   // the slice still holds the previous cell's data
    const int tot = half_finish(tl, cw, stab, spre);
    const int n_home = spre[1];
    if (n_home == 0) return;
    const int s_home = __float_as_int(stab[0].w);
    int T = 0;
    if (n_home <= 32 && tot <= 2 * k.cap && n3_stage<NC>(k, pos, S, stab, spre, tot, s_home, n_home, T))
        n3_compute<MODE, ENERGY>(k, fout, S, H, T, n_home, eacc, wacc);
    else
        n3_plain<MODE, ENERGY, NC>(k, pos, fout, stab, spre, s_home, n_home, eacc, wacc);
}

}  // namespace
