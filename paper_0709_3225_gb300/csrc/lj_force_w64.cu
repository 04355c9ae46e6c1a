// Lennard-Jones forces over cell lists in FP64, warp per home cell with the
// in-range pairs compacted before any FP64 arithmetic.
//
// Same method as the other force kernels (Section 3: a particle interacts
// with the particles of its own and the neighbouring cells; Section 2 pair
// force, truncated / shifted), organised for a GPU whose FP64 rate is a
// small fraction of its FP32 rate (GB300: about 2 FP64 FMAs per clock per
// SM against 128 FP32).  Only ~15-25 % of the stencil's candidates lie
// within rc, so FP64 work is spent on those alone:
//  * Staging (per home cell, as in the FP32-mixed warp kernel): the stencil
//    table, then one flat pass over the stencil's candidates.  Each is
//    converted to the home-cell frame twice: in FP64 (kept for the force)
//    and, from a truncated FP32 copy of its coordinates, in FP32 for the
//    filters.  Candidates farther than rc from the home particles' bounding
//    box are dropped.
//  * Phase A (FP32 and integer work only): for each home particle, the
//    indices of the staged candidates within rc (FP32 test with a relative
//    margin of 1e-4, far above the conversion error) are appended to one
//    list, particle after particle.
//  * Phase B (FP64): the 32 lanes split the concatenated list into equal
//    contiguous ranges, so every lane evaluates the same number of pairs
//    whatever the occupancy.  A lane sums its entries in order; a particle
//    whose entries all lie in one lane is stored by that lane; a particle
//    split over several lanes is combined by the lane holding its first
//    entry, adding the other lanes' partial sums in lane order.  The exact
//    FP64 cutoff test decides each pair (pair64).  Sums are in a fixed
//    order, so the forces are reproducible for a fixed in-cell order.
//  * Cells whose pruned stencil does not fit the warp's slice take a plain
//    FP64 path reading global memory per stencil cell.
// The same kernel, with the cotangents staged beside the positions, gives
// the FP64 VJP of the forces (OP 2, vjp64): the pair lists are the same,
// only the FP64 pair term and what is stored differ.
// Pair-once form (PO, forces and energies; the default outside the
// deterministic in-cell mode): the pair force is antisymmetric (Section 2),
// so each pair is evaluated once.  The stencil is the home cell and its 13
// neighbours of positive offset; Phase A lists, for home particle p, only
// the staged candidates j > p (the home cell stages first, so this is every
// pair of the home cell once and every pair with a neighbour cell once).
// Phase B adds the pair force to p's running sum and its reaction to j's
// sum by FP64 atomic adds, into a buffer in cell order (so that a cell's
// atomics and its neighbours' stay within a few MB of L2); one more
// coalesced kernel copies the buffer to f in particle order.  The FP64 pipe
// is the bound: the sign of -F/r is taken into the coefficients and the
// atomics carry no zero test, so that no FP64-pipe instruction is spent on
// anything but the pair arithmetic (measured 7.9 -> 4.8 ms at N = 4M
// against the 27-cell form; with zero tests and negations on the FP64 pipe
// it measured 6.5 ms).  The VJP (OP 2) has a pair-once form too: J_ij is
// even in d, so j receives the negative of i's J_ij (g_i - g_j) (vjp64_po);
// k_unsort_add64 then adds the scaled buffer to dL/dx.
#include <math.h>
#include <string.h>

#include "lj_force_cell.cuh"
#include "lj_force_n3.cuh"
#include "lj_pair.cuh"

namespace {

constexpr int kW64Threads = 32;    // one warp per CTA: residency set by each warp's slice alone
constexpr int kW64PMax = 64;       // home particles per list batch
constexpr int kW64Comp = 5;        // fx, fy, fz, energy, virial

struct W64Params {
    int n, nc, cap, lcap, grab;
    unsigned *work;
    int64_t ncell;
    float cwf;                                    // cell side (FP32, filter shifts)
    float rc2_box, rc2_pair;                      // FP32 filter cutoffs squared (with margins)
    double cw;                                    // cell side (FP64 shifts)
    double rc2, rc, a12, b6, c12, c6, uc, fc;     // pair coefficients, as in Coef<double>
    // VJP (OP 2) only: sorted cotangents, dx += scale dL/dx, and the
    // coefficients of the derivative terms (eps = 1 forms, see vjp64)
    const double4_16a *g4;
    double *dxo;
    double scale;
    double va1, vb1, vfc1, vdfc1, veps, visg;
};

// Byte layout of one warp's shared-memory slice:
//   X64, Y64, Z64   double[cap]   staged candidates, home frame, FP64
//   HX64 .. HZ64    double[cap]   their cotangents (VJP only)
//   part            double[2][kW64Comp][32]   per-lane partial sums (first,
//                                 head; not in the pair-once form)
//   stab            float4[NS]    stencil table: FP32 shift xyz, start index
//   S64             double[3][NS] stencil shifts in FP64 (padded to 16 B)
//   X, Y, Z         float[cap]    staged candidates, home frame, FP32
//   spre            int[NS + 1]   stencil prefix sums (padded to 4)
//   off             int[kW64PMax + 4]   list offsets of the batch's particles
//   list            uint16[lcap]  in-range candidate indices
//   iw              int[cap]      sorted slot of each staged candidate (the
//                                 pair-once form only)
struct W64Layout {
    int x64, h64, part, stab, s64, x32, spre, off, list, iw, bytes;
    __host__ __device__ W64Layout(int cap, int R, int lcap, bool vjp = false, bool po = false)
    {
        const int ns = (2 * R + 1) * (2 * R + 1) * (2 * R + 1);
        x64 = 0;
        h64 = x64 + 24 * cap;
        part = h64 + (vjp ? 24 * cap : 0);
        stab = part + (po ? 0 : 2 * kW64Comp * 32 * 8);
        s64 = stab + 16 * ns;
        x32 = s64 + ((24 * ns + 15) & ~15);
        spre = x32 + 12 * cap;
        off = spre + 4 * ((ns + 1 + 3) & ~3);
        list = off + 4 * (kW64PMax + 4);
        iw = (list + 2 * lcap + 15) & ~15;
        bytes = (iw + (po ? 4 * cap : 0) + 15) & ~15;
    }
};

// FP32 value of a double by truncation of its IEEE-754 fields (relative
// error below 2^-23; |x| < 2^-126 gives 0).  Exponent bias 1023 -> 127 is a
// subtraction of 896 << 20 from the high word; the 23-bit mantissa is the
// high word's 20 bits and the top 3 bits of the low word.  Integer
// operations only: the filters never touch the FP64 pipe.
__device__ __forceinline__ float f32_trunc(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned mag = hi & 0x7fffffffu;
    const unsigned b = mag >= (897u << 20) ? (((mag - (896u << 20)) << 3) | (lo >> 29)) : 0u;
    return __uint_as_float(b | (hi & 0x80000000u));
}

__device__ __forceinline__ double3 load_xyz(const double4_16a *__restrict__ pos, int i)
{
    const double2 *p2 = reinterpret_cast<const double2 *>(pos + i);
    const double2 a = __ldg(p2);
    const double2 b = __ldg(p2 + 1);
    return make_double3(a.x, a.y, b.x);
}

// The FP64 pair term of Phase B.  Same formulas as pair_accum<double>, with
// two changes that keep FP64-pipe work down and the result at FP64 accuracy:
//  * the cutoff and self tests compare bit patterns as integers (r^2 >= +0,
//    and non-negative doubles order as their bit patterns), off the FP64 pipe;
//  * 1/r^2 (or 1/r for the force-shifted form) starts from the hardware's
//    approximate FP64 reciprocal (reciprocal square root), relative error
//    h ~ 1e-6, and takes one third-order correction: the first three terms
//    of the series of 1/(1 - h) (of (1 - h)^(-1/2)), which cube the error.
//    Against IEEE division and square root the forces differ by ~1e-14
//    relative at most.
__device__ __forceinline__ double rcp64_approx(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}

__device__ __forceinline__ double rsqrt64_approx(double x)
{
    double r;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}

template <int MODE, bool ENERGY>
__device__ __forceinline__ void pair64(double dx, double dy, double dz, const Coef<double> &k, double &fx, double &fy,
                                       double &fz, double &e, double &w)
{
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const long long b = __double_as_longlong(r2);
    const bool in = b < __double_as_longlong(k.rc2) && b != 0;
    double ri, rinv = 0.0;
    if constexpr (MODE == 2) {
        double y = rsqrt64_approx(r2);
        const double h = fma(-r2 * y, y, 1.0);             // y = (1 - h)^(1/2) / sqrt(r2)
        y = fma(y, h * fma(h, 0.375, 0.5), y);               // (1 - h)^(-1/2) ~ 1 + h/2 + 3h^2/8
        rinv = in ? y : 0.0;
        ri = rinv * rinv;
    } else {
        double y = rcp64_approx(r2);
        const double h = fma(-r2, y, 1.0);                  // y = (1 - h) / r2
        y = fma(y, fma(h, h, h), y);                         // 1 / (1 - h) ~ 1 + h + h^2
        ri = in ? y : 0.0;
    }
    const double r6 = ri * ri * ri;
    double ff = ri * r6 * (k.a12 * r6 - k.b6);
    if constexpr (MODE == 2) ff -= k.fc * rinv;
    fx = fma(ff, dx, fx);
    fy = fma(ff, dy, fy);
    fz = fma(ff, dz, fz);
    if constexpr (ENERGY) {
        double u = r6 * (k.c12 * r6 - k.c6);
        if constexpr (MODE >= 1) u -= k.uc;
        if constexpr (MODE == 2) u += (r2 * rinv - k.rc) * k.fc;
        e += in ? u : 0.0;
        w += ff * r2;
    }
}

// The FP64 VJP term of one pair (the adjoint of the force, rc fixed): with
// d = x_i - x_j, phi = F(r)/r, g = g_i - g_j,
//   a  += phi g + (phi'(r)/r) (d . g) d      (J_ij (g_i - g_j)),
//   ae += phi|eps=1 (d . g_i)                (dF_i/deps . g_i),
//   as += eps (dphi/dsigma) (d . g_i)        (dF_i/dsigma . g_i);
// with q = r^2, phi = eps (A q^-7 - B q^-4) (A = 48 sigma^12, B = 24
// sigma^6), phi'(r)/r = eps q^-5 (8 B - 14 A q^-3), dphi/dsigma = eps (12 A
// q^-7 - 6 B q^-4) / sigma; the force shift adds -Fc/r to phi, +Fc/r^3 to
// phi'(r)/r and -(dFc/dsigma)/r to dphi/dsigma.  Same cutoff test and
// reciprocal as pair64.
template <int MODE>
__device__ __forceinline__ void vjp64(double dx, double dy, double dz, double gix, double giy, double giz,
                                      double gjx, double gjy, double gjz, const W64Params &k, double &ax,
                                      double &ay, double &az, double &ae, double &as)
{
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const long long b = __double_as_longlong(r2);
    const bool in = b < __double_as_longlong(k.rc2) && b != 0;
    double ri, rinv = 0.0;
    if constexpr (MODE == 2) {
        double y = rsqrt64_approx(r2);
        const double h = fma(-r2 * y, y, 1.0);
        y = fma(y, h * fma(h, 0.375, 0.5), y);
        rinv = in ? y : 0.0;
        ri = rinv * rinv;
    } else {
        double y = rcp64_approx(r2);
        const double h = fma(-r2, y, 1.0);
        y = fma(y, fma(h, h, h), y);
        ri = in ? y : 0.0;
    }
    const double r6 = ri * ri * ri;
    const double r8 = ri * r6;
    double phi1 = r8 * (k.va1 * r6 - k.vb1);
    double dphi1 = r8 * ri * (8.0 * k.vb1 - 14.0 * k.va1 * r6);
    double dsig1 = r8 * (12.0 * k.va1 * r6 - 6.0 * k.vb1) * k.visg;
    if constexpr (MODE == 2) {
        phi1 -= k.vfc1 * rinv;
        dphi1 += k.vfc1 * rinv * ri;
        dsig1 -= k.vdfc1 * rinv;
    }
    const double phi = k.veps * phi1, dphi = k.veps * dphi1;
    const double gx = gix - gjx, gy = giy - gjy, gz = giz - gjz;
    const double dot = fma(dz, gz, fma(dy, gy, dx * gx));
    const double gid = fma(dz, giz, fma(dy, giy, dx * gix));
    const double t = dphi * dot;
    ax = fma(t, dx, fma(phi, gx, ax));
    ay = fma(t, dy, fma(phi, gy, ay));
    az = fma(t, dz, fma(phi, gz, az));
    ae = fma(phi1, gid, ae);
    as = fma(k.veps * dsig1, gid, as);
}

struct Acc64 {
    double fx, fy, fz, e, w;
    __device__ __forceinline__ void zero() { fx = fy = fz = e = w = 0.0; }
};

// OP: 0 = forces, 1 = forces with energies and virials, 2 = VJP (the five
// sums are then dL/dx and the two parameter terms).

// Final sums of home particle `slot` (sorted index): the force, and its
// energy share and virial for OP 1; for OP 2 dx += scale a and the
// parameter terms into (eacc, wacc).
template <int OP>
__device__ __forceinline__ void w64_store(const W64Params &k, const double4_16a *__restrict__ pos,
                                          double4_16a *__restrict__ fout, int slot, const Acc64 &a, double &eacc,
                                          double &wacc)
{
    constexpr bool ENERGY = OP == 1;
    const int idx = (int)__ldg(&pos[slot].w);
    if ((unsigned)idx >= (unsigned)k.n) return;
    if constexpr (OP == 2) {
        k.dxo[3 * (int64_t)idx] += k.scale * a.fx;
        k.dxo[3 * (int64_t)idx + 1] += k.scale * a.fy;
        k.dxo[3 * (int64_t)idx + 2] += k.scale * a.fz;
        eacc += a.e;
        wacc += a.w;
        return;
    }
    double4_16a o;
    o.x = a.fx;
    o.y = a.fy;
    o.z = a.fz;
    o.w = ENERGY ? 0.5 * a.e : 0.0;
    fout[idx] = o;
    if constexpr (ENERGY) {
        eacc += 0.5 * a.e;
        wacc += 0.5 * a.w;
    }
}

// Plain path: lanes own home particles, FP64 over every candidate read from
// global memory per stencil cell (cells whose stencil overflows the slice).
template <int R, int MODE, int OP>
__device__ void w64_plain(const W64Params &k, const Coef<double> &kc, const double4_16a *__restrict__ pos,
                          double4_16a *__restrict__ fout, const float4 *stab, const double *S64, const int *spre,
                          int s_home, int n_home, double &eacc, double &wacc)
{
    constexpr int NS = Stencil<R>::NS;
    const int lane = threadIdx.x & 31;
    for (int p0 = 0; p0 < n_home; p0 += 32) {
        const int i = p0 + lane;
        const bool vi = i < n_home;
        const double3 pi = load_xyz(pos, s_home + (vi ? i : 0));
        double3 gi = make_double3(0.0, 0.0, 0.0);
        if constexpr (OP == 2) gi = load_xyz(k.g4, s_home + (vi ? i : 0));
        Acc64 a;
        a.zero();
        for (int kk = 0; kk < NS; kk++) {
            const int s = __float_as_int(stab[kk].w);
            const int nn = spre[kk + 1] - spre[kk];
            const double xs = pi.x - S64[kk], ys = pi.y - S64[NS + kk], zs = pi.z - S64[2 * NS + kk];
            for (int j = 0; j < nn; j++) {
                const double3 q = load_xyz(pos, s + j);
                if constexpr (OP == 2) {
                    const double3 h = load_xyz(k.g4, s + j);
                    vjp64<MODE>(xs - q.x, ys - q.y, zs - q.z, gi.x, gi.y, gi.z, h.x, h.y, h.z, k, a.fx, a.fy, a.fz,
                                a.e, a.w);
                } else {
                    pair_accum<double, MODE, OP == 1>(xs - q.x, ys - q.y, zs - q.z, kc, a.fx, a.fy, a.fz, a.e, a.w);
                }
            }
        }
        if (vi) w64_store<OP>(k, pos, fout, s_home + i, a, eacc, wacc);
    }
}

// Staging of one home cell's stencil: returns the number of kept candidates
// T, or -1 (nothing written that matters) when they would not fit the slice
// with the 64 padding entries Phase A reads.  With HX64 (VJP) the kept
// candidates' cotangents are staged too.
template <int NS, int P2>
__device__ __forceinline__ int w64_stage(const W64Params &k, const double4_16a *__restrict__ pos, float *X, float *Y,
                                         float *Z, double *X64, double *Y64, double *Z64, double *HX64,
                                         double *HY64, double *HZ64, int *Iw, const float4 *stab, const double *S64,
                                         const int *spre, int Ttot, int s_home, int n_home)
{
    const int lane = threadIdx.x & 31;
    float bxl = 3.4e38f, byl = 3.4e38f, bzl = 3.4e38f, bxh = -3.4e38f, byh = -3.4e38f, bzh = -3.4e38f;
    for (int p0 = 0; p0 < n_home; p0 += 32) {
        if (p0 + lane < n_home) {
            const double3 q = load_xyz(pos, s_home + p0 + lane);
            const float qx = f32_trunc(q.x), qy = f32_trunc(q.y), qz = f32_trunc(q.z);
            bxl = fminf(bxl, qx);
            byl = fminf(byl, qy);
            bzl = fminf(bzl, qz);
            bxh = fmaxf(bxh, qx);
            byh = fmaxf(byh, qy);
            bzh = fmaxf(bzh, qz);
        }
    }
    box_reduce(bxl, byl, bzl, bxh, byh, bzh);
    const unsigned lt = (1u << lane) - 1u;
    int T = 0;
    for (int t0 = 0; t0 < Ttot; t0 += 32 * kStageBatch) {
        double3 q[kStageBatch];
        float4 sh[kStageBatch];
        int kcs[kStageBatch], src[kStageBatch];
#pragma unroll
        for (int u = 0; u < kStageBatch; u++) {
            const int t = t0 + 32 * u + lane;
            q[u] = make_double3(0.0, 0.0, 0.0);
            sh[u] = make_float4(kFar, kFar, kFar, 0.f);
            kcs[u] = 0;
            src[u] = 0;
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
                sh[u] = stab[kc];
                kcs[u] = kc;
                src[u] = __float_as_int(sh[u].w) + (t - kb);
                q[u] = load_xyz(pos, src[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kStageBatch; u++) {
            if (T + 96 > k.cap) {   // this round (<= 32) plus 64 padding entries might not fit
                __syncwarp();
                return -1;
            }
            const int t = t0 + 32 * u + lane;
            const float cx = f32_trunc(q[u].x) + sh[u].x;
            const float cy = f32_trunc(q[u].y) + sh[u].y;
            const float cz = f32_trunc(q[u].z) + sh[u].z;
            const float dx = fmaxf(fmaxf(bxl - cx, cx - bxh), 0.f);
            const float dy = fmaxf(fmaxf(byl - cy, cy - byh), 0.f);
            const float dz = fmaxf(fmaxf(bzl - cz, cz - bzh), 0.f);
            const bool keep = t < Ttot && dx * dx + dy * dy + dz * dz < k.rc2_box;
            const unsigned kept = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int sl = T + __popc(kept & lt);
                const int kc = kcs[u];
                X[sl] = cx;
                Y[sl] = cy;
                Z[sl] = cz;
                X64[sl] = q[u].x + S64[kc];
                Y64[sl] = q[u].y + S64[NS + kc];
                Z64[sl] = q[u].z + S64[2 * NS + kc];
                if (HX64) {
                    const double3 h = load_xyz(k.g4, src[u]);
                    HX64[sl] = h.x;
                    HY64[sl] = h.y;
                    HZ64[sl] = h.z;
                }
                if (Iw) Iw[sl] = src[u];
            }
            T += __popc(kept);
        }
    }
    X[T + lane] = kFar;
    Y[T + lane] = kFar;
    Z[T + lane] = kFar;
    X[T + 32 + lane] = kFar;
    Y[T + 32 + lane] = kFar;
    Z[T + 32 + lane] = kFar;
    __syncwarp();
    return T;
}

// Phase B over one batch: entries [0, E) of the list, particles pb .. pb + P
// - 1 of the home cell with list offsets off[0 .. P].
template <int MODE, int OP>
__device__ __forceinline__ void w64_pairs(const W64Params &k, const Coef<double> &kc,
                                          const double4_16a *__restrict__ pos, double4_16a *__restrict__ fout,
                                          const double *X64, const double *Y64, const double *Z64,
                                          const double *HX64, const double *HY64, const double *HZ64,
                                          const uint16_t *list, const int *off, double *part, int E, int P,
                                          int pb, int s_home, double &eacc, double &wacc)
{
    constexpr bool ENERGY = OP >= 1;   // five sums, not three
    const int lane = threadIdx.x & 31;
    double *first = part;                 // [kW64Comp][32]
    double *head = part + kW64Comp * 32;  // [kW64Comp][32]
    const int lo = (lane * E) >> 5;
    const int hi = ((lane + 1) * E) >> 5;
    int headq = -1;
    if (lo < hi) {
        // q: the particle whose entries contain lo (largest q < P with off[q] <= lo)
        int q = 0;
#pragma unroll
        for (int step = kW64PMax / 2; step > 0; step >>= 1)
            if (q + step < P && off[q + step] <= lo) q += step;
        int nxt = off[q + 1];
        double xp = X64[pb + q], yp = Y64[pb + q], zp = Z64[pb + q];
        double gpx = 0.0, gpy = 0.0, gpz = 0.0;
        if constexpr (OP == 2) {
            gpx = HX64[pb + q];
            gpy = HY64[pb + q];
            gpz = HZ64[pb + q];
        }
        Acc64 a;
        a.zero();
        auto flush = [&]() {
            const bool starts = off[q] >= lo;
            const bool ends = nxt <= hi;
            if (starts && ends) {
                w64_store<OP>(k, pos, fout, s_home + pb + q, a, eacc, wacc);
            } else {
                double *dst = starts ? head : first;
                dst[0 * 32 + lane] = a.fx;
                dst[1 * 32 + lane] = a.fy;
                dst[2 * 32 + lane] = a.fz;
                if constexpr (ENERGY) {
                    dst[3 * 32 + lane] = a.e;
                    dst[4 * 32 + lane] = a.w;
                }
                if (starts) headq = q;
            }
        };
        for (int e = lo; e < hi; e++) {
            if (e == nxt) {
                flush();
                do {
                    q++;
                    nxt = off[q + 1];
                } while (nxt == e);   // particles without entries were stored in Phase A
                xp = X64[pb + q];
                yp = Y64[pb + q];
                zp = Z64[pb + q];
                if constexpr (OP == 2) {
                    gpx = HX64[pb + q];
                    gpy = HY64[pb + q];
                    gpz = HZ64[pb + q];
                }
                a.zero();
            }
            const int j = list[e];
            if constexpr (OP == 2) {
                vjp64<MODE>(xp - X64[j], yp - Y64[j], zp - Z64[j], gpx, gpy, gpz, HX64[j], HY64[j], HZ64[j], k, a.fx,
                            a.fy, a.fz, a.e, a.w);
            } else {
                pair64<MODE, ENERGY>(xp - X64[j], yp - Y64[j], zp - Z64[j], kc, a.fx, a.fy, a.fz, a.e, a.w);
            }
        }
        flush();
    }
    __syncwarp();
    if (headq >= 0) {
        // this lane holds the first entries of particle headq; the rest are
        // the first segments of the following non-empty lanes
        Acc64 a;
        a.fx = head[0 * 32 + lane];
        a.fy = head[1 * 32 + lane];
        a.fz = head[2 * 32 + lane];
        a.e = ENERGY ? head[3 * 32 + lane] : 0.0;
        a.w = ENERGY ? head[4 * 32 + lane] : 0.0;
        const int end = off[headq + 1];
        for (int l2 = lane + 1; l2 < 32; l2++) {
            const int lo2 = (l2 * E) >> 5, hi2 = ((l2 + 1) * E) >> 5;
            if (lo2 == hi2) continue;
            a.fx += first[0 * 32 + l2];
            a.fy += first[1 * 32 + l2];
            a.fz += first[2 * 32 + l2];
            if constexpr (ENERGY) {
                a.e += first[3 * 32 + l2];
                a.w += first[4 * 32 + l2];
            }
            if (end <= hi2) break;
        }
        w64_store<OP>(k, pos, fout, s_home + pb + headq, a, eacc, wacc);
    }
    __syncwarp();   // part, list and off are rewritten by the next batch
}

// Half-stencil table of home cell (cx, cy, cz) for the pair-once form:
// entries e = 0 (the home cell) .. 13 (the neighbours with (dz, dy, dx) > 0
// lexicographically), as stencil_table writes them for the full stencil
// (FP32 shift and first particle in stab, FP64 shifts in S64 with stride
// kN3Half, prefix sums in spre).  Returns the total.  All 32 lanes.
__device__ __forceinline__ int half_table64(const int32_t *__restrict__ start, int cx, int cy, int cz, int nc,
                                            float cw, float4 *stab, int *spre, double *S64, double cw64)
{
    const int lane = threadIdx.x & 31;
    int nn = 0;
    if (lane < kN3Half) {
        int dx, dy, dz;
        half_delta(lane, dx, dy, dz);
        int ux = cx + dx, uy = cy + dy, uz = cz + dz;
        ux += ux < 0 ? nc : 0;
        ux -= ux >= nc ? nc : 0;
        uy += uy < 0 ? nc : 0;
        uy -= uy >= nc ? nc : 0;
        uz += uz < 0 ? nc : 0;
        uz -= uz >= nc ? nc : 0;
        const int64_t cn = ux + (int64_t)nc * (uy + (int64_t)nc * uz);
        const int st = start[cn];
        nn = start[cn + 1] - st;
        stab[lane] = make_float4((float)dx * cw, (float)dy * cw, (float)dz * cw, __int_as_float(st));
        S64[lane] = (double)dx * cw64;
        S64[kN3Half + lane] = (double)dy * cw64;
        S64[2 * kN3Half + lane] = (double)dz * cw64;
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

// FP64 additions into the pair-once form's sums (zeroed before the launch),
// without a test for zero: a comparison of doubles would take FP64-pipe
// issue slots, the scarce resource here.
template <bool ENERGY>
__device__ __forceinline__ void add_force64(double4_16a *fs, int slot, double fx, double fy, double fz, double e)
{
    atomicAdd(&fs[slot].x, fx);
    atomicAdd(&fs[slot].y, fy);
    atomicAdd(&fs[slot].z, fz);
    if constexpr (ENERGY) atomicAdd(&fs[slot].w, e);
}

// The pair term of the pair-once form: returns -F(r)/r (0 outside rc or
// for r = 0), with the pair energy in u (ENERGY) and r^2.  Same formulas,
// cutoff test and reciprocal as pair64; the sign is taken into the
// coefficients, so that the reaction (-F/r d) and the home particle's
// subtraction need no negation.
template <int MODE, bool ENERGY>
__device__ __forceinline__ double pair64_nf(double dx, double dy, double dz, const Coef<double> &k, double &u,
                                            double &r2)
{
    r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const long long b = __double_as_longlong(r2);
    const bool in = b < __double_as_longlong(k.rc2) && b != 0;
    double ri, rinv = 0.0;
    if constexpr (MODE == 2) {
        double y = rsqrt64_approx(r2);
        const double h = fma(-r2 * y, y, 1.0);
        y = fma(y, h * fma(h, 0.375, 0.5), y);
        rinv = in ? y : 0.0;
        ri = rinv * rinv;
    } else {
        double y = rcp64_approx(r2);
        const double h = fma(-r2, y, 1.0);
        y = fma(y, fma(h, h, h), y);
        ri = in ? y : 0.0;
    }
    const double r6 = ri * ri * ri;
    double nf = ri * r6 * fma(-k.a12, r6, k.b6);
    if constexpr (MODE == 2) nf = fma(k.fc, rinv, nf);
    if constexpr (ENERGY) {
        double v = r6 * (k.c12 * r6 - k.c6);
        if constexpr (MODE >= 1) v -= k.uc;
        if constexpr (MODE == 2) v += (r2 * rinv - k.rc) * k.fc;
        u = in ? v : 0.0;
    }
    return nf;
}

// The VJP term of one pair in the pair-once form: with d = x_i - x_j and
// g = g_i - g_j (vjp64's notation), the contribution to i is J_ij g and,
// J_ij being even in d, the one to j is its negative.  Returns the one to j,
// r = -(phi g + (phi'(r)/r)(d . g) d), and adds the pair's two parameter
// terms, which over both particles are phi|eps=1 (d . g) and eps
// (dphi/dsigma) (d . g), to (ae, as).  The signs are folded into -eps, so
// that neither r nor i's subtraction of it needs a negation.
template <int MODE>
__device__ __forceinline__ void vjp64_po(double dx, double dy, double dz, double gx, double gy, double gz,
                                         const W64Params &k, double &rx, double &ry, double &rz, double &ae,
                                         double &as)
{
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const long long b = __double_as_longlong(r2);
    const bool in = b < __double_as_longlong(k.rc2) && b != 0;
    double ri, rinv = 0.0;
    if constexpr (MODE == 2) {
        double y = rsqrt64_approx(r2);
        const double h = fma(-r2 * y, y, 1.0);
        y = fma(y, h * fma(h, 0.375, 0.5), y);
        rinv = in ? y : 0.0;
        ri = rinv * rinv;
    } else {
        double y = rcp64_approx(r2);
        const double h = fma(-r2, y, 1.0);
        y = fma(y, fma(h, h, h), y);
        ri = in ? y : 0.0;
    }
    const double r6 = ri * ri * ri;
    const double r8 = ri * r6;
    double phi1 = r8 * (k.va1 * r6 - k.vb1);
    double dphi1 = r8 * ri * (8.0 * k.vb1 - 14.0 * k.va1 * r6);
    double dsig1 = r8 * (12.0 * k.va1 * r6 - 6.0 * k.vb1) * k.visg;
    if constexpr (MODE == 2) {
        phi1 -= k.vfc1 * rinv;
        dphi1 += k.vfc1 * rinv * ri;
        dsig1 -= k.vdfc1 * rinv;
    }
    const double dot = fma(dz, gz, fma(dy, gy, dx * gx));
    const double nphi = -k.veps * phi1;
    const double nt = (-k.veps * dphi1) * dot;
    rx = fma(nt, dx, nphi * gx);
    ry = fma(nt, dy, nphi * gy);
    rz = fma(nt, dz, nphi * gz);
    ae = fma(phi1, dot, ae);
    as = fma(k.veps * dsig1, dot, as);
}

// Phase B of the pair-once form over one batch (OP as w64_cell; for OP 2
// the sums are those of the VJP, vjp64_po): the list holds each pair
// once (home particle p, staged candidate j > p).  A lane evaluates its
// contiguous range of entries in FP64; the pair force goes to the home
// particle's running sum and, with the opposite sign, to the candidate's
// sum in fs (an FP64 atomic add per component); each running home sum is
// added to fs when the lane's entries of that particle end.  fs is in the
// cell order of the sorted positions, so the atomic adds of a cell and its
// neighbours stay within a few MB of L2.  Energies: half of each pair
// energy to both particles, the whole once to the FP64 totals.
template <int MODE, int OP>
__device__ __forceinline__ void w64_pairs_po(const W64Params &k, const Coef<double> &kc,
                                             double4_16a *__restrict__ fs, const double *X64, const double *Y64,
                                             const double *Z64, const double *HX64, const double *HY64,
                                             const double *HZ64, const int *Iw, const uint16_t *list, const int *off,
                                             int E, int P, int pb, int s_home, double &eacc, double &wacc)
{
    constexpr bool ENERGY = OP == 1;
    const int lane = threadIdx.x & 31;
    const int lo = (lane * E) >> 5;
    const int hi = ((lane + 1) * E) >> 5;
    if (lo < hi) {
        int q = 0;
#pragma unroll
        for (int step = kW64PMax / 2; step > 0; step >>= 1)
            if (q + step < P && off[q + step] <= lo) q += step;
        int nxt = off[q + 1];
        double xp = X64[pb + q], yp = Y64[pb + q], zp = Z64[pb + q];
        double gpx = 0.0, gpy = 0.0, gpz = 0.0;
        if constexpr (OP == 2) {
            gpx = HX64[pb + q];
            gpy = HY64[pb + q];
            gpz = HZ64[pb + q];
        }
        Acc64 a;
        a.zero();
        auto flush = [&]() {
            add_force64<ENERGY>(fs, s_home + pb + q, a.fx, a.fy, a.fz, 0.5 * a.e);
            if constexpr (OP >= 1) {   // energy and virial, or the two parameter sums: each pair once
                eacc += a.e;
                wacc += a.w;
            }
        };
        for (int e = lo; e < hi; e++) {
            if (e == nxt) {
                flush();
                do {
                    q++;
                    nxt = off[q + 1];
                } while (nxt == e);
                xp = X64[pb + q];
                yp = Y64[pb + q];
                zp = Z64[pb + q];
                if constexpr (OP == 2) {
                    gpx = HX64[pb + q];
                    gpy = HY64[pb + q];
                    gpz = HZ64[pb + q];
                }
                a.zero();
            }
            const int j = list[e];
            const double dx = xp - X64[j], dy = yp - Y64[j], dz = zp - Z64[j];
            double rx, ry, rz, u = 0.0;
            if constexpr (OP == 2) {
                vjp64_po<MODE>(dx, dy, dz, gpx - HX64[j], gpy - HY64[j], gpz - HZ64[j], k, rx, ry, rz, a.e, a.w);
            } else {
                double r2;
                const double nf = pair64_nf<MODE, ENERGY>(dx, dy, dz, kc, u, r2);
                rx = nf * dx;   // the reaction on j
                ry = nf * dy;
                rz = nf * dz;
                if constexpr (ENERGY) {
                    a.e += u;
                    a.w = fma(-nf, r2, a.w);
                }
            }
            a.fx -= rx;
            a.fy -= ry;
            a.fz -= rz;
            add_force64<ENERGY>(fs, Iw[j], rx, ry, rz, 0.5 * u);
        }
        flush();
    }
    __syncwarp();   // list and off are rewritten by the next batch
}

// Plain path of the pair-once form (a cell whose pruned half stencil
// overflows the slice): lanes own home particles, FP64 over the half
// stencil read from global memory, each pair's reaction added by the lane
// (fout: the sums in cell order).
template <int MODE, int OP>
__device__ void w64_plain_po(const W64Params &k, const Coef<double> &kc, const double4_16a *__restrict__ pos,
                             double4_16a *__restrict__ fout, const float4 *stab, const double *S64, const int *spre,
                             int s_home, int n_home, double &eacc, double &wacc)
{
    constexpr bool ENERGY = OP == 1;
    const int lane = threadIdx.x & 31;
    for (int p0 = 0; p0 < n_home; p0 += 32) {
        const int i = p0 + lane;
        const bool vi = i < n_home;
        const double3 pi = load_xyz(pos, s_home + (vi ? i : 0));
        double3 gi = make_double3(0.0, 0.0, 0.0);
        if constexpr (OP == 2) gi = load_xyz(k.g4, s_home + (vi ? i : 0));
        Acc64 a;
        a.zero();
        for (int kk = 0; kk < kN3Half; kk++) {
            const int st = __float_as_int(stab[kk].w);
            const int nn = spre[kk + 1] - spre[kk];
            const double xs = pi.x - S64[kk], ys = pi.y - S64[kN3Half + kk], zs = pi.z - S64[2 * kN3Half + kk];
            for (int j = (kk == 0 ? p0 + 1 : 0); j < nn; j++) {
                if (!vi || (kk == 0 && j <= i)) continue;
                const double3 q = load_xyz(pos, st + j);
                const double dx = xs - q.x, dy = ys - q.y, dz = zs - q.z;
                double rx, ry, rz, u = 0.0;
                if constexpr (OP == 2) {
                    const double3 h = load_xyz(k.g4, st + j);
                    vjp64_po<MODE>(dx, dy, dz, gi.x - h.x, gi.y - h.y, gi.z - h.z, k, rx, ry, rz, a.e, a.w);
                } else {
                    double r2;
                    const double nf = pair64_nf<MODE, ENERGY>(dx, dy, dz, kc, u, r2);
                    rx = nf * dx;
                    ry = nf * dy;
                    rz = nf * dz;
                    if constexpr (ENERGY) {
                        a.e += u;
                        a.w = fma(-nf, r2, a.w);
                    }
                }
                a.fx -= rx;
                a.fy -= ry;
                a.fz -= rz;
                add_force64<ENERGY>(fout, st + j, rx, ry, rz, 0.5 * u);
            }
        }
        if (vi) {
            add_force64<ENERGY>(fout, s_home + i, a.fx, a.fy, a.fz, 0.5 * a.e);
            if constexpr (OP >= 1) {
                eacc += a.e;
                wacc += a.w;
            }
        }
    }
}

// One home cell.  PO: the pair-once form (fout is then the zeroed sums in
// cell order: forces, or for OP 2 the VJP's dL/dx before the scale), over
// the half stencil, each in-range pair listed once.
template <int R, int MODE, int OP, bool PO>
__device__ void w64_cell(const W64Params &k, const Coef<double> &kc, const double4_16a *__restrict__ pos,
                         const int32_t *__restrict__ start, double4_16a *__restrict__ fout, unsigned char *slice,
                         int cx, int cy, int cz, double &eacc, double &wacc)
{
    static_assert(!PO || R == 1, "the pair-once form takes the 27-cell stencil's half");
    const W64Layout L(k.cap, R, k.lcap, OP == 2, PO);
    double *X64 = reinterpret_cast<double *>(slice + L.x64);
    double *Y64 = X64 + k.cap;
    double *Z64 = Y64 + k.cap;
    double *HX64 = OP == 2 ? reinterpret_cast<double *>(slice + L.h64) : nullptr;
    double *HY64 = OP == 2 ? HX64 + k.cap : nullptr;
    double *HZ64 = OP == 2 ? HY64 + k.cap : nullptr;
    double *part = reinterpret_cast<double *>(slice + L.part);
    float4 *stab = reinterpret_cast<float4 *>(slice + L.stab);
    double *S64 = reinterpret_cast<double *>(slice + L.s64);
    float *X = reinterpret_cast<float *>(slice + L.x32);
    float *Y = X + k.cap;
    float *Z = Y + k.cap;
    int *spre = reinterpret_cast<int *>(slice + L.spre);
    int *off = reinterpret_cast<int *>(slice + L.off);
    uint16_t *list = reinterpret_cast<uint16_t *>(slice + L.list);
    int *Iw = PO ? reinterpret_cast<int *>(slice + L.iw) : nullptr;
    const int lane = threadIdx.x & 31;
    const int nc = k.nc;

    __syncwarp();   // the slice still holds the previous cell's data
    const int carry = PO ? half_table64(start, cx, cy, cz, nc, k.cwf, stab, spre, S64, k.cw)
                         : stencil_table<R>(start, 0, cx, cy, cz, nc, k.cwf, stab, spre, S64, k.cw);
    const int n_home = spre[1];
    if (n_home == 0) return;
    const int s_home = __float_as_int(stab[0].w);
    int T = -1;
    if (carry <= 2 * k.cap) {
        if constexpr (PO)
            T = w64_stage<kN3Half, 16>(k, pos, X, Y, Z, X64, Y64, Z64, HX64, HY64, HZ64, Iw, stab, S64, spre,
                                       carry, s_home, n_home);
        else
            T = w64_stage<Stencil<R>::NS, 32>(k, pos, X, Y, Z, X64, Y64, Z64, HX64, HY64, HZ64, nullptr, stab, S64,
                                              spre, carry, s_home, n_home);
    }
    if (T < 0) {
        if constexpr (PO)
            w64_plain_po<MODE, OP>(k, kc, pos, fout, stab, S64, spre, s_home, n_home, eacc, wacc);
        else
            w64_plain<R, MODE, OP>(k, kc, pos, fout, stab, S64, spre, s_home, n_home, eacc, wacc);
        return;
    }
    const float2 *X2 = reinterpret_cast<const float2 *>(X);
    const float2 *Y2 = reinterpret_cast<const float2 *>(Y);
    const float2 *Z2 = reinterpret_cast<const float2 *>(Z);
    const unsigned lt = (1u << lane) - 1u;
    int p = 0;
    while (p < n_home) {
        // Phase A: lists of the batch's particles (home particle p sits at
        // staged position p; its list has at most T - 1 entries)
        const int pb = p;
        int E = 0;
        if (lane == 0) off[0] = 0;
        while (p < n_home && p - pb < kW64PMax && E + T <= k.lcap) {
            const float2 xs = make_float2(X[p], X[p]), ys = make_float2(Y[p], Y[p]), zs = make_float2(Z[p], Z[p]);
            const int E0 = E;
            for (int j0 = 0; j0 < T; j0 += 64) {
                const int jx = j0 + 2 * lane;
                const float2 qx = X2[(j0 >> 1) + lane], qy = Y2[(j0 >> 1) + lane], qz = Z2[(j0 >> 1) + lane];
                const float2 m1 = make_float2(-1.0f, -1.0f);
                const float2 dx = __ffma2_rn(qx, m1, xs);
                const float2 dy = __ffma2_rn(qy, m1, ys);
                const float2 dz = __ffma2_rn(qz, m1, zs);
                float2 r2 = __fmul2_rn(dx, dx);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                // pair-once: candidate j > p only (the home particles
                // before p listed p already; neighbour cells stage after
                // the home cell)
                const bool ina = r2.x < k.rc2_pair && (PO ? jx > p : jx != p);
                const bool inb = r2.y < k.rc2_pair && (PO ? jx + 1 > p : jx + 1 != p);
                const unsigned ba = __ballot_sync(0xffffffffu, ina);
                const unsigned bb = __ballot_sync(0xffffffffu, inb);
                if (ina) list[E + __popc(ba & lt)] = (uint16_t)jx;
                if (inb) list[E + __popc(ba) + __popc(bb & lt)] = (uint16_t)(jx + 1);
                E += __popc(ba) + __popc(bb);
            }
            if (lane == 0) off[p - pb + 1] = E;
            if (!PO && OP != 2 && E == E0 && lane == 0) {
                // no candidate within rc: the force is zero (a VJP adds nothing)
                Acc64 a;
                a.zero();
                w64_store<OP>(k, pos, fout, s_home + p, a, eacc, wacc);
            }
            p++;
        }
        __syncwarp();
        // Phase B
        if constexpr (PO)
            w64_pairs_po<MODE, OP>(k, kc, fout, X64, Y64, Z64, HX64, HY64, HZ64, Iw, list, off, E, p - pb, pb, s_home,
                                   eacc, wacc);
        else
            w64_pairs<MODE, OP>(k, kc, pos, fout, X64, Y64, Z64, HX64, HY64, HZ64, list, off, part, E, p - pb, pb,
                                s_home, eacc, wacc);
    }
}

template <int R, int MODE, int OP, bool PO>
__global__ void __launch_bounds__(kW64Threads) k_force_w64(W64Params k, const double4_16a *__restrict__ pos,
                                                           const int32_t *__restrict__ start,
                                                           double4_16a *__restrict__ fout,
                                                           double *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char w64smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const W64Layout L(k.cap, R, k.lcap, OP == 2, PO);
    unsigned char *slice = w64smem + (size_t)warp * L.bytes;
    const Coef<double> kc(k);
    const int nc = k.nc;
    double eacc = 0.0, wacc = 0.0;
    auto one_cell = [&](int64_t c) {
        const int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        w64_cell<R, MODE, OP, PO>(k, kc, pos, start, fout, slice, cx, cy, cz, eacc, wacc);
    };
    if (k.grab > 0) {
        for (;;) {
            unsigned c0 = 0;
            if (lane == 0) c0 = atomicAdd(k.work, (unsigned)k.grab);
            c0 = __shfl_sync(0xffffffffu, c0, 0);
            if ((int64_t)c0 >= k.ncell) break;
            const int64_t c1 = min((int64_t)c0 + k.grab, k.ncell);
            for (int64_t c = c0; c < c1; c++) one_cell(c);
        }
    } else {
        const int64_t nwarps = (int64_t)gridDim.x * (kW64Threads / 32);
        for (int64_t c = (int64_t)blockIdx.x * (kW64Threads / 32) + warp; c < k.ncell; c += nwarps) one_cell(c);
    }
    if constexpr (OP >= 1) {   // energy and virial, or the two parameter sums
        __shared__ double red[2 * (kW64Threads / 32)];
        for (int o = 16; o > 0; o >>= 1) {
            eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
            wacc += __shfl_xor_sync(0xffffffffu, wacc, o);
        }
        if (lane == 0) {
            red[2 * warp] = eacc;
            red[2 * warp + 1] = wacc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double es = 0.0, ws = 0.0;
            for (int q = 0; q < kW64Threads / 32; q++) {
                es += red[2 * q];
                ws += red[2 * q + 1];
            }
            partial[2 * blockIdx.x] = es;
            partial[2 * blockIdx.x + 1] = ws;
        }
    }
}

// FP64 contexts use the 27-cell stencil (subdivision 1) only.  op: see OP;
// po: the pair-once form.
void *w64_kernel(int mode, int op, bool po = false)
{
    if (op == 2) {   // modes 0 and 1: the same force
        if (po) return mode == 2 ? (void *)k_force_w64<1, 2, 2, true> : (void *)k_force_w64<1, 0, 2, true>;
        return mode == 2 ? (void *)k_force_w64<1, 2, 2, false> : (void *)k_force_w64<1, 0, 2, false>;
    }
    switch (mode * 4 + (op == 1 ? 2 : 0) + (po ? 1 : 0)) {
        case 0: return (void *)k_force_w64<1, 0, 0, false>;
        case 1: return (void *)k_force_w64<1, 0, 0, true>;
        case 2: return (void *)k_force_w64<1, 0, 1, false>;
        case 3: return (void *)k_force_w64<1, 0, 1, true>;
        case 4: return (void *)k_force_w64<1, 1, 0, false>;
        case 5: return (void *)k_force_w64<1, 1, 0, true>;
        case 6: return (void *)k_force_w64<1, 1, 1, false>;
        case 7: return (void *)k_force_w64<1, 1, 1, true>;
        case 8: return (void *)k_force_w64<1, 2, 0, false>;
        case 9: return (void *)k_force_w64<1, 2, 0, true>;
        case 10: return (void *)k_force_w64<1, 2, 1, false>;
        default: return (void *)k_force_w64<1, 2, 1, true>;
    }
}

// f[perm[s]] = fs[s]: the pair-once form's sums from cell order to
// particle order.
__global__ void k_unsort64(const double4_16a *__restrict__ fs, const int32_t *__restrict__ perm,
                           double4_16a *__restrict__ f, int n)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) f[perm[s]] = fs[s];
}

// dx[perm[s]] += scale vs[s]: the pair-once VJP's sums from cell order to
// particle order, (n, 3) rows.
__global__ void k_unsort_add64(const double4_16a *__restrict__ vs, const int32_t *__restrict__ perm,
                               double *__restrict__ dx, double scale, int n)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) {
        const double4_16a v = vs[s];
        double *o = dx + 3 * (int64_t)perm[s];
        o[0] = fma(scale, v.x, o[0]);
        o[1] = fma(scale, v.y, o[1]);
        o[2] = fma(scale, v.z, o[2]);
    }
}

W64Params w64_params_of(const lj_ctx *c)
{
    W64Params k;
    memset(&k, 0, sizeof(k));
    k.n = (int)c->p.n;
    k.nc = c->nc;
    k.cap = c->wcap;
    k.lcap = c->w64_lcap;
    k.grab = c->grab;
    k.work = c->work;
    k.ncell = c->ncell;
    k.cwf = (float)c->cw;
    k.cw = c->cw;
    const double eps = c->p.eps, sg = c->p.sigma, rc = c->p.rc;
    const double s6 = sg * sg * sg * sg * sg * sg, s12 = s6 * s6;
    const double rci2 = 1.0 / (rc * rc), rci6 = rci2 * rci2 * rci2;
    k.rc2 = rc * rc;
    k.rc = rc;
    // FP32 filters: the bounding-box test as in the FP32-mixed kernel, the
    // pair test with a relative margin of 1e-4 on rc^2 (the truncated FP32
    // coordinates are within ~1e-6 of the FP64 ones)
    k.rc2_box = (float)(rc * rc) * 1.0001f;
    k.rc2_pair = (float)(rc * rc * (1.0 + 1e-4));
    k.a12 = 48.0 * eps * s12;
    k.b6 = 24.0 * eps * s6;
    k.c12 = 4.0 * eps * s12;
    k.c6 = 4.0 * eps * s6;
    k.uc = rci6 * (4.0 * eps * s12 * rci6 - 4.0 * eps * s6);
    k.fc = rc * rci2 * rci6 * (48.0 * eps * s12 * rci6 - 24.0 * eps * s6);
    return k;
}

}  // namespace

cudaError_t w64_force_configure(lj_ctx *c)
{
    if (c->p.cell_subdiv == 2) return cudaErrorInvalidValue;
    const int subdiv = 1;
    const int ns = (2 * subdiv + 1) * (2 * subdiv + 1) * (2 * subdiv + 1);
    const double mean = c->ncell > 0 ? (double)c->p.n / (double)c->ncell : 0.0;
    // Kept candidates: about 0.65 of the stencil population m after the
    // bounding-box pruning; capacity 0.75 m + 4 sqrt(m) + the 96 entries of
    // the last round and the padding, at least 160, at most what fits 227 KB
    // per CTA.  The list holds 1024 entries (~55 per particle at liquid
    // density, ~730 per cell); a cell's particles whose lists exceed it are
    // taken in batches.  A smaller slice means more resident warps: 10 per
    // SM at liquid density (measured 8.40 -> 7.73 ms at 4M against 8 warps
    // with a 2048-entry list).
    // Denser systems than the slice holds take the plain path in the cells
    // that overflow.  lcap >= cap, so one particle's list always fits.
    const double m = (double)ns * mean;
    int cap = (int)(0.75 * m + 4.0 * sqrt(m)) + 96;
    cap = cap < 160 ? 160 : cap;
    cap = (cap + 7) & ~7;
    const int lcap = 1024;
    const int warps = kW64Threads / 32;
    const int limit = 227 * 1024 - 2 * warps * (int)sizeof(double) - 256;
    while (cap > 160 && (cap > lcap || warps * W64Layout(cap, subdiv, lcap).bytes > limit)) cap -= 8;
    if (warps * W64Layout(cap, subdiv, lcap).bytes > limit) return cudaErrorInvalidValue;
    c->wcap = cap;
    c->w64_lcap = lcap;
    c->wforce_smem = warps * W64Layout(cap, subdiv, lcap).bytes;
    int minblk = 1 << 30;
    for (int mode = 0; mode < 3; mode++)
        for (int en = 0; en < 2; en++) {
            void *kern = w64_kernel(mode, en);
            cudaError_t e = raise_dyn_smem(kern, c->wforce_smem);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kW64Threads, c->wforce_smem);
            if (e != cudaSuccess) return e;
            if (nb < minblk) minblk = nb;
        }
    if (minblk < 1) minblk = 1;
    const int64_t need = (c->ncell + warps - 1) / warps;
    int64_t grid = (int64_t)minblk * c->nsm;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    c->wforce_grid = (int)grid;

    // The pair-once form stages the half stencil: m = 14 n_cell raw
    // candidates, with the same capacity rule; its lists are half as long.
    // Its sums go to a buffer in cell order (the context's f_sorted),
    // copied to f in particle order after the launch.
    const double mh = (double)kN3Half * mean;
    int hcap = (int)(0.75 * mh + 4.0 * sqrt(mh)) + 96;
    hcap = hcap < 160 ? 160 : hcap;
    hcap = (hcap + 7) & ~7;
    while (hcap > 160 && (hcap > lcap || warps * W64Layout(hcap, subdiv, lcap, false, true).bytes > limit)) hcap -= 8;
    if (warps * W64Layout(hcap, subdiv, lcap, false, true).bytes > limit) return cudaErrorInvalidValue;
    c->n3cap = hcap;
    c->n3_smem = warps * W64Layout(hcap, subdiv, lcap, false, true).bytes;
    minblk = 1 << 30;
    for (int mode = 0; mode < 3; mode++)
        for (int en = 0; en < 2; en++) {
            void *kern = w64_kernel(mode, en, true);
            cudaError_t e = raise_dyn_smem(kern, c->n3_smem);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kW64Threads, c->n3_smem);
            if (e != cudaSuccess) return e;
            if (nb < minblk) minblk = nb;
        }
    if (minblk < 1) minblk = 1;
    grid = (int64_t)minblk * c->nsm;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    c->n3_grid = (int)grid;
    return cudaSuccess;
}

cudaError_t launch_force_w64(lj_ctx *c, void *f, bool energy)
{
    // pair-once form (sums by atomic adds, into the context's buffer in cell
    // order) unless the context asks for sums in a fixed order or has no
    // such buffer
    const bool po = c->n3 && !c->deterministic && c->f_sorted;
    W64Params k = w64_params_of(c);
    if (po) k.cap = c->n3cap;
    const double4_16a *pos = (const double4_16a *)c->pos;
    const int32_t *start = c->start;
    double *partial = c->partial;
    void *kern = w64_kernel(c->p.shift_mode, energy ? 1 : 0, po);
    const int grid = po ? c->n3_grid : c->wforce_grid;
    const int smem = po ? c->n3_smem : c->wforce_smem;
    void *fk = po ? c->f_sorted : f;
    void *args[] = {&k, (void *)&pos, (void *)&start, &fk, &partial};
    if (c->timing && c->ev_used + 2 <= c->nev) cudaEventRecord(c->ev[c->ev_used], c->stream);
    cudaError_t e = cudaSuccess;
    if (po && c->p.n > 0) e = cudaMemsetAsync(c->f_sorted, 0, (size_t)c->p.n * sizeof(double4_16a), c->stream);
    if (e == cudaSuccess)
        e = cudaLaunchKernel(kern, dim3(grid), dim3(kW64Threads), args, smem, c->stream);
    if (e == cudaSuccess && po && c->p.n > 0) {
        const int nb = (int)((c->p.n + 255) / 256);
        k_unsort64<<<nb, 256, 0, c->stream>>>((const double4_16a *)c->f_sorted, c->perm, (double4_16a *)f,
                                              (int)c->p.n);
        c->kernel_launches++;
        e = cudaGetLastError();
    }
    if (c->timing && c->ev_used + 2 <= c->nev) {
        cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
        c->ev_used += 2;
    }
    if (po) c->npartial = grid;
    c->kernel_launches++;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_vjp_w64(lj_ctx *c, double scale, double *dx, double a1, double b1, double fc1, double dfc1,
                           int *grid_out)
{
    // pair-once form (as launch_force_w64) into the cell-order buffer, then
    // dx += scale * the buffer in particle order
    const bool po = c->n3 && !c->deterministic && c->f_sorted && c->n3cap > 0;
    W64Params k = w64_params_of(c);
    if (po) k.cap = c->n3cap;
    k.g4 = (const double4_16a *)c->g4;
    k.dxo = dx;
    k.scale = scale;
    k.va1 = a1;
    k.vb1 = b1;
    k.vfc1 = fc1;
    k.vdfc1 = dfc1;
    k.veps = c->p.eps;
    k.visg = 1.0 / c->p.sigma;
    k.grab = 0;   // static striding: the work counter belongs to the force kernel
    const int smem = (kW64Threads / 32) * W64Layout(k.cap, 1, c->w64_lcap, true, po).bytes;
    void *kern = w64_kernel(c->p.shift_mode, 2, po);
    cudaError_t e = raise_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kW64Threads, smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)(nb > 0 ? nb : 1) * c->nsm;
    const int64_t need = (c->ncell + kW64Threads / 32 - 1) / (kW64Threads / 32);
    if (grid > need) grid = need;
    if (grid > c->npartial_cap) grid = c->npartial_cap;
    if (grid < 1) grid = 1;
    const double4_16a *pos = (const double4_16a *)c->pos;
    const int32_t *start = c->start;
    double4_16a *fout = po ? (double4_16a *)c->f_sorted : nullptr;
    double *partial = c->partial;
    void *args[] = {&k, (void *)&pos, (void *)&start, &fout, &partial};
    if (po && c->p.n > 0) {
        e = cudaMemsetAsync(c->f_sorted, 0, (size_t)c->p.n * sizeof(double4_16a), c->stream);
        if (e != cudaSuccess) return e;
    }
    e = cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kW64Threads), args, smem, c->stream);
    c->kernel_launches++;
    if (e != cudaSuccess) return e;
    if (po && c->p.n > 0) {
        const int nblk = (int)((c->p.n + 255) / 256);
        k_unsort_add64<<<nblk, 256, 0, c->stream>>>((const double4_16a *)c->f_sorted, c->perm, dx, scale,
                                                    (int)c->p.n);
        c->kernel_launches++;
    }
    *grid_out = (int)grid;
    return cudaGetLastError();
}
