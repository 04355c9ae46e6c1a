// Lennard-Jones forces over cell lists, warp-per-cell variant (FP32-mixed).
//
// Same method as lj_force.cu (Section 3: a particle interacts with the
// particles of its own and the neighbouring cells; Section 2 pair force),
// organised for GB300:
//  * Warps work independently (no CTA barriers): a persistent grid whose
//    warps pull runs of consecutive home cells from an atomic counter (or
//    take cells w, w + W, ... by static striding), so warps of one CTA work
//    on neighbouring cells and share L1 lines.
//  * Cell side >= rc / k for subdivision k = 1 (the paper's 27-cell stencil)
//    or k = 2 (125-cell stencil of half-size cells); the stencil radius is
//    the template parameter R = k.
//  * Per home cell the warp writes the stencil table (start, count, shift)
//    to its own slice of shared memory, then stages the stencil's particles
//    as one flat list, converting every candidate to coordinates relative to
//    the HOME cell centre (|x| <= (R + 1/2) cell sides, so FP32 keeps ~1e-7
//    absolute resolution) and dropping candidates farther than rc from the
//    home particles' bounding box.
//  * The compute phase takes the home particles in chunks of G lanes
//    (by default G = 16 for the 27-cell stencil and 4 for the 125-cell one,
//    compiled in; a general kernel takes G from the tuning or chooses it per
//    cell to minimise idle lanes): lane g of a
//    group owns particle g of the chunk, the S = 32/G groups split the
//    candidates.  Staged data are SoA, so one 8-byte shared load gives a
//    lane its next two candidates, evaluated together with packed FP32x2
//    arithmetic (__ffma2_rn / __fmul2_rn).
//  * Stencils that do not fit the warp's slice take a plain path reading
//    global memory per stencil cell.
#include <math.h>
#include <string.h>

#include "lj_force_cell.cuh"

namespace {

// EPI 0: store forces (and energies); EPI 1: apply the fused velocity-Verlet
// update (KickDriftBin) to each particle instead.
// GFIX > 0: that group width compiled in (the default); 0: chosen per cell
// or fixed at run time by the tuning (k.gw).
template <int R, int MODE, bool ENERGY, int EPI, int GFIX>
__global__ void __launch_bounds__(kWarpForceThreads, 4) k_force_warp(WarpParams k, const float4 *__restrict__ pos,
                                                                  const int32_t *__restrict__ start,
                                                                  float4 *__restrict__ fout,
                                                                  double *__restrict__ partial, KickDriftBin kd)
{
    extern __shared__ __align__(16) float wsmem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *slice = wsmem + (size_t)warp * warp_slice_words(k.cap, R);
    const int nc = k.nc;
    double eacc = 0.0, wacc = 0.0;
    auto one_cell = [&](int64_t c) {
        const int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        if constexpr (EPI == 0) {
            const StoreForce<MODE, ENERGY> out{fout, k.n};
            process_home_cell<R, MODE, ENERGY, true, GFIX>(k, pos, start, out, slice, cx, cy, cz, nc, 0, k.cw, eacc, wacc);
        } else {
            process_home_cell<R, MODE, ENERGY, true, GFIX>(k, pos, start, kd, slice, cx, cy, cz, nc, 0, k.cw, eacc, wacc);
        }
    };
    if (k.grab > 0) {
        // dynamic: warps pull chunks of `grab` consecutive cells
        for (;;) {
            unsigned c0 = 0;
            if (lane == 0) c0 = atomicAdd(k.work, (unsigned)k.grab);
            c0 = __shfl_sync(0xffffffffu, c0, 0);
            if ((int64_t)c0 >= k.ncell) break;
            const int64_t c1 = min((int64_t)c0 + k.grab, k.ncell);
            for (int64_t c = c0; c < c1; c++) one_cell(c);
        }
    } else {
        const int64_t nwarps = (int64_t)gridDim.x * (kWarpForceThreads / 32);
        for (int64_t c = (int64_t)blockIdx.x * (kWarpForceThreads / 32) + warp; c < k.ncell; c += nwarps) one_cell(c);
    }
    if constexpr (ENERGY) {
        __shared__ double red[2 * (kWarpForceThreads / 32)];
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
            for (int q = 0; q < kWarpForceThreads / 32; q++) {
                es += red[2 * q];
                ws += red[2 * q + 1];
            }
            partial[2 * blockIdx.x] = es;
            partial[2 * blockIdx.x + 1] = ws;
        }
    }
}

template <int R, int G>
void *warp_kernel_rg(int mode, bool energy, bool fused)
{
    if (fused) {
        switch (mode) {
            case 0: return (void *)k_force_warp<R, 0, false, 1, G>;
            case 1: return (void *)k_force_warp<R, 1, false, 1, G>;
            default: return (void *)k_force_warp<R, 2, false, 1, G>;
        }
    }
    switch (mode * 2 + (energy ? 1 : 0)) {
        case 0: return (void *)k_force_warp<R, 0, false, 0, G>;
        case 1: return (void *)k_force_warp<R, 0, true, 0, G>;
        case 2: return (void *)k_force_warp<R, 1, false, 0, G>;
        case 3: return (void *)k_force_warp<R, 1, true, 0, G>;
        case 4: return (void *)k_force_warp<R, 2, false, 0, G>;
        default: return (void *)k_force_warp<R, 2, true, 0, G>;
    }
}

// The default width (gw 0) runs the kernel with it compiled in; any other
// tuning (a fixed width, or -1 = choose per cell) runs the general kernel.
template <int R>
void *warp_kernel_r(int mode, bool energy, bool fused, int gw)
{
    if (gw == 0) return warp_kernel_rg<R, DefaultGroup<R>::value>(mode, energy, fused);
    return warp_kernel_rg<R, 0>(mode, energy, fused);
}

void *warp_kernel(int subdiv, int mode, bool energy, bool fused, int gw)
{
    return subdiv == 2 ? warp_kernel_r<2>(mode, energy, fused, gw) : warp_kernel_r<1>(mode, energy, fused, gw);
}

}  // namespace

int warp_stencil_cap(double mean_occupancy, int subdiv, int threads, int static_bytes)
{
    // Staged candidates per warp: the largest slice with which 4 CTAs fit in
    // an SM's shared memory (228 KB, 1 KB reserved per CTA).  Raised (then
    // fewer CTAs fit) only when the mean stencil population m plus 4 sqrt(m)
    // (a Poisson spread) plus the 32-entry padding exceeds it: dense systems.
    // Multiple of 8, at least 40.
    const int R = subdiv == 2 ? 2 : 1;
    const int warps = threads / 32;
    const int ns = (2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    auto cap_for = [&](int bytes_per_cta) {
        const int words = (bytes_per_cta - static_bytes) / (4 * warps);
        return ((words - warp_slice_words(0, R)) / 3) & ~7;
    };
    const int cap4 = cap_for(228 * 1024 / 4 - 1024);
    const int cap1 = cap_for(227 * 1024);
    const double m = (double)ns * mean_occupancy;
    int need = (int)(m + 4.0 * sqrt(m)) + 32;
    need = (need + 7) & ~7;
    int cap = need > cap4 ? (need < cap1 ? need : cap1) : cap4;
    return cap < 40 ? 40 : cap;
}

cudaError_t warp_force_configure(lj_ctx *c)
{
    const int subdiv = c->p.cell_subdiv == 2 ? 2 : 1;
    double mean = c->ncell > 0 ? (double)c->p.n / (double)c->ncell : 0.0;
    c->wcap = warp_stencil_cap(mean, subdiv, kWarpForceThreads, 2 * (kWarpForceThreads / 32) * (int)sizeof(double));
    c->wforce_smem = (kWarpForceThreads / 32) * warp_slice_words(c->wcap, subdiv) * (int)sizeof(float);
    int minblk = 1 << 30;
    for (int mode = 0; mode < 3; mode++)
        for (int en = 0; en < 6; en++) {
            void *kern = warp_kernel(subdiv, mode, en % 3 == 1, en % 3 == 2, en < 3 ? 0 : -1);
            cudaError_t e = raise_dyn_smem(kern, c->wforce_smem);
            if (e != cudaSuccess) return e;
            // shared memory for 4 resident CTAs and no more: the rest of the
            // SM's 256 KB stays L1, which caches the stencil reads
            const int pct = (int)((100.0 * 4.0 * (c->wforce_smem + 1024 + 2 * (kWarpForceThreads / 32) * 8)) /
                                  (228.0 * 1024.0)) + 1;
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct > 100 ? 100 : pct);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kWarpForceThreads, c->wforce_smem);
            if (e != cudaSuccess) return e;
            if (nb < minblk) minblk = nb;
        }
    if (minblk < 1) minblk = 1;
    int64_t cells_per_block = kWarpForceThreads / 32;
    int64_t need = (c->ncell + cells_per_block - 1) / cells_per_block;
    int64_t grid = (int64_t)minblk * c->nsm;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    c->wforce_grid = (int)grid;
    return cudaSuccess;
}

namespace {

cudaError_t launch_warp(lj_ctx *c, void *kern, WarpParams k, void *f, KickDriftBin kd)
{
    const float4 *pos = (const float4 *)c->pos;
    const int32_t *start = c->start;
    double *partial = c->partial;
    void *args[] = {&k, (void *)&pos, (void *)&start, &f, &partial, &kd};
    if (c->timing && c->ev_used + 2 <= c->nev) cudaEventRecord(c->ev[c->ev_used], c->stream);
    cudaError_t e = cudaLaunchKernel(kern, dim3(c->wforce_grid), dim3(kWarpForceThreads), args, c->wforce_smem,
                                     c->stream);
    if (c->timing && c->ev_used + 2 <= c->nev) {
        cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
        c->ev_used += 2;
    }
    c->kernel_launches++;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

bool uses_force_n3(const lj_ctx *c)
{
    return c->p.n > 0 && !c->use_aop && !c->use_run_kernel && c->p.precision != LJ_PREC_FP64 &&
           c->p.cell_subdiv != 2 && !c->pipe && c->n3 && !c->deterministic;
}

cudaError_t launch_force_warp(lj_ctx *c, void *f, bool energy)
{
    if (c->p.precision == LJ_PREC_FP64) return launch_force_w64(c, f, energy);
    // tuning choice: stencils bulk-copied one cell ahead (lj_force_pipe.cu)
    if (c->p.cell_subdiv != 2 && c->pipe) return launch_force_pipe(c, f, energy);
    // each pair once (lj_force_n3.cu); its atomic sums have no fixed order,
    // so the deterministic in-cell mode keeps this 27-cell kernel
    if (c->p.cell_subdiv != 2 && c->n3 && !c->deterministic) return launch_force_n3(c, f, energy);
    KickDriftBin kd;
    memset(&kd, 0, sizeof(kd));
    return launch_warp(c, warp_kernel(c->p.cell_subdiv, c->p.shift_mode, energy, false, c->gw), warp_params_of(c), f, kd);
}

cudaError_t launch_force_warp_fused(lj_ctx *c, void *f, double *x, double *v, bool last)
{
    KickDriftBin kd;
    memset(&kd, 0, sizeof(kd));
    kd.fout = (float4 *)f;
    kd.n = (int)c->p.n;
    kd.x = x;
    kd.v = v;
    kd.last = last ? 1 : 0;
    kd.hk = (last ? 0.5 : 1.0) * c->p.dt / c->p.mass;
    kd.dt = c->p.dt;
    kd.L = c->p.box;
    kd.whi = c->wrap_hi;
    kd.wlo = c->wrap_lo;
    kd.s = c->inv_cw;
    kd.nc = c->nc;
    kd.thb = c->thb;
    kd.cell_of = c->cell_of;
    kd.rank = c->rank;
    kd.count = c->count;
    kd.err = c->err;
    return launch_warp(c, warp_kernel(c->p.cell_subdiv, c->p.shift_mode, false, true, c->gw), warp_params_of(c), f, kd);
}
