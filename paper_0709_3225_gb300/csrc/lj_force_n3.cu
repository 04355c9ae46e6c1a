// The pair-once force kernel for single systems (FP32-mixed; the design and
// the device code are in lj_force_n3.cuh): configuration and launch.
#include <string.h>

#include "lj_force_n3.cuh"

namespace {

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kN3Threads, 6) k_force_n3(WarpParams k, const float4 *__restrict__ pos,
                                                         const int32_t *__restrict__ start, float4 *__restrict__ fout,
                                                         double *__restrict__ partial)
{
    extern __shared__ __align__(16) float nsmem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float4 *S = reinterpret_cast<float4 *>(nsmem + (size_t)warp * n3_slice_words(k.cap));
    float4 *stab = S + k.cap;
    int *spre = reinterpret_cast<int *>(stab + kN3Half);
    float4 *H = reinterpret_cast<float4 *>(spre + 16);
    const int nc = k.nc;
    double eacc = 0.0, wacc = 0.0;
    auto one_cell = [&](HalfLoad tl) {
        n3_cell<MODE, ENERGY, true>(k, pos, fout, tl, k.cw, S, stab, spre, H, eacc, wacc);
    };
    if (k.grab > 0) {
        // pulls of k.grab cells, then single cells over the last stretch (two
        // rounds of pulls of the whole grid), so that the warps finish closer
        // together
        const int64_t tail = 2 * (int64_t)k.grab * gridDim.x * (kN3Threads / 32);
        unsigned last = 0;
        for (;;) {
            const unsigned g = (int64_t)last + tail >= k.ncell ? 1u : (unsigned)k.grab;
            unsigned c0 = 0;
            if (lane == 0) c0 = atomicAdd(k.work, g);
            c0 = __shfl_sync(0xffffffffu, c0, 0);
            if ((int64_t)c0 >= k.ncell) break;
            last = c0;
            const int c1 = (int)min((int64_t)c0 + g, k.ncell);
            // the next cell's table loads are issued before this cell's work
            HalfLoad nxt = half_load<true>(start, (int)c0, nc, k.inv_nc);
            for (int c = (int)c0; c < c1; c++) {
                const HalfLoad cur = nxt;
                if (c + 1 < c1) nxt = half_load<true>(start, c + 1, nc, k.inv_nc);
                one_cell(cur);
            }
        }
    } else {
        const int nwarps = gridDim.x * (kN3Threads / 32);
        int c = blockIdx.x * (kN3Threads / 32) + warp;
        HalfLoad nxt = half_load<true>(start, c < k.ncell ? c : 0, nc, k.inv_nc);
        for (; c < k.ncell; c += nwarps) {
            const HalfLoad cur = nxt;
            if (c + nwarps < k.ncell) nxt = half_load<true>(start, c + nwarps, nc, k.inv_nc);
            one_cell(cur);
        }
    }
    if constexpr (ENERGY) {
        __shared__ double red[2 * (kN3Threads / 32)];
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
            for (int q = 0; q < kN3Threads / 32; q++) {
                es += red[2 * q];
                ws += red[2 * q + 1];
            }
            partial[2 * blockIdx.x] = es;
            partial[2 * blockIdx.x + 1] = ws;
        }
    }
}

void *n3_kernel(int mode, bool energy)
{
    switch (mode * 2 + (energy ? 1 : 0)) {
        case 0: return (void *)k_force_n3<0, false>;
        case 1: return (void *)k_force_n3<0, true>;
        case 2: return (void *)k_force_n3<1, false>;
        case 3: return (void *)k_force_n3<1, true>;
        case 4: return (void *)k_force_n3<2, false>;
        default: return (void *)k_force_n3<2, true>;
    }
}

}  // namespace

cudaError_t n3_force_configure(lj_ctx *c)
{
    // Staged candidates per warp: the pruned half stencil of a fluid cell
    // (~125 at rho 0.84) plus 32 padding, with room for a Poisson spread of
    // the raw half stencil m = 14 n_cell (4 sqrt(m) + 32), and at least the
    // home forces' transpose (kN3Home * 32), which reuses the same space.
    const double mean = c->ncell > 0 ? (double)c->p.n / (double)c->ncell : 0.0;
    const double m = kN3Half * mean;
    int cap = (int)(m + 4.0 * sqrt(m)) + 64;
    cap = cap < kN3Home * 32 ? kN3Home * 32 : cap;   // S also holds the home forces' transpose
    cap = (cap + 31) & ~31;
    const int max_cap = ((227 * 1024 - 2 * (kN3Threads / 32) * 8) / (4 * (kN3Threads / 32)) -
                         kN3FixedWords) / 4 & ~31;
    if (cap > max_cap) cap = max_cap;
    c->n3cap = cap;   // float4 slots
    c->n3_smem = (kN3Threads / 32) * n3_slice_words(cap) * (int)sizeof(float);
    int minblk = 1 << 30;
    for (int mode = 0; mode < 3; mode++)
        for (int en = 0; en < 2; en++) {
            void *kern = n3_kernel(mode, en != 0);
            cudaError_t e = raise_dyn_smem(kern, c->n3_smem);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kN3Threads, c->n3_smem);
            if (e != cudaSuccess) return e;
            if (en == 0 && nb < minblk) minblk = nb;   // the energy kernels get the same grid
        }
    if (minblk < 1) minblk = 1;
    int64_t need = (c->ncell + kN3Threads / 32 - 1) / (kN3Threads / 32);
    int64_t grid = (int64_t)minblk * c->nsm;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    c->n3_grid = (int)grid;
    return cudaSuccess;
}

cudaError_t launch_force_n3(lj_ctx *c, void *f, bool energy)
{
    if (c->p.n == 0) return cudaSuccess;
    WarpParams k = warp_params_of(c);
    k.cap = c->n3cap;
    k.inv_nc = c->inv_nc_f;
    const float4 *pos = (const float4 *)c->pos;
    const int32_t *start = c->start;
    double *partial = c->partial;
    void *args[] = {&k, (void *)&pos, (void *)&start, &f, &partial};
    if (c->timing && c->ev_used + 2 <= c->nev) cudaEventRecord(c->ev[c->ev_used], c->stream);
    // f must start at zero: zeroed here, unless the step zeroed it already
    // on its side stream
    cudaError_t e = cudaSuccess;
    if (!c->f_prezeroed) e = cudaMemsetAsync(f, 0, (size_t)c->p.n * sizeof(float4), c->stream);
    c->f_prezeroed = 0;
    if (e == cudaSuccess)
        e = cudaLaunchKernel(n3_kernel(c->p.shift_mode, energy), dim3(c->n3_grid), dim3(kN3Threads), args, c->n3_smem,
                             c->stream);
    if (c->timing && c->ev_used + 2 <= c->nev) {
        cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
        c->ev_used += 2;
    }
    c->npartial = c->n3_grid;
    c->kernel_launches++;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
