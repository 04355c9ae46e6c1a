// The paper's own cell data structure (Section 3.1): every cell owns a fixed
// array of kAopCap placeholders (the paper's capacity n = 32), particles are
// copied into it, and empty places act as virtual particles whose
// interactions are computed like the real ones.  One warp per home cell,
// lane l = placeholder l (the paper's one thread per placeholder); for each
// of the 27 stencil cells the warp loads that cell's 32 placeholders (one
// coalesced 512-byte read), shifts them into the home-cell frame and every
// lane runs over all 32 of them by warp shuffles.  The work is therefore
// 27 x 32 pair evaluations per placeholder whatever the density: run time
// follows the number of cells, the density dependence the paper reports.
// Kept as the comparison point for the CSR layout of the default kernels;
// selected with lj_set_tuning kernel 4 (FP32-mixed, subdivision 1).
#include "lj_force_cell.cuh"

namespace {

constexpr int kAopCap = 32;
constexpr int kAopThreads = 256;

// aop[c * cap + r] = pos[start[c] + r] for the r-th particle of cell c;
// particles past the capacity latch LJ_ERRBIT_OVERFLOW (the layout cannot
// hold them: the paper's density limit).
__global__ void k_aop_pack(const float4 *__restrict__ pos, const int32_t *__restrict__ start,
                           const int32_t *__restrict__ cell_of, const int32_t *__restrict__ rank, int n,
                           int64_t ncell, float4 *__restrict__ aop, int32_t *__restrict__ err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell_of[i];
    if ((int64_t)c >= ncell) return;   // the extra cell of non-finite particles
    const int r = rank[i];
    if (r < kAopCap) {
        aop[(int64_t)c * kAopCap + r] = pos[start[c] + r];
    } else {
        atomicOr(err, LJ_ERRBIT_OVERFLOW);
    }
}

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kAopThreads) k_force_aop(WarpParams k, const float4 *__restrict__ aop,
                                                           const int32_t *__restrict__ start,
                                                           float4 *__restrict__ fout, double *__restrict__ partial)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nc = k.nc;
    double eacc = 0.0, wacc = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * (kAopThreads / 32);
    for (int64_t c = (int64_t)blockIdx.x * (kAopThreads / 32) + warp; c < k.ncell; c += nwarps) {
        const int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        const int n_home = min(kAopCap, start[c + 1] - start[c]);
        float4 p = make_float4(kFar, kFar, kFar, 0.f);
        if (lane < n_home) p = __ldg(aop + c * kAopCap + lane);
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f, w = 0.f;
        for (int kk = 0; kk < 27; kk++) {
            const int dx = kk % 3 - 1, dy = (kk / 3) % 3 - 1, dz = kk / 9 - 1;
            int ux = cx + dx, uy = cy + dy, uz = cz + dz;
            ux += ux < 0 ? nc : 0;
            ux -= ux >= nc ? nc : 0;
            uy += uy < 0 ? nc : 0;
            uy -= uy >= nc ? nc : 0;
            uz += uz < 0 ? nc : 0;
            uz -= uz >= nc ? nc : 0;
            const int64_t cn = ux + (int64_t)nc * (uy + (int64_t)nc * uz);
            const int nk = min(kAopCap, start[cn + 1] - start[cn]);
            // placeholder `lane` of the neighbour cell in the home frame;
            // virtual placeholders sit far away
            float qx = kFar, qy = kFar, qz = kFar;
            if (lane < nk) {
                const float4 q = __ldg(aop + cn * kAopCap + lane);
                qx = q.x + (float)dx * k.cw;
                qy = q.y + (float)dy * k.cw;
                qz = q.z + (float)dz * k.cw;
            }
#pragma unroll 8
            for (int j = 0; j < kAopCap; j++) {
                const float ax = __shfl_sync(0xffffffffu, qx, j);
                const float ay = __shfl_sync(0xffffffffu, qy, j);
                const float az = __shfl_sync(0xffffffffu, qz, j);
                pair1<MODE, ENERGY>(p.x - ax, p.y - ay, p.z - az, k, fx, fy, fz, e, w);
            }
        }
        if (lane < n_home) {
            const int idx = __float_as_int(p.w);
            if ((unsigned)idx < (unsigned)k.n) {
                fout[idx] = make_float4(fx, fy, fz, ENERGY ? 0.5f * e : 0.0f);
                if constexpr (ENERGY) {
                    eacc += 0.5 * (double)e;
                    wacc += 0.5 * (double)w;
                }
            }
        }
    }
    if constexpr (ENERGY) {
        __shared__ double red[2 * (kAopThreads / 32)];
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
            for (int q = 0; q < kAopThreads / 32; q++) {
                es += red[2 * q];
                ws += red[2 * q + 1];
            }
            partial[2 * blockIdx.x] = es;
            partial[2 * blockIdx.x + 1] = ws;
        }
    }
}

void *aop_kernel(int mode, bool energy)
{
    switch (mode * 2 + (energy ? 1 : 0)) {
        case 0: return (void *)k_force_aop<0, false>;
        case 1: return (void *)k_force_aop<0, true>;
        case 2: return (void *)k_force_aop<1, false>;
        case 3: return (void *)k_force_aop<1, true>;
        case 4: return (void *)k_force_aop<2, false>;
        default: return (void *)k_force_aop<2, true>;
    }
}

}  // namespace

cudaError_t launch_force_aop(lj_ctx *c, void *f, bool energy)
{
    const int n = (int)c->p.n;
    if (n == 0) return cudaSuccess;
    const size_t need = (size_t)c->ncell * kAopCap * sizeof(float4);
    if (need > c->aop_bytes) {
        cudaFree(c->aop);
        c->aop = nullptr;
        c->aop_bytes = 0;
        cudaError_t e = cudaMalloc(&c->aop, need);
        if (e != cudaSuccess) return e;
        c->aop_bytes = need;
    }
    float4 *aop = (float4 *)c->aop;
    k_aop_pack<<<(n + 255) / 256, 256, 0, c->stream>>>((const float4 *)c->pos, c->start, c->cell_of, c->rank, n,
                                                         c->ncell, aop, c->err);
    int nb = 0;
    void *kern = aop_kernel(c->p.shift_mode, energy);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kAopThreads, 0);
    if (e != cudaSuccess) return e;
    int64_t need_blocks = (c->ncell + kAopThreads / 32 - 1) / (kAopThreads / 32);
    int64_t grid = (int64_t)(nb > 0 ? nb : 1) * c->nsm;
    if (grid > need_blocks) grid = need_blocks;
    if (grid > c->npartial_cap) grid = c->npartial_cap;
    if (grid < 1) grid = 1;
    c->npartial = (int)grid;
    WarpParams k = warp_params_of(c);
    const int32_t *start = c->start;
    double *partial = c->partial;
    void *args[] = {&k, (void *)&aop, (void *)&start, &f, &partial};
    if (c->timing && c->ev_used + 2 <= c->nev) cudaEventRecord(c->ev[c->ev_used], c->stream);
    e = cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kAopThreads), args, 0, c->stream);
    if (c->timing && c->ev_used + 2 <= c->nev) {
        cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
        c->ev_used += 2;
    }
    c->kernel_launches += 2;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
