// lj_forces_static: the forces of lj_forces for callers that cannot
// allocate device memory (a fixed memory budget, another runtime's pool,
// code paths where cudaMalloc is not allowed at call time).  The paper has
// no counterpart; it is an allocation-free variant of lj_forces.
//
// All scratch (cell arrays, sorted positions, scan sums) lives in one
// file-scope device array of fixed size.  Host code cannot use the array's
// name as a device address, so every call looks the address up with
// cudaGetSymbolAddress for the current device (a host-side lookup, no
// stream work).  The address is not cached: after a cudaDeviceReset the
// library's device code is loaded again and the array can move, and a kept
// address would then point at freed memory.  The first call on a device
// (and the first after a reset) loads the device code.  The same launchers
// as lj_forces run on a context built on the host stack whose pointers
// point into the array.  No cudaMalloc, cudaFree or allocating library
// routine is called.
#include <string.h>

#include "lj_internal.cuh"

namespace {

constexpr int64_t kMaxN = LJ_STATIC_MAX_N;
constexpr int64_t kMaxCells = LJ_STATIC_MAX_CELLS;
constexpr int kMaxNc = 32;               // 32^3 == kMaxCells
constexpr int64_t kMaxPartials = 4096;    // energy partials are not written here

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Byte offsets of the regions of the static buffer.
constexpr size_t kOffCellOf = 0;
constexpr size_t kOffRank = kOffCellOf + align256(4 * kMaxN);
constexpr size_t kOffPerm = kOffRank + align256(4 * kMaxN);
constexpr size_t kOffPos = kOffPerm + align256(4 * kMaxN);
constexpr size_t kOffCount = kOffPos + align256(32 * kMaxN);          // double4 in FP64 mode
constexpr size_t kOffStart = kOffCount + align256(4 * (kMaxCells + 1));
constexpr size_t kOffCentre = kOffStart + align256(4 * (kMaxCells + 2));
constexpr size_t kOffTiles = kOffCentre + align256(8 * kMaxNc);
constexpr size_t kOffPartial = kOffTiles + align256(4 * ((kMaxCells + 1 + kScanTile - 1) / kScanTile));
constexpr size_t kOffScalars = kOffPartial + align256(16 * kMaxPartials);
constexpr size_t kOffErr = kOffScalars + align256(4 * sizeof(double));
constexpr size_t kScratchBytes = kOffErr + 256;

static __device__ __align__(256) unsigned char g_lj_static_scratch[kScratchBytes];

__global__ void k_static_centres(double *centre, int nc, double cw)
{
    const int k = threadIdx.x;
    if (k < nc) centre[k] = ((double)k + 0.5) * cw;
}

int map_err(cudaError_t e) { return e == cudaErrorMemoryAllocation ? LJ_ENOMEM : LJ_ECUDA; }

int check_ptr(const void *ptr, size_t align)
{
    if (!ptr || ((uintptr_t)ptr) % align != 0) return LJ_EINVAL;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return LJ_EINVAL;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? LJ_OK : LJ_EINVAL;
}

// Device address of the static buffer on the current device, looked up on
// every call (see the file header for why it is not kept).
int scratch_for_current_device(unsigned char **out)
{
    void *addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_lj_static_scratch);
    if (e != cudaSuccess) return map_err(e);
    if (!addr) return LJ_ECUDA;
    *out = (unsigned char *)addr;
    return LJ_OK;
}

}  // namespace

extern "C" int lj_forces_static(const lj_params *p, const double *x, void *f, void *stream)
{
    int32_t nc = 0;
    int r = lj_grid(p, &nc);
    if (r != LJ_OK) return r;
    // Only the warp kernels: the run kernels' bounded waits report a timeout
    // through the error word, which no caller of this entry point can read.
    if (p->flags != 0) return LJ_EINVAL;
    const int64_t ncell = (int64_t)nc * nc * nc;
    if (p->n > kMaxN || ncell > kMaxCells) return LJ_EOVERFLOW;
    if (p->n > 0) {
        if ((r = check_ptr(x, 8)) != LJ_OK) return r;
        if ((r = check_ptr(f, 16)) != LJ_OK) return r;
    }
    unsigned char *base = nullptr;
    if ((r = scratch_for_current_device(&base)) != LJ_OK) return r;

    lj_ctx c;
    memset(&c, 0, sizeof(c));
    c.p = *p;
    if (c.p.cell_subdiv == 0) c.p.cell_subdiv = 1;
    c.nc = nc;
    c.ncell = ncell;
    c.inv_cw = (double)nc / p->box;
    c.cw = p->box / (double)nc;
    c.wrap_hi = p->box * (1.0 - ldexp(1.0, -50));
    c.wrap_lo = p->box * ldexp(1.0, -50);
    c.stream = (cudaStream_t)stream;
    c.use_tma = 1;
    c.use_run_kernel = 0;
    cudaError_t e = cudaGetDevice(&c.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, c.device);
    if (e != cudaSuccess) return map_err(e);
    c.cell_of = (int32_t *)(base + kOffCellOf);
    c.rank = (int32_t *)(base + kOffRank);
    c.perm = (int32_t *)(base + kOffPerm);
    c.pos = (void *)(base + kOffPos);
    c.count = (int32_t *)(base + kOffCount);
    c.start = (int32_t *)(base + kOffStart);
    c.centre = (double *)(base + kOffCentre);
    c.tile_sum = (int32_t *)(base + kOffTiles);
    c.ntiles = (int)((ncell + 1 + kScanTile - 1) / kScanTile);
    c.partial = (double *)(base + kOffPartial);
    c.scalars = (double *)(base + kOffScalars);
    c.err = (int32_t *)(base + kOffErr);

    if ((e = force_configure(&c)) != cudaSuccess) return map_err(e);
    e = p->precision == LJ_PREC_MIXED ? warp_force_configure(&c) : w64_force_configure(&c);
    if (e != cudaSuccess) return map_err(e);
    if (c.force_grid > kMaxPartials || c.wforce_grid > kMaxPartials) return LJ_EOVERFLOW;
    if (p->n == 0) return LJ_OK;

    // The buffer keeps the previous call's contents: clear what must start at 0.
    if ((e = cudaMemsetAsync(c.count, 0, (size_t)(ncell + 1) * sizeof(int32_t), c.stream)) != cudaSuccess)
        return map_err(e);
    if ((e = cudaMemsetAsync(c.err, 0, sizeof(int32_t), c.stream)) != cudaSuccess) return map_err(e);
    k_static_centres<<<1, kMaxNc, 0, c.stream>>>(c.centre, nc, c.cw);
    if ((e = cudaGetLastError()) != cudaSuccess) return map_err(e);
    if ((e = launch_bin_count(&c, x)) != cudaSuccess) return map_err(e);
    if ((e = launch_scan(&c)) != cudaSuccess) return map_err(e);
    if ((e = launch_scatter(&c, x, true)) != cudaSuccess) return map_err(e);
    if ((e = launch_force(&c, f, false)) != cudaSuccess) return map_err(e);
    return LJ_OK;
}
