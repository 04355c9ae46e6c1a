// C ABI of liblj.so (declared in include/lj.h): context management,
// argument checking and the sequencing of the kernels of one MD step.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lj_internal.cuh"

// Device (or managed) memory check for caller arrays.
int check_dev_ptr(const void *ptr, size_t align)
{
    if (!ptr) return LJ_EINVAL;
    if (((uintptr_t)ptr) % align != 0) return LJ_EINVAL;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LJ_EINVAL;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return LJ_EINVAL;
    return LJ_OK;
}

namespace {

constexpr int kEventPool = 2 * 8192;

int map_cuda(cudaError_t e)
{
    return e == cudaErrorMemoryAllocation ? LJ_ENOMEM : LJ_ECUDA;
}

#define LJ_CK(call)                                     \
    do {                                                \
        cudaError_t lj_ck_e_ = (call);                  \
        if (lj_ck_e_ != cudaSuccess) return map_cuda(lj_ck_e_); \
    } while (0)

// Smallest double t >= 0 with trunc(t * s) >= k (IEEE double multiply, the
// same operation the kernels use): the lower edge of cell k.
double cell_threshold(int k, double s)
{
    double t = (double)k / s;
    while (t > 0.0 && nextafter(t, 0.0) * s >= (double)k) t = nextafter(t, 0.0);
    while (!(t * s >= (double)k)) t = nextafter(t, INFINITY);
    return t;
}

int validate(const lj_params *p, int *nc_out)
{
    if (!p) return LJ_EINVAL;
    if (p->n < 0) return LJ_EINVAL;
    if (p->n >= INT32_MAX) return LJ_EOVERFLOW;
    if (!(p->box > 0.0) || !isfinite(p->box)) return LJ_EINVAL;
    if (!(p->sigma > 0.0) || !isfinite(p->sigma)) return LJ_EINVAL;
    if (!(p->rc > 0.0) || !isfinite(p->rc)) return LJ_EINVAL;
    if (!(p->mass > 0.0) || !isfinite(p->mass)) return LJ_EINVAL;
    if (!(p->eps >= 0.0) || !isfinite(p->eps)) return LJ_EINVAL;
    if (!isfinite(p->dt)) return LJ_EINVAL;
    if (p->shift_mode < LJ_SHIFT_NONE || p->shift_mode > LJ_SHIFT_FORCE) return LJ_EINVAL;
    if (p->precision != LJ_PREC_MIXED && p->precision != LJ_PREC_FP64) return LJ_EINVAL;
    if (p->cell_subdiv < 0 || p->cell_subdiv > 2) return LJ_EINVAL;
    // subdivision 2 runs on the warp kernel only (FP32-mixed, no run-kernel flag)
    if (p->cell_subdiv == 2 && (p->precision != LJ_PREC_MIXED || p->flags != 0)) return LJ_EINVAL;
    if ((p->flags & ~(LJ_FLAG_RUN_STAGED | LJ_FLAG_RUN_DIRECT)) != 0) return LJ_EINVAL;
    if ((p->flags & LJ_FLAG_RUN_STAGED) && (p->flags & LJ_FLAG_RUN_DIRECT)) return LJ_EINVAL;
    const int k = p->cell_subdiv == 2 ? 2 : 1;
    double q = floor(((double)k * p->box) / p->rc);
    if (!(q >= 2.0 * k + 1.0)) return LJ_EBOX;
    if (q > 1290.0) return LJ_EOVERFLOW;   // nc^3 + 1 must fit in int32
    if (nc_out) *nc_out = (int)q;
    return LJ_OK;
}

size_t force_vsize(const lj_ctx *c)
{
    return c->p.precision == LJ_PREC_FP64 ? sizeof(double4_16a) : sizeof(float4);
}

void free_ctx(lj_ctx *c)
{
    if (!c) return;
    cudaFree(c->cell_of);
    cudaFree(c->rank);
    cudaFree(c->count);
    cudaFree(c->start);
    cudaFree(c->perm);
    cudaFree(c->pos);
    cudaFree(c->tile_sum);
    cudaFree(c->scan_status);
    cudaFree(c->scan_ctl);
    cudaFree(c->centre);
    cudaFree(c->work);
    cudaFree(c->thb);
    cudaFree(c->partial);
    cudaFree(c->ekin_partial);
    cudaFree(c->scalars);
    cudaFree(c->err);
    cudaFree(c->xs);
    cudaFree(c->vs);
    cudaFree(c->fs);
    cudaFree(c->g4);
    cudaFree(c->n2_scratch);
    cudaFree(c->f_sorted);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->zero_stream) cudaStreamDestroy(c->zero_stream);
    if (c->ev_zfork) cudaEventDestroy(c->ev_zfork);
    if (c->ev_zjoin) cudaEventDestroy(c->ev_zjoin);
    if (c->ev_xfinal) cudaEventDestroy(c->ev_xfinal);
    if (c->ev_entry) cudaEventDestroy(c->ev_entry);
    for (int k = 0; k < 4; k++)
        if (c->ev_chunk[k]) cudaEventDestroy(c->ev_chunk[k]);
    cudaFree(c->pos_alt);
    cudaFree(c->perm_alt);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    cudaFree(c->aop);
    cudaFree(c->r48_state);
    cudaFree(c->disp);
    cudaFree(c->skin_flags);
    cudaFree(c->skin_counts);
    if (c->host_scalars) cudaFreeHost(c->host_scalars);
    if (c->host_err) cudaFreeHost(c->host_err);
    if (c->pers) lj_batch_destroy(c->pers);
    if (c->ev) {
        for (int i = 0; i < c->nev; i++) cudaEventDestroy(c->ev[i]);
        free(c->ev);
    }
    free(c);
}

// Synchronize, read and clear latched kernel errors.
int sync_and_check(lj_ctx *c)
{
    LJ_CK(cudaStreamSynchronize(c->stream));
    LJ_CK(cudaMemcpyAsync(c->host_err, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    LJ_CK(cudaStreamSynchronize(c->stream));
    int32_t bits = *c->host_err;
    if (bits) {
        LJ_CK(cudaMemsetAsync(c->err, 0, sizeof(int32_t), c->stream));
        LJ_CK(cudaStreamSynchronize(c->stream));
    }
    // steps taken by the persistent one-replica batch latch their own flags
    const int rp = c->pers ? lj_batch_check(c->pers) : LJ_OK;
    if (bits & LJ_ERRBIT_NONFINITE) return LJ_ENONFINITE;
    if (bits & LJ_ERRBIT_TIMEOUT) return LJ_ETIMEOUT;
    if (bits & LJ_ERRBIT_SCAN) return LJ_ECUDA;
    if (bits & LJ_ERRBIT_OVERFLOW) return LJ_EOVERFLOW;
    return rp;
}

// Restart the skin bookkeeping after a full rebuild (the ungated count
// kernel has cleared the displacements).
int skin_restart(lj_ctx *c)
{
    if (c->skin > 0.0) {
        LJ_CK(cudaMemsetAsync(c->skin_flags, 0, sizeof(int32_t), c->stream));
        LJ_CK(cudaMemsetAsync(c->skin_flags + 2, 0, sizeof(int32_t), c->stream));
        c->skin_dirty = 0;
    }
    return LJ_OK;
}

int do_bin(lj_ctx *c, const double *x, bool wrap_in_scatter)
{
    LJ_CK(launch_bin_count(c, x));
    LJ_CK(launch_scan(c));
    LJ_CK(launch_scatter(c, x, wrap_in_scatter));
    return skin_restart(c);
}

// Cell lists with a skin: the cells are rebuilt only when the device-side
// decision (k_skin_decide) asks for it; otherwise the sorted positions are
// refreshed from x in the old cell order (the scatter with the old ranks).
bool fused_mode(const lj_ctx *c) { return !c->use_run_kernel && c->fuse_update && c->skin <= 0.0; }

// The launches of step s of an nsteps-call (see do_steps).  Steps other
// than the first and the last issue the same launches, which is what the
// graph replay captures.
int one_step(lj_ctx *c, double *x, double *v, void *f, int s, int nsteps, cudaEvent_t x_final = nullptr)
{
    if (c->skin > 0.0) {
        // cell lists with a skin: the cells are rebuilt only when the
        // device-side decision (k_skin_decide) asks for it; otherwise the
        // sorted positions are refreshed from x in the old cell order
        LJ_CK(launch_kick_drift_skin(c, x, v, f, s == 0 ? 1 : 2));
        const bool gated = !c->skin_dirty;
        LJ_CK(launch_bin_count(c, x, gated));
        LJ_CK(launch_scan(c, gated));
        LJ_CK(launch_scatter(c, x, false));
        if (x_final) LJ_CK(cudaEventRecord(x_final, c->stream));
        if (!gated) {
            int r = skin_restart(c);
            if (r) return r;
        }
        LJ_CK(launch_force(c, f, false));
        return LJ_OK;
    }
    if (fused_mode(c)) {
        // FP32-mixed warp kernel with the update fused: every force launch
        // applies the next step's update to the particles it has just
        // finished (the last one only the closing half kick)
        LJ_CK(launch_scan(c));
        LJ_CK(launch_scatter(c, x, false));
        LJ_CK(launch_force_warp_fused(c, f, x, v, s == nsteps - 1));
        return LJ_OK;
    }
    if (s == 0 && c->kdb_done) {
        c->kdb_done = 0;   // lj_step_host ran step 0's update chunk by chunk
    } else {
        LJ_CK(launch_kick_drift_bin(c, x, v, f, s == 0 ? 1 : 2));
    }
    // the update has read f: the pair-once kernel's zeroing of f forks off
    // here and overlaps the scan (latency-bound) and the scatter
    const bool zfork = c->zero_stream && uses_force_n3(c);
    if (zfork) {
        LJ_CK(cudaEventRecord(c->ev_zfork, c->stream));
        LJ_CK(cudaStreamWaitEvent(c->zero_stream, c->ev_zfork, 0));
        LJ_CK(cudaMemsetAsync(f, 0, (size_t)c->p.n * force_vsize(c), c->zero_stream));
        LJ_CK(cudaEventRecord(c->ev_zjoin, c->zero_stream));
    }
    LJ_CK(launch_scan(c));
    LJ_CK(launch_scatter(c, x, false));
    if (x_final) LJ_CK(cudaEventRecord(x_final, c->stream));   // x holds its final value
    if (zfork) {
        LJ_CK(cudaStreamWaitEvent(c->stream, c->ev_zjoin, 0));
        c->f_prezeroed = 1;
    }
    const cudaError_t e = launch_force(c, f, false);
    c->f_prezeroed = 0;
    LJ_CK(e);
    return LJ_OK;
}

// The side stream and events of the zeroing fork (outside any capture).
int ensure_zero_stream(lj_ctx *c)
{
    if (c->zero_stream) return LJ_OK;
    LJ_CK(cudaEventCreateWithFlags(&c->ev_zfork, cudaEventDisableTiming));
    LJ_CK(cudaEventCreateWithFlags(&c->ev_zjoin, cudaEventDisableTiming));
    LJ_CK(cudaStreamCreateWithFlags(&c->zero_stream, cudaStreamNonBlocking));
    return LJ_OK;
}

// Capture the launches of one middle step for (x, v, f) into c->gexec.
int capture_middle_step(lj_ctx *c, double *x, double *v, void *f)
{
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    cudaStream_t cs = c->stream;
    bool own = false;
    if (!cs) {   // the legacy stream cannot be captured
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return LJ_ECUDA;
        own = true;
    }
    cudaGraph_t g = nullptr;
    const int64_t k0 = c->kernel_launches;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int r = LJ_OK;
    if (e == cudaSuccess) {
        cudaStream_t keep = c->stream;
        c->stream = cs;
        r = one_step(c, x, v, f, 1, 3);
        c->stream = keep;
        e = cudaStreamEndCapture(cs, &g);
    }
    c->glaunches = c->kernel_launches - k0;
    c->kernel_launches = k0;
    if (e == cudaSuccess && r == LJ_OK) e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (own) cudaStreamDestroy(cs);
    if (e != cudaSuccess || r != LJ_OK || !c->gexec) {
        cudaGetLastError();
        c->gexec = nullptr;
        return r != LJ_OK ? r : LJ_ECUDA;
    }
    c->gx = x;
    c->gv = v;
    c->gf = f;
    c->ggen = c->gen;
    return LJ_OK;
}

// nsteps velocity-Verlet steps: [fused: the first kick + drift + bin],
// the steps, [unfused: the closing half kick].  With graph replay on, the
// middle steps are replays of one captured step.
// x_final (optional): recorded once x holds its final value (after the
// last step's scatter; unfused updates only), so that its copy can overlap
// the last force evaluation.
// Tuning kernel 6: the steps run as one cooperative persistent launch each
// (the batched-ensemble kernel with one replica), which removes the gaps
// between the five kernels of a step; for small systems.  Cells with a skin
// and the deterministic in-cell order keep the regular path.
bool persistent_mode(const lj_ctx *c)
{
    return c->use_pers && c->skin <= 0.0 && !c->deterministic && c->p.precision == LJ_PREC_MIXED &&
           c->p.cell_subdiv == 1 && c->p.n > 0;
}

int persistent_steps(lj_ctx *c, double *x, double *v, void *f, int nsteps, cudaEvent_t x_final)
{
    if (!c->pers) {
        const int64_t n = c->p.n;
        const double box = c->p.box;
        int r = lj_batch_create(&c->pers, 1, &n, &box, &c->p, (void *)c->stream);
        if (r != LJ_OK) {
            c->pers = nullptr;
            return r;
        }
        c->pers_gen = c->gen - 1;
    }
    if (c->pers_gen != c->gen) {   // cells per pull and lane-group width of the tuning
        const int r = lj_batch_set_tuning(c->pers, c->grab > 0 ? c->grab : 1, 1, c->gw);
        if (r != LJ_OK) return r;
        c->pers_gen = c->gen;
    }
    int64_t l0 = 0, l1 = 0;
    lj_batch_launches(c->pers, &l0, nullptr);
    const int r = lj_batch_step(c->pers, x, v, f, nsteps);
    lj_batch_launches(c->pers, &l1, nullptr);
    c->kernel_launches += l1 - l0;
    if (r != LJ_OK) return r;
    if (x_final) LJ_CK(cudaEventRecord(x_final, c->stream));
    return LJ_OK;
}

constexpr int kHostChunks = 4;   // parts of lj_step_host's copies in

int do_steps(lj_ctx *c, double *x, double *v, void *f, int nsteps, cudaEvent_t x_final = nullptr)
{
    if (nsteps <= 0) return LJ_OK;
    if (persistent_mode(c)) return persistent_steps(c, x, v, f, nsteps, x_final);
    if (fused_mode(c)) LJ_CK(launch_kick_drift_bin(c, x, v, f, 1));
    if (c->skin <= 0.0 && !fused_mode(c) && uses_force_n3(c)) {
        int r = ensure_zero_stream(c);
        if (r) return r;
    }
    const bool graph = c->use_graph && !c->timing && nsteps >= 3;
    for (int s = 0; s < nsteps; s++) {
        // after step 0 (which does any lazy set-up outside the capture and
        // settles a pending skin rebuild) the middle steps are graph replays
        if (graph && s > 0 && s < nsteps - 1 && !c->skin_dirty) {
            if (!c->gexec || c->gx != x || c->gv != v || c->gf != f || c->ggen != c->gen) {
                int r = capture_middle_step(c, x, v, f);
                if (r) return r;
            }
            LJ_CK(cudaGraphLaunch(c->gexec, c->stream));
            c->kernel_launches += c->glaunches;
        } else {
            int r = one_step(c, x, v, f, s, nsteps, s == nsteps - 1 && !fused_mode(c) ? x_final : nullptr);
            if (r) return r;
        }
    }
    if (!fused_mode(c)) LJ_CK(launch_kick(c, v, f));
    if (x_final && fused_mode(c)) LJ_CK(cudaEventRecord(x_final, c->stream));
    return LJ_OK;
}

// The adjoint's buffers: the cell-ordered cotangents and, for the
// pair-once FP32-mixed VJP, its float4 accumulator (in f_sorted, which
// FP32-mixed contexts do not otherwise use).
int ensure_vjp_buffers(lj_ctx *c)
{
    if (!c->g4) LJ_CK(cudaMalloc(&c->g4, (size_t)c->p.n * force_vsize(c)));
    if (c->p.precision == LJ_PREC_MIXED && uses_vjp_n3(c) && !c->f_sorted)
        LJ_CK(cudaMalloc(&c->f_sorted, (size_t)c->p.n * sizeof(float4)));
    return LJ_OK;
}

int ensure_staging(lj_ctx *c)
{
    size_t n1 = (size_t)(c->p.n > 0 ? c->p.n : 1);
    if (!c->xs) LJ_CK(cudaMalloc(&c->xs, 3 * n1 * sizeof(double)));
    if (!c->vs) LJ_CK(cudaMalloc(&c->vs, 3 * n1 * sizeof(double)));
    if (!c->fs) LJ_CK(cudaMalloc(&c->fs, n1 * force_vsize(c)));
    return LJ_OK;
}

}  // namespace

extern "C" int lj_version(void) { return LJ_ABI_VERSION; }

extern "C" const char *lj_strerror(int code)
{
    switch (code) {
        case LJ_OK: return "ok";
        case LJ_EINVAL: return "invalid argument";
        case LJ_EBOX: return "box too small for the cell stencil (need at least 3 cells per side)";
        case LJ_ECUDA: return "CUDA runtime error";
        case LJ_ENONFINITE: return "non-finite particle coordinate";
        case LJ_ETIMEOUT: return "bounded device wait timed out";
        case LJ_EOVERFLOW: return "size exceeds 32-bit indexing";
        case LJ_ENOMEM: return "out of memory";
        default: return "unknown lj status";
    }
}

extern "C" int lj_grid(const lj_params *p, int32_t *nc_out)
{
    int nc = 0;
    int r = validate(p, &nc);
    if (r != LJ_OK) return r;
    if (nc_out) *nc_out = nc;
    return LJ_OK;
}

// (Re)build the cell grid of a context for n cells per axis: cell geometry,
// count / start / scan arrays, cell-centre and threshold tables, kernel
// configurations and the energy partials.  Frees what an earlier grid held.
int setup_grid(lj_ctx *c, int nc)
{
    cudaFree(c->count);
    cudaFree(c->start);
    cudaFree(c->centre);
    cudaFree(c->thb);
    cudaFree(c->tile_sum);
    cudaFree(c->scan_status);
    cudaFree(c->scan_ctl);
    cudaFree(c->partial);
    c->count = c->start = c->tile_sum = nullptr;
    c->scan_status = nullptr;
    c->scan_ctl = nullptr;
    c->centre = nullptr;
    c->thb = nullptr;
    c->partial = nullptr;
    c->nc = nc;
    c->ncell = (int64_t)nc * nc * nc;
    c->inv_cw = (double)nc / c->p.box;
    c->inv_nc_f = c->ncell + 1 < (1 << 24) ? 1.0f / (float)nc : 0.0f;
    c->cw = c->p.box / (double)nc;
#define LJ_GRID_CK(call)             \
    do {                             \
        cudaError_t e_ = (call);     \
        if (e_ != cudaSuccess) return map_cuda(e_); \
    } while (0)
    LJ_GRID_CK(cudaMalloc(&c->count, (size_t)(c->ncell + 1) * sizeof(int32_t)));
    LJ_GRID_CK(cudaMalloc(&c->start, (size_t)(c->ncell + 2) * sizeof(int32_t)));
    {
        double *h = (double *)malloc(sizeof(double) * (size_t)nc);
        if (!h) return LJ_ENOMEM;
        for (int k = 0; k < nc; k++) h[k] = ((double)k + 0.5) * c->cw;
        cudaError_t e = cudaMalloc(&c->centre, sizeof(double) * (size_t)nc);
        if (e == cudaSuccess) e = cudaMemcpy(c->centre, h, sizeof(double) * (size_t)nc, cudaMemcpyHostToDevice);
        free(h);
        long long *tb = (long long *)malloc(sizeof(long long) * (size_t)(nc + 1));
        if (!tb && e == cudaSuccess) e = cudaErrorMemoryAllocation;
        if (tb) {
            tb[0] = 0;
            for (int k = 1; k < nc; k++) {
                double t = cell_threshold(k, c->inv_cw);
                memcpy(&tb[k], &t, sizeof(double));
            }
            tb[nc] = INT64_MAX;
            if (e == cudaSuccess) e = cudaMalloc(&c->thb, sizeof(long long) * (size_t)(nc + 1));
            if (e == cudaSuccess)
                e = cudaMemcpy(c->thb, tb, sizeof(long long) * (size_t)(nc + 1), cudaMemcpyHostToDevice);
            free(tb);
        }
        if (e != cudaSuccess) return map_cuda(e);
    }
    c->ntiles = (int)((c->ncell + 1 + kScanTile - 1) / kScanTile);
    LJ_GRID_CK(cudaMalloc(&c->tile_sum, (size_t)c->ntiles * sizeof(int32_t)));
    LJ_GRID_CK(cudaMalloc(&c->scan_status, (size_t)c->ntiles * sizeof(unsigned long long)));
    LJ_GRID_CK(cudaMalloc(&c->scan_ctl, 4 * sizeof(unsigned)));
    LJ_GRID_CK(cudaMemsetAsync(c->scan_status, 0, (size_t)c->ntiles * sizeof(unsigned long long), c->stream));
    LJ_GRID_CK(cudaMemsetAsync(c->scan_ctl, 0, 4 * sizeof(unsigned), c->stream));
    LJ_GRID_CK(force_configure(c));
    LJ_GRID_CK(c->p.precision == LJ_PREC_MIXED ? warp_force_configure(c) : w64_force_configure(c));
    c->pipe_grid = 0;
    if (c->p.precision == LJ_PREC_MIXED && c->p.cell_subdiv != 2) LJ_GRID_CK(pipe_force_configure(c));
    if (c->p.precision == LJ_PREC_MIXED && c->p.cell_subdiv != 2) LJ_GRID_CK(n3_force_configure(c));
    if (c->p.precision == LJ_PREC_FP64 && !c->f_sorted && c->p.n > 0)   // the FP64 pair-once sums, in cell order
        LJ_GRID_CK(cudaMalloc(&c->f_sorted, (size_t)c->p.n * 4 * sizeof(double)));
    {
        int np = c->force_grid > c->wforce_grid ? c->force_grid : c->wforce_grid;
        if (c->n3_grid > np) np = c->n3_grid;
        if (np < 32 * c->nsm) np = 32 * c->nsm;   // room for the adjoint kernel's grid
        c->npartial_cap = np;
        LJ_GRID_CK(cudaMalloc(&c->partial, 2 * (size_t)np * sizeof(double)));
    }
    LJ_GRID_CK(cudaMemsetAsync(c->count, 0, (size_t)(c->ncell + 1) * sizeof(int32_t), c->stream));
    LJ_GRID_CK(cudaMemsetAsync(c->start, 0, (size_t)(c->ncell + 2) * sizeof(int32_t), c->stream));
#undef LJ_GRID_CK
    return LJ_OK;
}

extern "C" int lj_create(lj_ctx **out, const lj_params *p, void *stream)
{
    if (!out) return LJ_EINVAL;
    *out = nullptr;
    int nc = 0;
    int r = validate(p, &nc);
    if (r != LJ_OK) return r;
    lj_ctx *c = (lj_ctx *)calloc(1, sizeof(lj_ctx));
    if (!c) return LJ_ENOMEM;
    c->p = *p;
    if (c->p.cell_subdiv == 0) c->p.cell_subdiv = 1;
    c->wrap_hi = p->box * (1.0 - ldexp(1.0, -50));
    c->wrap_lo = p->box * ldexp(1.0, -50);
    c->stream = (cudaStream_t)stream;
    // Kernel choice: the warp-per-cell kernels (FP32-mixed, and FP64 with
    // compacted pair lists) by default; the flags force a run kernel.
    c->use_tma = (p->flags & LJ_FLAG_RUN_DIRECT) ? 0 : 1;
    c->use_run_kernel = (p->flags & (LJ_FLAG_RUN_STAGED | LJ_FLAG_RUN_DIRECT)) ? 1 : 0;
    // The update runs as its own coalesced kernel by default: fused into the
    // force kernel (lj_set_tuning kernel 0) it measured slower at N = 4M
    // (1.35 vs 1.20 ms per step) from the scattered x, v accesses.
    c->fuse_update = 0;
    // Forces with cell subdivision 1 take each pair once (Newton's third
    // law, lj_set_tuning kernel 7; FP32-mixed and FP64) unless a flag asks
    // for a run kernel.
    c->n3 = (c->p.cell_subdiv == 1 && !c->use_run_kernel) ? 1 : 0;

#define LJ_CREATE_CK(call)            \
    do {                              \
        cudaError_t e_ = (call);      \
        if (e_ != cudaSuccess) {      \
            free_ctx(c);              \
            return map_cuda(e_);      \
        }                             \
    } while (0)

    LJ_CREATE_CK(cudaGetDevice(&c->device));
    LJ_CREATE_CK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));
    const size_t n1 = (size_t)(p->n > 0 ? p->n : 1);
    LJ_CREATE_CK(cudaMalloc(&c->cell_of, n1 * sizeof(int32_t)));
    LJ_CREATE_CK(cudaMalloc(&c->rank, n1 * sizeof(int32_t)));
    LJ_CREATE_CK(cudaMalloc(&c->perm, n1 * sizeof(int32_t)));
    LJ_CREATE_CK(cudaMalloc(&c->pos, n1 * force_vsize(c)));
    {
        const int gr = setup_grid(c, nc);
        if (gr != LJ_OK) {
            free_ctx(c);
            return gr;
        }
    }
    int64_t eb = (3 * (int64_t)n1 + kReduceThreads - 1) / kReduceThreads;
    c->ekin_grid = (int)(eb < 4 * (int64_t)c->nsm ? eb : 4 * (int64_t)c->nsm);
    LJ_CREATE_CK(cudaMalloc(&c->ekin_partial, (size_t)c->ekin_grid * sizeof(double)));
    LJ_CREATE_CK(cudaMalloc(&c->scalars, 8 * sizeof(double)));
    LJ_CREATE_CK(cudaMalloc(&c->err, sizeof(int32_t)));
    LJ_CREATE_CK(cudaMalloc(&c->work, sizeof(unsigned)));
    LJ_CREATE_CK(cudaMemset(c->work, 0, sizeof(unsigned)));
    c->grab = 4;   // dynamic pulls of 4 cells: measured fastest at 4M (static striding 5% slower)
    LJ_CREATE_CK(cudaMallocHost(&c->host_scalars, 8 * sizeof(double)));
    LJ_CREATE_CK(cudaMallocHost(&c->host_err, sizeof(int32_t)));
    LJ_CREATE_CK(cudaMemsetAsync(c->cell_of, 0, n1 * sizeof(int32_t), c->stream));
    LJ_CREATE_CK(cudaMemsetAsync(c->scalars, 0, 8 * sizeof(double), c->stream));
    LJ_CREATE_CK(cudaMemsetAsync(c->err, 0, sizeof(int32_t), c->stream));
    LJ_CREATE_CK(cudaStreamSynchronize(c->stream));
#undef LJ_CREATE_CK
    *out = c;
    return LJ_OK;
}

extern "C" void lj_destroy(lj_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

extern "C" int lj_bin(lj_ctx *c, const double *x)
{
    if (!c) return LJ_EINVAL;
    if (c->p.n > 0) {
        int r = check_dev_ptr(x, 8);
        if (r) return r;
    }
    return do_bin(c, x, true);
}

extern "C" int lj_get_cells(lj_ctx *c, int32_t *cell_of, int32_t *count, int32_t *start, int32_t *perm)
{
    if (!c) return LJ_EINVAL;
    const size_t n = (size_t)c->p.n;
    if (cell_of && n) {
        int r = check_dev_ptr(cell_of, 4);
        if (r) return r;
        LJ_CK(cudaMemcpyAsync(cell_of, c->cell_of, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
    }
    if (perm && n) {
        int r = check_dev_ptr(perm, 4);
        if (r) return r;
        LJ_CK(cudaMemcpyAsync(perm, c->perm, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
    }
    if (start) {
        int r = check_dev_ptr(start, 4);
        if (r) return r;
        LJ_CK(cudaMemcpyAsync(start, c->start, (size_t)(c->ncell + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                              c->stream));
    }
    if (count) {
        int r = check_dev_ptr(count, 4);
        if (r) return r;
        LJ_CK(launch_counts_from_start(c, count));
    }
    return LJ_OK;
}

extern "C" int lj_forces(lj_ctx *c, const double *x, void *f, double *e_pot, double *virial)
{
    if (!c) return LJ_EINVAL;
    if (c->p.n > 0) {
        int r = check_dev_ptr(x, 8);
        if (r) return r;
        r = check_dev_ptr(f, 16);
        if (r) return r;
    }
    int r = do_bin(c, x, true);
    if (r) return r;
    const bool energy = e_pot || virial;
    LJ_CK(launch_force(c, f, energy));
    if (!energy) return LJ_OK;
    LJ_CK(cudaMemsetAsync(c->scalars, 0, 2 * sizeof(double), c->stream));
    if (c->p.n > 0) LJ_CK(launch_energy_reduce(c));
    LJ_CK(cudaMemcpyAsync(c->host_scalars, c->scalars, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    r = sync_and_check(c);
    if (r) return r;
    if (e_pot) *e_pot = c->host_scalars[0];
    if (virial) *virial = c->host_scalars[1];
    return LJ_OK;
}

extern "C" int lj_langevin_seed(lj_ctx *c, int64_t seed)
{
    if (!c) return LJ_EINVAL;
    if (c->p.n == 0) return LJ_OK;
    if (!c->r48_state) LJ_CK(cudaMalloc(&c->r48_state, (size_t)c->p.n * sizeof(uint64_t)));
    LJ_CK(launch_r48_seed(c->r48_state, c->p.n, lj_srand48_state(seed), c->stream));
    c->kernel_launches++;
    return LJ_OK;
}

extern "C" int lj_get_rng_state(lj_ctx *c, uint64_t *state)
{
    if (!c) return LJ_EINVAL;
    if (c->p.n == 0) return LJ_OK;
    if (!c->r48_state) return LJ_EINVAL;   // no series yet
    int r = check_dev_ptr(state, 8);
    if (r) return r;
    LJ_CK(cudaMemcpyAsync(state, c->r48_state, (size_t)c->p.n * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                          c->stream));
    return LJ_OK;
}

extern "C" int lj_set_rng_state(lj_ctx *c, const uint64_t *state)
{
    if (!c) return LJ_EINVAL;
    if (c->p.n == 0) return LJ_OK;
    int r = check_dev_ptr(state, 8);
    if (r) return r;
    if (!c->r48_state) LJ_CK(cudaMalloc(&c->r48_state, (size_t)c->p.n * sizeof(uint64_t)));
    LJ_CK(cudaMemcpyAsync(c->r48_state, state, (size_t)c->p.n * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                          c->stream));
    return LJ_OK;
}

extern "C" int lj_langevin_step(lj_ctx *c, double *x, double *v, void *f, int32_t nsteps, double gamma, double kT)
{
    if (!c || nsteps < 0 || !(gamma >= 0.0) || !isfinite(gamma) || !(kT >= 0.0) || !isfinite(kT)) return LJ_EINVAL;
    if (c->p.n == 0 || nsteps == 0) return LJ_OK;
    if (!c->r48_state) return LJ_EINVAL;   // lj_langevin_seed first
    int r = check_dev_ptr(x, 8);
    if (r) return r;
    r = check_dev_ptr(v, 8);
    if (r) return r;
    r = check_dev_ptr(f, 16);
    if (r) return r;
    for (int s = 0; s < nsteps; s++) {
        LJ_CK(launch_langevin_bin(c, x, v, f, s == 0 ? 1 : 2, gamma, kT));
        LJ_CK(launch_scan(c));
        LJ_CK(launch_scatter(c, x, false));
        LJ_CK(launch_force(c, f, false));
    }
    LJ_CK(launch_kick(c, v, f));
    return LJ_OK;
}

extern "C" int lj_forces_n2(lj_ctx *c, const double *x, void *f, double *e_pot, double *virial)
{
    if (!c) return LJ_EINVAL;
    if (c->p.n > 0) {
        int r = check_dev_ptr(x, 8);
        if (r) return r;
        r = check_dev_ptr(f, 16);
        if (r) return r;
    }
    const bool energy = e_pot || virial;
    if (energy) LJ_CK(cudaMemsetAsync(c->scalars, 0, 2 * sizeof(double), c->stream));
    LJ_CK(launch_forces_n2(c, x, f, energy));
    if (!energy) return LJ_OK;
    LJ_CK(cudaMemcpyAsync(c->host_scalars, c->scalars, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    int r = sync_and_check(c);
    if (r) return r;
    if (e_pot) *e_pot = c->host_scalars[0];
    if (virial) *virial = c->host_scalars[1];
    return LJ_OK;
}

extern "C" int lj_step(lj_ctx *c, double *x, double *v, void *f, int32_t nsteps)
{
    if (!c || nsteps < 0) return LJ_EINVAL;
    if (c->p.n > 0 && nsteps > 0) {
        int r = check_dev_ptr(x, 8);
        if (r) return r;
        r = check_dev_ptr(v, 8);
        if (r) return r;
        r = check_dev_ptr(f, 16);
        if (r) return r;
    }
    return do_steps(c, x, v, f, nsteps);
}

extern "C" int lj_step_host(lj_ctx *c, double *x, double *v, void *f, int32_t nsteps)
{
    if (!c || nsteps < 0) return LJ_EINVAL;
    const size_t n = (size_t)c->p.n;
    if (n > 0 && (!x || !v || !f)) return LJ_EINVAL;
    int r = ensure_staging(c);
    if (r) return r;
    const size_t bx = 3 * n * sizeof(double), bf = n * force_vsize(c);
    if (!c->copy_stream) LJ_CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    if (!c->ev_xfinal) LJ_CK(cudaEventCreateWithFlags(&c->ev_xfinal, cudaEventDisableTiming));
    if (!c->ev_entry) LJ_CK(cudaEventCreateWithFlags(&c->ev_entry, cudaEventDisableTiming));
    for (int k = 0; k < kHostChunks; k++)
        if (!c->ev_chunk[k]) LJ_CK(cudaEventCreateWithFlags(&c->ev_chunk[k], cudaEventDisableTiming));
    // The regular step's first kernel (kick, drift, bin) works on each part
    // of x, v, f as soon as its copy has arrived on the second stream; the
    // other update paths take the whole arrays first.
    const bool chunked = n >= (size_t)(kHostChunks * 1024) && nsteps > 0 && c->skin <= 0.0 && !fused_mode(c) &&
                         !persistent_mode(c);
    if (chunked) {
        LJ_CK(cudaEventRecord(c->ev_entry, c->stream));
        LJ_CK(cudaStreamWaitEvent(c->copy_stream, c->ev_entry, 0));
        const size_t fv = force_vsize(c);
        for (int k = 0; k < kHostChunks; k++) {
            const size_t i0 = n * k / kHostChunks, i1 = n * (k + 1) / kHostChunks;
            LJ_CK(cudaMemcpyAsync(c->xs + 3 * i0, x + 3 * i0, 3 * (i1 - i0) * sizeof(double), cudaMemcpyHostToDevice,
                                  c->copy_stream));
            LJ_CK(cudaMemcpyAsync(c->vs + 3 * i0, v + 3 * i0, 3 * (i1 - i0) * sizeof(double), cudaMemcpyHostToDevice,
                                  c->copy_stream));
            LJ_CK(cudaMemcpyAsync((char *)c->fs + fv * i0, (const char *)f + fv * i0, fv * (i1 - i0),
                                  cudaMemcpyHostToDevice, c->copy_stream));
            LJ_CK(cudaEventRecord(c->ev_chunk[k], c->copy_stream));
            LJ_CK(cudaStreamWaitEvent(c->stream, c->ev_chunk[k], 0));
            LJ_CK(launch_kick_drift_bin(c, c->xs, c->vs, c->fs, 1, (int64_t)i0, (int64_t)i1));
        }
        c->kdb_done = 1;
    } else if (n > 0) {
        LJ_CK(cudaMemcpyAsync(c->xs, x, bx, cudaMemcpyHostToDevice, c->stream));
        LJ_CK(cudaMemcpyAsync(c->vs, v, bx, cudaMemcpyHostToDevice, c->stream));
        LJ_CK(cudaMemcpyAsync(c->fs, f, bf, cudaMemcpyHostToDevice, c->stream));
    }
    // x is final after the last scatter: its copy back runs on the second
    // stream while the last force evaluation and kick run
    const bool overlap = n > 0 && nsteps > 0;
    r = do_steps(c, c->xs, c->vs, c->fs, nsteps, overlap ? c->ev_xfinal : nullptr);
    c->kdb_done = 0;
    if (r) return r;
    if (n > 0) {
        if (overlap) {
            LJ_CK(cudaStreamWaitEvent(c->copy_stream, c->ev_xfinal, 0));
            LJ_CK(cudaMemcpyAsync(x, c->xs, bx, cudaMemcpyDeviceToHost, c->copy_stream));
        } else {
            LJ_CK(cudaMemcpyAsync(x, c->xs, bx, cudaMemcpyDeviceToHost, c->stream));
        }
        LJ_CK(cudaMemcpyAsync(v, c->vs, bx, cudaMemcpyDeviceToHost, c->stream));
        LJ_CK(cudaMemcpyAsync(f, c->fs, bf, cudaMemcpyDeviceToHost, c->stream));
    }
    LJ_CK(cudaStreamSynchronize(c->copy_stream));
    return sync_and_check(c);
}

extern "C" int lj_energy(lj_ctx *c, const double *x, const double *v, double *out)
{
    if (!c || !out) return LJ_EINVAL;
    if (c->p.n > 0) {
        int r = check_dev_ptr(x, 8);
        if (r) return r;
        r = check_dev_ptr(v, 8);
        if (r) return r;
    }
    int r = ensure_staging(c);
    if (r) return r;
    LJ_CK(cudaMemsetAsync(c->scalars, 0, 4 * sizeof(double), c->stream));
    if (c->p.n > 0) {
        LJ_CK(launch_ekin(c, v));
        r = do_bin(c, x, true);
        if (r) return r;
        LJ_CK(launch_force(c, c->fs, true));
        LJ_CK(launch_energy_reduce(c));
    }
    LJ_CK(cudaMemcpyAsync(c->host_scalars, c->scalars, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    r = sync_and_check(c);
    if (r) return r;
    out[0] = c->host_scalars[2];
    out[1] = c->host_scalars[0];
    out[2] = out[0] + out[1];
    return LJ_OK;
}

extern "C" int lj_observables(lj_ctx *c, const double *x, const double *v, double *out)
{
    if (!c || !out) return LJ_EINVAL;
    if (c->p.n > 0) {
        int r = check_dev_ptr(x, 8);
        if (r) return r;
        r = check_dev_ptr(v, 8);
        if (r) return r;
    }
    int r = ensure_staging(c);
    if (r) return r;
    LJ_CK(cudaMemsetAsync(c->scalars, 0, 8 * sizeof(double), c->stream));
    if (c->p.n > 0) {
        LJ_CK(launch_ekin(c, v));
        r = do_bin(c, x, true);
        if (r) return r;
        LJ_CK(launch_force(c, c->fs, true));
        LJ_CK(launch_energy_reduce(c));
    }
    LJ_CK(launch_observables(c));
    LJ_CK(cudaMemcpyAsync(c->host_scalars, c->scalars, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    r = sync_and_check(c);
    if (r) return r;
    out[0] = c->host_scalars[2];
    out[1] = c->host_scalars[0];
    out[2] = c->host_scalars[3];
    out[3] = c->host_scalars[1];
    out[4] = c->host_scalars[4];
    out[5] = c->host_scalars[5];
    return LJ_OK;
}

extern "C" int lj_check(lj_ctx *c)
{
    if (!c) return LJ_EINVAL;
    return sync_and_check(c);
}

extern "C" int lj_set_params(lj_ctx *c, double eps, double sigma)
{
    if (!c || !(sigma > 0.0) || !isfinite(sigma) || !(eps >= 0.0) || !isfinite(eps)) return LJ_EINVAL;
    c->p.eps = eps;
    c->p.sigma = sigma;
    c->gen++;   // captured steps hold the old coefficients
    if (c->pers) {   // the persistent batch holds them too: rebuilt at the next step
        LJ_CK(cudaStreamSynchronize(c->stream));
        lj_batch_destroy(c->pers);
        c->pers = nullptr;
    }
    return LJ_OK;
}

extern "C" int lj_forces_vjp(lj_ctx *c, const double *x, const double *g, double scale, double *dx, double *dparam)
{
    if (!c || !isfinite(scale)) return LJ_EINVAL;
    int r;
    if ((r = check_dev_ptr(dparam, 8)) != LJ_OK) return r;
    if (c->p.n == 0) return LJ_OK;
    if ((r = check_dev_ptr(x, 8)) != LJ_OK) return r;
    if ((r = check_dev_ptr(g, 8)) != LJ_OK) return r;
    if ((r = check_dev_ptr(dx, 8)) != LJ_OK) return r;
    if ((r = ensure_vjp_buffers(c)) != LJ_OK) return r;
    if ((r = do_bin(c, x, true)) != LJ_OK) return r;
    LJ_CK(launch_vjp(c, g, scale, dx, dparam));
    return LJ_OK;
}

extern "C" int lj_vv_adjoint_step(lj_ctx *c, const double *x_n, const double *x_n1, double *lam_x, double *lam_v,
                                  double *dparam)
{
    if (!c) return LJ_EINVAL;
    int r;
    if ((r = check_dev_ptr(dparam, 8)) != LJ_OK) return r;
    if (c->p.n == 0) return LJ_OK;
    if ((r = check_dev_ptr(x_n, 8)) != LJ_OK) return r;
    if ((r = check_dev_ptr(x_n1, 8)) != LJ_OK) return r;
    if ((r = check_dev_ptr(lam_x, 8)) != LJ_OK) return r;
    if ((r = check_dev_ptr(lam_v, 8)) != LJ_OK) return r;
    if ((r = ensure_vjp_buffers(c)) != LJ_OK) return r;
    const double h = 0.5 * c->p.dt / c->p.mass;
    // v_{n+1} = v_half + h F(x_{n+1})
    if ((r = do_bin(c, x_n1, true)) != LJ_OK) return r;
    LJ_CK(launch_vjp(c, lam_v, h, lam_x, dparam));
    // x_{n+1} = x_n + dt v_half
    LJ_CK(launch_axpy(c, lam_v, lam_x, c->p.dt));
    // v_half = v_n + h F(x_n)
    if ((r = do_bin(c, x_n, true)) != LJ_OK) return r;
    LJ_CK(launch_vjp(c, lam_v, h, lam_x, dparam));
    return LJ_OK;
}

extern "C" int lj_set_skin(lj_ctx *c, double skin, int32_t max_interval)
{
    if (c) c->gen++;   // captured steps hold the old configuration
    if (!c || !(skin >= 0.0) || !isfinite(skin) || max_interval < 0) return LJ_EINVAL;
    if (skin > 0.0 && c->fuse_update) return LJ_EINVAL;   // the fused update bins in the force kernel
    const int k = c->p.cell_subdiv == 2 ? 2 : 1;
    const double q = floor(((double)k * c->p.box) / (c->p.rc + skin));
    if (!(q >= 2.0 * k + 1.0)) return LJ_EBOX;
    const int nc = (int)q;
    if (nc != c->nc) {
        LJ_CK(cudaStreamSynchronize(c->stream));
        int r = setup_grid(c, nc);
        if (r) return r;
    }
    if (skin > 0.0) {
        const size_t n1 = (size_t)(c->p.n > 0 ? c->p.n : 1);
        if (!c->disp) LJ_CK(cudaMalloc(&c->disp, n1 * sizeof(float4)));
        if (!c->skin_flags) LJ_CK(cudaMalloc(&c->skin_flags, 4 * sizeof(int32_t)));
        if (!c->skin_counts) LJ_CK(cudaMalloc(&c->skin_counts, 2 * sizeof(long long)));
        LJ_CK(cudaMemsetAsync(c->disp, 0, n1 * sizeof(float4), c->stream));
        LJ_CK(cudaMemsetAsync(c->skin_flags, 0, 4 * sizeof(int32_t), c->stream));
        LJ_CK(cudaMemsetAsync(c->skin_counts, 0, 2 * sizeof(long long), c->stream));
    }
    c->skin = skin;
    c->skin_max_interval = max_interval;
    c->skin_dirty = 1;
    LJ_CK(cudaStreamSynchronize(c->stream));
    return LJ_OK;
}

extern "C" int lj_wait_selftest(lj_ctx *c)
{
    if (!c) return LJ_EINVAL;
    LJ_CK(launch_wait_selftest(c));
    return sync_and_check(c);
}

extern "C" int lj_set_deterministic(lj_ctx *c, int32_t enable)
{
    if (!c || (enable != 0 && enable != 1)) return LJ_EINVAL;
    if (enable && !c->pos_alt) {
        const size_t n1 = (size_t)(c->p.n > 0 ? c->p.n : 1);
        LJ_CK(cudaMalloc(&c->pos_alt, n1 * force_vsize(c)));
        LJ_CK(cudaMalloc(&c->perm_alt, n1 * sizeof(int32_t)));
    }
    c->deterministic = enable;
    c->gen++;   // captured steps do not sort
    return LJ_OK;
}

extern "C" int lj_set_graph(lj_ctx *c, int32_t enable)
{
    if (!c || (enable != 0 && enable != 1)) return LJ_EINVAL;
    c->use_graph = enable;
    if (!enable && c->gexec) {
        LJ_CK(cudaStreamSynchronize(c->stream));
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return LJ_OK;
}

extern "C" int lj_skin_stats(lj_ctx *c, int64_t *rebuilds, int64_t *steps)
{
    if (!c) return LJ_EINVAL;
    long long h[2] = {0, 0};
    if (c->skin_counts) {
        LJ_CK(cudaStreamSynchronize(c->stream));
        LJ_CK(cudaMemcpy(h, c->skin_counts, sizeof(h), cudaMemcpyDeviceToHost));
    }
    if (rebuilds) *rebuilds = h[0];
    if (steps) *steps = h[1];
    return LJ_OK;
}

extern "C" int lj_set_tuning(lj_ctx *c, int32_t kernel, int32_t group_width, int32_t cells_per_grab)
{
    if (c) c->gen++;   // captured steps hold the old configuration
    if (!c || kernel < 0 || kernel > 7 || cells_per_grab < 0 || cells_per_grab > 1024) return LJ_EINVAL;
    if (kernel == 7) {   // each pair once (Newton's third law), 27-cell stencil: FP32-mixed or FP64
        if (c->p.cell_subdiv == 2) return LJ_EINVAL;
        const int r = lj_set_tuning(c, 3, group_width, cells_per_grab);   // gw: for the deterministic fallback
        if (r != LJ_OK) return r;
        c->n3 = 1;
        return LJ_OK;
    }
    c->n3 = 0;
    if (kernel == 6) {   // lj_step as one persistent launch per step; forces by the warp kernel
        if (c->p.precision != LJ_PREC_MIXED || c->p.cell_subdiv == 2) return LJ_EINVAL;
        const int r = lj_set_tuning(c, 3, group_width, cells_per_grab);
        if (r != LJ_OK) return r;
        c->use_pers = 1;
        return LJ_OK;
    }
    c->use_pers = 0;
    if (kernel == 4) {   // the paper's fixed-capacity cell arrays: FP32-mixed, 27-cell stencil
        if (c->p.precision != LJ_PREC_MIXED || c->p.cell_subdiv == 2) return LJ_EINVAL;
        c->use_aop = 1;
        c->use_run_kernel = 0;
        c->fuse_update = 0;
        return LJ_OK;
    }
    c->use_aop = 0;
    if (kernel == 5 && (c->p.precision != LJ_PREC_MIXED || c->p.cell_subdiv == 2)) return LJ_EINVAL;
    c->pipe = kernel == 5 ? 1 : 0;
    if (kernel == 5) kernel = 3;   // warp kernel, stencils bulk-copied one cell ahead
    if (group_width != 0 && group_width != -1 && group_width != 2 && group_width != 4 && group_width != 8 &&
        group_width != 16 && group_width != 32)
        return LJ_EINVAL;
    const bool warp = kernel == 0 || kernel == 3;
    if (kernel == 0 && c->p.precision == LJ_PREC_FP64) return LJ_EINVAL;   // fused update: FP32-mixed
    if (!warp && c->p.cell_subdiv == 2) return LJ_EINVAL;            // run kernels: 27-cell stencil only
    if (kernel == 0 && c->skin > 0.0) return LJ_EINVAL;              // fused update bins every step
    if (warp && c->wforce_grid == 0)
        LJ_CK(c->p.precision == LJ_PREC_MIXED ? warp_force_configure(c) : w64_force_configure(c));
    c->use_run_kernel = warp ? 0 : 1;
    c->fuse_update = kernel == 0 ? 1 : 0;
    c->grab = cells_per_grab;
    c->use_tma = kernel == 2 ? 0 : 1;
    c->gw = group_width;
    return LJ_OK;
}

extern "C" int lj_set_timing(lj_ctx *c, int32_t enable)
{
    if (!c) return LJ_EINVAL;
    if (enable) {
        if (!c->ev) {
            c->ev = (cudaEvent_t *)calloc(kEventPool, sizeof(cudaEvent_t));
            if (!c->ev) return LJ_ENOMEM;
            for (int i = 0; i < kEventPool; i++) {
                cudaError_t e = cudaEventCreate(&c->ev[i]);
                if (e != cudaSuccess) {
                    c->nev = i;
                    return map_cuda(e);
                }
            }
            c->nev = kEventPool;
        }
        LJ_CK(cudaStreamSynchronize(c->stream));
        c->ev_used = 0;
        c->force_ms = 0.0;
        c->force_launches = 0;
    }
    c->timing = enable ? 1 : 0;
    return LJ_OK;
}

extern "C" int lj_read_timing(lj_ctx *c, double *force_ms, int64_t *force_launches, int64_t *kernel_launches)
{
    if (!c) return LJ_EINVAL;
    LJ_CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i + 1 < c->ev_used; i += 2) {
        float ms = 0.0f;
        LJ_CK(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
        c->force_ms += ms;
        c->force_launches++;
    }
    c->ev_used = 0;
    if (force_ms) *force_ms = c->force_ms;
    if (force_launches) *force_launches = c->force_launches;
    if (kernel_launches) *kernel_launches = c->kernel_launches;
    return LJ_OK;
}
