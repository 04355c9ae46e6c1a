// Device helpers shared by the run kernel (lj_force.cu) and the all-pairs
// kernel (lj_n2.cu): shared-memory bulk copies completing on mbarriers with
// bounded waits, and the scalar Lennard-Jones pair term in FP32 or FP64.
#pragma once

#include "lj_internal.cuh"

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Global -> shared bulk copy completing on an mbarrier.  dst, src 16-byte
// aligned, bytes a positive multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait on an mbarrier phase: gives up after ~2^31 SM cycles (about
// one second), latches LJ_ERRBIT_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int32_t *err)
{
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) {
            atomicOr(err, LJ_ERRBIT_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ float fast_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float fast_rsqrt(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <typename T> struct PairMath;

template <> struct PairMath<float> {
    static __device__ __forceinline__ float rcp(float x) { return fast_rcp(x); }
    static __device__ __forceinline__ float rsqrt(float x) { return fast_rsqrt(x); }
};

template <> struct PairMath<double> {
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / sqrt(x); }
};

template <typename T> struct Coef {
    T rc2, rc, a12, b6, c12, c6, uc, fc;
    template <class P>
    __device__ __forceinline__ explicit Coef(const P &p)
        : rc2((T)p.rc2), rc((T)p.rc), a12((T)p.a12), b6((T)p.b6), c12((T)p.c12), c6((T)p.c6), uc((T)p.uc),
          fc((T)p.fc)
    {
    }
};

// One candidate pair.  d = x_i - x_j (already shifted to the neighbour
// cell).  F(r)/r = (24 eps / r^2) [2 (sigma/r)^12 - (sigma/r)^6]
//               = ri r6i (48 eps sigma^12 r6i - 24 eps sigma^6),
// ri = 1/r^2, r6i = ri^3; MODE 2 subtracts F(rc)/r; MODE >= 1 shifts U.
template <typename T, int MODE, bool ENERGY>
__device__ __forceinline__ void pair_accum(T dx, T dy, T dz, const Coef<T> &k, T &fx, T &fy, T &fz, T &e, T &w)
{
    T r2 = dx * dx + dy * dy + dz * dz;
    bool in = (r2 < k.rc2) && (r2 > (T)0);
    T ri, rinv = (T)0;
    if constexpr (MODE == 2) {
        rinv = PairMath<T>::rsqrt(r2);
        rinv = in ? rinv : (T)0;
        ri = rinv * rinv;
    } else {
        ri = PairMath<T>::rcp(r2);
        ri = in ? ri : (T)0;
    }
    T r6i = ri * ri * ri;
    T ff = ri * r6i * (k.a12 * r6i - k.b6);
    if constexpr (MODE == 2) ff -= k.fc * rinv;
    fx += ff * dx;
    fy += ff * dy;
    fz += ff * dz;
    if constexpr (ENERGY) {
        T u = r6i * (k.c12 * r6i - k.c6);
        if constexpr (MODE >= 1) u -= k.uc;
        if constexpr (MODE == 2) u += (r2 * rinv - k.rc) * k.fc;
        e += in ? u : (T)0;
        w += ff * r2;
    }
}

}  // namespace
