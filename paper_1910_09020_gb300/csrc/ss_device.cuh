// ss_device.cuh -- device-side helpers shared by the filter kernels.
//
// Packed format (SS_FMT_PACKED2, include/ss.h): 16 bases per uint32; bit t
// holds code bit 0 of base t and bit 16+t holds code bit 1.  The kernels work
// on "bit planes" of 32 columns: lo32/hi32 hold code bits 0/1 of 32
// consecutive bases, so one XOR per plane compares 32 bases at once.
#pragma once
#include <cstdint>

// The routing functions are __host__ __device__ so that the test suite can
// also compile them for the host and check their logic on the CPU; the
// wrappers below are the device intrinsics on the GPU.
#define SS_HD __host__ __device__ __forceinline__

namespace ssk {

SS_HD uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t s)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_r(lo, hi, s);
#else
    return (uint32_t)(((((uint64_t)hi) << 32) | lo) >> (s & 31u));
#endif
}

SS_HD uint32_t funnel_l(uint32_t lo, uint32_t hi, uint32_t s)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_l(lo, hi, s);
#else
    return (uint32_t)((((((uint64_t)hi) << 32) | lo) << (s & 31u)) >> 32);
#endif
}

SS_HD int ffs32(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return __ffs((int)x);
#else
    return __builtin_ffs((int)x);
#endif
}

SS_HD int imax(int a, int b) { return a > b ? a : b; }
SS_HD int imin(int a, int b) { return a < b ? a : b; }

template <class T>
SS_HD T ldg(const T *p)
{
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// Device status bits latched in the context (returned by ss_sync).
constexpr int kStatusInvalidBase = 1;
constexpr int kStatusInvalidArg = 2;
constexpr int kStatusTimeout = 4;
constexpr int kStatusUnsupported = 8;

// Two packed words (bases 32k..32k+15 and 32k+16..32k+31) -> the two
// 32-column planes of word k.
SS_HD void planes_of(uint32_t p0, uint32_t p1, uint32_t &lo, uint32_t &hi)
{
#ifdef __CUDA_ARCH__
    lo = __byte_perm(p0, p1, 0x5410);  // low halves: code bit 0
    hi = __byte_perm(p0, p1, 0x7632);  // high halves: code bit 1
#else
    lo = (p0 & 0xffffu) | (p1 << 16);
    hi = (p0 >> 16) | (p1 & 0xffff0000u);
#endif
}

// Byte permute: byte i of the result is byte (s >> 4i) & 7 of the 8-byte
// value b:a (selector nibbles 0..7 only).
SS_HD uint32_t prmt(uint32_t a, uint32_t b, uint32_t s)
{
#ifdef __CUDA_ARCH__
    return __byte_perm(a, b, s);
#else
    const uint64_t v = ((uint64_t)b << 32) | a;
    uint32_t r = 0;
    for (int i = 0; i < 4; ++i)
        r |= (uint32_t)((v >> (8 * ((s >> (4 * i)) & 7u))) & 0xffu) << (8 * i);
    return r;
#endif
}

#ifdef __CUDACC__
// ---- bulk asynchronous copies and mbarriers (sm_90 and later) ----------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                     smem_addr(bar)),
                 "r"(count)
                 : "memory");
}

// Make initialised barriers visible to the asynchronous (copy) proxy.
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces `bytes` of copies completing on `bar`.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar,
                                                      uint32_t bytes)
{
    asm volatile(
        "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
            smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

// Global -> shared bulk copy (addresses 16-byte aligned, bytes a multiple
// of 16) completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src,
                                          uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
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
    return ok != 0u;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` to complete, for at most about limit_ns
// (and at most kWaitMaxPolls polls, should the timer not advance); false on
// timeout.
constexpr uint32_t kWaitMaxPolls = 1u << 22;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar,
                                                  uint32_t parity,
                                                  uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = global_ns();
    for (uint32_t polls = 0; polls < kWaitMaxPolls; ++polls) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (global_ns() - t0 > limit_ns)
            return false;
    }
    return false;
}
#endif

// Bits t >= lim of a 32-column word set (lim <= 0: all, lim >= 32: none).
SS_HD uint32_t mask_from(int lim)
{
    return lim <= 0 ? 0xffffffffu : (lim >= 32 ? 0u : (0xffffffffu << lim));
}

// Bits t < lim set (lim <= 0: none, lim >= 32: all).
SS_HD uint32_t mask_below(int lim)
{
#ifdef __CUDA_ARCH__
    // shl.b32 clamps shift amounts above 32 to 32 (giving 0)
    uint32_t b;
    asm("shl.b32 %0, 1, %1;" : "=r"(b) : "r"((uint32_t)imax(lim, 0)));
    return b - 1u;
#else
    return lim <= 0 ? 0u : (lim >= 32 ? 0xffffffffu : ((1u << lim) - 1u));
#endif
}

// ceil(2^32 / d) for d >= 2 (0 for d <= 1, where fast_div returns x):
// __umulhi(x, magic) equals x / d whenever x * d < 2^32.
__host__ __device__ inline uint32_t div_magic(uint32_t d)
{
    return d <= 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + d - 1) / d);
}

__device__ __forceinline__ uint32_t fast_div(uint32_t x, uint32_t d,
                                             uint32_t magic)
{
    return d <= 1 ? x : __umulhi(x, magic);
}

}  // namespace ssk
