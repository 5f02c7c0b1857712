// ss_verify.cu -- accuracy harness kernels: banded edit distance per pair
// and the confusion counts of filter decisions against it.
#include <cuda_runtime.h>

#include <cstdint>

#include "ss_internal.h"
#include "ss_verify.cuh"

namespace ssk {

template <int E>
__global__ void __launch_bounds__(128) k_ed_banded(const EdArgs a)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t *q = a.reads + p * a.w16;
        const uint32_t *r = a.refs + p * a.w16;
        a.ed[p] = ed_banded<E>(q, r, a.m, a.w16);
    }
}

// counts[0..3] += (accepted & ED<=E, accepted & ED>E, rejected & ED<=E,
// rejected & ED>E): true accepts, false accepts, false rejects, true
// rejects (Section 3.2's rates are false accepts / (ED>E) and false
// rejects / (ED<=E)).
__global__ void k_confusion(const uint8_t *__restrict__ acc,
                            const int32_t *__restrict__ ed, int64_t n, int E,
                            unsigned long long *counts)
{
    unsigned long long c[4] = {0, 0, 0, 0};
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const bool a = acc[p] != 0, close = ed[p] <= E;
        c[(a ? 0 : 2) + (close ? 0 : 1)] += 1;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        unsigned long long v = c[k];
        for (int off = 16; off > 0; off >>= 1)
            v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v)
            atomicAdd(&counts[k], v);
    }
}

// Warp per pair, pairs of any length and threshold; the launch for class C
// (2E+1 <= 32 C, E <= 511) routes the pairs of that class and skips the
// others; the first launch also flags unsupported thresholds.
struct EdVarArgs {
    const uint32_t *reads;
    const uint32_t *refs;
    const int64_t *off;   // words
    const int32_t *len;   // bases
    const int32_t *E;
    int64_t n;
    int32_t *ed;
    int *status;
};

template <int C, int CLO>
__global__ void __launch_bounds__(128) k_ed_warp(const EdVarArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp =
        ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < a.n; p += nwarps) {
        const int m = a.len[p], E = a.E[p];
        if (m < 0 || E < 0 || E > kEdWarpMaxE) {
            if (CLO == 0 && lane == 0) {
                a.ed[p] = -1;
                atomicOr(a.status, m < 0 || E < 0 ? kStatusInvalidArg
                                                  : kStatusUnsupported);
            }
            continue;
        }
        const int need = (2 * E + 1 + 31) >> 5;  // cells per lane
        if (need <= CLO || need > C)
            continue;
        const int v = ed_band_warp<C>(a.reads + a.off[p], a.refs + a.off[p],
                                      m, E);
        if (lane == 0)
            a.ed[p] = v;
    }
}

namespace {
template <int E>
cudaError_t launch_ed_one(const EdArgs &a, int sm_count, cudaStream_t st)
{
    const int64_t want = (a.n + 127) / 128;
    const int grid = (int)(want < (int64_t)sm_count * 16 ? want
                                                         : (int64_t)sm_count * 16);
    k_ed_banded<E><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <int... Es>
cudaError_t launch_ed_dispatch(int E, const EdArgs &a, int sm_count,
                               cudaStream_t st,
                               std::integer_sequence<int, Es...>)
{
    cudaError_t out = cudaErrorInvalidValue;
    ((E == Es ? (out = launch_ed_one<Es>(a, sm_count, st), 0) : 0), ...);
    return out;
}
}  // namespace

cudaError_t launch_ed_banded(int E, const uint32_t *reads,
                             const uint32_t *refs, int64_t n, int32_t m,
                             int32_t *ed, int sm_count, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    EdArgs a{reads, refs, n, m, (m + 15) / 16, ed};
    return launch_ed_dispatch(E, a, sm_count, st,
                              std::make_integer_sequence<int, kEdMaxE + 1>{});
}

cudaError_t launch_ed_var(const uint32_t *reads, const uint32_t *refs,
                          const int64_t *off, const int32_t *len,
                          const int32_t *E, int64_t n, int32_t *ed,
                          int *status, int sm_count, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    const EdVarArgs a{reads, refs, off, len, E, n, ed, status};
    const int64_t want = (n * 32 + 127) / 128;
    const int grid = (int)(want < (int64_t)sm_count * 16
                               ? want
                               : (int64_t)sm_count * 16);
    k_ed_warp<1, 0><<<grid, 128, 0, st>>>(a);
    k_ed_warp<2, 1><<<grid, 128, 0, st>>>(a);
    k_ed_warp<4, 2><<<grid, 128, 0, st>>>(a);
    k_ed_warp<8, 4><<<grid, 128, 0, st>>>(a);
    k_ed_warp<16, 8><<<grid, 128, 0, st>>>(a);
    k_ed_warp<32, 16><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_confusion(const uint8_t *acc, const int32_t *ed,
                             int64_t n, int E, unsigned long long *counts,
                             int sm_count, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long),
                                    st);
    if (e != cudaSuccess || n <= 0)
        return e;
    const int64_t want = (n + 255) / 256;
    const int grid = (int)(want < (int64_t)sm_count * 8 ? want
                                                        : (int64_t)sm_count * 8);
    k_confusion<<<grid, 256, 0, st>>>(acc, ed, n, E, counts);
    return cudaGetLastError();
}

}  // namespace ssk
