// ss_submaze.cu -- kernels of the sub-maze approximate mode (Section 2.5).
#include <cuda_runtime.h>

#include <cstdint>

#include "ss_internal.h"
#include "ss_submaze.cuh"

namespace ssk {

struct SubmazeArgs {
    const uint32_t *reads;
    const uint32_t *refs;
    int64_t n;
    int32_t m, E, t, y, w16;
    uint32_t neg1;
    uint8_t *acc;
    int32_t *obs;
};

// The pair's route: the column walk from EMAX = 7 (it walks at least one
// 8-column chunk, which row-wise routing of up to 7 rows undercuts); the
// row-wise form for 63 rows.
template <int EMAX, class Seq>
__device__ __forceinline__ int submaze_pair(const Seq &q, const Seq &r,
                                            int m, int E, int t, int y,
                                            uint32_t neg1)
{
    if constexpr (EMAX >= 7 && EMAX <= 15)
        return submaze_route_cols<EMAX>(q, r, m, E, t, y);
    else
        return submaze_route<EMAX>(q, r, m, E, t, y, neg1);
}

// m <= 256: the plain launch's pipeline (bulk-copied stages, tiles ordered
// by predicted cost, so a warp holds pairs of similar routing work).
template <int EMAX>
__global__ void __launch_bounds__(128) k_submaze_pipe(const RwPipeArgs a,
                                                       const int E,
                                                       const int t,
                                                       const int y)
{
    rw_pipe_run<true>(a, E, [&](const SmemSeqPad &q, const SmemSeqPad &r) {
        return submaze_pair<EMAX>(q, r, a.m, E, t, y, a.neg1);
    });
}

// Longer pairs: one thread per pair straight from global memory.
template <int EMAX>
__global__ void __launch_bounds__(128) k_submaze(const SubmazeArgs a)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const GlobalSeq q{a.reads + p * a.w16, a.w16};
        const GlobalSeq r{a.refs + p * a.w16, a.w16};
        const int cnt =
            submaze_pair<EMAX>(q, r, a.m, a.E, a.t, a.y, a.neg1);
        a.acc[p] = (uint8_t)(cnt <= a.E);
        a.obs[p] = cnt;
    }
}

template <int EMAX>
cudaError_t submaze_launch_one(const uint32_t *reads, const uint32_t *refs,
                               int64_t n, int32_t m, int32_t E, int32_t t,
                               int32_t y, uint8_t *acc, int32_t *obs,
                               int *status, int sm_count, cudaStream_t st)
{
    if ((m + 15) / 16 <= kRwPipeMaxW16) {
        RwPipeArgs a;
        unsigned grid;
        size_t smem;
        if (!rw_pipe_config(reads, refs, n, m, acc, obs, status, a, grid,
                            smem))
            return cudaErrorInvalidValue;
        k_submaze_pipe<EMAX><<<grid, kRwThreads, smem, st>>>(a, E, t, y);
    } else {
        SubmazeArgs a{reads, refs, n, m, E, t, y, (m + 15) / 16,
                      0xffffffffu, acc, obs};
        const int64_t want = (n + 127) / 128;
        const int64_t cap = (int64_t)sm_count * 16;
        const int grid = (int)(want < cap ? want : cap);
        k_submaze<EMAX><<<grid, 128, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_submaze(const uint32_t *reads, const uint32_t *refs,
                           int64_t n, int32_t m, int32_t E, int32_t t,
                           int32_t y, uint8_t *acc, int32_t *obs,
                           int *status, int sm_count, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    const int Ee = E < m - 1 ? E : (m > 0 ? m - 1 : 0);
    if (Ee <= 3)
        return submaze_launch_one<3>(reads, refs, n, m, E, t, y, acc, obs,
                                     status, sm_count, st);
    if (Ee <= 7)
        return submaze_launch_one<7>(reads, refs, n, m, E, t, y, acc, obs,
                                     status, sm_count, st);
    if (Ee <= 15)
        return submaze_launch_one<15>(reads, refs, n, m, E, t, y, acc, obs,
                                      status, sm_count, st);
    if (Ee <= 31)
        return submaze_launch_one<31>(reads, refs, n, m, E, t, y, acc, obs,
                                      status, sm_count, st);
    return cudaErrorInvalidValue;
}

}  // namespace ssk
