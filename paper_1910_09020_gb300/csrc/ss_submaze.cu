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

template <int EMAX>
__global__ void __launch_bounds__(128) k_submaze(const SubmazeArgs a)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const GlobalSeq q{a.reads + p * a.w16, a.w16};
        const GlobalSeq r{a.refs + p * a.w16, a.w16};
        // the column walk from EMAX = 7 (it walks at least one 8-column
        // chunk, which row-wise routing of up to 7 rows undercuts); the
        // row-wise form for 63 rows
        int cnt;
        if constexpr (EMAX >= 7 && EMAX <= 15)
            cnt = submaze_route_cols<EMAX>(q, r, a.m, a.E, a.t, a.y);
        else
            cnt = submaze_route<EMAX>(q, r, a.m, a.E, a.t, a.y, a.neg1);
        a.acc[p] = (uint8_t)(cnt <= a.E);
        a.obs[p] = cnt;
    }
}

cudaError_t launch_submaze(const uint32_t *reads, const uint32_t *refs,
                           int64_t n, int32_t m, int32_t E, int32_t t,
                           int32_t y, uint8_t *acc, int32_t *obs,
                           int sm_count, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    SubmazeArgs a{reads, refs, n, m, E, t, y, (m + 15) / 16, 0xffffffffu,
                  acc, obs};
    const int64_t want = (n + 127) / 128;
    const int64_t cap = (int64_t)sm_count * 16;
    const int grid = (int)(want < cap ? want : cap);
    const int Ee = E < m - 1 ? E : (m > 0 ? m - 1 : 0);
    if (Ee <= 3)
        k_submaze<3><<<grid, 128, 0, st>>>(a);
    else if (Ee <= 7)
        k_submaze<7><<<grid, 128, 0, st>>>(a);
    else if (Ee <= 15)
        k_submaze<15><<<grid, 128, 0, st>>>(a);
    else if (Ee <= 31)
        k_submaze<31><<<grid, 128, 0, st>>>(a);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace ssk
