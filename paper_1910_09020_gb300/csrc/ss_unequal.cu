// ss_unequal.cu -- launches for pairs of different lengths, thread per
// pair (the kernel is in ss_unequal_tile.cuh).
//
// A uniform threshold e gets one launch with the routine for exactly e
// (ss_unequal_x0.cu, ss_unequal_x1.cu); per-pair thresholds get one launch
// per row class (E' <= 3, 7, 15, 31), each walking all pairs and skipping
// the others.  The first launch also writes the pairs that need no routing
// and flags the invalid and unsupported ones.
#include "ss_unequal_tile.cuh"

namespace ssk {

cudaError_t launch_unequal(const uint32_t *reads, const int64_t *read_off,
                           const int32_t *read_len, const uint32_t *refs,
                           const int64_t *ref_off, const int32_t *ref_len,
                           const int32_t *E, int32_t e, int64_t n,
                           uint8_t *acc, int32_t *obs, int *status,
                           int sm_count, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    const UnequalArgs a{reads, read_off, read_len, refs, ref_off, ref_len,
                        E, e, n, acc, obs, status};
    const unsigned grid = unequal_grid(n);
    if (grid == 0)
        return cudaErrorInvalidValue;
    if (!E) {
        // a uniform threshold: every pair routed for exactly that threshold
        if (e < 0)
            return cudaErrorInvalidValue;
        const int ex = e < kRwMaxE ? e : kRwMaxE;
        // e above 31 leaves pairs past 31 rows: flagged unsupported by the
        // class launch, which also answers the others
        if (e > kRwMaxE) {
            k_unequal_tile<31, -1, false><<<grid, kRwThreads, 0, st>>>(a);
            return cudaGetLastError();
        }
        return ex <= 15 ? launch_unequal_exact_x0(ex, a, grid, st)
                        : launch_unequal_exact_x1(ex, a, grid, st);
    }
    // per-pair thresholds: one launch per row class
    k_unequal_tile<3, -1, false><<<grid, kRwThreads, 0, st>>>(a);
    k_unequal_tile<7, 3, false><<<grid, kRwThreads, 0, st>>>(a);
    k_unequal_tile<15, 7, false><<<grid, kRwThreads, 0, st>>>(a);
    k_unequal_tile<31, 15, false><<<grid, kRwThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ssk
