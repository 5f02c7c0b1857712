// ss_unequal.cu -- kernel for pairs of different lengths, thread per pair.
//
// Pairs are routed by the launch of their row class (E' <= 3, 7, 15, 31);
// each launch walks all pairs and skips the others, so a batch with mixed
// thresholds and lengths needs no sort.  The first launch also writes the
// pairs that need no routing and flags the invalid and unsupported ones.
#include <cuda_runtime.h>

#include <cstdint>

#include "ss_internal.h"
#include "ss_rw.cuh"
#include "ss_unequal.cuh"

namespace ssk {

struct UnequalArgs {
    const uint32_t *reads;
    const int64_t *read_off;  // words
    const int32_t *read_len;  // bases
    const uint32_t *refs;
    const int64_t *ref_off;
    const int32_t *ref_len;
    const int32_t *E;         // per pair, or nullptr: e for all
    int32_t e;
    int64_t n;
    uint8_t *acc;
    int32_t *obs;
    int *status;
};

template <int EMAX, int ELO>
__global__ void __launch_bounds__(128) k_rw_unequal(const UnequalArgs a)
{
    int bad = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int mQ = a.read_len[p];
        const int mR = a.ref_len[p];
        const int E = a.E ? a.E[p] : a.e;
        if (mQ < 0 || mR < 0 || E < 0) {
            if (ELO < 0) {
                a.acc[p] = 0;
                a.obs[p] = -1;
                bad |= kStatusInvalidArg;
            }
            continue;
        }
        const int rows = unequal_rows(mQ, mR, E);
        if (rows < 0) {
            if (ELO < 0) {
                a.acc[p] = 1;
                a.obs[p] = 0;
            }
            continue;
        }
        if (rows > kRwMaxE) {
            if (ELO < 0) {
                a.acc[p] = 0;
                a.obs[p] = -1;
                bad |= kStatusUnsupported;
            }
            continue;
        }
        if (rows <= ELO || rows > EMAX)
            continue;
        const GlobalSeq q{a.reads + a.read_off[p], (mQ + 15) >> 4};
        const GlobalSeq r{a.refs + a.ref_off[p], (mR + 15) >> 4};
        // the column walk from 15 rows; row-wise below and for 63 rows
        int cnt;
        if constexpr (EMAX >= 7 && EMAX <= 15)
            cnt = rw_route2_cols<EMAX>(q, mQ, r, mR, E);
        else
            cnt = rw_route2<EMAX>(q, mQ, r, mR, E, 0xffffffffu);
        a.acc[p] = (uint8_t)(cnt <= E);
        a.obs[p] = cnt;
    }
    if (bad)
        atomicOr(a.status, bad);
}

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
    const int64_t want = (n + 127) / 128;
    const int grid = (int)(want < (int64_t)sm_count * 16
                               ? want
                               : (int64_t)sm_count * 16);
    // a uniform threshold bounds the rows: skip the classes above it
    const int top = E ? kRwMaxE : (e < kRwMaxE ? e : kRwMaxE);
    k_rw_unequal<3, -1><<<grid, 128, 0, st>>>(a);
    if (top > 3)
        k_rw_unequal<7, 3><<<grid, 128, 0, st>>>(a);
    if (top > 7)
        k_rw_unequal<15, 7><<<grid, 128, 0, st>>>(a);
    if (top > 15)
        k_rw_unequal<31, 15><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ssk
