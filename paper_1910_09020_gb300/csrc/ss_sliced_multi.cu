// ss_sliced_multi.cu -- the plain launch over several batches of one
// threshold, reads and references of one length per batch (k_sliced_seg in
// ss_sliced_seg.cuh): a batch mixing lengths, bucketed into uniform
// segments, in one launch per threshold.
#include "ss_sliced_seg.cuh"

namespace ssk {

cudaError_t launch_sliced_segments(const SlicedSegment *segs, int nseg,
                                   int32_t E, cudaStream_t st)
{
    if (nseg == 1)
        return launch_sliced(segs[0].reads, segs[0].refs, segs[0].n,
                             segs[0].m, E, segs[0].acc, segs[0].obs, st);
    return sliced_seg_launch<false>(segs, nseg, E, st);
}

}  // namespace ssk
