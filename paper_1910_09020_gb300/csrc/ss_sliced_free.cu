// ss_sliced_free.cu -- pairs whose read and reference differ in length over
// the bit-sliced layout (reads of m bases, references of m_ref, uniform
// per batch): the walk of ss_sliced.cuh over the reference's m_ref columns
// with Section 2.4's correction -- the leading and trailing cells where a
// diagonal reads no base of the read are free, not obstacles
// (k_sliced_seg<E, true> in ss_sliced_seg.cuh).  Up to kSlicedMaxSegments
// batches of one threshold per launch.
#include "ss_sliced_seg.cuh"

namespace ssk {

cudaError_t launch_sliced_free_segments(const SlicedSegment *segs, int nseg,
                                        int32_t E, cudaStream_t st)
{
    return sliced_seg_launch<true>(segs, nseg, E, st);
}

}  // namespace ssk
