// ss_unequal_x0.cu -- exact-threshold instantiations of the tile kernel
// for pairs of different lengths, E = 0..15 (split across
// translation units so that they compile in parallel).
#include "ss_unequal_tile.cuh"

namespace ssk {

cudaError_t launch_unequal_exact_x0(int e, const UnequalArgs &a,
                                    unsigned grid, cudaStream_t st)
{
    return unequal_exact_range<0>(e, a, grid, st,
                                    std::make_integer_sequence<int, 16>{});
}

}  // namespace ssk
