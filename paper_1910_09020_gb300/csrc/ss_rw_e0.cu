// ss_rw_e0.cu -- instantiations of K3a for E = 0..9 (split across
// translation units so that they compile in parallel).
#include "ss_rw_launch.cuh"

namespace ssk {

cudaError_t launch_rw_uniform_e0(int E, const RwLaunch &L, cudaStream_t st)
{
    return rw_launch_range<0>(E, L, st,
                                 std::make_integer_sequence<int, 10>{});
}

cudaError_t rw_init_e0()
{
    return rw_init_range<0>(std::make_integer_sequence<int, 10>{});
}

}  // namespace ssk
