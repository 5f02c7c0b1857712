// ss_rw_e3.cu -- instantiations of K3a for E = 25..31 (split across
// translation units so that they compile in parallel).
#include "ss_rw_launch.cuh"

namespace ssk {

cudaError_t launch_rw_uniform_e3(int E, const RwLaunch &L, cudaStream_t st)
{
    return rw_launch_range<25>(E, L, st,
                                 std::make_integer_sequence<int, 7>{});
}

cudaError_t rw_init_e3()
{
    return rw_init_range<25>(std::make_integer_sequence<int, 7>{});
}

}  // namespace ssk
