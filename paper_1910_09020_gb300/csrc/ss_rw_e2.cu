// ss_rw_e2.cu -- instantiations of K3a for E = 18..24 (split across
// translation units so that they compile in parallel).
#include "ss_rw_launch.cuh"

namespace ssk {

cudaError_t launch_rw_uniform_e2(int E, const RwLaunch &L, cudaStream_t st)
{
    return rw_launch_range<18>(E, L, st,
                                 std::make_integer_sequence<int, 7>{});
}

cudaError_t rw_init_e2()
{
    return rw_init_range<18>(std::make_integer_sequence<int, 7>{});
}

}  // namespace ssk
