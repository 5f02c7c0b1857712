// ss_rw_e1.cu -- instantiations of K3a for E = 10..17 (split across
// translation units so that they compile in parallel).
#include "ss_rw_launch.cuh"

namespace ssk {

cudaError_t launch_rw_uniform_e1(int E, const RwLaunch &L, cudaStream_t st)
{
    return rw_launch_range<10>(E, L, st,
                                 std::make_integer_sequence<int, 8>{});
}

cudaError_t rw_init_e1()
{
    return rw_init_range<10>(std::make_integer_sequence<int, 8>{});
}

}  // namespace ssk
