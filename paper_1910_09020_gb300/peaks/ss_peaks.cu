// ss_peaks.cu -- throughput microbenchmarks of the integer pipes the filter
// uses (logic, add, funnel shift, find-first), measured on the device the
// filter runs on.  They give the ALU denominator of the filter's roofline
// the way a STREAM copy gives the HBM one.  Measurement code only: not part
// of the filter library.
//
// Each thread runs 8 independent dependency chains of one instruction kind
// (inline PTX, so the compiler cannot fold or fuse the chain); with many
// resident warps the chains are throughput-bound.
#include <cuda_runtime.h>
#include <cstdint>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <int KIND>
__global__ void __launch_bounds__(512) k_peak(uint32_t *out, int iters,
                                              uint32_t seed)
{
    uint32_t r[kChains];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t b = seed * 2654435761u + tid;
    const uint32_t c = (seed ^ tid) | 1u;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        r[j] = tid * (j + 3) + seed;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) {
                if (KIND == 0)  // 3-input logic op (LOP3)
                    asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;"
                                 : "+r"(r[j]) : "r"(b), "r"(c));
                else if (KIND == 1)  // integer add
                    asm volatile("add.u32 %0, %0, %1;" : "+r"(r[j]) : "r"(b));
                else if (KIND == 2)  // funnel shift
                    asm volatile("shf.r.wrap.b32 %0, %0, %1, %2;"
                                 : "+r"(r[j]) : "r"(b), "r"(c));
                else  // find leading one (count-leading-zeros class)
                    asm volatile("bfind.u32 %0, %0;" : "+r"(r[j]));
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        acc ^= r[j];
    if (acc == 0x9e3779b9u)
        out[0] = acc;  // practically never: keeps the chains alive
}

}  // namespace

extern "C" {

// kind: 0 = lop3, 1 = add, 2 = funnel shift, 3 = bfind.  Writes the measured
// rate in warp-lane operations per second and the kernel time.  Returns 0 on
// success, else a CUDA error code.
int ss_peak_int(int device, int kind, double *ops_per_s, double *ms)
{
    if (cudaSetDevice(device) != cudaSuccess)
        return 1;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess)
        return 2;
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, 4) != cudaSuccess)
        return 3;
    const int threads = 512;
    const int blocks = p.multiProcessorCount * 4;
    const int iters = kind == 3 ? 256 : 1024;
    cudaEvent_t a, z;
    cudaEventCreate(&a);
    cudaEventCreate(&z);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a);
        switch (kind) {
        case 0: k_peak<0><<<blocks, threads>>>(out, iters, rep + 1); break;
        case 1: k_peak<1><<<blocks, threads>>>(out, iters, rep + 1); break;
        case 2: k_peak<2><<<blocks, threads>>>(out, iters, rep + 1); break;
        default: k_peak<3><<<blocks, threads>>>(out, iters, rep + 1); break;
        }
        cudaEventRecord(z);
        cudaEventSynchronize(z);
        float t = 0;
        cudaEventElapsedTime(&t, a, z);
        if (rep > 0 && t < best)
            best = t;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    cudaFree(out);
    if (err != cudaSuccess)
        return (int)err;
    const double ops =
        (double)blocks * threads * iters * kUnroll * kChains;
    *ops_per_s = ops / (best * 1e-3);
    *ms = best;
    return 0;
}

}  // extern "C"
