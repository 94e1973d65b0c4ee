// probe.cu -- the FP32 FMA throughput of the device, measured by a kernel of its own: the
// ceiling of the plain-FP32 contraction (CUDA cores, one FFMA per multiply-add).
//
// Every thread runs 8 independent chains x <- x * a + b for `iters` steps (8 FMAs in
// flight per thread hide the FMA latency at 8 or more warps per SM); the chains' sum is
// stored so that none of the work can be dropped.  The values stay finite: |a| < 1.
#include "mtk_internal.cuh"

namespace mtk {
namespace {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) ffma_probe_kernel(float* out, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t launch_ffma_probe(int blocks, int iters, float* out, cudaStream_t s) {
    ffma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(out, iters, 0.999f, 1e-4f);
    note_launches(1);
    return cudaGetLastError();
}

int ffma_probe_threads() { return kProbeThreads; }

}  // namespace mtk
