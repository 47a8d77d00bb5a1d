// probe.cu -- FP32 throughput probe for the roofline of the compositing
// kernels (not part of the rendering path).  Every thread runs kChains
// independent fused multiply-add chains, so that each SM sub-partition
// always has a ready FFMA to issue; the rate the caller measures (lane FMAs
// per second) is the SM count x FP32 lanes x clock the part sustains.
#include "../../include/pvg.h"
#include "pvg_internal.cuh"

namespace pvg {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(float *__restrict__ dst, int64_t iters, float a,
                                                             float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = (float)(threadIdx.x + c) * 1e-3f;
#pragma unroll 1
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    dst[blockIdx.x * (size_t)kProbeThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace pvg

extern "C" pvg_status_t pvg_fma_probe(float *dst, int32_t blocks, int64_t iters, float a, float b, void *stream) {
    if (!dst || blocks < 1 || iters < 1) return PVG_ERR_INVALID;
    pvg::note_launch();
    pvg::k_fma_probe<<<blocks, pvg::kProbeThreads, 0, (cudaStream_t)stream>>>(dst, iters, a, b);
    return cudaGetLastError() == cudaSuccess ? PVG_OK : PVG_ERR_CUDA;
}

extern "C" int32_t pvg_device_sm_count(void) { return pvg::device_sm_count(); }
