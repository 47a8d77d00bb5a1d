// loss.cu -- L1 photometric loss and its gradient (the L1 term of the
// objective, Sec. 3.4), so that a training step needs no kernel outside
// this library: loss = scale * sum |pred - target|,
// dl = scale * sign(pred - target).
#include "../../include/pvg.h"
#include "pvg_internal.cuh"

namespace pvg {
namespace {

__global__ void __launch_bounds__(256) k_l1(const float *__restrict__ pred, const float *__restrict__ tgt,
                                            size_t n, float scale, float *__restrict__ dl, float *loss) {
    __shared__ float warp_sum[8];
    float acc = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = pred[i] - tgt[i];
        acc += fabsf(d);
        if (dl) dl[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < 8; w++) b += warp_sum[w];
        atomicAdd(loss, b * scale);
    }
}

}  // namespace
}  // namespace pvg

extern "C" pvg_status_t pvg_l1_loss(const float *pred, const float *target, int64_t n, float scale, float *dl,
                                    float *loss, void *stream) {
    if (!pred || !target || !loss || n < 0) return PVG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return PVG_ERR_CUDA;
    if (n == 0) return PVG_OK;
    size_t blocks = ((size_t)n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    pvg::note_launch();
    pvg::k_l1<<<(unsigned)blocks, 256, 0, s>>>(pred, target, (size_t)n, scale, dl, loss);
    return cudaGetLastError() == cudaSuccess ? PVG_OK : PVG_ERR_CUDA;
}
