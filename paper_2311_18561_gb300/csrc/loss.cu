// loss.cu -- L1 photometric loss and its gradient (the L1 term of the
// objective, Sec. 3.4), so that a training step needs no kernel outside
// this library: loss = scale * sum |pred - target|,
// dl = scale * sign(pred - target).
//
// The sum is taken in a fixed order, so the loss is the same bit for bit
// on every run with the same inputs on the same device: a fixed grid of
// blocks (a multiple of the SM count) walks the elements with a fixed
// stride, each block reduces its threads in a fixed pattern into one
// partial sum, and the last block to finish adds the partial sums in block
// order.  Nothing waits on another block.
#include "../../include/pvg.h"
#include "pvg_internal.cuh"

namespace pvg {
namespace {

constexpr int kL1Threads = 256;
constexpr int kL1BlocksPerSm = 8;
constexpr size_t kL1PartialsOffset = 16;  // bytes: the ticket counter comes first

__device__ __forceinline__ float block_sum(float v, float *warp_sum) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = v;
    __syncthreads();
    float b = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < kL1Threads / 32; w++) b += warp_sum[w];
    return b;  // valid in thread 0
}

__global__ void __launch_bounds__(kL1Threads) k_l1(const float *__restrict__ pred, const float *__restrict__ tgt,
                                                   size_t n, float scale, float *__restrict__ dl,
                                                   unsigned int *ticket, float *partials, float *loss) {
    pdl_enter();
    __shared__ float warp_sum[kL1Threads / 32];
    __shared__ bool is_last;
    float acc = 0.f;
    auto sgn = [scale](float d) { return d > 0.f ? scale : (d < 0.f ? -scale : 0.f); };
    const size_t stride = (size_t)gridDim.x * kL1Threads;
    size_t head = 0;  // elements before it are taken four at a time
    if ((((uintptr_t)pred | (uintptr_t)tgt | (uintptr_t)dl) & 15u) == 0) {
        // 16-byte aligned arrays: float4 loads and stores, the same sum
        // order on every run (a fixed stride over fixed groups of four)
        head = n & ~(size_t)3;
        const float4 *p4 = reinterpret_cast<const float4 *>(pred);
        const float4 *t4 = reinterpret_cast<const float4 *>(tgt);
        float4 *d4 = reinterpret_cast<float4 *>(dl);
        for (size_t i = blockIdx.x * (size_t)kL1Threads + threadIdx.x; i < head / 4; i += stride) {
            const float4 a = p4[i], b = t4[i];
            const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
            acc += fabsf(d.x) + fabsf(d.y) + fabsf(d.z) + fabsf(d.w);
            if (dl) d4[i] = make_float4(sgn(d.x), sgn(d.y), sgn(d.z), sgn(d.w));
        }
    }
    for (size_t i = head + blockIdx.x * (size_t)kL1Threads + threadIdx.x; i < n; i += stride) {
        const float d = pred[i] - tgt[i];
        acc += fabsf(d);
        if (dl) dl[i] = sgn(d);
    }
    const float b = block_sum(acc, warp_sum);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b;
        __threadfence();
        is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    // the last block: every other block's partial is visible
    __threadfence();
    float s = 0.f;
    for (unsigned int k = threadIdx.x; k < gridDim.x; k += kL1Threads) s += ((volatile float *)partials)[k];
    __syncthreads();  // warp_sum is reused
    const float total = block_sum(s, warp_sum);
    if (threadIdx.x == 0) {
        *loss = total * scale;
        *ticket = 0u;  // ready for the next call
    }
}

unsigned l1_blocks(int64_t n) {
    size_t blocks = ((size_t)n + kL1Threads - 1) / kL1Threads;
    const size_t cap = (size_t)kL1BlocksPerSm * device_sm_count();
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1u : (unsigned)blocks;
}

}  // namespace

size_t l1_loss_scratch_bytes() { return kL1PartialsOffset + sizeof(float) * kL1BlocksPerSm * device_sm_count(); }

cudaError_t launch_l1_loss(const float *pred, const float *target, int64_t n, float scale, float *dl, float *loss,
                           void *scratch, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(loss, 0, sizeof(float), s);
    unsigned int *ticket = (unsigned int *)scratch;
    float *partials = (float *)((char *)scratch + kL1PartialsOffset);
    note_launch();
    pdl_launch(k_l1, l1_blocks(n), kL1Threads, 0, s, pred, target, (size_t)n, scale, dl, ticket, partials, loss);
    return cudaGetLastError();
}

}  // namespace pvg
