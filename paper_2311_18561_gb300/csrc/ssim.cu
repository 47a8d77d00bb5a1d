// ssim.cu -- the photometric loss of the objective (Sec. 3.4),
//   L = (1 - lambda_r) L1 + lambda_r (1 - SSIM),
// and dL/dpred in one fused pass, so a training step with the paper's RGB
// supervision needs no kernel outside this library.
//
// SSIM follows 3D Gaussian Splatting, whose losses the paper reuses: per
// channel, an 11 x 11 Gaussian window (sigma 1.5, normalised) applied with
// zero padding, C1 = 0.01^2, C2 = 0.03^2, averaged over channels and
// pixels; L1 is the mean absolute difference (sign(0) = 0).
//
// One CTA per 32 x 32 output tile and channel.  The window is separable
// and symmetric, so the gradient of SSIM is itself a windowed sum:
//   dSSIM/dx_p = sum_q G(q - p) [a_q + 2 x_p b_q + y_p c_q],
// a, b, c the derivatives of S_q with respect to the windowed moments
// G*x, G*x^2, G*xy.  The CTA stages x and y with a 10-pixel halo in
// shared memory, computes the five moments (row pass, then column pass) on
// the tile plus a 5-pixel halo, turns them into S, a, b, c (zero outside
// the image), filters a, b, c the same way and writes the gradient of its
// 32 x 32 pixels.  HBM traffic is one read of both images and one write of
// the gradient; the per-CTA sums of S and |x - y| go to a partial array
// that one small kernel adds in a fixed order (the loss is deterministic).
#include "pvg_internal.cuh"

namespace pvg {
namespace {

constexpr int kT = 32;               // output tile
constexpr int kR = 5;                // window radius
constexpr int kA = kT + 2 * kR;      // S / a / b / c region (42)
constexpr int kX = kT + 4 * kR;      // staged input region (52)
constexpr int kThreads = 384;  // one round of the largest pass (364 strips)
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// shared layout, in floats.  The staged inputs are dead after the first
// row pass, so a, b, c take their place (the gradient pass reads x and y
// of its own pixels from global memory again, where they are L2 hits):
// 65 KB per CTA, three CTAs per SM.
constexpr int kOffX = 0, kOffY = kX * kX;
constexpr int kOffABC = 0;                         // [3][kA][kA] over the inputs
static_assert(3 * kA * kA <= 2 * kX * kX, "a, b, c fit where the inputs were");
constexpr int kOffH = 2 * kX * kX;                 // 5 row-filtered moments [5][kX][kA]
constexpr int kOffH2 = kOffH;                      // row-filtered a, b, c [3][kA][kT] (reuses the moments)
constexpr int kOffG = kOffH + 5 * kX * kA;         // 11 window taps
constexpr int kOffRed = kOffG + 12;                // 2 x 16 warp partials
constexpr int kSmemFloats = kOffRed + 32;

__global__ void __launch_bounds__(kThreads, 3) k_rgb_loss(const float *__restrict__ pred,
                                                       const float *__restrict__ tgt, int H, int W,
                                                       float lambda_r, float inv_n, float *__restrict__ dl,
                                                       float2 *__restrict__ partial) {
    pdl_enter();
    extern __shared__ float sm[];
    float *sx = sm + kOffX, *sy = sm + kOffY, *hm = sm + kOffH, *abc = sm + kOffABC, *h2 = sm + kOffH2;
    float *g = sm + kOffG, *red = sm + kOffRed;
    const int tid = threadIdx.x;
    const size_t plane = (size_t)H * W;
    const float *X = pred + blockIdx.z * plane, *Y = tgt + blockIdx.z * plane;
    const int tx0 = blockIdx.x * kT, ty0 = blockIdx.y * kT;
    if (tid < 11) {
        float s = 0.f;
        for (int j = 0; j < 11; j++) s += expf(-(float)((j - kR) * (j - kR)) / (2.0f * 1.5f * 1.5f));
        g[tid] = expf(-(float)((tid - kR) * (tid - kR)) / (2.0f * 1.5f * 1.5f)) / s;
    }
    // inputs with a 2R halo, zero outside the image
    for (int k = tid; k < kX * kX; k += kThreads) {
        const int r = k / kX, c = k % kX, gy = ty0 - 2 * kR + r, gx = tx0 - 2 * kR + c;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        sx[k] = in ? X[(size_t)gy * W + gx] : 0.f;
        sy[k] = in ? Y[(size_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    float gw[11];  // the taps, in registers
#pragma unroll
    for (int j = 0; j < 11; j++) gw[j] = g[j];
    // Each pass is register-blocked: a thread filters a strip of outputs
    // along the pass direction from one run of staged values, so a value is
    // read from shared memory once per strip instead of once per tap.
    //
    // row pass of the five moments: every staged row, strips of 6 columns
    // of the 42-wide S region (7 per row)
    for (int k = tid; k < kX * 7; k += kThreads) {
        const int r = k / 7, c0 = (k % 7) * 6;
        float xa[16], ya[16];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            xa[j] = sx[r * kX + c0 + j];
            ya[j] = sy[r * kX + c0 + j];
        }
        float m[5][6];
#pragma unroll
        for (int o = 0; o < 6; o++) {
            float mx = 0.f, my = 0.f, mxx = 0.f, myy = 0.f, mxy = 0.f;
#pragma unroll
            for (int j = 0; j < 11; j++) {
                const float a = xa[o + j], b = ya[o + j], w = gw[j];
                mx = fmaf(w, a, mx);
                my = fmaf(w, b, my);
                mxx = fmaf(w, a * a, mxx);
                myy = fmaf(w, b * b, myy);
                mxy = fmaf(w, a * b, mxy);
            }
            m[0][o] = mx; m[1][o] = my; m[2][o] = mxx; m[3][o] = myy; m[4][o] = mxy;
        }
#pragma unroll
        for (int q = 0; q < 5; q++)
#pragma unroll
            for (int o = 0; o < 6; o++) hm[q * kX * kA + r * kA + c0 + o] = m[q][o];
    }
    __syncthreads();
    // column pass -> S and its moment derivatives a, b, c on the tile + R
    // halo: every column, strips of 6 rows (7 per column).  The row pass
    // was the inputs' last reader (barrier above), so a, b, c are written
    // over them.
    float ssum = 0.f, l1sum = 0.f;
    for (int k = tid; k < kA * 7; k += kThreads) {
        const int c = k % kA, r0 = (k / kA) * 6;
        float m[5][6];
#pragma unroll
        for (int q = 0; q < 5; q++) {
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; i++) v[i] = hm[q * kX * kA + (r0 + i) * kA + c];
#pragma unroll
            for (int o = 0; o < 6; o++) {
                float acc = 0.f;
#pragma unroll
                for (int i = 0; i < 11; i++) acc = fmaf(gw[i], v[o + i], acc);
                m[q][o] = acc;
            }
        }
        const int gx = tx0 - kR + c;
#pragma unroll
        for (int o = 0; o < 6; o++) {
            const int r = r0 + o, gy = ty0 - kR + r;
            float a = 0.f, b = 0.f, cc = 0.f;
            if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
                const float mx = m[0][o], my = m[1][o];
                const float vx = fmaf(-mx, mx, m[2][o]), vy = fmaf(-my, my, m[3][o]);
                const float cxy = fmaf(-mx, my, m[4][o]);
                const float A1 = fmaf(2.f * mx, my, kC1), A2 = fmaf(2.f, cxy, kC2);
                const float B1 = fmaf(mx, mx, fmaf(my, my, kC1)), B2 = vx + vy + kC2;
                // SFU reciprocals (within 2 ulp)
                const float iA1 = __fdividef(1.f, A1), iA2 = __fdividef(1.f, A2);
                const float iB1 = __fdividef(1.f, B1), iB2 = __fdividef(1.f, B2);
                const float S = A1 * A2 * iB1 * iB2;
                const float dmu = 2.f * S * fmaf(my, iA1, -mx * iB1);
                const float dvx = -S * iB2, dcxy = 2.f * S * iA2;
                a = fmaf(-2.f * mx, dvx, fmaf(-my, dcxy, dmu));
                b = dvx;
                cc = dcxy;
                if (r >= kR && r < kR + kT && c >= kR && c < kR + kT) ssum += S;
            }
            abc[0 * kA * kA + r * kA + c] = a;
            abc[1 * kA * kA + r * kA + c] = b;
            abc[2 * kA * kA + r * kA + c] = cc;
        }
    }
    __syncthreads();
    // row pass of a, b, c (into the moments' space, no longer needed):
    // every row of the S region, strips of 8 of the 32 tile columns
    for (int k = tid; k < kA * 4; k += kThreads) {
        const int r = k / 4, c0 = (k % 4) * 8;
#pragma unroll
        for (int t = 0; t < 3; t++) {
            float v[18];
#pragma unroll
            for (int j = 0; j < 18; j++) v[j] = abc[t * kA * kA + r * kA + c0 + j];
#pragma unroll
            for (int o = 0; o < 8; o++) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < 11; j++) acc = fmaf(gw[j], v[o + j], acc);
                h2[t * kA * kT + r * kT + c0 + o] = acc;
            }
        }
    }
    __syncthreads();
    // column pass and the gradient of the tile's pixels (strips of 4 rows),
    // and the L1 term of those pixels (x, y again from global memory)
    {
        const float kl1 = (1.0f - lambda_r) * inv_n, kss = lambda_r * inv_n;
        float *D = dl ? dl + blockIdx.z * plane : nullptr;
        for (int k = tid; k < kT * 8; k += kThreads) {
            const int c = k % kT, r0 = (k / kT) * 4, gx = tx0 + c;
            float q[3][4];
            if (D) {
#pragma unroll
                for (int t = 0; t < 3; t++) {
                    float v[14];
#pragma unroll
                    for (int i = 0; i < 14; i++) v[i] = h2[t * kA * kT + (r0 + i) * kT + c];
#pragma unroll
                    for (int o = 0; o < 4; o++) {
                        float acc = 0.f;
#pragma unroll
                        for (int i = 0; i < 11; i++) acc = fmaf(gw[i], v[o + i], acc);
                        q[t][o] = acc;
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < 4; o++) {
                const int r = r0 + o, gy = ty0 + r;
                if (gx >= W || gy >= H) continue;
                const float x = X[(size_t)gy * W + gx], y = Y[(size_t)gy * W + gx], d = x - y;
                l1sum += fabsf(d);
                if (D) {
                    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                    const float dssim = q[0][o] + 2.f * x * q[1][o] + y * q[2][o];
                    D[(size_t)gy * W + gx] = kl1 * sgn - kss * dssim;
                }
            }
        }
    }
    // per-CTA sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
        l1sum += __shfl_xor_sync(0xffffffffu, l1sum, o);
    }
    if ((tid & 31) == 0) {
        red[tid >> 5] = ssum;
        red[16 + (tid >> 5)] = l1sum;
    }
    __syncthreads();
    if (tid == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < kThreads / 32; w++) {
            a += red[w];
            b += red[16 + w];
        }
        partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = make_float2(a, b);
    }
}

// loss[0..2] = (L, L1, SSIM) from the per-CTA partial sums, added in a
// fixed order in double precision
__global__ void __launch_bounds__(1024) k_rgb_loss_finish(const float2 *__restrict__ partial, int n,
                                                          double inv_n, float lambda_r, float *loss) {
    pdl_enter();
    __shared__ double ss[1024], sl[1024];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += (double)partial[i].x;
        b += (double)partial[i].y;
    }
    ss[threadIdx.x] = a;
    sl[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            ss[threadIdx.x] += ss[threadIdx.x + s];
            sl[threadIdx.x] += sl[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double ssim = ss[0] * inv_n, l1 = sl[0] * inv_n;
        loss[0] = (float)((1.0 - lambda_r) * l1 + lambda_r * (1.0 - ssim));
        loss[1] = (float)l1;
        loss[2] = (float)ssim;
    }
}

}  // namespace

size_t rgb_loss_partials(int channels, int height, int width) {
    return (size_t)channels * ((height + kT - 1) / kT) * ((width + kT - 1) / kT);
}

cudaError_t launch_rgb_loss(const float *pred, const float *target, int channels, int height, int width,
                            float lambda_r, float *dl, float *loss, void *partials, cudaStream_t s) {
    const size_t smem = sizeof(float) * kSmemFloats;
    static_assert(sizeof(float) * kSmemFloats <= 227 * 1024, "shared memory of the loss kernel");
    cudaError_t e = cudaFuncSetAttribute(k_rgb_loss, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((width + kT - 1) / kT, (height + kT - 1) / kT, channels);
    const double n = (double)channels * height * width;
    note_launch();
    pdl_launch(k_rgb_loss, grid, kThreads, smem, s, pred, target, height, width, lambda_r, (float)(1.0 / n), dl,
                                            reinterpret_cast<float2 *>(partials));
    note_launch();
    pdl_launch(k_rgb_loss_finish, 1, 1024, 0, s, reinterpret_cast<const float2 *>(partials),
                                         (int)rgb_loss_partials(channels, height, width), 1.0 / n, lambda_r, loss);
    return cudaGetLastError();
}

}  // namespace pvg
