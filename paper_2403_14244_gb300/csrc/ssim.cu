// The training loss of Sec. 3 with its structural term,
//   L = (1 - lambda) mean |img - target| + lambda (1 - SSIM(img, target)),
// and dL/dimg, in two kernels over 32 x 32 tiles of one channel.
//
// SSIM per channel and pixel q (Wang et al.'s index; the paper names it
// without a definition):
//   S_q = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sxx + syy + C2)),
// where mx, my, E[x^2], E[y^2], E[xy] are window means, sxx = E[x^2] - mx^2,
// syy = E[y^2] - my^2, sxy = E[xy] - mx my, the window is the 11 x 11 Gaussian
// of standard deviation 1.5 normalised to sum 1 (applied as two passes of its
// 1-D factor) with zeros outside the image, C1 = 0.01^2 and C2 = 0.03^2.
//
// Forward: the five window means of a tile (inputs staged with a 5-pixel halo),
// then S and its partials A = dS/dmx, B = dS/dE[x^2], C = dS/dE[xy], written as
// three maps scaled by -lambda / count. Backward: the same window over those maps
// (the window is symmetric, so the adjoint of the zero-padded filter is the
// filter itself) gives dL/dx_p = (1 - lambda) sign(x_p - y_p) / count
// + wA + 2 x_p wB + y_p wC.
#include <cmath>

#include "common.cuh"

namespace igs {
namespace {

constexpr int kWinR = 5;                         // window radius (11 taps)
constexpr int kWinN = 2 * kWinR + 1;
constexpr int kSsimTile = 32;                    // output tile edge
constexpr int kSsimHalo = kSsimTile + 2 * kWinR;  // staged tile edge (42)
constexpr int kSsimThreads = 256;                // 8 warps, 4 output rows each
constexpr int kRowsPerThread = kSsimTile / (kSsimThreads / 32);
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct SsimParams {
    float g[kWinN];    // 1-D window, normalised; the 2-D window is g (x) g
    int width, height;
    float l1_scale;    // (1 - lambda) / count
    float s_scale;     // lambda / count
    float lambda;
    float inv_count;
};

// Packed two-lane FP32 arithmetic of sm_100+ (each lane rounded as its scalar
// _rn counterpart): the filters carry (x, y) or (A, B) pairs through one
// instruction per step.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// Stage a (kSsimHalo x kSsimHalo) window of one channel as elements of type T
// (load(i) gives the element at flat index i), zeros outside the image. Warp w
// stages rows w, w + 8, ..., lanes the columns; every load of a thread is
// issued before the first store.
constexpr int kStageRows = (kSsimHalo + kSsimThreads / 32 - 1) / (kSsimThreads / 32);  // 6
constexpr int kStageCols = (kSsimHalo + 31) / 32;                                     // 2
template <typename T, int LD, typename Load>
__device__ __forceinline__ void stage(Load load, int W, int H, int x0, int y0, T (*dst)[LD]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T v[kStageRows][kStageCols];
#pragma unroll
    for (int i = 0; i < kStageRows; ++i) {
        const int r = w + i * (kSsimThreads / 32), gy = y0 + r;
        const bool row_in = r < kSsimHalo && gy >= 0 && gy < H;
        const size_t row = (size_t)(row_in ? gy : 0) * W;
#pragma unroll
        for (int j = 0; j < kStageCols; ++j) {
            const int c = lane + 32 * j, gx = x0 + c;
            v[i][j] = (row_in && c < kSsimHalo && gx >= 0 && gx < W) ? load(row + gx) : T{};
        }
    }
#pragma unroll
    for (int i = 0; i < kStageRows; ++i) {
        const int r = w + i * (kSsimThreads / 32);
#pragma unroll
        for (int j = 0; j < kStageCols; ++j) {
            const int c = lane + 32 * j;
            if (r < kSsimHalo && c < kSsimHalo) dst[r][c] = v[i][j];
        }
    }
}

// Sum of the two block-wide partials, returned to thread 0.
__device__ __forceinline__ void block_sum2(float a, float b, float (*s_red)[kSsimThreads / 32], float* a_sum,
                                           float* b_sum) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_red[0][threadIdx.x >> 5] = a;
        s_red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float ta = 0.f, tb = 0.f;
        for (int k = 0; k < kSsimThreads / 32; ++k) {
            ta += s_red[0][k];
            tb += s_red[1][k];
        }
        *a_sum = ta;
        *b_sum = tb;
    }
}

// Shared memory of the forward kernel: the staged (x, y) pairs, then the
// horizontally filtered (mx, my), (E[x^2], E[y^2]) pairs and E[xy].
struct SsimFwdSmem {
    float2 p[kSsimHalo][kSsimHalo + 2];
    float2 h_m[kSsimHalo][kSsimTile];
    float2 h_q[kSsimHalo][kSsimTile];
    float h_xy[kSsimHalo][kSsimTile];
    float red[2][kSsimThreads / 32];
};

__global__ void __launch_bounds__(kSsimThreads) k_ssim_fwd(const float* __restrict__ img, const float* __restrict__ target,
                                                          SsimParams P, float2* __restrict__ mAB,
                                                          float* __restrict__ mC, float* __restrict__ loss,
                                                          float* __restrict__ ssim) {
    __shared__ SsimFwdSmem sm;
    const int W = P.width, H = P.height;
    const size_t plane = (size_t)W * H, base = (size_t)blockIdx.z * plane;
    const int tx0 = blockIdx.x * kSsimTile, ty0 = blockIdx.y * kSsimTile;
    {
        const float* a = img + base;
        const float* b = target + base;
        stage(
            [a, b](size_t i) { return make_float2(a[i], b[i]); }, W, H, tx0 - kWinR, ty0 - kWinR, sm.p);
    }
    const int lane = threadIdx.x & 31;
    float2 G[kWinN];  // (g_k, g_k), kept in registers for the packed steps
#pragma unroll
    for (int k = 0; k < kWinN; ++k) G[k] = dup2(P.g[k]);
    __syncthreads();
    // horizontal pass: warp w filters staged rows w, w + 8, ... along x; lane = output column
    for (int r = threadIdx.x >> 5; r < kSsimHalo; r += kSsimThreads / 32) {
        float2 m = make_float2(0.f, 0.f), q = make_float2(0.f, 0.f);
        float xy = 0.f;
#pragma unroll
        for (int k = 0; k < kWinN; ++k) {
            const float2 v = sm.p[r][lane + k];      // (x, y)
            const float2 w = mul2(G[k], v);          // (g x, g y)
            m = add2(m, w);
            q = fma2(w, v, q);
            xy = fmaf(w.x, v.y, xy);
        }
        sm.h_m[r][lane] = m;
        sm.h_q[r][lane] = q;
        sm.h_xy[r][lane] = xy;
    }
    __syncthreads();
    // vertical pass: kRowsPerThread consecutive output rows of column `lane`
    const int r0 = (threadIdx.x >> 5) * kRowsPerThread;
    float2 am[kRowsPerThread], aq[kRowsPerThread];
    float axy[kRowsPerThread];
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
        am[q] = aq[q] = make_float2(0.f, 0.f);
        axy[q] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < kWinN + kRowsPerThread - 1; ++j) {
        const float2 hm = sm.h_m[r0 + j][lane], hq = sm.h_q[r0 + j][lane];
        const float hxy = sm.h_xy[r0 + j][lane];
#pragma unroll
        for (int q = 0; q < kRowsPerThread; ++q) {
            const int k = j - q;
            if (k >= 0 && k < kWinN) {
                am[q] = fma2(G[k], hm, am[q]);
                aq[q] = fma2(G[k], hq, aq[q]);
                axy[q] = fmaf(G[k].x, hxy, axy[q]);
            }
        }
    }
    float part_l1 = 0.f, part_s = 0.f;
    const int px = tx0 + lane;
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
        const int py = ty0 + r0 + q;
        if (px >= W || py >= H) continue;
        const float mx = am[q].x, my = am[q].y;
        const float sxx = aq[q].x - mx * mx, syy = aq[q].y - my * my, sxy = axy[q] - mx * my;
        const float n1 = 2.f * mx * my + kC1, n2 = 2.f * sxy + kC2;
        const float d1 = mx * mx + my * my + kC1, d2 = sxx + syy + kC2;
        const float inv = 1.f / (d1 * d2);
        const float r1 = d2 * inv, r2 = d1 * inv;  // 1 / d1, 1 / d2
        const float S = n1 * n2 * inv;
        // dS/dmx with n1' = 2 my, n2' = -2 my, d1' = 2 mx, d2' = -2 mx (E[.] held)
        const float A = 2.f * my * (n2 - n1) * inv - 2.f * mx * S * (r1 - r2);
        const float B = -S * r2;
        const float Cc = 2.f * n1 * inv;
        const size_t o = base + (size_t)py * W + px;
        mAB[o] = make_float2(-P.s_scale * A, -P.s_scale * B);
        mC[o] = -P.s_scale * Cc;
        const float2 v = sm.p[r0 + q + kWinR][lane + kWinR];
        part_l1 += fabsf(v.x - v.y);
        part_s += S;
    }
    float sum_l1, sum_s;
    block_sum2(part_l1, part_s, sm.red, &sum_l1, &sum_s);
    if (threadIdx.x == 0) {
        const bool first = blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
        atomicAdd(loss, P.l1_scale * sum_l1 - P.s_scale * sum_s + (first ? P.lambda : 0.f));
        if (ssim) atomicAdd(ssim, sum_s * P.inv_count);
    }
}

struct SsimBwdSmem {
    float2 ab[kSsimHalo][kSsimHalo + 2];
    float c[kSsimHalo][kSsimHalo + 1];
    float2 h_ab[kSsimHalo][kSsimTile];
    float h_c[kSsimHalo][kSsimTile];
};

__global__ void __launch_bounds__(kSsimThreads) k_ssim_bwd(const float* __restrict__ img, const float* __restrict__ target,
                                                          const float2* __restrict__ mAB, const float* __restrict__ mC,
                                                          SsimParams P, float* __restrict__ grad) {
    __shared__ SsimBwdSmem sm;
    const int W = P.width, H = P.height;
    const size_t plane = (size_t)W * H, base = (size_t)blockIdx.z * plane;
    const int tx0 = blockIdx.x * kSsimTile, ty0 = blockIdx.y * kSsimTile;
    const int lane = threadIdx.x & 31;
    {
        const float2* ab = mAB + base;
        const float* c = mC + base;
        stage([ab](size_t i) { return ab[i]; }, W, H, tx0 - kWinR, ty0 - kWinR, sm.ab);
        stage([c](size_t i) { return c[i]; }, W, H, tx0 - kWinR, ty0 - kWinR, sm.c);
    }
    float2 G[kWinN];
#pragma unroll
    for (int k = 0; k < kWinN; ++k) G[k] = dup2(P.g[k]);
    __syncthreads();
    for (int r = threadIdx.x >> 5; r < kSsimHalo; r += kSsimThreads / 32) {
        float2 ab = make_float2(0.f, 0.f);
        float c = 0.f;
#pragma unroll
        for (int k = 0; k < kWinN; ++k) {
            ab = fma2(G[k], sm.ab[r][lane + k], ab);
            c = fmaf(G[k].x, sm.c[r][lane + k], c);
        }
        sm.h_ab[r][lane] = ab;
        sm.h_c[r][lane] = c;
    }
    __syncthreads();
    const int r0 = (threadIdx.x >> 5) * kRowsPerThread;
    float2 aab[kRowsPerThread];
    float ac[kRowsPerThread];
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
        aab[q] = make_float2(0.f, 0.f);
        ac[q] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < kWinN + kRowsPerThread - 1; ++j) {
        const float2 hab = sm.h_ab[r0 + j][lane];
        const float hc = sm.h_c[r0 + j][lane];
#pragma unroll
        for (int q = 0; q < kRowsPerThread; ++q) {
            const int k = j - q;
            if (k >= 0 && k < kWinN) {
                aab[q] = fma2(G[k], hab, aab[q]);
                ac[q] = fmaf(G[k].x, hc, ac[q]);
            }
        }
    }
    const int px = tx0 + lane;
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
        const int py = ty0 + r0 + q;
        if (px >= W || py >= H) continue;
        const size_t o = base + (size_t)py * W + px;
        const float x = img[o], y = target[o], d = x - y;
        const float l1 = d > 0.f ? P.l1_scale : (d < 0.f ? -P.l1_scale : 0.f);
        grad[o] = l1 + aab[q].x + 2.f * x * aab[q].y + y * ac[q];
    }
}

}  // namespace

size_t ssim_work_floats(int channels, int height, int width) { return 3 * (size_t)channels * height * width; }

cudaError_t launch_l1_ssim(const float* img, const float* target, int channels, int height, int width, float lambda,
                           float* loss, float* ssim, float* grad, float* work, cudaStream_t st) {
    SsimParams P;
    double g[kWinN], sum = 0.0;
    for (int k = 0; k < kWinN; ++k) {
        const double d = (double)(k - kWinR);
        g[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        sum += g[k];
    }
    for (int k = 0; k < kWinN; ++k) P.g[k] = (float)(g[k] / sum);
    const double count = (double)channels * height * width;
    P.width = width;
    P.height = height;
    P.l1_scale = (float)((1.0 - lambda) / count);
    P.s_scale = (float)(lambda / count);
    P.lambda = lambda;
    P.inv_count = (float)(1.0 / count);
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e == cudaSuccess && ssim) e = cudaMemsetAsync(ssim, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    const size_t count_e = (size_t)channels * height * width;
    float2* mAB = reinterpret_cast<float2*>(work);  // (A, B) pairs, then C
    float* mC = work + 2 * count_e;
    const dim3 grid((unsigned)ceil_div(width, kSsimTile), (unsigned)ceil_div(height, kSsimTile), (unsigned)channels);
    k_ssim_fwd<<<grid, kSsimThreads, 0, st>>>(img, target, P, mAB, mC, loss, ssim);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ssim_bwd<<<grid, kSsimThreads, 0, st>>>(img, target, mAB, mC, P, grad);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace igs
