// Per-tile front-to-back compositing (Eq. 4), shared by the one-view forward
// kernel (blend.cu) and the persistent multi-view kernel (batch.cu), so both
// produce bit-identical pixels. Internal to libigs.
#pragma once

#include "common.cuh"

namespace igs {
namespace {

struct Alpha {
    float alpha, g, og, d2, dx, dy;
};

// The alpha of one (pixel, entry) pair, written with explicit roundings so the
// forward and backward kernels take exactly the same skip / stop / clamp decisions.
__device__ __forceinline__ Alpha eval_alpha(float px, float py, float4 a, float alpha_max) {
    Alpha r;
    r.dx = __fsub_rn(px, a.x);
    r.dy = __fsub_rn(py, a.y);
    r.d2 = __fmaf_rn(r.dx, r.dx, __fmul_rn(r.dy, r.dy));
    r.g = fast_exp2(-__fmul_rn(a.z, r.d2));
    r.og = __fmul_rn(a.w, r.g);
    r.alpha = fminf(alpha_max, r.og);
    return r;
}

// One CTA of TS*TS threads composites one tile (one thread per pixel), staging
// B entries at a time in shared memory (s_a, s_c hold B float4 each), and leaves
// the batch loop once every pixel has stopped. Writes img (planar, `plane`
// floats per channel, row stride `width`) and, if given, T_final / n_contrib.
template <int TS, int B>
__device__ __forceinline__ void blend_tile_fwd(int tx, int ty, int width, int height, uint2 rg,
                                               const uint32_t* __restrict__ vals, const float4* __restrict__ rec,
                                               float alpha_min, float alpha_max, float t_min, const float* bg,
                                               float4* s_a, float4* s_c, float* __restrict__ img,
                                               float* __restrict__ T_final, uint32_t* __restrict__ n_contrib) {
    constexpr int NT = TS * TS;
    static_assert(B <= NT, "staging batch larger than the tile");
    const int x = tx * TS + (threadIdx.x % TS), y = ty * TS + (threadIdx.x / TS);
    const bool inside = x < width && y < height;
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    for (uint32_t b0 = rg.x; b0 < rg.y; b0 += B) {
        if (__syncthreads_count(done) == NT) break;
        const uint32_t j = b0 + threadIdx.x;
        if (threadIdx.x < B && j < rg.y) {
            const uint32_t g = vals[j];
            s_a[threadIdx.x] = rec[2 * g];
            s_c[threadIdx.x] = rec[2 * g + 1];
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)B, rg.y - b0);
        for (int k = 0; k < nb && !done; ++k) {
            const Alpha a = eval_alpha(px, py, s_a[k], alpha_max);
            if (a.alpha < alpha_min) continue;
            const float Tn = T * (1.f - a.alpha);
            if (Tn < t_min) {
                done = true;
                break;
            }
            const float4 c = s_c[k];
            const float w = a.alpha * T;
            C0 = fmaf(c.x, w, C0);
            C1 = fmaf(c.y, w, C1);
            C2 = fmaf(c.z, w, C2);
            T = Tn;
            last = b0 - rg.x + k + 1;
        }
    }
    if (!inside) return;
    const size_t pix = (size_t)y * width + x, plane = (size_t)width * height;
    img[pix] = fmaf(T, bg[0], C0);
    img[plane + pix] = fmaf(T, bg[1], C1);
    img[2 * plane + pix] = fmaf(T, bg[2], C2);
    if (T_final) T_final[pix] = T;
    if (n_contrib) n_contrib[pix] = last;
}

}  // namespace
}  // namespace igs
