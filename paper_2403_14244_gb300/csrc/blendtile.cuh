// Per-tile front-to-back compositing (Eq. 4), shared by the one-view forward
// kernel (blend.cu) and the persistent multi-view kernel (batch.cu), so both
// produce bit-identical pixels. Internal to libigs.
#pragma once

#include "common.cuh"

namespace igs {
namespace {

// A record's first float4 is (u, v, w2, pmax), its second (r, g, b, o); the
// exponent of a pixel is w2 d^2 and pmax = log2(o / alpha_min) + margin bounds
// it: a larger exponent gives alpha < alpha_min.
struct Dist {
    float dx, dy, d2, pw;
};

// Squared distance and exponent of one (pixel, entry) pair, each step rounded
// once in a fixed order, so that forward and backward take the same decisions.
__device__ __forceinline__ Dist eval_dist(float px, float py, float4 a) {
    Dist r;
    r.dx = __fsub_rn(px, a.x);
    r.dy = __fsub_rn(py, a.y);
    r.d2 = __fmaf_rn(r.dx, r.dx, __fmul_rn(r.dy, r.dy));
    r.pw = __fmul_rn(a.z, r.d2);
    return r;
}

// Whether the entry can reach a pixel centre in [xlo, xhi] x [ylo, yhi] (first
// and last centres of a block of rows): the exponent test at the centre nearest
// to (u, v). Each rounded step of eval_dist is monotone in |dx| and |dy|, so that
// centre has the smallest exponent of the block and a false answer never drops
// a pair that the per-pixel test would keep.
__device__ __forceinline__ bool may_reach(float4 a, float xlo, float xhi, float ylo, float yhi) {
    const float cx = fminf(fmaxf(floorf(a.x) + 0.5f, xlo), xhi);
    const float cy = fminf(fmaxf(floorf(a.y) + 0.5f, ylo), yhi);
    return !(eval_dist(cx, cy, a).pw > a.w);
}

// One CTA of TS*TS threads composites one tile (one thread per pixel), staging
// B entries at a time in shared memory (s_a, s_c hold B float4 each), and leaves
// the batch loop once every pixel has stopped. Each warp owns an 8 x 4 block of
// the tile (compact blocks are reached by fewer entries than whole rows, and
// their pixels stop at similar depths) and walks, in order, only the staged
// entries that may reach it (one ballot per 32 entries). Writes img (planar,
// `plane` floats per channel, row stride `width`) and, if given, T_final /
// n_contrib.
template <int TS, int B>
__device__ __forceinline__ void blend_tile_fwd(int tx, int ty, int width, int height, uint2 rg,
                                               const uint32_t* __restrict__ vals, const float4* __restrict__ rec,
                                               float alpha_min, float alpha_max, float t_min, const float* bg,
                                               float4* s_a, float4* s_c, float* __restrict__ img,
                                               float* __restrict__ T_final, uint32_t* __restrict__ n_contrib) {
    constexpr int NT = TS * TS;
    constexpr int BPR = TS / 8;  // 8 x 4 warp blocks per block row of the tile
    static_assert(B <= NT, "staging batch larger than the tile");
    static_assert(TS >= 8 && TS <= 32, "the tile holds whole 8 x 4 warp blocks");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int bx = tx * TS + (w % BPR) * 8, by = ty * TS + (w / BPR) * 4;  // the warp's block
    const int x = bx + (lane & 7), y = by + (lane >> 3);
    const bool inside = x < width && y < height;
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    // pixel centres of this warp's block
    const float bx0 = (float)bx + 0.5f, bx1 = bx0 + 7.f;
    const float by0 = (float)by + 0.5f, by1 = by0 + 3.f;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    // Software-pipelined staging: thread t < B stages entry b0 + t of every
    // batch, its ids fetched two batches ahead and its records one batch ahead,
    // so that a long walk does not wait out two dependent gathers per batch.
    const bool stager = threadIdx.x < B;
    uint32_t g_nxt = 0;
    float4 a_cur = make_float4(0.f, 0.f, 0.f, 0.f), c_cur = a_cur;
    if (stager) {
        const uint32_t j0 = rg.x + threadIdx.x, j1 = j0 + B;
        if (j0 < rg.y) {
            const uint32_t g = vals[j0];
            a_cur = rec[2 * g];
            c_cur = rec[2 * g + 1];
        }
        if (j1 < rg.y) g_nxt = vals[j1];
    }
    for (uint32_t b0 = rg.x; b0 < rg.y; b0 += B) {
        if (__syncthreads_count(done) == NT) break;
        if (stager) {
            const uint32_t j = b0 + threadIdx.x;
            if (j < rg.y) {
                s_a[threadIdx.x] = a_cur;
                s_c[threadIdx.x] = c_cur;
            }
            if (j + B < rg.y) {  // the next batch's record, then the id of the one after it
                a_cur = rec[2 * g_nxt];
                c_cur = rec[2 * g_nxt + 1];
            }
            if (j + 2 * B < rg.y) g_nxt = vals[j + 2 * B];
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)B, rg.y - b0);
        for (int c0 = 0; c0 < nb; c0 += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            const bool reach = c0 + lane < nb && may_reach(s_a[c0 + lane], bx0, bx1, by0, by1);
            uint32_t bits = __ballot_sync(0xffffffffu, reach);
            while (bits && !done) {
                const int k = c0 + __ffs(bits) - 1;
                bits &= bits - 1;
                const float4 a = s_a[k];
                const float pw = eval_dist(px, py, a).pw;
                if (pw > a.w) continue;
                const float4 c = s_c[k];
                const float alpha = fminf(alpha_max, __fmul_rn(c.w, fast_exp2(-pw)));
                if (alpha < alpha_min) continue;
                const float Tn = T * (1.f - alpha);
                if (Tn < t_min) {
                    done = true;
                    break;
                }
                const float w = alpha * T;
                C0 = fmaf(c.x, w, C0);
                C1 = fmaf(c.y, w, C1);
                C2 = fmaf(c.z, w, C2);
                T = Tn;
                last = b0 - rg.x + k + 1;
            }
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
