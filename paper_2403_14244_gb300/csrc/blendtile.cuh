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

// Block-wide last blend (max of last, +1 positions) into *s_hi of the caller's
// shared memory.
__device__ __forceinline__ void seg_reduce_into(uint32_t last, int lane, uint32_t* s_hi) {
    const uint32_t whi = __reduce_max_sync(0xffffffffu, last);
    if (lane == 0) atomicMax(s_hi, whi);
}

// One CTA of TS*TS threads composites one tile (one thread per pixel), staging
// B entries at a time in shared memory (s_a, s_c hold B float4 each), and leaves
// the batch loop once every pixel has stopped. Each warp owns an 8 x 4 block of
// the tile (compact blocks are reached by fewer entries than whole rows, and
// their pixels stop at similar depths) and walks, in order, only the staged
// entries that may reach it (one ballot per 32 entries). Writes img (planar,
// `plane` floats per channel, row stride `width`) and, if given, T_final /
// n_contrib. SEG (one 8 x 8 block per CTA): the walk is cut into segments for
// the backward (SegLayout), `block` naming this block.
template <int TS, int B, bool SEG = false>
__device__ __forceinline__ void blend_tile_fwd(int tx, int ty, int width, int height, uint2 rg,
                                               const uint32_t* __restrict__ vals, const float4* __restrict__ rec,
                                               float alpha_min, float alpha_max, float t_min, const float* bg,
                                               float4* s_a, float4* s_c, float* __restrict__ img,
                                               float* __restrict__ T_final, uint32_t* __restrict__ n_contrib,
                                               const SegLayout seg = SegLayout{}, uint32_t block = 0) {
    constexpr int NT = TS * TS;
    static_assert(!SEG || NT == 64, "segments are cut per 8 x 8 block, one thread per pixel");
    // segment state: where the open segment starts (the last cut), the block's
    // last blend, and the slots of the segments closed so far
    __shared__ uint32_t s_lo, s_hi, s_slot, s_n, s_stop;
    __shared__ uint32_t s_slots[SEG ? kSegMaxPerBlock : 1];
    uint32_t reserved = kSegNone;  // thread 0: the pool slot taken for the next close (its atomic
                                   // is in flight meanwhile, off the block's path)
    const bool segs = SEG && seg.slots != 0;
    if (segs) {
        if (threadIdx.x == 0) {
            s_lo = 0;
            s_hi = 0;
            s_n = 0;
            s_stop = 0;
        }
        __syncthreads();
    }
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
        if constexpr (SEG) {
            const uint32_t P = b0 - rg.x;
            if (segs && P > 0 && P % kSegStride == 0) {
                // close the open segment here if it holds blends: each pixel's state is
                // that after every entry before P (its colour is turned into the colour
                // behind once the walk has ended)
                seg_reduce_into(last, lane, &s_hi);
                __syncthreads();
                if (threadIdx.x == 0) {
                    uint32_t slot = kSegNone;
                    if (s_hi > s_lo && !s_stop && s_n < kSegMaxPerBlock) {  // blends since the last cut
                        if (reserved == kSegNone) {  // first close: this slot and the next one
                            slot = atomicAdd(&seg.ctrl->slots_used, 2u);
                            reserved = slot + 1;
                        } else {
                            slot = reserved;
                            reserved = atomicAdd(&seg.ctrl->slots_used, 1u);
                        }
                        if (slot >= seg.slots) {
                            slot = kSegNone;
                            s_stop = 1;  // pool full: the block's last segment takes the rest
                        } else {
                            seg.items[slot] = make_uint4(block, s_lo, s_hi, slot);
                            s_slots[s_n++] = slot;
                            s_lo = P;
                        }
                    }
                    s_slot = slot;
                }
                __syncthreads();
                if (s_slot != kSegNone) seg.pool[(size_t)s_slot * 64 + threadIdx.x] = make_float4(T, C0, C1, C2);
            }
        }
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
    if constexpr (SEG) {
        if (segs) {
            seg_reduce_into(last, lane, &s_hi);
            __syncthreads();
            if (threadIdx.x == 0) {
                // (no segment closed: the last segment is the whole walk; lo = kSegNone:
                // no blend after the last cut)
                seg.last[block] = s_n == 0 ? make_uint4(0u, 0u, kSegNone, 0u)
                                           : make_uint4(s_n, s_hi > s_lo ? s_lo : kSegNone, s_hi, 0u);
                if (reserved != kSegNone && reserved < seg.slots)
                    seg.items[reserved] = make_uint4(kSegNone, 0u, 0u, kSegNone);  // taken, not used
            }
            // the saved colours become the colour composited behind each cut
            for (uint32_t i = 0; i < s_n; ++i) {
                float4* q = seg.pool + (size_t)s_slots[i] * 64 + threadIdx.x;
                const float4 v = *q;
                *q = make_float4(v.x, fmaf(T, bg[0], C0 - v.y), fmaf(T, bg[1], C1 - v.z), fmaf(T, bg[2], C2 - v.w));
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
