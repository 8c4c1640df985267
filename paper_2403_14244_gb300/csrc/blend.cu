// Per-tile front-to-back compositing (Eq. 4) and its adjoint.
//
// One CTA per tile, one thread per pixel. The tile's entries (already in
// front-to-back order) are staged in shared memory in batches; each pixel walks
// them with
//   alpha = min(alpha_max, o * 2^(-w2 d^2)),  w2 = log2(e) / (2 s^2)   (Eq. 8)
//   skip if alpha < alpha_min; stop (without blending) if T (1 - alpha) < t_min
//   C += c alpha T; T *= (1 - alpha)
// and the CTA leaves the batch loop as soon as every pixel has stopped
// (__syncthreads_count). Each warp first ballots which staged entries can reach
// its rows at all (w2 d^2 <= pmax at the nearest pixel centre) and walks only
// those; the per-pixel test w2 d^2 > pmax skips the exponential where alpha must
// fall below alpha_min. The backward pass walks each pixel's blended entries
// in reverse from n_contrib, recovering T_k = T_{k+1} / (1 - alpha_k) from the
// saved T_final, and reduces the per-pixel gradient terms of each entry over
// the tile before one vector atomic per (entry, 4 floats).
#include "blendtile.cuh"
#include "warp.cuh"

namespace igs {
namespace {

// Zeros to n4 float4 at p (none if p is null), spread over the grid: the
// forward blend of a training step clears the 2D gradient for the adjoint that
// follows. The blend is bound by instruction issue and leaves HBM mostly idle,
// so the stores cost it a few instructions per thread, not a pass of their own.
__device__ __forceinline__ void clear_slice(float4* __restrict__ p, uint64_t n4) {
    if (!p) return;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int TS>
__global__ void __launch_bounds__(TS* TS) k_blend_fwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                                                      const float4* __restrict__ rec, BlendParams P,
                                                      float* __restrict__ img, float* __restrict__ T_final,
                                                      uint32_t* __restrict__ n_contrib,
                                                      const uint32_t* __restrict__ info, float4* __restrict__ clear,
                                                      uint64_t clear4) {
    constexpr int NT = TS * TS;
    __shared__ float4 s_a[NT];
    __shared__ float4 s_c[NT];
    clear_slice(clear, clear4);
    if (info[kInfoAbort]) return;
    const int tile = blockIdx.x;
    blend_tile_fwd<TS, NT>(tile % P.tiles_x, tile / P.tiles_x, P.width, P.height, ranges[tile], vals, rec, P.alpha_min,
                           P.alpha_max, P.t_min, P.bg, s_a, s_c, img, T_final, n_contrib);
}


// Entries staged per barrier pair in the backward: 64 (two ballot words per
// warp) for 16x16 tiles; 32 for 32x32 tiles (whose per-warp partials would not
// fit otherwise) and for the one-warp 8x8 blocks (measured faster than 64: a
// block stops on its own, so smaller batches waste fewer staged entries).
template <int TS>
constexpr int bwd_batch() { return TS == 16 ? 64 : 32; }

// One pixel's state in the reverse walk. The colour composited behind the
// current entry, S, enters the adjoint only through G . S, so the walk carries
// that scalar (GS = G . (T_final bg) at the start, then GS += w T (G . c) per
// blended entry) instead of S itself.
struct BwdPixel {
    float px, py, G0, G1, G2, T, GS;
    uint32_t nc;
};

// Per-entry factors of the adjoint, shared by the pixels that walk the entry:
// d alpha / d power = -ln 2 o g, d power / d(u, v) = -2 w2 (dx, dy).
struct BwdEntry {
    float4 a, c;
    float ocl;  // -ln 2 o
    float m2z;  // -2 w2
};

// The adjoint of one (pixel, entry) pair, added to v[0..6]; false if the pixel
// did not blend the entry.
__device__ __forceinline__ bool bwd_pair(BwdPixel& q, uint32_t pos, const BwdEntry& e, const BlendParams& P,
                                         float v[8]) {
    if (pos >= q.nc) return false;
    const float4 a4 = e.a, c = e.c;
    const Dist d = eval_dist(q.px, q.py, a4);
    if (d.pw > a4.w) return false;
    const float g = fast_exp2(-d.pw);
    const float og = __fmul_rn(c.w, g);
    const float alpha = fminf(P.alpha_max, og);
    if (alpha < P.alpha_min) return false;
    const float oma = 1.f - alpha;              // >= 1 - alpha_max > 0
    const float inv = __fdividef(1.f, oma);
    const float Tk = q.T * inv;                 // transmittance before this entry
    const float wT = alpha * Tk;
    v[4] += wT * q.G0;
    v[5] += wT * q.G1;
    v[6] += wT * q.G2;
    const float Gc = q.G0 * c.x + q.G1 * c.y + q.G2 * c.z;
    const float dalpha = Tk * Gc - q.GS * inv;
    q.GS = fmaf(wT, Gc, q.GS);
    q.T = Tk;
    if (og <= P.alpha_max) {                    // alpha not clamped
        const float dg = dalpha * g;
        v[3] += dg;                             // d/do
        const float dpow = dg * e.ocl;          // d/d(power), power = w2 d^2
        v[2] += dpow * d.d2;                    // d/dw2
        const float k2 = dpow * e.m2z;
        v[0] += k2 * d.dx;                      // d/du  (dx = px - u)
        v[1] += k2 * d.dy;                      // d/dv
    }
    return true;
}

// Two pixels per thread: warp w holds an 8 x 8 block of the TS x TS pixel tile
// (tx, ty), pixel A in its upper 8 x 4 half and pixel B four rows below, so one
// warp reduction per entry serves 64 pixels (a compact block is reached by fewer
// entries than whole rows). rg: the entries to walk (those of the tile, or of an
// enclosing binning tile). A walk segment (TS = 8) walks only list positions
// [seg_lo, seg_hi) from the pixels' saved state at seg_hi (seg_state: 64 pixels
// (T, colour behind); nullptr: the final state).
template <int TS>
__device__ __forceinline__ void blend_tile_bwd(int tx, int ty, uint2 rg, const uint32_t* __restrict__ vals,
                                               const float4* __restrict__ rec, const BlendParams& P,
                                               const float* __restrict__ dL, const float* __restrict__ T_final,
                                               const uint32_t* __restrict__ n_contrib, float4* __restrict__ g2d,
                                               uint32_t seg_lo = 0, uint32_t seg_hi = kSegNone,
                                               const float4* __restrict__ seg_state = nullptr) {
    constexpr int NT = TS * TS / 2;
    constexpr int NW = NT / 32;
    constexpr int BPR = TS / 8;  // 8 x 8 warp blocks per block row of the tile
    constexpr int BB = bwd_batch<TS>();
    constexpr int NBW = BB / 32;  // ballot words per warp
    __shared__ float4 s_a[BB];
    __shared__ float4 s_c[BB];
    __shared__ uint32_t s_id[BB];
    __shared__ float s_red[NW][BB][8];
    __shared__ uint32_t s_bits[NW][NBW];
    __shared__ uint32_t s_max;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int bx = tx * TS + (w % BPR) * 8, by = ty * TS + (w / BPR) * 8;  // the warp's block
    const int x = bx + (lane & 7);
    const int yA = by + (lane >> 3), yB = yA + 4;
    const float bx0 = (float)bx + 0.5f, bx1 = bx0 + 7.f;
    const float by0 = (float)by + 0.5f, by1 = by0 + 7.f;
    const size_t plane = (size_t)P.width * P.height;
    BwdPixel q[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int y = i ? yB : yA;
        BwdPixel& p = q[i];
        p.px = (float)x + 0.5f;
        p.py = (float)y + 0.5f;
        p.G0 = p.G1 = p.G2 = 0.f;
        p.T = 1.f;
        p.nc = 0;
        if (x < P.width && y < P.height) {
            const size_t pix = (size_t)y * P.width + x;
            p.G0 = dL[pix];
            p.G1 = dL[plane + pix];
            p.G2 = dL[2 * plane + pix];
            p.T = T_final[pix];
            p.nc = n_contrib[pix];
        }
        p.GS = p.T * (p.G0 * P.bg[0] + p.G1 * P.bg[1] + p.G2 * P.bg[2]);
        if (TS == 8 && seg_state) {  // pixel index in the 8 x 8 block: row * 8 + column = lane + 32 i
            const float4 v = seg_state[lane + 32 * i];
            p.T = v.x;
            p.GS = p.G0 * v.y + p.G1 * v.z + p.G2 * v.w;
        }
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, max(q[0].nc, q[1].nc));  // nothing blended past wmax
    if (lane == 0 && wmax) atomicMax(&s_max, wmax);
    __syncthreads();
    // no pixel blended anything at or past this entry; the walk ends at L
    const uint32_t hi_end = rg.x + min(min(s_max, seg_hi), rg.y - rg.x);
    const uint32_t L = rg.x + min(seg_lo, rg.y - rg.x);
    // Batches walk [lo, hi) downwards, BB entries each; k = 0 is the last entry
    // of a batch. With one thread per staged entry, the staging is software
    // pipelined: the thread's entry ids come two batches ahead and its records
    // one batch ahead, so a long walk does not wait out two dependent gathers
    // per batch.
    const uint32_t st = threadIdx.x;  // this thread's staged entry (NT == BB)
    auto stages = [&](uint32_t h) { return h > L && st < min((uint32_t)BB, h - L); };
    auto next_hi = [&](uint32_t h) { return h > L ? h - min((uint32_t)BB, h - L) : L; };
    uint32_t g_cur = 0, g_nxt = 0;
    float4 a_cur = make_float4(0.f, 0.f, 0.f, 0.f), c_cur = a_cur;
    if constexpr (NT == BB) {
        if (stages(hi_end)) {
            g_cur = vals[hi_end - 1 - st];
            a_cur = rec[2 * g_cur];
            c_cur = rec[2 * g_cur + 1];
        }
        const uint32_t h1 = next_hi(hi_end);
        if (stages(h1)) g_nxt = vals[h1 - 1 - st];
    }
    for (uint32_t hi = hi_end; hi > L;) {
        const uint32_t lo = hi - min((uint32_t)BB, hi - L);
        const int nb = (int)(hi - lo);
        if constexpr (NT == BB) {
            if ((int)st < nb) {
                s_id[st] = g_cur;
                s_a[st] = a_cur;
                s_c[st] = c_cur;
            }
            if (stages(lo)) {  // the next batch's records, then the ids of the one after it
                a_cur = rec[2 * g_nxt];
                c_cur = rec[2 * g_nxt + 1];
            }
            g_cur = g_nxt;
            const uint32_t h2 = next_hi(lo);
            if (stages(h2)) g_nxt = vals[h2 - 1 - st];
        } else {
            for (int t = threadIdx.x; t < nb; t += NT) {
                const uint32_t g = vals[hi - 1 - t];
                s_id[t] = g;
                s_a[t] = rec[2 * g];
                s_c[t] = rec[2 * g + 1];
            }
        }
        __syncthreads();
#pragma unroll
        for (int hw = 0; hw < NBW; ++hw) {
            // the entries this warp may have blended: before its last contributor, reaching its block
            const int kl = hw * 32 + lane;
            const bool reach = kl < nb && hi - 1 - kl - rg.x < wmax && may_reach(s_a[kl], bx0, bx1, by0, by1);
            uint32_t bits = __ballot_sync(0xffffffffu, reach);
            if (lane == 0) s_bits[w][hw] = bits;
            while (bits) {
                const int k = hw * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                const uint32_t pos = hi - 1 - k - rg.x;  // list position within the tile
                BwdEntry e;
                e.a = s_a[k];
                e.c = s_c[k];
                e.ocl = -kLn2 * e.c.w;
                e.m2z = -2.f * e.a.z;
                float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                const bool active0 = bwd_pair(q[0], pos, e, P, v);
                const bool active1 = bwd_pair(q[1], pos, e, P, v);
                if (__any_sync(0xffffffffu, active0 || active1)) {
                    const float r = warp_reduce8(v, lane);
                    if ((lane & 3) == 0) s_red[w][k][lane >> 2] = r;
                } else if (lane < 8) {
                    s_red[w][k][lane] = 0.f;
                }
            }
        }
        __syncthreads();
        // sum the warps' partials of each (entry, half) and add them to the entry's Gaussian
        for (int t = threadIdx.x; t < nb * 2; t += NT) {
            const int k = t >> 1, h = (t & 1) * 4;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int ww = 0; ww < NW; ++ww) {
                if (!((s_bits[ww][k >> 5] >> (k & 31)) & 1u)) continue;
                acc.x += s_red[ww][k][h + 0];
                acc.y += s_red[ww][k][h + 1];
                acc.z += s_red[ww][k][h + 2];
                acc.w += s_red[ww][k][h + 3];
            }
            if (acc.x != 0.f || acc.y != 0.f || acc.z != 0.f || acc.w != 0.f)
                atomicAdd(&g2d[2 * s_id[k] + (h >> 2)], acc);
        }
        __syncthreads();
        hi = lo;
    }
}

template <int TS>
__global__ void __launch_bounds__(TS * TS / 2, (2560 / (TS * TS) < 32 ? 2560 / (TS * TS) : 32)) k_blend_bwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                                                      const float4* __restrict__ rec, BlendParams P,
                                                      const float* __restrict__ dL, const float* __restrict__ T_final,
                                                      const uint32_t* __restrict__ n_contrib,
                                                      float4* __restrict__ g2d, const uint32_t* __restrict__ info) {
    if (info[kInfoAbort]) return;
    const int tile = blockIdx.x;
    blend_tile_bwd<TS>(tile % P.tiles_x, tile / P.tiles_x, ranges[tile], vals, rec, P, dL, T_final, n_contrib, g2d);
}

// Sub-tile kernels: one CTA per 8 x 8 pixel block of a TS x TS binning tile,
// walking the binning tile's entries; each block stops on its own (its
// pixels' last contributors), and entries that miss it cost one reach test.
// Per pixel the walk, the arithmetic and the result are those of the whole-tile
// kernels.
template <int TS>
__global__ void __launch_bounds__(64) k_blend_fwd_sub(const uint2* __restrict__ ranges,
                                                      const uint32_t* __restrict__ vals,
                                                      const float4* __restrict__ rec, BlendParams P,
                                                      float* __restrict__ img, float* __restrict__ T_final,
                                                      uint32_t* __restrict__ n_contrib,
                                                      const uint32_t* __restrict__ info, SegLayout seg,
                                                      float4* __restrict__ clear, uint64_t clear4) {
    pdl_wait();
    constexpr int SUB = TS / 8;
    __shared__ float4 s_a[64];
    __shared__ float4 s_c[64];
    clear_slice(clear, clear4);
    if (info[kInfoAbort]) return;
    const int tile = blockIdx.x / (SUB * SUB), q = blockIdx.x % (SUB * SUB);
    const int tx = tile % P.tiles_x, ty = tile / P.tiles_x;
    blend_tile_fwd<8, 64, true>(tx * SUB + q % SUB, ty * SUB + q / SUB, P.width, P.height, ranges[tile], vals, rec,
                                P.alpha_min, P.alpha_max, P.t_min, P.bg, s_a, s_c, img, T_final, n_contrib, seg,
                                blockIdx.x);
}

// The backward of a block's whole walk (no walk segments: the forward cut none,
// or the frame has no room for them).
template <int TS>
__global__ void __launch_bounds__(32, 32) k_blend_bwd_sub(const uint2* __restrict__ ranges,
                                                          const uint32_t* __restrict__ vals,
                                                          const float4* __restrict__ rec, BlendParams P,
                                                          const float* __restrict__ dL,
                                                          const float* __restrict__ T_final,
                                                          const uint32_t* __restrict__ n_contrib,
                                                          float4* __restrict__ g2d, const uint32_t* __restrict__ info) {
    pdl_wait();
    constexpr int SUB = TS / 8;
    if (info[kInfoAbort]) return;
    const int tile = blockIdx.x / (SUB * SUB), q = blockIdx.x % (SUB * SUB);
    const int tx = tile % P.tiles_x, ty = tile / P.tiles_x;
    blend_tile_bwd<8>(tx * SUB + q % SUB, ty * SUB + q / SUB, ranges[tile], vals, rec, P, dL, T_final, n_contrib,
                      g2d);
}

// The backward over walk segments: one-warp CTAs, all resident, take work from
// one counter: first the segments the forward closed, then each block's last
// segment (its whole walk when it closed none). Every piece walks at most
// kSegStride list positions (unless the pool ran out), so no block's long walk
// sets the kernel's length.
template <int TS>
__global__ void __launch_bounds__(32, 32) k_blend_bwd_segs(const uint2* __restrict__ ranges,
                                                           const uint32_t* __restrict__ vals,
                                                           const float4* __restrict__ rec, BlendParams P,
                                                           const float* __restrict__ dL,
                                                           const float* __restrict__ T_final,
                                                           const uint32_t* __restrict__ n_contrib,
                                                           float4* __restrict__ g2d,
                                                           const uint32_t* __restrict__ info, SegLayout seg) {
    pdl_wait();
    constexpr int SUB = TS / 8;
    if (info[kInfoAbort]) return;
    const uint32_t items = min(seg.ctrl->slots_used, seg.slots);  // closed segments, by pool slot
    const uint32_t total = items + seg.blocks;                       // then each block's last segment
    for (;;) {
        uint32_t u = 0;
        if (threadIdx.x == 0) u = atomicAdd(&seg.ctrl->next, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= total) break;
        uint32_t block, lo, hi, slot = kSegNone;
        if (u < items) {
            const uint4 it = seg.items[u];
            if (it.x == kSegNone) continue;  // a slot taken ahead and not used
            block = it.x;
            lo = it.y;
            hi = it.z;
            slot = it.w;
        } else {
            block = u - items;
            const uint4 l = seg.last[block];
            if (l.y == kSegNone) continue;  // its last segment holds no blend
            lo = l.y;
            hi = l.z;
        }
        const int tile = (int)(block / (SUB * SUB)), q = (int)(block % (SUB * SUB));
        const int tx = tile % P.tiles_x, ty = tile / P.tiles_x;
        blend_tile_bwd<8>(tx * SUB + q % SUB, ty * SUB + q / SUB, ranges[tile], vals, rec, P, dL, T_final,
                          n_contrib, g2d, lo, hi, slot == kSegNone ? nullptr : seg.pool + (size_t)slot * 64);
        __syncthreads();  // the shared staging of the next piece
    }
}

}  // namespace

// Walk segments of the sub-tile blends of frame f (off for 8-pixel tiles and
// when the frame's depth-item buffers cannot hold a useful pool).
SegLayout frame_segments(const igs_frame& f) {
    if (f.tile != 16 && f.tile != 32) return SegLayout{};
    const SortScratch s = sort_scratch(f);
    const int64_t sub = f.tile / 8;
    return seg_layout(s.seg_base, s.seg_bytes, (int64_t)f.tiles_x * f.tiles_y * sub * sub);
}

cudaError_t launch_blend_fwd(const igs_frame& f, const BlendParams& bp, float* img, cudaStream_t st, float* clear_g2d) {
    const unsigned tiles = (unsigned)(f.tiles_x * f.tiles_y);
    auto clear = reinterpret_cast<float4*>(clear_g2d);
    const uint64_t clear4 = clear_g2d ? 2 * (uint64_t)f.n : 0;  // [n][8] floats
    if (tiles == 0) {  // nothing to blend; the gradient is still cleared for the adjoint
        if (!clear || clear4 == 0) return cudaSuccess;
        ZeroRanges z = {};
        z.ptr[0] = clear;
        z.bytes[0] = clear4 * 16;
        z.count = 1;
        return launch_zero(z, st);
    }
    auto rg = reinterpret_cast<const uint2*>(f.ranges);
    auto rec = reinterpret_cast<const float4*>(f.rec);
    const SegLayout seg = frame_segments(f);
    cudaError_t e = cudaSuccess;
    if (seg.slots) {  // a fresh list of segments for this forward
        ZeroRanges z = {};
        z.ptr[0] = seg.ctrl;
        z.bytes[0] = sizeof(SegCtrl);
        z.count = 1;
        if ((e = launch_zero(z, st)) != cudaSuccess) return e;
    }
    switch (f.tile) {
        case 8: k_blend_fwd<8><<<tiles, 64, 0, st>>>(rg, f.vals, rec, bp, img, f.T_final, f.n_contrib, f.info, clear, clear4); break;
        case 16: e = launch_pdl(k_blend_fwd_sub<16>, dim3(tiles * 4), dim3(64), 0, st, rg, f.vals, rec, bp, img, f.T_final, f.n_contrib, f.info, seg, clear, clear4); break;
        case 32: e = launch_pdl(k_blend_fwd_sub<32>, dim3(tiles * 16), dim3(64), 0, st, rg, f.vals, rec, bp, img, f.T_final, f.n_contrib, f.info, seg, clear, clear4); break;
        default: return cudaErrorInvalidValue;
    }
    count_launches();
    return e != cudaSuccess ? e : cudaGetLastError();
}

// The segmented backward: one-warp CTAs, 32 resident per SM.
constexpr unsigned kSegCtas = 152 * 32;

cudaError_t launch_blend_bwd(const igs_frame& f, const BlendParams& bp, const float* dL, float* g2d, cudaStream_t st) {
    const unsigned tiles = (unsigned)(f.tiles_x * f.tiles_y);
    if (tiles == 0) return cudaSuccess;
    auto rg = reinterpret_cast<const uint2*>(f.ranges);
    auto rec = reinterpret_cast<const float4*>(f.rec);
    auto g = reinterpret_cast<float4*>(g2d);
    const SegLayout seg = frame_segments(f);
    cudaError_t e = cudaSuccess;
    switch (f.tile) {
        case 8: k_blend_bwd<8><<<tiles, 32, 0, st>>>(rg, f.vals, rec, bp, dL, f.T_final, f.n_contrib, g, f.info); break;
        case 16:
            if (seg.slots)
                e = launch_pdl(k_blend_bwd_segs<16>, dim3(kSegCtas), dim3(32), 0, st, rg, f.vals, rec, bp, dL, f.T_final, f.n_contrib, g, f.info, seg);
            else
                e = launch_pdl(k_blend_bwd_sub<16>, dim3(tiles * 4), dim3(32), 0, st, rg, f.vals, rec, bp, dL, f.T_final, f.n_contrib, g, f.info);
            break;
        case 32:
            if (seg.slots)
                e = launch_pdl(k_blend_bwd_segs<32>, dim3(kSegCtas), dim3(32), 0, st, rg, f.vals, rec, bp, dL, f.T_final, f.n_contrib, g, f.info, seg);
            else
                e = launch_pdl(k_blend_bwd_sub<32>, dim3(tiles * 16), dim3(32), 0, st, rg, f.vals, rec, bp, dL, f.T_final, f.n_contrib, g, f.info);
            break;
        default: return cudaErrorInvalidValue;
    }
    count_launches();
    return e != cudaSuccess ? e : cudaGetLastError();
}

// The backward's work counter of frame f (zeroed with the 2D gradient before
// each backward), or nullptr when the frame has no walk segments.
void* blend_bwd_counter(const igs_frame& f) {
    const SegLayout seg = frame_segments(f);
    return seg.slots ? &seg.ctrl->next : nullptr;
}

const uint32_t* blend_segments_used(const igs_frame& f) {
    const SegLayout seg = frame_segments(f);
    return seg.slots ? &seg.ctrl->slots_used : nullptr;
}

}  // namespace igs
