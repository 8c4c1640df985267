// The paper's 2D experiment (Sec. 3): an image as a sum of isotropic kernels,
//   f^(x) = sum over k with |mu_k - x| < D of A_k exp(-|x - mu_k|^2 / (2 sigma_k^2)),
// its adjoint, an Adam step that keeps its step count on the device (so that a
// captured CUDA graph can replay iterations), and the QuadTree initialisation
// of Sec. 3.1.
//
// Particles are float4 pairs (mu_x, mu_y, log sigma, A_r | A_g, A_b, 0, 0) in
// pixel units; pixel (x, y) samples at (x + 0.5, y + 0.5). The support test is
// canonical FP32 (dx = px - mu_x, dy = py - mu_y, d2 = dx*dx + dy*dy, each step
// rounded once; reached iff d2 < D*D), so that every implementation reaches the
// same (pixel, particle) pairs.
//
// Render and adjoint: one CTA per 16 x 16 tile. Particles are staged 256 (128
// in the adjoint) at a time with their tile test (the nearest pixel centre of
// the tile, where every rounded step of d2 is smallest), and each pixel walks
// the staged particles that reach the tile in index order, so the sums are
// deterministic. The adjoint reduces each particle's six terms over a warp
// (butterfly reduce-scatter), sums the warps in shared memory and adds the
// result with one atomic per term and tile.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "fit2d.cuh"
#include "warp.cuh"

namespace igs {
namespace {

constexpr int kFitTile = 16;
constexpr int kFitThreads = kFitTile * kFitTile;
constexpr int kFitBatch = kFitThreads;  // particles staged per batch (render)
constexpr int kFitBwdBatch = 128;       // (adjoint: its per-warp partials take 32 KB)
constexpr int kFitWarps = kFitThreads / 32;

struct FitParams {
    float D2;
    int width, height, tiles_x, k;
};

__device__ __forceinline__ float fit_d2(float px, float py, float mx, float my) {
    const float dx = __fsub_rn(px, mx), dy = __fsub_rn(py, my);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// Stage particles [b0, b0 + B) (thread t takes b0 + t): s_p = (mu_x, mu_y,
// log2(e) / (2 sigma^2), 1 / sigma^2), s_a = (A_r, A_g, A_b, 0), and bit t of
// s_bits = whether the particle reaches a pixel centre of the tile [bx0, bx1] x
// [by0, by1]. Non-finite parameters reach nothing.
template <int B>
__device__ __forceinline__ void stage_particles(const float4* __restrict__ pr, int k, int b0, float D2, float bx0,
                                                float bx1, float by0, float by1, float4* s_p, float4* s_a,
                                                uint32_t* s_bits) {
    const int t = threadIdx.x;
    if (t >= B) return;
    const int j = b0 + t;
    bool reach = false;
    if (j < k) {
        const float4 a = pr[2 * j], b = pr[2 * j + 1];
        const float s = expf(a.z);
        const float inv_s2 = 1.f / (s * s);
        s_p[t] = make_float4(a.x, a.y, 0.5f * kLog2e * inv_s2, inv_s2);
        s_a[t] = make_float4(a.w, b.x, b.y, 0.f);
        const float cx = fminf(fmaxf(floorf(a.x) + 0.5f, bx0), bx1);
        const float cy = fminf(fmaxf(floorf(a.y) + 0.5f, by0), by1);
        reach = fit_d2(cx, cy, a.x, a.y) < D2;
    }
    const uint32_t bits = __ballot_sync(0xffffffffu, reach);
    if ((t & 31) == 0) s_bits[t >> 5] = bits;
}

__global__ void __launch_bounds__(kFitThreads) k_fit2d_render(const float4* __restrict__ pr, FitParams P,
                                                             float* __restrict__ img) {
    __shared__ float4 s_p[kFitBatch];
    __shared__ float4 s_a[kFitBatch];
    __shared__ uint32_t s_bits[kFitBatch / 32];
    const int tx = blockIdx.x % P.tiles_x, ty = blockIdx.x / P.tiles_x;
    const int x = tx * kFitTile + (threadIdx.x % kFitTile), y = ty * kFitTile + (threadIdx.x / kFitTile);
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    const float bx0 = (float)(tx * kFitTile) + 0.5f, bx1 = bx0 + (float)(kFitTile - 1);
    const float by0 = (float)(ty * kFitTile) + 0.5f, by1 = by0 + (float)(kFitTile - 1);
    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
    for (int b0 = 0; b0 < P.k; b0 += kFitBatch) {
        __syncthreads();
        stage_particles<kFitBatch>(pr, P.k, b0, P.D2, bx0, bx1, by0, by1, s_p, s_a, s_bits);
        __syncthreads();
#pragma unroll 1
        for (int wd = 0; wd < kFitBatch / 32; ++wd) {
            uint32_t bits = s_bits[wd];
            while (bits) {
                const int j = wd * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                const float4 p = s_p[j];
                const float d2 = fit_d2(px, py, p.x, p.y);
                if (d2 < P.D2) {
                    const float g = fast_exp2(-d2 * p.z);
                    const float4 a = s_a[j];
                    c0 = fmaf(a.x, g, c0);
                    c1 = fmaf(a.y, g, c1);
                    c2 = fmaf(a.z, g, c2);
                }
            }
        }
    }
    if (x >= P.width || y >= P.height) return;
    const size_t pix = (size_t)y * P.width + x, plane = (size_t)P.width * P.height;
    img[pix] = c0;
    img[plane + pix] = c1;
    img[2 * plane + pix] = c2;
}

// d_particles must be zero on entry (the launcher clears it).
__global__ void __launch_bounds__(kFitThreads) k_fit2d_bwd(const float4* __restrict__ pr, FitParams P,
                                                          const float* __restrict__ dL, float* __restrict__ dpr) {
    constexpr int B = kFitBwdBatch;
    __shared__ float4 s_p[B];
    __shared__ float4 s_a[B];
    __shared__ uint32_t s_bits[B / 32];
    __shared__ float s_red[kFitWarps][B][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tx = blockIdx.x % P.tiles_x, ty = blockIdx.x / P.tiles_x;
    const int x = tx * kFitTile + (threadIdx.x % kFitTile), y = ty * kFitTile + (threadIdx.x / kFitTile);
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    const float bx0 = (float)(tx * kFitTile) + 0.5f, bx1 = bx0 + (float)(kFitTile - 1);
    const float by0 = (float)(ty * kFitTile) + 0.5f, by1 = by0 + (float)(kFitTile - 1);
    float G0 = 0.f, G1 = 0.f, G2 = 0.f;  // pixels outside the image carry no gradient
    if (x < P.width && y < P.height) {
        const size_t pix = (size_t)y * P.width + x, plane = (size_t)P.width * P.height;
        G0 = dL[pix];
        G1 = dL[plane + pix];
        G2 = dL[2 * plane + pix];
    }
    for (int b0 = 0; b0 < P.k; b0 += B) {
        __syncthreads();
        stage_particles<B>(pr, P.k, b0, P.D2, bx0, bx1, by0, by1, s_p, s_a, s_bits);
        __syncthreads();
#pragma unroll 1
        for (int wd = 0; wd < B / 32; ++wd) {
            uint32_t bits = s_bits[wd];
            while (bits) {
                const int j = wd * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                const float4 p = s_p[j];
                const float dx = __fsub_rn(px, p.x), dy = __fsub_rn(py, p.y);
                const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                const bool active = d2 < P.D2;
                float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (active) {
                    const float g = fast_exp2(-d2 * p.z);
                    const float4 a = s_a[j];
                    const float sg = (a.x * G0 + a.y * G1 + a.z * G2) * g * p.w;  // s g / sigma^2
                    v[0] = sg * dx;
                    v[1] = sg * dy;
                    v[2] = sg * d2;
                    v[3] = g * G0;
                    v[4] = g * G1;
                    v[5] = g * G2;
                }
                if (__any_sync(0xffffffffu, active)) {
                    const float r = warp_reduce8(v, lane);
                    if ((lane & 3) == 0) s_red[w][j][lane >> 2] = r;
                } else if (lane < 8) {
                    s_red[w][j][lane] = 0.f;
                }
            }
        }
        __syncthreads();
        // sum the warps' partials of every particle that reaches the tile
        for (int t = threadIdx.x; t < B * 6; t += kFitThreads) {
            const int j = t / 6, c = t - 6 * j;
            if (!((s_bits[j >> 5] >> (j & 31)) & 1u)) continue;
            float acc = 0.f;
#pragma unroll
            for (int ww = 0; ww < kFitWarps; ++ww) acc += s_red[ww][j][c];
            if (acc != 0.f) atomicAdd(&dpr[8 * (size_t)(b0 + j) + c], acc);
        }
    }
}

// One Adam step over the particles (2 float4 per particle, slot j of the 8 with
// learning rate lr[j]); the step count t - 1 is state[0], read by every block,
// and the last block to finish increments it (state[1] is its ticket counter).
__global__ void __launch_bounds__(256) k_fit2d_adam(float4* __restrict__ p, const float4* __restrict__ g,
                                                   float4* __restrict__ m, float4* __restrict__ v, int n4,
                                                   Fit2dAdam a, int32_t* __restrict__ state) {
    __shared__ float s_step[8];
    __shared__ float s_bc2_sqrt;
    if (threadIdx.x == 0) {
        const int t = state[0] + 1;
        const double bc1 = 1.0 - pow(a.b1d, (double)t), bc2 = 1.0 - pow(a.b2d, (double)t);
        for (int j = 0; j < 8; ++j) s_step[j] = (float)((double)a.lr[j] / bc1);
        s_bc2_sqrt = (float)sqrt(bc2);
    }
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
        float4 pp = p[i], gg = g[i], mm = m[i], vv = v[i];
        const int s0 = (i & 1) * 4;
        float* pf = &pp.x;
        const float* gf = &gg.x;
        float* mf = &mm.x;
        float* vf = &vv.x;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            mf[c] = a.b1 * mf[c] + a.omb1 * gf[c];
            vf[c] = a.b2 * vf[c] + a.omb2 * gf[c] * gf[c];
            const float denom = sqrtf(vf[c]) / s_bc2_sqrt + a.eps;
            pf[c] -= s_step[s0 + c] * mf[c] / denom;
        }
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(reinterpret_cast<unsigned*>(&state[1]), 1u);
        if (ticket == gridDim.x - 1) {
            state[0] += 1;
            state[1] = 0;
        }
    }
}

// ------------------------------------------------------------- QuadTree ----
//
// Cells of level l (0 = the whole image) are 2^l x 2^l, id = (4^l - 1) / 3 +
// row 2^l + column. Each holds the exact integer sums S1_c, S2_c of the 12-bit
// quantised image q = rint(clamp(v, 0, 1) 4096) and of q^2. The greedy rule
// (split the leaf of largest error first) splits the cells that come first in
// the order (error key descending, id ascending): a cell's error is never below
// a child's and its id is smaller, so that order lists every parent before its
// children, and the greedy frontier always holds the next cell of it. So the
// tree is "the first m cells of that order are split", m = min((k_max - 1) / 3,
// splittable cells), found by bisection on the key and then on the id.

struct CellStats {
    long long s1[3], s2[3];
};

__host__ __device__ inline long long level_off(int l) { return (((long long)1 << (2 * l)) - 1) / 3; }

__global__ void k_qt_base(const float* __restrict__ img, int side, int lf, CellStats* __restrict__ st) {
    const int per = 1 << lf, cs = side >> lf;
    const long long n = (long long)per * per;
    const size_t plane = (size_t)side * side;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int iy = (int)(c / per), ix = (int)(c % per);
        CellStats s;
        for (int ch = 0; ch < 3; ++ch) {
            long long a = 0, b = 0;
            for (int y = iy * cs; y < (iy + 1) * cs; ++y)
                for (int x = ix * cs; x < (ix + 1) * cs; ++x) {
                    const float v = fminf(fmaxf(img[ch * plane + (size_t)y * side + x], 0.f), 1.f);
                    const long long q = (long long)rintf(v * 4096.f);
                    a += q;
                    b += q * q;
                }
            s.s1[ch] = a;
            s.s2[ch] = b;
        }
        st[level_off(lf) + c] = s;
    }
}

__global__ void k_qt_up(CellStats* __restrict__ st, int l) {
    const int per = 1 << l;
    const long long n = (long long)per * per;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int iy = (int)(c / per), ix = (int)(c % per);
        CellStats s;
        for (int ch = 0; ch < 3; ++ch) s.s1[ch] = s.s2[ch] = 0;
        for (int d = 0; d < 4; ++d) {
            const CellStats& k = st[level_off(l + 1) + (long long)(2 * iy + (d >> 1)) * (2 * per) + 2 * ix + (d & 1)];
            for (int ch = 0; ch < 3; ++ch) {
                s.s1[ch] += k.s1[ch];
                s.s2[ch] += k.s2[ch];
            }
        }
        st[level_off(l) + c] = s;
    }
}

constexpr int kQtThreads = 1024;

// Error key of a cell of n pixels: T / n as a double (T = sum_c n S2_c - S1_c^2,
// exact), returned as its bit pattern (ordered like the value: T / n >= 0).
__device__ __forceinline__ unsigned long long cell_key(const CellStats& s, long long n) {
    unsigned long long T = 0;
    for (int ch = 0; ch < 3; ++ch)
        T += (unsigned long long)(n * s.s2[ch]) - (unsigned long long)(s.s1[ch] * s.s1[ch]);
    const double k = __ddiv_rn(__ull2double_rn(T), (double)n);
    return (unsigned long long)__double_as_longlong(k);
}

__device__ __forceinline__ long long block_sum_ll(long long v, long long* s_tmp) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = v;
    __syncthreads();
    long long t = 0;
    for (int i = 0; i < kQtThreads / 32; ++i) t += s_tmp[i];
    return t;
}

// One CTA: keys of the splittable cells (levels < lf), the m-th largest in
// (key desc, id asc), and the split flags.
__global__ void __launch_bounds__(kQtThreads) k_qt_select(const CellStats* __restrict__ st, int side, int lf, int k_max,
                                                         unsigned long long* __restrict__ keys,
                                                         uint8_t* __restrict__ split) {
    __shared__ long long s_tmp[kQtThreads / 32];
    const long long items = level_off(lf);
    for (int l = 0; l < lf; ++l) {
        const long long per = 1LL << l, cs = side >> l;
        for (long long c = threadIdx.x; c < per * per; c += kQtThreads)
            keys[level_off(l) + c] = cell_key(st[level_off(l) + c], cs * cs);
    }
    __syncthreads();
    const long long m = min((long long)((k_max - 1) / 3), items);
    // X = max{X : count(key >= X) >= m}
    unsigned long long X = 0, Ihi = 0;
    if (m > 0 && m < items) {
        unsigned long long lo = 0, hi = ~0ULL;  // invariant: count(>= lo) >= m, count(>= hi + 1) < m (hi + 1 may wrap)
        while (lo < hi) {
            const unsigned long long mid = lo + (hi - lo) / 2 + 1;
            long long cnt = 0;
            for (long long i = threadIdx.x; i < items; i += kQtThreads) cnt += keys[i] >= mid;
            if (block_sum_ll(cnt, s_tmp) >= m)
                lo = mid;
            else
                hi = mid - 1;
        }
        X = lo;
        long long gt = 0;
        for (long long i = threadIdx.x; i < items; i += kQtThreads) gt += keys[i] > X;
        const long long r = m - block_sum_ll(gt, s_tmp);  // >= 1 cells with key == X, smallest ids
        // I = min{I : count(key == X and id <= I) >= r}
        unsigned long long a = 0, b = (unsigned long long)items - 1;
        while (a < b) {
            const unsigned long long mid = a + (b - a) / 2;
            long long cnt = 0;
            for (long long i = threadIdx.x; i <= (long long)mid; i += kQtThreads) cnt += keys[i] == X;
            if (block_sum_ll(cnt, s_tmp) >= r)
                b = mid;
            else
                a = mid + 1;
        }
        Ihi = a;
    }
    for (long long i = threadIdx.x; i < items; i += kQtThreads) {
        bool s;
        if (m <= 0)
            s = false;
        else if (m >= items)
            s = true;
        else
            s = keys[i] > X || (keys[i] == X && (unsigned long long)i <= Ihi);
        split[i] = s ? 1 : 0;
    }
}

// One CTA: the leaves in id order (a cell is a leaf if it is the root or its
// parent is split, and it is not split itself), one particle each.
__global__ void __launch_bounds__(kQtThreads) k_qt_emit(const CellStats* __restrict__ st,
                                                       const uint8_t* __restrict__ split, int side, int lf, int k_max,
                                                       float4* __restrict__ out, int32_t* __restrict__ count) {
    __shared__ int s_warp[kQtThreads / 32];
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long cells = level_off(lf + 1);
    for (long long c0 = 0; c0 < cells; c0 += kQtThreads) {
        const long long id = c0 + threadIdx.x;
        bool leaf = false;
        int l = 0, iy = 0, ix = 0;
        if (id < cells) {
            while (level_off(l + 1) <= id) ++l;
            const long long r = id - level_off(l), per = 1LL << l;
            iy = (int)(r / per);
            ix = (int)(r % per);
            const bool parent_split = l == 0 || split[level_off(l - 1) + (long long)(iy >> 1) * (per >> 1) + (ix >> 1)];
            leaf = parent_split && (l == lf || !split[id]);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, leaf);
        if (lane == 0) s_warp[w] = __popc(bal);
        __syncthreads();
        int before = s_base, total = 0;
        for (int i = 0; i < kQtThreads / 32; ++i) {
            if (i < w) before += s_warp[i];
            total += s_warp[i];
        }
        const int pos = before + __popc(bal & ((1u << lane) - 1u));
        if (leaf && pos < k_max) {
            const CellStats& s = st[id];
            const int cs = side >> l;
            const double n = (double)cs * (double)cs;
            int lg = 0;
            while ((1 << lg) < cs) ++lg;
            float4 a, b;
            a.x = (float)((double)ix * cs + 0.5 * cs);
            a.y = (float)((double)iy * cs + 0.5 * cs);
            a.z = (float)((double)(lg - 1) * 0.6931471805599453);
            a.w = (float)__ddiv_rn((double)s.s1[0], 4096.0 * n);
            b.x = (float)__ddiv_rn((double)s.s1[1], 4096.0 * n);
            b.y = (float)__ddiv_rn((double)s.s1[2], 4096.0 * n);
            b.z = b.w = 0.f;
            out[2 * pos] = a;
            out[2 * pos + 1] = b;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = min(s_base, k_max);
}

// ------------------------------------------------------- densify / prune ----
//
// Sec. 3.2 deletes particles whose amplitude falls below a threshold, and
// Sec. 2's multiscale property divides coarse particles into finer ones. The
// statistic for division is the position-gradient norm summed over the
// iterations since the last densify (k_fit2d_grad_accum, called after each
// adjoint). One CTA walks the particles in chunks of kDensThreads: a first pass
// counts the kept particles and the division candidates (which fixes how many
// candidates fit the capacity), a second pass gives each particle its output
// slot (exclusive scan of 0 / 1 / 4 outputs, carried across chunks) and writes
// the kept particle or its four children, so the output is in index order with
// children in place of their parent.

constexpr int kDensThreads = 1024;

struct DensifyParams {
    float thr, tau_a, log_sigma_min;
    int k, capacity;
};

// accum_i += |dL/dmu_i| in FP32, one rounding per step.
__global__ void __launch_bounds__(256) k_fit2d_grad_accum(const float4* __restrict__ g, int k,
                                                         float* __restrict__ accum) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const float4 a = g[2 * i];
        const float sq = __fadd_rn(__fmul_rn(a.x, a.x), __fmul_rn(a.y, a.y));
        accum[i] = __fadd_rn(accum[i], __fsqrt_rn(sq));
    }
}

// Keep: max_c |A_c| is not below tau_a (the comparisons run in this order, so a
// NaN amplitude keeps its particle). Candidate: kept, accum_i > thr and
// log sigma >= log_sigma_min.
__device__ __forceinline__ void densify_flags(const float4* __restrict__ pr, const float* __restrict__ accum, int i,
                                              const DensifyParams& P, bool& keep, bool& cand) {
    const float4 a = pr[2 * i], b = pr[2 * i + 1];
    float amax = fabsf(a.w);
    if (fabsf(b.x) > amax) amax = fabsf(b.x);
    if (fabsf(b.y) > amax) amax = fabsf(b.y);
    keep = !(amax < P.tau_a);
    cand = keep && accum[i] > P.thr && a.z >= P.log_sigma_min;
}

__global__ void __launch_bounds__(kDensThreads) k_fit2d_densify(const float4* __restrict__ pr,
                                                               const float4* __restrict__ m,
                                                               const float4* __restrict__ v,
                                                               const float* __restrict__ accum, DensifyParams P,
                                                               float4* __restrict__ out, float4* __restrict__ om,
                                                               float4* __restrict__ ov, int32_t* __restrict__ count) {
    __shared__ uint32_t s_warp[kDensThreads / 32];
    __shared__ uint32_t s_tot[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // pass 1: kept particles and division candidates
    uint32_t nk = 0, nc = 0;
    for (int i = threadIdx.x; i < P.k; i += kDensThreads) {
        bool keep, cand;
        densify_flags(pr, accum, i, P, keep, cand);
        nk += keep;
        nc += cand;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nk += __shfl_xor_sync(0xffffffffu, nk, o);
        nc += __shfl_xor_sync(0xffffffffu, nc, o);
    }
    if (threadIdx.x == 0) s_tot[0] = s_tot[1] = 0;
    __syncthreads();
    if (lane == 0) {
        atomicAdd(&s_tot[0], nk);
        atomicAdd(&s_tot[1], nc);
    }
    __syncthreads();
    const long long keep_total = s_tot[0], cand_total = s_tot[1];
    const long long allowed = min(P.capacity > keep_total ? ((long long)P.capacity - keep_total) / 3 : 0LL, cand_total);
    // pass 2: slots (outputs in the low 16 bits, candidates in the high 16 bits of one scan)
    long long base_out = 0, base_cand = 0;
    for (int c0 = 0; c0 < P.k; c0 += kDensThreads) {
        const int i = c0 + threadIdx.x;
        bool keep = false, cand = false;
        if (i < P.k) densify_flags(pr, accum, i, P, keep, cand);
        // a candidate divides iff its rank among candidates is < allowed; outputs
        // depend on that rank, so scan the candidates first
        uint32_t x = cand ? 1u : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[w] = incl;
        __syncthreads();
        uint32_t wpre = 0, ctot = 0;
        for (int j = 0; j < kDensThreads / 32; ++j) {
            if (j < w) wpre += s_warp[j];
            ctot += s_warp[j];
        }
        const long long crank = base_cand + wpre + incl - x;
        const bool divide = cand && crank < allowed;
        __syncthreads();
        const uint32_t n_out = divide ? 4u : (keep ? 1u : 0u);
        incl = n_out;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[w] = incl;
        __syncthreads();
        uint32_t opre = 0, otot = 0;
        for (int j = 0; j < kDensThreads / 32; ++j) {
            if (j < w) opre += s_warp[j];
            otot += s_warp[j];
        }
        const long long slot = base_out + opre + incl - n_out;
        if (divide) {
            // four children with half the scale at mu +- sigma / 2, zero moments
            const float4 a = pr[2 * i], b = pr[2 * i + 1];
            const float h = __fmul_rn(0.5f, (float)exp((double)a.z));
            const float ls = __fsub_rn(a.z, 0.6931472f);
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float x0 = (c & 1) ? __fadd_rn(a.x, h) : __fsub_rn(a.x, h);
                const float y0 = (c & 2) ? __fadd_rn(a.y, h) : __fsub_rn(a.y, h);
                const long long o = slot + c;
                out[2 * o] = make_float4(x0, y0, ls, a.w);
                out[2 * o + 1] = make_float4(b.x, b.y, 0.f, 0.f);
                om[2 * o] = om[2 * o + 1] = zero;
                ov[2 * o] = ov[2 * o + 1] = zero;
            }
        } else if (keep && slot < P.capacity) {
            out[2 * slot] = pr[2 * i];
            out[2 * slot + 1] = pr[2 * i + 1];
            om[2 * slot] = m[2 * i];
            om[2 * slot + 1] = m[2 * i + 1];
            ov[2 * slot] = v[2 * i];
            ov[2 * slot + 1] = v[2 * i + 1];
        }
        base_out += otot;
        base_cand += ctot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = (int32_t)min(base_out, (long long)P.capacity);
}

int finest_level(int side, int min_cell) {
    int lf = 0;
    while ((side >> (lf + 1)) >= min_cell && (side >> (lf + 1)) >= 1) ++lf;
    return lf;
}

}  // namespace

cudaError_t launch_fit2d_render(const float* particles, int k, float D, int width, int height, float* img,
                                cudaStream_t st) {
    FitParams P;
    P.D2 = D * D;
    P.width = width;
    P.height = height;
    P.tiles_x = (int)ceil_div(width, kFitTile);
    P.k = k;
    const unsigned tiles = (unsigned)(P.tiles_x * ceil_div(height, kFitTile));
    k_fit2d_render<<<tiles, kFitThreads, 0, st>>>(reinterpret_cast<const float4*>(particles), P, img);
    count_launches();
    return cudaGetLastError();
}

cudaError_t launch_fit2d_backward(const float* particles, int k, float D, int width, int height, const float* dL,
                                  float* d_particles, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d_particles, 0, sizeof(float) * 8 * (size_t)k, st);
    if (e != cudaSuccess || k == 0) return e;
    FitParams P;
    P.D2 = D * D;
    P.width = width;
    P.height = height;
    P.tiles_x = (int)ceil_div(width, kFitTile);
    P.k = k;
    const unsigned tiles = (unsigned)(P.tiles_x * ceil_div(height, kFitTile));
    k_fit2d_bwd<<<tiles, kFitThreads, 0, st>>>(reinterpret_cast<const float4*>(particles), P, dL, d_particles);
    count_launches();
    return cudaGetLastError();
}

cudaError_t launch_fit2d_adam(float* particles, const float* d_particles, float* m, float* v, int k,
                              const Fit2dAdam& a, int32_t* state, cudaStream_t st) {
    if (k == 0) return cudaSuccess;
    const int n4 = 2 * k;
    const int blocks = (int)std::min<int64_t>(ceil_div(n4, 256), 152 * 4);
    k_fit2d_adam<<<blocks, 256, 0, st>>>(reinterpret_cast<float4*>(particles),
                                         reinterpret_cast<const float4*>(d_particles), reinterpret_cast<float4*>(m),
                                         reinterpret_cast<float4*>(v), n4, a, state);
    count_launches();
    return cudaGetLastError();
}

cudaError_t launch_fit2d_grad_accum(const float* d_particles, int k, float* accum, cudaStream_t st) {
    if (k == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>(ceil_div(k, 256), 152 * 4);
    k_fit2d_grad_accum<<<blocks, 256, 0, st>>>(reinterpret_cast<const float4*>(d_particles), k, accum);
    count_launches();
    return cudaGetLastError();
}

cudaError_t launch_fit2d_densify(const float* particles, const float* m, const float* v, const float* accum, int k,
                                 float thr, float tau_a, float log_sigma_min, int capacity, float* out, float* out_m,
                                 float* out_v, int32_t* count, cudaStream_t st) {
    DensifyParams P;
    P.thr = thr;
    P.tau_a = tau_a;
    P.log_sigma_min = log_sigma_min;
    P.k = k;
    P.capacity = capacity;
    k_fit2d_densify<<<1, kDensThreads, 0, st>>>(
        reinterpret_cast<const float4*>(particles), reinterpret_cast<const float4*>(m),
        reinterpret_cast<const float4*>(v), accum, P, reinterpret_cast<float4*>(out), reinterpret_cast<float4*>(out_m),
        reinterpret_cast<float4*>(out_v), count);
    count_launches();
    return cudaGetLastError();
}

size_t quadtree_work_bytes(int side, int min_cell) {
    const int lf = finest_level(side, min_cell);
    const size_t cells = (size_t)level_off(lf + 1), items = (size_t)level_off(lf);
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return up(cells * sizeof(CellStats)) + up(items * sizeof(unsigned long long)) + up(items + 1);
}

cudaError_t launch_quadtree_init(const float* img, int side, int k_max, int min_cell, float* particles,
                                 int32_t* count, void* work, cudaStream_t st) {
    const int lf = finest_level(side, min_cell);
    const size_t cells = (size_t)level_off(lf + 1), items = (size_t)level_off(lf);
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    char* w = static_cast<char*>(work);
    auto* stats = reinterpret_cast<CellStats*>(w);
    auto* keys = reinterpret_cast<unsigned long long*>(w + up(cells * sizeof(CellStats)));
    auto* split = reinterpret_cast<uint8_t*>(w + up(cells * sizeof(CellStats)) + up(items * sizeof(unsigned long long)));
    const long long base = 1LL << (2 * lf);
    k_qt_base<<<(unsigned)std::min<long long>(ceil_div(base, 256), 152 * 8), 256, 0, st>>>(img, side, lf, stats);
    cudaError_t e = cudaGetLastError();
    int launches = 1;
    for (int l = lf - 1; l >= 0 && e == cudaSuccess; --l) {
        const long long n = 1LL << (2 * l);
        k_qt_up<<<(unsigned)std::min<long long>(ceil_div(n, 256), 152 * 8), 256, 0, st>>>(stats, l);
        e = cudaGetLastError();
        ++launches;
    }
    if (e == cudaSuccess) {
        k_qt_select<<<1, kQtThreads, 0, st>>>(stats, side, lf, k_max, keys, split);
        e = cudaGetLastError();
        ++launches;
    }
    if (e == cudaSuccess) {
        k_qt_emit<<<1, kQtThreads, 0, st>>>(stats, split, side, lf, k_max, reinterpret_cast<float4*>(particles),
                                            count);
        e = cudaGetLastError();
        ++launches;
    }
    count_launches(launches);
    return e;
}

}  // namespace igs
