// Merging of the 3D Gaussians (Sec. 3.2: particles may be merged or divided;
// Sec. 2.5's multiscale property; the Octree of Sec. 3.1 as the pattern, so a
// merge is the inverse of the octant division): the eligible Gaussians that
// share a cell of a grid, two or more of them, become one Gaussian at the
// place of the first; every other Gaussian is kept. Output in index order.
//
//   k_merge_keys     per Gaussian: its cell key (x | y << 10 | z << 20) if it
//                    is eligible, else 0xFFFFFFFF (FP32 cell indices, each step
//                    rounded once; the opacity floor tested on the stored value)
//   k_hist, 4 passes stable radix sort of (key, index): a cell's Gaussians end
//                    up together, in index order
//   k_merge_mark     per sorted position that starts a cell of two or more:
//                    its members' roles (the first leads, the others go), and
//                    the position appended to the list of merged cells
//   k_merge_count    per block of Gaussians: how many are written
//   k_merge_scan     one CTA: each block's first output slot, the total
//   k_merge_write    per block of Gaussians: output slots; kept Gaussians copy
//                    parameters and moments (colour rows cooperatively); a
//                    leader records its slot for its cell
//   k_merge_cells    one warp per merged cell: the merged Gaussian (FP32,
//                    compensated sums over the members in index order, means
//                    relative to the first member), zero moments
//
// The arithmetic of a merged Gaussian is FP32 (this part's FP64 rate is a small
// fraction of its FP32 rate): Kahan-compensated sums keep each sum's error at a
// few units in the last place of its largest term whatever the number of
// members, and the means are summed as offsets from the first member (exact
// differences within a cell), so that the distances in the variance do not
// lose their digits to the cell's position.
#include <algorithm>
#include <type_traits>

#include "binning.cuh"

namespace igs {
namespace {

constexpr uint32_t kRoleKept = 0xFFFFFFFFu;  // not merged
constexpr uint32_t kRoleGone = 0xFFFFFFFEu;  // merged into an earlier Gaussian
constexpr int kMergeThreads = 256;
constexpr int kMergeScanThreads = 1024;

struct MergeArrays {
    const float4* ms;
    const float* op;
    const float* col;
    const float4* m_ms;
    const float* m_op;
    const float* m_col;
    const float4* v_ms;
    const float* v_op;
    const float* v_col;
};
struct MergeOut {
    float4* ms;
    float* op;
    float* col;
    float4* m_ms;
    float* m_op;
    float* m_col;
    float4* v_ms;
    float* v_op;
    float* v_col;
};

// Opacity floor of an eligible Gaussian, on the stored value: 2^-60 <= o <= 1,
// or logit >= -41.58883f (the FP32 value nearest the logit of 2^-60).
__device__ __forceinline__ bool opacity_eligible(float o, int param_mode) {
    return param_mode == 1 ? o >= -41.58883f : (o >= 0x1p-60f && o <= 1.0f);
}

// Linear opacity o and log(1 - o) of a stored value (logit with param_mode 1), FP32.
__device__ __forceinline__ void opacity_terms(float x, int param_mode, float& o, float& log_keep) {
    if (param_mode == 1) {
        const float e = expf(-fabsf(x));
        const float sp = log1pf(e);                       // softplus(-|x|)
        o = x >= 0.f ? 1.0f / (1.0f + e) : e / (1.0f + e);
        log_keep = -(x >= 0.f ? x + sp : sp);             // log(1 - sigmoid(x)) = -softplus(x)
    } else {
        o = x;
        log_keep = log1pf(-x);
    }
}

__global__ void __launch_bounds__(kMergeThreads) k_merge_keys(const float4* __restrict__ ms,
                                                              const float* __restrict__ op, int64_t n,
                                                              int param_mode, float lox, float loy, float loz,
                                                              float inv, float scale_max, uint32_t* __restrict__ key) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 m = ms[i];
    uint32_t k = 0xFFFFFFFFu;
    if (isfinite(m.x) && isfinite(m.y) && isfinite(m.z) && m.w <= scale_max && opacity_eligible(op[i], param_mode)) {
        const float cx = floorf(__fmul_rn(__fsub_rn(m.x, lox), inv));
        const float cy = floorf(__fmul_rn(__fsub_rn(m.y, loy), inv));
        const float cz = floorf(__fmul_rn(__fsub_rn(m.z, loz), inv));
        if (cx >= 0.f && cx < 1024.f && cy >= 0.f && cy < 1024.f && cz >= 0.f && cz < 1024.f)
            k = (uint32_t)cx | ((uint32_t)cy << 10) | ((uint32_t)cz << 20);
    }
    key[i] = k;
}

// Sorted items (key << 32 | index). A position that starts a cell of two or
// more eligible Gaussians marks its members: role[first] = the start position,
// role[other members] = gone; and appends the position to `cells`. role is
// kRoleKept everywhere on entry.
__global__ void __launch_bounds__(kMergeThreads) k_merge_mark(const u64* __restrict__ items, int64_t n,
                                                              uint32_t* __restrict__ role,
                                                              uint32_t* __restrict__ cells,
                                                              uint32_t* __restrict__ n_cells,
                                                              const uint32_t* __restrict__ info) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || info[kInfoAbort]) return;  // after a sort that gave up, the items are not a permutation
    const uint32_t key = (uint32_t)(items[p] >> 32);
    if (key == 0xFFFFFFFFu) return;
    if (p > 0 && (uint32_t)(items[p - 1] >> 32) == key) return;  // not the cell's first
    if (p + 1 >= n || (uint32_t)(items[p + 1] >> 32) != key) return;  // alone in its cell: kept
    role[(uint32_t)items[p]] = (uint32_t)p;
    for (int64_t r = p + 1; r < n && (uint32_t)(items[r] >> 32) == key; ++r) role[(uint32_t)items[r]] = kRoleGone;
    cells[atomicAdd(n_cells, 1u)] = (uint32_t)p;  // (list order is free: each cell's output slot is fixed)
    // (a cell of many Gaussians is marked by one thread: the cost grows with the
    // largest cell, not with n)
}

// Per block of kMergeThreads Gaussians: the number written (all but the gone).
__global__ void __launch_bounds__(kMergeThreads) k_merge_count(const uint32_t* __restrict__ role, int64_t n,
                                                               uint32_t* __restrict__ blk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool out = i < n && role[i] != kRoleGone;
    const uint32_t c = __syncthreads_count(out);
    if (threadIdx.x == 0) blk[blockIdx.x] = c;
}

// One CTA: the exclusive scan of the block counts in place, and the total
// (-1 when the sort gave up; nothing is written then).
__global__ void __launch_bounds__(kMergeScanThreads) k_merge_scan(uint32_t* __restrict__ blk, int64_t blocks,
                                                                  int64_t* __restrict__ d_count,
                                                                  const uint32_t* __restrict__ info) {
    if (info[kInfoAbort]) {
        if (threadIdx.x == 0) *d_count = -1;
        return;
    }
    __shared__ uint32_t s_warp[kMergeScanThreads / 32];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0) s_carry = 0ull;
    __syncthreads();
    for (int64_t b0 = 0; b0 < blocks; b0 += kMergeScanThreads) {
        const int64_t b = b0 + threadIdx.x;
        const uint32_t v = b < blocks ? blk[b] : 0u;
        const uint32_t ex = block_excl_scan<kMergeScanThreads>(v, s_warp);
        const unsigned long long carry = s_carry;
        if (b < blocks) blk[b] = (uint32_t)(carry + ex);
        __syncthreads();
        if (threadIdx.x == kMergeScanThreads - 1) s_carry = carry + ex + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *d_count = (int64_t)s_carry;
}

// Per block of kMergeThreads Gaussians: output slots by a block scan; kept
// Gaussians copy their means, scales, opacities and moments (one thread each)
// and then, cooperatively, their colour rows and moments (float4 when C is a
// multiple of 4); the leader of a merged cell records its slot at its cell's
// sorted start position (cell_slot, indexed like the sorted items).
template <int C>
__global__ void __launch_bounds__(kMergeThreads) k_merge_write(MergeArrays in, MergeOut out, int64_t n,
                                                               const uint32_t* __restrict__ role,
                                                               const uint32_t* __restrict__ blk,
                                                               uint32_t* __restrict__ cell_slot,
                                                               const uint32_t* __restrict__ info) {
    if (info[kInfoAbort]) return;
    __shared__ uint32_t s_warp[kMergeThreads / 32];
    __shared__ uint32_t s_dst[kMergeThreads];  // output slot of a kept Gaussian, else ~0
    const int64_t i0 = (int64_t)blockIdx.x * kMergeThreads, i = i0 + threadIdx.x;
    const uint32_t rl = i < n ? role[i] : kRoleGone;
    const bool emit = rl != kRoleGone;
    const uint32_t slot = blk[blockIdx.x] + block_excl_scan<kMergeThreads>(emit ? 1u : 0u, s_warp);
    s_dst[threadIdx.x] = rl == kRoleKept ? slot : 0xFFFFFFFFu;
    const size_t d = slot, s = (size_t)i;
    if (rl == kRoleKept) {
        out.ms[d] = in.ms[s];
        out.m_ms[d] = in.m_ms[s];
        out.v_ms[d] = in.v_ms[s];
        out.op[d] = in.op[s];
        out.m_op[d] = in.m_op[s];
        out.v_op[d] = in.v_op[s];
    } else if (emit) {
        cell_slot[rl] = slot;
    }
    __syncthreads();
    const int nr = (int)min((int64_t)kMergeThreads, n - i0);
    constexpr int V = (C % 4 == 0) ? 4 : 1;  // floats per access
    constexpr int CV = C / V;                // accesses per row
    using T = typename std::conditional<V == 4, float4, float>::type;
    const T* icol = reinterpret_cast<const T*>(in.col);
    const T* imc = reinterpret_cast<const T*>(in.m_col);
    const T* ivc = reinterpret_cast<const T*>(in.v_col);
    T* ocol = reinterpret_cast<T*>(out.col);
    T* omc = reinterpret_cast<T*>(out.m_col);
    T* ovc = reinterpret_cast<T*>(out.v_col);
    for (int q = threadIdx.x; q < nr * CV; q += kMergeThreads) {
        const int j = q / CV, f = q - j * CV;
        const uint32_t dj = s_dst[j];
        if (dj == 0xFFFFFFFFu) continue;
        const size_t src = (size_t)(i0 + j) * CV + f, dst = (size_t)dj * CV + f;
        ocol[dst] = icol[src];
        omc[dst] = imc[src];
        ovc[dst] = ivc[src];
    }
}

// Kahan-compensated sum (s, c): add x.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Add the x of lanes 0..cnt-1 to (s, c) in lane order (the same in every lane).
__device__ __forceinline__ void kahan_lanes(float& s, float& c, float x, int cnt) {
    for (int j = 0; j < cnt; ++j) kahan_add(s, c, __shfl_sync(0xffffffffu, x, j));
}

// One warp per merged cell (a grid-stride loop over the list of cells): lane j
// holds member j of each run of 32 (index order), and every sum adds the
// members' terms in index order; colour coefficient c is lane c mod 32's.
template <int C>
__global__ void __launch_bounds__(kMergeThreads) k_merge_cells(MergeArrays in, MergeOut out, int64_t n,
                                                               int param_mode, const u64* __restrict__ items,
                                                               const uint32_t* __restrict__ cells,
                                                               const uint32_t* __restrict__ n_cells,
                                                               const uint32_t* __restrict__ cell_slot,
                                                               const uint32_t* __restrict__ info) {
    if (info[kInfoAbort]) return;
    const int lane = threadIdx.x & 31;
    const uint32_t total = *n_cells;
    const uint32_t warps = gridDim.x * (kMergeThreads / 32);
    for (uint32_t g = blockIdx.x * (kMergeThreads / 32) + (threadIdx.x >> 5); g < total; g += warps) {
        const int64_t p0 = cells[g];
        const uint32_t key = (uint32_t)(items[p0] >> 32);
        const size_t d = cell_slot[p0];
        const float4 m0 = in.ms[(uint32_t)items[p0]];  // the first member: origin of the offsets
        // W = sum o_k, offsets sum o_k (mu_k - mu_0), L = sum log(1 - o_k) over the members
        float W = 0.f, cW = 0.f, ox = 0.f, cx = 0.f, oy = 0.f, cy = 0.f, oz = 0.f, cz = 0.f, L = 0.f, cL = 0.f;
        bool opaque = false;  // a member of opacity 1: the coverage is 1
        int64_t end = p0;
        // this lane's member of the first run, kept for the later passes when
        // the cell has at most 32 members (the common case)
        uint32_t k1 = 0;
        float4 m1 = make_float4(0.f, 0.f, 0.f, 0.f);
        float o1 = 0.f;
        for (int64_t b = p0;; b += 32) {
            const int64_t r = b + lane;
            const bool mem = r < n && (uint32_t)(items[r] >> 32) == key;
            const uint32_t ball = __ballot_sync(0xffffffffu, mem);
            const int cnt = ball == 0xffffffffu ? 32 : __ffs(~ball) - 1;  // members in this run
            float o = 0.f, x = 0.f, y = 0.f, z = 0.f, lk = 0.f;
            if (lane < cnt) {
                const uint32_t k = (uint32_t)items[r];
                const float4 m = in.ms[k];
                opacity_terms(in.op[k], param_mode, o, lk);
                x = __fmul_rn(o, __fsub_rn(m.x, m0.x));
                y = __fmul_rn(o, __fsub_rn(m.y, m0.y));
                z = __fmul_rn(o, __fsub_rn(m.z, m0.z));
                if (b == p0) {
                    k1 = k;
                    m1 = m;
                    o1 = o;
                }
            }
            opaque |= __any_sync(0xffffffffu, lane < cnt && isinf(lk));
            if (isinf(lk)) lk = 0.f;
            kahan_lanes(W, cW, o, cnt);
            kahan_lanes(ox, cx, x, cnt);
            kahan_lanes(oy, cy, y, cnt);
            kahan_lanes(oz, cz, z, cnt);
            kahan_lanes(L, cL, lk, cnt);
            end = b + cnt;
            if (cnt < 32) break;
        }
        const float ex = __fdiv_rn(ox, W), ey = __fdiv_rn(oy, W), ez = __fdiv_rn(oz, W);  // mean - mu_0
        const bool one_run = end - p0 <= 32;
        float V = 0.f, cV = 0.f;  // sum o_k (sigma_k^2 + |mu_k - mu|^2 / 3)
        for (int64_t b = p0; b < end; b += 32) {
            const int cnt = (int)min((int64_t)32, end - b);
            float t = 0.f;
            if (lane < cnt) {
                uint32_t k = k1;
                float4 m = m1;
                float o = o1;
                if (!one_run) {
                    k = (uint32_t)items[b + lane];
                    m = in.ms[k];
                    float lk;
                    opacity_terms(in.op[k], param_mode, o, lk);
                }
                const float sk = param_mode == 1 ? expf(m.w) : m.w;
                const float dx = __fsub_rn(__fsub_rn(m.x, m0.x), ex), dy = __fsub_rn(__fsub_rn(m.y, m0.y), ey),
                            dz = __fsub_rn(__fsub_rn(m.z, m0.z), ez);
                const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                t = __fmul_rn(o, __fadd_rn(__fmul_rn(sk, sk), __fdiv_rn(d2, 3.0f)));
            }
            kahan_lanes(V, cV, t, cnt);
        }
        if (lane == 0) {
            const float sigma = sqrtf(__fdiv_rn(V, W));
            const float cover = opaque ? 1.0f : -expm1f(L);  // 1 - prod (1 - o_k)
            float o_out;
            if (param_mode == 1)  // logit: log(cover) - log(1 - cover), or that of 0.99
                o_out = cover >= 0.99f ? logf(99.0f) : __fsub_rn(logf(cover), L);
            else
                o_out = fminf(cover, 0.99f);
            out.ms[d] = make_float4(__fadd_rn(m0.x, ex), __fadd_rn(m0.y, ey), __fadd_rn(m0.z, ez),
                                    param_mode == 1 ? logf(sigma) : sigma);
            out.op[d] = o_out;
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            out.m_ms[d] = zero;
            out.v_ms[d] = zero;
            out.m_op[d] = 0.f;
            out.v_op[d] = 0.f;
        }
        // colour: coefficients lane, lane + 32, ...: sum o_k c_k / W
        constexpr int CP = (C + 31) / 32;  // coefficients per lane
        float acc[CP], cacc[CP];
#pragma unroll
        for (int t = 0; t < CP; ++t) acc[t] = cacc[t] = 0.f;
        for (int64_t b = p0; b < end; b += 32) {
            const int cnt = (int)min((int64_t)32, end - b);
            uint32_t k = k1;
            float o = o1;
            if (!one_run && lane < cnt) {
                k = (uint32_t)items[b + lane];
                float lk;
                opacity_terms(in.op[k], param_mode, o, lk);
            }
            for (int j0 = 0; j0 < cnt; j0 += 4) {  // the rows of four members loaded together
                float v[4][CP], w4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u;
                    const uint32_t kj = __shfl_sync(0xffffffffu, k, j & 31);
                    w4[u] = __shfl_sync(0xffffffffu, o, j & 31);
                    const float* row = in.col + (size_t)kj * C;
#pragma unroll
                    for (int t = 0; t < CP; ++t) {
                        const int c = lane + 32 * t;
                        v[u][t] = (j < cnt && c < C) ? row[c] : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (j0 + u < cnt)
#pragma unroll
                        for (int t = 0; t < CP; ++t)
                            if (lane + 32 * t < C) kahan_add(acc[t], cacc[t], __fmul_rn(w4[u], v[u][t]));
            }
        }
#pragma unroll
        for (int t = 0; t < CP; ++t) {
            const int c = lane + 32 * t;
            if (c < C) {
                out.col[d * C + c] = __fdiv_rn(acc[t], W);
                out.m_col[d * C + c] = 0.f;
                out.v_col[d * C + c] = 0.f;
            }
        }
    }
}

// Work layout (all 256-byte aligned pieces).
struct MergeWork {
    uint32_t* key;      // [n] cell keys; after the sort, the output slot of each merged cell (by sorted start)
    uint32_t* cells;    // [n] sorted start positions of the merged cells
    u64* items_a;       // [n]
    u64* items_b;       // [n]
    uint32_t* role;     // [n]
    uint32_t* blk;      // [blocks]
    uint32_t* hist;     // [4][256]
    uint32_t* status;   // [4][sort blocks][256]
    uint32_t* counters; // [16]
    uint32_t* info;     // [16]
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

MergeWork merge_work(void* w, int64_t n, size_t* bytes) {
    const int64_t blocks = std::max<int64_t>(1, ceil_div(n, kMergeThreads));
    const int64_t sb = std::max<int64_t>(1, ceil_div(n, kSortTile));
    char* p = static_cast<char*>(w);
    size_t off = 0;
    auto take = [&](size_t b) { char* q = p ? p + off : nullptr; off += al256(b); return q; };
    MergeWork m;
    m.key = (uint32_t*)take((size_t)n * 4);
    m.cells = (uint32_t*)take((size_t)n * 4);
    m.items_a = (u64*)take((size_t)n * 8);
    m.items_b = (u64*)take((size_t)n * 8);
    m.role = (uint32_t*)take((size_t)n * 4);
    m.blk = (uint32_t*)take((size_t)blocks * 4);
    m.hist = (uint32_t*)take(4 * kRadix * 4);
    m.status = (uint32_t*)take((size_t)4 * sb * kRadix * 4);
    m.counters = (uint32_t*)take(16 * 4);
    m.info = (uint32_t*)take(16 * 4);
    if (bytes) *bytes = off;
    return m;
}

}  // namespace

size_t merge_work_bytes(int64_t n) {
    size_t b = 0;
    merge_work(nullptr, n, &b);
    return b;
}

cudaError_t launch_merge(const float* const in_p[3], const float* const in_m[3], const float* const in_v[3], int64_t n,
                         int C, int param_mode, const float lo[3], float cell, float scale_max, float* const out_p[3],
                         float* const out_m[3], float* const out_v[3], int64_t* d_count, void* work,
                         cudaStream_t st) {
    cudaError_t e;
#define CK(x) do { if ((e = (x)) != cudaSuccess) { g_failed_call = #x " (merge.cu:" IGS_STR(__LINE__) ")"; return e; } } while (0)
    if (n == 0) return cudaMemsetAsync(d_count, 0, 8, st);
    const MergeWork w = merge_work(work, n, nullptr);
    const int64_t blocks = ceil_div(n, kMergeThreads), sb = ceil_div(n, kSortTile);
    const uint32_t nn = (uint32_t)n;
    const float inv = 1.0f / cell;
    CK(cudaMemsetAsync(w.hist, 0, 4 * kRadix * 4, st));
    CK(cudaMemsetAsync(w.status, 0, (size_t)4 * sb * kRadix * 4, st));
    CK(cudaMemsetAsync(w.counters, 0, 16 * 4, st));
    CK(cudaMemsetAsync(w.info, 0, 16 * 4, st));
    CK(cudaMemsetAsync(w.role, 0xFF, (size_t)n * 4, st));
    k_merge_keys<<<(unsigned)blocks, kMergeThreads, 0, st>>>(reinterpret_cast<const float4*>(in_p[0]), in_p[1], n,
                                                              param_mode, lo[0], lo[1], lo[2], inv, scale_max, w.key);
    count_launches();
    CK(cudaGetLastError());
    k_hist<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 4), 256, 0, st>>>(w.key, nn, 4, w.hist);
    count_launches();
    CK(cudaGetLastError());
    k_hist_to_offsets<<<1, 1024, 0, st>>>(w.hist, 4);
    count_launches();
    CK(cudaGetLastError());
    for (int p = 0; p < 4; ++p) {  // (key, index) -> A -> B -> A -> B
        uint32_t* status = w.status + (size_t)p * sb * kRadix;
        const uint32_t* hist = w.hist + p * kRadix;
        if (p == 0)
            k_radix_pass<true, false><<<(unsigned)sb, kSortThreads, 0, st>>>(w.key, w.items_a, nullptr, nn, 0, hist,
                                                                             status, w.counters + p, w.info);
        else
            k_radix_pass<false, false><<<(unsigned)sb, kSortThreads, 0, st>>>(
                p % 2 ? w.items_a : w.items_b, p % 2 ? w.items_b : w.items_a, nullptr, nn, 8 * p, hist, status,
                w.counters + p, w.info);
        count_launches();
        CK(cudaGetLastError());
    }
    const u64* sorted = w.items_b;
    k_merge_mark<<<(unsigned)blocks, kMergeThreads, 0, st>>>(sorted, n, w.role, w.cells, w.counters + 8, w.info);
    count_launches();
    CK(cudaGetLastError());
    k_merge_count<<<(unsigned)blocks, kMergeThreads, 0, st>>>(w.role, n, w.blk);
    count_launches();
    CK(cudaGetLastError());
    k_merge_scan<<<1, kMergeScanThreads, 0, st>>>(w.blk, blocks, d_count, w.info);
    count_launches();
    CK(cudaGetLastError());
    MergeArrays in{reinterpret_cast<const float4*>(in_p[0]), in_p[1], in_p[2], reinterpret_cast<const float4*>(in_m[0]),
                   in_m[1], in_m[2], reinterpret_cast<const float4*>(in_v[0]), in_v[1], in_v[2]};
    MergeOut out{reinterpret_cast<float4*>(out_p[0]), out_p[1], out_p[2], reinterpret_cast<float4*>(out_m[0]),
                 out_m[1], out_m[2], reinterpret_cast<float4*>(out_v[0]), out_v[1], out_v[2]};
    uint32_t* cell_slot = w.key;  // the keys are not read after the first radix pass
    const unsigned cell_blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 16), 152 * 8));
    switch (C) {  // colour floats per Gaussian: a compile-time row length for the cooperative copies
#define IGS_MERGE_C(CC)                                                                                             \
    case CC:                                                                                                        \
        k_merge_write<CC><<<(unsigned)blocks, kMergeThreads, 0, st>>>(in, out, n, w.role, w.blk, cell_slot, w.info); \
        count_launches();                                                                                           \
        CK(cudaGetLastError());                                                                                     \
        k_merge_cells<CC><<<cell_blocks, kMergeThreads, 0, st>>>(in, out, n, param_mode, sorted, w.cells,            \
                                                                 w.counters + 8, cell_slot, w.info);                \
        count_launches();                                                                                           \
        CK(cudaGetLastError());                                                                                     \
        break;
        IGS_MERGE_C(3)
        IGS_MERGE_C(12)
        IGS_MERGE_C(27)
        IGS_MERGE_C(48)
#undef IGS_MERGE_C
        default: return cudaErrorInvalidValue;
    }
#undef CK
    return cudaSuccess;
}

}  // namespace igs
