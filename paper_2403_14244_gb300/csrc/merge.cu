// Merging of the 3D Gaussians (Sec. 3.2: particles may be merged or divided;
// Sec. 2.5's multiscale property; the Octree of Sec. 3.1 as the pattern, so a
// merge is the inverse of the octant division): the eligible Gaussians that
// share a cell of a grid, two or more of them, become one Gaussian at the
// place of the first; every other Gaussian is kept. Output in index order.
//
//   k_merge_keys     per Gaussian: its cell key (x | y << 10 | z << 20) if it
//                    is eligible, else 0xFFFFFFFF (FP32 cell indices, each step
//                    rounded once)
//   k_hist, 4 passes stable radix sort of (key, index): a cell's Gaussians end
//                    up together, in index order
//   k_merge_mark     per sorted position that starts a cell of two or more:
//                    its members' roles (the first leads, the others go)
//   k_merge_count    per block of Gaussians: how many are written
//   k_merge_scan     one CTA: each block's first output slot, the total
//   k_merge_write    per Gaussian: kept ones copy parameters and moments; a
//                    leader writes the merged Gaussian (FP64 sums over its
//                    members in index order) with zero moments
#include <algorithm>

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

// Linear opacity of a stored value (logit with param_mode 1), in FP64.
__device__ __forceinline__ double lin_opacity(float o, int param_mode) {
    return param_mode == 1 ? __ddiv_rn(1.0, __dadd_rn(1.0, exp(-(double)o))) : (double)o;
}

__global__ void __launch_bounds__(kMergeThreads) k_merge_keys(const float4* __restrict__ ms,
                                                              const float* __restrict__ op, int64_t n,
                                                              int param_mode, float lox, float loy, float loz,
                                                              float inv, float scale_max, uint32_t* __restrict__ key) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 m = ms[i];
    uint32_t k = 0xFFFFFFFFu;
    if (isfinite(m.x) && isfinite(m.y) && isfinite(m.z) && m.w <= scale_max && lin_opacity(op[i], param_mode) > 0.0) {
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
// role[other members] = gone. role is kRoleKept everywhere on entry.
__global__ void __launch_bounds__(kMergeThreads) k_merge_mark(const u64* __restrict__ items, int64_t n,
                                                              uint32_t* __restrict__ role,
                                                              const uint32_t* __restrict__ info) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || info[kInfoAbort]) return;  // after a sort that gave up, the items are not a permutation
    const uint32_t key = (uint32_t)(items[p] >> 32);
    if (key == 0xFFFFFFFFu) return;
    if (p > 0 && (uint32_t)(items[p - 1] >> 32) == key) return;  // not the cell's first
    if (p + 1 >= n || (uint32_t)(items[p + 1] >> 32) != key) return;  // alone in its cell: kept
    role[(uint32_t)items[p]] = (uint32_t)p;
    for (int64_t r = p + 1; r < n && (uint32_t)(items[r] >> 32) == key; ++r) role[(uint32_t)items[r]] = kRoleGone;
    // (a cell of many Gaussians is marked, and later merged, by one thread: the
    // cost grows with the largest cell, not with n)
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

__global__ void __launch_bounds__(kMergeThreads) k_merge_write(MergeArrays in, MergeOut out, int64_t n, int C,
                                                               int param_mode, const u64* __restrict__ items,
                                                               const uint32_t* __restrict__ role,
                                                               const uint32_t* __restrict__ blk,
                                                               const uint32_t* __restrict__ info) {
    if (info[kInfoAbort]) return;
    __shared__ uint32_t s_warp[kMergeThreads / 32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t rl = i < n ? role[i] : kRoleGone;
    const bool emit = rl != kRoleGone;
    const uint32_t slot = blk[blockIdx.x] + block_excl_scan<kMergeThreads>(emit ? 1u : 0u, s_warp);
    if (!emit) return;
    const size_t d = slot, s = (size_t)i;
    if (rl == kRoleKept) {
        out.ms[d] = in.ms[s];
        out.m_ms[d] = in.m_ms[s];
        out.v_ms[d] = in.v_ms[s];
        out.op[d] = in.op[s];
        out.m_op[d] = in.m_op[s];
        out.v_op[d] = in.v_op[s];
        for (int c = 0; c < C; ++c) {
            out.col[d * C + c] = in.col[s * C + c];
            out.m_col[d * C + c] = in.m_col[s * C + c];
            out.v_col[d * C + c] = in.v_col[s * C + c];
        }
        return;
    }
    // the cell's merged Gaussian: members are items[rl ...] while the key holds,
    // in index order; every FP64 product and sum rounded once (no fused
    // multiply-add), so with linear parameters the result is that of the plain
    // FP64 formulas evaluated term by term
    const uint32_t key = (uint32_t)(items[rl] >> 32);
    double W = 0.0, mx = 0.0, my = 0.0, mz = 0.0, keep = 1.0;
    int64_t end = rl;
    for (int64_t r = rl; r < n && (uint32_t)(items[r] >> 32) == key; ++r, ++end) {
        const uint32_t k = (uint32_t)items[r];
        const double ok = lin_opacity(in.op[k], param_mode);
        const float4 m = in.ms[k];
        W = __dadd_rn(W, ok);
        mx = __dadd_rn(mx, __dmul_rn(ok, (double)m.x));
        my = __dadd_rn(my, __dmul_rn(ok, (double)m.y));
        mz = __dadd_rn(mz, __dmul_rn(ok, (double)m.z));
        keep = __dmul_rn(keep, __dsub_rn(1.0, ok));
    }
    mx = __ddiv_rn(mx, W);
    my = __ddiv_rn(my, W);
    mz = __ddiv_rn(mz, W);
    double var = 0.0;
    for (int64_t r = rl; r < end; ++r) {
        const uint32_t k = (uint32_t)items[r];
        const double ok = lin_opacity(in.op[k], param_mode);
        const float4 m = in.ms[k];
        const double sk = param_mode == 1 ? exp((double)m.w) : (double)m.w;
        const double dx = __dsub_rn((double)m.x, mx), dy = __dsub_rn((double)m.y, my), dz = __dsub_rn((double)m.z, mz);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        var = __dadd_rn(var, __dmul_rn(ok, __dadd_rn(__dmul_rn(sk, sk), __ddiv_rn(d2, 3.0))));
    }
    var = __ddiv_rn(var, W);
    const double sigma = __dsqrt_rn(var);
    const double o = fmin(__dsub_rn(1.0, keep), 0.99);
    out.ms[d] = make_float4((float)mx, (float)my, (float)mz, param_mode == 1 ? (float)log(sigma) : (float)sigma);
    out.op[d] = param_mode == 1 ? (float)log(__ddiv_rn(o, __dsub_rn(1.0, o))) : (float)o;
    for (int c = 0; c < C; ++c) {
        double acc = 0.0;
        for (int64_t r = rl; r < end; ++r) {
            const uint32_t k = (uint32_t)items[r];
            acc = __dadd_rn(acc, __dmul_rn(lin_opacity(in.op[k], param_mode), (double)in.col[(size_t)k * C + c]));
        }
        out.col[d * C + c] = (float)__ddiv_rn(acc, W);
        out.m_col[d * C + c] = 0.f;
        out.v_col[d * C + c] = 0.f;
    }
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    out.m_ms[d] = zero;
    out.v_ms[d] = zero;
    out.m_op[d] = 0.f;
    out.v_op[d] = 0.f;
}

// Work layout (all 256-byte aligned pieces).
struct MergeWork {
    uint32_t* key;      // [n]
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
    k_merge_mark<<<(unsigned)blocks, kMergeThreads, 0, st>>>(sorted, n, w.role, w.info);
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
    k_merge_write<<<(unsigned)blocks, kMergeThreads, 0, st>>>(in, out, n, C, param_mode, sorted, w.role, w.blk, w.info);
    count_launches();
    CK(cudaGetLastError());
#undef CK
    return cudaSuccess;
}

}  // namespace igs
