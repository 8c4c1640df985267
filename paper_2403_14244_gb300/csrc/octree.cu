// Octree initialisation of 3D Gaussians (Sec. 3.1: an Octree for 3D, as the
// QuadTree for 2D; colour = the cell average, sigma = half the cell width), from
// a coloured point set.
//
// Cells of level l (0 = the whole cube) are cubes of side side / 2^l, id =
// (8^l - 1) / 7 + Morton index (x lowest). Each holds the exact integer sums n,
// S1_c, S2_c of its points' colours quantised to 12 bits. The greedy growth
// (split the splittable leaf of largest error first, while the non-empty leaves
// stay within the budget) splits a prefix of the order (error descending, id
// ascending) over the splittable cells: a cell's error is never below a child's
// (the children partition its points) and its id is smaller, so every cell
// comes after its ancestors, and the greedy stops at the first cell of the
// order whose split (adding its non-empty children minus one) does not fit.
// The prefix is found by a radix selection on the 64-bit key (8 bits at a time,
// histograms weighted by the leaves each split adds), and then on the id among
// equal keys: each pass a histogram over all cells by many CTAs, then a scan of
// its 256 bins by one CTA picks the digit. The leaves are then emitted in id
// order, a CTA per chunk of cells placed after the leaves of the chunks before it.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace igs {
namespace {

struct OctCell {
    unsigned long long n, s1[3], s2[3];
};

__host__ __device__ inline long long oct_off(int l) { return (((long long)1 << (3 * l)) - 1) / 7; }

__device__ __forceinline__ uint32_t oct_morton(uint32_t x, uint32_t y, uint32_t z, int L) {
    uint32_t m = 0;
    for (int b = 0; b < L; ++b)
        m |= (((x >> b) & 1u) << (3 * b)) | (((y >> b) & 1u) << (3 * b + 1)) | (((z >> b) & 1u) << (3 * b + 2));
    return m;
}

struct OctParams {
    float lo[3];
    float inv;            // 2^L / side (FP32)
    double side;
    double y00;           // 1 / (2 sqrt(pi)), for the SH DC coefficient
    float log_half[8];    // per level: log(side / 2^(l+1)) (param_mode 1) or side / 2^(l+1)
    float op_value;       // stored opacity (logit with param_mode 1)
    int L, C, sh;
    long long k_max;
};

__global__ void k_oct_base(const float* __restrict__ pts, const float* __restrict__ cols, long long npts,
                           OctParams P, OctCell* __restrict__ st) {
    const int top = (1 << P.L) - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts;
         i += (long long)gridDim.x * blockDim.x) {
        const float px = pts[3 * i], py = pts[3 * i + 1], pz = pts[3 * i + 2];
        if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) continue;
        const float p3[3] = {px, py, pz};
        uint32_t ix[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float t = floorf(__fmul_rn(__fsub_rn(p3[a], P.lo[a]), P.inv));
            ix[a] = t < 0.f ? 0u : (t > (float)top ? (uint32_t)top : (uint32_t)t);
        }
        OctCell* c = st + oct_off(P.L) + oct_morton(ix[0], ix[1], ix[2], P.L);
        atomicAdd(&c->n, 1ull);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float v = fminf(fmaxf(cols[3 * i + ch], 0.f), 1.f);
            const unsigned long long q = (unsigned long long)rintf(__fmul_rn(v, 4096.f));
            atomicAdd(&c->s1[ch], q);
            atomicAdd(&c->s2[ch], q * q);
        }
    }
}

__global__ void k_oct_up(OctCell* __restrict__ st, int l) {
    const long long cells = 1LL << (3 * l);
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < cells;
         m += (long long)gridDim.x * blockDim.x) {
        OctCell s;
        s.n = 0;
        for (int ch = 0; ch < 3; ++ch) s.s1[ch] = s.s2[ch] = 0;
        for (int d = 0; d < 8; ++d) {
            const OctCell& k = st[oct_off(l + 1) + 8 * m + d];
            s.n += k.n;
            for (int ch = 0; ch < 3; ++ch) {
                s.s1[ch] += k.s1[ch];
                s.s2[ch] += k.s2[ch];
            }
        }
        st[oct_off(l) + m] = s;
    }
}

constexpr int kOctThreads = 256;
constexpr int kOctChunk = kOctThreads * 8;  // cells per CTA of the emission
constexpr int kOctPasses = 11;              // 8 digits of the key, then 3 of the id (ids < 2^24)

// Error of a cell: max(0, sum_c (S2_c - S1_c^2 / n)) in double, one rounding per
// step in channel order (0 for an empty cell).
__device__ __forceinline__ double oct_err(const OctCell& c) {
    if (c.n == 0) return 0.0;
    const double n = (double)c.n;
    double e = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
        const double s1 = (double)c.s1[ch];
        e = __dadd_rn(e, __dsub_rn((double)c.s2[ch], __ddiv_rn(__dmul_rn(s1, s1), n)));
    }
    return e > 0.0 ? e : 0.0;
}

// The leaves a split of cell id (level l) adds (non-empty children - 1), or
// 0xFF if the cell cannot split (fewer than 2 points, or the finest level).
__device__ __forceinline__ uint32_t oct_inc(const OctCell* __restrict__ st, long long id, int l, int L) {
    if (l >= L || st[id].n < 2) return 0xFFu;
    const long long m = id - oct_off(l);
    uint32_t kids = 0;
    for (int d = 0; d < 8; ++d) kids += st[oct_off(l + 1) + 8 * m + d].n > 0;
    return kids - 1;
}

__device__ __forceinline__ int oct_level(long long id) {
    int l = 0;
    while (oct_off(l + 1) <= id) ++l;
    return l;
}

// The selection's state between passes. X = max{X : 1 + W(X) > k_max}, W(X) the
// increments of the splittable cells with key >= X, is found 8 bits at a time
// from the top: `above` = 1 + the increments of keys whose fixed high bits exceed
// `prefix`. Then, among keys == X, the first id (in id order) whose cumulative
// increments no longer fit k_max - above is found the same way on the id bits.
struct OctSel {
    unsigned long long prefix;  // key bits fixed so far; X once the key passes end
    long long above;
    unsigned long long idp;     // id bits fixed so far
    long long below;            // increments of keys == X with ids below the fixed id bits
    long long ihi;              // the last id of key X that splits
    int done;                   // no pass left to run
    int all;                    // every splittable cell splits
};

// Keys and increments of level l (one launch per level, top down): key = min(error,
// parent's key), which keeps every child after its parent in the order whatever
// the rounding, stored as bits ordered like the value.
__global__ void k_oct_keys(const OctCell* __restrict__ st, int l, int L, unsigned long long* __restrict__ keys,
                           uint8_t* __restrict__ inc8) {
    const long long cells = 1LL << (3 * l);
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < cells;
         m += (long long)gridDim.x * blockDim.x) {
        const long long id = oct_off(l) + m;
        double k = oct_err(st[id]);
        if (l > 0) k = fmin(k, __longlong_as_double((long long)keys[oct_off(l - 1) + (m >> 3)]));
        keys[id] = (unsigned long long)__double_as_longlong(k);
        inc8[id] = (uint8_t)oct_inc(st, id, l, L);
    }
}

// One pass of the selection: the histogram, over one 8-bit digit, of the
// increments of the cells still in the running (a CTA-local histogram, then one
// atomic per bin and CTA).
__global__ void __launch_bounds__(kOctThreads) k_oct_hist(const unsigned long long* __restrict__ keys,
                                                          const uint8_t* __restrict__ inc8, long long items,
                                                          const OctSel* __restrict__ sel, int pass,
                                                          uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_h[256];
    if (sel->done) return;
    s_h[threadIdx.x] = 0;
    __syncthreads();
    const unsigned long long prefix = sel->prefix, idp = sel->idp;
    if (pass < 8) {
        const int sh = 8 * (7 - pass);
        const unsigned long long hi = pass == 0 ? 0ull : (~0ull << (sh + 8));
        for (long long i = blockIdx.x * (long long)kOctThreads + threadIdx.x; i < items;
             i += (long long)gridDim.x * kOctThreads) {
            const uint32_t c = inc8[i];
            if (c == 0xFFu || c == 0) continue;
            const unsigned long long k = keys[i];
            if ((k & hi) == prefix) atomicAdd(&s_h[(k >> sh) & 0xFFu], c);
        }
    } else {
        const int sh = 8 * (10 - pass);
        const unsigned long long hi = ~0ull << (sh + 8);
        for (long long i = blockIdx.x * (long long)kOctThreads + threadIdx.x; i < items;
             i += (long long)gridDim.x * kOctThreads) {
            const uint32_t c = inc8[i];
            if (c == 0xFFu || c == 0) continue;
            if (keys[i] == prefix && ((unsigned long long)i & hi) == idp)
                atomicAdd(&s_h[((unsigned long long)i >> sh) & 0xFFu], c);
        }
    }
    __syncthreads();
    if (s_h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], s_h[threadIdx.x]);
}

// One CTA of 256 fixes the pass's digit from its histogram: thread t holds one bin
// (bin 255 - t for the key, taken from the top; bin t for the id) and an
// inclusive scan gives each bin the increments at and above it (key) or at and
// below it (id).
__global__ void __launch_bounds__(256) k_oct_pick(const OctCell* __restrict__ st, const uint32_t* __restrict__ hist,
                                                  int pass, long long items, long long k_max,
                                                  OctSel* __restrict__ sel) {
    __shared__ long long s_scan[256];
    __shared__ OctSel s;
    __shared__ int s_b;
    const int t = threadIdx.x;
    const bool key = pass < 8;
    if (t == 0) {
        s = *sel;
        s_b = key ? 0 : 256;
    }
    __syncthreads();
    if (s.done) return;  // uniform over the CTA
    const int bin = key ? 255 - t : t;
    const long long h = hist[bin];
    long long v = h;
    s_scan[t] = v;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        const long long add = t >= o ? s_scan[t - o] : 0;
        __syncthreads();
        v += add;
        s_scan[t] = v;
        __syncthreads();
    }
    long long above = s.above;
    if (pass == 0) {
        // 1 + W(0): the leaves if every splittable cell split
        if (st[0].n == 0 || 1 + s_scan[255] <= k_max) {
            if (t == 0) {
                s.all = 1;
                s.done = 1;
                *sel = s;
            }
            return;
        }
        above = 1;
    }
    if (key) {
        // the highest digit at which above + the increments at and above it exceed k_max (0 if none)
        if (bin >= 1 && above + v > k_max) atomicMax(&s_b, bin);
    } else {
        // the lowest digit at which the increments of key X, in id order, leave k_max - above
        if (s.below + v > k_max - above) atomicMin(&s_b, bin);
    }
    __syncthreads();
    if (t != 0) return;
    const int d = s_b;
    if (key) {
        s.prefix |= (unsigned long long)d << (8 * (7 - pass));
        s.above = above + s_scan[255 - d] - (long long)hist[d];  // + the increments above digit d
    } else if (d == 256) {  // every cell of key X fits
        s.ihi = items - 1;
        s.done = 1;
    } else {
        s.idp |= (unsigned long long)d << (8 * (10 - pass));
        s.below += s_scan[d] - (long long)hist[d];  // + the increments below digit d
        if (pass == kOctPasses - 1) {
            s.ihi = (long long)s.idp - 1;  // idp: the first id whose increment does not fit
            s.done = 1;
        }
    }
    *sel = s;
}

__global__ void k_oct_split(const OctCell* __restrict__ st, const unsigned long long* __restrict__ keys,
                            const uint8_t* __restrict__ inc8, long long items, const OctSel* __restrict__ sel,
                            uint8_t* __restrict__ split) {
    const bool root = st[0].n > 0;
    const bool all = sel->all != 0;
    const unsigned long long X = sel->prefix;
    const long long ihi = sel->ihi;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < items;
         i += (long long)gridDim.x * blockDim.x) {
        bool sp = false;
        if (root && inc8[i] != 0xFFu) sp = all || keys[i] > X || (keys[i] == X && i <= ihi);
        split[i] = sp ? 1 : 0;
    }
}

// Whether cell id holds a Gaussian: non-empty, its parent split (or the root), and
// itself not split (or the finest level).
__device__ __forceinline__ bool oct_leaf(const OctCell* __restrict__ st, const uint8_t* __restrict__ split,
                                         long long id, long long cells, int L, int* lvl, long long* mor) {
    if (id >= cells || st[id].n == 0) return false;
    const int l = oct_level(id);
    const long long m = id - oct_off(l);
    *lvl = l;
    *mor = m;
    const bool parent_split = l == 0 || split[oct_off(l - 1) + (m >> 3)];
    return parent_split && (l == L || !split[id]);
}

__device__ __forceinline__ long long oct_block_sum(long long v, long long* s_tmp) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = v;
    __syncthreads();
    long long t = 0;
    for (int i = 0; i < kOctThreads / 32; ++i) t += s_tmp[i];
    return t;
}

// Leaves per chunk of kOctChunk cells.
__global__ void __launch_bounds__(kOctThreads) k_oct_count(const OctCell* __restrict__ st,
                                                           const uint8_t* __restrict__ split, int L,
                                                           uint32_t* __restrict__ chunk_leaves) {
    __shared__ long long s_tmp[kOctThreads / 32];
    const long long cells = oct_off(L + 1), c0 = (long long)blockIdx.x * kOctChunk;
    long long n = 0;
    for (int j = threadIdx.x; j < kOctChunk; j += kOctThreads) {
        int l;
        long long m;
        n += oct_leaf(st, split, c0 + j, cells, L, &l, &m);
    }
    n = oct_block_sum(n, s_tmp);
    if (threadIdx.x == 0) chunk_leaves[blockIdx.x] = (uint32_t)n;
}

// The non-empty leaves in id order, one Gaussian each: a CTA per chunk, placed
// after the leaves of the chunks before it.
__global__ void __launch_bounds__(kOctThreads) k_oct_emit(const OctCell* __restrict__ st,
                                                         const uint8_t* __restrict__ split,
                                                         const uint32_t* __restrict__ chunk_leaves, OctParams P,
                                                         float4* __restrict__ out_ms, float* __restrict__ out_op,
                                                         float* __restrict__ out_col, int32_t* __restrict__ count) {
    __shared__ long long s_tmp[kOctThreads / 32];
    __shared__ int s_warp[kOctThreads / 32];
    __shared__ float s_dc[3 * kOctThreads];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long before = 0;
    for (unsigned b = threadIdx.x; b < blockIdx.x; b += kOctThreads) before += chunk_leaves[b];
    long long base = oct_block_sum(before, s_tmp);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        *count = (int32_t)min(base + (long long)chunk_leaves[blockIdx.x], P.k_max);
    if (base >= P.k_max) return;  // uniform over the CTA
    const long long cells = oct_off(P.L + 1), c0 = (long long)blockIdx.x * kOctChunk;
    for (int j0 = 0; j0 < kOctChunk; j0 += kOctThreads) {
        const long long id = c0 + j0 + threadIdx.x;
        int l = 0;
        long long m = 0;
        const bool leaf = oct_leaf(st, split, id, cells, P.L, &l, &m);
        const uint32_t bal = __ballot_sync(0xffffffffu, leaf);
        if (lane == 0) s_warp[w] = __popc(bal);
        __syncthreads();
        long long pos = base, total = 0;
        for (int i = 0; i < kOctThreads / 32; ++i) {
            if (i < w) pos += s_warp[i];
            total += s_warp[i];
        }
        pos += __popc(bal & ((1u << lane) - 1u));
        if (leaf && pos < P.k_max) {
            const OctCell& s = st[id];
            uint32_t c3[3] = {0u, 0u, 0u};
            for (int b = 0; b < l; ++b)
                for (int a = 0; a < 3; ++a) c3[a] |= (uint32_t)((m >> (3 * b + a)) & 1) << b;
            const double cs = P.side / (double)(1 << l);
            out_ms[pos] = make_float4((float)__dadd_rn((double)P.lo[0], __dmul_rn((double)c3[0] + 0.5, cs)),
                                      (float)__dadd_rn((double)P.lo[1], __dmul_rn((double)c3[1] + 0.5, cs)),
                                      (float)__dadd_rn((double)P.lo[2], __dmul_rn((double)c3[2] + 0.5, cs)),
                                      P.log_half[l]);
            out_op[pos] = P.op_value;
            float* dc = s_dc + 3 * (pos - base);
            for (int ch = 0; ch < 3; ++ch) {
                const double mean = __ddiv_rn((double)s.s1[ch], __dmul_rn(4096.0, (double)s.n));
                dc[ch] = P.sh < 0 ? (float)mean : (float)__ddiv_rn(__dsub_rn(mean, 0.5), P.y00);
            }
        }
        __syncthreads();
        // the round's leaves hold positions [base, base + total): their colour rows are one
        // contiguous range, written by the whole CTA (DC from shared memory, the rest 0)
        const long long rows = min(total, P.k_max - base);
        for (long long i = threadIdx.x; i < rows * P.C; i += kOctThreads) {
            const long long r = i / P.C;
            const int k = (int)(i - r * P.C);
            out_col[(size_t)P.C * base + i] = k < 3 ? s_dc[3 * r + k] : 0.f;
        }
        base += total;
        __syncthreads();  // s_warp is rewritten by the next round
    }
}

}  // namespace

// Scratch: cell statistics, keys and increments of the cells above the finest
// level, split flags, leaves per emission chunk, the selection's state and its
// histograms (one per pass).
struct OctWork {
    OctCell* stats;
    unsigned long long* keys;
    uint8_t *inc8, *split;
    uint32_t* chunk_leaves;
    OctSel* sel;
    uint32_t* hist;
    size_t bytes;
};

OctWork oct_work(int L, void* base) {
    const size_t cells = (size_t)oct_off(L + 1), items = (size_t)oct_off(L);
    const size_t chunks = (cells + kOctChunk - 1) / kOctChunk;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const uintptr_t w = reinterpret_cast<uintptr_t>(base);
    OctWork o;
    size_t at = 0;
    o.stats = reinterpret_cast<OctCell*>(w + at);
    at += up(cells * sizeof(OctCell));
    o.keys = reinterpret_cast<unsigned long long*>(w + at);
    at += up(items * 8);
    o.inc8 = reinterpret_cast<uint8_t*>(w + at);
    at += up(items + 1);
    o.split = reinterpret_cast<uint8_t*>(w + at);
    at += up(items + 1);
    o.chunk_leaves = reinterpret_cast<uint32_t*>(w + at);
    at += up(chunks * 4);
    o.sel = reinterpret_cast<OctSel*>(w + at);  // the state and the histograms are zeroed together
    at += up(sizeof(OctSel));
    o.hist = reinterpret_cast<uint32_t*>(w + at);
    at += up((size_t)kOctPasses * 256 * 4);
    o.bytes = at;
    return o;
}

size_t octree_work_bytes(int L) {
    if (L < 0 || L > 7) return 0;
    return oct_work(L, nullptr).bytes;
}

cudaError_t launch_octree_init(const float* pts, const float* cols, long long npts, const float lo[3], float side,
                               int L, long long k_max, float opacity, int sh_degree, int param_mode, float* out_ms,
                               float* out_op, float* out_col, int32_t* count, void* work, cudaStream_t st) {
    const long long cells = oct_off(L + 1), items = oct_off(L);
    const OctWork o = oct_work(L, work);
    OctCell* stats = o.stats;
    OctParams P;
    for (int a = 0; a < 3; ++a) P.lo[a] = lo[a];
    P.inv = (float)((double)(1 << L) / (double)side);
    P.side = (double)side;
    P.y00 = 0.5 / std::sqrt(3.14159265358979323846);
    for (int l = 0; l < 8; ++l) {
        const double half = 0.5 * (double)side / (double)(1 << l);
        P.log_half[l] = param_mode == 1 ? (float)std::log(half) : (float)half;
    }
    P.op_value = param_mode == 1 ? (float)std::log((double)opacity / (1.0 - (double)opacity)) : opacity;
    P.L = L;
    P.sh = sh_degree;
    P.C = sh_degree < 0 ? 3 : 3 * (sh_degree + 1) * (sh_degree + 1);
    P.k_max = k_max;
    cudaError_t e = cudaMemsetAsync(stats + oct_off(L), 0, sizeof(OctCell) * ((size_t)1 << (3 * L)), st);
    if (e != cudaSuccess) return e;
    int launches = 0;
    if (npts > 0) {
        k_oct_base<<<(unsigned)std::min<long long>(ceil_div(npts, 256), 152 * 8), 256, 0, st>>>(pts, cols, npts, P,
                                                                                                stats);
        ++launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int l = L - 1; l >= 0; --l) {
        const long long n = 1LL << (3 * l);
        k_oct_up<<<(unsigned)std::min<long long>(ceil_div(n, 256), 152 * 8), 256, 0, st>>>(stats, l);
        ++launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int l = 0; l < L; ++l) {
        const long long n = 1LL << (3 * l);
        k_oct_keys<<<(unsigned)std::min<long long>(ceil_div(n, 256), 152 * 8), 256, 0, st>>>(stats, l, L, o.keys,
                                                                                           o.inc8);
        ++launches;
    }
    if (L > 0) {
        e = cudaMemsetAsync(o.sel, 0, reinterpret_cast<char*>(o.hist + kOctPasses * 256) -
                                          reinterpret_cast<char*>(o.sel), st);
        if (e != cudaSuccess) return e;
        const unsigned hblocks = (unsigned)std::min<long long>(ceil_div(items, kOctThreads * 4), 152 * 4);
        for (int pass = 0; pass < kOctPasses; ++pass) {
            k_oct_hist<<<hblocks, kOctThreads, 0, st>>>(o.keys, o.inc8, items, o.sel, pass, o.hist + 256 * pass);
            k_oct_pick<<<1, 256, 0, st>>>(stats, o.hist + 256 * pass, pass, items, k_max, o.sel);
            launches += 2;
        }
        k_oct_split<<<(unsigned)std::min<long long>(ceil_div(items, 256), 152 * 8), 256, 0, st>>>(
            stats, o.keys, o.inc8, items, o.sel, o.split);
        ++launches;
    }
    const unsigned chunks = (unsigned)ceil_div(cells, kOctChunk);
    k_oct_count<<<chunks, kOctThreads, 0, st>>>(stats, o.split, L, o.chunk_leaves);
    k_oct_emit<<<chunks, kOctThreads, 0, st>>>(stats, o.split, o.chunk_leaves, P, reinterpret_cast<float4*>(out_ms),
                                               out_op, out_col, count);
    launches += 2;
    count_launches(launches);
    return cudaGetLastError();
}

}  // namespace igs
