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
// One CTA finds that prefix by bisection on the 64-bit error key, weighted by
// the leaves each split adds, and then on the id among equal keys.
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

constexpr int kOctThreads = 1024;

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

__device__ __forceinline__ long long block_sum(long long v, long long* s_tmp) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = v;
    __syncthreads();
    long long t = 0;
    for (int i = 0; i < kOctThreads / 32; ++i) t += s_tmp[i];
    return t;
}

__device__ __forceinline__ int oct_level(long long id) {
    int l = 0;
    while (oct_off(l + 1) <= id) ++l;
    return l;
}

// One CTA: keys and increments of every cell below the finest level, the split
// prefix of the order, and the split flags.
__global__ void __launch_bounds__(kOctThreads) k_oct_select(const OctCell* __restrict__ st, OctParams P,
                                                           unsigned long long* __restrict__ keys,
                                                           uint8_t* __restrict__ inc8, uint8_t* __restrict__ split) {
    __shared__ long long s_tmp[kOctThreads / 32];
    const long long items = oct_off(P.L);
    // key = min(error, parent's key), level by level (keeps every child after its
    // parent in the order whatever the rounding), as bits ordered like the value
    for (int l = 0; l < P.L; ++l) {
        for (long long m = threadIdx.x; m < (1LL << (3 * l)); m += kOctThreads) {
            const long long id = oct_off(l) + m;
            double k = oct_err(st[id]);
            if (l > 0) k = fmin(k, __longlong_as_double((long long)keys[oct_off(l - 1) + (m >> 3)]));
            keys[id] = (unsigned long long)__double_as_longlong(k);
            inc8[id] = (uint8_t)oct_inc(st, id, l, P.L);
        }
        __syncthreads();
    }
    const bool root = st[0].n > 0;
    // W(X) = sum of the increments of splittable cells with key >= X
    auto W = [&](unsigned long long X) {
        long long w = 0;
        for (long long i = threadIdx.x; i < items; i += kOctThreads)
            if (inc8[i] != 0xFFu && keys[i] >= X) w += inc8[i];
        return block_sum(w, s_tmp);
    };
    bool all = true;
    unsigned long long X = 0;
    long long Ihi = -1;
    if (root && 1 + W(0) > P.k_max) {
        all = false;
        // X = max{X : 1 + W(X) > k_max}; invariant: 1 + W(lo) > k_max, 1 + W(hi + 1) <= k_max
        unsigned long long lo = 0, hi = ~0ULL;
        while (lo < hi) {
            const unsigned long long mid = lo + (hi - lo) / 2 + 1;
            if (1 + W(mid) > P.k_max) lo = mid; else hi = mid - 1;
        }
        X = lo;
        long long gt = 0;
        for (long long i = threadIdx.x; i < items; i += kOctThreads)
            if (inc8[i] != 0xFFu && keys[i] > X) gt += inc8[i];
        const long long base = 1 + block_sum(gt, s_tmp);  // <= k_max
        // Ihi = max{I : base + sum of increments of cells with key == X and id <= I <= k_max} (-1: none)
        long long a = -1, b = items - 1;
        while (a < b) {
            const long long mid = a + (b - a + 1) / 2;
            long long w = 0;
            for (long long i = threadIdx.x; i <= mid; i += kOctThreads)
                if (inc8[i] != 0xFFu && keys[i] == X) w += inc8[i];
            if (base + block_sum(w, s_tmp) <= P.k_max) a = mid; else b = mid - 1;
        }
        Ihi = a;
    }
    for (long long i = threadIdx.x; i < items; i += kOctThreads) {
        bool sp = false;
        if (root && inc8[i] != 0xFFu) sp = all || keys[i] > X || (keys[i] == X && i <= Ihi);
        split[i] = sp ? 1 : 0;
    }
}

// One CTA: the non-empty leaves in id order, one Gaussian each.
__global__ void __launch_bounds__(kOctThreads) k_oct_emit(const OctCell* __restrict__ st,
                                                         const uint8_t* __restrict__ split, OctParams P,
                                                         float4* __restrict__ out_ms, float* __restrict__ out_op,
                                                         float* __restrict__ out_col, int32_t* __restrict__ count) {
    __shared__ int s_warp[kOctThreads / 32];
    __shared__ long long s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long cells = oct_off(P.L + 1);
    for (long long c0 = 0; c0 < cells; c0 += kOctThreads) {
        const long long id = c0 + threadIdx.x;
        bool leaf = false;
        int l = 0;
        long long m = 0;
        if (id < cells && st[id].n > 0) {
            l = oct_level(id);
            m = id - oct_off(l);
            const bool parent_split = l == 0 || split[oct_off(l - 1) + (m >> 3)];
            leaf = parent_split && (l == P.L || !split[id]);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, leaf);
        if (lane == 0) s_warp[w] = __popc(bal);
        __syncthreads();
        long long before = s_base, total = 0;
        for (int i = 0; i < kOctThreads / 32; ++i) {
            if (i < w) before += s_warp[i];
            total += s_warp[i];
        }
        const long long pos = before + __popc(bal & ((1u << lane) - 1u));
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
            float* cc = out_col + (size_t)P.C * pos;
            for (int k = 3; k < P.C; ++k) cc[k] = 0.f;
            for (int ch = 0; ch < 3; ++ch) {
                const double mean = __ddiv_rn((double)s.s1[ch], __dmul_rn(4096.0, (double)s.n));
                cc[ch] = P.sh < 0 ? (float)mean : (float)__ddiv_rn(__dsub_rn(mean, 0.5), P.y00);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = (int32_t)min(s_base, P.k_max);
}

}  // namespace

size_t octree_work_bytes(int L) {
    if (L < 0 || L > 7) return 0;
    const size_t cells = (size_t)oct_off(L + 1), items = (size_t)oct_off(L);
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return up(cells * sizeof(OctCell)) + up(items * 8) + up(items + 1) + up(items + 1);
}

cudaError_t launch_octree_init(const float* pts, const float* cols, long long npts, const float lo[3], float side,
                               int L, long long k_max, float opacity, int sh_degree, int param_mode, float* out_ms,
                               float* out_op, float* out_col, int32_t* count, void* work, cudaStream_t st) {
    const size_t cells = (size_t)oct_off(L + 1), items = (size_t)oct_off(L);
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    char* w = static_cast<char*>(work);
    auto* stats = reinterpret_cast<OctCell*>(w);
    auto* keys = reinterpret_cast<unsigned long long*>(w + up(cells * sizeof(OctCell)));
    auto* inc8 = reinterpret_cast<uint8_t*>(w + up(cells * sizeof(OctCell)) + up(items * 8));
    auto* split = inc8 + up(items + 1);
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
    k_oct_select<<<1, kOctThreads, 0, st>>>(stats, P, keys, inc8, split);
    k_oct_emit<<<1, kOctThreads, 0, st>>>(stats, split, P, reinterpret_cast<float4*>(out_ms), out_op, out_col,
                                          count);
    launches += 2;
    count_launches(launches);
    return cudaGetLastError();
}

}  // namespace igs
