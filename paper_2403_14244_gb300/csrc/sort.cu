// Binning and sorting: front-to-back order of the kept Gaussians, their
// duplication into one entry per touched tile, a stable sort of the entries by
// tile id, and per-tile ranges.
//
// Eq. 4 composites each pixel front to back, so every tile needs its Gaussians
// in depth order. Instead of one radix sort over 64-bit (tile << 32 | depth)
// keys, this does:
//   1. a stable 32-bit LSD radix sort of the n depth keys (culled ones carry
//      0xFFFFFFFF and sort last), which gives `order`;
//   2. an exclusive scan of the tile counts in that order and the duplication
//      of each Gaussian, in that order, into (tile id, Gaussian id) entries;
//   3. a stable LSD radix sort of the M entries by tile id only
//      (ceil(log2(tiles) / 8) passes).
// Stability makes the result identical to the stable 64-bit key sort: within a
// tile, entries are in (depth bits, Gaussian index) order. The sort traffic per
// entry drops from 6 passes of 12-byte pairs to 2 passes of 8-byte pairs.
//
// Each radix pass is a single sweep (one read, one write of the pairs): a block
// ranks its 4096 keys in shared memory, publishes its digit counts, and finds
// its global digit offsets by looking back at earlier blocks (decoupled
// look-back). Every wait on another block is bounded (kMaxSpin polls); on
// expiry the block records IGS_ERR_DEVICE_TIMEOUT and carries on.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace igs {
namespace {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 2u << 30;
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValMask = kFlagAgg - 1;
constexpr unsigned long long kScanAgg = 1ull << 62;
constexpr unsigned long long kScanPre = 2ull << 62;
constexpr unsigned long long kScanMask = 3ull << 62;
constexpr unsigned long long kScanVal = kScanAgg - 1;
constexpr int kWarps = kSortThreads / 32;

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t x, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    uint32_t wpre = 0, all = 0;
#pragma unroll
    for (int k = 0; k < kSortThreads / 32; ++k) {
        uint32_t v = s_warp[k];
        if (k < w) wpre += v;
        all += v;
    }
    __syncthreads();
    if (total) *total = all;
    return wpre + incl - x;
}

// Digit histograms of n 32-bit keys for `passes` 8-bit digits starting at bit 0.
__global__ void __launch_bounds__(256) k_hist(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ d_count,
                                              uint32_t count_host, int passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_h[4][kRadix];
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = 0;
    __syncthreads();
    const uint32_t count = d_count ? *d_count : count_host;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(k >> (8 * p)) & 0xFF], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < passes * kRadix; k += blockDim.x) {
        const uint32_t v = (&s_h[0][0])[k];
        if (v) atomicAdd(&hist[k], v);
    }
}

// One stable LSD radix pass over `count` (key, value) pairs on the 8-bit digit
// at `shift`. vals_in == nullptr means value = index (the first pass of a
// sort whose values are the identity). hist = this pass's digit counts over
// all keys. status = [blocks][256] look-back words, zero on entry.
__global__ void __launch_bounds__(kSortThreads) k_onesweep(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const uint32_t* __restrict__ d_count, uint32_t count_host, int shift,
    const uint32_t* __restrict__ hist, uint32_t* __restrict__ status, uint32_t* __restrict__ block_counter,
    uint32_t* __restrict__ info) {
    __shared__ uint32_t s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    __shared__ uint32_t s_whist[kWarps][kRadix];
    __shared__ uint32_t s_local[kRadix];
    __shared__ uint32_t s_gbase[kRadix];
    __shared__ uint32_t s_warp[kWarps];
    __shared__ uint32_t s_blk;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (info && info[kInfoAbort]) return;
    const uint32_t count = d_count ? *d_count : count_host;
    if (tid == 0) s_blk = atomicAdd(block_counter, 1u);
    for (int k = tid; k < kWarps * kRadix; k += kSortThreads) (&s_whist[0][0])[k] = 0;
    __syncthreads();
    const uint32_t blk = s_blk;
    const uint64_t base = (uint64_t)blk * kSortTile;
    if (base >= count) return;  // no later block depends on a block past the end
    const uint32_t valid = (uint32_t)min((uint64_t)kSortTile, (uint64_t)count - base);

    // warp-striped load: warp w owns [w*32*IPT, (w+1)*32*IPT), item i of lane l is i*32 + l
    uint32_t key[kSortIpt], val[kSortIpt], rank[kSortIpt];
    const uint32_t wbase = w * 32 * kSortIpt;
#pragma unroll
    for (int i = 0; i < kSortIpt; ++i) {
        const uint32_t loc = wbase + i * 32 + lane;
        const uint64_t g = base + loc;
        if (loc < valid) {
            key[i] = keys_in[g];
            val[i] = vals_in ? vals_in[g] : (uint32_t)g;
        } else {
            key[i] = 0xFFFFFFFFu;  // past the end: ranks after every valid key
            val[i] = 0u;
        }
    }
    // rank within the warp, in item order
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kSortIpt; ++i) {
        const uint32_t d = (key[i] >> shift) & 0xFF;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = s_whist[w][d];
        __syncwarp();
        if (lane == __ffs(peers) - 1) s_whist[w][d] = before + __popc(peers);
        __syncwarp();
        rank[i] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, block total, local and global offsets
    const uint32_t d = tid;
    uint32_t total = 0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
        const uint32_t c = s_whist[k][d];
        s_whist[k][d] = total;
        total += c;
    }
    const uint32_t local = block_excl_scan_256(total, s_warp, nullptr);
    s_local[d] = local;
    const uint32_t hcount = hist[d];
    const uint32_t hexcl = block_excl_scan_256(hcount, s_warp, nullptr);
    // decoupled look-back for digit d
    uint32_t* my = status + (size_t)blk * kRadix;
    uint32_t excl = 0;
    if (blk == 0) {
        st_release_u32(&my[d], kFlagPre | (total & kValMask));
    } else {
        st_release_u32(&my[d], kFlagAgg | (total & kValMask));
        int64_t b = (int64_t)blk - 1;
        while (b >= 0) {
            const uint32_t* p = status + (size_t)b * kRadix + d;
            uint32_t v = ld_acquire_u32(p);
            int spins = 0;
            while ((v & kFlagMask) == 0) {
                if (++spins > kMaxSpin) {
                    record_error(info, IGS_ERR_DEVICE_TIMEOUT);
                    break;
                }
                __nanosleep(32);
                v = ld_acquire_u32(p);
            }
            excl += v & kValMask;
            if ((v & kFlagMask) != kFlagAgg) break;  // inclusive prefix reached (or gave up)
            --b;
        }
        st_release_u32(&my[d], kFlagPre | ((excl + total) & kValMask));
    }
    s_gbase[d] = hexcl + excl;
    __syncthreads();
    // stage the block's pairs in digit order
#pragma unroll
    for (int i = 0; i < kSortIpt; ++i) {
        const uint32_t dd = (key[i] >> shift) & 0xFF;
        const uint32_t q = s_local[dd] + s_whist[w][dd] + rank[i];
        s_keys[q] = key[i];
        s_vals[q] = val[i];
    }
    __syncthreads();
    // write out: runs of one digit land contiguously; past-the-end pairs occupy the last slots
#pragma unroll
    for (int k = 0; k < kSortIpt; ++k) {
        const uint32_t q = k * kSortThreads + tid;
        if (q >= valid) continue;
        const uint32_t kk = s_keys[q];
        const uint32_t dd = (kk >> shift) & 0xFF;
        const uint32_t pos = s_gbase[dd] + (q - s_local[dd]);
        if (pos >= count) continue;  // only after a look-back that gave up
        if (keys_out) keys_out[pos] = kk;
        vals_out[pos] = s_vals[q];
    }
}

// Exclusive scan of count[order[p]] over p (the tile counts in front-to-back
// order) with decoupled look-back; writes offset[p], M and the kept count.
__global__ void __launch_bounds__(kScanThreads) k_scan_offsets(const uint32_t* __restrict__ order,
                                                               const uint32_t* __restrict__ count, uint32_t n,
                                                               uint32_t* __restrict__ offset,
                                                               unsigned long long* __restrict__ status,
                                                               uint32_t* __restrict__ block_counter,
                                                               uint32_t* __restrict__ info, uint64_t capacity) {
    __shared__ uint32_t s_blk;
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_excl;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (info[kInfoAbort]) return;
    if (tid == 0) s_blk = atomicAdd(block_counter, 1u);
    __syncthreads();
    const uint32_t blk = s_blk;
    const uint64_t base = (uint64_t)blk * kScanTile;
    if (base >= n) return;
    uint32_t c[kScanIpt];
    uint32_t sum = 0, kept = 0;
    const uint64_t first = base + (uint64_t)tid * kScanIpt;
#pragma unroll
    for (int k = 0; k < kScanIpt; ++k) {
        const uint64_t p = first + k;
        const uint32_t g = p < n ? order[p] : 0xFFFFFFFFu;
        c[k] = g < n ? count[g] : 0u;
        sum += c[k];
        kept += c[k] > 0;
    }
    // block scan of the per-thread sums (64-bit)
    unsigned long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    unsigned long long wpre = 0, btotal = 0;
#pragma unroll
    for (int k = 0; k < kScanThreads / 32; ++k) {
        if (k < w) wpre += s_warp[k];
        btotal += s_warp[k];
    }
    unsigned warp_kept = __reduce_add_sync(0xffffffffu, kept);
    if (lane == 0 && warp_kept) atomicAdd(&info[kInfoKept], warp_kept);
    if (tid == 0) {
        unsigned long long excl = 0;
        unsigned long long* my = status + blk;
        if (blk == 0) {
            st_release_u64(my, kScanPre | btotal);
        } else {
            st_release_u64(my, kScanAgg | btotal);
            int64_t b = (int64_t)blk - 1;
            while (b >= 0) {
                unsigned long long v = ld_acquire_u64(status + b);
                int spins = 0;
                while ((v & kScanMask) == 0) {
                    if (++spins > kMaxSpin) {
                        record_error(info, IGS_ERR_DEVICE_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);
                    v = ld_acquire_u64(status + b);
                }
                excl += v & kScanVal;
                if ((v & kScanMask) != kScanAgg) break;
                --b;
            }
            st_release_u64(my, kScanPre | (excl + btotal));
        }
        s_excl = excl;
        if (base + kScanTile >= n) {  // the block holding the last item knows M
            const unsigned long long M = excl + btotal;
            info[kInfoM] = (uint32_t)min(M, (unsigned long long)0xFFFFFFFFu);
            info[kInfoNeed] = (uint32_t)min(M, (unsigned long long)0xFFFFFFFFu);
            if (M > capacity) {
                record_error(info, IGS_ERR_CAPACITY);
                info[kInfoAbort] = 1u;
            }
        }
    }
    __syncthreads();
    unsigned long long run = s_excl + wpre + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanIpt; ++k) {
        const uint64_t p = first + k;
        if (p < n) offset[p] = (uint32_t)min(run, (unsigned long long)0xFFFFFFFFu);
        run += c[k];
    }
}

// One thread per position p of the front-to-back order: write the entries of
// Gaussian order[p] (row-major over its tile rectangle) at offset[p]; count the
// tile-id digits of the sort passes that follow.
__global__ void __launch_bounds__(256) k_duplicate(const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ offset,
                                                   const uint32_t* __restrict__ count,
                                                   const uint2* __restrict__ rect, uint32_t n, int tiles_x,
                                                   uint64_t capacity,
                                                   uint32_t* __restrict__ tile_key, uint32_t* __restrict__ vals,
                                                   int passes, uint32_t* __restrict__ hist,
                                                   const uint32_t* __restrict__ info) {
    __shared__ uint32_t s_h[4][kRadix];
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = 0;
    __syncthreads();
    const bool abort = info[kInfoAbort] != 0;
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (!abort && p < n) {
        const uint32_t g = order[p];
        const uint32_t c = g < n ? count[g] : 0u;
        if (c && (uint64_t)offset[p] + c <= capacity) {
            const uint32_t off = offset[p];
            const uint2 r = rect[g];
            const int x0 = r.x & 0xFFFF, y0 = r.x >> 16, x1 = r.y & 0xFFFF, y1 = r.y >> 16;
            uint32_t j = off;
            for (int ty = y0; ty <= y1; ++ty)
                for (int tx = x0; tx <= x1; ++tx, ++j) {
                    const uint32_t t = (uint32_t)ty * (uint32_t)tiles_x + (uint32_t)tx;
                    tile_key[j] = t;
                    vals[j] = g;
                    for (int q = 0; q < passes; ++q) atomicAdd(&s_h[q][(t >> (8 * q)) & 0xFF], 1u);
                }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < passes * kRadix; k += blockDim.x) {
        const uint32_t v = (&s_h[0][0])[k];
        if (v) atomicAdd(&hist[k], v);
    }
}

// Per-tile [start, end) of the sorted entries; ranges are zero on entry.
__global__ void __launch_bounds__(256) k_ranges(const uint32_t* __restrict__ tile_key, uint2* __restrict__ ranges,
                                                uint32_t tiles, const uint32_t* __restrict__ info) {
    if (info[kInfoAbort]) return;
    const uint32_t M = info[kInfoM];
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        const uint32_t t = tile_key[j];
        if (t >= tiles) continue;
        if (j == 0 || tile_key[j - 1] != t) ranges[t].x = j;
        if (j + 1 == M || tile_key[j + 1] != t) ranges[t].y = j + 1;
    }
}

__global__ void k_export_keys(const uint32_t* __restrict__ tile_key, const uint32_t* __restrict__ vals,
                              const uint32_t* __restrict__ depth_key, uint64_t* __restrict__ keys,
                              const uint32_t* __restrict__ info) {
    if (info[kInfoAbort]) return;
    const uint32_t M = info[kInfoM];
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
        keys[j] = ((uint64_t)tile_key[j] << 32) | (uint64_t)depth_key[vals[j]];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

int tile_passes_for(int64_t tiles) {
    int bits = 0;
    while (bits < 32 && ((int64_t)1 << bits) < tiles) ++bits;
    return bits == 0 ? 0 : (bits + 7) / 8;
}

size_t sort_scratch_bytes(int64_t n, int64_t capacity, int64_t tiles) {
    const int64_t bn = ceil_div(n, kSortTile), bc = ceil_div(capacity, kSortTile), bs = ceil_div(n, kScanTile);
    const int tp = tile_passes_for(tiles);
    size_t b = 0;
    b += 3 * align256((size_t)n * 4);                         // dkeys_a, dkeys_b, dvals_a
    b += align256(8 * kRadix * 4);                            // hist
    b += align256(16 * 4);                                    // counters
    b += align256((size_t)4 * bn * kRadix * 4);               // status_depth
    b += align256((size_t)(tp > 0 ? tp : 1) * bc * kRadix * 4);  // status_tile
    b += align256((size_t)bs * 8);                            // scan_status
    b += 2 * align256((size_t)capacity * 4);                  // tkey_alt, vals_alt
    return b;
}

SortScratch sort_scratch(const igs_frame& f) {
    SortScratch s;
    const int64_t n = f.n, cap = f.capacity, tiles = (int64_t)f.tiles_x * f.tiles_y;
    const int64_t bn = ceil_div(n, kSortTile), bc = ceil_div(cap, kSortTile), bs = ceil_div(n, kScanTile);
    s.tile_passes = tile_passes_for(tiles);
    char* p = static_cast<char*>(f.scratch);
    auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
    s.dkeys_a = (uint32_t*)take((size_t)n * 4);
    s.dkeys_b = (uint32_t*)take((size_t)n * 4);
    s.dvals_a = (uint32_t*)take((size_t)n * 4);
    s.hist = (uint32_t*)take(8 * kRadix * 4);
    s.counters = (uint32_t*)take(16 * 4);
    s.status_depth = (uint32_t*)take((size_t)4 * bn * kRadix * 4);
    s.status_tile = (uint32_t*)take((size_t)(s.tile_passes > 0 ? s.tile_passes : 1) * bc * kRadix * 4);
    s.scan_status = (unsigned long long*)take((size_t)bs * 8);
    s.tkey_alt = (uint32_t*)take((size_t)cap * 4);
    s.vals_alt = (uint32_t*)take((size_t)cap * 4);
    return s;
}

cudaError_t launch_bin_sort(const igs_frame& f, cudaStream_t st) {
    const SortScratch s = sort_scratch(f);
    const int64_t n = f.n, cap = f.capacity;
    const int64_t tiles = (int64_t)f.tiles_x * f.tiles_y;
    const int64_t bn = ceil_div(n, kSortTile), bc = ceil_div(cap, kSortTile), bs = ceil_div(n, kScanTile);
    const int tp = s.tile_passes;
    cudaError_t e;
#define CK(x) do { if ((e = (x)) != cudaSuccess) return e; } while (0)
    // reset state: status words, histograms, counters, look-back words, ranges
    CK(cudaMemsetAsync(f.info, 0, kInfoWords * 4, st));
    CK(cudaMemsetAsync(s.hist, 0, 8 * kRadix * 4, st));
    CK(cudaMemsetAsync(s.counters, 0, 16 * 4, st));
    CK(cudaMemsetAsync(s.status_depth, 0, (size_t)4 * bn * kRadix * 4, st));
    if (tp > 0) CK(cudaMemsetAsync(s.status_tile, 0, (size_t)tp * bc * kRadix * 4, st));
    CK(cudaMemsetAsync(s.scan_status, 0, (size_t)bs * 8, st));
    CK(cudaMemsetAsync(f.ranges, 0, (size_t)tiles * 8, st));
    if (n == 0) return cudaGetLastError();
    const uint32_t nn = (uint32_t)n;
    // 1. depth sort: 4 passes, (depth_key, iota) -> (A, vA) -> (B, order) -> (A, vA) -> (B, order)
    const int hist_blocks = (int)std::min<int64_t>(ceil_div(n, 256), 152 * 4);
    k_hist<<<hist_blocks, 256, 0, st>>>(f.depth_key, nullptr, nn, 4, s.hist);
    count_launches();
    CK(cudaGetLastError());
    const uint32_t* kin = f.depth_key;
    const uint32_t* vin = nullptr;
    for (int p = 0; p < 4; ++p) {
        uint32_t* kout = (p % 2 == 0) ? s.dkeys_a : s.dkeys_b;
        uint32_t* vout = (p % 2 == 0) ? s.dvals_a : f.order;
        k_onesweep<<<(unsigned)bn, kSortThreads, 0, st>>>(kin, vin, p == 3 ? nullptr : kout, vout, nullptr, nn,
                                                          8 * p, s.hist + p * kRadix,
                                                          s.status_depth + (size_t)p * bn * kRadix, s.counters + p,
                                                          f.info);
        count_launches();
    CK(cudaGetLastError());
        kin = kout;
        vin = vout;
    }
    // 2. scan of tile counts in depth order, M, capacity check
    k_scan_offsets<<<(unsigned)bs, kScanThreads, 0, st>>>(f.order, f.count, nn, f.offset, s.scan_status,
                                                          s.counters + 4, f.info, (uint64_t)cap);
    count_launches();
    CK(cudaGetLastError());
    // 3. duplication into the buffer that, after tp passes, leaves the result in (tile_key, vals)
    uint32_t* k0 = (tp % 2 == 0) ? f.tile_key : s.tkey_alt;
    uint32_t* v0 = (tp % 2 == 0) ? f.vals : s.vals_alt;
    uint32_t* k1 = (tp % 2 == 0) ? s.tkey_alt : f.tile_key;
    uint32_t* v1 = (tp % 2 == 0) ? s.vals_alt : f.vals;
    k_duplicate<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(f.order, f.offset, f.count,
                                                            reinterpret_cast<const uint2*>(f.rect), nn, f.tiles_x,
                                                            (uint64_t)cap, k0, v0, tp, s.hist + 4 * kRadix, f.info);
    count_launches();
    CK(cudaGetLastError());
    // 4. stable tile-id sort over the M entries (M read on the device; grid sized by capacity)
    for (int p = 0; p < tp; ++p) {
        const uint32_t* ki = (p % 2 == 0) ? k0 : k1;
        const uint32_t* vi = (p % 2 == 0) ? v0 : v1;
        uint32_t* ko = (p % 2 == 0) ? k1 : k0;
        uint32_t* vo = (p % 2 == 0) ? v1 : v0;
        k_onesweep<<<(unsigned)bc, kSortThreads, 0, st>>>(ki, vi, ko, vo, f.info + kInfoM, 0u, 8 * p,
                                                          s.hist + (4 + p) * kRadix,
                                                          s.status_tile + (size_t)p * bc * kRadix,
                                                          s.counters + 5 + p, f.info);
        count_launches();
    CK(cudaGetLastError());
    }
    // 5. ranges
    const int rb = (int)std::min<int64_t>(ceil_div(cap, 256), 152 * 8);
    k_ranges<<<rb, 256, 0, st>>>(f.tile_key, reinterpret_cast<uint2*>(f.ranges), (uint32_t)tiles, f.info);
    count_launches();
    CK(cudaGetLastError());
#undef CK
    return cudaSuccess;
}

cudaError_t launch_export_keys(const igs_frame& f, uint64_t* keys, cudaStream_t st) {
    const int rb = (int)std::min<int64_t>(ceil_div(f.capacity, 256), 152 * 8);
    k_export_keys<<<rb > 0 ? rb : 1, 256, 0, st>>>(f.tile_key, f.vals, f.depth_key, keys, f.info);
    count_launches();
    return cudaGetLastError();
}

}  // namespace igs

// ---------------------------------------------------------------------------
// Front-to-back ordering without any allocation (igs_sort_depth_noalloc).
//
// Some callers cannot allocate device memory around a call: code that runs
// while a CUDA graph is being captured, or an embedding host whose memory is
// owned by its own allocator. This entry point orders n depth keys exactly as
// igs_bin_sort orders its frame's depth_key into order (stable, ties by index),
// but takes its scratch from one fixed device array compiled into the library.
// ---------------------------------------------------------------------------
namespace igs {
namespace {

constexpr int64_t kNoAllocMaxKeys = (int64_t)1 << 20;
constexpr int64_t kNoAllocBlocks = kNoAllocMaxKeys / kSortTile;
// word offsets inside the static scratch
constexpr int64_t kNaKeysA = 0;
constexpr int64_t kNaKeysB = kNaKeysA + kNoAllocMaxKeys;
constexpr int64_t kNaValsA = kNaKeysB + kNoAllocMaxKeys;
constexpr int64_t kNaHist = kNaValsA + kNoAllocMaxKeys;     // [4][256]
constexpr int64_t kNaCounters = kNaHist + 4 * kRadix;       // [64]
constexpr int64_t kNaInfo = kNaCounters + 64;               // [64]
constexpr int64_t kNaStatus = kNaInfo + 64;                 // [4][blocks][256]
constexpr int64_t kNaWords = kNaStatus + 4 * kNoAllocBlocks * kRadix;
// words that must be zero at the start of every call
constexpr int64_t kNaZeroFrom = kNaHist;

// 13.6 MB (3409024 words), held by every device that loads the library until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNaWords];

std::mutex g_noalloc_mu;
uint32_t* g_noalloc_ptr[128] = {};

// Device address of the static scratch on the current device (looked up once per device).
cudaError_t noalloc_scratch(uint32_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace igs

extern "C" igs_status igs_sort_depth_noalloc(const uint32_t* depth_key, int64_t n, uint32_t* order, void* stream) {
    using namespace igs;
    if (n < 0 || n > kNoAllocMaxKeys) return IGS_ERR_INVALID_ARG;
    if (n > 0 && (!depth_key || !order)) return IGS_ERR_INVALID_ARG;
    if (n == 0) return IGS_OK;
    uint32_t* s = nullptr;
    if (noalloc_scratch(&s) != cudaSuccess) return IGS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(s + kNaZeroFrom, 0, (size_t)(kNaWords - kNaZeroFrom) * 4, st) != cudaSuccess)
        return IGS_ERR_CUDA;
    const uint32_t nn = (uint32_t)n;
    const unsigned blocks = (unsigned)ceil_div(n, kSortTile);
    const int hist_blocks = (int)std::min<int64_t>(ceil_div(n, 256), 152 * 4);
    k_hist<<<hist_blocks, 256, 0, st>>>(depth_key, nullptr, nn, 4, s + kNaHist);
    count_launches();
    const uint32_t* kin = depth_key;
    const uint32_t* vin = nullptr;
    for (int p = 0; p < 4; ++p) {
        uint32_t* kout = (p % 2 == 0) ? s + kNaKeysA : s + kNaKeysB;
        uint32_t* vout = (p % 2 == 0) ? s + kNaValsA : order;
        k_onesweep<<<blocks, kSortThreads, 0, st>>>(kin, vin, p == 3 ? nullptr : kout, vout, nullptr, nn, 8 * p,
                                                    s + kNaHist + p * kRadix,
                                                    s + kNaStatus + (size_t)p * kNoAllocBlocks * kRadix,
                                                    s + kNaCounters + p, s + kNaInfo);
        count_launches();
        kin = kout;
        vin = vout;
    }
    return cudaGetLastError() == cudaSuccess ? IGS_OK : IGS_ERR_CUDA;
}
