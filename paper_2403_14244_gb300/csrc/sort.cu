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
//      of each Gaussian, in that order, into (tile id | Gaussian id) items;
//   3. a stable LSD radix sort of the M items on the tile id only
//      (ceil(bits(tiles) / 8) passes).
// Stability makes the result identical to the stable 64-bit key sort: within a
// tile, entries are in (depth bits, Gaussian index) order.
//
// The per-tile entry counts, hence the tile ranges and the digit histograms of
// the tile passes, come from the rectangles alone: every kept Gaussian adds its
// rectangle to a 2D difference grid (four corner updates) whose 2D prefix sum is
// the number of entries of each tile. No pass over the M entries is needed for
// them.
//
// Each radix pass is a single sweep over (key | value) items: a block counts
// the digits of its 4096 items and publishes those counts at once, ranks the
// items within each warp with ballots, looks back over earlier blocks (eight
// at a time) for its global digit offsets, and scatters the items staged in
// digit order. Every wait on another block is bounded (kMaxSpin polls); on
// expiry the block records IGS_ERR_DEVICE_TIMEOUT, which aborts the frame.
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
constexpr int kLookWindow = 8;
// 2D corner grid kept in shared memory by the preparation kernel up to this many cells.
constexpr int kGridSmemCells = 10240;

using u64 = unsigned long long;

// Exclusive scan of one value per thread over a block of NT threads.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* s_warp) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    uint32_t wpre = 0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k)
        if (k < w) wpre += s_warp[k];
    __syncthreads();
    return wpre + incl - x;
}

// Digit histograms of 32-bit keys, `passes` 8-bit digits from bit 0 (used by the
// allocation-free ordering; the frame path counts depth digits in k_bin_prep).
__global__ void __launch_bounds__(256) k_hist(const uint32_t* __restrict__ keys, uint32_t count, int passes,
                                              uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_h[4][kRadix];
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = 0;
    __syncthreads();
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

// Depth-digit histograms of all n depth keys, and the rectangle corners of every
// kept Gaussian added into the (tiles_y+1) x (tiles_x+1) difference grid.
template <bool SMEM_GRID>
__global__ void __launch_bounds__(256) k_bin_prep(const uint32_t* __restrict__ depth_key, const uint2* __restrict__ rect,
                                                  const uint32_t* __restrict__ count, uint32_t n, int gx, int gy,
                                                  uint32_t* __restrict__ hist, int32_t* __restrict__ grid) {
    extern __shared__ int32_t s_grid[];
    __shared__ uint32_t s_h[4][kRadix];
    const int cells = gx * gy;
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = 0;
    if (SMEM_GRID)
        for (int k = threadIdx.x; k < cells; k += blockDim.x) s_grid[k] = 0;
    __syncthreads();
    int32_t* g = SMEM_GRID ? s_grid : grid;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = depth_key[i];
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&s_h[p][(k >> (8 * p)) & 0xFF], 1u);
        if (count[i]) {
            const uint2 r = rect[i];
            const int x0 = r.x & 0xFFFF, y0 = r.x >> 16, x1 = (r.y & 0xFFFF) + 1, y1 = (r.y >> 16) + 1;
            atomicAdd(&g[y0 * gx + x0], 1);
            atomicAdd(&g[y0 * gx + x1], -1);
            atomicAdd(&g[y1 * gx + x0], -1);
            atomicAdd(&g[y1 * gx + x1], 1);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) {
        const uint32_t v = (&s_h[0][0])[k];
        if (v) atomicAdd(&hist[k], v);
    }
    if (SMEM_GRID)
        for (int k = threadIdx.x; k < cells; k += blockDim.x)
            if (s_grid[k]) atomicAdd(&grid[k], s_grid[k]);
}

// 2D inclusive prefix of the corner grid, rows then columns: afterwards grid[y][x]
// holds the number of kept Gaussians whose rectangle contains tile (x, y).
__global__ void k_grid_rows(int32_t* __restrict__ grid, int gx, int tiles_x, int tiles_y) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= tiles_y) return;
    int32_t run = 0;
    int32_t* row = grid + (size_t)y * gx;
    for (int x = 0; x < tiles_x; ++x) {
        run += row[x];
        row[x] = run;
    }
}

__global__ void k_grid_cols(int32_t* __restrict__ grid, int gx, int tiles_x, int tiles_y) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= tiles_x) return;
    int32_t run = 0;
    for (int y = 0; y < tiles_y; ++y) {
        run += grid[(size_t)y * gx + x];
        grid[(size_t)y * gx + x] = run;
    }
}

// One block: tile ranges = exclusive scan of the per-tile counts (row-major tile
// order), (0, 0) for empty tiles; digit histograms of the tile-id passes.
constexpr int kTileScanThreads = 1024;
__global__ void __launch_bounds__(kTileScanThreads) k_tile_scan(const int32_t* __restrict__ grid, int gx, int tiles_x,
                                                                uint32_t tiles, int passes,
                                                                uint2* __restrict__ ranges,
                                                                uint32_t* __restrict__ hist_tile,
                                                                uint32_t* __restrict__ info) {
    __shared__ uint32_t s_h[4][kRadix];
    __shared__ uint32_t s_warp[kTileScanThreads / 32];
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = 0;
    const uint32_t per = (tiles + kTileScanThreads - 1) / kTileScanThreads;
    const uint32_t t0 = min(tiles, threadIdx.x * per), t1 = min(tiles, t0 + per);
    uint32_t sum = 0;
    for (uint32_t t = t0; t < t1; ++t) sum += (uint32_t)grid[(size_t)(t / tiles_x) * gx + (t % tiles_x)];
    __syncthreads();
    uint32_t start = block_excl_scan<kTileScanThreads>(sum, s_warp);
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t c = (uint32_t)grid[(size_t)(t / tiles_x) * gx + (t % tiles_x)];
        ranges[t] = c ? make_uint2(start, start + c) : make_uint2(0u, 0u);
        start += c;
        if (c)
            for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(t >> (8 * p)) & 0xFF], c);
    }
    if (t1 == tiles && t0 < t1) info[kInfoTileTotal] = start;  // checked against M by the scan
    __syncthreads();
    for (int k = threadIdx.x; k < passes * kRadix; k += blockDim.x) hist_tile[k] = (&s_h[0][0])[k];
}

// In place: each of `passes` (<= 8) rows of 256 digit counts becomes its
// exclusive prefix (the global start of each digit in that pass). One block of 1024.
__global__ void __launch_bounds__(1024) k_hist_to_offsets(uint32_t* __restrict__ hist, int passes) {
    const int n = passes * kRadix;
    uint32_t v[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int idx = threadIdx.x + r * 1024;
        v[r] = 0;
        if (idx < n) {
            const uint32_t* row = hist + (idx & ~255);
            for (int k = 0; k < (idx & 255); ++k) v[r] += row[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int idx = threadIdx.x + r * 1024;
        if (idx < n) hist[idx] = v[r];
    }
}

// One stable LSD radix pass over `count` items (key << 32 | value) on the 8-bit
// digit (key >> shift) & 255. IN_KEYS32: the input is the 32-bit key array and
// the value is the index (first pass of the depth sort). OUT_VALS: write only the
// values (last pass). digit_base = this pass's global start of every digit.
// status = [blocks][256] look-back words, zero on entry.
template <bool IN_KEYS32, bool OUT_VALS>
__global__ void __launch_bounds__(kSortThreads, 4) k_radix_pass(
    const void* __restrict__ in_, void* __restrict__ out_, const uint32_t* __restrict__ d_count, uint32_t count_host,
    int shift, const uint32_t* __restrict__ digit_base, uint32_t* __restrict__ status,
    uint32_t* __restrict__ block_counter, uint32_t* __restrict__ info) {
    __shared__ u64 s_items[kSortTile];
    __shared__ uint16_t s_whist[kWarps][kRadix];  // per warp: running count, then block-local start
    __shared__ uint32_t s_cnt[kRadix];
    __shared__ int32_t s_delta[kRadix];           // global position - staged position, per digit
    __shared__ uint32_t s_warp[kWarps];
    __shared__ uint32_t s_blk;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (info && info[kInfoAbort]) return;
    const uint32_t count = d_count ? *d_count : count_host;
    if (tid == 0) s_blk = atomicAdd(block_counter, 1u);
    {
        uint32_t* z = reinterpret_cast<uint32_t*>(&s_whist[0][0]);
#pragma unroll
        for (int k = 0; k < kWarps * kRadix / 2 / kSortThreads; ++k) z[k * kSortThreads + tid] = 0;
        s_cnt[tid] = 0;
    }
    __syncthreads();
    const uint32_t blk = s_blk;
    const uint64_t base = (uint64_t)blk * kSortTile;
    if (base >= count) return;  // no later block depends on a block past the end
    const uint32_t valid = (uint32_t)min((uint64_t)kSortTile, (uint64_t)count - base);

    // warp-striped load: warp w owns [w*32*IPT, (w+1)*32*IPT), item i of lane l is i*32 + l
    u64 it[kSortIpt];
    const uint32_t wbase = w * 32 * kSortIpt + lane;
    if (valid == kSortTile) {
#pragma unroll
        for (int i = 0; i < kSortIpt; ++i) {
            const uint64_t g = base + wbase + i * 32;
            if (IN_KEYS32)
                it[i] = ((u64)static_cast<const uint32_t*>(in_)[g] << 32) | (uint32_t)g;
            else
                it[i] = static_cast<const u64*>(in_)[g];
        }
    } else {
#pragma unroll
        for (int i = 0; i < kSortIpt; ++i) {
            const uint32_t loc = wbase + i * 32;
            const uint64_t g = base + loc;
            if (loc < valid)
                it[i] = IN_KEYS32 ? (((u64)static_cast<const uint32_t*>(in_)[g] << 32) | (uint32_t)g)
                                  : static_cast<const u64*>(in_)[g];
            else
                it[i] = ~0ull;  // past the end: digit 255, after every valid item
        }
    }
    // digit counts of the block's valid items, published before the ranking
#pragma unroll
    for (int i = 0; i < kSortIpt; ++i)
        if (wbase + i * 32 < valid) atomicAdd(&s_cnt[(uint32_t)(it[i] >> (32 + shift)) & 0xFFu], 1u);
    __syncthreads();
    uint32_t* my = status + (size_t)blk * kRadix;
    st_relaxed_u32(&my[tid], (blk == 0 ? kFlagPre : kFlagAgg) | (s_cnt[tid] & kValMask));
    // rank within the warp, in item order
    uint32_t rank2[kSortIpt / 2];  // two 16-bit ranks per register (ranks < 4096)
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kSortIpt; ++i) {
        const uint32_t d = (uint32_t)(it[i] >> (32 + shift)) & 0xFFu;
        // peers: lanes with the same digit, from 8 ballots (measured faster than match.any here)
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bal : ~bal;
        }
        const uint32_t before = s_whist[w][d];
        __syncwarp();
        if ((peers & lt) == 0) s_whist[w][d] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        const uint32_t r = before + __popc(peers & lt);
        if (i & 1) rank2[i >> 1] |= r << 16; else rank2[i >> 1] = r;
    }
    __syncthreads();
    // digit tid: block-local start of every warp's run, global offset by look-back
    const uint32_t cnt = s_cnt[tid];
    const uint32_t local = block_excl_scan<kSortThreads>(cnt, s_warp);
    {
        uint32_t run = local;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) {
            const uint32_t c = s_whist[k][tid];
            s_whist[k][tid] = (uint16_t)run;
            run += c;
        }
    }
    uint32_t excl = 0;
    if (blk > 0) {
        int64_t b = (int64_t)blk - 1;
        bool done = false;
        while (!done && b >= 0) {
            const int nw = b + 1 < kLookWindow ? (int)(b + 1) : kLookWindow;
            uint32_t v[kLookWindow];
#pragma unroll
            for (int j = 0; j < kLookWindow; ++j)
                v[j] = j < nw ? ld_relaxed_u32(status + (size_t)(b - j) * kRadix + tid) : 0u;
#pragma unroll
            for (int j = 0; j < kLookWindow; ++j) {
                if (done || j >= nw) break;
                int spins = 0;
                while ((v[j] & kFlagMask) == 0) {
                    if (++spins > kMaxSpin) {
                        record_error(info, IGS_ERR_DEVICE_TIMEOUT);
                        done = true;
                        break;
                    }
                    __nanosleep(32);
                    v[j] = ld_relaxed_u32(status + (size_t)(b - j) * kRadix + tid);
                }
                if (done) break;
                excl += v[j] & kValMask;
                if ((v[j] & kFlagMask) == kFlagPre) done = true;
            }
            b -= nw;
        }
        st_relaxed_u32(&my[tid], kFlagPre | ((excl + cnt) & kValMask));
    }
    s_delta[tid] = (int32_t)(digit_base[tid] + excl) - (int32_t)local;
    __syncthreads();
    // stage the block's items in digit order
#pragma unroll
    for (int i = 0; i < kSortIpt; ++i) {
        const uint32_t d = (uint32_t)(it[i] >> (32 + shift)) & 0xFFu;
        s_items[s_whist[w][d] + ((rank2[i >> 1] >> (16 * (i & 1))) & 0xFFFFu)] = it[i];
    }
    __syncthreads();
    // write out: runs of one digit land contiguously; past-the-end items hold the last slots
#pragma unroll
    for (int k = 0; k < kSortIpt; ++k) {
        const uint32_t q = k * kSortThreads + tid;
        if (q >= valid) continue;
        const u64 item = s_items[q];
        const uint32_t pos = (uint32_t)((int32_t)q + s_delta[(uint32_t)(item >> (32 + shift)) & 0xFFu]);
        if (pos >= count) continue;  // only after a look-back that gave up
        if (OUT_VALS)
            static_cast<uint32_t*>(out_)[pos] = (uint32_t)item;
        else
            static_cast<u64*>(out_)[pos] = item;
    }
}

// Exclusive scan of count[order[p]] over p (the tile counts in front-to-back
// order) with decoupled look-back (one warp reads 32 predecessors at a time);
// writes offset[p], M, the kept count, and for every duplication block the
// position in `order` of the Gaussian that holds its first entry.
__global__ void __launch_bounds__(kScanThreads) k_scan_offsets(const uint32_t* __restrict__ order,
                                                               const uint32_t* __restrict__ count, uint32_t n,
                                                               uint32_t* __restrict__ offset,
                                                               uint32_t* __restrict__ dup_start,
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
    unsigned long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
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
    const unsigned warp_kept = __reduce_add_sync(0xffffffffu, kept);
    if (lane == 0 && warp_kept) atomicAdd(&info[kInfoKept], warp_kept);
    if (w == 0) {
        unsigned long long* my = status + blk;
        if (lane == 0) st_relaxed_u64(my, (blk == 0 ? kScanPre : kScanAgg) | btotal);
        unsigned long long excl = 0;
        int64_t b = (int64_t)blk - 1;
        bool timed_out = false;
        while (b >= 0) {
            const int64_t j = b - lane;
            unsigned long long v = j >= 0 ? ld_relaxed_u64(status + j) : kScanPre;  // before block 0: prefix 0
            int spins = 0;
            while (__any_sync(0xffffffffu, (v & kScanMask) == 0)) {
                if (++spins > kMaxSpin) {
                    timed_out = true;
                    break;
                }
                __nanosleep(32);
                if ((v & kScanMask) == 0) v = ld_relaxed_u64(status + j);
            }
            if (timed_out) {
                if (lane == 0) record_error(info, IGS_ERR_DEVICE_TIMEOUT);
                break;
            }
            const uint32_t pre = __ballot_sync(0xffffffffu, (v & kScanMask) == kScanPre);
            const int stop = pre ? __ffs(pre) - 1 : 31;
            unsigned long long part = lane <= stop ? (v & kScanVal) : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            excl += part;
            if (pre) break;
            b -= 32;
        }
        if (lane == 0) {
            if (blk > 0) st_relaxed_u64(my, kScanPre | (excl + btotal));
            s_excl = excl;
            if (base + kScanTile >= n) {  // the block holding the last item knows M
                const unsigned long long M = excl + btotal;
                info[kInfoM] = (uint32_t)min(M, (unsigned long long)0xFFFFFFFFu);
                info[kInfoNeed] = (uint32_t)min(M, (unsigned long long)0xFFFFFFFFu);
                if (M > capacity) {
                    atomicCAS(&info[kInfoErr], 0u, (uint32_t)IGS_ERR_CAPACITY);
                    info[kInfoAbort] = 1u;
                } else if (M != info[kInfoTileTotal]) {
                    record_error(info, IGS_ERR_CUDA);  // tile counts disagree with the scan: never expected
                }
            }
        }
    }
    __syncthreads();
    unsigned long long run = s_excl + wpre + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanIpt; ++k) {
        const uint64_t p = first + k;
        if (p < n) {
            offset[p] = (uint32_t)min(run, (unsigned long long)0xFFFFFFFFu);
            // duplication blocks whose first entry belongs to this Gaussian
            if (c[k] && run < capacity) {
                for (unsigned long long m = (run + kDupTile - 1) / kDupTile * kDupTile; m < run + c[k] && m < capacity;
                     m += kDupTile)
                    dup_start[m / kDupTile] = (uint32_t)p;
            }
        }
        run += c[k];
    }
}

// Duplication by output position: block b writes entries [b*kDupTile, ...) of
// the front-to-back entry list. Each entry finds its Gaussian by a binary
// search of the block's window of offsets, then its tile inside the Gaussian's
// rectangle (row-major). Writes (tile id << 32 | Gaussian id), or only the
// Gaussian id when no tile pass follows.
__global__ void __launch_bounds__(256) k_duplicate(const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ offset,
                                                   const uint32_t* __restrict__ dup_start,
                                                   const uint2* __restrict__ rect, uint32_t n, int tiles_x,
                                                   u64* __restrict__ items, uint32_t* __restrict__ vals_direct,
                                                   const uint32_t* __restrict__ info) {
    __shared__ uint32_t s_off[kDupTile + 2];
    __shared__ uint32_t s_ord[kDupTile + 1];
    if (info[kInfoAbort]) return;
    const uint32_t M = info[kInfoM];
    const uint64_t e0 = (uint64_t)blockIdx.x * kDupTile;
    if (e0 >= M) return;
    const uint32_t pb = dup_start[blockIdx.x];
    if (pb >= n) return;
    const uint32_t cnt = min((uint32_t)kDupTile + 1u, n - pb);
    for (uint32_t k = threadIdx.x; k <= cnt; k += blockDim.x) s_off[k] = (pb + k < n) ? offset[pb + k] : M;
    for (uint32_t k = threadIdx.x; k < cnt; k += blockDim.x) s_ord[k] = order[pb + k];
    __syncthreads();
    const uint32_t e_end = (uint32_t)(e0 + kDupTile < (uint64_t)M ? e0 + kDupTile : (uint64_t)M);
    for (uint32_t e = (uint32_t)e0 + threadIdx.x; e < e_end; e += blockDim.x) {
        uint32_t lo = 0, hi = cnt;  // largest k with s_off[k] <= e
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_off[mid] <= e) lo = mid; else hi = mid;
        }
        const uint32_t g = s_ord[lo];
        if (g >= n) continue;
        const uint32_t j = e - s_off[lo];
        const uint2 r = rect[g];
        const uint32_t x0 = r.x & 0xFFFF, y0 = r.x >> 16, wdt = (r.y & 0xFFFF) - x0 + 1;
        // row = j / wdt: float estimate, then exact integer correction (j, wdt < 2^24)
        uint32_t row = (uint32_t)__fmul_rz((float)j, __frcp_rz((float)wdt));
        int32_t rem = (int32_t)j - (int32_t)(row * wdt);
        if (rem < 0) { --row; rem += (int32_t)wdt; }
        if (rem >= (int32_t)wdt) { ++row; rem -= (int32_t)wdt; }
        const uint32_t t = (y0 + row) * (uint32_t)tiles_x + x0 + (uint32_t)rem;
        if (vals_direct)
            vals_direct[e] = g;
        else
            items[e] = ((u64)t << 32) | g;
    }
}

// Sorted 64-bit keys (tile << 32 | depth bits) and the tile id of every entry,
// from the ranges: block t fills the entries of tile t.
__global__ void k_export_keys(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                              const uint32_t* __restrict__ depth_key, uint64_t* __restrict__ keys,
                              uint32_t* __restrict__ tile_key, const uint32_t* __restrict__ info) {
    if (info[kInfoAbort]) return;
    const uint32_t t = blockIdx.x;
    const uint2 r = ranges[t];
    for (uint32_t j = r.x + threadIdx.x; j < r.y; j += blockDim.x) {
        keys[j] = ((uint64_t)t << 32) | (uint64_t)depth_key[vals[j]];
        tile_key[j] = t;
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int tile_bits_for(int64_t tiles) {
    int bits = 0;
    while (bits < 32 && ((int64_t)1 << bits) < tiles) ++bits;
    return bits;
}

}  // namespace

int tile_passes_for(int64_t tiles) {
    const int bits = tile_bits_for(tiles);
    return (bits + 7) / 8;
}

// The corner grid has (tiles_y + 1)(tiles_x + 1) = tiles + tiles_x + tiles_y + 1
// <= 2 tiles + 2 cells.
size_t sort_scratch_bytes(int64_t n, int64_t capacity, int64_t tiles) {
    const int64_t bn = ceil_div(n, kSortTile), bc = ceil_div(capacity, kSortTile), bs = ceil_div(n, kScanTile);
    const int tp = tile_passes_for(tiles);
    size_t b = 0;
    b += 2 * align256((size_t)n * 8);                               // ditems_a, ditems_b
    b += 2 * align256((size_t)capacity * 8);                        // items_a, items_b
    b += align256(8 * kRadix * 4);                                  // hist
    b += align256(16 * 4);                                          // counters
    b += align256((size_t)4 * bn * kRadix * 4);                     // status_depth
    b += align256((size_t)(tp > 0 ? tp : 1) * bc * kRadix * 4);     // status_tile
    b += align256((size_t)bs * 8);                                  // scan_status
    b += align256((size_t)(ceil_div(capacity, kDupTile) + 1) * 4);  // dup_start
    b += align256((size_t)(2 * tiles + 2) * 4);                     // grid
    return b;
}

SortScratch sort_scratch(const igs_frame& f) {
    SortScratch s;
    const int64_t n = f.n, cap = f.capacity, tiles = (int64_t)f.tiles_x * f.tiles_y;
    const int64_t bn = ceil_div(n, kSortTile), bc = ceil_div(cap, kSortTile), bs = ceil_div(n, kScanTile);
    s.tile_bits = tile_bits_for(tiles);
    s.tile_passes = tile_passes_for(tiles);
    char* p = static_cast<char*>(f.scratch);
    auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
    s.ditems_a = (u64*)take((size_t)n * 8);
    s.ditems_b = (u64*)take((size_t)n * 8);
    s.items_a = (u64*)take((size_t)cap * 8);
    s.items_b = (u64*)take((size_t)cap * 8);
    s.hist = (uint32_t*)take(8 * kRadix * 4);
    s.counters = (uint32_t*)take(16 * 4);
    s.status_depth = (uint32_t*)take((size_t)4 * bn * kRadix * 4);
    s.status_tile = (uint32_t*)take((size_t)(s.tile_passes > 0 ? s.tile_passes : 1) * bc * kRadix * 4);
    s.scan_status = (unsigned long long*)take((size_t)bs * 8);
    s.dup_start = (uint32_t*)take((size_t)(ceil_div(cap, kDupTile) + 1) * 4);
    s.grid = (int32_t*)take((size_t)(2 * tiles + 2) * 4);
    return s;
}

cudaError_t launch_bin_sort(const igs_frame& f, cudaStream_t st) {
    const SortScratch s = sort_scratch(f);
    const int64_t n = f.n, cap = f.capacity;
    const int64_t tiles = (int64_t)f.tiles_x * f.tiles_y;
    const int64_t bn = ceil_div(n, kSortTile), bc = ceil_div(cap, kSortTile), bs = ceil_div(n, kScanTile);
    const int tp = s.tile_passes;
    const int gx = f.tiles_x + 1, gy = f.tiles_y + 1;
    cudaError_t e;
#define CK(x) do { if ((e = (x)) != cudaSuccess) return e; } while (0)
    // reset state: status words, histograms, counters, look-back words, corner grid
    CK(cudaMemsetAsync(f.info, 0, kInfoWords * 4, st));
    CK(cudaMemsetAsync(s.hist, 0, 8 * kRadix * 4, st));
    CK(cudaMemsetAsync(s.counters, 0, 16 * 4, st));
    CK(cudaMemsetAsync(s.status_depth, 0, (size_t)4 * bn * kRadix * 4, st));
    if (tp > 0) CK(cudaMemsetAsync(s.status_tile, 0, (size_t)tp * bc * kRadix * 4, st));
    CK(cudaMemsetAsync(s.scan_status, 0, (size_t)bs * 8, st));
    CK(cudaMemsetAsync(s.grid, 0, (size_t)gx * gy * 4, st));
    if (n == 0) {
        CK(cudaMemsetAsync(f.ranges, 0, (size_t)tiles * 8, st));
        return cudaSuccess;
    }
    const uint32_t nn = (uint32_t)n;
    // 0. depth-digit histograms; rectangle corners -> per-tile counts -> ranges, tile-digit histograms
    const int prep_blocks = (int)std::min<int64_t>(ceil_div(n, 256), 152 * 4);
    if ((int64_t)gx * gy <= kGridSmemCells)
        k_bin_prep<true><<<prep_blocks, 256, (size_t)gx * gy * 4, st>>>(
            f.depth_key, reinterpret_cast<const uint2*>(f.rect), f.count, nn, gx, gy, s.hist, s.grid);
    else
        k_bin_prep<false><<<prep_blocks, 256, 0, st>>>(f.depth_key, reinterpret_cast<const uint2*>(f.rect), f.count,
                                                       nn, gx, gy, s.hist, s.grid);
    count_launches();
    CK(cudaGetLastError());
    k_grid_rows<<<(unsigned)ceil_div(f.tiles_y, 128), 128, 0, st>>>(s.grid, gx, f.tiles_x, f.tiles_y);
    count_launches();
    CK(cudaGetLastError());
    k_grid_cols<<<(unsigned)ceil_div(f.tiles_x, 128), 128, 0, st>>>(s.grid, gx, f.tiles_x, f.tiles_y);
    count_launches();
    CK(cudaGetLastError());
    k_tile_scan<<<1, kTileScanThreads, 0, st>>>(s.grid, gx, f.tiles_x, (uint32_t)tiles, tp,
                                                reinterpret_cast<uint2*>(f.ranges), s.hist + 4 * kRadix, f.info);
    count_launches();
    CK(cudaGetLastError());
    k_hist_to_offsets<<<1, 1024, 0, st>>>(s.hist, 4 + tp);
    count_launches();
    CK(cudaGetLastError());
    // 1. depth sort: (depth_key, index) -> A -> B -> A -> order
    for (int p = 0; p < 4; ++p) {
        uint32_t* status = s.status_depth + (size_t)p * bn * kRadix;
        const uint32_t* hist = s.hist + p * kRadix;
        if (p == 0)
            k_radix_pass<true, false><<<(unsigned)bn, kSortThreads, 0, st>>>(
                f.depth_key, s.ditems_a, nullptr, nn, 0, hist, status, s.counters + 0, f.info);
        else if (p == 3)
            k_radix_pass<false, true><<<(unsigned)bn, kSortThreads, 0, st>>>(
                s.ditems_a, f.order, nullptr, nn, 24, hist, status, s.counters + 3, f.info);
        else
            k_radix_pass<false, false><<<(unsigned)bn, kSortThreads, 0, st>>>(
                p == 1 ? s.ditems_a : s.ditems_b, p == 1 ? s.ditems_b : s.ditems_a, nullptr, nn, 8 * p, hist,
                status, s.counters + p, f.info);
        count_launches();
        CK(cudaGetLastError());
    }
    // 2. scan of tile counts in depth order, M, capacity check, duplication block starts
    k_scan_offsets<<<(unsigned)bs, kScanThreads, 0, st>>>(f.order, f.count, nn, f.offset, s.dup_start,
                                                          s.scan_status, s.counters + 4, f.info, (uint64_t)cap);
    count_launches();
    CK(cudaGetLastError());
    // 3. duplication, in depth order, by output position
    const unsigned dup_blocks = (unsigned)std::max<int64_t>(1, ceil_div(cap, kDupTile));
    k_duplicate<<<dup_blocks, 256, 0, st>>>(f.order, f.offset, s.dup_start, reinterpret_cast<const uint2*>(f.rect), nn,
                                            f.tiles_x, s.items_a, tp == 0 ? f.vals : nullptr, f.info);
    count_launches();
    CK(cudaGetLastError());
    // 4. stable tile-id sort of the M items (M read on the device; grid sized by capacity)
    for (int p = 0; p < tp; ++p) {
        const u64* in = (p % 2 == 0) ? s.items_a : s.items_b;
        uint32_t* status = s.status_tile + (size_t)p * bc * kRadix;
        const uint32_t* hist = s.hist + (4 + p) * kRadix;
        if (p == tp - 1)
            k_radix_pass<false, true><<<(unsigned)bc, kSortThreads, 0, st>>>(
                in, f.vals, f.info + kInfoM, 0u, 8 * p, hist, status, s.counters + 5 + p, f.info);
        else
            k_radix_pass<false, false><<<(unsigned)bc, kSortThreads, 0, st>>>(
                in, (p % 2 == 0) ? s.items_b : s.items_a, f.info + kInfoM, 0u, 8 * p, hist, status,
                s.counters + 5 + p, f.info);
        count_launches();
        CK(cudaGetLastError());
    }
#undef CK
    return cudaSuccess;
}

cudaError_t launch_export_keys(const igs_frame& f, uint64_t* keys, cudaStream_t st) {
    const unsigned tiles = (unsigned)(f.tiles_x * f.tiles_y);
    if (tiles == 0) return cudaSuccess;
    k_export_keys<<<tiles, 128, 0, st>>>(reinterpret_cast<const uint2*>(f.ranges), f.vals, f.depth_key, keys,
                                         f.tile_key, f.info);
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
// 32-bit word offsets inside the static scratch
constexpr int64_t kNaItemsA = 0;                                // [max] u64
constexpr int64_t kNaItemsB = kNaItemsA + 2 * kNoAllocMaxKeys;  // [max] u64
constexpr int64_t kNaHist = kNaItemsB + 2 * kNoAllocMaxKeys;    // [4][256]
constexpr int64_t kNaCounters = kNaHist + 4 * kRadix;           // [64]
constexpr int64_t kNaInfo = kNaCounters + 64;                   // [64]
constexpr int64_t kNaStatus = kNaInfo + 64;                     // [4][blocks][256]
constexpr int64_t kNaWords = kNaStatus + 4 * kNoAllocBlocks * kRadix;
// words that must be zero at the start of every call
constexpr int64_t kNaZeroFrom = kNaHist;

// 17.8 MB (4457600 words), held by every device that loads the library until the process exits.
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
    k_hist<<<hist_blocks, 256, 0, st>>>(depth_key, nn, 4, s + kNaHist);
    count_launches();
    k_hist_to_offsets<<<1, 1024, 0, st>>>(s + kNaHist, 4);
    count_launches();
    u64* A = reinterpret_cast<u64*>(s + kNaItemsA);
    u64* B = reinterpret_cast<u64*>(s + kNaItemsB);
    for (int p = 0; p < 4; ++p) {
        uint32_t* status = s + kNaStatus + (size_t)p * kNoAllocBlocks * kRadix;
        const uint32_t* hist = s + kNaHist + p * kRadix;
        if (p == 0)
            k_radix_pass<true, false><<<blocks, kSortThreads, 0, st>>>(depth_key, A, nullptr, nn, 0, hist, status,
                                                                       s + kNaCounters + 0, s + kNaInfo);
        else if (p == 3)
            k_radix_pass<false, true><<<blocks, kSortThreads, 0, st>>>(A, order, nullptr, nn, 24, hist, status,
                                                                       s + kNaCounters + 3, s + kNaInfo);
        else
            k_radix_pass<false, false><<<blocks, kSortThreads, 0, st>>>(p == 1 ? A : B, p == 1 ? B : A, nullptr, nn,
                                                                        8 * p, hist, status, s + kNaCounters + p,
                                                                        s + kNaInfo);
        count_launches();
    }
    return cudaGetLastError() == cudaSuccess ? IGS_OK : IGS_ERR_CUDA;
}
