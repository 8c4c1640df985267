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

#include "binning.cuh"

namespace igs {
namespace {

// 2D corner grid kept in shared memory by the preparation kernel up to this many cells.
constexpr int kGridSmemCells = 10240;

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

// One block, grid in shared memory (cells <= kGridSmemCells): the 2D prefix of
// the corner grid, the tile ranges, the tile-digit histograms, and every digit
// histogram (4 depth + `passes` tile rows) turned into exclusive offsets.
constexpr int kTilesSmallThreads = 1024;
__global__ void __launch_bounds__(kTilesSmallThreads) k_tiles_small(const int32_t* __restrict__ grid, int tiles_x,
                                                                    int tiles_y, int passes,
                                                                    uint2* __restrict__ ranges,
                                                                    uint32_t* __restrict__ hist,
                                                                    uint32_t* __restrict__ info) {
    extern __shared__ int32_t s_g[];
    __shared__ uint32_t s_h[8][kRadix];
    __shared__ uint32_t s_warp[kTilesSmallThreads / 32];
    const int gx = tiles_x + 1, cells = gx * (tiles_y + 1);
    const int tid = threadIdx.x;
    for (int k = tid; k < cells; k += blockDim.x) s_g[k] = grid[k];
    for (int k = tid; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = hist[k];          // depth counts
    for (int k = tid; k < 4 * kRadix; k += blockDim.x) (&s_h[4][0])[k] = 0;                // tile counts
    __syncthreads();
    for (int y = tid; y < tiles_y; y += blockDim.x) {
        int32_t run = 0;
        for (int x = 0; x < tiles_x; ++x) { run += s_g[y * gx + x]; s_g[y * gx + x] = run; }
    }
    __syncthreads();
    for (int x = tid; x < tiles_x; x += blockDim.x) {
        int32_t run = 0;
        for (int y = 0; y < tiles_y; ++y) { run += s_g[y * gx + x]; s_g[y * gx + x] = run; }
    }
    __syncthreads();
    const uint32_t tiles = (uint32_t)tiles_x * tiles_y;
    const uint32_t per = (tiles + kTilesSmallThreads - 1) / kTilesSmallThreads;
    const uint32_t t0 = min(tiles, tid * per), t1 = min(tiles, t0 + per);
    uint32_t sum = 0;
    for (uint32_t t = t0; t < t1; ++t) sum += (uint32_t)s_g[(t / tiles_x) * gx + (t % tiles_x)];
    uint32_t start = block_excl_scan<kTilesSmallThreads>(sum, s_warp);
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t c = (uint32_t)s_g[(t / tiles_x) * gx + (t % tiles_x)];
        ranges[t] = c ? make_uint2(start, start + c) : make_uint2(0u, 0u);
        start += c;
        if (c)
            for (int p = 0; p < passes; ++p) atomicAdd(&s_h[4 + p][(t >> (8 * p)) & 0xFF], c);
    }
    if (t1 == tiles && t0 < t1) info[kInfoTileTotal] = start;
    __syncthreads();
    // exclusive offsets of every histogram row
    const int rows = 4 + passes;
    uint32_t v[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int idx = tid + r * kTilesSmallThreads;
        v[r] = 0;
        if (idx < rows * kRadix) {
            const uint32_t* row = &s_h[idx >> 8][0];
            for (int k = 0; k < (idx & 255); ++k) v[r] += row[k];
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int idx = tid + r * kTilesSmallThreads;
        if (idx < rows * kRadix) hist[idx] = v[r];
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
    // the last tile pass (p = passes - 1) reads items_a when p is even, items_b when odd
    const bool last_reads_a = s.tile_passes > 0 && (s.tile_passes - 1) % 2 == 0;
    s.vals = reinterpret_cast<uint32_t*>(last_reads_a ? s.items_b : s.items_a);
    s.tile_key = reinterpret_cast<uint32_t*>(last_reads_a ? s.items_a : s.items_b);
    if (s.tile_passes == 0) {  // the duplication writes the values directly
        s.vals = reinterpret_cast<uint32_t*>(s.items_a);
        s.tile_key = reinterpret_cast<uint32_t*>(s.items_b);
    }
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
    if ((int64_t)gx * gy <= kGridSmemCells) {
        k_tiles_small<<<1, kTilesSmallThreads, (size_t)gx * gy * 4, st>>>(s.grid, f.tiles_x, f.tiles_y, tp,
                                                                           reinterpret_cast<uint2*>(f.ranges), s.hist,
                                                                           f.info);
        count_launches();
        CK(cudaGetLastError());
    } else {
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
    }
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
    k_duplicate<false><<<dup_blocks, 256, 0, st>>>(f.order, f.offset, s.dup_start,
                                                   reinterpret_cast<const uint2*>(f.rect), nn, f.tiles_x, s.items_a,
                                                   tp == 0 ? f.vals : nullptr, f.info, nn, nullptr, nullptr);
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
