// Binning and sorting: front-to-back order of the kept Gaussians, their
// entries (one per touched tile) grouped by tile id, and per-tile ranges.
//
// Eq. 4 composites each pixel front to back, so every tile needs its Gaussians
// in depth order. Instead of one radix sort over 64-bit (tile << 32 | depth)
// keys, this does:
//   1. a stable 32-bit LSD radix sort of the n depth keys (culled ones carry
//      0xFFFFFFFF and sort last), which gives `order`. When every other key
//      has the same top byte (depths within one pair of binary exponents) and
//      none has its low 24 bits all ones, sorting the low 24 bits alone gives
//      the same order (culled keys, 0xFFFFFF there, still sort last and by
//      index), so the third pass writes `order` and the fourth does nothing;
//      the decision is taken on the device from the digit histograms;
//   2. an exclusive scan of the tile counts in that order (M, capacity check);
//   3. the entries in tile order, by one of two routes:
//      a. counting sort (at most 2048 tiles per axis): the tile ranges are
//         known in advance (below), so each entry's slot is its tile's start
//         plus the number of earlier Gaussians, in depth order, whose
//         rectangle holds the tile. Two counting sorts with few buckets each
//         get there: Gaussians into the lists of the tile rows they span, then
//         each row's items into the row's tiles. No (tile, Gaussian) item is
//         materialised before its final slot.
//      b. radix (larger frames): duplication of each Gaussian, in depth order,
//         into (tile id | Gaussian id) items, then a stable LSD radix sort of
//         the M items on the tile id (ceil(bits(tiles) / 8) passes).
// Both give the stable 64-bit key order: within a tile, entries are in
// (depth bits, Gaussian index) order.
//
// The per-tile entry counts, hence the tile ranges and the digit histograms of
// the tile passes, come from the footprints alone: in each tile row it touches,
// a kept Gaussian adds +1 at its first tile and -1 past its last to a
// difference grid whose prefix sum along the row is the entries of each tile.
// (A Gaussian touches, in each row of its bounding rectangle, the tiles whose
// column meets its footprint disc: row_span.)
//
// Each radix pass is a single sweep over (key | value) items: a block counts
// the digits of its 5120 items and publishes those counts at once, ranks the
// items within each warp with ballots, looks back over earlier blocks (eight
// at a time) for its global digit offsets, and scatters the items staged in
// digit order. Every wait on another block or warp is bounded (kMaxSpin polls);
// on expiry it records IGS_ERR_DEVICE_TIMEOUT, which aborts the frame.
#include <algorithm>
#include <mutex>

#include "binning.cuh"

namespace igs {
namespace {

// Difference grid kept in shared memory by the preparation kernel up to this many cells.
constexpr int kGridSmemCells = 10240;

// Counting sort of the entries (route a), below.
constexpr int kRowWalkMax = 2048;          // tiles per axis for route a (shared-memory buckets)
constexpr uint32_t kL1ChunksMax = 16384;   // most level-1 chunks (columns of H1), fewer for tall frames
constexpr uint32_t kL1ChunksMin = 1024;
constexpr uint32_t kH1Words = 1u << 22;    // H1 budget: rows x chunks
constexpr uint32_t kStage = 1536;          // staged entries per level-2 chunk
constexpr uint32_t kChunkTarget = kStage * 4 / 5;
constexpr uint32_t kStage1 = 768;          // staged 8-byte items per level-1 chunk
constexpr uint32_t kChunkTarget1 = kStage1 * 4 / 5;
constexpr int kWalkWarps = 4;              // warps per CTA of the walk kernels (one chunk each)
constexpr int kWalkUnroll = 8;             // items per lane per round of the counting walks

// Depth-digit histograms of all n depth keys, the kept count, and for every kept
// Gaussian, in each tile row, +1 at its first touched tile and -1 past its last
// in the (tiles_y+1) x (tiles_x+1) grid (a prefix sum along each row then gives
// the entries of every tile); with rectangle footprints on the shared-memory
// grid, +1/-1 at the rectangle's four corners instead (a prefix down each
// column, then along each row). Each thread has kPrepUnroll Gaussians in flight;
// the top byte of a view's depths is mostly one value, so a warp whose lanes
// share it adds its count once instead of 32 times to one shared-memory word.
// With rowd (the counting-sort route), also +1 at the first row of every kept
// Gaussian's rectangle and -1 past its last in rowd[tiles_y + 1] (a prefix
// sum over the rows then gives each tile row's level-1 list length); on the
// shared-memory grid these sit after the grid's cells.
constexpr int kPrepUnroll = 4;
template <bool SMEM_GRID>
__global__ void __launch_bounds__(256) k_bin_prep(const uint32_t* __restrict__ depth_key, const uint2* __restrict__ rect,
                                                  const float4* __restrict__ disc, int tile, int footprint,
                                                  const uint32_t* __restrict__ count, uint32_t n, int gx,
                                                  int gy, uint32_t* __restrict__ hist, int32_t* __restrict__ grid,
                                                  int32_t* __restrict__ rowd, uint32_t* __restrict__ info) {
    pdl_wait();
    extern __shared__ int32_t s_grid[];
    __shared__ uint32_t s_h[4][kRadix];
    const int cells = gx * gy;
    const int rowd_cells = rowd ? gy : 0;
    int32_t* rd = SMEM_GRID ? s_grid + cells : rowd;
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = 0;
    if (SMEM_GRID)
        for (int k = threadIdx.x; k < cells + rowd_cells; k += blockDim.x) s_grid[k] = 0;
    __syncthreads();
    int32_t* g = SMEM_GRID ? s_grid : grid;
    const float inv = 1.0f / (float)tile;
    uint32_t kept = 0;
    bool wrap = false;
    const uint32_t stride = gridDim.x * blockDim.x;
    // every lane of a warp runs the same iterations (the counts below are warp-collective)
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; i0 < n;
         i0 += (uint64_t)stride * kPrepUnroll) {
        uint32_t key[kPrepUnroll], cnt[kPrepUnroll];
        uint2 r[kPrepUnroll];
#pragma unroll
        for (int u = 0; u < kPrepUnroll; ++u) {  // independent loads first
            const uint64_t i = i0 + (uint64_t)u * stride + lane;
            const bool ok = i < n;
            key[u] = ok ? depth_key[i] : 0u;
            cnt[u] = ok ? count[i] : 0u;
            r[u] = ok ? rect[i] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kPrepUnroll; ++u) {
            const uint64_t i = i0 + (uint64_t)u * stride + lane;
            const bool ok = i < n;
            const uint32_t k = key[u];
            if (ok) {
                atomicAdd(&s_h[0][k & 0xFF], 1u);
                atomicAdd(&s_h[1][(k >> 8) & 0xFF], 1u);
            }
            if (ok) atomicAdd(&s_h[2][(k >> 16) & 0xFF], 1u);
            {  // the top byte: one count per warp when all its lanes share it (a view's depths do)
                const uint32_t d3 = k >> 24, okm = __ballot_sync(0xffffffffu, ok);
                const uint32_t lead = __shfl_sync(0xffffffffu, d3, okm ? __ffs(okm) - 1 : 0);
                if (__all_sync(0xffffffffu, !ok || d3 == lead)) {
                    if (okm && lane == __ffs(okm) - 1) atomicAdd(&s_h[3][lead], (uint32_t)__popc(okm));
                } else if (ok) {
                    atomicAdd(&s_h[3][d3], 1u);
                }
            }
            wrap |= ok && k != 0xFFFFFFFFu && ((k & 0xFFFFFFu) == 0xFFFFFFu || (k >> 24) == 0xFFu);
            if (cnt[u]) {
                ++kept;
                const int y0 = r[u].x >> 16, y1 = r[u].y >> 16;
                if (rowd) {
                    atomicAdd(&rd[y0], 1);
                    atomicAdd(&rd[y1 + 1], -1);
                }
                if (SMEM_GRID && footprint == 0) {  // the rectangle's four corners (a 2D difference)
                    const int x0 = r[u].x & 0xFFFF, x1 = r[u].y & 0xFFFF;
                    atomicAdd(&g[y0 * gx + x0], 1);
                    atomicAdd(&g[y0 * gx + x1 + 1], -1);
                    atomicAdd(&g[(y1 + 1) * gx + x0], -1);
                    atomicAdd(&g[(y1 + 1) * gx + x1 + 1], 1);
                } else {
                    for (int ty = y0; ty <= y1; ++ty) {  // +1 at the row's first touched tile, -1 past its last
                        const int2 sp = tile_span(footprint, r[u], disc, i, tile, inv, ty);
                        if (sp.y < sp.x) continue;
                        atomicAdd(&g[ty * gx + sp.x], 1);
                        atomicAdd(&g[ty * gx + sp.y + 1], -1);
                    }
                }
            }
        }
    }
    kept = __reduce_add_sync(0xffffffffu, kept);
    if (lane == 0 && kept) atomicAdd(&info[kInfoKept], kept);
    if (__any_sync(0xffffffffu, wrap) && lane == 0) atomicOr(&info[kInfoKeyWrap], 1u);
    __syncthreads();
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) {
        const uint32_t v = (&s_h[0][0])[k];
        if (v) atomicAdd(&hist[k], v);
    }
    if (SMEM_GRID) {
        for (int k = threadIdx.x; k < cells; k += blockDim.x)
            if (s_grid[k]) atomicAdd(&grid[k], s_grid[k]);
        for (int k = threadIdx.x; k < rowd_cells; k += blockDim.x)
            if (s_grid[cells + k]) atomicAdd(&rowd[k], s_grid[cells + k]);
    }
}

// Inclusive prefix of the difference grid along each row: afterwards grid[y][x]
// holds the number of kept Gaussians that touch tile (x, y).
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

// The tile total M (summed in 64 bits over the block's threads): entries the
// frame needs; over the capacity, the frame is aborted with IGS_ERR_CAPACITY.
__device__ __forceinline__ void publish_tile_total(unsigned long long* s_total, uint32_t sum, uint64_t capacity,
                                                   uint32_t* __restrict__ info) {
    unsigned long long w = sum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(s_total, w);  // one per warp
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long M = *s_total;
        const uint32_t m32 = (uint32_t)min(M, (unsigned long long)0xFFFFFFFFu);
        info[kInfoTileTotal] = m32;
        info[kInfoM] = m32;
        info[kInfoNeed] = m32;
        if (M > capacity) {
            atomicCAS(&info[kInfoErr], 0u, (uint32_t)IGS_ERR_CAPACITY);
            info[kInfoAbort] = 1u;
        }
    }
}

// Row layout of the counting sort, by one block of NT threads once the tile
// ranges are known (after publish_tile_total). len[y]: the kept Gaussians whose
// rectangle spans tile row y (prefix of the row differences rowd), the length
// of row y's level-1 list. rowinfo = [rows] list starts (prefix of len),
// [rows] first level-2 chunk, [rows] items per level-2 chunk, [1] level-2 chunk
// total. A row's level-2 chunks take about kChunkTarget entries each:
// kChunkTarget * len / entries items, at least 32, where the row's entries are
// rowstart[y + 1] - rowstart[y] (rowstart[y]: the first entry of the row's
// tiles, held in column tiles_x of the grid g; rowstart[rows] = M). Records an
// error if the chunks exceed max_chunks.
template <int NT>
__device__ __forceinline__ void row_layout(const int32_t* __restrict__ rowd, const int32_t* g, int gx, uint32_t rows,
                                           uint32_t tiles_x, uint32_t M, uint32_t max_chunks,
                                           uint32_t* __restrict__ len, uint32_t* __restrict__ rowinfo,
                                           uint32_t* __restrict__ info, uint32_t* s_warp) {
    __syncthreads();  // the row starts, written by other threads
    auto rowstart = [&](uint32_t y) { return y < rows ? (uint32_t)g[(size_t)y * gx + tiles_x] : M; };
    const uint32_t per = (rows + NT - 1) / NT;
    const uint32_t y0 = min(rows, threadIdx.x * per), y1 = min(rows, y0 + per);
    uint32_t dsum = 0;
    for (uint32_t y = y0; y < y1; ++y) dsum += (uint32_t)rowd[y];
    const uint32_t lfirst = block_excl_scan<NT>(dsum, s_warp);  // modulo 2^32: the differences' prefix
    uint32_t items = 0, chunks = 0, run = lfirst;
    for (uint32_t y = y0; y < y1; ++y) {
        run += (uint32_t)rowd[y];
        const uint32_t ly = run;
        const uint64_t entries = rowstart(y + 1) - rowstart(y);
        const uint32_t size =
            (uint32_t)max((uint64_t)32, entries ? (uint64_t)kChunkTarget * ly / entries : (uint64_t)kChunkTarget);
        len[y] = ly;
        rowinfo[2 * rows + y] = size;
        items += ly;
        chunks += (ly + size - 1) / size;
    }
    uint32_t start = block_excl_scan<NT>(items, s_warp);
    uint32_t base = block_excl_scan<NT>(chunks, s_warp);
    if (threadIdx.x == NT - 1) {
        rowinfo[3 * rows] = base + chunks;
        if (base + chunks > max_chunks) record_error(info, IGS_ERR_CUDA);  // never expected: chunks are bounded
    }
    run = lfirst;
    for (uint32_t y = y0; y < y1; ++y) {
        run += (uint32_t)rowd[y];
        const uint32_t size = rowinfo[2 * rows + y];
        rowinfo[y] = start;
        rowinfo[rows + y] = base;
        start += run;
        base += (run + size - 1) / size;
    }
}

// One block: tile ranges = exclusive scan of the per-tile counts (row-major tile
// order), (0, 0) for empty tiles; digit histograms of the tile-id passes; with
// rowd, the row layout of the counting sort (row_layout).
constexpr int kTileScanThreads = 1024;
__global__ void __launch_bounds__(kTileScanThreads) k_tile_scan(const int32_t* grid, int gx, int tiles_x,
                                                                uint32_t tiles, int passes,
                                                                uint2* __restrict__ ranges,
                                                                uint32_t* __restrict__ hist_tile,
                                                                uint32_t* __restrict__ info, uint64_t capacity,
                                                                int32_t* __restrict__ grid_w,
                                                                const int32_t* __restrict__ rowd,
                                                                uint32_t max_chunks, uint32_t* __restrict__ len,
                                                                uint32_t* __restrict__ rowinfo) {
    __shared__ uint32_t s_h[4][kRadix];
    __shared__ uint32_t s_warp[kTileScanThreads / 32];
    __shared__ unsigned long long s_total;
    if (threadIdx.x == 0) s_total = 0ull;
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = 0;
    const uint32_t per = (tiles + kTileScanThreads - 1) / kTileScanThreads;
    const uint32_t t0 = min(tiles, threadIdx.x * per), t1 = min(tiles, t0 + per);
    uint32_t sum = 0;
    for (uint32_t t = t0; t < t1; ++t) sum += (uint32_t)grid[(size_t)(t / tiles_x) * gx + (t % tiles_x)];
    __syncthreads();
    uint32_t start = block_excl_scan<kTileScanThreads>(sum, s_warp);
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t c = (uint32_t)grid[(size_t)(t / tiles_x) * gx + (t % tiles_x)];
        if (rowd && t % tiles_x == 0) grid_w[(size_t)(t / tiles_x) * gx + tiles_x] = (int32_t)start;  // row start
        ranges[t] = c ? make_uint2(start, start + c) : make_uint2(0u, 0u);
        start += c;
        if (c)
            for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(t >> (8 * p)) & 0xFF], c);
    }
    publish_tile_total(&s_total, sum, capacity, info);
    for (int k = threadIdx.x; k < passes * kRadix; k += blockDim.x) hist_tile[k] = (&s_h[0][0])[k];
    if (rowd) {
        __threadfence_block();
        row_layout<kTileScanThreads>(rowd, grid_w, gx, tiles / tiles_x, tiles_x,
                                     (uint32_t)min(s_total, (unsigned long long)0xFFFFFFFFu), max_chunks, len,
                                     rowinfo, info, s_warp);
    }
}

// One block, grid in shared memory (cells <= kGridSmemCells): the row prefix of
// the difference grid, the tile ranges, the tile-digit histograms, every digit
// histogram (4 depth + `passes` tile rows) turned into exclusive offsets, and
// with rowd the row layout of the counting sort (row_layout).
constexpr int kTilesSmallThreads = 1024;
__global__ void __launch_bounds__(kTilesSmallThreads) k_tiles_small(const int32_t* __restrict__ grid, int tiles_x,
                                                                    int tiles_y, int passes, int diff2d,
                                                                    uint2* __restrict__ ranges,
                                                                    uint32_t* __restrict__ hist,
                                                                    uint32_t* __restrict__ info, uint64_t capacity,
                                                                    const int32_t* __restrict__ rowd,
                                                                    uint32_t max_chunks, uint32_t* __restrict__ len,
                                                                    uint32_t* __restrict__ rowinfo) {
    pdl_wait();
    extern __shared__ int32_t s_g[];
    __shared__ uint32_t s_h[8][kRadix];
    __shared__ uint32_t s_warp[kTilesSmallThreads / 32];
    __shared__ unsigned long long s_total;
    if (threadIdx.x == 0) s_total = 0ull;
    const int gx = tiles_x + 1, cells = gx * (tiles_y + 1);
    const int tid = threadIdx.x;
    for (int k = tid; k < cells; k += blockDim.x) s_g[k] = grid[k];
    for (int k = tid; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = hist[k];          // depth counts
    for (int k = tid; k < 4 * kRadix; k += blockDim.x) (&s_h[4][0])[k] = 0;                // tile counts
    __syncthreads();
    if (tid < 32) {  // skip the top depth pass: at most one top byte other than the culled 0xFF, no wrap
        uint32_t nz = 0;
        for (int b = tid; b < kRadix - 1; b += 32) nz += s_h[3][b] != 0u;
        nz = __reduce_add_sync(0xffffffffu, nz);
        if (tid == 0) info[kInfoSkipTop] = (nz <= 1u && info[kInfoKeyWrap] == 0u) ? 1u : 0u;
    }
    if (diff2d) {  // rectangles were added as 2D differences: a prefix down each column first
        for (int x = tid; x < tiles_x; x += blockDim.x) {
            int32_t run = 0;
            for (int y = 0; y < tiles_y; ++y) { run += s_g[y * gx + x]; s_g[y * gx + x] = run; }
        }
        __syncthreads();
    }
    for (int y = tid; y < tiles_y; y += blockDim.x) {
        int32_t run = 0;
        for (int x = 0; x < tiles_x; ++x) { run += s_g[y * gx + x]; s_g[y * gx + x] = run; }
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
        if (t % tiles_x == 0) s_g[(t / tiles_x) * gx + tiles_x] = (int32_t)start;  // row start (column tiles_x is free)
        ranges[t] = c ? make_uint2(start, start + c) : make_uint2(0u, 0u);
        start += c;
        if (c)
            for (int p = 0; p < passes; ++p) atomicAdd(&s_h[4 + p][(t >> (8 * p)) & 0xFF], c);
    }
    publish_tile_total(&s_total, sum, capacity, info);
    // exclusive offsets of every histogram row: a warp scans 32 consecutive digits of one
    // row, then adds the totals of the row's earlier warps
    const int rows = 4 + passes;
    __shared__ uint32_t s_wt[8 * kRadix / 32];
    const int lane = tid & 31;
    uint32_t v[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int idx = tid + r * kTilesSmallThreads;
        const uint32_t x = idx < rows * kRadix ? (&s_h[0][0])[idx] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wt[idx >> 5] = incl;
        v[r] = incl - x;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int idx = tid + r * kTilesSmallThreads;
        if (idx < rows * kRadix) {
            uint32_t base = 0;
            for (int k = (idx >> 8) * (kRadix / 32); k < (idx >> 5); ++k) base += s_wt[k];
            hist[idx] = v[r] + base;
        }
    }
    if (rowd)
        row_layout<kTilesSmallThreads>(rowd, s_g, gx, (uint32_t)tiles_y, (uint32_t)tiles_x,
                                       (uint32_t)min(s_total, (unsigned long long)0xFFFFFFFFu), max_chunks, len,
                                       rowinfo, info, s_warp);
}

// ---- counting sort of the entries by tile (route a) ----
//
// Two levels, each a counting sort with few buckets:
//   level 1 places each kept Gaussian, in depth order, into the list of every
//            tile row its rectangle spans (buckets: rows; items: Gaussian ids);
//   level 2 places each item of a row, in list order, into every tile of that
//            row its rectangle spans (buckets: the row's tiles; items: entries).
// A level counts its chunks' items per bucket (shared memory), scans the counts
// down each bucket over the chunks, and walks the chunks again placing items.
// Placement keeps order within a bucket (Placer below). Chunks are sized
// so that their items fill about 4/5 of a shared-memory stage.

// Level-1 chunk c: positions [p0, p1) of the depth order among the kept
// Gaussians; `used` chunks hold Gaussians. A chunk takes about kChunkTarget1 /
// sqrt(M / kept) Gaussians (the rows of an isotropic footprint are about the
// square root of its tiles).
struct Chunk {
    uint32_t p0, p1, used;
};
__device__ __forceinline__ Chunk l1_chunk(uint32_t c, uint32_t cmax, const uint32_t* __restrict__ info) {
    const uint32_t kept = info[kInfoKept], M = info[kInfoM];
    const float rows_per = kept ? fmaxf(1.f, sqrtf((float)M / (float)kept)) : 1.f;
    const uint32_t target = max(32u, (uint32_t)((float)kChunkTarget1 / rows_per));
    const uint32_t per = max(target, (uint32_t)ceil_div(kept, cmax));
    Chunk ch;
    ch.used = (uint32_t)ceil_div(kept, per);
    ch.p0 = (uint32_t)min((uint64_t)kept, (uint64_t)c * per);
    ch.p1 = (uint32_t)min((uint64_t)kept, (uint64_t)ch.p0 + per);
    return ch;
}

// A warp's stable placement of one chunk whose items each span a contiguous
// range of buckets [lo, hi], one batch of 32 items (one per lane, in order) at
// a time. Each lane marks its bit at the start of its range (smask[lo]) and
// past its end (emask[hi + 1]); a warp-wide XOR prefix over the batch's
// buckets turns the marks into each bucket's covering mask (the lanes whose
// range holds it: a bit marked at both ends cancels); an item's slot in
// bucket q = the bucket's cursor + the earlier lanes of the covering mask, and
// each bucket's cursor then advances by the mask's size. Two marks per item
// instead of one per (item, bucket), and no per-bucket pass diverges but the
// slot writes. Items go to a shared-memory stage grouped by bucket and leave
// by stage slot (lane l takes slots l, l + 32, ..., each to its bucket's run
// in the output; a chunk too large for the stage writes its items directly). Items are of type T (the value an item
// takes in bucket q comes from a functor); the stage holds S of them. Shared
// memory: words(B) 32-bit words, an even count (8-byte items stay aligned).
template <typename T, uint32_t S>
struct Placer {
    uint32_t *pos, *smask, *emask, *cov, *first, *lstart;
    T* stage;
    uint32_t B;
    bool staged;
    __host__ __device__ static constexpr uint32_t words(uint32_t B) {
        return 6 * B + 6 + S * (uint32_t)(sizeof(T) / 4);
    }
    __device__ __forceinline__ Placer(uint32_t* ws, uint32_t nb) : B(nb), staged(false) {
        pos = ws;
        smask = pos + nb;          // nb + 1 words
        emask = smask + nb + 1;    // nb + 2 words
        cov = emask + nb + 2;      // nb words
        first = cov + nb;
        lstart = first + nb;       // nb + 1 words (+ 2 pad)
        stage = reinterpret_cast<T*>(ws + 6 * nb + 6);
    }
    // first_slot(q): the chunk's first slot in bucket q of the output; count(q): its items there
    template <typename First, typename Count>
    __device__ __forceinline__ void init(int lane, First first_slot, Count count) {
        for (uint32_t q = lane; q < B; q += 32) {  // coalesced, independent loads
            first[q] = first_slot(q);
            lstart[q] = count(q);
        }
        for (uint32_t q = lane; q < B + 2; q += 32) {
            emask[q] = 0u;
            if (q <= B) smask[q] = 0u;
        }
        __syncwarp();
        const uint32_t per = (B + 31) / 32, q0 = min(B, lane * per), q1 = min(B, q0 + per);
        uint32_t sum = 0;
        for (uint32_t q = q0; q < q1; ++q) sum += lstart[q];
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        staged = total <= S;
        uint32_t run = incl - sum;
        for (uint32_t q = q0; q < q1; ++q) {
            const uint32_t c = lstart[q];
            lstart[q] = run;
            pos[q] = staged ? run : first[q];
            run += c;
        }
        if (lane == 31) lstart[B] = total;
        __syncwarp();
    }
    // one batch: this lane's item (none if lo > hi) spans buckets lo..hi and takes value item(q) in bucket q
    template <typename Item>
    __device__ __forceinline__ void batch(uint32_t lo, uint32_t hi, Item item, int lane, T* __restrict__ out) {
        const uint32_t bit = 1u << lane, lt = bit - 1u;
        const bool any = lo <= hi;
        if (any) {
            atomicOr(&smask[lo], bit);
            atomicOr(&emask[hi + 1], bit);
        }
        const uint32_t qmin = __reduce_min_sync(0xffffffffu, any ? lo : 0xFFFFFFFFu);
        const uint32_t qmax = __reduce_max_sync(0xffffffffu, any ? hi : 0u);
        if (qmin > qmax) return;  // warp-uniform: no item spans a bucket
        __syncwarp();
        // covering masks: lanes whose span holds q = XOR of start and end marks up to q
        uint32_t carry = 0u;
        for (uint32_t base = qmin; base <= qmax; base += 32) {
            const uint32_t q = base + lane;
            uint32_t x = q <= qmax ? (smask[q] ^ emask[q]) : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x ^= y;
            }
            x ^= carry;
            if (q <= qmax) cov[q] = x;
            carry = __shfl_sync(0xffffffffu, x, 31);
        }
        __syncwarp();
        for (uint32_t q = lo; q <= hi; ++q) {
            const uint32_t at = pos[q] + __popc(cov[q] & lt);
            const T v = item(q);
            if (staged) stage[at] = v; else out[at] = v;
        }
        __syncwarp();
        for (uint32_t base = qmin; base <= qmax; base += 32) {
            const uint32_t q = base + lane;
            if (q <= qmax) {
                pos[q] += __popc(cov[q]);
                smask[q] = 0u;
                emask[q] = 0u;
            }
        }
        if (lane == 0) emask[qmax + 1] = 0u;  // ends past the last bucket of the batch
        __syncwarp();
    }
    // staged chunk: every bucket's run to out[first[q] ...]; lane l takes stage slots l, l + 32, ...,
    // each written to its bucket's output run (a warp store covers 32 consecutive slots)
    __device__ __forceinline__ void flush(T* __restrict__ out, int lane) {
        if (!staged) return;
        const uint32_t total = lstart[B];
        uint32_t q = 0;  // the bucket holding stage slot e: slots rise, so q only moves forward
        for (uint32_t e = lane; e < total; e += 32) {
            while (lstart[q + 1] <= e) ++q;
            out[first[q] + (e - lstart[q])] = stage[e];
        }
    }
};
// What the level-1 placement needs to give each row item the tiles its Gaussian
// touches in that row: the rectangles, or with footprint 1 the discs (disc_span).
struct DiscRef {
    const uint2* rect;
    const float4* disc;
    int tile;
    float inv_tile;
    int footprint;
};

using Placer1 = Placer<u64, kStage1>;      // level 1: (column span << 32 | Gaussian id) items
using Placer2 = Placer<uint32_t, kStage>;  // level 2: Gaussian ids

// In place: the warp turns the difference counts d[0..B) (+1 where an item's
// bucket range starts, -1 past its end) into each bucket's item count, and
// writes count q to out(q). Lanes take consecutive runs of buckets.
template <typename Out>
__device__ __forceinline__ void diff_to_counts(const uint32_t* d, uint32_t B, int lane, Out out) {
    const uint32_t per = (B + 31) / 32, q0 = min(B, lane * per), q1 = min(B, q0 + per);
    uint32_t sum = 0;
    for (uint32_t q = q0; q < q1; ++q) sum += d[q];
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    uint32_t run = incl - sum;  // modulo 2^32: the prefix of the differences is a count
    for (uint32_t q = q0; q < q1; ++q) {
        run += d[q];
        out(q, run);
    }
}

// Level 1, count: for each of its chunks c (grid-stride over warps), a warp adds,
// for each Gaussian of the chunk, one to every row of its rectangle (as +1 at
// its first row and -1 past its last, summed along the rows at the end); writes
// column c of H1 [rows][cmax], and the rectangles in depth order (srect[p] =
// rect[order[p]]) so that the placement reads them without a gather.
__global__ void __launch_bounds__(32 * kWalkWarps) k_rows_count(const uint32_t* __restrict__ order,
                                                                const uint2* __restrict__ rect, uint32_t rows,
                                                                uint32_t cmax, uint32_t* __restrict__ H1,
                                                                uint2* __restrict__ srect,
                                                                const uint32_t* __restrict__ info) {
    pdl_wait();
    extern __shared__ uint32_t s_walk[];
    const int lane = threadIdx.x & 31;
    uint32_t* cnt = s_walk + (size_t)(threadIdx.x >> 5) * (rows + 1);  // difference counts
    if (info[kInfoAbort]) return;
    const uint32_t used = l1_chunk(0, cmax, info).used;
    for (uint32_t c = blockIdx.x * kWalkWarps + (threadIdx.x >> 5); c < used; c += gridDim.x * kWalkWarps) {
        const Chunk ch = l1_chunk(c, cmax, info);
        for (uint32_t y = lane; y <= rows; y += 32) cnt[y] = 0u;
        __syncwarp();
        for (uint32_t b = ch.p0; b < ch.p1; b += 32 * kWalkUnroll) {
            uint32_t g[kWalkUnroll];
            uint32_t ry[kWalkUnroll];
#pragma unroll
            for (int k = 0; k < kWalkUnroll; ++k) {
                const uint32_t p = b + k * 32 + lane;
                g[k] = p < ch.p1 ? order[p] : 0xFFFFFFFFu;
            }
#pragma unroll
            for (int k = 0; k < kWalkUnroll; ++k) {
                const uint2 r = g[k] != 0xFFFFFFFFu ? rect[g[k]] : make_uint2(1u << 16, 0u);  // rows 1..0: none
                ry[k] = (r.x >> 16) | (r.y & 0xFFFF0000u);
                if (g[k] != 0xFFFFFFFFu) srect[b + k * 32 + lane] = r;  // the placement reads it in order
            }
#pragma unroll
            for (int k = 0; k < kWalkUnroll; ++k) {
                const uint32_t y0 = ry[k] & 0xFFFF, y1 = ry[k] >> 16;
                if (y0 <= y1) {
                    atomicAdd(&cnt[y0], 1u);
                    atomicAdd(&cnt[y1 + 1], 0xFFFFFFFFu);
                }
            }
        }
        __syncwarp();
        diff_to_counts(cnt, rows, lane, [&](uint32_t y, uint32_t v) { H1[(size_t)y * cmax + c] = v; });
        __syncwarp();  // the next chunk clears what this one read
    }
}

// Level 1, scan: block y turns row y of H1 (the used chunks' counts) into
// exclusive offsets in place. The row's total must equal len[y], the list
// length the row layout was built from (both count the kept Gaussians whose
// rectangle spans row y); a difference records an error and aborts the frame
// before any placement.
constexpr int kRowScanThreads = 1024;
__global__ void __launch_bounds__(kRowScanThreads) k_rows_scan(uint32_t* __restrict__ H1, uint32_t cmax,
                                                               const uint32_t* __restrict__ len,
                                                               uint32_t* __restrict__ info) {
    pdl_wait();
    __shared__ uint32_t s_warp[kRowScanThreads / 32];
    if (info[kInfoAbort]) return;
    uint32_t* row = H1 + (size_t)blockIdx.x * cmax;
    const uint32_t used = l1_chunk(0, cmax, info).used;
    const uint32_t per = (used + kRowScanThreads - 1) / kRowScanThreads;
    const uint32_t c0 = min(used, threadIdx.x * per), c1 = min(used, c0 + per);
    uint32_t sum = 0;
    for (uint32_t c = c0; c < c1; ++c) sum += row[c];
    uint32_t run = block_excl_scan<kRowScanThreads>(sum, s_warp);
    if (threadIdx.x == kRowScanThreads - 1 && run + sum != len[blockIdx.x])
        record_error(info, IGS_ERR_CUDA);  // never expected: the row counts disagree
    for (uint32_t c = c0; c < c1; ++c) {
        const uint32_t h = row[c];
        row[c] = run;
        run += h;
    }
}

// Level 1, place: a warp walks each of its chunks again and puts each Gaussian
// into the list of every row of its rectangle (R1, rows one after another), as
// the item (xa | xb << 16) << 32 | id with the tiles [xa, xb] it touches in
// that row ((1, 0): none), so that level 2 reads its items without a gather.
__global__ void __launch_bounds__(32 * kWalkWarps) k_rows_place(const uint32_t* __restrict__ order,
                                                                const uint2* __restrict__ srect, DiscRef disc,
                                                                uint32_t rows,
                                                                uint32_t cmax, const uint32_t* __restrict__ H1,
                                                                const uint32_t* __restrict__ len,
                                                                const uint32_t* __restrict__ rowinfo,
                                                                u64* __restrict__ R1,
                                                                const uint32_t* __restrict__ info) {
    pdl_wait();
    extern __shared__ uint32_t s_walk[];
    const int lane = threadIdx.x & 31;
    if (info[kInfoAbort]) return;
    const uint32_t used = l1_chunk(0, cmax, info).used;
    for (uint32_t c = blockIdx.x * kWalkWarps + (threadIdx.x >> 5); c < used; c += gridDim.x * kWalkWarps) {
        const Chunk ch = l1_chunk(c, cmax, info);
        // the first batch's items load while the placer reads the chunk's bucket offsets
        uint32_t g_next = ch.p0 + lane < ch.p1 ? order[ch.p0 + lane] : 0xFFFFFFFFu;
        uint2 r_next = ch.p0 + lane < ch.p1 ? srect[ch.p0 + lane] : make_uint2(1u << 16, 0u);  // rows 1..0: none
        Placer1 rs(s_walk + (size_t)(threadIdx.x >> 5) * Placer1::words(rows), rows);
        auto first = [&](uint32_t y) { return rowinfo[y] + H1[(size_t)y * cmax + c]; };
        rs.init(lane, first, [&](uint32_t y) {
            const uint32_t* h = H1 + (size_t)y * cmax;
            return (c + 1 < ch.used ? h[c + 1] : len[y]) - h[c];
        });
        for (uint32_t b = ch.p0; b < ch.p1; b += 32) {
            const uint32_t g = g_next;
            const uint2 r = r_next;
            const bool more = b + 32 + lane < ch.p1;
            g_next = more ? order[b + 32 + lane] : 0xFFFFFFFFu;
            r_next = more ? srect[b + 32 + lane] : make_uint2(1u << 16, 0u);
            if (disc.footprint == 0) {  // every row: the rectangle's columns
                const u64 item = (u64)g | ((u64)((r.x & 0xFFFFu) | (r.y << 16)) << 32);
                rs.batch(r.x >> 16, r.y >> 16, [&](uint32_t) { return item; }, lane, R1);
            } else {  // per row: the columns the disc meets there
                const float4 d = g != 0xFFFFFFFFu ? disc.disc[g] : make_float4(0.f, 0.f, 0.f, 0.f);
                rs.batch(r.x >> 16, r.y >> 16, [&](uint32_t y) {
                    int2 sp = disc_span(d, disc.tile, disc.inv_tile, (int)y);
                    if (sp.y < sp.x) sp = make_int2(1, 0);
                    return (u64)g | ((u64)((uint32_t)sp.x | ((uint32_t)sp.y << 16)) << 32);
                }, lane, R1);
            }
        }
        rs.flush(R1, lane);
        __syncwarp();  // the next chunk's init rewrites what the flush reads
    }
}

// Level-2 chunk j: row y (largest y whose first chunk is <= j; rows without
// chunks share the next row's base) and items [i0, i1) of R1.
struct RowChunk {
    uint32_t y, i0, i1;
};
__device__ __forceinline__ RowChunk l2_chunk(uint32_t j, uint32_t rows, const uint32_t* __restrict__ rowinfo,
                                             const uint32_t* __restrict__ len) {
    uint32_t lo = 0, hi = rows;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (rowinfo[rows + mid] <= j) lo = mid; else hi = mid;
    }
    RowChunk rc;
    rc.y = lo;
    const uint32_t start = rowinfo[lo], size = rowinfo[2 * rows + lo];
    rc.i0 = start + (j - rowinfo[rows + lo]) * size;
    rc.i1 = min(start + len[lo], rc.i0 + size);
    return rc;
}

// Level 2, count: for each of its chunks j, a warp adds, for each item of the
// chunk, one to every tile of the row that the item's Gaussian touches (the
// span the item carries, as +1 at its first tile and -1 past its last, summed
// along the row at the end); writes row j of H2 [chunks][tiles_x].
__global__ void __launch_bounds__(32 * kWalkWarps) k_cols_count(const u64* __restrict__ R1, uint32_t rows,
                                                                uint32_t tiles_x, const uint32_t* __restrict__ len,
                                                                const uint32_t* __restrict__ rowinfo,
                                                                uint32_t* __restrict__ H2,
                                                                const uint32_t* __restrict__ info) {
    pdl_wait();
    extern __shared__ uint32_t s_walk[];
    const int lane = threadIdx.x & 31;
    uint32_t* cnt = s_walk + (size_t)(threadIdx.x >> 5) * (tiles_x + 1);  // difference counts
    if (info[kInfoAbort]) return;
    const uint32_t total = rowinfo[3 * rows];
    for (uint32_t j = blockIdx.x * kWalkWarps + (threadIdx.x >> 5); j < total; j += gridDim.x * kWalkWarps) {
        const RowChunk rc = l2_chunk(j, rows, rowinfo, len);
        for (uint32_t x = lane; x <= tiles_x; x += 32) cnt[x] = 0u;
        __syncwarp();
        for (uint32_t b = rc.i0; b < rc.i1; b += 32 * kWalkUnroll) {
            uint32_t sp[kWalkUnroll];
#pragma unroll
            for (int k = 0; k < kWalkUnroll; ++k) {
                const uint32_t i = b + k * 32 + lane;
                sp[k] = i < rc.i1 ? (uint32_t)(R1[i] >> 32) : 1u;  // (1, 0): no tiles
            }
#pragma unroll
            for (int k = 0; k < kWalkUnroll; ++k) {
                const uint32_t x0 = sp[k] & 0xFFFFu, x1 = sp[k] >> 16;
                if (x0 <= x1) {
                    atomicAdd(&cnt[x0], 1u);
                    atomicAdd(&cnt[x1 + 1], 0xFFFFFFFFu);
                }
            }
        }
        __syncwarp();
        uint32_t* out = H2 + (size_t)j * tiles_x;
        diff_to_counts(cnt, tiles_x, lane, [&](uint32_t x, uint32_t v) { out[x] = v; });
        __syncwarp();  // the next chunk clears what this one read
    }
}

// Level 2, scan: block (y, b) turns, for tiles 32 b .. 32 b + 31 of row y, the
// counts of the row's chunks into slots (tile start + earlier chunks), in
// place. Lanes take tiles, the block's warps take consecutive segments of the
// row's chunks.
constexpr int kColScanWarps = 16;
__global__ void __launch_bounds__(32 * kColScanWarps) k_cols_scan(uint32_t* __restrict__ H2, uint32_t rows,
                                                                  uint32_t tiles_x, const uint2* __restrict__ ranges,
                                                                  const uint32_t* __restrict__ rowinfo,
                                                                  const uint32_t* __restrict__ info) {
    pdl_wait();
    __shared__ uint32_t s_seg[kColScanWarps][32];
    if (info[kInfoAbort]) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t y = blockIdx.x;
    const uint32_t j0 = rowinfo[rows + y], j1 = y + 1 < rows ? rowinfo[rows + y + 1] : rowinfo[3 * rows];
    const uint32_t per = (j1 - j0 + kColScanWarps - 1) / kColScanWarps;
    const uint32_t s0 = min(j1, j0 + w * per), s1 = min(j1, s0 + per);
    for (uint32_t x0 = blockIdx.y * 32; x0 < min(tiles_x, blockIdx.y * 32 + 32); x0 += 32) {
        const uint32_t x = x0 + lane;
        const bool on = x < tiles_x;
        uint32_t sum = 0;
        if (on)
            for (uint32_t j = s0; j < s1; ++j) sum += H2[(size_t)j * tiles_x + x];
        s_seg[w][lane] = sum;
        __syncthreads();
        uint32_t run = on ? ranges[(size_t)y * tiles_x + x].x : 0u;
        for (int k = 0; k < w; ++k) run += s_seg[k][lane];
        if (on)
            for (uint32_t j = s0; j < s1; ++j) {
                const uint32_t h = H2[(size_t)j * tiles_x + x];
                H2[(size_t)j * tiles_x + x] = run;
                run += h;
            }
        __syncthreads();
    }
}

// Level 2, place: a warp walks each of its chunks again and puts each item's
// Gaussian id into its slot in every tile of the row that the Gaussian touches.
__global__ void __launch_bounds__(32 * kWalkWarps) k_cols_place(const u64* __restrict__ R1, uint32_t rows,
                                                                uint32_t tiles_x, const uint32_t* __restrict__ len,
                                                                const uint32_t* __restrict__ rowinfo,
                                                                const uint32_t* __restrict__ H2,
                                                                const uint2* __restrict__ ranges,
                                                                uint32_t* __restrict__ vals,
                                                                const uint32_t* __restrict__ info) {
    pdl_wait();
    extern __shared__ uint32_t s_walk[];
    const int lane = threadIdx.x & 31;
    if (info[kInfoAbort]) return;
    const uint32_t total = rowinfo[3 * rows];
    for (uint32_t j = blockIdx.x * kWalkWarps + (threadIdx.x >> 5); j < total; j += gridDim.x * kWalkWarps) {
        const RowChunk rc = l2_chunk(j, rows, rowinfo, len);
        const bool last = j + 1 == (rc.y + 1 < rows ? rowinfo[rows + rc.y + 1] : rowinfo[3 * rows]);
        // the first batch's items load while the placer reads the chunk's tile offsets
        const u64 none = 0xFFFFFFFFull | (1ull << 32);  // past the chunk: (1, 0), no tiles
        u64 it_next = rc.i0 + lane < rc.i1 ? R1[rc.i0 + lane] : none;
        Placer2 rs(s_walk + (size_t)(threadIdx.x >> 5) * Placer2::words(tiles_x), tiles_x);
        const uint32_t* h = H2 + (size_t)j * tiles_x;
        const uint2* rg = ranges + (size_t)rc.y * tiles_x;
        auto first = [&](uint32_t x) { return h[x]; };
        rs.init(lane, first, [&](uint32_t x) { return (last ? rg[x].y : h[x + tiles_x]) - h[x]; });
        for (uint32_t b = rc.i0; b < rc.i1; b += 32) {
            const u64 it = it_next;
            it_next = b + 32 + lane < rc.i1 ? R1[b + 32 + lane] : none;
            const uint32_t g = (uint32_t)it, sp = (uint32_t)(it >> 32);
            rs.batch(sp & 0xFFFFu, sp >> 16, [&](uint32_t) { return g; }, lane, vals);
        }
        rs.flush(vals, lane);
        __syncwarp();  // the next chunk's init rewrites what the flush reads
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

// Blocks of a grid-stride walk kernel: enough for `warps` chunks, at most as
// many as the GPU holds at once (cached per device, kernel and size).
static unsigned walk_blocks(const void* kernel, size_t smem, int64_t warps) {
    static std::mutex mu;
    struct Entry {
        int dev;
        const void* k;
        size_t smem;
        int64_t blocks;
    };
    static Entry cache[64];
    static int used = 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    int64_t resident = -1;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (int i = 0; i < used; ++i)
            if (cache[i].dev == dev && cache[i].k == kernel && cache[i].smem == smem) resident = cache[i].blocks;
        if (resident < 0) {
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * kWalkWarps, smem) != cudaSuccess) {
                cudaGetLastError();
                sms = 1;
                per_sm = 1;
            }
            resident = (int64_t)std::max(per_sm, 1) * sms;
            if (used < 64) cache[used++] = Entry{dev, kernel, smem, resident};
        }
    }
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(warps, kWalkWarps), resident));
}

// Lets the placing kernels use the route's largest shared-memory size
// (kWalkWarps placement states for kRowWalkMax buckets), once per device; never lowers it.
static cudaError_t walk_opt_in() {
    static std::mutex mu;
    static bool done[128] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    const int bytes1 = kWalkWarps * (int)Placer1::words(kRowWalkMax) * 4;
    const int bytes2 = kWalkWarps * (int)Placer2::words(kRowWalkMax) * 4;
    if ((e = cudaFuncSetAttribute(k_rows_place, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes1)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_cols_place, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes2)) != cudaSuccess)
        return e;
    done[dev] = true;
    return cudaSuccess;
}

// Level-1 chunks of a route-a frame (a multiple of kWalkWarps), or 0 for route b.
int64_t sort_walk_chunks(int64_t tiles_x, int64_t tiles_y) {
    if (tiles_x < 1 || tiles_y < 1 || tiles_x > kRowWalkMax || tiles_y > kRowWalkMax) return 0;
    const int64_t c = std::min<int64_t>(kL1ChunksMax, std::max<int64_t>(kL1ChunksMin, kH1Words / tiles_y));
    return c / kWalkWarps * kWalkWarps;
}

// Level-2 chunks a frame can need: a row's chunks hold at least kChunkTarget * len /
// entries items (or 32, which is more), so a row needs at most entries /
// kChunkTarget + 1 of them; twice that over all rows, for rounding.
static int64_t l2_chunks_max(int64_t capacity, int64_t tiles_y) {
    return 2 * (ceil_div(capacity, kChunkTarget) + tiles_y) + 16;
}

// The difference grid has (tiles_y + 1)(tiles_x + 1) = tiles + tiles_x + tiles_y + 1
// <= 2 tiles + 2 cells. Route a: vals takes 4 bytes per entry and the second
// buffer 8 (the 8-byte level-1 items, which never outnumber the entries, live
// there until the keys are exported into it as tile ids); route b's two 8-byte
// item buffers hold vals and tile_key.
size_t sort_scratch_bytes(int64_t n, int64_t capacity, int64_t tiles_x, int64_t tiles_y, int64_t chunks) {
    const int64_t tiles = tiles_x * tiles_y;
    const int64_t bn = ceil_div(n, kSortTile), bc = ceil_div(capacity, kSortTile), bs = ceil_div(n, kScanTile);
    const int tp = chunks > 0 ? 0 : tile_passes_for(tiles);
    const size_t entry = chunks > 0 ? 4 : 8;
    const int64_t rows = chunks > 0 ? tiles_y : 0;
    size_t b = 0;
    b += 2 * align256((size_t)n * 8);                                        // ditems_a, ditems_b
    b += align256((size_t)capacity * entry);                                 // items_a
    b += align256((size_t)capacity * 8);                                     // items_b
    b += align256(8 * kRadix * 4);                                           // hist
    b += align256(16 * 4);                                                   // counters
    b += align256((size_t)4 * bn * kRadix * 4);                              // status_depth
    b += align256((size_t)(tp > 0 ? tp : 1) * bc * kRadix * 4);              // status_tile
    b += align256((size_t)bs * 8);                                           // scan_status
    b += align256((size_t)(ceil_div(capacity, kDupTile) + 1) * 4);           // dup_start
    b += align256((size_t)(2 * tiles + 2 + tiles_y + 1) * 4);                // grid, row differences
    b += align256((size_t)chunks * rows * 4);                                // walk_h1 [rows][chunks]
    b += align256((size_t)rows * 4);                                         // walk_len
    b += align256((size_t)(3 * rows + 1) * 4);                               // walk_rows
    b += align256((size_t)(chunks > 0 ? l2_chunks_max(capacity, tiles_y) * tiles_x : 0) * 4);  // walk_h2
    b += align256((size_t)(chunks > 0 ? n : 0) * 8);                         // walk_rect
    return b;
}

SortScratch sort_scratch(const igs_frame& f) {
    SortScratch s;
    const int64_t n = f.n, cap = f.capacity, tiles = (int64_t)f.tiles_x * f.tiles_y;
    const int64_t bn = ceil_div(n, kSortTile), bc = ceil_div(cap, kSortTile), bs = ceil_div(n, kScanTile);
    const int64_t chunks = f.sort_chunks;
    const size_t entry = chunks > 0 ? 4 : 8;
    s.tile_bits = tile_bits_for(tiles);
    s.tile_passes = chunks > 0 ? 0 : tile_passes_for(tiles);
    s.walk_chunks = chunks;
    char* p = static_cast<char*>(f.scratch);
    auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
    s.ditems_a = (u64*)take((size_t)n * 8);
    s.ditems_b = (u64*)take((size_t)n * 8);
    s.seg_base = s.ditems_a;
    s.seg_bytes = 2 * align256((size_t)n * 8);
    s.items_a = (u64*)take((size_t)cap * entry);
    s.items_b = (u64*)take((size_t)cap * 8);
    s.hist = (uint32_t*)take(8 * kRadix * 4);
    s.counters = (uint32_t*)take(16 * 4);
    s.status_depth = (uint32_t*)take((size_t)4 * bn * kRadix * 4);
    s.status_tile = (uint32_t*)take((size_t)(s.tile_passes > 0 ? s.tile_passes : 1) * bc * kRadix * 4);
    s.scan_status = (unsigned long long*)take((size_t)bs * 8);
    s.dup_start = (uint32_t*)take((size_t)(ceil_div(cap, kDupTile) + 1) * 4);
    s.grid = (int32_t*)take((size_t)(2 * tiles + 2 + f.tiles_y + 1) * 4);
    const int64_t rows = chunks > 0 ? f.tiles_y : 0;
    s.walk_h1 = (uint32_t*)take((size_t)chunks * rows * 4);
    s.walk_len = (uint32_t*)take((size_t)rows * 4);
    s.walk_rows = (uint32_t*)take((size_t)(3 * rows + 1) * 4);
    s.walk_h2 = (uint32_t*)take((size_t)(chunks > 0 ? l2_chunks_max(cap, f.tiles_y) * f.tiles_x : 0) * 4);
    s.walk_rect = (uint2*)take((size_t)(chunks > 0 ? n : 0) * 8);
    // the last tile pass (p = passes - 1) reads items_a when p is even, items_b when odd
    const bool last_reads_a = s.tile_passes > 0 && (s.tile_passes - 1) % 2 == 0;
    s.vals = reinterpret_cast<uint32_t*>(last_reads_a ? s.items_b : s.items_a);
    s.tile_key = reinterpret_cast<uint32_t*>(last_reads_a ? s.items_a : s.items_b);
    if (s.tile_passes == 0) {  // route a, or one tile: the values are written directly
        s.vals = reinterpret_cast<uint32_t*>(s.items_a);
        s.tile_key = reinterpret_cast<uint32_t*>(s.items_b);
    }
    return s;
}

// Failure-detection tests: when set, the next binning's first depth pass runs
// with one silent block (igs_debug_silence_lookback_once).
std::atomic<int> g_silence_next{0};

cudaError_t launch_bin_sort(const igs_frame& f, int footprint, cudaStream_t st) {
    const SortScratch s = sort_scratch(f);
    const int64_t n = f.n, cap = f.capacity;
    const int64_t tiles = (int64_t)f.tiles_x * f.tiles_y;
    const int64_t bn = ceil_div(n, kSortTile), bc = ceil_div(cap, kSortTile), bs = ceil_div(n, kScanTile);
    const int tp = s.tile_passes;
    const int gx = f.tiles_x + 1, gy = f.tiles_y + 1;
    cudaError_t e;
#define CK(x) do { if ((e = (x)) != cudaSuccess) { g_failed_call = #x " (sort.cu:" IGS_STR(__LINE__) ")"; return e; } } while (0)
    // reset state: status words, histograms, counters, look-back words, difference grid (one launch)
    {
        ZeroRanges z = {};
        auto add = [&](void* p, size_t bytes) {
            z.ptr[z.count] = p;
            z.bytes[z.count++] = bytes;
        };
        add(f.info, kInfoWords * 4);
        add(s.hist, 8 * kRadix * 4);
        add(s.counters, 16 * 4);
        add(s.status_depth, (size_t)4 * bn * kRadix * 4);
        if (tp > 0) add(s.status_tile, (size_t)tp * bc * kRadix * 4);
        if (s.walk_chunks == 0) add(s.scan_status, (size_t)bs * 8);
        add(s.grid, (size_t)(gx * gy + (s.walk_chunks > 0 ? gy : 0)) * 4);  // grid (route a: and row differences)
        if (n == 0) add(f.ranges, (size_t)tiles * 8);
        CK(launch_zero(z, st));
    }
    if (n == 0) return cudaSuccess;
    const uint32_t nn = (uint32_t)n;
    const bool walk = s.walk_chunks > 0;
    int32_t* rowd = walk ? s.grid + (size_t)gx * gy : nullptr;  // row differences (route a)
    const uint32_t max2 = walk ? (uint32_t)l2_chunks_max(cap, f.tiles_y) : 0u;
    // 0. depth-digit histograms; footprint rows -> per-tile counts -> ranges, tile-digit histograms
    const int prep_blocks = (int)std::min<int64_t>(ceil_div(n, 256), 152 * 4);
    if ((int64_t)gx * gy <= kGridSmemCells)
        CK(launch_pdl(k_bin_prep<true>, dim3(prep_blocks), dim3(256), (size_t)(gx * gy + (walk ? gy : 0)) * 4, st,
            f.depth_key, reinterpret_cast<const uint2*>(f.rect), reinterpret_cast<const float4*>(f.disc), f.tile,
            footprint, f.count, nn, gx, gy, s.hist, s.grid, rowd, f.info));
    else
        CK(launch_pdl(k_bin_prep<false>, dim3(prep_blocks), dim3(256), 0, st, f.depth_key, reinterpret_cast<const uint2*>(f.rect),
                                                       reinterpret_cast<const float4*>(f.disc), f.tile, footprint,
                                                       f.count, nn, gx, gy, s.hist, s.grid, rowd, f.info));
    count_launches();
    CK(cudaGetLastError());
    if ((int64_t)gx * gy <= kGridSmemCells) {
        CK(launch_pdl(k_tiles_small, dim3(1), dim3(kTilesSmallThreads), (size_t)gx * gy * 4, st, s.grid, f.tiles_x, f.tiles_y, tp,
                      footprint == 0 ? 1 : 0,
                                                                           reinterpret_cast<uint2*>(f.ranges), s.hist,
                                                                           f.info, (uint64_t)cap, rowd, max2,
                                                                           s.walk_len, s.walk_rows));
        count_launches();
        CK(cudaGetLastError());
    } else {
        k_grid_rows<<<(unsigned)ceil_div(f.tiles_y, 128), 128, 0, st>>>(s.grid, gx, f.tiles_x, f.tiles_y);
        count_launches();
        CK(cudaGetLastError());
        k_tile_scan<<<1, kTileScanThreads, 0, st>>>(s.grid, gx, f.tiles_x, (uint32_t)tiles, tp,
                                                    reinterpret_cast<uint2*>(f.ranges), s.hist + 4 * kRadix, f.info,
                                                    (uint64_t)cap, s.grid, rowd, max2, s.walk_len, s.walk_rows);
        count_launches();
        CK(cudaGetLastError());
        k_hist_to_offsets<<<1, 1024, 0, st>>>(s.hist, 4 + tp);
        count_launches();
        CK(cudaGetLastError());
    }
    // 1. depth sort: (depth_key, index) -> A -> B -> A -> order (or -> order after the third pass)
    const bool small_grid = (int64_t)gx * gy <= kGridSmemCells;  // k_tiles_small decides the top-pass skip
    for (int p = 0; p < 4; ++p) {
        uint32_t* status = s.status_depth + (size_t)p * bn * kRadix;
        const uint32_t* hist = s.hist + p * kRadix;
        if (p == 0)
            CK(launch_pdl(k_radix_pass<true, false>, dim3((unsigned)bn), dim3(kSortThreads), 0, st, 
                f.depth_key, s.ditems_a, nullptr, nn, 0, hist, status, s.counters + 0, f.info,
                g_silence_next.exchange(0) ? 1u : 0xFFFFFFFFu, nullptr, nullptr));
        else if (p == 3 && small_grid)  // nothing to do when the top pass is skipped (k_tiles_small decides)
            CK(launch_pdl(k_radix_pass<false, true, true>, dim3((unsigned)bn), dim3(kSortThreads), 0, st, 
                s.ditems_a, f.order, nullptr, nn, 24, hist, status, s.counters + 3, f.info, 0xFFFFFFFFu,
                f.info + kInfoSkipTop, nullptr));
        else if (p == 3)
            CK(launch_pdl(k_radix_pass<false, true>, dim3((unsigned)bn), dim3(kSortThreads), 0, st, 
                s.ditems_a, f.order, nullptr, nn, 24, hist, status, s.counters + 3, f.info, 0xFFFFFFFFu,
                nullptr, nullptr));
        else if (p == 2 && small_grid)  // writes the order itself when the top pass is skipped
            CK(launch_pdl(k_radix_pass<false, false, true>, dim3((unsigned)bn), dim3(kSortThreads), 0, st, 
                s.ditems_b, s.ditems_a, nullptr, nn, 16, hist, status, s.counters + 2, f.info, 0xFFFFFFFFu,
                f.info + kInfoSkipTop, f.order));
        else
            CK(launch_pdl(k_radix_pass<false, false>, dim3((unsigned)bn), dim3(kSortThreads), 0, st, 
                p == 1 ? s.ditems_a : s.ditems_b, p == 1 ? s.ditems_b : s.ditems_a, nullptr, nn, 8 * p, hist,
                status, s.counters + p, f.info, 0xFFFFFFFFu, nullptr, nullptr));
        count_launches();
        CK(cudaGetLastError());
    }
    // kept count (k_bin_prep), M and the capacity check (tile-range kernel) are known here
    if (s.walk_chunks > 0) {
        // 3a. two-level counting sort: Gaussians into tile-row lists, then row items into tiles
        const uint32_t rows = (uint32_t)f.tiles_y, cols = (uint32_t)f.tiles_x;
        u64* R1 = s.items_b;  // level-1 lists: free until the keys are exported (as tile_key) into it
        const size_t count1 = (size_t)kWalkWarps * (rows + 1) * 4, count2 = (size_t)kWalkWarps * (cols + 1) * 4;
        const size_t place1 = (size_t)kWalkWarps * Placer1::words(rows) * 4;
        const size_t place2 = (size_t)kWalkWarps * Placer2::words(cols) * 4;
        if (std::max(place1, place2) > 48 * 1024) CK(walk_opt_in());
        const uint32_t cmax = (uint32_t)s.walk_chunks;

        const uint2* rect = reinterpret_cast<const uint2*>(f.rect);
        const uint2* rg = reinterpret_cast<const uint2*>(f.ranges);
        CK(launch_pdl(k_rows_count, dim3(walk_blocks((const void*)k_rows_count, count1, cmax)), dim3(32 * kWalkWarps), count1, st, f.order, rect, rows, cmax, s.walk_h1, s.walk_rect, f.info));
        count_launches();
        CK(cudaGetLastError());
        CK(launch_pdl(k_rows_scan, dim3(rows), dim3(kRowScanThreads), 0, st, s.walk_h1, cmax, s.walk_len, f.info));
        count_launches();
        CK(cudaGetLastError());
        const DiscRef disc{rect, reinterpret_cast<const float4*>(f.disc), f.tile, 1.0f / (float)f.tile, footprint};
        CK(launch_pdl(k_rows_place, dim3(walk_blocks((const void*)k_rows_place, place1, cmax)), dim3(32 * kWalkWarps), place1, st, f.order, s.walk_rect, disc, rows, cmax, s.walk_h1, s.walk_len,
                                                                s.walk_rows, R1, f.info));
        count_launches();
        CK(cudaGetLastError());
        CK(launch_pdl(k_cols_count, dim3(walk_blocks((const void*)k_cols_count, count2, max2)), dim3(32 * kWalkWarps), count2, st, (const u64*)R1, rows, cols, s.walk_len, s.walk_rows,
                                                                s.walk_h2, f.info));
        count_launches();
        CK(cudaGetLastError());
        CK(launch_pdl(k_cols_scan, dim3(rows, (unsigned)ceil_div(cols, 32)), dim3(32 * kColScanWarps), 0, st, s.walk_h2, rows, cols, rg, s.walk_rows, f.info));
        count_launches();
        CK(cudaGetLastError());
        CK(launch_pdl(k_cols_place, dim3(walk_blocks((const void*)k_cols_place, place2, max2)), dim3(32 * kWalkWarps), place2, st, (const u64*)R1, rows, cols, s.walk_len, s.walk_rows,
                                                                s.walk_h2, rg, f.vals, f.info));
        count_launches();
        CK(cudaGetLastError());
        return cudaSuccess;
    }
    // 2b. scan of tile counts in depth order (checked against the tile total), duplication block starts
    k_scan_offsets<<<(unsigned)bs, kScanThreads, 0, st>>>(f.order, f.count, nn, f.offset, s.dup_start,
                                                          s.scan_status, s.counters + 4, f.info, (uint64_t)cap, false);
    count_launches();
    CK(cudaGetLastError());
    // 3b. duplication, in depth order, by output position
    const unsigned dup_blocks = (unsigned)std::max<int64_t>(1, ceil_div(cap, kDupTile));
    k_duplicate<<<dup_blocks, 256, 0, st>>>(f.order, f.offset, s.dup_start, reinterpret_cast<const uint2*>(f.rect),
                                            reinterpret_cast<const float4*>(f.disc), f.tile, footprint, nn, f.tiles_x,
                                            s.items_a, tp == 0 ? f.vals : nullptr, f.info);
    count_launches();
    CK(cudaGetLastError());
    // 4b. stable tile-id sort of the M items (M read on the device; grid sized by capacity)
    for (int p = 0; p < tp; ++p) {
        const u64* in = (p % 2 == 0) ? s.items_a : s.items_b;
        uint32_t* status = s.status_tile + (size_t)p * bc * kRadix;
        const uint32_t* hist = s.hist + (4 + p) * kRadix;
        if (p == tp - 1)
            CK(launch_pdl(k_radix_pass<false, true>, dim3((unsigned)bc), dim3(kSortThreads), 0, st, 
                in, f.vals, f.info + kInfoM, 0u, 8 * p, hist, status, s.counters + 5 + p, f.info, 0xFFFFFFFFu,
                nullptr, nullptr));
        else
            CK(launch_pdl(k_radix_pass<false, false>, dim3((unsigned)bc), dim3(kSortThreads), 0, st, 
                in, (p % 2 == 0) ? s.items_b : s.items_a, f.info + kInfoM, 0u, 8 * p, hist, status,
                s.counters + 5 + p, f.info, 0xFFFFFFFFu, nullptr, nullptr));
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
// Some callers cannot allocate device memory around a call: an embedding host
// whose device memory all belongs to its own allocator (reserved at start-up,
// none left for cudaMalloc), or a latency-critical loop that must not call
// cudaMalloc/cudaFree, which can synchronise the whole device. This entry point
// orders n depth keys exactly as igs_bin_sort orders its frame's depth_key
// into order (stable, ties by index), but takes its scratch from one fixed
// device array compiled into the library.
// ---------------------------------------------------------------------------
namespace igs {
namespace {

constexpr int64_t kNoAllocMaxKeys = (int64_t)1 << 20;
constexpr int64_t kNoAllocBlocks = (kNoAllocMaxKeys + kSortTile - 1) / kSortTile;
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

// 17.6 MB (4405376 words), held by every device that loads the library until the process exits.
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

// The six launches of one call; the first failing CUDA call is named in g_failed_call.
cudaError_t launch_sort_depth_noalloc(const uint32_t* depth_key, uint32_t nn, uint32_t* order, cudaStream_t st) {
    cudaError_t e;
#define CK(x) do { if ((e = (x)) != cudaSuccess) { g_failed_call = #x " (sort.cu:" IGS_STR(__LINE__) ")"; return e; } } while (0)
    uint32_t* s = nullptr;
    CK(noalloc_scratch(&s));
    CK(cudaMemsetAsync(s + kNaZeroFrom, 0, (size_t)(kNaWords - kNaZeroFrom) * 4, st));
    const unsigned blocks = (unsigned)ceil_div(nn, kSortTile);
    const int hist_blocks = (int)std::min<int64_t>(ceil_div(nn, 256), 152 * 4);
    k_hist<<<hist_blocks, 256, 0, st>>>(depth_key, nn, 4, s + kNaHist);
    count_launches();
    CK(cudaGetLastError());
    k_hist_to_offsets<<<1, 1024, 0, st>>>(s + kNaHist, 4);
    count_launches();
    CK(cudaGetLastError());
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
        CK(cudaGetLastError());
    }
#undef CK
    return cudaSuccess;
}

}  // namespace
}  // namespace igs

extern "C" igs_status igs_sort_depth_noalloc(const uint32_t* depth_key, int64_t n, uint32_t* order, void* stream) {
    using namespace igs;
    if (n < 0 || n > kNoAllocMaxKeys)
        return report_invalid("igs_sort_depth_noalloc: n must be in [0, 2^20] (the size of its fixed scratch)");
    if (n > 0 && (!depth_key || !order)) return report_invalid("igs_sort_depth_noalloc: depth_key or order is NULL");
    if (n == 0) return IGS_OK;
    return report_cuda(launch_sort_depth_noalloc(depth_key, (uint32_t)n, order, (cudaStream_t)stream),
                       "igs_sort_depth_noalloc");
}
