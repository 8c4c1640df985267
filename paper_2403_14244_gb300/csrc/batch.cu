// Multi-view batch rendering: V views of one scene, each with its own pose and
// image size, rendered by one chain of launches with no host synchronisation
// (so the chain can be captured in a CUDA graph and replayed):
//   project all (view, Gaussian) pairs            one launch, grid (blocks, V)
//   depth-digit histograms, footprint rows        one launch per step, per view in grid.y
//   per-view tile counts -> global tile ranges
//   per-view depth sorts                          4 segmented radix passes
//   scan of tile counts over all views            one launch (view-major entry order)
//   duplication with global tile ids              one launch
//   tile-id sort over all entries                 ceil(bits(total tiles) / 8) passes
//   persistent blend                              one launch: CTAs pull (view, tile)
//                                                 work items from an atomic counter
// A view's pixels are bit-identical to rendering it alone (same projection,
// same order, same per-tile compositing routine).
#include <algorithm>
#include <cstring>

#include "binning.cuh"
#include "blendtile.cuh"
#include "projection.cuh"

namespace igs {

namespace {

constexpr int kBatchGridSmemCells = 24576;  // 96 KB of corner grid in shared memory
constexpr int kPrepThreads = 256;

struct BatchScratch {
    BatchView* views;        // [V]
    int32_t* tiles_x;        // [V]
    uint32_t* tile_base;     // [V]
    uint32_t* view_total;    // [V] entries per view
    uint32_t* entry_base;    // [V] first entry of each view
    unsigned long long* ditems_a;  // [V n]
    unsigned long long* ditems_b;  // [V n]
    unsigned long long* items_a;   // [capacity]
    unsigned long long* items_b;   // [capacity]
    uint32_t* hist_depth;    // [4][V][256]
    uint32_t* hist_tile;     // [4][256]
    uint32_t* counters;      // [4 V + 16]
    uint32_t* status_depth;  // [4][V][blocks(n)][256]
    uint32_t* status_tile;   // [tile passes][blocks(capacity)][256]
    unsigned long long* scan_status;  // [blocks(V n)]
    uint32_t* dup_start;     // [blocks(capacity) + 1]
    int32_t* grid;           // corner grids of all views
    uint32_t* work;          // [1] persistent-blend work counter
    int tile_passes;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct Sizes {
    int64_t n, V, cap, tiles, cells, bn, bc, bs;
    int tp;
};

Sizes sizes_of(const igs_batch& b, int64_t cells) {
    Sizes z;
    z.n = b.n;
    z.V = b.views;
    z.cap = b.capacity;
    z.tiles = b.tiles_total;
    z.cells = cells;
    z.bn = ceil_div(b.n, kSortTile);
    z.bc = ceil_div(b.capacity, kSortTile);
    z.bs = ceil_div(b.n * b.views, kScanTile);
    z.tp = tile_passes_for(b.tiles_total);
    return z;
}

// Carve the batch scratch; with base == nullptr only the size is computed.
size_t carve(const Sizes& z, char* base, BatchScratch* s) {
    size_t off = 0;
    auto take = [&](size_t bytes) { char* q = base ? base + off : nullptr; off += al(bytes); return q; };
    const int64_t Vn = z.V * z.n;
    BatchScratch t;
    t.views = (BatchView*)take(sizeof(BatchView) * z.V);
    t.tiles_x = (int32_t*)take(4 * z.V);
    t.tile_base = (uint32_t*)take(4 * z.V);
    t.view_total = (uint32_t*)take(4 * z.V);
    t.entry_base = (uint32_t*)take(4 * z.V);
    t.ditems_a = (unsigned long long*)take(8 * (size_t)Vn);
    t.ditems_b = (unsigned long long*)take(8 * (size_t)Vn);
    t.items_a = (unsigned long long*)take(8 * (size_t)z.cap);
    t.items_b = (unsigned long long*)take(8 * (size_t)z.cap);
    t.hist_depth = (uint32_t*)take(4 * 4 * z.V * kRadix);
    t.hist_tile = (uint32_t*)take(4 * 4 * kRadix);
    t.counters = (uint32_t*)take(4 * (4 * z.V + 16));
    t.status_depth = (uint32_t*)take(4 * (size_t)4 * z.V * z.bn * kRadix);
    t.status_tile = (uint32_t*)take(4 * (size_t)(z.tp > 0 ? z.tp : 1) * z.bc * kRadix);
    t.scan_status = (unsigned long long*)take(8 * (size_t)z.bs);
    t.dup_start = (uint32_t*)take(4 * (size_t)(ceil_div(z.cap, kDupTile) + 1));
    t.grid = (int32_t*)take(4 * (size_t)z.cells);
    t.work = (uint32_t*)take(4 * 16);
    t.tile_passes = z.tp;
    if (s) *s = t;
    return off;
}

template <int DEG>
__global__ void __launch_bounds__(256) k_project_batch(const float4* __restrict__ ms, const float* __restrict__ op,
                                                       const float* __restrict__ col, int64_t n,
                                                       const BatchView* __restrict__ views,
                                                       float4* __restrict__ rec, uint2* __restrict__ rect,
                                                       float4* __restrict__ disc, uint32_t* __restrict__ count,
                                                       uint32_t* __restrict__ depth_key) {
    __shared__ ViewParams s_vp;
    const int v = blockIdx.y;
    if (threadIdx.x == 0) s_vp = views[v].vp;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t r = (int64_t)v * n + i;
    project_one<DEG>(ms, op, col, i, s_vp, rec + 2 * r, rect + r, disc + r, count + r, depth_key + r);
}

// Per view (grid.y): depth-digit histograms, and for each record, in each tile
// row it touches, +1 at its first tile and -1 past its last (difference grid).
template <bool SMEM_GRID>
__global__ void __launch_bounds__(kPrepThreads) k_bin_prep_batch(const uint32_t* __restrict__ depth_key,
                                                                 const uint2* __restrict__ rect,
                                                                 const float4* __restrict__ disc,
                                                                 const uint32_t* __restrict__ count, uint32_t n,
                                                                 int V, const BatchView* __restrict__ views,
                                                                 uint32_t* __restrict__ hist_depth,
                                                                 int32_t* __restrict__ grid) {
    extern __shared__ int32_t s_grid[];
    __shared__ uint32_t s_h[4][kRadix];
    const int v = blockIdx.y;
    const int gx = views[v].vp.tiles_x + 1, gy = views[v].vp.tiles_y + 1;
    const int cells = gx * gy;
    int32_t* vg = grid + views[v].grid_off;
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = 0;
    if (SMEM_GRID)
        for (int k = threadIdx.x; k < cells; k += blockDim.x) s_grid[k] = 0;
    __syncthreads();
    int32_t* g = SMEM_GRID ? s_grid : vg;
    const size_t r0 = (size_t)v * n;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = depth_key[r0 + i];
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&s_h[p][(k >> (8 * p)) & 0xFF], 1u);
        if (count[r0 + i]) {
            const uint2 r = rect[r0 + i];
            const int tile = views[v].vp.tile, fp = views[v].vp.footprint;
            const float inv = 1.0f / (float)tile;
            const int y0 = r.x >> 16, y1 = r.y >> 16;
            for (int ty = y0; ty <= y1; ++ty) {  // +1 at the row's first touched tile, -1 past its last
                const int2 sp = tile_span(fp, r, disc, r0 + i, tile, inv, ty);
                if (sp.y < sp.x) continue;
                atomicAdd(&g[ty * gx + sp.x], 1);
                atomicAdd(&g[ty * gx + sp.y + 1], -1);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) {
        const uint32_t c = (&s_h[0][0])[k];
        const int p = k >> 8, d = k & 255;
        if (c) atomicAdd(&hist_depth[((size_t)p * V + v) * kRadix + d], c);
    }
    if (SMEM_GRID)
        for (int k = threadIdx.x; k < cells; k += blockDim.x)
            if (s_grid[k]) atomicAdd(&vg[k], s_grid[k]);
}

// Prefix of each view's difference grid along its rows: per-tile entry counts.
__global__ void k_grid_rows_batch(int32_t* __restrict__ grid, const BatchView* __restrict__ views) {
    const int v = blockIdx.y;
    const int tx = views[v].vp.tiles_x, ty = views[v].vp.tiles_y, gx = tx + 1;
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= ty) return;
    int32_t* row = grid + views[v].grid_off + (size_t)y * gx;
    int32_t run = 0;
    for (int x = 0; x < tx; ++x) {
        run += row[x];
        row[x] = run;
    }
}

// One block per view: view-local tile ranges into the global range table, the
// view's entry total, and the digit histogram of the global tile ids.
constexpr int kTsThreads = 1024;
__global__ void __launch_bounds__(kTsThreads) k_tile_scan_batch(const int32_t* __restrict__ grid,
                                                                const BatchView* __restrict__ views, int passes,
                                                                uint2* __restrict__ ranges,
                                                                uint32_t* __restrict__ hist_tile,
                                                                uint32_t* __restrict__ view_total) {
    __shared__ uint32_t s_h[4][kRadix];
    __shared__ uint32_t s_warp[kTsThreads / 32];
    const int v = blockIdx.x;
    const int tiles_x = views[v].vp.tiles_x, gx = tiles_x + 1;
    const uint32_t tiles = (uint32_t)tiles_x * (uint32_t)views[v].vp.tiles_y;
    const uint32_t base = views[v].tile_base;
    const int32_t* g = grid + views[v].grid_off;
    for (int k = threadIdx.x; k < 4 * kRadix; k += blockDim.x) (&s_h[0][0])[k] = 0;
    const uint32_t per = (tiles + kTsThreads - 1) / kTsThreads;
    const uint32_t t0 = min(tiles, threadIdx.x * per), t1 = min(tiles, t0 + per);
    uint32_t sum = 0;
    for (uint32_t t = t0; t < t1; ++t) sum += (uint32_t)g[(size_t)(t / tiles_x) * gx + (t % tiles_x)];
    __syncthreads();
    uint32_t start = block_excl_scan<kTsThreads>(sum, s_warp);
    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t c = (uint32_t)g[(size_t)(t / tiles_x) * gx + (t % tiles_x)];
        ranges[base + t] = c ? make_uint2(start, start + c) : make_uint2(0u, 0u);
        start += c;
        if (c)
            for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][((base + t) >> (8 * p)) & 0xFF], c);
    }
    if (t1 == tiles && t0 < t1) view_total[v] = start;
    if (tiles == 0 && threadIdx.x == 0) view_total[v] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < passes * kRadix; k += blockDim.x) {
        const uint32_t c = (&s_h[0][0])[k];
        if (c) atomicAdd(&hist_tile[k], c);
    }
}

// One thread: first entry of every view (exclusive scan of the view totals) and
// the total, for the scan's consistency check.
__global__ void k_view_bases(const uint32_t* __restrict__ view_total, int V, uint32_t* __restrict__ entry_base,
                             uint32_t* __restrict__ info) {
    uint64_t run = 0;
    for (int v = 0; v < V; ++v) {
        entry_base[v] = (uint32_t)run;
        run += view_total[v];
    }
    info[kInfoTileTotal] = (uint32_t)min(run, (uint64_t)0xFFFFFFFFu);
}

// Shift every non-empty range of view v by the view's first entry.
__global__ void k_ranges_rebase(uint2* __restrict__ ranges, const BatchView* __restrict__ views,
                                const uint32_t* __restrict__ entry_base) {
    const int v = blockIdx.y;
    const uint32_t tiles = (uint32_t)views[v].vp.tiles_x * (uint32_t)views[v].vp.tiles_y;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles) return;
    uint2* r = ranges + views[v].tile_base + t;
    const uint2 x = *r;
    if (x.y > x.x) *r = make_uint2(x.x + entry_base[v], x.y + entry_base[v]);
}

// Persistent blend: every CTA takes (view, tile) work items from one counter
// until none is left. Work item w is global tile w; its view is found by binary
// search of the views' first tiles.
template <int TS, int B>
__global__ void __launch_bounds__(TS* TS) k_blend_persistent(const uint2* __restrict__ ranges,
                                                             const uint32_t* __restrict__ vals,
                                                             const float4* __restrict__ rec,
                                                             const BatchView* __restrict__ views, int V,
                                                             uint32_t tiles_total, BlendParams P,
                                                             float* __restrict__ images, uint32_t* __restrict__ work,
                                                             const uint32_t* __restrict__ info) {
    __shared__ float4 s_a[B];
    __shared__ float4 s_c[B];
    __shared__ uint32_t s_base[IGS_MAX_VIEWS + 1];
    __shared__ uint32_t s_item;
    if (info[kInfoAbort]) return;
    for (int k = threadIdx.x; k < V; k += blockDim.x) s_base[k] = views[k].tile_base;
    if (threadIdx.x == 0) s_base[V] = tiles_total;
    for (;;) {
        __syncthreads();  // s_item / s_a / s_c are free again
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t w = s_item;
        if (w >= tiles_total) break;
        int lo = 0, hi = V;  // view: largest v with s_base[v] <= w
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_base[mid] <= w) lo = mid; else hi = mid;
        }
        const ViewParams& vp = views[lo].vp;
        const uint32_t t = w - s_base[lo];
        blend_tile_fwd<TS, B>((int)(t % (uint32_t)vp.tiles_x), (int)(t / (uint32_t)vp.tiles_x), vp.width, vp.height,
                              ranges[w], vals, rec, P.alpha_min, P.alpha_max, P.t_min, P.bg, s_a, s_c,
                              images + views[lo].img_off, nullptr, nullptr);
    }
}

// Sub-tile blend: one 64-thread CTA per 8 x 8 pixel block of every view's
// binning tiles (item w: tile w / (TS/8)^2, block w % (TS/8)^2), walking the
// tile's entries; each block stops on its own. The hardware block scheduler
// balances the mixed view sizes, so the launch is not persistent.
template <int TS>
__global__ void __launch_bounds__(64) k_blend_batch_sub(const uint2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ vals,
                                                        const float4* __restrict__ rec,
                                                        const BatchView* __restrict__ views, int V,
                                                        uint32_t tiles_total, BlendParams P,
                                                        float* __restrict__ images, uint32_t* __restrict__ work,
                                                        const uint32_t* __restrict__ info) {
    constexpr int SUB = TS / 8, NS = SUB * SUB;
    __shared__ float4 s_a[64];
    __shared__ float4 s_c[64];
    if (info[kInfoAbort]) return;
    const uint32_t w = blockIdx.x / NS, q = blockIdx.x % NS;
    int lo = 0, hi = V;  // view: largest v with tile_base[v] <= w
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (views[mid].tile_base <= w) lo = mid; else hi = mid;
    }
    const ViewParams& vp = views[lo].vp;
    const uint32_t t = w - views[lo].tile_base;
    const int tx = (int)(t % (uint32_t)vp.tiles_x), ty = (int)(t / (uint32_t)vp.tiles_x);
    blend_tile_fwd<8, 64>(tx * SUB + (int)(q % SUB), ty * SUB + (int)(q / SUB), vp.width, vp.height, ranges[w], vals,
                          rec, P.alpha_min, P.alpha_max, P.t_min, P.bg, s_a, s_c, images + views[lo].img_off, nullptr,
                          nullptr);
}

template <int TS, int B>
void* persistent_kernel() {
    return reinterpret_cast<void*>(k_blend_persistent<TS, B>);
}

// The blend variants the batch path (and its autotuner) can pick: a staging
// depth of 64 with 16- or 32-pixel tiles selects the sub-tile blend (`sub`:
// one CTA of 64 threads per 8 x 8 block), the others the persistent whole-tile
// blend.
bool blend_variant(int tile, int batch, void** fn, bool* sub = nullptr) {
    bool sb = false;
    switch (tile * 10000 + batch) {
        case 8 * 10000 + 32: *fn = persistent_kernel<8, 32>(); break;
        case 8 * 10000 + 64: *fn = persistent_kernel<8, 64>(); break;
        case 16 * 10000 + 64: *fn = reinterpret_cast<void*>(k_blend_batch_sub<16>); sb = true; break;
        case 16 * 10000 + 128: *fn = persistent_kernel<16, 128>(); break;
        case 16 * 10000 + 256: *fn = persistent_kernel<16, 256>(); break;
        case 32 * 10000 + 64: *fn = reinterpret_cast<void*>(k_blend_batch_sub<32>); sb = true; break;
        case 32 * 10000 + 256: *fn = persistent_kernel<32, 256>(); break;
        case 32 * 10000 + 512: *fn = persistent_kernel<32, 512>(); break;
        case 32 * 10000 + 1024: *fn = persistent_kernel<32, 1024>(); break;
        default: return false;
    }
    if (sub) *sub = sb;
    return true;
}

}  // namespace

int batch_persistent_blocks(int tile, int batch) {
    void* fn = nullptr;
    bool sub = false;
    if (!blend_variant(tile, batch, &fn, &sub)) return 0;
    if (sub) return 1;  // not persistent: one CTA per 8 x 8 block
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, tile * tile, 0) != cudaSuccess) return 0;
    return sms * std::max(per_sm, 1);
}

int64_t batch_grid_cells(const igs_batch& b) {
    int64_t cells = 0;
    for (int v = 0; v < b.views; ++v) {
        const int64_t tx = (b.width[v] + b.tile - 1) / b.tile, ty = (b.height[v] + b.tile - 1) / b.tile;
        cells += (tx + 1) * (ty + 1);
    }
    return cells;
}

int64_t batch_max_cells(const igs_batch& b) {
    int64_t m = 0;
    for (int v = 0; v < b.views; ++v) {
        const int64_t tx = (b.width[v] + b.tile - 1) / b.tile, ty = (b.height[v] + b.tile - 1) / b.tile;
        m = std::max(m, (tx + 1) * (ty + 1));
    }
    return m;
}

size_t batch_scratch_bytes(const igs_batch& b) { return carve(sizes_of(b, batch_grid_cells(b)), nullptr, nullptr); }

const uint32_t* batch_view_totals(const igs_batch& b) {
    BatchScratch s;
    carve(sizes_of(b, batch_grid_cells(b)), static_cast<char*>(b.scratch), &s);
    return s.view_total;
}

bool batch_blend_variant_ok(int tile, int batch) {
    void* fn;
    return blend_variant(tile, batch, &fn);
}

cudaError_t batch_set_views(const igs_batch& b, const BatchView* host_views, cudaStream_t st) {
    BatchScratch s;
    carve(sizes_of(b, batch_grid_cells(b)), static_cast<char*>(b.scratch), &s);
    int32_t tx[IGS_MAX_VIEWS];
    uint32_t tb[IGS_MAX_VIEWS];
    for (int v = 0; v < b.views; ++v) {
        tx[v] = host_views[v].vp.tiles_x;
        tb[v] = host_views[v].tile_base;
    }
    cudaError_t e = cudaMemcpyAsync(s.views, host_views, sizeof(BatchView) * b.views, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.tiles_x, tx, 4 * b.views, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.tile_base, tb, 4 * b.views, cudaMemcpyHostToDevice, st);
    return e;
}

cudaError_t batch_prepare_kernels(const igs_batch& b) {
    // opt-in shared memory sizes, set once outside any stream capture
    const int64_t mc = batch_max_cells(b);
    if (mc <= kBatchGridSmemCells) {
        cudaError_t e = cudaFuncSetAttribute(k_bin_prep_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kBatchGridSmemCells * 4));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_render_batch(const igs_batch& b, const igs_scene& sc, const BlendParams& bp, int sh_degree,
                                float* images, cudaStream_t st, int opts_footprint) {
    BatchScratch s;
    const int64_t cells = batch_grid_cells(b);
    const Sizes z = sizes_of(b, cells);
    carve(z, static_cast<char*>(b.scratch), &s);
    const int V = b.views;
    const int64_t n = b.n, cap = b.capacity;
    const uint32_t Vn = (uint32_t)(n * V);
    const int tp = s.tile_passes;
    cudaError_t e;
#define CK(x) do { if ((e = (x)) != cudaSuccess) { g_failed_call = #x " (batch.cu:" IGS_STR(__LINE__) ")"; return e; } } while (0)
    CK(cudaMemsetAsync(b.info, 0, kInfoWords * 4, st));
    CK(cudaMemsetAsync(s.hist_depth, 0, 4 * 4 * (size_t)V * kRadix, st));
    CK(cudaMemsetAsync(s.hist_tile, 0, 4 * 4 * kRadix, st));
    CK(cudaMemsetAsync(s.counters, 0, 4 * (4 * (size_t)V + 16), st));
    CK(cudaMemsetAsync(s.status_depth, 0, 4 * (size_t)4 * V * z.bn * kRadix, st));
    if (tp > 0) CK(cudaMemsetAsync(s.status_tile, 0, 4 * (size_t)tp * z.bc * kRadix, st));
    CK(cudaMemsetAsync(s.scan_status, 0, 8 * (size_t)z.bs, st));
    CK(cudaMemsetAsync(s.grid, 0, 4 * (size_t)cells, st));
    CK(cudaMemsetAsync(s.work, 0, 64, st));
    if (n == 0 || V == 0) return cudaSuccess;
    // 1. projection of every (view, Gaussian)
    {
        const dim3 grid((unsigned)ceil_div(n, 256), (unsigned)V);
        auto ms = reinterpret_cast<const float4*>(sc.means_sigma);
        auto rec = reinterpret_cast<float4*>(b.rec);
        auto rect = reinterpret_cast<uint2*>(b.rect);
#define IGS_PB(D) k_project_batch<D><<<grid, 256, 0, st>>>(ms, sc.opacity, sc.color, n, s.views, rec, rect, reinterpret_cast<float4*>(b.disc), b.count, b.depth_key)
        switch (sh_degree) {
            case -1: IGS_PB(-1); break;
            case 0: IGS_PB(0); break;
            case 1: IGS_PB(1); break;
            case 2: IGS_PB(2); break;
            case 3: IGS_PB(3); break;
            default: return cudaErrorInvalidValue;
        }
#undef IGS_PB
        count_launches();
        CK(cudaGetLastError());
    }
    // 2. histograms, corner grids, per-view tile counts -> global tile ranges
    {
        const int64_t mc = batch_max_cells(b);
        const dim3 grid((unsigned)std::min<int64_t>(ceil_div(n, kPrepThreads), 64), (unsigned)V);
        if (mc <= kBatchGridSmemCells)
            k_bin_prep_batch<true><<<grid, kPrepThreads, (size_t)mc * 4, st>>>(
                b.depth_key, reinterpret_cast<const uint2*>(b.rect), reinterpret_cast<const float4*>(b.disc),
                b.count, (uint32_t)n, V, s.views, s.hist_depth, s.grid);
        else
            k_bin_prep_batch<false><<<grid, kPrepThreads, 0, st>>>(
                b.depth_key, reinterpret_cast<const uint2*>(b.rect), reinterpret_cast<const float4*>(b.disc),
                b.count, (uint32_t)n, V, s.views, s.hist_depth, s.grid);
        count_launches();
        CK(cudaGetLastError());
        int max_tx = 1, max_ty = 1;
        for (int v = 0; v < V; ++v) {
            max_tx = std::max(max_tx, (b.width[v] + b.tile - 1) / b.tile);
            max_ty = std::max(max_ty, (b.height[v] + b.tile - 1) / b.tile);
        }
        k_grid_rows_batch<<<dim3((unsigned)ceil_div(max_ty, 128), V), 128, 0, st>>>(s.grid, s.views);
        count_launches();
        k_tile_scan_batch<<<V, kTsThreads, 0, st>>>(s.grid, s.views, tp, reinterpret_cast<uint2*>(b.ranges),
                                                     s.hist_tile, s.view_total);
        count_launches();
        k_view_bases<<<1, 1, 0, st>>>(s.view_total, V, s.entry_base, b.info);
        count_launches();
        k_ranges_rebase<<<dim3((unsigned)ceil_div((int64_t)max_tx * max_ty, 256), V), 256, 0, st>>>(
            reinterpret_cast<uint2*>(b.ranges), s.views, s.entry_base);
        count_launches();
        const int rows = 4 * V;  // depth histograms [4][V] rows
        k_hist_to_offsets<<<(unsigned)ceil_div(rows, 8), 1024, 0, st>>>(s.hist_depth, rows);
        count_launches();
        if (tp > 0) {
            k_hist_to_offsets<<<1, 1024, 0, st>>>(s.hist_tile, tp);
            count_launches();
        }
        CK(cudaGetLastError());
    }
    // 3. per-view depth sorts: segment v = records [v n, (v + 1) n)
    for (int p = 0; p < 4; ++p) {
        const dim3 grid((unsigned)z.bn, (unsigned)V);
        uint32_t* status = s.status_depth + (size_t)p * V * z.bn * kRadix;
        const uint32_t* base = s.hist_depth + (size_t)p * V * kRadix;
        uint32_t* cnt = s.counters + p * V;
        if (p == 0)
            k_radix_pass<true, false><<<grid, kSortThreads, 0, st>>>(b.depth_key, s.ditems_a, nullptr, (uint32_t)n,
                                                                     0, base, status, cnt, b.info);
        else if (p == 3)
            k_radix_pass<false, true><<<grid, kSortThreads, 0, st>>>(s.ditems_a, b.order, nullptr, (uint32_t)n, 24,
                                                                     base, status, cnt, b.info);
        else
            k_radix_pass<false, false><<<grid, kSortThreads, 0, st>>>(
                p == 1 ? s.ditems_a : s.ditems_b, p == 1 ? s.ditems_b : s.ditems_a, nullptr, (uint32_t)n, 8 * p, base,
                status, cnt, b.info);
        count_launches();
        CK(cudaGetLastError());
    }
    // 4. scan over all views, 5. duplication with global tile ids
    k_scan_offsets<<<(unsigned)z.bs, kScanThreads, 0, st>>>(b.order, b.count, Vn, b.offset, s.dup_start,
                                                            s.scan_status, s.counters + 4 * V, b.info, (uint64_t)cap, true);
    count_launches();
    CK(cudaGetLastError());
    const unsigned dup_blocks = (unsigned)std::max<int64_t>(1, ceil_div(cap, kDupTile));
    k_duplicate<true><<<dup_blocks, 256, 0, st>>>(b.order, b.offset, s.dup_start, reinterpret_cast<const uint2*>(b.rect),
                                                  reinterpret_cast<const float4*>(b.disc), b.tile, opts_footprint, Vn, 0,
                                                  s.items_a, tp == 0 ? b.vals : nullptr, b.info, (uint32_t)n,
                                                  s.tiles_x, s.tile_base);
    count_launches();
    CK(cudaGetLastError());
    // 6. tile-id sort of all entries
    for (int p = 0; p < tp; ++p) {
        const unsigned long long* in = (p % 2 == 0) ? s.items_a : s.items_b;
        uint32_t* status = s.status_tile + (size_t)p * z.bc * kRadix;
        const uint32_t* base = s.hist_tile + p * kRadix;
        if (p == tp - 1)
            k_radix_pass<false, true><<<(unsigned)z.bc, kSortThreads, 0, st>>>(
                in, b.vals, b.info + kInfoM, 0u, 8 * p, base, status, s.counters + 4 * V + 1 + p, b.info);
        else
            k_radix_pass<false, false><<<(unsigned)z.bc, kSortThreads, 0, st>>>(
                in, (p % 2 == 0) ? s.items_b : s.items_a, b.info + kInfoM, 0u, 8 * p, base, status,
                s.counters + 4 * V + 1 + p, b.info);
        count_launches();
        CK(cudaGetLastError());
    }
    // 7. persistent blend over every (view, tile)
    void* fn = nullptr;
    bool sub = false;
    if (!blend_variant(b.tile, b.blend_batch, &fn, &sub)) return cudaErrorInvalidValue;
    const int64_t per_tile = sub ? (int64_t)(b.tile / 8) * (b.tile / 8) : 1;
    const unsigned nblocks = (unsigned)(sub ? std::max<int64_t>(1, b.tiles_total * per_tile)
                                            : std::max<int64_t>(1, std::min<int64_t>(b.persistent_blocks, b.tiles_total)));
    const float4* recp = reinterpret_cast<const float4*>(b.rec);
    const uint2* rg = reinterpret_cast<const uint2*>(b.ranges);
    uint32_t tt = (uint32_t)b.tiles_total;
    BlendParams bpp = bp;
    void* args[] = {(void*)&rg, (void*)&b.vals, (void*)&recp, (void*)&s.views, (void*)&V, (void*)&tt, (void*)&bpp,
                    (void*)&images, (void*)&s.work, (void*)&b.info};
    CK(cudaLaunchKernel(fn, dim3(nblocks), dim3(sub ? 64 : b.tile * b.tile), args, 0, st));
    count_launches();
#undef CK
    return cudaSuccess;
}

}  // namespace igs
