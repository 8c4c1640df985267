// Internal declarations shared by the CUDA translation units of libigs.
// Nothing here is part of the C ABI (include/igs.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>

#include "igs.h"

namespace igs {

// Footprint radius in units of the screen-space scale s: o exp(-K^2/2) < 1/255
// for every o <= 1 (compact support of the particle, Eq. 2).
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
// Slack added to the record's exponent bound pmax = log2(o / alpha_min): it
// covers the rounding of that logarithm and the relative error of ex2.approx
// (both below 2^-19), so w2 d^2 > pmax proves alpha < alpha_min.
constexpr float kPowMargin = 1.0f / 1024.0f;

// Status words of a frame (igs_frame::info). kInfoKeyWrap: some depth key other
// than the culled 0xFFFFFFFF has its low 24 bits all ones or its top byte 0xFF;
// kInfoSkipTop: the depth sort's top-byte pass is redundant and skipped (below).
enum : int { kInfoM = 0, kInfoKept = 1, kInfoErr = 2, kInfoNeed = 3, kInfoAbort = 4, kInfoTileTotal = 5,
             kInfoKeyWrap = 6, kInfoSkipTop = 7, kInfoWords = 16 };

// Radix sort geometry: 256 threads x 20 (key | value) items per block, 8-bit digits
// (5120 items: a 3M-key pass fits one wave of four blocks per SM).
constexpr int kSortThreads = 256;
constexpr int kSortIpt = 20;
constexpr int kSortTile = kSortThreads * kSortIpt;
constexpr int kRadix = 256;
constexpr int kScanThreads = 256;
constexpr int kScanIpt = 16;
constexpr int kScanTile = kScanThreads * kScanIpt;
// Entries written per block by the duplication kernel.
constexpr int kDupTile = 2048;
// Upper bound on polls of a look-back flag before a block gives up (about 0.1 s).
constexpr int kMaxSpin = 1 << 21;

// Set by igs_debug_silence_lookback_once, consumed by the next launch_bin_sort.
extern std::atomic<int> g_silence_next;
// Kernel launches made by the library (igs_launch_count).
extern std::atomic<uint64_t> g_launches;
inline void count_launches(uint64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }
// The CUDA call of a multi-launch step that failed last on this thread (for the error message).
extern thread_local const char* g_failed_call;
// Status of a finished call for the C ABI: IGS_OK, or IGS_ERR_CUDA / IGS_ERR_INVALID_ARG
// with the message igs_last_error() returns (naming g_failed_call, if set).
igs_status report_cuda(cudaError_t e, const char* what);
igs_status report_invalid(const char* msg);
#define IGS_STR2(x) #x
#define IGS_STR(x) IGS_STR2(x)

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Programmatic dependent launch: a kernel launched with launch_pdl is set up
// while its stream predecessor (a kernel) still runs, and calls pdl_wait()
// before it touches memory, which returns once the predecessor has finished and
// its writes are visible. Without the launch attribute pdl_wait() is a no-op.
// (Kernels do not trigger their successors early: resident waiting CTAs then
// slowed the predecessors' last waves, measured.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Zero up to kZeroRanges byte ranges in one launch (16-byte aligned starts and
// sizes multiple of 4), so that a chain of kernels is not split by memset nodes.
constexpr int kZeroRanges = 8;
struct ZeroRanges {
    void* ptr[kZeroRanges];
    unsigned long long bytes[kZeroRanges];
    int count;
};
cudaError_t launch_zero(const ZeroRanges& z, cudaStream_t s);

// Record the first device error of a frame and tell every later step to skip
// its work (outputs are left untouched).
__device__ __forceinline__ void record_error(uint32_t* info, uint32_t code) {
    atomicCAS(&info[kInfoErr], 0u, code);
    atomicExch(&info[kInfoAbort], 1u);
}

// Look-back status words carry their own flag and count in one word, and a
// reader uses nothing else its predecessor wrote, so relaxed GPU-scope accesses
// suffice (an acquire load would also hold back every later load until it
// completes, serialising a window of polls).
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// 2^x with the SFU (ex2.approx, flush-to-zero): alpha only needs ~22 bits.
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Everything a projection kernel needs about the view (passed by value).
struct ViewParams {
    float R[9], t[3];
    float fx, fy, cx, cy, znear;
    float alpha_min;      // the blend's skip threshold, for the record's exponent bound
    float cam_center[3];  // -R^T t, for the SH view direction
    int32_t width, height, tile, tiles_x, tiles_y;
    int32_t sh_degree, param_mode;
    int32_t footprint;  // 0: the bounding rectangle's tiles; 1: the tiles the disc meets
};

struct BlendParams {
    int32_t width, height, tiles_x, tiles_y;
    float alpha_min, alpha_max, t_min;
    float bg[3];
};

// Tiles [x, y] (inclusive) of tile row ty that the disc of radius r around
// (u, v) touches, within [x0, x1] (empty when x > y). The row's band
// [ty tile, (ty + 1) tile) lies dy = max(0, ty tile - v, v - (ty + 1) tile) from
// v, where the disc spans u +- sqrt(r^2 - dy^2); a tile is touched when its
// column meets that span. One rounding per step in a fixed order, so that every
// kernel (and the key path) finds the same tiles. The tile size is a power of
// two, so dividing by it is exact and equals multiplying by inv_tile.
__device__ __forceinline__ int2 row_span(float u, float v, float r, int tile, float inv_tile, int ty, int x0,
                                         int x1) {
    const float lo = (float)(ty * tile), hi = (float)((ty + 1) * tile);
    const float dy = fmaxf(0.0f, fmaxf(__fsub_rn(lo, v), __fsub_rn(v, hi)));
    // the row holding v: sqrt(fl(r r)) is r exactly (correctly rounded square and root)
    const float hw = dy == 0.0f ? r : __fsqrt_rn(fmaxf(__fsub_rn(__fmul_rn(r, r), __fmul_rn(dy, dy)), 0.0f));
    const float fa = floorf(__fmul_rn(__fsub_rn(u, hw), inv_tile));
    const float fb = floorf(__fmul_rn(__fadd_rn(u, hw), inv_tile));
    return make_int2((int)fminf(fmaxf(fa, (float)x0), (float)(x1 + 1)),
                     (int)fmaxf(fminf(fb, (float)x1), (float)(x0 - 1)));
}

// A kept Gaussian's footprint for the tile walks: centre, radius, and the
// column range of its bounding rectangle (x0 | x1 << 16, as float bits).
__device__ __forceinline__ float4 make_disc(float u, float v, float r, int x0, int x1) {
    return make_float4(u, v, r, __uint_as_float((uint32_t)x0 | ((uint32_t)x1 << 16)));
}
// Tiles of tile row ty (inside the rectangle's rows) that the footprint touches.
__device__ __forceinline__ int2 disc_span(float4 d, int tile, float inv_tile, int ty) {
    const uint32_t xr = __float_as_uint(d.w);
    return row_span(d.x, d.y, d.z, tile, inv_tile, ty, (int)(xr & 0xFFFF), (int)(xr >> 16));
}
// Tiles of tile row ty that kept Gaussian g touches: the whole row of its
// rectangle (footprint 0, the disc record is not read) or the disc's columns.
__device__ __forceinline__ int2 tile_span(int footprint, uint2 rect, const float4* __restrict__ disc, size_t g,
                                          int tile, float inv_tile, int ty) {
    if (footprint == 0) return make_int2((int)(rect.x & 0xFFFF), (int)(rect.y & 0xFFFF));
    return disc_span(disc[g], tile, inv_tile, ty);
}

// ---- launchers (defined in the .cu files, called from api.cu) ----
cudaError_t launch_project(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, cudaStream_t s);
cudaError_t launch_project_bwd(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, const float* g2d,
                               float* d_ms, float* d_op, float* d_col, cudaStream_t s);
struct AdamParams;
// With vp_next and f_next, the same pass also projects every Gaussian for the
// next view from its updated parameters (what launch_project would write there).
cudaError_t launch_project_bwd_adam(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, const float* g2d,
                                    float* m_ms, float* m_op, float* m_col, float* v_ms, float* v_op, float* v_col,
                                    const AdamParams& ap, cudaStream_t s, const ViewParams* vp_next = nullptr,
                                    const igs_frame* f_next = nullptr);
cudaError_t launch_bin_sort(const igs_frame& f, int footprint, cudaStream_t s);
cudaError_t launch_export_keys(const igs_frame& f, uint64_t* keys, cudaStream_t s);
// clear_g2d (optional, [n][8] floats, 16-byte aligned): zeroed by the blend's
// CTAs for the adjoint that follows (the frame's backward work counter is
// zeroed with the segment list whenever the frame has walk segments).
cudaError_t launch_blend_fwd(const igs_frame& f, const BlendParams& bp, float* img, cudaStream_t s,
                             float* clear_g2d = nullptr);
// The segmented backward's work counter of a frame (4 bytes, 16-byte aligned), to
// be zeroed before each launch_blend_bwd; nullptr when the frame has none.
void* blend_bwd_counter(const igs_frame& f);
// The pool slots the last forward of a frame took; nullptr when it has no segments.
const uint32_t* blend_segments_used(const igs_frame& f);
cudaError_t launch_blend_bwd(const igs_frame& f, const BlendParams& bp, const float* dL, float* g2d,
                             cudaStream_t s);
cudaError_t launch_l1(const float* img, const float* target, int64_t count, float* loss, float* grad,
                      cudaStream_t s);
// (1 - lambda) L1 + lambda (1 - SSIM) and its image gradient (ssim.cu); work holds ssim_work_floats floats.
size_t ssim_work_floats(int channels, int height, int width);
cudaError_t launch_l1_ssim(const float* img, const float* target, int channels, int height, int width, float lambda,
                           float* loss, float* ssim, float* grad, float* work, cudaStream_t s);
// Adam constants, formed in double on the host and rounded once.
struct AdamParams {
    float b1, b2, omb1, omb2;  // beta1, beta2, 1 - beta1, 1 - beta2
    float step_size;           // lr / (1 - beta1^t)
    float bc2_sqrt;            // sqrt(1 - beta2^t)
    float inv_bc2_sqrt;        // 1 / sqrt(1 - beta2^t)
    float eps;
    // If set: device floats (step_size, inv_bc2_sqrt, bc2_sqrt) written by
    // k_adam_advance, which replace the three host values (step count on the device).
    const float* dev_consts;
};
// Advance a device Adam step count (state[0] += 1) and write the bias-corrected
// constants of that step to state[1..3] as floats (one thread).
cudaError_t launch_adam_advance(int32_t* state, double lr, double b1, double b2, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t count, const AdamParams& a,
                        cudaStream_t s);

// Densify / prune of the 3D Gaussians (densify.cu): the per-step statistic and the
// keep / delete / divide pass into new buffers (arrays: means_sigma, opacity, color).
cudaError_t launch_grad_accum3d(const float* g2d, const uint32_t* count, int64_t n, float* accum, uint32_t* vis,
                                cudaStream_t s);
size_t densify_work_bytes(int64_t n);
cudaError_t launch_densify(const float* const in_p[3], const float* const in_m[3], const float* const in_v[3],
                           const float* accum, const uint32_t* vis, int64_t n, int C, int param_mode, float op_min,
                           float tau_g, float scale_min, int64_t capacity, float* const out_p[3],
                           float* const out_m[3], float* const out_v[3], int64_t* d_count, void* work,
                           cudaStream_t s);

// Merging of the 3D Gaussians that share a grid cell (merge.cu).
size_t merge_work_bytes(int64_t n);
cudaError_t launch_merge(const float* const in_p[3], const float* const in_m[3], const float* const in_v[3], int64_t n,
                         int C, int param_mode, const float lo[3], float cell, float scale_max, float* const out_p[3],
                         float* const out_m[3], float* const out_v[3], int64_t* d_count, void* work, cudaStream_t st);

// Octree initialisation of 3D Gaussians from a coloured point set (octree.cu).
size_t octree_work_bytes(int L);
cudaError_t launch_octree_init(const float* pts, const float* cols, long long npts, const float lo[3], float side,
                               int L, long long k_max, float opacity, int sh_degree, int param_mode, float* out_ms,
                               float* out_op, float* out_col, int32_t* count, void* work, cudaStream_t s);

// Multi-view batch (batch.cu): per-view record in device memory (the view table):
// the pose, where the view's tiles and image sit in the batch, and its frame.
struct BatchView {
    ViewParams vp;
    uint32_t tile_base;  // global id of the view's first tile (blend work items)
    uint32_t pad;
    int64_t img_off;     // first float of the view's image in the packed buffer
    float4* rec;         // the view's frame: projection outputs ...
    uint2* rect;
    float4* disc;
    uint32_t* count;
    uint32_t* depth_key;
    const uint2* ranges;  // ... and the binning's
    const uint32_t* vals;
    const uint32_t* info;
};
// Control words of a batch (igs_batch::info points at them): [16] status, [16] work counter, [V] entries.
constexpr int kBatchCtrlWords = 32;
size_t batch_table_bytes(int views);
bool batch_blend_variant_ok(int tile, int batch);
int batch_persistent_blocks(int tile, int batch);
// Fan-out streams of a batch (igs_batch::fanout), made once outside any capture.
cudaError_t batch_fanout_make(igs_batch& b);
void batch_fanout_free(igs_batch& b);
cudaError_t launch_render_batch(const igs_batch& b, const igs_frame* frames, const igs_scene& sc,
                                const BlendParams& bp, int sh_degree, float* images, cudaStream_t st, int footprint);

// Scratch layout of a frame (pieces of igs_frame::scratch).
struct SortScratch {
    unsigned long long* ditems_a;     // [n] (depth key | index) items
    unsigned long long* ditems_b;     // [n]
    unsigned long long* items_a;      // [capacity] (tile id | Gaussian id) items
    unsigned long long* items_b;      // [capacity] (route a: the level-1 items, then the exported tile ids)
    uint32_t* hist;                   // [8][256]: 4 depth passes, then up to 4 tile passes
    uint32_t* counters;               // [16] virtual block counters
    uint32_t* status_depth;           // [4][blocks(n)][256]
    uint32_t* status_tile;            // [tile_passes][blocks(capacity)][256]
    unsigned long long* scan_status;  // [scan blocks(n)]
    uint32_t* dup_start;              // [blocks(capacity) + 1] first Gaussian (in depth order) of each duplication block
    int32_t* grid;                    // [(tiles_y + 1) * (tiles_x + 1)] rectangle corner counts -> per-tile counts,
                                      // then (counting-sort route) [tiles_y + 1] tile-row differences
    uint32_t* vals;                   // sorted values: in the item buffer the last tile pass does not read
    uint32_t* tile_key;               // exported tile ids: in the item buffer the last tile pass reads
    uint32_t* walk_h1;                // [tiles_y][walk_chunks] level-1 row counts per chunk, then offsets
    uint32_t* walk_len;               // [tiles_y] items per tile-row list
    uint32_t* walk_rows;              // [tiles_y] list starts, first level-2 chunks, chunk sizes; [1] chunk total
    uint32_t* walk_h2;                // [level-2 chunks][tiles_x] level-2 tile counts per chunk, then slots
    uint2* walk_rect;                 // [n] rectangle of order[p] (level-1 count writes, level-1 place reads)
    void* seg_base;                   // the depth items' buffers (ditems_a, ditems_b), reused by the blends'
    size_t seg_bytes;                 // walk segments once binning is done
    int64_t walk_chunks;              // > 0: counting sort of the entries; 0: duplication + tile radix passes
    int tile_passes;
    int tile_bits;
};
SortScratch sort_scratch(const igs_frame& f);
size_t sort_scratch_bytes(int64_t n, int64_t capacity, int64_t tiles_x, int64_t tiles_y, int64_t chunks);

// Walk segments of the one-view blends (16- and 32-pixel binning tiles, one
// 8 x 8 pixel block per CTA). A block whose walk is long closes a segment at
// a list position that is a multiple of kSegStride when the open segment holds
// blends: it saves each pixel's state there (T, and the colour composited
// behind that position, once the walk has ended) in a pool slot, so that the
// backward can walk every segment in parallel instead of one block walking its
// whole list. A closed segment is items[slot] = (block, lo, hi, slot): list
// positions relative to the tile's first entry, lo = the cut it starts at, hi =
// one past its last blend, the state at hi in pool[slot]; a slot taken but not used
// holds block = kSegNone. A block's last segment, which ends with the final
// state (T_final and the background), is last[block] = (segments closed, lo,
// hi, -); lo = kSegNone when it holds no blend. The pieces live in the frame's
// depth-sort item buffers, which binning no longer needs once the entries are
// placed.
constexpr uint32_t kSegStride = 1024;        // list positions; a multiple of the forward's 64-entry batches
constexpr uint32_t kSegNone = 0xFFFFFFFFu;
constexpr int kSegMaxPerBlock = 64;          // segments a block closes at most (the rest stay in its last one)
struct SegCtrl {                             // all zeroed before each forward; next (the
    uint32_t next, slots_used, pad0, pad1;   // backward's work counter) also before each backward
};
struct SegLayout {
    SegCtrl* ctrl;
    uint4* last;      // [blocks] (closed, lo, hi, -) of each block's last segment
    uint4* items;     // [slots] (block, lo, hi, slot) of each closed segment
    float4* pool;     // [slots][64] (T, S_r, S_g, S_b) per pixel of the block, pixel = row * 8 + column
    uint32_t slots;   // 0: segments off
    uint32_t blocks;
};
// Carved from [base, base + bytes) for `blocks` 8 x 8 blocks (slots = 0 when it does not fit).
__host__ __device__ inline SegLayout seg_layout(void* base, size_t bytes, int64_t blocks) {
    SegLayout L{};
    const size_t head = 256 + (((size_t)blocks * 16 + 255) & ~(size_t)255);
    if (!base || bytes < head + 1040 || blocks <= 0 || blocks >= (1 << 24)) return L;
    int64_t slots = (int64_t)((bytes - head) / 1040);  // 16 B item + 1 KB of pixel states per slot
    if (slots > (1 << 20)) slots = 1 << 20;
    char* p = static_cast<char*>(base);
    L.ctrl = reinterpret_cast<SegCtrl*>(p);
    L.last = reinterpret_cast<uint4*>(p + 256);
    L.items = reinterpret_cast<uint4*>(p + head);
    L.pool = reinterpret_cast<float4*>(p + head + (((size_t)slots * 16 + 255) & ~(size_t)255));
    if ((size_t)(reinterpret_cast<char*>(L.pool) - p) + (size_t)slots * 1024 > bytes) --slots;
    L.slots = slots > 0 ? (uint32_t)slots : 0;
    L.blocks = (uint32_t)blocks;
    return L;
}
int64_t sort_walk_chunks(int64_t tiles_x, int64_t tiles_y);
int tile_passes_for(int64_t tiles);

}  // namespace igs
