// Multi-view batch rendering: V views of one scene, each with its own pose and
// image size, rendered by one chain of launches with no host synchronisation
// (so the chain can be captured in a CUDA graph and replayed with new poses):
//   project all (view, Gaussian) pairs     one launch, a thread per Gaussian that
//                                          reads it once and projects it for every
//                                          view; the poses come from the device
//                                          view table
//   bin and sort each view                 each view's frame as igs_bin_sort does it,
//                                          the views spread over up to 16 streams
//                                          that fork from the caller's stream and
//                                          join it again
//   batch status                           one block: the views' status words summed
//   blend                                  one launch over every view's tiles: one
//                                          64-thread CTA per 8 x 8 block, or a
//                                          persistent whole-tile blend whose CTAs
//                                          take (view, tile) items from a counter
// A view's pixels are bit-identical to rendering it alone (same projection,
// same binning, same per-tile compositing routine). Each view's binning alone
// is a chain of short, partly single-wave kernels; running the views' chains
// concurrently fills the GPU where one view's chain cannot.
#include <algorithm>
#include <cstring>
#include <vector>

#include "blendtile.cuh"
#include "projection.cuh"

namespace igs {

namespace {

constexpr int kFanout = 16;  // most streams the views' binnings spread over

// Streams and events of one batch (host object behind igs_batch::fanout).
struct Fanout {
    int dev = -1;
    int k = 0;
    cudaStream_t st[kFanout] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kFanout] = {};
};

// Every view of the batch for one Gaussian per thread: the Gaussian's mean,
// scale, opacity and colour row are read once and projected for each view in
// turn (what project_one writes into that view's frame), the view table staged
// kViewChunk entries at a time in shared memory. The scene is read once per
// batch, not once per view; the per-view writes stay coalesced across a warp.
constexpr int kViewChunk = 16;
template <int DEG>
__global__ void __launch_bounds__(256) k_project_views(const float4* __restrict__ ms, const float* __restrict__ op,
                                                       const float* __restrict__ col, int64_t n,
                                                       const BatchView* __restrict__ views, int V) {
    constexpr int C = DEG < 0 ? 3 : 3 * (DEG + 1) * (DEG + 1);
    static_assert(sizeof(BatchView) % 4 == 0, "the view table is staged as 32-bit words");
    __shared__ BatchView s_v[kViewChunk];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = i < n;
    float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
    float o = 0.f;
    float c[48];
    if (on) {
        m = __ldg(ms + i);
        o = __ldg(op + i);
        load_color<DEG>(col, i, c);
    }
    constexpr int kWords = (int)(sizeof(BatchView) / 4);
    for (int v0 = 0; v0 < V; v0 += kViewChunk) {
        const int nv = min(kViewChunk, V - v0);
        __syncthreads();  // the previous chunk's views are no longer read
        for (int k = threadIdx.x; k < nv * kWords; k += blockDim.x)
            reinterpret_cast<uint32_t*>(s_v)[k] = reinterpret_cast<const uint32_t*>(views + v0)[k];
        __syncthreads();
        if (!on) continue;
        for (int k = 0; k < nv; ++k) {
            const BatchView& bv = s_v[k];
            project_one_vals<DEG>(m, o, [&](float cc[48]) {
#pragma unroll
                for (int q = 0; q < C; ++q) cc[q] = c[q];
            }, bv.vp, bv.rec + 2 * i, bv.rect + i, bv.disc + i, bv.count + i, bv.depth_key + i);
        }
    }
}

// One block: the batch's status words from the views' (entries summed, the
// first error, entries needed summed, abort if any view aborted) and each
// view's entry count.
__global__ void __launch_bounds__(256) k_batch_info(const BatchView* __restrict__ views, int V,
                                                    uint32_t* __restrict__ info, uint32_t* __restrict__ entries) {
    __shared__ unsigned long long s_m, s_need, s_kept;
    __shared__ uint32_t s_abort;
    if (threadIdx.x == 0) {
        s_m = s_need = s_kept = 0ull;
        s_abort = 0u;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        const uint32_t* f = views[v].info;
        entries[v] = f[kInfoM];
        atomicAdd(&s_m, (unsigned long long)f[kInfoM]);
        atomicAdd(&s_need, (unsigned long long)f[kInfoNeed]);
        atomicAdd(&s_kept, (unsigned long long)f[kInfoKept]);
        if (f[kInfoAbort]) atomicExch(&s_abort, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t err = 0u;
        for (int v = 0; v < V && !err; ++v) err = views[v].info[kInfoErr];  // the first view's error
        info[kInfoM] = (uint32_t)min(s_m, 0xFFFFFFFFull);
        info[kInfoKept] = (uint32_t)min(s_kept, 0xFFFFFFFFull);
        info[kInfoNeed] = (uint32_t)min(s_need, 0xFFFFFFFFull);
        info[kInfoErr] = err;
        info[kInfoAbort] = s_abort;
    }
}

// The view of global tile w: the largest v with tile_base[v] <= w.
__device__ __forceinline__ int view_of(const BatchView* __restrict__ views, int V, uint32_t w) {
    int lo = 0, hi = V;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (views[mid].tile_base <= w) lo = mid; else hi = mid;
    }
    return lo;
}

// Persistent blend: every CTA takes (view, tile) work items from one counter
// until none is left; work item w is global tile w. A view whose binning
// aborted is skipped (its image untouched).
template <int TS, int B>
__global__ void __launch_bounds__(TS* TS) k_blend_persistent(const BatchView* __restrict__ views, int V,
                                                             uint32_t tiles_total, BlendParams P,
                                                             float* __restrict__ images, uint32_t* __restrict__ work) {
    __shared__ float4 s_a[B];
    __shared__ float4 s_c[B];
    __shared__ uint32_t s_item;
    for (;;) {
        __syncthreads();  // s_item / s_a / s_c are free again
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t w = s_item;
        if (w >= tiles_total) break;
        const BatchView& bv = views[view_of(views, V, w)];
        if (bv.info[kInfoAbort]) continue;
        const ViewParams& vp = bv.vp;
        const uint32_t t = w - bv.tile_base;
        blend_tile_fwd<TS, B>((int)(t % (uint32_t)vp.tiles_x), (int)(t / (uint32_t)vp.tiles_x), vp.width, vp.height,
                              bv.ranges[t], bv.vals, bv.rec, P.alpha_min, P.alpha_max, P.t_min, P.bg, s_a, s_c,
                              images + bv.img_off, nullptr, nullptr);
    }
}

// Sub-tile blend: one 64-thread CTA per 8 x 8 pixel block of every view's
// binning tiles (item w: tile w / (TS/8)^2, block w % (TS/8)^2), walking the
// tile's entries; each block stops on its own. The hardware block scheduler
// balances the mixed view sizes, so the launch is not persistent.
template <int TS>
__global__ void __launch_bounds__(64) k_blend_batch_sub(const BatchView* __restrict__ views, int V,
                                                        uint32_t tiles_total, BlendParams P,
                                                        float* __restrict__ images, uint32_t* __restrict__ work) {
    constexpr int SUB = TS / 8, NS = SUB * SUB;
    __shared__ float4 s_a[64];
    __shared__ float4 s_c[64];
    const uint32_t w = blockIdx.x / NS, q = blockIdx.x % NS;
    const BatchView& bv = views[view_of(views, V, w)];
    if (bv.info[kInfoAbort]) return;
    const ViewParams& vp = bv.vp;
    const uint32_t t = w - bv.tile_base;
    const int tx = (int)(t % (uint32_t)vp.tiles_x), ty = (int)(t / (uint32_t)vp.tiles_x);
    blend_tile_fwd<8, 64>(tx * SUB + (int)(q % SUB), ty * SUB + (int)(q / SUB), vp.width, vp.height, bv.ranges[t],
                          bv.vals, bv.rec, P.alpha_min, P.alpha_max, P.t_min, P.bg, s_a, s_c, images + bv.img_off,
                          nullptr, nullptr);
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

size_t batch_table_bytes(int views) { return sizeof(BatchView) * (size_t)views; }

bool batch_blend_variant_ok(int tile, int batch) {
    void* fn;
    return blend_variant(tile, batch, &fn);
}

cudaError_t batch_fanout_make(igs_batch& b) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (b.fanout) return static_cast<Fanout*>(b.fanout)->dev == dev ? cudaSuccess : cudaErrorInvalidDevice;
    Fanout* f = new Fanout();
    f->dev = dev;
    f->k = std::min(kFanout, std::max(1, (int)b.views));
    b.fanout = f;  // (freed by batch_fanout_free whatever happens below)
    if ((e = cudaEventCreateWithFlags(&f->fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    for (int k = 0; k < f->k; ++k) {
        if ((e = cudaStreamCreateWithFlags(&f->st[k], cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&f->join[k], cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void batch_fanout_free(igs_batch& b) {
    Fanout* f = static_cast<Fanout*>(b.fanout);
    if (!f) return;
    for (int k = 0; k < kFanout; ++k) {
        if (f->st[k]) {
            cudaStreamSynchronize(f->st[k]);
            cudaStreamDestroy(f->st[k]);
        }
        if (f->join[k]) cudaEventDestroy(f->join[k]);
    }
    if (f->fork) cudaEventDestroy(f->fork);
    delete f;
    b.fanout = nullptr;
}

cudaError_t launch_render_batch(const igs_batch& b, const igs_frame* frames, const igs_scene& sc,
                                const BlendParams& bp, int sh_degree, float* images, cudaStream_t st,
                                int footprint) {
    const int V = b.views;
    const int64_t n = b.n;
    const Fanout* fo = static_cast<const Fanout*>(b.fanout);
    const BatchView* table = static_cast<const BatchView*>(b.table);
    uint32_t* work = b.info + 16;
    cudaError_t e;
#define CK(x) do { if ((e = (x)) != cudaSuccess) { g_failed_call = #x " (batch.cu:" IGS_STR(__LINE__) ")"; return e; } } while (0)
    if (!fo || fo->k < 1) return cudaErrorInvalidValue;
    CK(cudaMemsetAsync(b.info, 0, 4 * (size_t)kBatchCtrlWords, st));
    if (V == 0) return cudaSuccess;
    // 1. projection of every (view, Gaussian) into the views' frames (an empty
    //    scene still bins to empty tiles and blends the background)
    if (n > 0) {
        const unsigned grid = (unsigned)ceil_div(n, 256);
        auto ms = reinterpret_cast<const float4*>(sc.means_sigma);
#define IGS_PB(D) k_project_views<D><<<grid, 256, 0, st>>>(ms, sc.opacity, sc.color, n, table, V)
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
    // 2. each view's binning on a fan-out stream (fork from st, join back into st)
    const int K = std::min(fo->k, V);
    CK(cudaEventRecord(fo->fork, st));
    for (int k = 0; k < K; ++k) CK(cudaStreamWaitEvent(fo->st[k], fo->fork, 0));
    {  // longest first, each onto the stream with the least work so far: a view's binning takes
       // about a fixed latency plus time in proportion to its entries (its capacity stands in)
        constexpr int64_t kViewFloor = 8 << 20;  // the fixed part, in entries
        std::vector<int> order(V);
        for (int v = 0; v < V; ++v) order[v] = v;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int c) { return frames[a].capacity > frames[c].capacity; });
        std::vector<int64_t> load(K, 0);
        for (int v : order) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            CK(launch_bin_sort(frames[v], footprint, fo->st[k]));
            load[k] += frames[v].capacity + kViewFloor;
        }
    }
    for (int k = 0; k < K; ++k) {
        CK(cudaEventRecord(fo->join[k], fo->st[k]));
        CK(cudaStreamWaitEvent(st, fo->join[k], 0));
    }
    // 3. the batch's status words and each view's entries
    k_batch_info<<<1, 256, 0, st>>>(table, V, b.info, b.view_entries);
    count_launches();
    CK(cudaGetLastError());
    // 4. one blend over every view's tiles
    void* fn = nullptr;
    bool sub = false;
    if (!blend_variant(b.tile, b.blend_batch, &fn, &sub)) return cudaErrorInvalidValue;
    const int64_t per_tile = sub ? (int64_t)(b.tile / 8) * (b.tile / 8) : 1;
    const unsigned nblocks = (unsigned)(sub ? std::max<int64_t>(1, b.tiles_total * per_tile)
                                            : std::max<int64_t>(1, std::min<int64_t>(b.persistent_blocks, b.tiles_total)));
    uint32_t tt = (uint32_t)b.tiles_total;
    int Vi = V;
    BlendParams bpp = bp;
    void* args[] = {(void*)&table, (void*)&Vi, (void*)&tt, (void*)&bpp, (void*)&images, (void*)&work};
    CK(cudaLaunchKernel(fn, dim3(nblocks), dim3(sub ? 64 : b.tile * b.tile), args, 0, st));
    count_launches();
#undef CK
    return cudaSuccess;
}

}  // namespace igs
