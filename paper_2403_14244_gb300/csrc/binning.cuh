// Radix-sort, scan and duplication kernels of the binning (sort.cu) and the
// allocation-free ordering. Internal to libigs.
//
// Each radix pass is a single sweep over (key | value) items: a block counts
// the digits of its 5120 items and publishes those counts at once, ranks the
// items within each warp with ballots, looks back over earlier blocks (eight
// at a time) for its global digit offsets, and scatters the items staged in
// digit order. Every wait on another block is bounded (kMaxSpin polls); on
// expiry the block records IGS_ERR_DEVICE_TIMEOUT, which aborts the frame.
#pragma once

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
// Consecutive entries one duplication thread writes.
constexpr int kDupPerThread = kDupTile / 256;

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

// In place: each of `rows` rows of 256 digit counts becomes its exclusive
// prefix (the global start of each digit in that pass). Blocks of 1024 threads,
// block b handling rows [8b, 8b + 8).
__global__ void __launch_bounds__(1024) k_hist_to_offsets(uint32_t* __restrict__ hist, int rows) {
    const int r0 = blockIdx.x * 8;
    const int n = min(8, rows - r0) * kRadix;
    uint32_t* h = hist + (size_t)r0 * kRadix;
    uint32_t v[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int idx = threadIdx.x + r * 1024;
        v[r] = 0;
        if (idx < n) {
            const uint32_t* row = h + (idx & ~255);
            for (int k = 0; k < (idx & 255); ++k) v[r] += row[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int idx = threadIdx.x + r * 1024;
        if (idx < n) h[idx] = v[r];
    }
}

// One stable LSD radix pass over `count` items (key << 32 | value) on the 8-bit
// digit (key >> shift) & 255. IN_KEYS32: the input is the 32-bit key array and
// the value is the index (first pass of the depth sort). OUT_VALS: write only the
// values (last pass). digit_base = this pass's global start of every digit.
// status = [blocks][256] look-back words, zero on entry.
// With gridDim.y > 1 the launch sorts gridDim.y independent segments of
// count_host items each (segment y at items [y * count_host, ...)); every
// segment has its own counter, look-back words and digit bases, and the first
// pass's values are the global item index.
// SKIPPABLE (one segment only): when *skip_flag is set, the pass writes only
// the values, to skip_vals, or, without skip_vals, does nothing (the redundant
// top pass of a depth sort whose third pass wrote the order).
template <bool IN_KEYS32, bool OUT_VALS, bool SKIPPABLE = false>
__global__ void __launch_bounds__(kSortThreads, 4) k_radix_pass(
    const void* __restrict__ in_, void* __restrict__ out_, const uint32_t* __restrict__ d_count, uint32_t count_host,
    int shift, const uint32_t* __restrict__ digit_base, uint32_t* __restrict__ status,
    uint32_t* __restrict__ block_counter, uint32_t* __restrict__ info, uint32_t silent_blk = 0xFFFFFFFFu,
    const uint32_t* __restrict__ skip_flag = nullptr, uint32_t* __restrict__ skip_vals = nullptr) {
    pdl_wait();
    if (SKIPPABLE && !skip_vals && *skip_flag) return;
    {
        const uint64_t seg = blockIdx.y;
        if (IN_KEYS32)
            in_ = static_cast<const uint32_t*>(in_) + seg * count_host;
        else
            in_ = static_cast<const unsigned long long*>(in_) + seg * count_host;
        if (OUT_VALS)
            out_ = static_cast<uint32_t*>(out_) + seg * count_host;
        else
            out_ = static_cast<unsigned long long*>(out_) + seg * count_host;
        digit_base += seg * kRadix;
        status += seg * gridDim.x * kRadix;
        block_counter += seg;
    }
    const uint64_t seg_base = (uint64_t)blockIdx.y * count_host;
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
                it[i] = ((u64)static_cast<const uint32_t*>(in_)[g] << 32) | (uint32_t)(seg_base + g);
            else
                it[i] = static_cast<const u64*>(in_)[g];
        }
    } else {
#pragma unroll
        for (int i = 0; i < kSortIpt; ++i) {
            const uint32_t loc = wbase + i * 32;
            const uint64_t g = base + loc;
            if (loc < valid)
                it[i] = IN_KEYS32 ? (((u64)static_cast<const uint32_t*>(in_)[g] << 32) | (uint32_t)(seg_base + g))
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
    // silent_blk (failure-detection tests only): that block never publishes, so
    // every later block's bounded look-back runs out
    const bool silent = blk == silent_blk;
    if (!silent) st_relaxed_u32(&my[tid], (blk == 0 ? kFlagPre : kFlagAgg) | (s_cnt[tid] & kValMask));
    // rank within the warp, in item order
    uint32_t rank2[kSortIpt / 2];  // two 16-bit ranks per register (ranks < kSortTile)
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
    __syncthreads();
    // stage the block's items in digit order (needs only block-local offsets, so it
    // runs before the look-back and gives earlier blocks time to publish)
#pragma unroll
    for (int i = 0; i < kSortIpt; ++i) {
        const uint32_t d = (uint32_t)(it[i] >> (32 + shift)) & 0xFFu;
        s_items[s_whist[w][d] + ((rank2[i >> 1] >> (16 * (i & 1))) & 0xFFFFu)] = it[i];
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
                    __nanosleep(200);
                    v[j] = ld_relaxed_u32(status + (size_t)(b - j) * kRadix + tid);
                }
                if (done) break;
                excl += v[j] & kValMask;
                if ((v[j] & kFlagMask) == kFlagPre) done = true;
            }
            b -= nw;
        }
        if (!silent) st_relaxed_u32(&my[tid], kFlagPre | ((excl + cnt) & kValMask));
    }
    s_delta[tid] = (int32_t)(digit_base[tid] + excl) - (int32_t)local;
    const bool skipped = SKIPPABLE && !OUT_VALS && skip_vals && *skip_flag;  // (read late: fewer live registers)
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
        else if (skipped)
            skip_vals[pos] = (uint32_t)item;
        else
            static_cast<u64*>(out_)[pos] = item;
    }
}

// Exclusive scan of count[order[p]] over p (the tile counts in front-to-back
// order) with decoupled look-back (one warp reads 32 predecessors at a time);
// writes offset[p], M, the kept count (if add_kept), and for every duplication
// block the position in `order` of the Gaussian that holds its first entry.
__global__ void __launch_bounds__(kScanThreads) k_scan_offsets(const uint32_t* __restrict__ order,
                                                               const uint32_t* __restrict__ count, uint32_t n,
                                                               uint32_t* __restrict__ offset,
                                                               uint32_t* __restrict__ dup_start,
                                                               unsigned long long* __restrict__ status,
                                                               uint32_t* __restrict__ block_counter,
                                                               uint32_t* __restrict__ info, uint64_t capacity,
                                                               bool add_kept) {
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
    if (add_kept && lane == 0 && warp_kept) atomicAdd(&info[kInfoKept], warp_kept);
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
// search of the block's window of offsets, then its tile among the tiles the
// Gaussian touches (row by row of its rectangle, row_span in each row). Writes (tile id << 32 | Gaussian id), or only the
// Gaussian id when no tile pass follows.
__global__ void __launch_bounds__(256) k_duplicate(const uint32_t* __restrict__ order,
                                                   const uint32_t* __restrict__ offset,
                                                   const uint32_t* __restrict__ dup_start,
                                                   const uint2* __restrict__ rect,
                                                   const float4* __restrict__ disc, int tile, int footprint,
                                                   uint32_t n, int tiles_x,
                                                   u64* __restrict__ items, uint32_t* __restrict__ vals_direct,
                                                   const uint32_t* __restrict__ info) {
    __shared__ uint32_t s_off[kDupTile + 2];
    __shared__ uint32_t s_ord[kDupTile + 1];
    __shared__ u64 s_items[kDupTile];  // the block's entries, written out coalesced at the end
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
    // Entries at or past `reach` belong to Gaussians after the window (when
    // Gaussians without entries sit inside it); those entries search the
    // global offsets.
    const uint32_t reach = s_off[cnt];
    // each thread: kDupPerThread consecutive entries, one search then a walk
    const uint32_t first = min((uint32_t)e0 + threadIdx.x * kDupPerThread, e_end);
    const uint32_t last = min(first + kDupPerThread, e_end);
    uint32_t k;       // window slot (or global position) of the current Gaussian
    bool global;
    auto locate = [&](uint32_t e) {
        if (e < reach) {
            uint32_t lo = 0, hi = cnt;  // largest k with s_off[k] <= e
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_off[mid] <= e) lo = mid; else hi = mid;
            }
            k = lo;
            global = false;
        } else {
            uint32_t lo = pb, hi = n;  // largest p with offset[p] <= e
            while (hi - lo > 1) {
                const uint32_t mid = lo + ((hi - lo) >> 1);
                if (offset[mid] <= e) lo = mid; else hi = mid;
            }
            k = lo;
            global = true;
        }
    };
    uint32_t e = first;
    if (e < last) locate(first);
    while (e < last) {
        const uint32_t g = global ? order[k] : s_ord[k];
        const uint32_t start = global ? offset[k] : s_off[k];
        const uint32_t next = global ? (k + 1 < n ? offset[k + 1] : M) : s_off[k + 1];
        const uint32_t stop = min(last, next);
        if (g < n && start <= e) {
            const uint2 r = rect[g];
            const float inv = 1.0f / (float)tile;
            const int y0 = r.x >> 16, y1 = r.y >> 16;
            // the row holding entry j (rows in order, each its touched tiles) and its span
            uint32_t j = e - start;
            int ty = y0;
            int2 sp = tile_span(footprint, r, disc, g, tile, inv, ty);
            for (;;) {
                const uint32_t w = sp.y >= sp.x ? (uint32_t)(sp.y - sp.x + 1) : 0u;
                if (j < w || ty >= y1) break;
                j -= w;
                sp = tile_span(footprint, r, disc, g, tile, inv, ++ty);
            }
            int col = sp.x + (int)j;
            for (; e < stop; ++e) {
                if (col > sp.y) break;  // never: the count is the total of the spans
                const uint32_t t = (uint32_t)ty * (uint32_t)tiles_x + (uint32_t)col;
                s_items[e - (uint32_t)e0] = ((u64)t << 32) | g;
                // next touched tile, row by row
                if (++col > sp.y) {
                    while (ty < y1) {
                        sp = tile_span(footprint, r, disc, g, tile, inv, ++ty);
                        if (sp.y >= sp.x) break;
                    }
                    col = sp.x;
                }
            }
            e = stop;
        } else {
            e = stop;
        }
        if (e >= last) break;
        // the next Gaussian with entries
        if (!global && k + 1 < cnt && e < reach) {
            ++k;
            while (k + 1 < cnt && s_off[k + 1] <= e) ++k;
        } else {
            locate(e);
        }
    }
    __syncthreads();
    // coalesced write-out of the block's entries [e0, e_end)
    const uint32_t ne = e_end - (uint32_t)e0;
    if (vals_direct)
        for (uint32_t q = threadIdx.x; q < ne; q += blockDim.x) vals_direct[e0 + q] = (uint32_t)s_items[q];
    else
        for (uint32_t q = threadIdx.x; q < ne; q += blockDim.x) items[e0 + q] = s_items[q];
}

}  // namespace
}  // namespace igs
