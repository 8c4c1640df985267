// Densify / prune of the 3D Gaussians (Sec. 3.2: a particle whose A_k falls
// below a threshold is deleted, and particles may be divided; Sec. 2.5's
// multiscale property, with the Octree of Sec. 3.1 as the division pattern).
//
// The statistic (k_grad_accum3d, after each backward blend): for every
// Gaussian that touched a tile, accum += |(du, dv)| of its screen-space
// gradient (FP32, one rounding per step) and vis += 1.
//
// The densify pass keeps, deletes or divides every Gaussian into new buffers
// in index order (children in place of their parent), in three launches:
//   k_dens_count  per block of kDensTile Gaussians: kept and candidate counts
//   k_dens_scan   one CTA: block prefixes, how many candidates fit the
//                 capacity (each division adds 7), each block's first output slot
//   k_dens_write  per block: each Gaussian's slot (block scans of 256 at a
//                 time), then the block copies parameters and moments (kept) or
//                 writes the eight children (zero moments), rows cooperatively.
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace igs {
namespace {

constexpr int kDensThreads = 256;
constexpr int kDensRounds = 8;
constexpr int kDensTile = kDensThreads * kDensRounds;

struct DensIn {
    const float4* ms;
    const float* op;
    const float* col;
    const float4* m_ms;
    const float* m_op;
    const float* m_col;
    const float4* v_ms;
    const float* v_op;
    const float* v_col;
    const float* accum;
    const uint32_t* vis;
};
struct DensOut {
    float4* ms;
    float* op;
    float* col;
    float4* m_ms;
    float* m_op;
    float* m_col;
    float4* v_ms;
    float* v_op;
    float* v_col;
};
struct DensParams {
    int64_t n, capacity;
    int C, param_mode;
    float op_min, tau_g, scale_min;
};

__global__ void __launch_bounds__(256) k_grad_accum3d(const float4* __restrict__ g2d, const uint32_t* __restrict__ count,
                                                      int64_t n, float* __restrict__ accum, uint32_t* __restrict__ vis) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (count[i] == 0) continue;
        const float4 g = g2d[2 * i];
        const float sq = __fadd_rn(__fmul_rn(g.x, g.x), __fmul_rn(g.y, g.y));
        accum[i] = __fadd_rn(accum[i], __fsqrt_rn(sq));
        vis[i] += 1u;
    }
}

// Kept: stored opacity not below op_min. Candidate: kept, seen (vis > 0), mean
// gradient above tau_g (accum > tau_g * vis, one FP32 product) and stored scale
// not below scale_min.
__device__ __forceinline__ void dens_flags(const DensIn& in, const DensParams& P, int64_t i, bool& keep, bool& cand) {
    keep = !(in.op[i] < P.op_min);
    const uint32_t vs = in.vis[i];
    cand = keep && vs > 0 && in.accum[i] > __fmul_rn(P.tau_g, (float)vs) && in.ms[i].w >= P.scale_min;
}

__global__ void __launch_bounds__(kDensThreads) k_dens_count(DensIn in, DensParams P, uint2* __restrict__ blk) {
    __shared__ uint32_t s_k[kDensThreads / 32], s_c[kDensThreads / 32];
    uint32_t nk = 0, nc = 0;
    const int64_t b0 = (int64_t)blockIdx.x * kDensTile;
    for (int r = 0; r < kDensRounds; ++r) {
        const int64_t i = b0 + r * kDensThreads + threadIdx.x;
        if (i < P.n) {
            bool keep, cand;
            dens_flags(in, P, i, keep, cand);
            nk += keep;
            nc += cand;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nk += __shfl_xor_sync(0xffffffffu, nk, o);
        nc += __shfl_xor_sync(0xffffffffu, nc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_k[threadIdx.x >> 5] = nk;
        s_c[threadIdx.x >> 5] = nc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tk = 0, tc = 0;
        for (int w = 0; w < kDensThreads / 32; ++w) {
            tk += s_k[w];
            tc += s_c[w];
        }
        blk[blockIdx.x] = make_uint2(tk, tc);
    }
}

// One CTA: base[b] = (first output slot of block b, candidates before block b);
// meta = (allowed divisions, output count).
constexpr int kDensScanThreads = 1024;
__global__ void __launch_bounds__(kDensScanThreads) k_dens_scan(const uint2* __restrict__ blk, int64_t blocks,
                                                                DensParams P, unsigned long long* __restrict__ base,
                                                                long long* __restrict__ meta,
                                                                int64_t* __restrict__ d_count) {
    __shared__ unsigned long long s_w[kDensScanThreads / 32][2];
    __shared__ unsigned long long s_carry[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // totals first: the number of divisions that fit depends on all of them
    unsigned long long tk = 0, tc = 0;
    for (int64_t b = threadIdx.x; b < blocks; b += kDensScanThreads) {
        tk += blk[b].x;
        tc += blk[b].y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tk += __shfl_xor_sync(0xffffffffu, tk, o);
        tc += __shfl_xor_sync(0xffffffffu, tc, o);
    }
    if (lane == 0) {
        s_w[w][0] = tk;
        s_w[w][1] = tc;
    }
    __syncthreads();
    long long keep = 0, cand = 0;
    for (int k = 0; k < kDensScanThreads / 32; ++k) {
        keep += (long long)s_w[k][0];
        cand += (long long)s_w[k][1];
    }
    const long long allowed = min(P.capacity > keep ? (P.capacity - keep) / 7 : 0LL, cand);
    __syncthreads();
    if (threadIdx.x == 0) {
        s_carry[0] = s_carry[1] = 0ull;
        meta[0] = allowed;
        meta[1] = min(keep + 7 * allowed, (long long)P.capacity);
        *d_count = meta[1];
    }
    __syncthreads();
    for (int64_t b0 = 0; b0 < blocks; b0 += kDensScanThreads) {
        const int64_t b = b0 + threadIdx.x;
        const uint2 v = b < blocks ? blk[b] : make_uint2(0u, 0u);
        unsigned long long ik = v.x, ic = v.y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long yk = __shfl_up_sync(0xffffffffu, ik, o);
            const unsigned long long yc = __shfl_up_sync(0xffffffffu, ic, o);
            if (lane >= o) {
                ik += yk;
                ic += yc;
            }
        }
        if (lane == 31) {
            s_w[w][0] = ik;
            s_w[w][1] = ic;
        }
        __syncthreads();
        unsigned long long pk = s_carry[0], pc = s_carry[1], sk = 0, sc = 0;
        for (int k = 0; k < kDensScanThreads / 32; ++k) {
            if (k < w) {
                pk += s_w[k][0];
                pc += s_w[k][1];
            }
            sk += s_w[k][0];
            sc += s_w[k][1];
        }
        pk += ik - v.x;  // kept before block b
        pc += ic - v.y;  // candidates before block b
        if (b < blocks) {
            const unsigned long long div_before = min((unsigned long long)allowed, pc);
            base[2 * b] = pk + 7ull * div_before;
            base[2 * b + 1] = pc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_carry[0] += sk;
            s_carry[1] += sc;
        }
        __syncthreads();
    }
}

template <int C>
__global__ void __launch_bounds__(kDensThreads) k_dens_write(DensIn in, DensOut out, DensParams P,
                                                             const unsigned long long* __restrict__ base,
                                                             const long long* __restrict__ meta) {
    __shared__ uint32_t s_wk[kDensThreads / 32], s_wc[kDensThreads / 32];
    __shared__ long long s_dst[kDensThreads];
    __shared__ int s_nout[kDensThreads];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * kDensTile;
    const long long allowed = meta[0], cap = P.capacity;
    long long slot = (long long)base[2 * blockIdx.x];
    long long crank = (long long)base[2 * blockIdx.x + 1];
    for (int r = 0; r < kDensRounds; ++r) {
        const int64_t r0 = b0 + r * kDensThreads;
        if (r0 >= P.n) break;
        const int64_t i = r0 + threadIdx.x;
        bool keep = false, cand = false;
        if (i < P.n) dens_flags(in, P, i, keep, cand);
        // candidates before this one (index order), then outputs before this one
        const uint32_t bc = __ballot_sync(0xffffffffu, cand);
        if (lane == 0) s_wc[w] = __popc(bc);
        __syncthreads();
        long long cpre = crank + __popc(bc & ((1u << lane) - 1u)), ctot = 0;
        for (int k = 0; k < kDensThreads / 32; ++k) {
            if (k < w) cpre += s_wc[k];
            ctot += s_wc[k];
        }
        const bool divide = cand && cpre < allowed;
        const int nout = divide ? 8 : (keep ? 1 : 0);
        // exclusive scan of nout (0, 1 or 8) over the round
        uint32_t incl = (uint32_t)nout;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wk[w] = incl;
        __syncthreads();
        long long opre = slot + incl - (uint32_t)nout, otot = 0;
        for (int k = 0; k < kDensThreads / 32; ++k) {
            if (k < w) opre += s_wk[k];
            otot += s_wk[k];
        }
        s_dst[threadIdx.x] = opre;
        s_nout[threadIdx.x] = nout;
        // means, scale, opacity and their moments: one thread per Gaussian
        if (divide) {
            const float4 m = in.ms[i];
            const float sigma = P.param_mode == 1 ? (float)exp((double)m.w) : m.w;
            const float h = __fmul_rn(0.5f, sigma);
            const float cs = P.param_mode == 1 ? __fsub_rn(m.w, 0.6931472f) : __fmul_rn(0.5f, m.w);
            const float o = in.op[i];
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const long long d = opre + c;  // < cap: the divisions were counted to fit
                out.ms[d] = make_float4((c & 1) ? __fadd_rn(m.x, h) : __fsub_rn(m.x, h),
                                        (c & 2) ? __fadd_rn(m.y, h) : __fsub_rn(m.y, h),
                                        (c & 4) ? __fadd_rn(m.z, h) : __fsub_rn(m.z, h), cs);
                out.op[d] = o;
                out.m_ms[d] = zero;
                out.v_ms[d] = zero;
                out.m_op[d] = 0.f;
                out.v_op[d] = 0.f;
            }
        } else if (keep && opre < cap) {
            out.ms[opre] = in.ms[i];
            out.m_ms[opre] = in.m_ms[i];
            out.v_ms[opre] = in.v_ms[i];
            out.op[opre] = in.op[i];
            out.m_op[opre] = in.m_op[i];
            out.v_op[opre] = in.v_op[i];
        }
        __syncthreads();
        // colour rows and their moments, cooperatively: consecutive float4 (rows of
        // a multiple of 4 floats, 16-byte aligned) or floats per thread
        const int nr = (int)min((int64_t)kDensThreads, P.n - r0);
        constexpr int V = (C % 4 == 0) ? 4 : 1;  // floats per access
        constexpr int CV = C / V;                // accesses per row
        using T = typename std::conditional<V == 4, float4, float>::type;
        const T zero{};
        const T* icol = reinterpret_cast<const T*>(in.col);
        const T* imc = reinterpret_cast<const T*>(in.m_col);
        const T* ivc = reinterpret_cast<const T*>(in.v_col);
        T* ocol = reinterpret_cast<T*>(out.col);
        T* omc = reinterpret_cast<T*>(out.m_col);
        T* ovc = reinterpret_cast<T*>(out.v_col);
        for (int q = threadIdx.x; q < nr * CV; q += kDensThreads) {
            const int j = q / CV, f = q - j * CV;
            const int no = s_nout[j];
            if (no == 0) continue;
            const long long d = s_dst[j];
            const size_t src = (size_t)(r0 + j) * CV + f;
            const T cv = icol[src];
            if (no == 1) {
                if (d < cap) {
                    ocol[(size_t)d * CV + f] = cv;
                    omc[(size_t)d * CV + f] = imc[src];
                    ovc[(size_t)d * CV + f] = ivc[src];
                }
            } else {
                for (int c = 0; c < 8; ++c) {
                    const size_t o = (size_t)(d + c) * CV + f;
                    ocol[o] = cv;
                    omc[o] = zero;
                    ovc[o] = zero;
                }
            }
        }
        slot += otot;
        crank += ctot;
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_grad_accum3d(const float* g2d, const uint32_t* count, int64_t n, float* accum, uint32_t* vis,
                                cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
    k_grad_accum3d<<<blocks, 256, 0, st>>>(reinterpret_cast<const float4*>(g2d), count, n, accum, vis);
    count_launches();
    return cudaGetLastError();
}

size_t densify_work_bytes(int64_t n) {
    const int64_t blocks = std::max<int64_t>(1, ceil_div(n, kDensTile));
    return (size_t)blocks * 8 + 256 + (size_t)blocks * 16 + 256 + 16;
}

cudaError_t launch_densify(const float* const in_p[3], const float* const in_m[3], const float* const in_v[3],
                           const float* accum, const uint32_t* vis, int64_t n, int C, int param_mode, float op_min,
                           float tau_g, float scale_min, int64_t capacity, float* const out_p[3],
                           float* const out_m[3], float* const out_v[3], int64_t* d_count, void* work,
                           cudaStream_t st) {
    const int64_t blocks = std::max<int64_t>(1, ceil_div(n, kDensTile));
    char* w = static_cast<char*>(work);
    auto* blk = reinterpret_cast<uint2*>(w);
    auto* base = reinterpret_cast<unsigned long long*>(w + ((size_t)blocks * 8 + 255) / 256 * 256);
    auto* meta = reinterpret_cast<long long*>(reinterpret_cast<char*>(base) + ((size_t)blocks * 16 + 255) / 256 * 256);
    DensIn in{reinterpret_cast<const float4*>(in_p[0]), in_p[1], in_p[2], reinterpret_cast<const float4*>(in_m[0]),
              in_m[1], in_m[2], reinterpret_cast<const float4*>(in_v[0]), in_v[1], in_v[2], accum, vis};
    DensOut out{reinterpret_cast<float4*>(out_p[0]), out_p[1], out_p[2], reinterpret_cast<float4*>(out_m[0]),
                out_m[1], out_m[2], reinterpret_cast<float4*>(out_v[0]), out_v[1], out_v[2]};
    DensParams P{n, capacity, C, param_mode, op_min, tau_g, scale_min};
    if (n > 0) {
        k_dens_count<<<(unsigned)blocks, kDensThreads, 0, st>>>(in, P, blk);
        count_launches();
    } else {
        cudaError_t e = cudaMemsetAsync(blk, 0, 8, st);
        if (e != cudaSuccess) return e;
    }
    k_dens_scan<<<1, kDensScanThreads, 0, st>>>(blk, blocks, P, base, meta, d_count);
    count_launches();
    if (n > 0) {
        switch (C) {  // colour floats per Gaussian: a compile-time row length for the cooperative copies
            case 3: k_dens_write<3><<<(unsigned)blocks, kDensThreads, 0, st>>>(in, out, P, base, meta); break;
            case 12: k_dens_write<12><<<(unsigned)blocks, kDensThreads, 0, st>>>(in, out, P, base, meta); break;
            case 27: k_dens_write<27><<<(unsigned)blocks, kDensThreads, 0, st>>>(in, out, P, base, meta); break;
            case 48: k_dens_write<48><<<(unsigned)blocks, kDensThreads, 0, st>>>(in, out, P, base, meta); break;
            default: return cudaErrorInvalidValue;
        }
        count_launches();
    }
    return cudaGetLastError();
}

}  // namespace igs
