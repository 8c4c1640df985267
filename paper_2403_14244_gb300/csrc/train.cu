// Training-step kernels: the L1 part of the loss of Sec. 3 and the Adam update
// of the back-propagation optimiser of Sec. 3.2.
#include <algorithm>

#include "common.cuh"

namespace igs {
namespace {

// loss += sum |img - target| / count (loss zeroed beforehand); grad = sign / count.
// VEC: 16-byte aligned arrays and count a multiple of 4, read and written as float4.
__device__ __forceinline__ float l1_term(float a, float b, float inv_count, float& acc) {
    const float d = a - b;
    acc += fabsf(d);
    return d > 0.f ? inv_count : (d < 0.f ? -inv_count : 0.f);
}
template <bool VEC>
__global__ void __launch_bounds__(256) k_l1(const float* __restrict__ img, const float* __restrict__ target,
                                            int64_t count, float inv_count, float* __restrict__ loss,
                                            float* __restrict__ grad) {
    pdl_wait();
    __shared__ float s_w[8];
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if constexpr (VEC) {
        const float4* a4 = reinterpret_cast<const float4*>(img);
        const float4* b4 = reinterpret_cast<const float4*>(target);
        float4* g4 = reinterpret_cast<float4*>(grad);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count / 4; i += stride) {
            const float4 a = a4[i], b = b4[i];
            float4 g;
            g.x = l1_term(a.x, b.x, inv_count, acc);
            g.y = l1_term(a.y, b.y, inv_count, acc);
            g.z = l1_term(a.z, b.z, inv_count, acc);
            g.w = l1_term(a.w, b.w, inv_count, acc);
            g4[i] = g;
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
            grad[i] = l1_term(img[i], target[i], inv_count, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_w[k];
        atomicAdd(loss, t * inv_count);
    }
}

// torch.optim.Adam's update order: m, v, then p -= step_size m / (sqrt(v) / sqrt(bc2) + eps).
__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, const AdamParams& a) {
    m = a.b1 * m + a.omb1 * g;
    v = a.b2 * v + a.omb2 * g * g;
    const float denom = sqrtf(v) / a.bc2_sqrt + a.eps;
    p -= a.step_size * m / denom;
}

// Vectorised body over count/4 float4 groups plus a scalar tail.
__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                              float* __restrict__ v, int64_t count, AdamParams a) {
    const int64_t n4 = count / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float4* p4 = reinterpret_cast<float4*>(p);
    const float4* g4 = reinterpret_cast<const float4*>(g);
    float4* m4 = reinterpret_cast<float4*>(m);
    float4* v4 = reinterpret_cast<float4*>(v);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 pp = p4[i], gg = g4[i], mm = m4[i], vv = v4[i];
        adam1(pp.x, gg.x, mm.x, vv.x, a);
        adam1(pp.y, gg.y, mm.y, vv.y, a);
        adam1(pp.z, gg.z, mm.z, vv.z, a);
        adam1(pp.w, gg.w, mm.w, vv.w, a);
        p4[i] = pp; m4[i] = mm; v4[i] = vv;
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        adam1(p[i], g[i], m[i], v[i], a);
}

__global__ void k_adam_scalar(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                              float* __restrict__ v, int64_t count, AdamParams a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        adam1(p[i], g[i], m[i], v[i], a);
}

// Range blockIdx.y of z, as 16-byte stores with a 4-byte tail.
__global__ void __launch_bounds__(256) k_zero(ZeroRanges z) {
    pdl_wait();
    const int r = blockIdx.y;
    if (r >= z.count) return;
    char* p = static_cast<char*>(z.ptr[r]);
    const unsigned long long n16 = z.bytes[r] / 16;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n16;
         i += (unsigned long long)gridDim.x * blockDim.x)
        reinterpret_cast<float4*>(p)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const unsigned long long tail = (z.bytes[r] - 16 * n16) / 4;
    if (blockIdx.x == 0 && threadIdx.x < tail) reinterpret_cast<float*>(p + 16 * n16)[threadIdx.x] = 0.f;
}

}  // namespace

cudaError_t launch_zero(const ZeroRanges& z, cudaStream_t st) {
    if (z.count <= 0) return cudaSuccess;
    unsigned long long most = 0;
    for (int r = 0; r < z.count; ++r) most = std::max(most, z.bytes[r]);
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)(most / 16), 256), 152 * 8));
    cudaError_t e = launch_pdl(k_zero, dim3(gx, (unsigned)z.count), dim3(256), 0, st, z);
    count_launches();
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_l1(const float* img, const float* target, int64_t count, float* loss, float* grad,
                      cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess || count == 0) return e;
    const bool vec = count % 4 == 0 && ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(target) |
                                         reinterpret_cast<uintptr_t>(grad)) & 15) == 0;
    const int blocks = (int)std::min<int64_t>(ceil_div(vec ? count / 4 : count, 256), 152 * 8);
    if (vec)
        k_l1<true><<<blocks, 256, 0, st>>>(img, target, count, 1.f / (float)count, loss, grad);
    else
        k_l1<false><<<blocks, 256, 0, st>>>(img, target, count, 1.f / (float)count, loss, grad);
    count_launches();
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t count, const AdamParams& a,
                        cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const bool aligned = ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(g) |
                           reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
    const int blocks = (int)std::min<int64_t>(ceil_div(count, 1024), 152 * 16);
    if (aligned)
        k_adam<<<blocks, 256, 0, st>>>(p, g, m, v, count, a);
    else
        k_adam_scalar<<<blocks, 256, 0, st>>>(p, g, m, v, count, a);
    count_launches();
    return cudaGetLastError();
}

}  // namespace igs
