// Projection of isotropic Gaussians to screen-space discs (with the
// activation of log sigma and the opacity logit fused in) and its adjoint; the
// per-Gaussian math is in projection.cuh.
#include "projection.cuh"

namespace igs {
namespace {

template <int DEG>
__global__ void __launch_bounds__(256) k_project(const float4* __restrict__ ms, const float* __restrict__ op,
                                                 const float* __restrict__ col, int64_t n, ViewParams P,
                                                 float4* __restrict__ rec, uint2* __restrict__ rect,
                                                 float4* __restrict__ disc, uint32_t* __restrict__ count,
                                                 uint32_t* __restrict__ depth_key) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    project_one<DEG>(ms, op, col, i, P, rec + 2 * i, rect + i, disc + i, count + i, depth_key + i);
}

// Projection with one warp per CTA and the warp's 32 colour rows (SH degree 3)
// staged in shared memory by coalesced 16-byte asynchronous copies (odd row
// stride: conflict-free row reads), instead of 32 rows read lane by lane.
constexpr int kProjRowStride = 13;  // float4 per staged row (12 used)

__global__ void __launch_bounds__(32) k_project_rows3(const float4* __restrict__ ms, const float* __restrict__ op,
                                                      const float* __restrict__ col, int64_t n, ViewParams P,
                                                      float4* __restrict__ rec, uint2* __restrict__ rect,
                                                      float4* __restrict__ disc, uint32_t* __restrict__ count,
                                                      uint32_t* __restrict__ depth_key) {
    pdl_wait();
    __shared__ float4 s_rows[32 * kProjRowStride];
    const int lane = threadIdx.x;
    const int64_t wb = (int64_t)blockIdx.x * 32;
    const int nv = (int)min((int64_t)32, n - wb);
    const float4* src = reinterpret_cast<const float4*>(col) + wb * 12;
    for (int q = lane; q < nv * 12; q += 32) {
        const int g = q / 12;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&s_rows[g * kProjRowStride + (q - g * 12)])),
                     "l"(src + q)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    if (lane >= nv) return;
    const int64_t i = wb + lane;
    const float4* row = s_rows + lane * kProjRowStride;
    project_one_with<3>(ms, op, [&](float c[48]) {
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float4 v = row[q];
            c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
        }
    }, i, P, rec + 2 * i, rect + i, disc + i, count + i, depth_key + i);
}

// Colour rows of a warp's 32 Gaussians are staged in shared memory (16-byte
// asynchronous copies) so that global reads and writes of the (3 (deg+1)^2)-float
// rows are coalesced float4 accesses; the row stride (in float4) is odd, so
// lane-strided float4 reads of one row per lane hit distinct banks. With Adam
// fused, the rows' moments m, v are staged the same way (dense) and stream in
// while the warp computes the gradient.
// The gradient of coefficient (k, ch) is Y_k * drgb_ch, so instead of staging 3K
// gradients per Gaussian the warp stages the K basis values and the 3 masked
// colour gradients (one row of kYStride floats per Gaussian).
template <int C>
struct ColorTile {
    static constexpr bool kStaged = (C % 4) == 0;
    static constexpr int kF4 = C / 4;
    static constexpr int kStride = kStaged ? ((kF4 % 2 == 1) ? kF4 : kF4 + 1) : 1;  // float4 units
    static constexpr int kYStride = C / 3 + 4;                                      // K basis values + 3 (+ pad)
    static constexpr int kWarpFloat4 = 32 * kStride + (32 * kYStride + 3) / 4;     // params, then basis rows
};

// One warp per CTA: a CTA's shared memory (21.5 KB with the Adam moments staged)
// is released as soon as its 32 Gaussians are done, so the ten resident warps
// of an SM run out of phase and keep HBM busy while others compute.
constexpr int kPbThreads = 32;

// 16-byte asynchronous global -> shared copy (completed by cp_async_wait).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Adam on one parameter (the fused kernel's hot loop: 53 updates per Gaussian);
// the bias correction is a multiplication, the square root the SFU's
// approximation (sqrt.approx, a few ulp) and the step a fast division (2 ulp).
__device__ __forceinline__ void adam_update(float& p, float g, float& m, float& v, const AdamParams& a) {
    m = a.b1 * m + a.omb1 * g;
    v = a.b2 * v + a.omb2 * g * g;
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    p -= __fdividef(a.step_size * m, fmaf(r, a.inv_bc2_sqrt, a.eps));
}
__device__ __forceinline__ void adam_update4(float4& p, float4 g, float4& m, float4& v, const AdamParams& a) {
    adam_update(p.x, g.x, m.x, v.x, a);
    adam_update(p.y, g.y, m.y, v.y, a);
    adam_update(p.z, g.z, m.z, v.z, a);
    adam_update(p.w, g.w, m.w, v.w, a);
}

struct AdamState {
    float4* m_ms; float* m_op; float* m_col;
    float4* v_ms; float* v_op; float* v_col;
};

// Where the projection of the next view goes (a frame's per-Gaussian arrays).
struct ProjOut {
    float4* rec; uint2* rect; float4* disc; uint32_t* count; uint32_t* depth_key;
};

// Adjoint of the projection and colour: g2d holds (du, dv, dw2, do, dr, dg, db, -)
// per Gaussian, accumulated by the backward blend. ADAM = false writes the
// gradients w.r.t. the stored parameters to d_ms / d_op / d_col; ADAM = true
// applies one Adam step to the parameters in place (ms / op / col) instead,
// without materialising the gradient. NEXT (with ADAM): each Gaussian is then
// projected for the next view (P2, into o2) from its updated parameters, still
// in registers and shared memory, so the next step needs no projection pass of
// its own. o2 may be the frame of this view: each thread reads its Gaussian's
// count before it writes the next view's.
template <int DEG, bool ADAM, bool NEXT = false>
__global__ void __launch_bounds__(kPbThreads, 10) k_project_bwd(float4* __restrict__ ms, float* __restrict__ op,
                                                            float* __restrict__ col, int64_t n, ViewParams P,
                                                            const uint32_t* count,
                                                            const float4* __restrict__ g2d, float4* __restrict__ d_ms,
                                                            float* __restrict__ d_op, float* __restrict__ d_col,
                                                            AdamState st, AdamParams ap, ViewParams P2, ProjOut o2) {
    pdl_wait();
    constexpr int C = DEG < 0 ? 3 : 3 * (DEG + 1) * (DEG + 1);
    using CT = ColorTile<C>;
    extern __shared__ float4 s_tiles[];
    AdamParams a = ap;
    if (ADAM && ap.dev_consts) {  // this step's constants from the device step count
        a.step_size = __ldg(ap.dev_consts);
        a.inv_bc2_sqrt = __ldg(ap.dev_consts + 1);
        a.bc2_sqrt = __ldg(ap.dev_consts + 2);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t wb = ((int64_t)blockIdx.x * (kPbThreads / 32) + w) * 32;
    if (wb >= n) return;  // whole warp past the end (no block-wide barrier below)
    const int nv = (int)min((int64_t)32, n - wb);
    const int64_t i = wb + lane;
    const bool active = lane < nv;
    constexpr int kWarpF4 = CT::kWarpFloat4 + (ADAM && CT::kStaged ? 2 * 32 * CT::kF4 : 0);
    float4* A = s_tiles + (size_t)w * kWarpF4;                   // this warp's parameter rows
    float* Ys = reinterpret_cast<float*>(A + 32 * CT::kStride);  // this warp's basis rows
    float* Af = reinterpret_cast<float*>(A) + lane * CT::kStride * 4;
    float4* Mrows = A + CT::kWarpFloat4;                         // Adam moments of the colour rows (dense)
    float4* Vrows = Mrows + 32 * CT::kF4;
    if constexpr (CT::kStaged) {
        const float4* src = reinterpret_cast<const float4*>(col) + wb * CT::kF4;
        for (int q = lane; q < nv * CT::kF4; q += 32) {
            const int g = q / CT::kF4;
            cp_async16(&A[g * CT::kStride + (q - g * CT::kF4)], src + q);
        }
        cp_async_commit();
        if constexpr (ADAM) {  // the colour moments stream in while the gradient is computed
            const float4* m4 = reinterpret_cast<const float4*>(st.m_col) + wb * CT::kF4;
            const float4* v4 = reinterpret_cast<const float4*>(st.v_col) + wb * CT::kF4;
            for (int q = lane; q < nv * CT::kF4; q += 32) {
                cp_async16(&Mrows[q], m4 + q);
                cp_async16(&Vrows[q], v4 + q);
            }
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
    }
    float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
    float raw_op = 0.f;
    float dmx = 0.f, dmy = 0.f, dmz = 0.f, dsig_out = 0.f, dop_out = 0.f;
    // colour coefficients of this lane's Gaussian (staged rows, or its own strided row)
    auto coef = [&](int k) -> float { return CT::kStaged ? Af[k] : col[(size_t)C * (size_t)i + k]; };
    bool has_grad = false;
    float drgb[3] = {0.f, 0.f, 0.f}, draw[3] = {0.f, 0.f, 0.f};
    float Y[16];
    float dx = 0.f, dy = 0.f, dz = 0.f;
    float4 e_mm = make_float4(0.f, 0.f, 0.f, 0.f), e_vv = e_mm;
    float e_mo = 0.f, e_vo = 0.f;
    float4 ga = e_mm, gb = e_mm;
    if (active) {
        m = ms[i];
        raw_op = op[i];
        // the screen-space gradient with the other loads, not after the count that decides
        // whether it is used: one memory round trip on the warp's path instead of two
        ga = __ldg(g2d + 2 * i);
        gb = __ldg(g2d + 2 * i + 1);
        has_grad = count[i] != 0;
        if constexpr (ADAM) {  // independent of the gradient: in flight during the compute
            e_mm = st.m_ms[i];
            e_vv = st.v_ms[i];
            e_mo = st.m_op[i];
            e_vo = st.v_op[i];
        }
    }
    if (has_grad) {
        float sg, o;
        activate(P.param_mode, m.w, raw_op, sg, o);
        const float xc = P.R[0] * m.x + P.R[1] * m.y + P.R[2] * m.z + P.t[0];
        const float yc = P.R[3] * m.x + P.R[4] * m.y + P.R[5] * m.z + P.t[1];
        const float zc = P.R[6] * m.x + P.R[7] * m.y + P.R[8] * m.z + P.t[2];
        const float iz = 1.f / zc;
        const float s = P.fx * sg * iz;
        const float w2 = 0.5f * kLog2e / (s * s);
        const float ds = ga.z * (-2.f * w2 / s);  // w2 = log2(e) / (2 s^2)
        const float dxc = ga.x * P.fx * iz;
        const float dyc = ga.y * P.fy * iz;
        const float dzc = -(ga.x * P.fx * xc + ga.y * P.fy * yc + ds * P.fx * sg) * iz * iz;
        dmx = P.R[0] * dxc + P.R[3] * dyc + P.R[6] * dzc;
        dmy = P.R[1] * dxc + P.R[4] * dyc + P.R[7] * dzc;
        dmz = P.R[2] * dxc + P.R[5] * dyc + P.R[8] * dzc;
        const float dsg = ds * P.fx * iz;
        dsig_out = P.param_mode == 1 ? dsg * sg : dsg;
        dop_out = P.param_mode == 1 ? ga.w * o * (1.f - o) : ga.w;
        drgb[0] = gb.x; drgb[1] = gb.y; drgb[2] = gb.z;
        if constexpr (DEG >= 0) {
            dx = m.x - P.cam_center[0]; dy = m.y - P.cam_center[1]; dz = m.z - P.cam_center[2];
            const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= inv; dy *= inv; dz *= inv;
            sh_basis(DEG, dx, dy, dz, Y);
            constexpr int K = (DEG + 1) * (DEG + 1);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < K; ++k) acc = fmaf(coef(3 * k + ch), Y[k], acc);
                draw[ch] = (acc + 0.5f > 0.f) ? drgb[ch] : 0.f;  // rgb = max(0, raw + 0.5)
            }
            float gd0 = 0.f, gd1 = 0.f, gd2 = 0.f;
#pragma unroll
            for (int k = 1; k < K; ++k) {
                const float wk = draw[0] * coef(3 * k) + draw[1] * coef(3 * k + 1) + draw[2] * coef(3 * k + 2);
                float gx, gy, gz;
                sh_grad_one(k, dx, dy, dz, gx, gy, gz);
                gd0 = fmaf(wk, gx, gd0);
                gd1 = fmaf(wk, gy, gd1);
                gd2 = fmaf(wk, gz, gd2);
            }
            const float dot = gd0 * dx + gd1 * dy + gd2 * dz;
            dmx += (gd0 - dot * dx) * inv;
            dmy += (gd1 - dot * dy) * inv;
            dmz += (gd2 - dot * dz) * inv;
        }
    }
    // gradient of colour coefficient k (zero for culled Gaussians)
    auto dcoef = [&](int k) -> float {
        if constexpr (DEG < 0) return drgb[k];
        else return Y[k / 3] * draw[k % 3];
    };
    // means, sigma, opacity: one lane per Gaussian (coalesced rows of 16 and 4 bytes)
    ProjGeom pg{};
    if (active) {
        const float4 g4 = make_float4(dmx, dmy, dmz, dsig_out);
        if constexpr (ADAM) {
            float4 mm = e_mm, vv = e_vv;
            adam_update4(m, g4, mm, vv, a);
            ms[i] = m; st.m_ms[i] = mm; st.v_ms[i] = vv;
            float mo = e_mo, vo = e_vo;
            adam_update(raw_op, dop_out, mo, vo, a);
            op[i] = raw_op; st.m_op[i] = mo; st.v_op[i] = vo;
            // the next view's geometry while the colour moments are still in flight
            if constexpr (NEXT) pg = project_geom(m, raw_op, P2, o2.rec + 2 * i, o2.rect + i, o2.disc + i,
                                                  o2.count + i, o2.depth_key + i);
        } else {
            d_ms[i] = g4;
            d_op[i] = dop_out;
        }
    }
    // colour rows
    if constexpr (CT::kStaged) {
        constexpr int K = C / 3;
        if (active) {
            float* yr = Ys + lane * CT::kYStride;
#pragma unroll
            for (int k = 0; k < K; ++k) yr[k] = has_grad ? Y[k] : 0.f;
            yr[K] = draw[0]; yr[K + 1] = draw[1]; yr[K + 2] = draw[2];
        }
        if constexpr (ADAM) cp_async_wait<0>();
        __syncwarp();
        const size_t row0 = (size_t)wb * CT::kF4;
#pragma unroll 6
        for (int q = lane; q < nv * CT::kF4; q += 32) {
            const int g = q / CT::kF4;
            const int c0 = 4 * (q - g * CT::kF4);  // first coefficient of this float4
            const float* yr = Ys + g * CT::kYStride;
            float4 g4;
            g4.x = yr[(c0 + 0) / 3] * yr[K + (c0 + 0) % 3];
            g4.y = yr[(c0 + 1) / 3] * yr[K + (c0 + 1) % 3];
            g4.z = yr[(c0 + 2) / 3] * yr[K + (c0 + 2) % 3];
            g4.w = yr[(c0 + 3) / 3] * yr[K + (c0 + 3) % 3];
            if constexpr (ADAM) {
                float4 p4 = A[g * CT::kStride + (q - g * CT::kF4)];
                float4 mm = Mrows[q];
                float4 vv = Vrows[q];
                adam_update4(p4, g4, mm, vv, a);
                if constexpr (NEXT) A[g * CT::kStride + (q - g * CT::kF4)] = p4;  // for the next view's colour
                reinterpret_cast<float4*>(col)[row0 + q] = p4;
                reinterpret_cast<float4*>(st.m_col)[row0 + q] = mm;
                reinterpret_cast<float4*>(st.v_col)[row0 + q] = vv;
            } else {
                reinterpret_cast<float4*>(d_col)[row0 + q] = g4;
            }
        }
    } else if (active) {
        const size_t r = (size_t)C * (size_t)i;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const float gk = has_grad ? dcoef(k) : 0.f;
            if constexpr (ADAM) {
                float pk = col[r + k], mk = st.m_col[r + k], vk = st.v_col[r + k];
                adam_update(pk, gk, mk, vk, a);
                col[r + k] = pk; st.m_col[r + k] = mk; st.v_col[r + k] = vk;
            } else {
                d_col[r + k] = gk;
            }
        }
    }
    if constexpr (NEXT) {  // the next view's colour from the updated coefficients
        static_assert(ADAM, "the next view is projected from the updated parameters");
        if constexpr (CT::kStaged) __syncwarp();  // the staged rows hold the updated coefficients
        if (active && pg.keep) {
            float c[48];
            if constexpr (CT::kStaged) {
                const float4* row = A + lane * CT::kStride;  // odd float4 stride: conflict-free
#pragma unroll
                for (int q = 0; q < CT::kF4; ++q) {
                    const float4 t = row[q];
                    c[4 * q] = t.x; c[4 * q + 1] = t.y; c[4 * q + 2] = t.z; c[4 * q + 3] = t.w;
                }
            } else {
#pragma unroll
                for (int k = 0; k < C; ++k) c[k] = col[(size_t)C * (size_t)i + k];  // this thread's own writes
            }
            project_color<DEG>(m, pg, c, P2, o2.rec + 2 * i);
        }
    }
}

template <int DEG, bool ADAM, bool NEXT = false>
cudaError_t launch_pb(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, const float* g2d, float* d_ms,
                      float* d_op, float* d_col, const AdamState& st, const AdamParams& ap, cudaStream_t stream,
                      const ViewParams& vp2 = ViewParams{}, const ProjOut& o2 = ProjOut{}) {
    constexpr int C = DEG < 0 ? 3 : 3 * (DEG + 1) * (DEG + 1);
    const size_t smem = (size_t)(kPbThreads / 32) *
                        (ColorTile<C>::kWarpFloat4 + (ADAM && ColorTile<C>::kStaged ? 2 * 32 * ColorTile<C>::kF4 : 0)) *
                        sizeof(float4);
    auto k = k_project_bwd<DEG, ADAM, NEXT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (unsigned)ceil_div(sc.n, kPbThreads);
    cudaError_t e = launch_pdl(k, dim3(blocks), dim3(kPbThreads), smem, stream,
                               const_cast<float4*>(reinterpret_cast<const float4*>(sc.means_sigma)),
                               const_cast<float*>(sc.opacity), const_cast<float*>(sc.color), sc.n, vp, f.count,
                               reinterpret_cast<const float4*>(g2d), reinterpret_cast<float4*>(d_ms), d_op, d_col, st,
                               ap, vp2, o2);
    count_launches();
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <bool ADAM, bool NEXT = false>
cudaError_t dispatch_pb(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, const float* g2d, float* d_ms,
                        float* d_op, float* d_col, const AdamState& st, const AdamParams& ap, cudaStream_t stream,
                        const ViewParams& vp2 = ViewParams{}, const ProjOut& o2 = ProjOut{}) {
    switch (vp.sh_degree) {
        case -1: return launch_pb<-1, ADAM, NEXT>(sc, vp, f, g2d, d_ms, d_op, d_col, st, ap, stream, vp2, o2);
        case 0: return launch_pb<0, ADAM, NEXT>(sc, vp, f, g2d, d_ms, d_op, d_col, st, ap, stream, vp2, o2);
        case 1: return launch_pb<1, ADAM, NEXT>(sc, vp, f, g2d, d_ms, d_op, d_col, st, ap, stream, vp2, o2);
        case 2: return launch_pb<2, ADAM, NEXT>(sc, vp, f, g2d, d_ms, d_op, d_col, st, ap, stream, vp2, o2);
        case 3: return launch_pb<3, ADAM, NEXT>(sc, vp, f, g2d, d_ms, d_op, d_col, st, ap, stream, vp2, o2);
        default: return cudaErrorInvalidValue;
    }
}

__global__ void k_adam_advance(int32_t* __restrict__ state, double lr, double b1, double b2) {
    pdl_wait();
    const int t = state[0] + 1;
    state[0] = t;
    const double bc1 = 1.0 - pow(b1, (double)t), bc2 = 1.0 - pow(b2, (double)t);
    float* f = reinterpret_cast<float*>(state + 1);
    f[0] = (float)(lr / bc1);
    f[1] = (float)(1.0 / sqrt(bc2));
    f[2] = (float)sqrt(bc2);
}

}  // namespace

cudaError_t launch_adam_advance(int32_t* state, double lr, double b1, double b2, cudaStream_t st) {
    cudaError_t e = launch_pdl(k_adam_advance, dim3(1), dim3(1), 0, st, state, lr, b1, b2);
    count_launches();
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_project(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, cudaStream_t st) {
    if (sc.n == 0) return cudaSuccess;
    const int threads = 256;
    const unsigned blocks = (unsigned)ceil_div(sc.n, threads);
    auto ms = reinterpret_cast<const float4*>(sc.means_sigma);
    auto rec = reinterpret_cast<float4*>(f.rec);
    auto rect = reinterpret_cast<uint2*>(f.rect);
#define IGS_PROJ(D) k_project<D><<<blocks, threads, 0, st>>>(ms, sc.opacity, sc.color, sc.n, vp, rec, rect, reinterpret_cast<float4*>(f.disc), f.count, f.depth_key)
    if (vp.sh_degree == 3 && (reinterpret_cast<uintptr_t>(sc.color) & 15) == 0) {
        cudaError_t e = launch_pdl(k_project_rows3, dim3((unsigned)ceil_div(sc.n, 32)), dim3(32), 0, st, ms,
                                   sc.opacity, sc.color, sc.n, vp, rec, rect, reinterpret_cast<float4*>(f.disc),
                                   f.count, f.depth_key);
        count_launches();
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    switch (vp.sh_degree) {
        case -1: IGS_PROJ(-1); break;
        case 0: IGS_PROJ(0); break;
        case 1: IGS_PROJ(1); break;
        case 2: IGS_PROJ(2); break;
        case 3: IGS_PROJ(3); break;
        default: return cudaErrorInvalidValue;
    }
#undef IGS_PROJ
    count_launches();
    return cudaGetLastError();
}

cudaError_t launch_project_bwd(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, const float* g2d,
                               float* d_ms, float* d_op, float* d_col, cudaStream_t st) {
    if (sc.n == 0) return cudaSuccess;
    return dispatch_pb<false>(sc, vp, f, g2d, d_ms, d_op, d_col, AdamState{}, AdamParams{}, st);
}

cudaError_t launch_project_bwd_adam(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, const float* g2d,
                                    float* m_ms, float* m_op, float* m_col, float* v_ms, float* v_op, float* v_col,
                                    const AdamParams& ap, cudaStream_t st, const ViewParams* vp_next,
                                    const igs_frame* f_next) {
    if (sc.n == 0) return cudaSuccess;
    AdamState s{reinterpret_cast<float4*>(m_ms), m_op, m_col, reinterpret_cast<float4*>(v_ms), v_op, v_col};
    if (vp_next && f_next) {
        const ProjOut o2{reinterpret_cast<float4*>(f_next->rec), reinterpret_cast<uint2*>(f_next->rect),
                         reinterpret_cast<float4*>(f_next->disc), f_next->count, f_next->depth_key};
        return dispatch_pb<true, true>(sc, vp, f, g2d, nullptr, nullptr, nullptr, s, ap, st, *vp_next, o2);
    }
    return dispatch_pb<true>(sc, vp, f, g2d, nullptr, nullptr, nullptr, s, ap, st);
}

}  // namespace igs
