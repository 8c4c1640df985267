// Projection of isotropic Gaussians to screen-space discs (with the
// activation of log sigma and the opacity logit fused in) and its adjoint.
//
// Eq. 7 with Sigma = sigma^2 I projects to a disc; the on-axis radius
// s = fx sigma / z_c depends only on the depth (Sec. 2.4). The support radius
// r = 3.33 s bounds the tiles a Gaussian can touch (compact support, Eq. 2).
// The key path (cull decisions, depth bits, tile rectangle) uses explicitly
// rounded FP32 operations in a fixed order so that it is bit-reproducible.
#include "common.cuh"

namespace igs {
namespace {

// Real orthonormal spherical harmonics without Condon-Shortley phase, written
// as polynomials of the unit direction (x, y, z); index k = l^2 + l + m.
// Constants: sqrt(2) K_lm times the leading factor of d^m P_l / dz^m, with
// K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
constexpr float kSh0 = 0.28209479177387814f;
constexpr float kSh1 = 0.4886025119029199f;
constexpr float kSh2a = 1.0925484305920792f;   // xy, yz, xz
constexpr float kSh2b = 0.31539156525252005f;  // (3z^2 - 1)
constexpr float kSh2c = 0.5462742152960396f;   // (x^2 - y^2)
constexpr float kSh3a = 0.5900435899266435f;   // (3x^2 y - y^3), (x^3 - 3 x y^2)
constexpr float kSh3b = 2.890611442640554f;    // xyz
constexpr float kSh3c = 0.4570457994644658f;   // y (5z^2 - 1), x (5z^2 - 1)
constexpr float kSh3d = 0.3731763325901154f;   // (5z^3 - 3z)
constexpr float kSh3e = 1.445305721320277f;    // z (x^2 - y^2)

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float Y[16]) {
    Y[0] = kSh0;
    if (deg < 1) return;
    Y[1] = kSh1 * y;
    Y[2] = kSh1 * z;
    Y[3] = kSh1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kSh2a * x * y;
    Y[5] = kSh2a * y * z;
    Y[6] = kSh2b * (3.f * zz - 1.f);
    Y[7] = kSh2a * x * z;
    Y[8] = kSh2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = kSh3a * y * (3.f * xx - yy);
    Y[10] = kSh3b * x * y * z;
    Y[11] = kSh3c * y * (5.f * zz - 1.f);
    Y[12] = kSh3d * z * (5.f * zz - 3.f);
    Y[13] = kSh3c * x * (5.f * zz - 1.f);
    Y[14] = kSh3e * z * (xx - yy);
    Y[15] = kSh3a * x * (xx - 3.f * yy);
}

// Gradient of the polynomial extension of each basis function.
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float G[16][3]) {
    G[0][0] = G[0][1] = G[0][2] = 0.f;
    if (deg < 1) return;
    G[1][0] = 0.f;   G[1][1] = kSh1; G[1][2] = 0.f;
    G[2][0] = 0.f;   G[2][1] = 0.f;  G[2][2] = kSh1;
    G[3][0] = kSh1;  G[3][1] = 0.f;  G[3][2] = 0.f;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    G[4][0] = kSh2a * y;        G[4][1] = kSh2a * x;         G[4][2] = 0.f;
    G[5][0] = 0.f;              G[5][1] = kSh2a * z;         G[5][2] = kSh2a * y;
    G[6][0] = 0.f;              G[6][1] = 0.f;               G[6][2] = kSh2b * 6.f * z;
    G[7][0] = kSh2a * z;        G[7][1] = 0.f;               G[7][2] = kSh2a * x;
    G[8][0] = kSh2c * 2.f * x;  G[8][1] = -kSh2c * 2.f * y;  G[8][2] = 0.f;
    if (deg < 3) return;
    G[9][0] = kSh3a * 6.f * x * y;        G[9][1] = kSh3a * 3.f * (xx - yy);   G[9][2] = 0.f;
    G[10][0] = kSh3b * y * z;             G[10][1] = kSh3b * x * z;            G[10][2] = kSh3b * x * y;
    G[11][0] = 0.f;                       G[11][1] = kSh3c * (5.f * zz - 1.f); G[11][2] = kSh3c * 10.f * y * z;
    G[12][0] = 0.f;                       G[12][1] = 0.f;                      G[12][2] = kSh3d * (15.f * zz - 3.f);
    G[13][0] = kSh3c * (5.f * zz - 1.f);  G[13][1] = 0.f;                      G[13][2] = kSh3c * 10.f * x * z;
    G[14][0] = kSh3e * 2.f * x * z;       G[14][1] = -kSh3e * 2.f * y * z;     G[14][2] = kSh3e * (xx - yy);
    G[15][0] = kSh3a * 3.f * (xx - yy);   G[15][1] = -kSh3a * 6.f * x * y;    G[15][2] = 0.f;
}

// Gradient of basis function k alone (k is a compile-time constant after unrolling).
__device__ __forceinline__ void sh_grad_one(int k, float x, float y, float z, float& gx, float& gy, float& gz) {
    const float xx = x * x, yy = y * y, zz = z * z;
    switch (k) {
        case 1: gx = 0.f; gy = kSh1; gz = 0.f; break;
        case 2: gx = 0.f; gy = 0.f; gz = kSh1; break;
        case 3: gx = kSh1; gy = 0.f; gz = 0.f; break;
        case 4: gx = kSh2a * y; gy = kSh2a * x; gz = 0.f; break;
        case 5: gx = 0.f; gy = kSh2a * z; gz = kSh2a * y; break;
        case 6: gx = 0.f; gy = 0.f; gz = kSh2b * 6.f * z; break;
        case 7: gx = kSh2a * z; gy = 0.f; gz = kSh2a * x; break;
        case 8: gx = kSh2c * 2.f * x; gy = -kSh2c * 2.f * y; gz = 0.f; break;
        case 9: gx = kSh3a * 6.f * x * y; gy = kSh3a * 3.f * (xx - yy); gz = 0.f; break;
        case 10: gx = kSh3b * y * z; gy = kSh3b * x * z; gz = kSh3b * x * y; break;
        case 11: gx = 0.f; gy = kSh3c * (5.f * zz - 1.f); gz = kSh3c * 10.f * y * z; break;
        case 12: gx = 0.f; gy = 0.f; gz = kSh3d * (15.f * zz - 3.f); break;
        case 13: gx = kSh3c * (5.f * zz - 1.f); gy = 0.f; gz = kSh3c * 10.f * x * z; break;
        case 14: gx = kSh3e * 2.f * x * z; gy = -kSh3e * 2.f * y * z; gz = kSh3e * (xx - yy); break;
        case 15: gx = kSh3a * 3.f * (xx - yy); gy = -kSh3a * 6.f * x * y; gz = 0.f; break;
        default: gx = gy = gz = 0.f; break;
    }
}

__device__ __forceinline__ bool finite4(float a, float b, float c, float d) {
    return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d);
}

// Camera-space position in the canonical order ((R0 x + R1 y) + R2 z) + t0,
// every operation rounded once.
__device__ __forceinline__ float cam_row(const float* R, float t, float x, float y, float z) {
    return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(R[0], x), __fmul_rn(R[1], y)), __fmul_rn(R[2], z)), t);
}

__device__ __forceinline__ void activate(int mode, float raw_sigma, float raw_op, float& sg, float& o) {
    if (mode == 1) {
        sg = expf(raw_sigma);
        o = 1.f / (1.f + expf(-raw_op));
    } else {
        sg = raw_sigma;
        o = raw_op;
    }
}

template <int DEG>
__device__ __forceinline__ void load_color(const float* __restrict__ col, int64_t i, float c[48]) {
    constexpr int C = DEG < 0 ? 3 : 3 * (DEG + 1) * (DEG + 1);
    const float* p = col + (size_t)C * (size_t)i;
    if constexpr (C % 4 == 0) {
        const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
            float4 v = __ldg(p4 + q);
            c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < C; ++q) c[q] = __ldg(p + q);
    }
}

template <int DEG>
__global__ void __launch_bounds__(256) k_project(const float4* __restrict__ ms, const float* __restrict__ op,
                                                 const float* __restrict__ col, int64_t n, ViewParams P,
                                                 float4* __restrict__ rec, uint2* __restrict__ rect,
                                                 uint32_t* __restrict__ count, uint32_t* __restrict__ depth_key) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 m = __ldg(ms + i);
    float sg, o;
    activate(P.param_mode, m.w, __ldg(op + i), sg, o);
    bool keep = finite4(m.x, m.y, m.z, sg) && isfinite(o);
    float xc = 0.f, yc = 0.f, zc = 0.f;
    if (keep) {
        xc = cam_row(P.R + 0, P.t[0], m.x, m.y, m.z);
        yc = cam_row(P.R + 3, P.t[1], m.x, m.y, m.z);
        zc = cam_row(P.R + 6, P.t[2], m.x, m.y, m.z);
        keep = (zc > P.znear) && (sg > 0.f) && (o >= 1.0f / 255.0f);
    }
    float s = 0.f, u = 0.f, v = 0.f;
    int x0 = 0, y0 = 0, x1 = -1, y1 = -1;
    if (keep) {
        s = __fdiv_rn(__fmul_rn(P.fx, sg), zc);
        u = __fadd_rn(__fdiv_rn(__fmul_rn(P.fx, xc), zc), P.cx);
        v = __fadd_rn(__fdiv_rn(__fmul_rn(P.fy, yc), zc), P.cy);
        const float r = __fmul_rn(kRadiusK, s);
        keep = isfinite(u) && isfinite(v) && isfinite(r);
        if (keep) {
            const float ts = (float)P.tile;
            const float fx0 = floorf(__fdiv_rn(__fsub_rn(u, r), ts));
            const float fx1 = floorf(__fdiv_rn(__fadd_rn(u, r), ts));
            const float fy0 = floorf(__fdiv_rn(__fsub_rn(v, r), ts));
            const float fy1 = floorf(__fdiv_rn(__fadd_rn(v, r), ts));
            keep = !(fx1 < 0.f || fx0 > (float)(P.tiles_x - 1) || fy1 < 0.f || fy0 > (float)(P.tiles_y - 1));
            if (keep) {
                x0 = (int)fmaxf(fx0, 0.f);
                y0 = (int)fmaxf(fy0, 0.f);
                x1 = (int)fminf(fx1, (float)(P.tiles_x - 1));
                y1 = (int)fminf(fy1, (float)(P.tiles_y - 1));
            }
        }
    }
    if (!keep) {
        count[i] = 0;
        depth_key[i] = 0xFFFFFFFFu;
        rect[i] = make_uint2(0u, 0u);
        rec[2 * i] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec[2 * i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    count[i] = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
    depth_key[i] = __float_as_uint(zc);
    rect[i] = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
    // colour
    float c[48];
    load_color<DEG>(col, i, c);
    float rgb[3];
    if constexpr (DEG < 0) {
        rgb[0] = c[0]; rgb[1] = c[1]; rgb[2] = c[2];
    } else {
        float dx = m.x - P.cam_center[0], dy = m.y - P.cam_center[1], dz = m.z - P.cam_center[2];
        const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv; dy *= inv; dz *= inv;
        float Y[16];
        sh_basis(DEG, dx, dy, dz, Y);
        constexpr int K = (DEG + 1) * (DEG + 1);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc = fmaf(c[3 * k + ch], Y[k], acc);
            rgb[ch] = fmaxf(acc + 0.5f, 0.f);
        }
    }
    const float w2 = 0.5f * kLog2e / (s * s);
    rec[2 * i] = make_float4(u, v, w2, o);
    rec[2 * i + 1] = make_float4(rgb[0], rgb[1], rgb[2], s);
}

// Colour rows of a warp's 32 Gaussians are staged in shared memory so that
// global reads and writes of the (3 (deg+1)^2)-float rows are coalesced float4
// accesses; the row stride (in float4) is odd, so lane-strided float4 reads of
// one row per lane hit distinct banks.
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

constexpr int kPbThreads = 128;

__device__ __forceinline__ void adam_update(float& p, float g, float& m, float& v, const AdamParams& a) {
    m = a.b1 * m + a.omb1 * g;
    v = a.b2 * v + a.omb2 * g * g;
    p -= a.step_size * m / (sqrtf(v) / a.bc2_sqrt + a.eps);
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

// Adjoint of the projection and colour: g2d holds (du, dv, dw2, do, dr, dg, db, -)
// per Gaussian, accumulated by the backward blend. ADAM = false writes the
// gradients w.r.t. the stored parameters to d_ms / d_op / d_col; ADAM = true
// applies one Adam step to the parameters in place (ms / op / col) instead,
// without materialising the gradient.
template <int DEG, bool ADAM>
__global__ void __launch_bounds__(kPbThreads, 6) k_project_bwd(float4* __restrict__ ms, float* __restrict__ op,
                                                            float* __restrict__ col, int64_t n, ViewParams P,
                                                            const uint32_t* __restrict__ count,
                                                            const float4* __restrict__ g2d, float4* __restrict__ d_ms,
                                                            float* __restrict__ d_op, float* __restrict__ d_col,
                                                            AdamState st, AdamParams ap) {
    constexpr int C = DEG < 0 ? 3 : 3 * (DEG + 1) * (DEG + 1);
    using CT = ColorTile<C>;
    extern __shared__ float4 s_tiles[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t wb = ((int64_t)blockIdx.x * (kPbThreads / 32) + w) * 32;
    if (wb >= n) return;  // whole warp past the end (no block-wide barrier below)
    const int nv = (int)min((int64_t)32, n - wb);
    const int64_t i = wb + lane;
    const bool active = lane < nv;
    float4* A = s_tiles + (size_t)w * CT::kWarpFloat4;           // this warp's parameter rows
    float* Ys = reinterpret_cast<float*>(A + 32 * CT::kStride);  // this warp's basis rows
    float* Af = reinterpret_cast<float*>(A) + lane * CT::kStride * 4;
    if constexpr (CT::kStaged) {
        const float4* src = reinterpret_cast<const float4*>(col) + wb * CT::kF4;
        for (int q = lane; q < nv * CT::kF4; q += 32) {
            const int g = q / CT::kF4;
            A[g * CT::kStride + (q - g * CT::kF4)] = src[q];
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
    if (active) {
        m = ms[i];
        raw_op = op[i];
        has_grad = count[i] != 0;
    }
    if (has_grad) {
        float sg, o;
        activate(P.param_mode, m.w, raw_op, sg, o);
        const float4 ga = __ldg(g2d + 2 * i), gb = __ldg(g2d + 2 * i + 1);
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
    if (active) {
        const float4 g4 = make_float4(dmx, dmy, dmz, dsig_out);
        if constexpr (ADAM) {
            float4 mm = st.m_ms[i], vv = st.v_ms[i];
            adam_update4(m, g4, mm, vv, ap);
            ms[i] = m; st.m_ms[i] = mm; st.v_ms[i] = vv;
            float mo = st.m_op[i], vo = st.v_op[i];
            adam_update(raw_op, dop_out, mo, vo, ap);
            op[i] = raw_op; st.m_op[i] = mo; st.v_op[i] = vo;
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
        __syncwarp();
        const size_t row0 = (size_t)wb * CT::kF4;
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
                float4 mm = reinterpret_cast<float4*>(st.m_col)[row0 + q];
                float4 vv = reinterpret_cast<float4*>(st.v_col)[row0 + q];
                adam_update4(p4, g4, mm, vv, ap);
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
                adam_update(pk, gk, mk, vk, ap);
                col[r + k] = pk; st.m_col[r + k] = mk; st.v_col[r + k] = vk;
            } else {
                d_col[r + k] = gk;
            }
        }
    }
}

template <int DEG, bool ADAM>
cudaError_t launch_pb(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, const float* g2d, float* d_ms,
                      float* d_op, float* d_col, const AdamState& st, const AdamParams& ap, cudaStream_t stream) {
    constexpr int C = DEG < 0 ? 3 : 3 * (DEG + 1) * (DEG + 1);
    const size_t smem = (size_t)(kPbThreads / 32) * ColorTile<C>::kWarpFloat4 * sizeof(float4);
    auto k = k_project_bwd<DEG, ADAM>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (unsigned)ceil_div(sc.n, kPbThreads);
    k<<<blocks, kPbThreads, smem, stream>>>(const_cast<float4*>(reinterpret_cast<const float4*>(sc.means_sigma)),
                                            const_cast<float*>(sc.opacity), const_cast<float*>(sc.color), sc.n, vp,
                                            f.count, reinterpret_cast<const float4*>(g2d),
                                            reinterpret_cast<float4*>(d_ms), d_op, d_col, st, ap);
    count_launches();
    return cudaGetLastError();
}

template <bool ADAM>
cudaError_t dispatch_pb(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, const float* g2d, float* d_ms,
                        float* d_op, float* d_col, const AdamState& st, const AdamParams& ap, cudaStream_t stream) {
    switch (vp.sh_degree) {
        case -1: return launch_pb<-1, ADAM>(sc, vp, f, g2d, d_ms, d_op, d_col, st, ap, stream);
        case 0: return launch_pb<0, ADAM>(sc, vp, f, g2d, d_ms, d_op, d_col, st, ap, stream);
        case 1: return launch_pb<1, ADAM>(sc, vp, f, g2d, d_ms, d_op, d_col, st, ap, stream);
        case 2: return launch_pb<2, ADAM>(sc, vp, f, g2d, d_ms, d_op, d_col, st, ap, stream);
        case 3: return launch_pb<3, ADAM>(sc, vp, f, g2d, d_ms, d_op, d_col, st, ap, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_project(const igs_scene& sc, const ViewParams& vp, const igs_frame& f, cudaStream_t st) {
    if (sc.n == 0) return cudaSuccess;
    const int threads = 256;
    const unsigned blocks = (unsigned)ceil_div(sc.n, threads);
    auto ms = reinterpret_cast<const float4*>(sc.means_sigma);
    auto rec = reinterpret_cast<float4*>(f.rec);
    auto rect = reinterpret_cast<uint2*>(f.rect);
#define IGS_PROJ(D) k_project<D><<<blocks, threads, 0, st>>>(ms, sc.opacity, sc.color, sc.n, vp, rec, rect, f.count, f.depth_key)
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
                                    const AdamParams& ap, cudaStream_t st) {
    if (sc.n == 0) return cudaSuccess;
    AdamState s{reinterpret_cast<float4*>(m_ms), m_op, m_col, reinterpret_cast<float4*>(v_ms), v_op, v_col};
    return dispatch_pb<true>(sc, vp, f, g2d, nullptr, nullptr, nullptr, s, ap, st);
}

}  // namespace igs
