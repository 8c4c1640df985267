// Per-Gaussian projection math shared by the one-view kernels (project.cu)
// and the multi-view batch kernels (batch.cu). Internal to libigs.
//
// Eq. 7 with Sigma = sigma^2 I projects an isotropic Gaussian to a disc; the
// on-axis radius s = fx sigma / z_c depends only on the depth (Sec. 2.4). The
// support radius r (support_radius, from s and the opacity) bounds the tiles a
// Gaussian can touch (compact support, Eq. 2). The key path (cull decisions, depth bits, tile rectangle)
// uses explicitly rounded FP32 operations in a fixed order so that it is
// bit-reproducible.
#pragma once

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

// Projection of Gaussian i for one view: disc, culling, tile rectangle, depth
// key and colour (the per-Gaussian body shared by the one-view and batch kernels).
// Footprint radius (Eq. 2's support, per particle): an FP32 upper bound of
// s sqrt(2 (ln(255 o) + 2^-9)). x = 255 o = 2^e m with m in [1, 2); ln m =
// 2 (t + t^3/3 + t^5/5 + t^7/7 + ...), t = (m - 1)/(m + 1) < 1/3, cut after t^7
// with the coefficients and ln 2 rounded up; the 2^-9 of slack covers the cut
// (< 1.2e-5), the roundings and the blend's exponent slack (2^-10 ln 2). Every
// step is rounded once in a fixed order, so the rectangle is reproducible.
__device__ __forceinline__ float support_radius(float s, float o) {
    const float x = __fmul_rn(255.0f, o);
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xFFu) - 127;
    const float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    const float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float t2 = __fmul_rn(t, t);
    float p = 0.2857143f;
    p = __fadd_rn(0.4f, __fmul_rn(t2, p));
    p = __fadd_rn(0.6666667f, __fmul_rn(t2, p));
    p = __fadd_rn(2.0f, __fmul_rn(t2, p));
    float U = __fadd_rn(__fmul_rn((float)e, 0.6931472f), __fmul_rn(t, p));
    U = __fadd_rn(fmaxf(U, 0.0f), 0.001953125f);
    const float k = __fsqrt_rn(__fmul_rn(2.0f, U));
    return __fmul_rn(__fmul_rn(s, k), 1.000244140625f);
}

// The geometric half of a Gaussian's projection (culling, disc, tiles, depth),
// kept for its colour half.
struct ProjGeom {
    bool keep;
    float u, v, w2, pmax, o;
};

// Geometric half from the stored parameters m (mean, scale) and raw_op: writes
// count, depth key, rectangle (and disc), or the culled values with a zero
// record.
__device__ __forceinline__ ProjGeom project_geom(float4 m, float raw_op, const ViewParams& P,
                                                 float4* __restrict__ rec, uint2* __restrict__ rect,
                                                 float4* __restrict__ disc, uint32_t* __restrict__ count,
                                                 uint32_t* __restrict__ depth_key) {
    ProjGeom g;
    float sg, o;
    activate(P.param_mode, m.w, raw_op, sg, o);
    bool keep = finite4(m.x, m.y, m.z, sg) && isfinite(o);
    float xc = 0.f, yc = 0.f, zc = 0.f;
    if (keep) {
        xc = cam_row(P.R + 0, P.t[0], m.x, m.y, m.z);
        yc = cam_row(P.R + 3, P.t[1], m.x, m.y, m.z);
        zc = cam_row(P.R + 6, P.t[2], m.x, m.y, m.z);
        keep = (zc > P.znear) && (sg > 0.f) && (o >= 1.0f / 255.0f);
    }
    float s = 0.f, u = 0.f, v = 0.f, r = 0.f;
    int x0 = 0, y0 = 0, x1 = -1, y1 = -1;
    uint32_t touched = 0;
    if (keep) {
        s = __fdiv_rn(__fmul_rn(P.fx, sg), zc);
        u = __fadd_rn(__fdiv_rn(__fmul_rn(P.fx, xc), zc), P.cx);
        v = __fadd_rn(__fdiv_rn(__fmul_rn(P.fy, yc), zc), P.cy);
        r = support_radius(s, o);
        keep = isfinite(u) && isfinite(v) && isfinite(r);
        if (keep) {
            const float inv = 1.0f / (float)P.tile;  // exact: the tile size is a power of two
            const float fx0 = floorf(__fmul_rn(__fsub_rn(u, r), inv));
            const float fx1 = floorf(__fmul_rn(__fadd_rn(u, r), inv));
            const float fy0 = floorf(__fmul_rn(__fsub_rn(v, r), inv));
            const float fy1 = floorf(__fmul_rn(__fadd_rn(v, r), inv));
            keep = !(fx1 < 0.f || fx0 > (float)(P.tiles_x - 1) || fy1 < 0.f || fy0 > (float)(P.tiles_y - 1));
            if (keep) {
                x0 = (int)fmaxf(fx0, 0.f);
                y0 = (int)fmaxf(fy0, 0.f);
                x1 = (int)fminf(fx1, (float)(P.tiles_x - 1));
                y1 = (int)fminf(fy1, (float)(P.tiles_y - 1));
                if (P.footprint == 0) {
                    touched = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
                } else {  // the tiles the disc meets, row by row of its bounding rectangle
                    for (int ty = y0; ty <= y1; ++ty) {
                        const int2 sp = row_span(u, v, r, P.tile, inv, ty, x0, x1);
                        if (sp.y >= sp.x) touched += (uint32_t)(sp.y - sp.x + 1);
                    }
                }
                keep = touched > 0;
            }
        }
    }
    g.keep = keep;
    if (!keep) {
        *count = 0;
        *depth_key = 0xFFFFFFFFu;
        *rect = make_uint2(0u, 0u);
        if (P.footprint) *disc = make_float4(0.f, 0.f, 0.f, 0.f);
        rec[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        return g;
    }
    *count = touched;
    if (P.footprint) *disc = make_disc(u, v, r, x0, x1);  // read only by the per-row walks
    *depth_key = __float_as_uint(zc);
    *rect = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
    g.u = u;
    g.v = v;
    g.w2 = 0.5f * kLog2e / (s * s);
    // every pixel with w2 d^2 above pmax has alpha < alpha_min (skipped in Eq. 4)
    g.pmax = __fadd_rn(log2f(__fdiv_rn(o, P.alpha_min)), kPowMargin);
    g.o = o;
    return g;
}

// Colour half of a kept Gaussian's projection: its colour from the
// coefficients c[0 .. C) (SH evaluated toward the camera centre), and the record.
template <int DEG>
__device__ __forceinline__ void project_color(float4 m, const ProjGeom& g, const float* c, const ViewParams& P,
                                              float4* __restrict__ rec) {
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
    rec[0] = make_float4(g.u, g.v, g.w2, g.pmax);
    rec[1] = make_float4(rgb[0], rgb[1], rgb[2], g.o);
}

// The Gaussian's stored parameters are m (mean, scale) and raw_op; load_c(c)
// fills c[0 .. C) with its colour coefficients and is called only for
// Gaussians that are kept.
template <int DEG, typename LoadC>
__device__ __forceinline__ void project_one_vals(float4 m, float raw_op, LoadC load_c, const ViewParams& P,
                                                 float4* __restrict__ rec, uint2* __restrict__ rect,
                                                 float4* __restrict__ disc, uint32_t* __restrict__ count,
                                                 uint32_t* __restrict__ depth_key) {
    const ProjGeom g = project_geom(m, raw_op, P, rec, rect, disc, count, depth_key);
    if (!g.keep) return;
    float c[48];
    load_c(c);
    project_color<DEG>(m, g, c, P, rec);
}

template <int DEG, typename LoadC>
__device__ __forceinline__ void project_one_with(const float4* __restrict__ ms, const float* __restrict__ op,
                                                 LoadC load_c, int64_t i, const ViewParams& P,
                                                 float4* __restrict__ rec, uint2* __restrict__ rect,
                                                 float4* __restrict__ disc, uint32_t* __restrict__ count,
                                                 uint32_t* __restrict__ depth_key) {
    project_one_vals<DEG>(__ldg(ms + i), __ldg(op + i), load_c, P, rec, rect, disc, count, depth_key);
}

template <int DEG>
__device__ __forceinline__ void project_one(const float4* __restrict__ ms, const float* __restrict__ op,
                                            const float* __restrict__ col, int64_t i, const ViewParams& P,
                                            float4* __restrict__ rec, uint2* __restrict__ rect,
                                            float4* __restrict__ disc, uint32_t* __restrict__ count,
                                            uint32_t* __restrict__ depth_key) {
    project_one_with<DEG>(ms, op, [&](float c[48]) { load_color<DEG>(col, i, c); }, i, P, rec, rect, disc, count,
                          depth_key);
}

}  // namespace
}  // namespace igs
