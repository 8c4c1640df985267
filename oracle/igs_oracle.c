/*
 * CPU oracle for isotropic Gaussian splatting (arXiv 2403.14244).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no code, header, table or constant with the
 * CUDA path; the only thing the two sides share is the seeded input
 * generator, which holds none of the method's arithmetic.
 *
 * What it computes, and where the paper states it:
 *   - isotropic kernel g = exp(-|x - mu|^2 / (2 s^2))          Eq. 8 (reading: the
 *     paper writes sigma^2 in the denominator; with s = sigma/sqrt(2) the two agree)
 *   - projection of an isotropic Gaussian to a screen disc      Eq. 7 with Sigma = sigma^2 I,
 *     radius s = f sigma / z_c, "size only depends on the distance to the view
 *     point" (Sec. 2.4); centre u = fx x_c/z_c + cx, v = fy y_c/z_c + cy
 *   - front-to-back alpha compositing                           Eq. 4
 *     C = sum_k c_k a_k prod_{j<k} (1 - a_j), a_k = min(0.99, o_k g_k),
 *     entries with a_k < 1/255 skipped, stop before the entry that would take
 *     the transmittance below 1e-4, background added with the final T
 *   - compact support of each particle                           Eq. 2 (support D),
 *     read per particle: the footprint radius r bounds s sqrt(2 ln(255 o)) from
 *     above (plus a small slack), so o exp(-d^2/(2 s^2)) < 1/255 beyond it
 *   - gradients of the loss w.r.t. every particle parameter      Eq. 3 and the
 *     position gradient that follows it, by the chain rule through Eq. 4, Eq. 8
 *     and the projection
 *   - colour as real spherical harmonics up to degree 3 (the particle property
 *     A_k of Sec. 3, view dependent)
 *   - the training loss of Sec. 3, (1 - lambda) L1 + lambda (1 - SSIM), and its
 *     gradient w.r.t. the rendered image
 *   - the paper's 2D experiment (Sec. 3): the additive image model
 *     f^ = sum A_k g(x - mu_k, sigma_k) over particles within the support D,
 *     its gradient, and the QuadTree initialisation of Sec. 3.1
 *
 * Two arithmetics:
 *   - the key path (culling, tile rectangle, depth key) is canonical FP32 with
 *     every operation rounded once, in a fixed order (compile with
 *     -ffp-contract=off), so that keys and tile ranges can be compared bit for bit;
 *   - compositing and gradients are FP64. With proj64 = 0 the disc (u, v, s) is
 *     the canonical FP32 value widened to FP64; with proj64 = 1 it is computed in
 *     FP64 from the inputs (used for finite differences).
 *
 * Two traversal modes give bit-identical results, because each pixel sees the
 * same Gaussians in the same order with the same arithmetic:
 *   mode 0 "literal": every pixel walks every visible Gaussian, front to back;
 *   mode 1 "lists":   each image row walks only the Gaussians whose support
 *                     reaches the row, still front to back.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    float R[9];          /* world -> camera rotation, row-major */
    float t[3];          /* x_c = R x_w + t */
    float fx, fy, cx, cy;
    float znear;
    int32_t width, height;
} orc_camera;

typedef struct {
    float alpha_min;     /* 1/255 */
    float alpha_max;     /* 0.99 */
    float t_min;         /* 1e-4 */
    float bg[3];
    int32_t sh_degree;   /* -1: RGB, 0..3: SH */
    int32_t log_params;  /* 1: sigma column is log sigma, opacity is a logit */
    int32_t proj64;      /* 1: disc in FP64 from the inputs */
    int32_t mode;        /* 0 literal, 1 lists */
    double flag_margin;  /* relative margin for near-threshold decisions */
} orc_opts;

/* Footprint radius of a Gaussian of screen size s and opacity o (Eq. 2's
 * support, per particle): r >= s sqrt(2 (ln(255 o) + 2^-9)). With
 * x = 255 o = 2^e m, m in [1, 2): ln x = e ln 2 + ln m, and ln m =
 * 2 (t + t^3/3 + t^5/5 + ...) with t = (m - 1)/(m + 1) in [0, 1/3); the sum is
 * cut after t^7 (remainder < 1.2e-5) with its coefficients and ln 2 rounded up,
 * and 2^-9 of slack covers the remainder and the roundings. Every step is one
 * FP32 operation rounded once, in this order (no contraction). */
static float support_radius(float s, float o) {
    float x = 255.0f * o;
    uint32_t b;
    memcpy(&b, &x, 4);
    const int e = (int)((b >> 23) & 0xFFu) - 127;
    const uint32_t mb = (b & 0x007FFFFFu) | 0x3F800000u;
    float m;
    memcpy(&m, &mb, 4);
    const float t = (m - 1.0f) / (m + 1.0f);
    const float t2 = t * t;
    float p = 0.2857143f;
    p = 0.4f + t2 * p;
    p = 0.6666667f + t2 * p;
    p = 2.0f + t2 * p;
    const float a = (float)e * 0.6931472f;
    const float q = t * p;
    float U = a + q;
    U = fmaxf(U, 0.0f) + 0.001953125f;
    const float k = sqrtf(2.0f * U);
    const float r = s * k;
    return r * 1.000244140625f;
}

/* the radius for given (s, o) pairs (for the tests) */
void orc_radius(int64_t n, const float* s, const float* o, float* r) {
    for (int64_t i = 0; i < n; ++i) r[i] = support_radius(s[i], o[i]);
}

/* Tiles of tile row ty that the disc of radius r around (u, v) touches, within
 * [x0, x1]: [*xa, *xb] (empty when *xa > *xb). The row's band
 * [ty*tile, (ty+1)*tile) lies dy = max(0, ty*tile - v, v - (ty+1)*tile) from v,
 * where the disc spans u +- sqrt(r^2 - dy^2); a tile is touched when its column
 * meets that span. One rounding per step, in this order. */
static void row_span(float u, float v, float r, int tile, int ty, int x0, int x1, int* xa, int* xb) {
    const float ts = (float)tile;
    const float lo = (float)(ty * tile), hi = (float)((ty + 1) * tile);
    const float d1 = lo - v, d2 = v - hi;
    const float dy = fmaxf(0.0f, fmaxf(d1, d2));
    const float rr = r * r, dd = dy * dy;
    const float h2 = rr - dd;
    const float hw = sqrtf(fmaxf(h2, 0.0f));
    const float fa = floorf((u - hw) / ts), fb = floorf((u + hw) / ts);
    *xa = (int)fminf(fmaxf(fa, (float)x0), (float)(x1 + 1));
    *xb = (int)fmaxf(fminf(fb, (float)x1), (float)(x0 - 1));
}

/* Tiles touched over the rows of the rectangle. */
static int32_t span_count(float u, float v, float r, int tile, const int32_t rc[4]) {
    int32_t c = 0;
    for (int ty = rc[1]; ty <= rc[3]; ++ty) {
        int xa, xb;
        row_span(u, v, r, tile, ty, rc[0], rc[2], &xa, &xb);
        if (xb >= xa) c += xb - xa + 1;
    }
    return c;
}

/* spans of given rows (for the tests): per query (u, v, r, ty, x0, x1) -> (xa, xb) */
void orc_row_span(int64_t n, const float* u, const float* v, const float* r, const int32_t* ty,
                  const int32_t* x0, const int32_t* x1, int32_t tile, int32_t* xa, int32_t* xb) {
    for (int64_t i = 0; i < n; ++i) {
        int a, b;
        row_span(u[i], v[i], r[i], tile, ty[i], x0[i], x1[i], &a, &b);
        xa[i] = a;
        xb[i] = b;
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static uint32_t f32_bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* ------------------------------------------------------------ activation -- */
/* sigma = exp(log sigma), o = 1/(1+exp(-logit)); FP64, rounded once to FP32. */
void orc_activate(int64_t n, const float* log_sigma, int64_t ls_stride, const float* logit,
                  float* sigma_out, float* opac_out) {
    for (int64_t i = 0; i < n; ++i) {
        double l = (double)log_sigma[i * ls_stride];
        sigma_out[i] = (float)exp(l);
        opac_out[i] = (float)(1.0 / (1.0 + exp(-(double)logit[i])));
    }
}

/* ------------------------------------------------------ FP32 key path ----- */
/* Canonical FP32 projection of one Gaussian. Returns the tiles it touches (0 = culled).
 * Culled when: an input is not finite, sigma <= 0, z_c <= znear,
 * o < 1/255 (no pixel could reach the alpha cutoff), or its tiles miss the
 * grid. rect is the bounding rectangle of the disc's tiles; the Gaussian touches
 * every tile of it (footprint 0) or, in each row ty, the tiles of row_span
 * (footprint 1). */
static int key_path_one(const orc_camera* c, int tile, int tiles_x, int tiles_y, int footprint,
                        float mx, float my, float mz, float sg, float o,
                        float* pu, float* pv, float* ps, float* pz, float* pr, int32_t rect[4]) {
    if (!(isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(sg) && isfinite(o)))
        return 0;
    float xc = ((c->R[0] * mx + c->R[1] * my) + c->R[2] * mz) + c->t[0];
    float yc = ((c->R[3] * mx + c->R[4] * my) + c->R[5] * mz) + c->t[1];
    float zc = ((c->R[6] * mx + c->R[7] * my) + c->R[8] * mz) + c->t[2];
    if (!(zc > c->znear)) return 0;
    if (!(sg > 0.0f)) return 0;
    if (!(o >= 1.0f / 255.0f)) return 0;
    float s = (c->fx * sg) / zc;
    float u = (c->fx * xc) / zc + c->cx;
    float v = (c->fy * yc) / zc + c->cy;
    float r = support_radius(s, o);
    if (!(isfinite(u) && isfinite(v) && isfinite(r))) return 0;
    float ts = (float)tile;
    float fx0 = floorf((u - r) / ts), fx1 = floorf((u + r) / ts);
    float fy0 = floorf((v - r) / ts), fy1 = floorf((v + r) / ts);
    if (fx1 < 0.0f || fx0 > (float)(tiles_x - 1) || fy1 < 0.0f || fy0 > (float)(tiles_y - 1))
        return 0;
    rect[0] = (int32_t)fmaxf(fx0, 0.0f);
    rect[1] = (int32_t)fmaxf(fy0, 0.0f);
    rect[2] = (int32_t)fminf(fx1, (float)(tiles_x - 1));
    rect[3] = (int32_t)fminf(fy1, (float)(tiles_y - 1));
    const int32_t cnt = footprint ? span_count(u, v, r, tile, rect)
                                  : (rect[2] - rect[0] + 1) * (rect[3] - rect[1] + 1);
    if (cnt == 0) return 0;  /* the disc meets no tile of the grid */
    *pu = u; *pv = v; *ps = s; *pz = zc; *pr = r;
    return cnt;
}

/* Per-Gaussian canonical projection (linear sigma and opacity given in FP32).
 * rect = (x0, y0, x1, y1) inclusive tile bounds; count = tiles touched (0 if culled). */
void orc_project(int64_t n, const float* means_sigma, const float* opacity, const orc_camera* cam,
                 int32_t tile, int32_t footprint, float* u, float* v, float* s, float* depth, float* radius,
                 int32_t* rect, int32_t* count) {
    int tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
    for (int64_t i = 0; i < n; ++i) {
        const float* m = means_sigma + 4 * i;
        int32_t rc[4] = {0, 0, -1, -1};
        float uu = 0, vv = 0, ss = 0, zz = 0, rr = 0;
        int cnt = key_path_one(cam, tile, tiles_x, tiles_y, footprint, m[0], m[1], m[2], m[3], opacity[i],
                               &uu, &vv, &ss, &zz, &rr, rc);
        if (cnt == 0) { rc[0] = 0; rc[1] = 0; rc[2] = -1; rc[3] = -1; }
        u[i] = uu; v[i] = vv; s[i] = ss; depth[i] = zz; radius[i] = rr;
        memcpy(rect + 4 * i, rc, sizeof rc);
        count[i] = cnt;
    }
}

typedef struct { uint64_t key; int64_t pos; uint32_t val; } key_entry;

static int cmp_key_entry(const void* a, const void* b) {
    const key_entry* x = (const key_entry*)a;
    const key_entry* y = (const key_entry*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->pos < y->pos ? -1 : (x->pos > y->pos);  /* generation order: a stable sort */
}

/* Duplicate every kept Gaussian into one (key, value) pair per tile it touches
 * (its rectangle, or row_span of each row of it with footprint 1), key = (tile_base + ty*tiles_x + tx)
 * << 32 | bits(depth), generated in index order and row-major tile order; sort by key keeping generation order among
 * equal keys; record for every tile the half-open range [start, end) of its
 * entries ((0, 0) if it has none). Returns M. */
int64_t orc_keys(int64_t n, const int32_t* rect, const int32_t* count, const float* depth,
                 const float* u, const float* v, const float* radius, int32_t tile, int32_t footprint,
                 int32_t tiles_x, int32_t tiles_y, uint32_t tile_base,
                 uint64_t* keys_out, uint32_t* vals_out, uint32_t* ranges_out) {
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) m += count[i];
    key_entry* e = (key_entry*)malloc(sizeof(key_entry) * (size_t)(m > 0 ? m : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (count[i] == 0) continue;
        const int32_t* rc = rect + 4 * i;
        for (int32_t ty = rc[1]; ty <= rc[3]; ++ty) {
            int xa = rc[0], xb = rc[2];
            if (footprint) row_span(u[i], v[i], radius[i], tile, ty, rc[0], rc[2], &xa, &xb);
            for (int32_t tx = xa; tx <= xb; ++tx) {
                uint64_t tid = (uint64_t)tile_base + (uint64_t)ty * (uint64_t)tiles_x + (uint64_t)tx;
                e[k].key = (tid << 32) | (uint64_t)f32_bits(depth[i]);
                e[k].pos = k;
                e[k].val = (uint32_t)i;
                ++k;
            }
        }
    }
    qsort(e, (size_t)m, sizeof(key_entry), cmp_key_entry);
    int64_t tiles = (int64_t)tiles_x * tiles_y;
    if (ranges_out) memset(ranges_out, 0, sizeof(uint32_t) * 2 * (size_t)tiles);
    for (int64_t j = 0; j < m; ++j) {
        if (keys_out) keys_out[j] = e[j].key;
        if (vals_out) vals_out[j] = e[j].val;
        if (ranges_out) {
            int64_t t = (int64_t)(e[j].key >> 32) - (int64_t)tile_base;
            if (j == 0 || (e[j - 1].key >> 32) != (e[j].key >> 32)) ranges_out[2 * t] = (uint32_t)j;
            ranges_out[2 * t + 1] = (uint32_t)(j + 1);
        }
    }
    free(e);
    return m;
}

/* ---------------------------------------------- real spherical harmonics -- */
/* Real orthonormal SH on the unit sphere, without the Condon-Shortley phase:
 *   Y_l0  = K_l0 P_l(z)
 *   Y_lm  = sqrt(2) K_lm P_l^m(z) cos(m phi)        m > 0
 *   Y_l-m = sqrt(2) K_lm P_l^m(z) sin(m phi)        m > 0
 * with K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^m(z) = (1-z^2)^{m/2} d^m P_l/dz^m.
 * On the sphere (1-z^2)^{m/2} cos(m phi) = Re (x+iy)^m and ... sin = Im (x+iy)^m,
 * so Y is the polynomial K d^mP_l/dz^m(z) * {Re,Im}(x+iy)^m, evaluated and
 * differentiated below from the explicit expansion of P_l. Index k = l^2 + l + m. */
static double fact(int a) { double r = 1; for (int i = 2; i <= a; ++i) r *= i; return r; }
static double binom(int a, int b) { return fact(a) / (fact(b) * fact(a - b)); }

/* d^m/dz^m of P_l at z, from P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) z^(l-2k). */
static double legendre_deriv(int l, int m, double z) {
    double acc = 0.0;
    for (int k = 0; 2 * k <= l; ++k) {
        int p = l - 2 * k;
        if (p < m) continue;
        double coef = ((k & 1) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l) / pow(2.0, l);
        double falling = fact(p) / fact(p - m);
        acc += coef * falling * pow(z, p - m);
    }
    return acc;
}

/* (x+iy)^m as (re, im); m >= 0. */
static void cpow_xy(double x, double y, int m, double* re, double* im) {
    double a = 1.0, b = 0.0;
    for (int i = 0; i < m; ++i) { double na = a * x - b * y, nb = a * y + b * x; a = na; b = nb; }
    *re = a; *im = b;
}

/* Basis values Y[k] and gradients dY[k][3] of the polynomial extension at d. */
static void sh_basis(int deg, const double d[3], double* Y, double (*dY)[3]) {
    const double x = d[0], y = d[1], z = d[2];
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            int k = l * l + l + m;
            double K = sqrt((2 * l + 1) / (4.0 * M_PI) * fact(l - am) / fact(l + am));
            if (m != 0) K *= sqrt(2.0);
            double P = legendre_deriv(l, am, z);
            double P1 = legendre_deriv(l, am + 1, z);
            double re, im, re1 = 0, im1 = 0;
            cpow_xy(x, y, am, &re, &im);
            if (am > 0) cpow_xy(x, y, am - 1, &re1, &im1);
            double A, Ax, Ay;
            if (m >= 0) { A = re; Ax = am * re1; Ay = -am * im1; }
            else        { A = im; Ax = am * im1; Ay = am * re1; }
            if (m == 0) { A = 1.0; Ax = 0.0; Ay = 0.0; }
            Y[k] = K * P * A;
            if (dY) { dY[k][0] = K * P * Ax; dY[k][1] = K * P * Ay; dY[k][2] = K * P1 * A; }
        }
    }
}

void orc_sh_basis(int32_t deg, int64_t n, const double* dirs, double* Y, double* dY) {
    int K = (deg + 1) * (deg + 1);
    for (int64_t i = 0; i < n; ++i)
        sh_basis(deg, dirs + 3 * i, Y + (size_t)K * i, dY ? (double (*)[3])(dY + (size_t)3 * K * i) : NULL);
}

/* --------------------------------------------------- prepared Gaussians --- */
typedef struct {
    double u, v, s, o, sigma;
    double xc, yc, zc;
    double rgb[3], raw[3];
    double dir[3], dist;
    double reach;        /* distance beyond which a < alpha_min, with margin */
    uint32_t zbits;      /* FP32 depth bits (canonical order key) */
    int vis;
} orc_g;

static int ncoef(int deg) { return deg < 0 ? 3 : 3 * (deg + 1) * (deg + 1); }

static void prepare(int64_t n, const float* ms, const float* op, const float* color, const orc_camera* c,
                    const orc_opts* o, orc_g* g) {
    int C = ncoef(o->sh_degree);
    double R[9], t[3];
    for (int i = 0; i < 9; ++i) R[i] = c->R[i];
    for (int i = 0; i < 3; ++i) t[i] = c->t[i];
    /* camera centre -R^T t */
    double cc[3];
    for (int a = 0; a < 3; ++a) cc[a] = -(R[0 * 3 + a] * t[0] + R[1 * 3 + a] * t[1] + R[2 * 3 + a] * t[2]);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        orc_g* G = &g[i];
        memset(G, 0, sizeof *G);
        const float* m = ms + 4 * i;
        double sig_d, op_d;
        float sig_f, op_f;
        if (o->log_params) {
            sig_d = exp((double)m[3]);
            op_d = 1.0 / (1.0 + exp(-(double)op[i]));
            sig_f = (float)sig_d; op_f = (float)op_d;
        } else {
            sig_f = m[3]; op_f = op[i];
            sig_d = sig_f; op_d = op_f;
        }
        /* visibility: the FP32 decisions of the key path, without the tile test
         * (a Gaussian off the tile grid cannot reach alpha_min on any pixel). */
        if (!(isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2]) && isfinite(sig_f) && isfinite(op_f))) continue;
        float xf = ((c->R[0] * m[0] + c->R[1] * m[1]) + c->R[2] * m[2]) + c->t[0];
        float yf = ((c->R[3] * m[0] + c->R[4] * m[1]) + c->R[5] * m[2]) + c->t[1];
        float zf = ((c->R[6] * m[0] + c->R[7] * m[1]) + c->R[8] * m[2]) + c->t[2];
        if (!(zf > c->znear) || !(sig_f > 0.0f) || !(op_f >= 1.0f / 255.0f)) continue;
        float sf = (c->fx * sig_f) / zf;
        float uf = (c->fx * xf) / zf + c->cx;
        float vf = (c->fy * yf) / zf + c->cy;
        if (!(isfinite(uf) && isfinite(vf) && isfinite(sf))) continue;
        G->vis = 1;
        G->zbits = f32_bits(zf);
        double mx = m[0], my = m[1], mz = m[2];
        G->xc = R[0] * mx + R[1] * my + R[2] * mz + t[0];
        G->yc = R[3] * mx + R[4] * my + R[5] * mz + t[1];
        G->zc = R[6] * mx + R[7] * my + R[8] * mz + t[2];
        G->sigma = sig_d;
        if (o->proj64) {
            G->s = (double)c->fx * sig_d / G->zc;
            G->u = (double)c->fx * G->xc / G->zc + (double)c->cx;
            G->v = (double)c->fy * G->yc / G->zc + (double)c->cy;
            G->o = op_d;
        } else {
            G->s = sf; G->u = uf; G->v = vf; G->o = op_f;
        }
        /* distance beyond which o g < alpha_min (1 - margin): nothing there can be
         * blended or flagged, so the lists mode may skip it (same result as literal) */
        double am = (double)o->alpha_min * (1.0 - o->flag_margin);
        G->reach = (G->o > am) ? G->s * sqrt(2.0 * log(G->o / am)) * (1.0 + 1e-6) + 1e-9 : 0.0;
        /* colour */
        const float* col = color + (size_t)C * i;
        double dv[3] = {mx - cc[0], my - cc[1], mz - cc[2]};
        double dist = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        G->dist = dist;
        for (int a = 0; a < 3; ++a) G->dir[a] = dv[a] / dist;
        if (o->sh_degree < 0) {
            for (int ch = 0; ch < 3; ++ch) { G->rgb[ch] = col[ch]; G->raw[ch] = col[ch]; }
        } else {
            double Y[16];
            sh_basis(o->sh_degree, G->dir, Y, NULL);
            int K = (o->sh_degree + 1) * (o->sh_degree + 1);
            for (int ch = 0; ch < 3; ++ch) {
                double acc = 0.0;
                for (int k = 0; k < K; ++k) acc += (double)col[3 * k + ch] * Y[k];
                G->raw[ch] = acc + 0.5;
                G->rgb[ch] = G->raw[ch] > 0.0 ? G->raw[ch] : 0.0;
            }
        }
    }
}

typedef struct { uint32_t zb; int64_t id; double z; } ord_entry;
static int cmp_ord32(const void* a, const void* b) {
    const ord_entry* x = (const ord_entry*)a; const ord_entry* y = (const ord_entry*)b;
    if (x->zb != y->zb) return x->zb < y->zb ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}
static int cmp_ord64(const void* a, const void* b) {
    const ord_entry* x = (const ord_entry*)a; const ord_entry* y = (const ord_entry*)b;
    if (x->z != y->z) return x->z < y->z ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}

/* Front-to-back order of the visible Gaussians: ascending depth (the FP32
 * depth bits on the canonical path, the FP64 depth with proj64), ties by index. */
static int64_t depth_order(int64_t n, const orc_g* g, int proj64, int64_t* order) {
    ord_entry* e = (ord_entry*)malloc(sizeof(ord_entry) * (size_t)(n > 0 ? n : 1));
    int64_t nv = 0;
    for (int64_t i = 0; i < n; ++i)
        if (g[i].vis) { e[nv].zb = g[i].zbits; e[nv].id = i; e[nv].z = g[i].zc; ++nv; }
    qsort(e, (size_t)nv, sizeof(ord_entry), proj64 ? cmp_ord64 : cmp_ord32);
    for (int64_t k = 0; k < nv; ++k) order[k] = e[k].id;
    free(e);
    return nv;
}

/* --------------------------------------------------------- compositing ---- */
typedef struct { int64_t id; double a, gval, T; int clamped; } blend_rec;

typedef struct {
    double C[3], T;
    int32_t nb;
    int64_t last;
    int alive, flag;
    uint64_t hash;
    blend_rec* rec; int64_t nrec, cap;   /* blended entries, only when recording */
} pix_state;

static void pix_init(pix_state* p) {
    p->C[0] = p->C[1] = p->C[2] = 0.0; p->T = 1.0; p->nb = 0; p->last = -1;
    p->alive = 1; p->flag = 0; p->hash = 1469598103934665603ull; p->nrec = 0;
}

static void hash_mix(uint64_t* h, uint64_t v) {
    for (int b = 0; b < 8; ++b) { *h ^= (v >> (8 * b)) & 0xff; *h *= 1099511628211ull; }
}

/* One front-to-back step of Eq. 4 for pixel centre (px, py). */
static void composite_step(pix_state* p, const orc_g* G, int64_t id, double px, double py,
                           const orc_opts* o, int record) {
    double dx = px - G->u, dy = py - G->v;
    double d2 = dx * dx + dy * dy;
    double gval = exp(-d2 / (2.0 * G->s * G->s));
    double og = G->o * gval;
    int clamped = og > (double)o->alpha_max;
    double a = clamped ? (double)o->alpha_max : og;
    double amin = (double)o->alpha_min, tmin = (double)o->t_min, mg = o->flag_margin;
    if (fabs(a - amin) <= mg * amin) p->flag = 1;
    if (a < amin) return;
    double Tn = p->T * (1.0 - a);
    if (fabs(Tn - tmin) <= mg * tmin) p->flag = 1;
    if (Tn < tmin) { p->alive = 0; hash_mix(&p->hash, (uint64_t)id ^ 0x8000000000000000ull); return; }
    for (int ch = 0; ch < 3; ++ch) p->C[ch] += G->rgb[ch] * a * p->T;
    if (record) {
        if (p->nrec == p->cap) {
            p->cap = p->cap ? 2 * p->cap : 16;
            p->rec = (blend_rec*)realloc(p->rec, sizeof(blend_rec) * (size_t)p->cap);
        }
        blend_rec* r = &p->rec[p->nrec++];
        r->id = id; r->a = a; r->gval = gval; r->T = p->T; r->clamped = clamped;
    }
    p->T = Tn;
    p->nb += 1;
    p->last = id;
    hash_mix(&p->hash, (uint64_t)id * 2u + (uint64_t)clamped);
}

/* 2D gradient accumulators per Gaussian: du, dv, ds, do, dr, dg, db. */
static void atomic_add(double* x, double v) {
#pragma omp atomic
    *x += v;
}

/* Reverse walk of one pixel (adjoint of Eq. 4). dC/da_k = T_k c_k - S_k/(1-a_k)
 * where S_k is everything composited behind entry k, background included. */
static void pixel_backward(const pix_state* p, const orc_g* g, double px, double py, const double G3[3],
                           const orc_opts* o, double* g2d) {
    double S[3];
    for (int ch = 0; ch < 3; ++ch) S[ch] = p->T * (double)o->bg[ch];
    for (int64_t k = p->nrec - 1; k >= 0; --k) {
        const blend_rec* r = &p->rec[k];
        const orc_g* G = &g[r->id];
        double* acc = g2d + 7 * r->id;
        double da = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            atomic_add(&acc[4 + ch], r->a * r->T * G3[ch]);
            da += G3[ch] * (r->T * G->rgb[ch] - S[ch] / (1.0 - r->a));
            S[ch] += r->a * r->T * G->rgb[ch];
        }
        if (r->clamped) continue;
        double d_o = da * r->gval;
        double dgv = da * G->o;
        double s2 = G->s * G->s;
        double dx = px - G->u, dy = py - G->v;
        atomic_add(&acc[0], dgv * r->gval * dx / s2);
        atomic_add(&acc[1], dgv * r->gval * dy / s2);
        atomic_add(&acc[2], dgv * r->gval * (dx * dx + dy * dy) / (s2 * G->s));
        atomic_add(&acc[3], d_o);
    }
}

static void write_pixel(const pix_state* p, int64_t pix, int64_t P, const orc_opts* o,
                        double* img, double* T, int32_t* nb, int32_t* last, uint8_t* flag, uint64_t* hash) {
    for (int ch = 0; ch < 3; ++ch) img[ch * P + pix] = p->C[ch] + p->T * (double)o->bg[ch];
    if (T) T[pix] = p->T;
    if (nb) nb[pix] = p->nb;
    if (last) last[pix] = (int32_t)p->last;
    if (flag) flag[pix] = (uint8_t)p->flag;
    if (hash) hash[pix] = p->hash;
}

/* Core renderer. dL_dimg != NULL additionally runs the adjoint into g2d [n][7]. */
static void render_core(int64_t n, const orc_g* g, const int64_t* order, int64_t nv, const orc_camera* c,
                        const orc_opts* o, double* img, double* T, int32_t* nb, int32_t* last,
                        uint8_t* flag, uint64_t* hash, const double* dL, double* g2d) {
    const int W = c->width, H = c->height;
    const int64_t P = (int64_t)W * H;
    const int record = dL != NULL;
    if (o->mode == 0) {
#pragma omp parallel
        {
            pix_state ps; memset(&ps, 0, sizeof ps);
#pragma omp for schedule(dynamic, 16)
            for (int64_t pix = 0; pix < P; ++pix) {
                double px = (double)(pix % W) + 0.5, py = (double)(pix / W) + 0.5;
                pix_init(&ps);
                for (int64_t k = 0; k < nv && ps.alive; ++k)
                    composite_step(&ps, &g[order[k]], order[k], px, py, o, record);
                write_pixel(&ps, pix, P, o, img, T, nb, last, flag, hash);
                if (record) {
                    double G3[3] = {dL[pix], dL[P + pix], dL[2 * P + pix]};
                    pixel_backward(&ps, g, px, py, G3, o, g2d);
                }
            }
            free(ps.rec);
        }
        return;
    }
    /* lists mode: bucket the Gaussians by the rows their support reaches, in depth order */
    int64_t* rcount = (int64_t*)calloc((size_t)H + 1, sizeof(int64_t));
    int32_t* r0 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    int32_t* r1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    for (int64_t k = 0; k < nv; ++k) {
        const orc_g* G = &g[order[k]];
        double lo = ceil(G->v - G->reach - 0.5), hi = floor(G->v + G->reach - 0.5);
        if (lo < 0) lo = 0;
        if (hi > H - 1) hi = H - 1;
        if (!(G->reach > 0.0) || lo > hi) { r0[k] = 1; r1[k] = 0; continue; }
        r0[k] = (int32_t)lo; r1[k] = (int32_t)hi;
        for (int32_t y = r0[k]; y <= r1[k]; ++y) rcount[y + 1]++;
    }
    for (int y = 0; y < H; ++y) rcount[y + 1] += rcount[y];
    int64_t total = rcount[H];
    int64_t* bucket = (int64_t*)malloc(sizeof(int64_t) * (size_t)(total > 0 ? total : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)H);
    for (int y = 0; y < H; ++y) fill[y] = rcount[y];
    for (int64_t k = 0; k < nv; ++k)
        for (int32_t y = r0[k]; y <= r1[k]; ++y) bucket[fill[y]++] = order[k];
    free(fill); free(r0); free(r1);
#pragma omp parallel
    {
        pix_state* row = (pix_state*)calloc((size_t)W, sizeof(pix_state));
#pragma omp for schedule(dynamic, 1)
        for (int y = 0; y < H; ++y) {
            double py = (double)y + 0.5;
            for (int x = 0; x < W; ++x) pix_init(&row[x]);
            int alive = W;
            for (int64_t b = rcount[y]; b < rcount[y + 1] && alive > 0; ++b) {
                int64_t id = bucket[b];
                const orc_g* G = &g[id];
                double dy = py - G->v;
                double w2 = G->reach * G->reach - dy * dy;
                if (w2 < 0) continue;
                double w = sqrt(w2);
                double lo = ceil(G->u - w - 0.5), hi = floor(G->u + w - 0.5);
                if (lo < 0) lo = 0;
                if (hi > W - 1) hi = W - 1;
                for (int x = (int)lo; x <= (int)hi; ++x) {
                    if (!row[x].alive) continue;
                    composite_step(&row[x], G, id, (double)x + 0.5, py, o, record);
                    if (!row[x].alive) --alive;
                }
            }
            for (int x = 0; x < W; ++x) {
                int64_t pix = (int64_t)y * W + x;
                write_pixel(&row[x], pix, P, o, img, T, nb, last, flag, hash);
                if (record) {
                    double G3[3] = {dL[pix], dL[P + pix], dL[2 * P + pix]};
                    pixel_backward(&row[x], g, (double)x + 0.5, py, G3, o, g2d);
                }
            }
        }
        for (int x = 0; x < W; ++x) free(row[x].rec);
        free(row);
    }
    free(bucket); free(rcount);
}

/* Forward render. img [3][H][W], T [H][W], nb (entries blended), last (index of
 * the last blended Gaussian or -1), flag (a cutoff/stop decision within the
 * relative margin), hash (digest of the decision sequence). Any output may be NULL
 * except img. Returns the number of visible Gaussians. */
int64_t orc_render(int64_t n, const float* means_sigma, const float* opacity, const float* color,
                   const orc_camera* cam, const orc_opts* o, double* img, double* T, int32_t* nb,
                   int32_t* last, uint8_t* flag, uint64_t* hash) {
    orc_g* g = (orc_g*)malloc(sizeof(orc_g) * (size_t)(n > 0 ? n : 1));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    prepare(n, means_sigma, opacity, color, cam, o, g);
    int64_t nv = depth_order(n, g, o->proj64, order);
    render_core(n, g, order, nv, cam, o, img, T, nb, last, flag, hash, NULL, NULL);
    free(g); free(order);
    return nv;
}

/* Chain rule from the screen-space disc to the parameters of one Gaussian. */
static void chain_one(const orc_g* G, const double* acc, const float* ms, const float* col,
                      const orc_camera* c, const orc_opts* o,
                      double* dmean, double* dsig, double* dop, double* dcol) {
    int C = ncoef(o->sh_degree);
    double fx = c->fx, fy = c->fy;
    double du = acc[0], dv = acc[1], ds = acc[2], d_o = acc[3];
    double zc = G->zc, xc = G->xc, yc = G->yc;
    double dxc = du * fx / zc;
    double dyc = dv * fy / zc;
    double dzc = -du * fx * xc / (zc * zc) - dv * fy * yc / (zc * zc) - ds * fx * G->sigma / (zc * zc);
    for (int a = 0; a < 3; ++a)
        dmean[a] = c->R[0 * 3 + a] * dxc + c->R[1 * 3 + a] * dyc + c->R[2 * 3 + a] * dzc;
    double dsigma = ds * fx / zc;
    *dsig = o->log_params ? dsigma * G->sigma : dsigma;
    *dop = o->log_params ? d_o * G->o * (1.0 - G->o) : d_o;
    if (o->sh_degree < 0) {
        for (int ch = 0; ch < 3; ++ch) dcol[ch] = acc[4 + ch];
        return;
    }
    int K = (o->sh_degree + 1) * (o->sh_degree + 1);
    double Y[16], dY[16][3];
    sh_basis(o->sh_degree, G->dir, Y, dY);
    double draw[3];
    for (int ch = 0; ch < 3; ++ch) draw[ch] = G->raw[ch] > 0.0 ? acc[4 + ch] : 0.0;
    for (int k = 0; k < K; ++k)
        for (int ch = 0; ch < 3; ++ch) dcol[3 * k + ch] = Y[k] * draw[ch];
    double ddir[3] = {0, 0, 0};
    for (int k = 0; k < K; ++k)
        for (int ch = 0; ch < 3; ++ch) {
            double w = draw[ch] * (double)col[3 * k + ch];
            for (int a = 0; a < 3; ++a) ddir[a] += w * dY[k][a];
        }
    double dot = ddir[0] * G->dir[0] + ddir[1] * G->dir[1] + ddir[2] * G->dir[2];
    for (int a = 0; a < 3; ++a) dmean[a] += (ddir[a] - dot * G->dir[a]) / G->dist;
    (void)ms; (void)C;
}

/* Forward + adjoint. dL_dimg [3][H][W]. Outputs: d_means [n][3], d_sigma [n]
 * (w.r.t. sigma, or log sigma), d_opac [n] (opacity, or logit), d_color [n][C],
 * g2d [n][7] (du, dv, ds, do, dr, dg, db; may be NULL). The forward outputs
 * are as in orc_render and may be NULL. */
int64_t orc_backward(int64_t n, const float* means_sigma, const float* opacity, const float* color,
                     const orc_camera* cam, const orc_opts* o, const double* dL_dimg,
                     double* d_means, double* d_sigma, double* d_opac, double* d_color, double* g2d_out,
                     double* img, double* T, int32_t* nb, int32_t* last, uint8_t* flag, uint64_t* hash) {
    orc_g* g = (orc_g*)malloc(sizeof(orc_g) * (size_t)(n > 0 ? n : 1));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double* g2d = (double*)calloc((size_t)(n > 0 ? n : 1) * 7, sizeof(double));
    int64_t P = (int64_t)cam->width * cam->height;
    double* img_tmp = img ? img : (double*)malloc(sizeof(double) * 3 * (size_t)P);
    prepare(n, means_sigma, opacity, color, cam, o, g);
    int64_t nv = depth_order(n, g, o->proj64, order);
    render_core(n, g, order, nv, cam, o, img_tmp, T, nb, last, flag, hash, dL_dimg, g2d);
    int C = ncoef(o->sh_degree);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double* dm = d_means + 3 * i;
        double* dc = d_color + (size_t)C * i;
        if (!g[i].vis) {
            dm[0] = dm[1] = dm[2] = 0.0; d_sigma[i] = 0.0; d_opac[i] = 0.0;
            for (int k = 0; k < C; ++k) dc[k] = 0.0;
            continue;
        }
        chain_one(&g[i], g2d + 7 * i, means_sigma + 4 * i, color + (size_t)C * i, cam, o,
                  dm, &d_sigma[i], &d_opac[i], dc);
    }
    if (g2d_out) memcpy(g2d_out, g2d, sizeof(double) * 7 * (size_t)n);
    if (!img) free(img_tmp);
    free(g); free(order); free(g2d);
    return nv;
}

/* ------------------------------------------------------- loss and Adam ---- */
/* L1 loss, mean over 3 H W entries, and its gradient sign(C - target)/(3HW)
 * (the l1 part of the training loss of Sec. 3, lambda = 0). */
double orc_l1(int64_t count, const double* img, const float* target, double* grad) {
    double acc = 0.0;
    for (int64_t i = 0; i < count; ++i) {
        double d = img[i] - (double)target[i];
        acc += fabs(d);
        if (grad) grad[i] = (d > 0) ? 1.0 / (double)count : (d < 0 ? -1.0 / (double)count : 0.0);
    }
    return acc / (double)count;
}

/* The loss of Sec. 3 with its structural term, L = (1 - lambda) |f - f^|_1 +
 * lambda (1 - SSIM(f, f^)) (the paper prints "+ lambda SSIM"; a loss has to
 * fall as the images grow alike, so the term is read as 1 - SSIM). The L1 part
 * is the mean absolute difference over all channels x height x width entries.
 * SSIM (the paper gives no definition; read as the structural similarity index
 * of Wang et al.): per channel and pixel q,
 *   S_q = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sxx + syy + C2)),
 * with mx, my, E[x^2], E[y^2], E[xy] the window means around q, sxx = E[x^2] -
 * mx^2, syy = E[y^2] - my^2, sxy = E[xy] - mx my; the window is the 11 x 11
 * Gaussian of standard deviation 1.5 pixels, normalised to sum 1, with zero
 * values outside the image (the "same"-size, zero-padded convention);
 * C1 = 0.01^2, C2 = 0.03^2 (dynamic range 1). SSIM is the mean of S over all
 * entries. Images are planar [channels][height][width].
 *
 * Gradient w.r.t. img (FP64, analytic): with A_q = dS_q/dmx, B_q = dS_q/dE[x^2],
 * Cq = dS_q/dE[xy] (holding the other window means), and w the window,
 *   dSSIM/dx_p = (1/count) sum_q w(q - p) (A_q + 2 x_p B_q + y_p C_q),
 * the sum over pixels q of the image within 5 of p in both axes.
 * Returns L; *ssim_out = SSIM (if not NULL); smap (if not NULL) = S per entry;
 * grad (if not NULL) = dL/dimg. */
static void ssim_window2d(double w[11][11]) {
    double sum = 0.0;
    for (int a = 0; a < 11; ++a)
        for (int b = 0; b < 11; ++b) {
            double da = a - 5, db = b - 5;
            w[a][b] = exp(-(da * da + db * db) / (2.0 * 1.5 * 1.5));
            sum += w[a][b];
        }
    for (int a = 0; a < 11; ++a)
        for (int b = 0; b < 11; ++b) w[a][b] /= sum;
}

double orc_l1_ssim(int64_t channels, int64_t height, int64_t width, const double* img, const double* target,
                   double lambda, double* ssim_out, double* smap, double* grad) {
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    const int64_t plane = height * width, count = channels * plane;
    double w[11][11];
    ssim_window2d(w);
    double* dA = (double*)calloc((size_t)count * 3 + 1, sizeof(double));
    double* dB = dA + count;
    double* dC = dB + count;
    double s_sum = 0.0, l1_sum = 0.0;
    for (int64_t c = 0; c < channels; ++c) {
        const double* x = img + c * plane;
        const double* y = target + c * plane;
#pragma omp parallel for reduction(+ : s_sum) schedule(static)
        for (int64_t i = 0; i < height; ++i)
            for (int64_t j = 0; j < width; ++j) {
                double mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
                for (int a = 0; a < 11; ++a) {
                    int64_t ii = i + a - 5;
                    if (ii < 0 || ii >= height) continue;
                    for (int b = 0; b < 11; ++b) {
                        int64_t jj = j + b - 5;
                        if (jj < 0 || jj >= width) continue;
                        double xv = x[ii * width + jj], yv = y[ii * width + jj], wv = w[a][b];
                        mx += wv * xv;
                        my += wv * yv;
                        exx += wv * xv * xv;
                        eyy += wv * yv * yv;
                        exy += wv * xv * yv;
                    }
                }
                double sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
                double n1 = 2 * mx * my + C1, n2 = 2 * sxy + C2;
                double d1 = mx * mx + my * my + C1, d2 = sxx + syy + C2;
                double S = (n1 * n2) / (d1 * d2);
                s_sum += S;
                int64_t q = c * plane + i * width + j;
                if (smap) smap[q] = S;
                /* dS/dmx: n1' = 2 my, n2' = -2 my, d1' = 2 mx, d2' = -2 mx */
                dA[q] = (2 * my * n2 - 2 * my * n1) / (d1 * d2) - S * (2 * mx / d1 - 2 * mx / d2);
                dB[q] = -S / d2;
                dC[q] = 2 * n1 / (d1 * d2);
            }
    }
    for (int64_t q = 0; q < count; ++q) l1_sum += fabs(img[q] - target[q]);
    if (grad) {
        for (int64_t c = 0; c < channels; ++c) {
            const double* x = img + c * plane;
            const double* y = target + c * plane;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < height; ++i)
                for (int64_t j = 0; j < width; ++j) {
                    double fa = 0, fb = 0, fc = 0;
                    for (int a = 0; a < 11; ++a) {
                        int64_t ii = i + (a - 5);   /* q = p + (a - 5, b - 5), weight w(q - p) */
                        if (ii < 0 || ii >= height) continue;
                        for (int b = 0; b < 11; ++b) {
                            int64_t jj = j + (b - 5);
                            if (jj < 0 || jj >= width) continue;
                            int64_t q = c * plane + ii * width + jj;
                            fa += w[a][b] * dA[q];
                            fb += w[a][b] * dB[q];
                            fc += w[a][b] * dC[q];
                        }
                    }
                    int64_t p = i * width + j;
                    double d = x[p] - y[p];
                    double g1 = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
                    double gs = fa + 2 * x[p] * fb + y[p] * fc;
                    grad[c * plane + p] = ((1.0 - lambda) * g1 - lambda * gs) / (double)count;
                }
        }
    }
    free(dA);
    double ssim = s_sum / (double)count;
    if (ssim_out) *ssim_out = ssim;
    return (1.0 - lambda) * l1_sum / (double)count + lambda * (1.0 - ssim);
}

/* Adam with bias correction (step t >= 1), FP64, in place on p, m, v. */
void orc_adam(int64_t count, double* p, const double* grad, double* m, double* v,
              double lr, double b1, double b2, double eps, int64_t t) {
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < count; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ---------------------------------------------------------------------------
 * The paper's 2D experiment (Sec. 3): an image as a sum of isotropic kernels,
 *   f^(x) = sum over k with |tau_k - x| < D of A_k g(x - mu_k, sigma_k),
 * with tau_k read as the particle centre mu_k and g = exp(-d^2 / (2 sigma^2))
 * (Eq. 8 with the normalisation of reading 1). A particle is 8 floats:
 * (mu_x, mu_y, log sigma, A_r, A_g, A_b, 0, 0) in pixel units (x right, y down);
 * pixel (x, y) samples at (x + 0.5, y + 0.5). Images are planar [3][H][W].
 *
 * The support test is canonical FP32 with one rounding per step, so that both
 * implementations take the same decision: dx = px - mu_x, dy = py - mu_y,
 * d2 = dx*dx + dy*dy, reached iff d2 < D*D. Values and gradients are FP64 on
 * the FP32 parameters.
 * ------------------------------------------------------------------------- */
static int fit_reach(float px, float py, const float* p, float D2) {
    float dx = px - p[0];
    float dy = py - p[1];
    float a = dx * dx;
    float b = dy * dy;
    float d2 = a + b;
    return d2 < D2;
}

void orc_fit2d_render(int64_t k, const float* params, float D, int32_t width, int32_t height, double* img) {
    const float D2 = D * D;
    const int64_t plane = (int64_t)width * height;
#pragma omp parallel for schedule(static)
    for (int32_t y = 0; y < height; ++y)
        for (int32_t x = 0; x < width; ++x) {
            const float px = (float)x + 0.5f, py = (float)y + 0.5f;
            double acc[3] = {0.0, 0.0, 0.0};
            for (int64_t i = 0; i < k; ++i) {
                const float* p = params + 8 * i;
                if (!fit_reach(px, py, p, D2)) continue;
                double dx = (double)px - p[0], dy = (double)py - p[1], s = exp((double)p[2]);
                double g = exp(-(dx * dx + dy * dy) / (2.0 * s * s));
                for (int c = 0; c < 3; ++c) acc[c] += (double)p[3 + c] * g;
            }
            for (int c = 0; c < 3; ++c) img[c * plane + (int64_t)y * width + x] = acc[c];
        }
}

/* Gradient of a loss with image gradient G ([3][H][W]) w.r.t. every particle
 * (grad [k][8], overwritten; the last two slots are 0), the set of reached
 * pixels held fixed: with g as above and s = sum_c A_c G_c(x),
 *   dA_c = sum_x g G_c,  dmu = sum_x s g (x - mu) / sigma^2,
 *   dlog sigma = sum_x s g |x - mu|^2 / sigma^2. */
void orc_fit2d_backward(int64_t k, const float* params, float D, int32_t width, int32_t height, const double* G,
                        double* grad) {
    const float D2 = D * D;
    const int64_t plane = (int64_t)width * height;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < k; ++i) {
        const float* p = params + 8 * i;
        double* gr = grad + 8 * i;
        for (int j = 0; j < 8; ++j) gr[j] = 0.0;
        /* every pixel the FP32 test can accept lies within D + 1 of the centre */
        int64_t x0 = (int64_t)floor((double)p[0] - D - 1.0), x1 = (int64_t)ceil((double)p[0] + D + 1.0);
        int64_t y0 = (int64_t)floor((double)p[1] - D - 1.0), y1 = (int64_t)ceil((double)p[1] + D + 1.0);
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > width - 1) x1 = width - 1;
        if (y1 > height - 1) y1 = height - 1;
        const double s = exp((double)p[2]), inv_s2 = 1.0 / (s * s);
        for (int64_t y = y0; y <= y1; ++y)
            for (int64_t x = x0; x <= x1; ++x) {
                const float px = (float)x + 0.5f, py = (float)y + 0.5f;
                if (!fit_reach(px, py, p, D2)) continue;
                double dx = (double)px - p[0], dy = (double)py - p[1], d2 = dx * dx + dy * dy;
                double g = exp(-d2 * inv_s2 / 2.0);
                double sg = 0.0;
                for (int c = 0; c < 3; ++c) {
                    double Gc = G[c * plane + y * width + x];
                    gr[3 + c] += g * Gc;
                    sg += (double)p[3 + c] * Gc;
                }
                gr[0] += sg * g * dx * inv_s2;
                gr[1] += sg * g * dy * inv_s2;
                gr[2] += sg * g * d2 * inv_s2;
            }
    }
}

/* QuadTree initialisation (Sec. 3.1): each leaf cell of a quad tree over the
 * image holds one particle at the cell centre, with A = the cell's mean colour
 * and sigma = half the cell width. The paper does not say how the tree is
 * grown; read as: starting from the whole image, split the leaf with the
 * largest squared error about its mean colour (SSE, summed over channels) into
 * four, as long as the leaves stay at most k_max (each split adds 3) and the
 * children are at least min_cell pixels wide. The image is square with a power
 * of two side of at most 512; the split statistics use it quantised to 12 bits,
 * q = rint(clamp(v, 0, 1) * 4096), so that they are exact integers:
 * T = sum_c (n S2_c - S1_c^2) with S1, S2 the sums of q and q^2 over the n
 * pixels, and the order key n * SSE * 4096^2 / n^2 = T / n is the double
 * quotient of (double)T and n. Ties: the lower level, then the upper row,
 * then the left column. A_c = S1_c / (4096 n) (double, rounded once to
 * float); log sigma = log2(side / 2) * ln 2 (double, rounded once).
 * Particles are written in (level, row, column) order; returns their number. */
typedef struct {
    int32_t level, iy, ix, side;
    double key;
    int64_t s1[3];
} orc_cell;

static void cell_stats(const int32_t* q, int32_t W, orc_cell* c) {
    uint64_t T = 0;
    const int64_t n = (int64_t)c->side * c->side, plane = (int64_t)W * W;
    for (int ch = 0; ch < 3; ++ch) {
        int64_t s1 = 0, s2 = 0;
        for (int32_t y = c->iy * c->side; y < (c->iy + 1) * c->side; ++y)
            for (int32_t x = c->ix * c->side; x < (c->ix + 1) * c->side; ++x) {
                int64_t v = q[ch * plane + (int64_t)y * W + x];
                s1 += v;
                s2 += v * v;
            }
        c->s1[ch] = s1;
        T += (uint64_t)(n * s2) - (uint64_t)(s1 * s1);
    }
    c->key = (double)T / (double)n;
}

static int cell_before(const orc_cell* a, const orc_cell* b) { /* a split before b? */
    if (a->key != b->key) return a->key > b->key;
    if (a->level != b->level) return a->level < b->level;
    if (a->iy != b->iy) return a->iy < b->iy;
    return a->ix < b->ix;
}

static int cell_order(const void* pa, const void* pb) {
    const orc_cell *a = (const orc_cell*)pa, *b = (const orc_cell*)pb;
    if (a->level != b->level) return a->level < b->level ? -1 : 1;
    if (a->iy != b->iy) return a->iy < b->iy ? -1 : 1;
    return a->ix < b->ix ? -1 : (a->ix > b->ix);
}

int64_t orc_quadtree_init(const float* img, int32_t side, int32_t k_max, int32_t min_cell, float* params) {
    if (side < 1 || side > 512 || (side & (side - 1)) || k_max < 1 || min_cell < 1) return -1;
    const int64_t plane = (int64_t)side * side;
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * 3 * plane);
    for (int64_t i = 0; i < 3 * plane; ++i) {
        float v = img[i];
        v = v < 0.f ? 0.f : (v > 1.f ? 1.f : v);
        q[i] = (int32_t)rint((double)v * 4096.0);
    }
    orc_cell* leaves = (orc_cell*)malloc(sizeof(orc_cell) * (size_t)(k_max + 3));
    int64_t n_leaves = 1;
    leaves[0].level = 0;
    leaves[0].iy = leaves[0].ix = 0;
    leaves[0].side = side;
    cell_stats(q, side, &leaves[0]);
    while (n_leaves + 3 <= k_max) {
        int64_t best = -1;
        for (int64_t i = 0; i < n_leaves; ++i) {
            if (leaves[i].side / 2 < min_cell) continue;
            if (best < 0 || cell_before(&leaves[i], &leaves[best])) best = i;
        }
        if (best < 0) break;
        orc_cell parent = leaves[best];
        for (int j = 0; j < 4; ++j) {
            orc_cell c;
            c.level = parent.level + 1;
            c.side = parent.side / 2;
            c.iy = 2 * parent.iy + (j >> 1);
            c.ix = 2 * parent.ix + (j & 1);
            cell_stats(q, side, &c);
            if (j == 0)
                leaves[best] = c;
            else
                leaves[n_leaves++] = c;
        }
    }
    qsort(leaves, (size_t)n_leaves, sizeof(orc_cell), cell_order);
    for (int64_t i = 0; i < n_leaves; ++i) {
        const orc_cell* c = &leaves[i];
        const double n = (double)c->side * c->side;
        float* p = params + 8 * i;
        p[0] = (float)((double)c->ix * c->side + 0.5 * c->side);
        p[1] = (float)((double)c->iy * c->side + 0.5 * c->side);
        int32_t lg = 0;
        while ((1 << lg) < c->side) ++lg;
        p[2] = (float)((double)(lg - 1) * 0.6931471805599453);
        for (int ch = 0; ch < 3; ++ch) p[3 + ch] = (float)((double)c->s1[ch] / (4096.0 * n));
        p[6] = p[7] = 0.f;
    }
    free(leaves);
    free(q);
    return n_leaves;
}

/* Accumulated position-gradient norm of each 2D particle, the statistic the
 * division rule below reads (Sec. 3.2 names no statistic; reading: the norm of
 * dL/dmu summed over the iterations since the last densify). FP32, one rounding
 * per step: accum_i += sqrt(g_x * g_x + g_y * g_y), g = d_particles[i][0..1]. */
void orc_fit2d_grad_accum(int64_t k, const float* d_particles, float* accum) {
    for (int64_t i = 0; i < k; ++i) {
        const float gx = d_particles[8 * i], gy = d_particles[8 * i + 1];
        const float sq = gx * gx + gy * gy;
        accum[i] = accum[i] + sqrtf(sq);
    }
}

/* Densify / prune of the 2D particles (Sec. 3.2: particles "can be deleted if
 * A_k is smaller than a threshold", and divided, Sec. 2's multiscale property).
 * Reading: particle i is
 *   deleted  if max_c |A_c| < tau_a;
 *   divided  otherwise, if its summed position-gradient norm accum_i exceeds
 *            tau_g * n_iters (FP32 product) and log sigma >= log_sigma_min,
 *            into four children with sigma / 2 at mu + (-/+ sigma/2, -/+ sigma/2)
 *            (order: (-,-), (+,-), (-,+), (+,+)), sigma = exp(log sigma) in FP64
 *            rounded to FP32, half of it exact; child log sigma = log sigma -
 *            ln 2 (FP32), same A;
 *   kept     otherwise.
 * If the result would exceed `capacity`, only the first (by index) division
 * candidates that fit divide (each adds 3), the others are kept. Output in
 * index order (children in place of their parent); kept particles keep their
 * Adam moments, children start with zero moments. Returns the output count. */
int64_t orc_fit2d_densify(int64_t k, const float* params, const float* m, const float* v, const float* accum,
                          int32_t n_iters, float tau_a, float tau_g, float log_sigma_min, int64_t capacity,
                          float* out, float* out_m, float* out_v) {
    const float thr = tau_g * (float)n_iters;
    int64_t keep = 0, cand = 0;
    for (int64_t i = 0; i < k; ++i) {
        const float* p = params + 8 * i;
        float amax = fabsf(p[3]);
        if (fabsf(p[4]) > amax) amax = fabsf(p[4]);
        if (fabsf(p[5]) > amax) amax = fabsf(p[5]);
        if (amax < tau_a) continue;
        ++keep;
        if (accum[i] > thr && p[2] >= log_sigma_min) ++cand;
    }
    int64_t allowed = capacity > keep ? (capacity - keep) / 3 : 0;
    if (allowed > cand) allowed = cand;
    int64_t o = 0, seen = 0;
    for (int64_t i = 0; i < k; ++i) {
        const float* p = params + 8 * i;
        float amax = fabsf(p[3]);
        if (fabsf(p[4]) > amax) amax = fabsf(p[4]);
        if (fabsf(p[5]) > amax) amax = fabsf(p[5]);
        if (amax < tau_a) continue;
        int divide = accum[i] > thr && p[2] >= log_sigma_min;
        if (divide) divide = seen++ < allowed;
        if (!divide) {
            if (o >= capacity) break;
            for (int j = 0; j < 8; ++j) {
                out[8 * o + j] = p[j];
                out_m[8 * o + j] = m[8 * i + j];
                out_v[8 * o + j] = v[8 * i + j];
            }
            ++o;
            continue;
        }
        const float h = 0.5f * (float)exp((double)p[2]);
        for (int c = 0; c < 4; ++c) {
            float* q = out + 8 * o;
            q[0] = (c & 1) ? p[0] + h : p[0] - h;
            q[1] = (c & 2) ? p[1] + h : p[1] - h;
            q[2] = p[2] - 0.6931472f;
            q[3] = p[3];
            q[4] = p[4];
            q[5] = p[5];
            q[6] = q[7] = 0.f;
            for (int j = 0; j < 8; ++j) out_m[8 * o + j] = out_v[8 * o + j] = 0.f;
            ++o;
        }
    }
    return o;
}

/* ------------------------------------------------------------------------- */
/* Densify / prune of the 3D Gaussians (Sec. 3.2: particles whose A_k falls
 * below a threshold are deleted, and particles may be divided; Sec. 2.5's
 * multiscale property, with the Octree of Sec. 3.1 as the division pattern).
 *
 * Statistic, per training step in which Gaussian i touched a tile (count_i > 0):
 *   accum_i += sqrt(du^2 + dv^2)   (its screen-space position gradient, g2d
 *   slots 0 and 1; FP32, one rounding per step),  vis_i += 1. */
void orc_grad_accum3d(int64_t n, const float* g2d, const uint32_t* count, float* accum, uint32_t* vis) {
    for (int64_t i = 0; i < n; ++i) {
        if (count[i] == 0) continue;
        const float du = g2d[8 * i], dv = g2d[8 * i + 1];
        const float sq = du * du + dv * dv;
        accum[i] = accum[i] + sqrtf(sq);
        vis[i] += 1u;
    }
}

/* Reading (parameters as stored: param_mode 1 keeps log sigma and the opacity
 * logit, 0 keeps sigma and the opacity). Gaussian i is
 *   deleted  if its stored opacity < op_min (op_min given in the same
 *            parameterisation, so the test is one FP32 comparison);
 *   divided  otherwise, if vis_i > 0, accum_i > tau_g * vis_i (one FP32
 *            product) and its stored scale >= scale_min, into eight children
 *            (one per octant, child c at mu + (+-h, +-h, +-h) with the sign of
 *            axis a from bit a of c, '-' for 0), h = sigma / 2 (sigma = exp(log
 *            sigma) in double rounded to FP32, or sigma itself), child scale
 *            log sigma - ln 2 (FP32) or sigma / 2; same opacity and colour; zero
 *            Adam moments;
 *   kept     otherwise, with its moments.
 * Output in index order, children in place of their parent; when the result
 * would exceed `capacity`, only the first candidates (by index) that fit
 * divide (each adds 7); if even the kept Gaussians exceed it, the first
 * `capacity` of them are written. Arrays: means_sigma [n][4], opacity [n],
 * color [n][C]; the moments m_*, v_* alike; outputs [capacity] alike. */
int64_t orc_densify3d(int64_t n, int32_t C, int32_t param_mode, const float* ms, const float* op, const float* col,
                      const float* m_ms, const float* m_op, const float* m_col, const float* v_ms, const float* v_op,
                      const float* v_col, const float* accum, const uint32_t* vis, float op_min, float tau_g,
                      float scale_min, int64_t capacity, float* o_ms, float* o_op, float* o_col, float* om_ms,
                      float* om_op, float* om_col, float* ov_ms, float* ov_op, float* ov_col) {
    int64_t keep = 0, cand = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (op[i] < op_min) continue;
        ++keep;
        if (vis[i] > 0 && accum[i] > tau_g * (float)vis[i] && ms[4 * i + 3] >= scale_min) ++cand;
    }
    int64_t allowed = capacity > keep ? (capacity - keep) / 7 : 0;
    if (allowed > cand) allowed = cand;
    int64_t o = 0, seen = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (op[i] < op_min) continue;
        int divide = vis[i] > 0 && accum[i] > tau_g * (float)vis[i] && ms[4 * i + 3] >= scale_min;
        if (divide) divide = seen++ < allowed;
        if (!divide) {
            if (o >= capacity) break;
            memcpy(o_ms + 4 * o, ms + 4 * i, 16);
            memcpy(om_ms + 4 * o, m_ms + 4 * i, 16);
            memcpy(ov_ms + 4 * o, v_ms + 4 * i, 16);
            o_op[o] = op[i];
            om_op[o] = m_op[i];
            ov_op[o] = v_op[i];
            memcpy(o_col + (size_t)C * o, col + (size_t)C * i, 4 * (size_t)C);
            memcpy(om_col + (size_t)C * o, m_col + (size_t)C * i, 4 * (size_t)C);
            memcpy(ov_col + (size_t)C * o, v_col + (size_t)C * i, 4 * (size_t)C);
            ++o;
            continue;
        }
        const float s = ms[4 * i + 3];
        const float sigma = param_mode == 1 ? (float)exp((double)s) : s;
        const float h = 0.5f * sigma;
        const float child_scale = param_mode == 1 ? s - 0.6931472f : 0.5f * s;
        for (int c = 0; c < 8; ++c) {
            for (int a = 0; a < 3; ++a) {
                const float mu = ms[4 * i + a];
                o_ms[4 * o + a] = ((c >> a) & 1) ? mu + h : mu - h;
            }
            o_ms[4 * o + 3] = child_scale;
            o_op[o] = op[i];
            memcpy(o_col + (size_t)C * o, col + (size_t)C * i, 4 * (size_t)C);
            memset(om_ms + 4 * o, 0, 16);
            memset(ov_ms + 4 * o, 0, 16);
            om_op[o] = ov_op[o] = 0.f;
            memset(om_col + (size_t)C * o, 0, 4 * (size_t)C);
            memset(ov_col + (size_t)C * o, 0, 4 * (size_t)C);
            ++o;
        }
    }
    return o;
}

/* ------------------------------------------------------------------------- */
/* Merging of 3D Gaussians (Sec. 3.2: particles may be merged or divided;
 * Sec. 2.5's multiscale property; the Octree of Sec. 3.1 as the pattern, so
 * merging is read as the inverse of the octant division). Reading:
 *   - grid: cells of side h from the corner lo, at most 1024 per axis; with
 *     inv = 1 / h in FP32, Gaussian i's cell index on axis a is
 *     floor((mu_a - lo_a) * inv), each operation rounded once in FP32;
 *   - eligible: finite mean, stored scale <= scale_max (the same
 *     parameterisation as stored), opacity at least 2^-60 (a lighter one
 *     weighs nothing in the merged sums), tested on the stored value: 2^-60 <=
 *     opacity <= 1, or logit >= -41.58883f (the FP32 value nearest the logit of
 *     2^-60) with param_mode 1; and all three cell indices in [0, 1024);
 *   - the eligible Gaussians of one cell, two or more of them, become one
 *     Gaussian at the place (in index order) of the first; with o_k the linear
 *     opacity and sigma_k the linear scale of member k (sums over members in
 *     index order, FP64):
 *       W = sum o_k,  mu = sum o_k mu_k / W,
 *       sigma^2 = sum o_k (sigma_k^2 + |mu_k - mu|^2 / 3) / W   (the mixture's
 *                 covariance, made isotropic by its mean eigenvalue),
 *       o = min(0.99, 1 - prod (1 - o_k)),   colour = sum o_k c_k / W,
 *     with 1 - prod (1 - o_k) evaluated as -expm1(sum log1p(-o_k)) (the same
 *     value, without the cancellation that loses small opacities),
 *     stored back in the input's parameterisation and rounded once to FP32;
 *     zero Adam moments;
 *   - every other Gaussian is kept with its moments; output in index order.
 * Returns the number of Gaussians written (at most n).                     */
typedef struct {
    uint32_t key;
    int64_t idx;
} merge_entry;

static int cmp_merge(const void* a, const void* b) {
    const merge_entry* x = (const merge_entry*)a;
    const merge_entry* y = (const merge_entry*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

/* Cell key (x | y << 10 | z << 20) of Gaussian i, or 0xFFFFFFFF if it is not eligible. */
static uint32_t merge_key(const float* ms, const float* op, int64_t i, int32_t param_mode, const float* lo,
                          float inv, float scale_max) {
    const float* m = ms + 4 * i;
    if (!isfinite(m[0]) || !isfinite(m[1]) || !isfinite(m[2])) return 0xFFFFFFFFu;
    if (!(m[3] <= scale_max)) return 0xFFFFFFFFu;
    const float op_floor = param_mode == 1 ? -41.58883f : 0x1p-60f;
    if (!(op[i] >= op_floor)) return 0xFFFFFFFFu;
    if (param_mode == 0 && !(op[i] <= 1.0f)) return 0xFFFFFFFFu;
    uint32_t key = 0;
    for (int a = 0; a < 3; ++a) {
        const float t = m[a] - lo[a];
        const float c = floorf(t * inv);
        if (!(c >= 0.0f && c < 1024.0f)) return 0xFFFFFFFFu;
        key |= (uint32_t)c << (10 * a);
    }
    return key;
}

int64_t orc_merge3d(int64_t n, int32_t C, int32_t param_mode, const float* ms, const float* op, const float* col,
                    const float* m_ms, const float* m_op, const float* m_col, const float* v_ms, const float* v_op,
                    const float* v_col, const float* lo, float h, float scale_max, float* o_ms, float* o_op,
                    float* o_col, float* om_ms, float* om_op, float* om_col, float* ov_ms, float* ov_op,
                    float* ov_col) {
    const float inv = 1.0f / h;
    merge_entry* e = (merge_entry*)malloc(sizeof(merge_entry) * (size_t)(n > 0 ? n : 1));
    int64_t* first = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));   /* group head of each i */
    int64_t* gbeg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));    /* sorted range of a head */
    int64_t* gend = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        e[i].key = merge_key(ms, op, i, param_mode, lo, inv, scale_max);
        e[i].idx = i;
        first[i] = i;
        gbeg[i] = gend[i] = -1;
    }
    qsort(e, (size_t)n, sizeof(merge_entry), cmp_merge);
    for (int64_t p = 0; p < n;) {
        int64_t q = p + 1;
        while (q < n && e[q].key == e[p].key) ++q;
        if (e[p].key != 0xFFFFFFFFu && q - p >= 2) {
            for (int64_t r = p; r < q; ++r) first[e[r].idx] = e[p].idx;
            gbeg[e[p].idx] = p;
            gend[e[p].idx] = q;
        }
        p = q;
    }
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (first[i] != i) continue;               /* merged into an earlier Gaussian */
        if (gbeg[i] < 0) {                          /* kept */
            memcpy(o_ms + 4 * o, ms + 4 * i, 16);
            memcpy(om_ms + 4 * o, m_ms + 4 * i, 16);
            memcpy(ov_ms + 4 * o, v_ms + 4 * i, 16);
            o_op[o] = op[i];
            om_op[o] = m_op[i];
            ov_op[o] = v_op[i];
            memcpy(o_col + (size_t)C * o, col + (size_t)C * i, 4 * (size_t)C);
            memcpy(om_col + (size_t)C * o, m_col + (size_t)C * i, 4 * (size_t)C);
            memcpy(ov_col + (size_t)C * o, v_col + (size_t)C * i, 4 * (size_t)C);
            ++o;
            continue;
        }
        double W = 0.0, mu[3] = {0.0, 0.0, 0.0}, log_keep = 0.0;
        for (int64_t r = gbeg[i]; r < gend[i]; ++r) {
            const int64_t k = e[r].idx;
            const double ok = param_mode == 1 ? 1.0 / (1.0 + exp(-(double)op[k])) : (double)op[k];
            W += ok;
            for (int a = 0; a < 3; ++a) mu[a] += ok * (double)ms[4 * k + a];
            log_keep += log1p(-ok);
        }
        for (int a = 0; a < 3; ++a) mu[a] /= W;
        double var = 0.0;
        double* acc = (double*)calloc((size_t)C, sizeof(double));
        for (int64_t r = gbeg[i]; r < gend[i]; ++r) {
            const int64_t k = e[r].idx;
            const double ok = param_mode == 1 ? 1.0 / (1.0 + exp(-(double)op[k])) : (double)op[k];
            const double sk = param_mode == 1 ? exp((double)ms[4 * k + 3]) : (double)ms[4 * k + 3];
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double d = (double)ms[4 * k + a] - mu[a];
                d2 += d * d;
            }
            var += ok * (sk * sk + d2 / 3.0);
            for (int c = 0; c < C; ++c) acc[c] += ok * (double)col[(size_t)C * k + c];
        }
        var /= W;
        const double sigma = sqrt(var);
        double om = -expm1(log_keep);
        if (om > 0.99) om = 0.99;
        for (int a = 0; a < 3; ++a) o_ms[4 * o + a] = (float)mu[a];
        o_ms[4 * o + 3] = param_mode == 1 ? (float)log(sigma) : (float)sigma;
        o_op[o] = param_mode == 1 ? (float)log(om / (1.0 - om)) : (float)om;
        for (int c = 0; c < C; ++c) o_col[(size_t)C * o + c] = (float)(acc[c] / W);
        free(acc);
        memset(om_ms + 4 * o, 0, 16);
        memset(ov_ms + 4 * o, 0, 16);
        om_op[o] = ov_op[o] = 0.f;
        memset(om_col + (size_t)C * o, 0, 4 * (size_t)C);
        memset(ov_col + (size_t)C * o, 0, 4 * (size_t)C);
        ++o;
    }
    free(e);
    free(first);
    free(gbeg);
    free(gend);
    return o;
}

/* ------------------------------------------------------------------------- */
/* Octree initialisation of 3D Gaussians (Sec. 3.1: an Octree for 3D, as the
 * QuadTree for 2D; colour = the cell average, sigma = half the cell width),
 * from a coloured point set standing in for the points a reconstruction
 * starts from. Reading:
 *   - domain: the cube [lo, lo + side)^3, levels 0..L (L <= 7), cell of level l
 *     = a cube of side side / 2^l; point p falls in finest cell
 *     i_a = clamp(floor((p_a - lo_a) * inv), 0, 2^L - 1), inv = 2^L / side in
 *     FP32, each operation rounded once; non-finite points are ignored;
 *   - cell id = (8^l - 1) / 7 + Morton index (bits of x, y, z interleaved,
 *     x lowest);
 *   - statistics on colours quantised to 12 bits, q = rint(clamp(c, 0, 1) 4096):
 *     n, S1_c, S2_c exact integers;
 *   - error of a cell: e = max(0, sum_c (S2_c - S1_c * S1_c / n)) in double,
 *     one rounding per step in channel order; its key = min(e, key of its
 *     parent) (the parent's error is never below the child's; the cap only
 *     keeps rounding from putting a child before its parent); a cell with
 *     n >= 2 points and level < L is splittable; order: key descending, id
 *     ascending;
 *   - growth: start from the root (one leaf); repeatedly take the splittable
 *     leaf first in that order; splitting it replaces it by its non-empty
 *     children; stop when that would make more than k_max leaves (or no leaf
 *     is splittable);
 *   - one Gaussian per non-empty leaf in id order: mean = cell centre
 *     lo + (i + 1/2) side / 2^l (double, rounded once), sigma = half the cell
 *     side, colour = S1_c / (4096 n) (double, rounded once) as RGB, or as the
 *     DC coefficient (colour - 1/2) / Y00 of SH of degree sh_degree with the
 *     others 0, opacity `opacity`; param_mode 1 stores log sigma and the
 *     opacity logit (double, rounded once).
 * Returns the number of Gaussians, or -1 for invalid arguments. */
typedef struct {
    int64_t n, s1[3], s2[3];
} orc_ocell;

static int64_t oct_off(int l) { return ((((int64_t)1) << (3 * l)) - 1) / 7; }

static uint32_t oct_morton(uint32_t x, uint32_t y, uint32_t z, int L) {
    uint32_t m = 0;
    for (int b = 0; b < L; ++b)
        m |= (((x >> b) & 1u) << (3 * b)) | (((y >> b) & 1u) << (3 * b + 1)) | (((z >> b) & 1u) << (3 * b + 2));
    return m;
}

static double oct_err(const orc_ocell* c) {
    const double n = (double)c->n;
    double e = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
        const double s1 = (double)c->s1[ch];
        e = e + ((double)c->s2[ch] - s1 * s1 / n);
    }
    return e > 0.0 ? e : 0.0;
}

int64_t orc_octree_init(int64_t npts, const float* pts, const float* cols, const float* lo, float side, int32_t L,
                        int64_t k_max, float opacity, int32_t sh_degree, int32_t param_mode, float* out_ms,
                        float* out_op, float* out_col) {
    if (L < 0 || L > 7 || k_max < 1 || !(side > 0.f) || sh_degree < -1 || sh_degree > 3) return -1;
    const int64_t cells = oct_off(L + 1);
    orc_ocell* st = (orc_ocell*)calloc((size_t)cells, sizeof(orc_ocell));
    uint8_t* split = (uint8_t*)calloc((size_t)cells, 1);
    uint8_t* leaf = (uint8_t*)calloc((size_t)cells, 1);
    const float inv = (float)((double)(1 << L) / (double)side);
    const int32_t top = (1 << L) - 1;
    for (int64_t i = 0; i < npts; ++i) {
        const float* p = pts + 3 * i;
        if (!isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) continue;
        int32_t ix[3];
        for (int a = 0; a < 3; ++a) {
            const float t = floorf((p[a] - lo[a]) * inv);
            ix[a] = t < 0.f ? 0 : (t > (float)top ? top : (int32_t)t);
        }
        orc_ocell* c = st + oct_off(L) + oct_morton((uint32_t)ix[0], (uint32_t)ix[1], (uint32_t)ix[2], L);
        c->n += 1;
        for (int ch = 0; ch < 3; ++ch) {
            float v = cols[3 * i + ch];
            v = v < 0.f ? 0.f : (v > 1.f ? 1.f : v);
            const int64_t q = (int64_t)rintf(v * 4096.f);
            c->s1[ch] += q;
            c->s2[ch] += q * q;
        }
    }
    for (int l = L - 1; l >= 0; --l)
        for (int64_t m = 0; m < ((int64_t)1 << (3 * l)); ++m) {
            orc_ocell* c = st + oct_off(l) + m;
            for (int d = 0; d < 8; ++d) {
                const orc_ocell* k = st + oct_off(l + 1) + 8 * m + d;
                c->n += k->n;
                for (int ch = 0; ch < 3; ++ch) {
                    c->s1[ch] += k->s1[ch];
                    c->s2[ch] += k->s2[ch];
                }
            }
        }
    double* key = (double*)calloc((size_t)cells, sizeof(double));
    for (int l = 0; l <= L; ++l)
        for (int64_t m = 0; m < ((int64_t)1 << (3 * l)); ++m) {
            const int64_t id = oct_off(l) + m;
            const double e = st[id].n > 0 ? oct_err(st + id) : 0.0;
            const double kp = l > 0 ? key[oct_off(l - 1) + (m >> 3)] : e;
            key[id] = e < kp ? e : kp;
        }
    int64_t leaves = st[0].n > 0 ? 1 : 0;
    if (leaves) leaf[0] = 1;
    for (;;) {  /* the greedy rule as written: scan the leaves for the first in the order */
        int64_t best = -1;
        double be = -1.0;
        for (int l = 0; l < L; ++l)
            for (int64_t m = 0; m < ((int64_t)1 << (3 * l)); ++m) {
                const int64_t id = oct_off(l) + m;
                if (!leaf[id] || st[id].n < 2) continue;
                const double e = key[id];
                if (e > be) {
                    be = e;
                    best = id;
                }
            }
        if (best < 0) break;
        int l = 0;
        while (oct_off(l + 1) <= best) ++l;
        const int64_t m = best - oct_off(l);
        int64_t kids = 0;
        for (int d = 0; d < 8; ++d) kids += st[oct_off(l + 1) + 8 * m + d].n > 0;
        if (leaves + kids - 1 > k_max) break;
        leaf[best] = 0;
        split[best] = 1;
        for (int d = 0; d < 8; ++d)
            if (st[oct_off(l + 1) + 8 * m + d].n > 0) leaf[oct_off(l + 1) + 8 * m + d] = 1;
        leaves += kids - 1;
    }
    const int C = sh_degree < 0 ? 3 : 3 * (sh_degree + 1) * (sh_degree + 1);
    const double y00 = 0.5 / sqrt(3.14159265358979323846);
    int64_t o = 0;
    for (int l = 0; l <= L; ++l)
        for (int64_t m = 0; m < ((int64_t)1 << (3 * l)); ++m) {
            const int64_t id = oct_off(l) + m;
            if (!leaf[id]) continue;
            uint32_t c3[3] = {0, 0, 0};
            for (int b = 0; b < l; ++b)
                for (int a = 0; a < 3; ++a) c3[a] |= (uint32_t)((m >> (3 * b + a)) & 1) << b;
            const double cs = (double)side / (double)(1 << l);
            float* q = out_ms + 4 * o;
            for (int a = 0; a < 3; ++a) q[a] = (float)((double)lo[a] + ((double)c3[a] + 0.5) * cs);
            q[3] = param_mode == 1 ? (float)log(0.5 * cs) : (float)(0.5 * cs);
            out_op[o] = param_mode == 1 ? (float)log((double)opacity / (1.0 - (double)opacity)) : opacity;
            float* cc = out_col + (size_t)C * o;
            for (int k = 0; k < C; ++k) cc[k] = 0.f;
            for (int ch = 0; ch < 3; ++ch) {
                const double mean = (double)st[id].s1[ch] / (4096.0 * (double)st[id].n);
                cc[ch] = sh_degree < 0 ? (float)mean : (float)((mean - 0.5) / y00);
            }
            ++o;
        }
    free(st);
    free(split);
    free(leaf);
    free(key);
    return o;
}
