/*
 * igs.h — C ABI of the GB300 (sm_103a) isotropic Gaussian splatting library.
 *
 * Method: arXiv 2403.14244, "Isotropic Gaussian Splatting for Real-Time
 * Radiance Field Rendering". Each particle is an isotropic Gaussian (Eq. 8)
 * with centre mu, one scale sigma, an opacity and a colour (plain RGB or real
 * spherical harmonics up to degree 3). A view is rendered by projecting every
 * Gaussian to a screen-space disc (Eq. 7 with Sigma = sigma^2 I: centre
 * u = fx x_c/z_c + cx, v = fy y_c/z_c + cy, radius s = fx sigma / z_c, which
 * depends only on the depth, Sec. 2.4), by compositing the discs front to
 * back per pixel (Eq. 4), and trained by the gradients of Eq. 3 and the
 * position gradient after it. Compositing rules fixed by this library where
 * the paper is silent:
 *   alpha = min(alpha_max, o * exp(-d^2 / (2 s^2)))  (Eq. 8 with s = sigma/sqrt 2)
 *   entries with alpha < alpha_min are skipped;
 *   an entry that would take the transmittance below t_min is not blended and
 *   ends the pixel; the final colour is C + T_final * bg;
 *   pixel centres are at (x + 0.5, y + 0.5);
 *   footprint radius r >= s sqrt(2 (ln(255 o) + 2^-9)) (compact support, Eq. 2, per
 *   particle): beyond it alpha < 1/255.
 *
 * Conventions for every entry point
 *   - Pointers marked "device" are CUDA device pointers of the current device;
 *     "host" pointers are ordinary host memory. The caller owns every buffer it
 *     passes. The library never allocates device memory: scratch comes from the
 *     caller through igs_frame_layout().
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Every call
 *     is asynchronous on `stream` unless it says otherwise.
 *   - Argument errors (NULL pointers, sizes out of range, tile not 8/16/32,
 *     fx != fy, a frame laid out for other sizes) return IGS_ERR_INVALID_ARG
 *     synchronously and launch nothing. Launch failures return IGS_ERR_CUDA.
 *   - Errors found on the device (capacity overflow, a bounded spin-wait that
 *     ran out) are written to the frame's device status words; read them with
 *     igs_frame_status(). A kernel never traps: it records the error and returns.
 *   - igs_last_error() gives a thread-local message for the last failed call.
 *
 * Data layout (structure of arrays, FP32, C order):
 *   means_sigma [n][4]  (x, y, z, sigma) or (x, y, z, log sigma) with param_mode 1
 *   opacity     [n]     opacity, or its logit with param_mode 1
 *   color       [n][C]  C = 3 (RGB, sh_degree -1) or 3 (deg+1)^2 SH coefficients,
 *                       coefficient-major: color[i][3*k + channel], k = l^2 + l + m,
 *                       real orthonormal basis without Condon-Shortley phase;
 *                       rgb = max(0, sum_k color[k] Y_k(dir) + 0.5), dir from the
 *                       camera centre to mu.
 *   images      [3][H][W] planar RGB; per-pixel buffers [H][W].
 */
#ifndef IGS_H
#define IGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IGS_ABI_VERSION 3

#if defined(__GNUC__)
#define IGS_API __attribute__((visibility("default")))
#else
#define IGS_API
#endif

typedef enum igs_status {
    IGS_OK = 0,
    IGS_ERR_INVALID_ARG = 1,
    IGS_ERR_OOM = 2,             /* a caller-sized buffer is too small */
    IGS_ERR_CUDA = 3,            /* a CUDA launch or call failed */
    IGS_ERR_CAPACITY = 4,        /* more (Gaussian, tile) entries than the frame holds */
    IGS_ERR_NOT_READY = 5,
    IGS_ERR_DEVICE_TIMEOUT = 6,  /* a bounded device spin-wait gave up */
    IGS_ERR_UNSUPPORTED = 7
} igs_status;

/* Pinhole camera, world -> camera x_c = R x_w + t (R row-major); image x to the
 * right, y down, z forward. fx must equal fy (an isotropic Gaussian projects to
 * a disc only then). znear: Gaussians with z_c <= znear are culled. */
typedef struct igs_camera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float znear;
    int32_t width, height;
} igs_camera;

typedef struct igs_opts {
    int32_t tile;        /* tile edge in pixels: 8, 16 or 32 */
    int32_t sh_degree;   /* -1: colour is RGB; 0..3: SH of that degree */
    int32_t param_mode;  /* 0: sigma and opacity stored as is; 1: log sigma and logit */
    float alpha_min;     /* 1/255 (at least 1/255: the footprint holds every pixel with alpha >= 1/255) */
    float alpha_max;     /* 0.99 */
    float t_min;         /* 1e-4 */
    float bg[3];         /* background colour, added with the final transmittance */
    int32_t footprint;   /* tiles of a Gaussian (Eq. 2's support, radius r from s and o): 0 = every tile of
                            the bounding rectangle of its disc; 1 = in each row of that rectangle, only the
                            tiles whose column meets the disc (fewer entries, more arithmetic). The image
                            is the same either way; igs_project and igs_bin_sort of a frame take the same. */
} igs_opts;

/* Scene buffers (device), layout above. */
typedef struct igs_scene {
    const float* means_sigma;
    const float* opacity;
    const float* color;
    int64_t n;
} igs_scene;

/* Per-view state. igs_frame_layout() carves every pointer out of ONE caller
 * buffer; the same frame serves igs_project, igs_bin_sort, igs_render_fwd and
 * igs_render_bwd of one view, and can be reused for the next view of the same
 * size. Contents after each step:
 *   igs_project:    rec, rect, count, depth_key
 *   igs_bin_sort:   order, vals, ranges, info[0..1]; offset only when sort_chunks == 0
 *   igs_render_fwd: T_final, n_contrib
 * Status words (device, uint32): info[0] = M entries, info[1] = Gaussians kept,
 * info[2] = error code (igs_status, 0 = none), info[3] = M the view needs. */
typedef struct igs_frame {
    int64_t n;               /* Gaussians the frame was laid out for */
    int64_t capacity;        /* (Gaussian, tile) entries it can hold */
    int32_t width, height, tile, tiles_x, tiles_y;
    int32_t sort_chunks;     /* > 0: entries placed by a counting sort over this many chunks of
                                the depth order; 0: duplication + radix sort on the tile id */
    float* rec;              /* [n][8] u, v, w2 = log2(e)/(2 s^2), pmax, r, g, b, o; pmax = log2(o / alpha_min)
                                + 2^-10 bounds the exponent w2 d^2 of every pixel with alpha >= alpha_min */
    uint32_t* rect;          /* [n][2] x0 | y0 << 16, x1 | y1 << 16 (inclusive tiles): the bounding
                                rectangle of the tiles the footprint disc meets */
    float* disc;             /* [n][4] u, v, footprint radius r, x0 | x1 << 16 (as float bits); zero if
                                culled. In tile row ty of the rectangle the Gaussian touches the tiles
                                whose column meets u +- sqrt(r^2 - dy^2) (dy: distance from v to the row) */
    uint32_t* count;         /* [n] tiles touched; 0 = culled */
    uint32_t* depth_key;     /* [n] bits of the FP32 depth z_c; 0xFFFFFFFF if culled */
    uint32_t* order;         /* [n] Gaussian ids, front to back (culled ones last) */
    uint32_t* offset;        /* [n] first entry of order[p]: exclusive scan of count in depth order */
    uint32_t* tile_key;      /* [capacity] tile id of each sorted entry (written by igs_export_keys) */
    uint32_t* vals;          /* [capacity] Gaussian id of each sorted entry (tile_key and vals share
                                the sort's scratch: valid until the next igs_bin_sort of this frame) */
    uint32_t* ranges;        /* [tiles][2] [start, end) of each tile's entries; (0, 0) if empty */
    float* T_final;          /* [H][W] transmittance after the last blended entry */
    uint32_t* n_contrib;     /* [H][W] 1 + list position (within the tile) of the last blended entry */
    uint32_t* info;          /* [16] status words, see above */
    void* scratch;           /* sort double buffers, histograms, look-back state */
    size_t scratch_bytes;
} igs_frame;

/* Lay out a frame for n Gaussians, at most `capacity` entries, and the camera's
 * image size and opts->tile. With workspace == NULL only *bytes is written (the
 * size to allocate, 256-byte aligned). Otherwise `workspace` (device, >= *bytes,
 * 256-byte aligned) is carved into `frame`; nothing is launched and the
 * workspace is not cleared (each step initialises what it reads). */
IGS_API igs_status igs_frame_layout(int64_t n, int64_t capacity, const igs_camera* cam, const igs_opts* opts,
                            void* workspace, size_t* bytes, igs_frame* frame);

/* Project every Gaussian to its screen disc and tile rectangle
 * (Eq. 7 with Sigma = sigma^2 I, Eq. 2 support radius from s and o; culling of z_c <=
 * znear, sigma <= 0, opacity < 1/255, non-finite input, off-grid rectangle), and
 * evaluate its colour (RGB, or SH at the direction from the camera centre).
 * With param_mode 1 sigma = exp(log sigma) and opacity = sigmoid(logit) here.
 * The culling decisions, depth key and rectangle use FP32 with every operation
 * rounded once in a fixed order (bit-reproducible). Writes rec, rect, count,
 * depth_key. */
IGS_API igs_status igs_project(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                       igs_frame* frame, void* stream);

/* Order the kept Gaussians front to back (stable radix sort of the
 * depth keys; ties keep index order), count every tile's entries from the
 * footprints (the per-tile ranges), and place one entry per (Gaussian, touched
 * tile) in tile order, front to back within each tile. Frames at most 2048
 * tiles wide and high (frame->sort_chunks > 0) place the entries by two stable
 * counting sorts (Gaussians into the lists of the tile rows they span, then
 * each row's list into its tiles); wider frames duplicate each Gaussian, in
 * depth order, into one (tile, Gaussian) item per touched tile and radix sort
 * the items by tile id (and write offset). Either way the entry order is that
 * of the 64-bit key (tile << 32 | depth bits) sorted stably: within a tile,
 * front to back as Eq. 4 requires. If M exceeds frame->capacity, info[2] is
 * set to IGS_ERR_CAPACITY, info[3] to M, and the later steps leave their
 * outputs untouched. Writes order, vals, ranges, info (and offset on the
 * radix route). */
IGS_API igs_status igs_bin_sort(igs_frame* frame, const igs_opts* opts, void* stream);

/* Front-to-back order of n depth keys WITHOUT allocating anything. The paper
 * has no counterpart: this exists for callers that cannot allocate device
 * memory around the call, such as a host application whose device memory all
 * belongs to its own allocator (reserved at start-up, so a cudaMalloc here
 * would fail or steal from it), or a latency-critical loop that must not call
 * cudaMalloc/cudaFree because they can synchronise the whole device.
 * It computes exactly what igs_bin_sort writes to frame->order for the same
 * depth_key: a stable ascending sort of the keys (ties keep index order), the
 * output being the indices. depth_key (device, n) is read; order (device, n)
 * is overwritten. Limit: n <= 1048576 (2^20); larger n returns
 * IGS_ERR_INVALID_ARG and launches nothing.
 * Scratch lives in one fixed 17.6 MB device array compiled into the library,
 * which every GPU that loads the library holds until the process exits. The
 * first call on each device looks up that array's device address; make that
 * first call before any stream capture. Every call on a device shares the
 * array (the call clears what must start at zero), so calls that overlap on
 * the GPU race: serialise them (one stream, or events). Asynchronous on
 * `stream`; a failed launch returns IGS_ERR_CUDA and igs_last_error() names
 * it; a device-side bounded wait that runs out leaves order incomplete and is
 * not reported here. */
IGS_API igs_status igs_sort_depth_noalloc(const uint32_t* depth_key, int64_t n, uint32_t* order, void* stream);

/* Export the sorted 64-bit keys (tile << 32 | depth bits), M = info[0] of them,
 * into keys (device, >= capacity entries), and the tile id of every sorted entry
 * into frame->tile_key. For inspection and tests. */
IGS_API igs_status igs_export_keys(const igs_frame* frame, uint64_t* keys, void* stream);

/* Per tile, front-to-back compositing of its entries (Eq. 4) at every pixel
 * centre. Writes img (device, [3][H][W]) = C + T_final * bg, and the frame's
 * T_final and n_contrib (saved for the backward pass). */
IGS_API igs_status igs_render_fwd(igs_frame* frame, const igs_opts* opts, float* img, void* stream);

/* Adjoint of igs_render_fwd and igs_project for dL_dimg (device,
 * [3][H][W]). Walks each pixel's blended entries back to front, recovering the
 * transmittance from T_final (no forward re-run), accumulates per-Gaussian
 * screen-space gradients in g2d (device, [n][8], caller scratch, cleared here),
 * then chains them to the stored parameters. Gradients are OVERWRITTEN:
 * d_means_sigma [n][4] (mu, and sigma or log sigma), d_opacity [n] (opacity or
 * logit), d_color [n][C]. Culled Gaussians get 0. The set of blended entries is
 * held fixed (almost-everywhere derivative). */
IGS_API igs_status igs_render_bwd(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                          const igs_frame* frame, const float* dL_dimg, float* g2d,
                          float* d_means_sigma, float* d_opacity, float* d_color, void* stream);

/* The two halves of igs_render_bwd, for callers that time or overlap them:
 * igs_blend_bwd clears g2d ([n][8], device) and accumulates the screen-space
 * gradients (du, dv, dw2, do, dr, dg, db, 0) of every Gaussian over all pixels;
 * igs_project_bwd chains g2d to the stored parameters (same outputs and rules
 * as igs_render_bwd). The projection backward reads every Gaussian's row of
 * g2d, culled ones included (their values are not used), so g2d must hold all
 * n rows; the same holds for the fused variants below. */
IGS_API igs_status igs_blend_bwd(const igs_frame* frame, const igs_opts* opts, const float* dL_dimg, float* g2d,
                                 void* stream);
IGS_API igs_status igs_project_bwd(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                                   const igs_frame* frame, const float* g2d, float* d_means_sigma,
                                   float* d_opacity, float* d_color, void* stream);

/* The forward and the first half of the adjoint of a training step (Eq. 4 and
 * its adjoint, Eq. 3 for the screen-space parameters), with the clearing of
 * the 2D gradient moved into the forward: igs_render_fwd_clear is
 * igs_render_fwd that also sets g2d ([n][8] floats, device, 16-byte aligned) to
 * zero, its CTAs writing the zeros while they blend (the forward is bound by
 * instruction issue, not by memory); igs_blend_bwd_acc is igs_blend_bwd
 * without the clearing: it accumulates into g2d as that forward left it. Use
 * them as a pair on one frame and stream, one igs_blend_bwd_acc per
 * igs_render_fwd_clear, with nothing writing g2d in between (the forward also
 * resets the backward's work counter of the frame). Same outputs as
 * igs_render_fwd + igs_blend_bwd; g2d is cleared even when the frame is
 * aborted (capacity), as igs_blend_bwd does. Errors as igs_render_fwd /
 * igs_blend_bwd; a NULL or unaligned g2d returns IGS_ERR_INVALID_ARG. */
IGS_API igs_status igs_render_fwd_clear(igs_frame* frame, const igs_opts* opts, float* img, float* g2d,
                                        void* stream);
IGS_API igs_status igs_blend_bwd_acc(const igs_frame* frame, const igs_opts* opts, const float* dL_dimg,
                                     float* g2d, void* stream);

/* The projection backward fused with one Adam step, for training: the same
 * gradient as igs_project_bwd, applied at once to the parameters without
 * writing it out. scene->means_sigma, scene->opacity and scene->color (device,
 * layout above, log sigma / logit with param_mode 1) are UPDATED IN PLACE; m_*
 * and v_* (device, same shapes; 16-byte aligned means_sigma and color rows) are
 * the Adam moments, updated in place. Every Gaussian is stepped, culled ones with
 * a zero gradient (their moments decay), exactly as igs_adam over the gradient
 * of igs_project_bwd would. Step and hyper-parameters as in igs_adam. */
IGS_API igs_status igs_project_bwd_adam(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                                        const igs_frame* frame, const float* g2d, float* m_means_sigma,
                                        float* m_opacity, float* m_color, float* v_means_sigma, float* v_opacity,
                                        float* v_color, double lr, double b1, double b2, double eps, int64_t step,
                                        void* stream);

/* igs_project_bwd_adam with the Adam step count on the device, so that a
 * training step can be captured in a CUDA graph and replayed: d_state (device
 * int32[4], 16-byte aligned, zero before the first step, caller-owned) holds
 * the count of steps taken; the call first advances it (t = d_state[0] + 1,
 * stored back) and writes that step's bias-corrected constants (lr / (1 - b1^t),
 * 1 / sqrt(1 - b2^t), sqrt(1 - b2^t), formed in double, rounded to FP32) to
 * d_state[1..3], then applies the same update as igs_project_bwd_adam. Two
 * launches; errors as igs_project_bwd_adam, plus a NULL or misaligned d_state. */
IGS_API igs_status igs_project_bwd_adam_dev(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                                            const igs_frame* frame, const float* g2d, float* m_means_sigma,
                                            float* m_opacity, float* m_color, float* v_means_sigma, float* v_opacity,
                                            float* v_color, double lr, double b1, double b2, double eps,
                                            int32_t* d_state, void* stream);

/* igs_project_bwd_adam_dev followed, in the same pass over the Gaussians, by
 * the projection of the NEXT view (Eq. 7 with Sigma = sigma^2 I, Sec. 2.4: as
 * igs_project) from the parameters just updated: next_frame receives exactly
 * what igs_project(scene after this step, next_cam, opts, next_frame) would
 * write (rec, rect, disc, count, depth_key, bit for bit), so that the next
 * view's step starts at igs_bin_sort. next_frame (laid out for next_cam's size
 * and scene->n) may be `frame` itself: each Gaussian's count of this view is
 * read before the next view's is written. The parameters are read once for
 * both: one pass over HBM instead of two. Two launches; errors as
 * igs_project_bwd_adam_dev, plus a NULL, invalid or mismatched next_cam or
 * next_frame. */
IGS_API igs_status igs_project_bwd_adam_next(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                                             const igs_frame* frame, const float* g2d, float* m_means_sigma,
                                             float* m_opacity, float* m_color, float* v_means_sigma,
                                             float* v_opacity, float* v_color, double lr, double b1, double b2,
                                             double eps, int32_t* d_state, const igs_camera* next_cam,
                                             const igs_frame* next_frame, void* stream);

/* L1 loss of Sec. 3 (lambda = 0): loss = mean |img - target| over `count`
 * entries, written to *loss (device float, overwritten), and
 * dL_dimg = sign(img - target) / count (device, count entries; sign(0) = 0). */
IGS_API igs_status igs_l1_loss(const float* img, const float* target, int64_t count, float* loss,
                       float* dL_dimg, void* stream);

/* Bytes of device scratch igs_l1_ssim_loss needs for planar [channels][height]
 * [width] images (three FP32 maps of that size); 0 for an empty or invalid size. */
IGS_API size_t igs_ssim_work_bytes(int32_t channels, int32_t height, int32_t width);

/* The loss of Sec. 3 with its structural term,
 *   loss = (1 - lambda) mean |img - target| + lambda (1 - SSIM(img, target)),
 * (the paper prints "+ lambda SSIM"; as a loss it is read as 1 - SSIM;
 * lambda = 0.2 in the paper). SSIM is the mean over all entries of Wang et al.'s
 * index, per channel, with the 11 x 11 Gaussian window of standard deviation
 * 1.5 (normalised to sum 1; zero values outside the image), C1 = 0.01^2,
 * C2 = 0.03^2 (dynamic range 1).
 * img, target: device FP32, planar [channels][height][width]. *loss (device
 * float) is overwritten; *ssim (device float, may be NULL) receives the mean
 * SSIM; dL_dimg (device, same layout) receives dloss/dimg, with
 * sign(0) = 0 in the L1 part. work: device scratch of igs_ssim_work_bytes bytes,
 * 16-byte aligned, caller-owned, overwritten. Asynchronous on `stream`.
 * Errors: NULL buffers, channels outside 1..65535, height or width < 1, lambda
 * outside [0, 1], work not 16-byte aligned -> IGS_ERR_INVALID_ARG; launch failures -> IGS_ERR_CUDA.
 * loss and ssim are sums of per-tile partials added in arbitrary order (not
 * bit-reproducible); dL_dimg is deterministic. */
IGS_API igs_status igs_l1_ssim_loss(const float* img, const float* target, int32_t channels, int32_t height,
                                    int32_t width, float lambda, float* loss, float* ssim, float* dL_dimg,
                                    void* work, void* stream);

/* ---------------------------------------------------------------------------
 * The paper's 2D experiment (Sec. 3): an image as a sum of isotropic kernels,
 *   f^(x) = sum over k with |mu_k - x| < D of A_k exp(-|x - mu_k|^2 / (2 sigma_k^2))
 * (Eq. 8 with the 1/2 of the Gaussian; the support centre tau_k read as mu_k).
 * A particle is 8 floats (mu_x, mu_y, log sigma, A_r, A_g, A_b, 0, 0) in pixel
 * units (x right, y down); particle arrays are device [k][8], 16-byte aligned.
 * Pixel (x, y) samples at (x + 0.5, y + 0.5); images are planar [3][H][W] FP32.
 * The support test is canonical FP32: dx = px - mu_x, dy = py - mu_y,
 * d2 = dx*dx + dy*dy, each step rounded once; reached iff d2 < D*D (D*D rounded
 * once). Non-finite particles reach nothing. All calls are asynchronous.
 * ------------------------------------------------------------------------- */

/* img = f^ over all width x height pixels (overwritten). Each pixel sums its
 * particles in index order (deterministic). D > 0 (+inf: no cutoff).
 * Errors: k outside 0..2^27, size outside 1..2^20, D <= 0 or NaN, NULL or
 * misaligned buffers -> IGS_ERR_INVALID_ARG. */
IGS_API igs_status igs_fit2d_render(const float* particles, int32_t k, float D, int32_t width, int32_t height,
                                    float* img, void* stream);

/* d_particles [k][8] (device, overwritten) = the gradient of a loss whose image
 * gradient is dL_dimg ([3][H][W]), the reached pixels held fixed:
 *   dA_c = sum_x g G_c,  dmu = sum_x s g (x - mu) / sigma^2,
 *   dlog sigma = sum_x s g |x - mu|^2 / sigma^2,  s = sum_c A_c G_c(x);
 * slots 6, 7 are 0. Sums over tiles are added atomically (not bit-reproducible). */
IGS_API igs_status igs_fit2d_backward(const float* particles, int32_t k, float D, int32_t width, int32_t height,
                                      const float* dL_dimg, float* d_particles, void* stream);

/* One bias-corrected Adam step over the particles in place (m, v: device [k][8],
 * the moments), slot j of every particle with learning rate lr[j] (host, 8
 * floats >= 0). The step count lives on the device so that captured graphs can
 * replay steps: d_state is device int32[2], zero before the first step; the
 * step uses t = d_state[0] + 1 and increments d_state[0] when it completes
 * (d_state[1] is internal). Update as igs_adam: m = b1 m + (1-b1) g;
 * v = b2 v + (1-b2) g^2; p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
IGS_API igs_status igs_fit2d_adam(float* particles, const float* d_particles, float* m, float* v, int32_t k,
                                  const float* lr, double b1, double b2, double eps, int32_t* d_state,
                                  void* stream);

/* Densify / prune of the 2D particles (Sec. 3.2: particles may be deleted when
 * A_k falls below a threshold, and divided; Sec. 2's multiscale property).
 *
 * igs_fit2d_grad_accum: accum[i] += sqrt(g_x^2 + g_y^2) for each particle,
 * g = d_particles[i][0..1] (the position gradient from igs_fit2d_backward);
 * FP32, each step rounded once. accum: device float[k], caller-owned, zeroed by
 * the caller when a densify interval starts. Asynchronous.
 *
 * igs_fit2d_densify: from particles, m, v (device [k][8], the Adam moments) and
 * accum (device float[k], summed over the n_iters iterations since the last
 * densify), writes new particles and moments to out, out_m, out_v (device
 * [capacity][8], caller-owned, 16-byte aligned, not overlapping the inputs) and
 * their number to *d_count (device int32). Particle i is
 *   deleted  if max_c |A_c| < tau_a (compared in channel order);
 *   divided  else, if accum[i] > tau_g * n_iters (one FP32 product) and
 *            log sigma >= log_sigma_min, into four children of half the scale
 *            (log sigma - ln 2 in FP32) at mu + (-h, -h), (+h, -h), (-h, +h),
 *            (+h, +h), h = sigma / 2 with sigma = exp(log sigma) in double
 *            rounded to FP32; same A; zero moments;
 *   kept     otherwise, with its moments.
 * Output is in index order, children in place of their parent. If the result
 * would exceed capacity, only the first candidates (by index) that fit divide,
 * each adding 3; if even the kept particles exceed it, the first capacity of
 * them are written. One CTA; intended for periodic use (e.g. every 100
 * iterations). Errors: k or capacity outside 0..2^27, n_iters < 1, a NaN
 * threshold, NULL, misaligned or overlapping buffers -> IGS_ERR_INVALID_ARG. */
IGS_API igs_status igs_fit2d_grad_accum(const float* d_particles, int32_t k, float* accum, void* stream);
IGS_API igs_status igs_fit2d_densify(const float* particles, const float* m, const float* v, const float* accum,
                                     int32_t k, int32_t n_iters, float tau_a, float tau_g, float log_sigma_min,
                                     int32_t capacity, float* out, float* out_m, float* out_v, int32_t* d_count,
                                     void* stream);

/* ---------------------------------------------------------------------------
 * Densify / prune of the 3D Gaussians (Sec. 3.2: a particle whose A_k falls
 * below a threshold is deleted, and particles may be divided; Sec. 2.5's
 * multiscale property, with the Octree of Sec. 3.1 as the division pattern).
 * ------------------------------------------------------------------------- */

/* Mutable parameter arrays of n Gaussians (device, caller-owned): means_sigma
 * [n][4] (16-byte aligned), opacity [n], color [n][C] (16-byte aligned),
 * C = 3 (RGB) or 3 (deg + 1)^2 (SH). Also used for Adam moments. */
typedef struct igs_params {
    float* means_sigma;
    float* opacity;
    float* color;
} igs_params;

/* Densify statistic after one training step: for every Gaussian i with
 * count[i] > 0 (it touched a tile of the view: igs_frame::count), accum[i] +=
 * sqrt(du^2 + dv^2) of its screen-space position gradient (g2d [n][8], slots 0
 * and 1, from igs_blend_bwd; FP32, each step rounded once) and vis[i] += 1.
 * accum (float[n]) and vis (uint32[n]) are device, caller-owned, zeroed by the
 * caller when an interval starts. Asynchronous. */
IGS_API igs_status igs_grad_accum(const float* g2d, const uint32_t* count, int64_t n, float* accum, uint32_t* vis,
                                  void* stream);

/* Bytes of device scratch igs_densify needs for n Gaussians. */
IGS_API size_t igs_densify_work_bytes(int64_t n);

/* From the scene (stored parameters), its Adam moments m, v (same layout) and
 * the statistic (accum, vis over the steps since the last densify), writes the
 * new parameters and moments to out, out_m, out_v (device arrays of `capacity`
 * Gaussians, caller-owned, not overlapping any input) and their number to
 * *d_count (device int64). With parameters as stored (param_mode 1: log sigma
 * and the opacity logit; 0: sigma and opacity), Gaussian i is
 *   deleted  if opacity_i < op_min (op_min in the same parameterisation);
 *   divided  else, if vis_i > 0, accum_i > tau_g * vis_i (one FP32 product)
 *            and its scale (means_sigma slot 3) >= scale_min, into eight
 *            children, child c at mu + (+-h, +-h, +-h) with the sign of axis a
 *            from bit a of c ('-' for 0), h = sigma / 2 (sigma = exp(log sigma)
 *            in double rounded to FP32, or sigma itself), child scale log sigma
 *            - ln 2 (FP32) or sigma / 2; same opacity and colour; zero moments;
 *   kept     otherwise, with its moments.
 * Output in index order, children in place of their parent. When the result
 * would exceed capacity, only the first candidates (by index) that fit divide
 * (each adds 7); if even the kept Gaussians exceed it, the first capacity of
 * them are written. work: igs_densify_work_bytes(n) bytes of device scratch,
 * 16-byte aligned. Three launches, no host synchronisation.
 * Errors: NULL, misaligned or overlapping buffers, n or capacity outside
 * 0..2^31, a bad sh_degree or param_mode, a NaN threshold -> IGS_ERR_INVALID_ARG. */
IGS_API igs_status igs_densify(const igs_scene* scene, const igs_params* m, const igs_params* v, int32_t sh_degree,
                               int32_t param_mode, const float* accum, const uint32_t* vis, float op_min, float tau_g,
                               float scale_min, int64_t capacity, const igs_params* out, const igs_params* out_m,
                               const igs_params* out_v, int64_t* d_count, void* work, void* stream);

/* Bytes of device scratch igs_merge needs for n Gaussians (0 for n outside 0..2^30 - 1). */
IGS_API size_t igs_merge_work_bytes(int64_t n);

/* Merging of the 3D Gaussians (Sec. 3.2: particles are merged as well as
 * divided; Sec. 2.5: the scale of a particle follows the detail it covers;
 * Sec. 3.1's Octree as the pattern, so a merge undoes an octant division):
 * the grid has cells of side `cell` from the corner lo (host float[3]), at
 * most 1024 per axis; with inv = 1 / cell in FP32, Gaussian i lies in the cell
 * floor((mu_a - lo_a) * inv) on each axis a (each operation rounded once in
 * FP32). Gaussian i is eligible if its mean is finite, its stored scale
 * (means_sigma slot 3, as stored) <= scale_max, its stored opacity is in
 * [2^-60, 1] (param_mode 0) or its stored logit >= -41.58883f (param_mode 1,
 * the logit of 2^-60) and all three cell indices are in [0, 1024). The eligible Gaussians of one cell, two
 * or more of them, become one Gaussian at the place (in index order) of the
 * first; with o_k the linear opacity and sigma_k the linear scale of member k
 * (sums over the members in index order):
 *   W = sum o_k,  mu = sum o_k mu_k / W,
 *   sigma^2 = sum o_k (sigma_k^2 + |mu_k - mu|^2 / 3) / W,
 *   opacity = min(0.99, 1 - prod (1 - o_k)),  colour = sum o_k c_k / W,
 * stored in the input's parameterisation (param_mode 1: log sigma and the
 * opacity logit; 0: sigma and opacity), with zero Adam moments. Arithmetic:
 * FP32 with compensated sums and the means as offsets from the first member
 * (with u = 2^-24 and h = cell: mean within 32u h + 4u |mu| of the exact value,
 * scale within 64u relative, opacity within 16u relative, colour within
 * 16u max|c| + 4u |c|). Every other Gaussian is kept with its moments. Output in index
 * order to out, out_m, out_v (device arrays of at least n Gaussians,
 * caller-owned, not overlapping any input); their number to *d_count (device
 * int64; -1 if the device sort gave up on a bounded wait, nothing written).
 * work: igs_merge_work_bytes(n) bytes of device scratch, 16-byte aligned.
 * Twelve launches, no host synchronisation.
 * Errors: NULL, misaligned or overlapping buffers, n outside 0..2^30 - 1, a bad
 * sh_degree or param_mode, cell not finite and > 0, a NaN scale_max or a
 * non-finite lo -> IGS_ERR_INVALID_ARG. */
IGS_API igs_status igs_merge(const igs_scene* scene, const igs_params* m, const igs_params* v, int32_t sh_degree,
                             int32_t param_mode, const float* lo, float cell, float scale_max, const igs_params* out,
                             const igs_params* out_m, const igs_params* out_v, int64_t* d_count, void* work,
                             void* stream);

/* Bytes of device scratch igs_octree_init needs for `levels` (0..7; 0 otherwise). */
IGS_API size_t igs_octree_work_bytes(int32_t levels);

/* Octree initialisation of 3D Gaussians (Sec. 3.1: an Octree for 3D, as the
 * QuadTree for 2D; colour = the cell average, sigma = half the cell width) from a
 * coloured point set: points [n][3] and colors [n][3] (device FP32, RGB in
 * [0, 1], clamped), in the cube [lo, lo + side)^3 (lo: host float[3]; points
 * outside are clamped into the boundary cells, non-finite points ignored),
 * cells down to level `levels` (cube side / 2^levels, levels <= 7). Cell of a
 * point: i_a = clamp(floor((p_a - lo_a) * inv), 0, 2^levels - 1) with inv =
 * 2^levels / side in FP32, each step rounded once. Statistics use colours
 * quantised to 12 bits (exact integers). A cell's error is
 * max(0, sum_c (S2_c - S1_c^2 / n)) (double, one rounding per step), its key
 * the smaller of its error and its parent's key; cells with >= 2 points above
 * the finest level can split. Growth: from the root, split the splittable leaf
 * first in the order (key descending, id = (8^l - 1)/7 + Morton index
 * ascending), replacing it by its non-empty children, and stop when that would
 * make more than k_max leaves. Writes one Gaussian per non-empty leaf in id
 * order to means_sigma [k_max][4] (cell centre, double rounded once; sigma =
 * half the cell side, or its log with param_mode 1), opacity [k_max]
 * (`opacity` in (0, 1), or its logit with param_mode 1) and color [k_max][C]
 * (mean colour as RGB, C = 3, for sh_degree -1; for sh_degree 0..3 the DC
 * coefficient (mean - 1/2) / Y00 and zeros), and their number to *d_count
 * (device int32). work: igs_octree_work_bytes(levels) bytes of device scratch,
 * 16-byte aligned. Errors: n outside 0..2^31, levels outside 0..7, k_max < 1,
 * side <= 0, opacity outside (0, 1), bad sh_degree / param_mode, NULL or
 * misaligned buffers -> IGS_ERR_INVALID_ARG. */
IGS_API igs_status igs_octree_init(const float* points, const float* colors, int64_t n, const float* lo, float side,
                                   int32_t levels, int32_t k_max, float opacity, int32_t sh_degree,
                                   int32_t param_mode, float* means_sigma, float* opacity_out, float* color,
                                   int32_t* d_count, void* work, void* stream);

/* Bytes of device scratch igs_quadtree_init needs (0 for an invalid size). */
IGS_API size_t igs_quadtree_work_bytes(int32_t side, int32_t min_cell);

/* QuadTree initialisation (Sec. 3.1) of a square RGB image (device
 * [3][side][side], side a power of two <= 512): one particle per leaf cell, at
 * the cell centre, with A = the cell's mean colour and sigma = half the cell
 * width. Growth rule (the paper gives none): starting from the whole image,
 * split the leaf with the largest squared error about its mean colour, summed
 * over channels, while the leaves stay at most k_max (a split adds 3) and the
 * children are at least min_cell pixels wide. The errors use the image
 * quantised to 12 bits, q = rint(clamp(v, 0, 1) 4096), as exact integers; the
 * key is T / n in double, T = sum_c n S2_c - S1_c^2 over the cell's n pixels;
 * ties go to the lower level, then the upper row, then the left column.
 * A_c = S1_c / (4096 n) (double, rounded once to float); log sigma =
 * log2(width / 2) ln 2 (double, rounded once). Writes the particles in (level,
 * row, column) order to particles (device, >= k_max x 8 floats, 16-byte
 * aligned) and their number to *d_count (device int32). work: device scratch
 * of igs_quadtree_work_bytes(side, min_cell) bytes, 16-byte aligned. */
IGS_API igs_status igs_quadtree_init(const float* img, int32_t side, int32_t k_max, int32_t min_cell,
                                     float* particles, int32_t* d_count, void* work, void* stream);

/* One bias-corrected Adam step (step >= 1) in place on p, m, v (device,
 * count FP32 each), from gradient g. The host scalars are double so that 1 - b1,
 * 1 - b2 and the bias corrections are formed exactly before rounding to FP32:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr (m/(1-b1^step)) / (sqrt(v/(1-b2^step)) + eps). */
IGS_API igs_status igs_adam(float* p, const float* g, float* m, float* v, int64_t count, double lr, double b1,
                            double b2, double eps, int64_t step, void* stream);

/* Copy the frame's four status words to host_info (host, 4 uint32) and wait for
 * `stream`. Returns the recorded device error (IGS_OK if none). Synchronous. */
IGS_API igs_status igs_frame_status(const igs_frame* frame, uint32_t* host_info, void* stream);

/* For failure-detection tests (the paper has no counterpart): the next
 * igs_bin_sort in this process runs its first depth-sort pass with one block
 * that never publishes its digit counts, so every later block's bounded wait
 * for them runs out (about half a second). Those blocks record
 * IGS_ERR_DEVICE_TIMEOUT, the frame is aborted (later kernels of the frame skip
 * their work and leave their outputs untouched) and igs_frame_status reports
 * the error; the GPU context stays usable. Needs n > 8192 (three or more
 * blocks). Host-only, takes effect once. */
IGS_API void igs_debug_silence_lookback_once(void);

/* Walk segments (observability; the paper has no counterpart). With 16- and
 * 32-pixel tiles the forward blend (igs_render_fwd) cuts the walk of an 8 x 8
 * pixel block through its tile's entries every 1024 list positions where the
 * block has blended since the previous cut, and saves the pixels' state there,
 * so that igs_blend_bwd walks the pieces in parallel (Eq. 4's adjoint is the same;
 * only the order of the additions changes). Writes to *host_count the pool slots
 * the last forward of this frame took (cut segments, and at most one slot per
 * block taken ahead and left unused); -1 when the frame has no segments (8-pixel
 * tiles, or no room). Waits for `stream`. Synchronous. */
IGS_API igs_status igs_frame_walk_segments(const igs_frame* frame, int64_t* host_count, void* stream);

/* Clear the frame's status words (asynchronous). */
IGS_API igs_status igs_frame_reset_status(igs_frame* frame, void* stream);

/* ---------------------------------------------------------------------------
 * Multi-view batch: V views of one scene, each with its own pose and image
 * size, rendered by one chain of launches with no host synchronisation: one
 * projection launch over every (view, Gaussian), each view's binning (depth
 * sort and tile lists, as igs_bin_sort) on one of up to 16 streams that run
 * concurrently, and one blend launch over the tiles of every view (the
 * hardware block scheduler, or for the persistent variant an atomic work
 * counter, balances views of different sizes). The chain can be captured in a
 * CUDA graph once and replayed with new poses. Each view's image is
 * bit-identical to rendering it alone with igs_project / igs_bin_sort /
 * igs_render_fwd.
 * ------------------------------------------------------------------------- */
#define IGS_MAX_VIEWS 256

typedef struct igs_batch {
    int64_t n;                  /* Gaussians */
    int64_t capacity;           /* (Gaussian, tile) entries over all views: the sum of view_capacity */
    int32_t views;              /* V, 1 .. IGS_MAX_VIEWS */
    int32_t tile;               /* 8, 16 or 32 */
    int32_t blend_batch;        /* entries staged per shared-memory batch in the blend */
    int32_t persistent_blocks;  /* CTAs of the persistent blend (set by igs_batch_set_views) */
    int64_t tiles_total;        /* tiles over all views */
    int64_t image_floats;       /* size of the packed image buffer: sum over views of 3 W H */
    int64_t image_offset[IGS_MAX_VIEWS];  /* first float of view v's [3][H][W] image */
    uint32_t tile_base[IGS_MAX_VIEWS];    /* global id of view v's first tile (blend work items) */
    int32_t width[IGS_MAX_VIEWS], height[IGS_MAX_VIEWS];
    int64_t view_capacity[IGS_MAX_VIEWS]; /* entries of view v's frame */
    int64_t frame_offset[IGS_MAX_VIEWS];  /* byte offset of view v's frame in the workspace */
    char* workspace;            /* the caller's buffer (device) */
    uint32_t* info;             /* [16] status words of the batch: info[0] = entries of all views, info[2]
                                   = the first error of a view, info[3] = entries all views need */
    uint32_t* view_entries;     /* [V] entries of each view (device), after igs_render_batch */
    void* table;                /* device view table (poses, frame pointers), written by igs_batch_set_views */
    void* fanout;               /* library-owned host object: the streams the views' binnings fan out
                                   to; made by igs_batch_set_views, freed by igs_batch_release */
} igs_batch;

/* Lay out a batch for n Gaussians and the V cameras' image sizes (the poses may
 * change later, the sizes may not). Each view gets a frame of its own (as from
 * igs_frame_layout) with capacities[v] entries (host array of V);
 * blend_batch = entries per shared-memory batch of the blend: 32 or 64 for tile
 * 8, 64, 128 or 256 for tile 16, 64, 256, 512 or 1024 for tile 32 (0 = tile^2).
 * 64 with tile 16 or 32 selects the sub-tile blend: one 64-thread CTA per 8 x 8
 * pixel block, walking its tile's entries and stopping on its own (not
 * persistent); the others run the persistent whole-tile blend.
 * workspace == NULL: only *bytes. Host-only, no launch. Laying out a batch
 * struct again forgets its fan-out streams: igs_batch_release it first. */
IGS_API igs_status igs_batch_layout(int64_t n, int32_t views, const igs_camera* cams, const igs_opts* opts,
                                    const int64_t* capacities, int32_t blend_batch, void* workspace, size_t* bytes,
                                    igs_batch* batch);

/* Upload the V cameras (same sizes as at layout) and the views' frame pointers
 * to the batch's device view table, asynchronously on `stream` (cams may be
 * reused on return). Call it before igs_render_batch whenever the poses
 * change, outside any stream capture. The first call also makes the batch's
 * fan-out streams (min(V, 8) CUDA streams and their events; no device memory). */
IGS_API igs_status igs_batch_set_views(igs_batch* batch, const igs_camera* cams, const igs_opts* opts,
                                       void* stream);

/* Render every view of the batch into `images` (device, batch->image_floats
 * floats; view v at image_offset[v], [3][H][W]): one projection launch for all
 * views (poses read from the view table), then each view's binning (as
 * igs_bin_sort) on one of the fan-out streams, joined back into `stream`, then
 * one blend launch over every view's tiles. No host synchronisation, so the
 * call can be captured in a CUDA graph (the fan-out streams join the capture).
 * A view whose entries overflow its frame leaves its image untouched; info[2]
 * = IGS_ERR_CAPACITY and info[3] = the entries the views need. */
IGS_API igs_status igs_render_batch(igs_batch* batch, const igs_scene* scene, const igs_opts* opts, float* images,
                                    void* stream);

/* Copy the batch's four status words to host_info and wait for `stream`. */
IGS_API igs_status igs_batch_status(const igs_batch* batch, uint32_t* host_info, void* stream);

/* Free the batch's fan-out streams and events (after its work has finished).
 * The workspace is the caller's. Safe on a batch that never made them. */
IGS_API void igs_batch_release(igs_batch* batch);

/* ---------------------------------------------------------------------------
 * Render server with continuous batching. Scenes stay resident (the caller
 * keeps their buffers alive); requests are queued and admitted in arrival
 * order as soon as a slot (a CUDA stream) is free and the request's frame
 * workspace fits in the caller's device pool, so requests that arrive while
 * others run overlap with them on the GPU. The entries a request needs are
 * sized from earlier requests of the same scene and image size; a request that
 * overflows is re-queued at the head with the capacity it reported. With
 * grouping on (igs_serve_set_grouping), requests of one scene that wait
 * together share one batched chain of launches. One host thread per server
 * schedules; the library allocates no device memory (the pool is the caller's)
 * and 80 bytes of pinned host memory per slot.
 * ------------------------------------------------------------------------- */
typedef struct igs_server igs_server;

typedef struct igs_timing {
    int64_t arrival_ns;  /* submit time (steady clock) */
    int64_t admit_ns;    /* slot and memory granted */
    int64_t start_ns;    /* first launch enqueued */
    int64_t done_ns;     /* completion seen by the scheduler */
    uint32_t entries;    /* (Gaussian, tile) entries of the view */
    int32_t status;      /* igs_status of the request */
    int32_t retries;     /* re-queues after a capacity overflow */
    int32_t group;       /* views rendered by the same chain of launches (1: alone) */
} igs_timing;

/* Create a server on the current device. pool (device, 256-byte aligned,
 * pool_bytes) holds every in-flight frame workspace; max_slots (1..64) requests
 * run at once, each on its own stream. opts->tile, thresholds and background
 * apply to every request; sh_degree / param_mode come with each scene. */
IGS_API igs_status igs_serve_create(void* pool, size_t pool_bytes, int32_t max_slots, const igs_opts* opts,
                                    igs_server** out);
/* Grouping: requests of one scene that wait together (among the first 64
 * queued) are rendered, up to max_views of them, by one batched chain of
 * launches (igs_render_batch: one projection, binning and blend launch for all
 * of them) on one slot, each image then copied to its request's output. The
 * pixels are those of rendering each request alone. 1 (the default) renders
 * every request by itself; 1 <= max_views <= 16. A group whose entries
 * overflow is split: its requests are redone one by one. Takes effect for
 * admissions after the call. */
IGS_API igs_status igs_serve_set_grouping(igs_server* server, int32_t max_views);
/* Register a resident scene (device buffers, layout as above); *scene_id
 * identifies it in igs_serve_submit. */
IGS_API igs_status igs_serve_add_scene(igs_server* server, const igs_scene* scene, int32_t sh_degree,
                                       int32_t param_mode, int32_t* scene_id);
/* Queue one render of scene_id from cam into img_out (device, [3][H][W]);
 * returns at once with *req_id. IGS_ERR_CAPACITY if even an empty frame of this
 * size cannot fit the pool. */
IGS_API igs_status igs_serve_submit(igs_server* server, int32_t scene_id, const igs_camera* cam, float* img_out,
                                    uint64_t* req_id);
/* Wait up to timeout_ns for request req_id; IGS_ERR_NOT_READY if it is still
 * running (poll again), otherwise the request's status, its timings in *t, and
 * the request is forgotten (poll a finished request once). */
IGS_API igs_status igs_serve_poll(igs_server* server, uint64_t req_id, int64_t timeout_ns, igs_timing* t);
/* Queue length, requests in flight, pool bytes in use and the peak in use. */
IGS_API igs_status igs_serve_stats(igs_server* server, int64_t* pending, int64_t* in_flight, int64_t* pool_used,
                                   int64_t* pool_peak);
/* Finish every queued request, then free the server's streams and host state. */
IGS_API void igs_serve_destroy(igs_server* server);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all threads). For accounting in benchmarks; host-only, never fails. */
IGS_API uint64_t igs_launch_count(void);

IGS_API const char* igs_status_string(igs_status s);
IGS_API const char* igs_last_error(void);
IGS_API int32_t igs_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IGS_H */
