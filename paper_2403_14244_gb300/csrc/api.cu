// C ABI of libigs (declared in include/igs.h): argument checks, frame layout,
// and the launches of each step. Nothing here allocates device memory.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "fit2d.cuh"

namespace igs {
std::atomic<uint64_t> g_launches{0};
thread_local const char* g_failed_call = nullptr;
}

namespace {

thread_local char g_last_error[512] = "";

igs_status fail(igs_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
igs_status fail(igs_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return s;
}

igs_status cuda_status(cudaError_t e, const char* what) {
    const char* call = igs::g_failed_call;
    igs::g_failed_call = nullptr;
    if (e == cudaSuccess) return IGS_OK;
    if (call) return fail(IGS_ERR_CUDA, "%s: %s (at %.160s)", what, cudaGetErrorString(e), call);
    return fail(IGS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace igs {
igs_status report_cuda(cudaError_t e, const char* what) { return cuda_status(e, what); }
igs_status report_invalid(const char* msg) { return fail(IGS_ERR_INVALID_ARG, "%s", msg); }
}  // namespace igs

namespace {

igs_status check_camera(const igs_camera* cam) {
    if (!cam) return fail(IGS_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width <= 0 || cam->height <= 0) return fail(IGS_ERR_INVALID_ARG, "image size must be positive");
    if (!(cam->fx > 0.f) || cam->fx != cam->fy)
        return fail(IGS_ERR_INVALID_ARG, "fx must be positive and equal fy (isotropic discs)");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(cam->R[i])) return fail(IGS_ERR_INVALID_ARG, "camera R not finite");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(cam->t[i])) return fail(IGS_ERR_INVALID_ARG, "camera t not finite");
    if (!std::isfinite(cam->cx) || !std::isfinite(cam->cy) || !std::isfinite(cam->znear))
        return fail(IGS_ERR_INVALID_ARG, "camera intrinsics not finite");
    return IGS_OK;
}

igs_status check_opts(const igs_opts* o) {
    if (!o) return fail(IGS_ERR_INVALID_ARG, "opts is NULL");
    if (o->tile != 8 && o->tile != 16 && o->tile != 32) return fail(IGS_ERR_INVALID_ARG, "tile must be 8, 16 or 32");
    if (o->sh_degree < -1 || o->sh_degree > 3) return fail(IGS_ERR_INVALID_ARG, "sh_degree must be -1..3");
    if (o->param_mode != 0 && o->param_mode != 1) return fail(IGS_ERR_INVALID_ARG, "param_mode must be 0 or 1");
    if (o->footprint != 0 && o->footprint != 1) return fail(IGS_ERR_INVALID_ARG, "footprint must be 0 or 1");
    if (!(o->alpha_min >= 1.0f / 255.0f) || !(o->alpha_max <= 1.f) || !(o->alpha_min < o->alpha_max) ||
        !(o->t_min > 0.f) || !(o->t_min < 1.f))
        return fail(IGS_ERR_INVALID_ARG,
                    "need 1/255 <= alpha_min < alpha_max <= 1 and 0 < t_min < 1 (the footprint holds alpha >= 1/255)");
    return IGS_OK;
}

igs_status check_scene(const igs_scene* s) {
    if (!s) return fail(IGS_ERR_INVALID_ARG, "scene is NULL");
    if (s->n < 0 || s->n >= ((int64_t)1 << 31)) return fail(IGS_ERR_INVALID_ARG, "n out of range");
    if (s->n > 0 && (!s->means_sigma || !s->opacity || !s->color))
        return fail(IGS_ERR_INVALID_ARG, "scene buffer is NULL");
    if (reinterpret_cast<uintptr_t>(s->means_sigma) & 15)
        return fail(IGS_ERR_INVALID_ARG, "means_sigma must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(s->color) & 15)
        return fail(IGS_ERR_INVALID_ARG, "color must be 16-byte aligned");
    return IGS_OK;
}

igs_status check_frame(const igs_frame* f) {
    if (!f || !f->info || !f->rec) return fail(IGS_ERR_INVALID_ARG, "frame is NULL or not laid out");
    return IGS_OK;
}

igs::ViewParams view_params(const igs_camera* c, const igs_opts* o, const igs_frame* f) {
    igs::ViewParams v;
    std::memcpy(v.R, c->R, sizeof v.R);
    std::memcpy(v.t, c->t, sizeof v.t);
    v.fx = c->fx; v.fy = c->fy; v.cx = c->cx; v.cy = c->cy; v.znear = c->znear;
    v.alpha_min = o->alpha_min;
    for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int r = 0; r < 3; ++r) acc -= (double)c->R[3 * r + a] * (double)c->t[r];
        v.cam_center[a] = (float)acc;
    }
    v.width = c->width; v.height = c->height;
    v.tile = o->tile;
    v.tiles_x = f ? f->tiles_x : (c->width + o->tile - 1) / o->tile;
    v.tiles_y = f ? f->tiles_y : (c->height + o->tile - 1) / o->tile;
    v.sh_degree = o->sh_degree;
    v.param_mode = o->param_mode;
    v.footprint = o->footprint;
    return v;
}

igs::BlendParams blend_params(const igs_frame* f, const igs_opts* o) {
    igs::BlendParams b;
    b.width = f->width; b.height = f->height; b.tiles_x = f->tiles_x; b.tiles_y = f->tiles_y;
    b.alpha_min = o->alpha_min; b.alpha_max = o->alpha_max; b.t_min = o->t_min;
    for (int i = 0; i < 3; ++i) b.bg[i] = o->bg[i];
    return b;
}

}  // namespace

extern "C" {

int32_t igs_abi_version(void) { return IGS_ABI_VERSION; }

uint64_t igs_launch_count(void) { return igs::g_launches.load(std::memory_order_relaxed); }

const char* igs_last_error(void) { return g_last_error; }

const char* igs_status_string(igs_status s) {
    switch (s) {
        case IGS_OK: return "ok";
        case IGS_ERR_INVALID_ARG: return "invalid argument";
        case IGS_ERR_OOM: return "buffer too small";
        case IGS_ERR_CUDA: return "CUDA error";
        case IGS_ERR_CAPACITY: return "entry capacity exceeded";
        case IGS_ERR_NOT_READY: return "not ready";
        case IGS_ERR_DEVICE_TIMEOUT: return "device wait timed out";
        case IGS_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

igs_status igs_frame_layout(int64_t n, int64_t capacity, const igs_camera* cam, const igs_opts* opts,
                            void* workspace, size_t* bytes, igs_frame* frame) {
    igs_status st;
    if ((st = check_camera(cam)) != IGS_OK || (st = check_opts(opts)) != IGS_OK) return st;
    if (!bytes) return fail(IGS_ERR_INVALID_ARG, "bytes is NULL");
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(IGS_ERR_INVALID_ARG, "n out of range");
    if (capacity < 0 || capacity >= ((int64_t)1 << 30)) return fail(IGS_ERR_INVALID_ARG, "capacity must be < 2^30");
    const int64_t tx = (cam->width + opts->tile - 1) / opts->tile, ty = (cam->height + opts->tile - 1) / opts->tile;
    if (tx >= 65536 || ty >= 65536) return fail(IGS_ERR_INVALID_ARG, "too many tiles per axis");
    const int64_t tiles = tx * ty, P = (int64_t)cam->width * cam->height;
    size_t off = 0;
    size_t o_rec = off; off += align256((size_t)n * 32);
    size_t o_rect = off; off += align256((size_t)n * 8);
    size_t o_disc = off; off += align256((size_t)n * 16);
    size_t o_count = off; off += align256((size_t)n * 4);
    size_t o_dkey = off; off += align256((size_t)n * 4);
    size_t o_order = off; off += align256((size_t)n * 4);
    size_t o_offset = off; off += align256((size_t)n * 4);
    size_t o_ranges = off; off += align256((size_t)tiles * 8);
    size_t o_T = off; off += align256((size_t)P * 4);
    size_t o_nc = off; off += align256((size_t)P * 4);
    size_t o_info = off; off += align256(igs::kInfoWords * 4);
    size_t o_scr = off;
    const int64_t chunks = igs::sort_walk_chunks(tx, ty);
    const size_t scr = igs::sort_scratch_bytes(n, capacity, tx, ty, chunks);
    off += align256(scr);
    *bytes = off;
    if (!workspace) return IGS_OK;
    if (!frame) return fail(IGS_ERR_INVALID_ARG, "frame is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return fail(IGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    char* b = static_cast<char*>(workspace);
    std::memset(frame, 0, sizeof *frame);
    frame->n = n;
    frame->capacity = capacity;
    frame->width = cam->width;
    frame->height = cam->height;
    frame->tile = opts->tile;
    frame->tiles_x = (int32_t)tx;
    frame->tiles_y = (int32_t)ty;
    frame->sort_chunks = (int32_t)chunks;
    frame->rec = reinterpret_cast<float*>(b + o_rec);
    frame->rect = reinterpret_cast<uint32_t*>(b + o_rect);
    frame->disc = reinterpret_cast<float*>(b + o_disc);
    frame->count = reinterpret_cast<uint32_t*>(b + o_count);
    frame->depth_key = reinterpret_cast<uint32_t*>(b + o_dkey);
    frame->order = reinterpret_cast<uint32_t*>(b + o_order);
    frame->offset = reinterpret_cast<uint32_t*>(b + o_offset);
    frame->ranges = reinterpret_cast<uint32_t*>(b + o_ranges);
    frame->T_final = reinterpret_cast<float*>(b + o_T);
    frame->n_contrib = reinterpret_cast<uint32_t*>(b + o_nc);
    frame->info = reinterpret_cast<uint32_t*>(b + o_info);
    frame->scratch = b + o_scr;
    frame->scratch_bytes = scr;
    // vals and tile_key live in the sort's entry buffers: a frame costs 12 bytes per
    // entry of capacity (counting sort: vals, and the 8-byte level-1 items whose
    // buffer later takes tile_key) or 16 (radix tile passes: the ping-pong item
    // buffers, each free when they are written)
    const igs::SortScratch ss = igs::sort_scratch(*frame);
    frame->vals = ss.vals;
    frame->tile_key = ss.tile_key;
    return IGS_OK;
}

static igs_status frame_matches(const igs_frame* f, const igs_scene* s, const igs_camera* cam, const igs_opts* o) {
    if (s && s->n != f->n) return fail(IGS_ERR_INVALID_ARG, "frame laid out for n=%lld, scene has %lld",
                                       (long long)f->n, (long long)s->n);
    if (cam && (cam->width != f->width || cam->height != f->height))
        return fail(IGS_ERR_INVALID_ARG, "frame laid out for another image size");
    if (o && o->tile != f->tile) return fail(IGS_ERR_INVALID_ARG, "frame laid out for another tile size");
    return IGS_OK;
}

igs_status igs_project(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts, igs_frame* frame,
                       void* stream) {
    igs_status st;
    if ((st = check_scene(scene)) || (st = check_camera(cam)) || (st = check_opts(opts)) || (st = check_frame(frame)) ||
        (st = frame_matches(frame, scene, cam, opts)))
        return st;
    const igs::ViewParams vp = view_params(cam, opts, frame);
    return cuda_status(igs::launch_project(*scene, vp, *frame, (cudaStream_t)stream), "igs_project");
}

igs_status igs_bin_sort(igs_frame* frame, const igs_opts* opts, void* stream) {
    igs_status st;
    if ((st = check_opts(opts)) || (st = check_frame(frame)) || (st = frame_matches(frame, nullptr, nullptr, opts)))
        return st;
    return cuda_status(igs::launch_bin_sort(*frame, opts->footprint, (cudaStream_t)stream), "igs_bin_sort");
}

igs_status igs_export_keys(const igs_frame* frame, uint64_t* keys, void* stream) {
    igs_status st;
    if ((st = check_frame(frame))) return st;
    if (!keys) return fail(IGS_ERR_INVALID_ARG, "keys is NULL");
    return cuda_status(igs::launch_export_keys(*frame, keys, (cudaStream_t)stream), "igs_export_keys");
}

igs_status igs_render_fwd(igs_frame* frame, const igs_opts* opts, float* img, void* stream) {
    igs_status st;
    if ((st = check_opts(opts)) || (st = check_frame(frame)) || (st = frame_matches(frame, nullptr, nullptr, opts)))
        return st;
    if (!img) return fail(IGS_ERR_INVALID_ARG, "img is NULL");
    const igs::BlendParams bp = blend_params(frame, opts);
    return cuda_status(igs::launch_blend_fwd(*frame, bp, img, (cudaStream_t)stream), "igs_render_fwd");
}

igs_status igs_render_fwd_clear(igs_frame* frame, const igs_opts* opts, float* img, float* g2d, void* stream) {
    igs_status st;
    if ((st = check_opts(opts)) || (st = check_frame(frame)) || (st = frame_matches(frame, nullptr, nullptr, opts)))
        return st;
    if (!img || !g2d) return fail(IGS_ERR_INVALID_ARG, "img or g2d is NULL");
    if (reinterpret_cast<uintptr_t>(g2d) & 15) return fail(IGS_ERR_INVALID_ARG, "g2d must be 16-byte aligned");
    const igs::BlendParams bp = blend_params(frame, opts);
    return cuda_status(igs::launch_blend_fwd(*frame, bp, img, (cudaStream_t)stream, g2d), "igs_render_fwd_clear");
}

igs_status igs_blend_bwd_acc(const igs_frame* frame, const igs_opts* opts, const float* dL_dimg, float* g2d,
                             void* stream) {
    igs_status st;
    if ((st = check_opts(opts)) || (st = check_frame(frame)) || (st = frame_matches(frame, nullptr, nullptr, opts)))
        return st;
    if (!dL_dimg || !g2d) return fail(IGS_ERR_INVALID_ARG, "dL_dimg or g2d is NULL");
    if (reinterpret_cast<uintptr_t>(g2d) & 15) return fail(IGS_ERR_INVALID_ARG, "g2d must be 16-byte aligned");
    const igs::BlendParams bp = blend_params(frame, opts);
    return cuda_status(igs::launch_blend_bwd(*frame, bp, dL_dimg, g2d, (cudaStream_t)stream), "igs_blend_bwd_acc");
}

igs_status igs_blend_bwd(const igs_frame* frame, const igs_opts* opts, const float* dL_dimg, float* g2d,
                         void* stream) {
    igs_status st;
    if ((st = check_opts(opts)) || (st = check_frame(frame)) || (st = frame_matches(frame, nullptr, nullptr, opts)))
        return st;
    if (!dL_dimg || !g2d) return fail(IGS_ERR_INVALID_ARG, "dL_dimg or g2d is NULL");
    if (reinterpret_cast<uintptr_t>(g2d) & 15) return fail(IGS_ERR_INVALID_ARG, "g2d must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    igs::ZeroRanges z = {};
    if (frame->n > 0) {
        z.ptr[z.count] = g2d;
        z.bytes[z.count++] = (unsigned long long)frame->n * 32;
    }
    if (void* next = igs::blend_bwd_counter(*frame)) {  // the backward's work counter
        z.ptr[z.count] = next;
        z.bytes[z.count++] = 4;
    }
    cudaError_t e = igs::launch_zero(z, s);
    if (e != cudaSuccess) return cuda_status(e, "igs_blend_bwd");
    const igs::BlendParams bp = blend_params(frame, opts);
    return cuda_status(igs::launch_blend_bwd(*frame, bp, dL_dimg, g2d, s), "igs_blend_bwd");
}

igs_status igs_project_bwd(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                           const igs_frame* frame, const float* g2d, float* d_means_sigma, float* d_opacity,
                           float* d_color, void* stream) {
    igs_status st;
    if ((st = check_scene(scene)) || (st = check_camera(cam)) || (st = check_opts(opts)) || (st = check_frame(frame)) ||
        (st = frame_matches(frame, scene, cam, opts)))
        return st;
    if (!g2d || !d_means_sigma || !d_opacity || !d_color) return fail(IGS_ERR_INVALID_ARG, "gradient buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(g2d) | reinterpret_cast<uintptr_t>(d_means_sigma)) & 15)
        return fail(IGS_ERR_INVALID_ARG, "g2d and d_means_sigma must be 16-byte aligned");
    const igs::ViewParams vp = view_params(cam, opts, frame);
    return cuda_status(igs::launch_project_bwd(*scene, vp, *frame, g2d, d_means_sigma, d_opacity, d_color,
                                               (cudaStream_t)stream),
                       "igs_project_bwd");
}

static igs_status adam_params(double lr, double b1, double b2, double eps, int64_t step, igs::AdamParams* a) {
    if (step < 1) return fail(IGS_ERR_INVALID_ARG, "Adam step must be >= 1");
    if (!(b1 >= 0.0 && b1 < 1.0 && b2 >= 0.0 && b2 < 1.0 && lr >= 0.0 && eps > 0.0))
        return fail(IGS_ERR_INVALID_ARG, "need 0 <= b1, b2 < 1, lr >= 0, eps > 0");
    const double bc1 = 1.0 - std::pow(b1, (double)step);
    const double bc2 = 1.0 - std::pow(b2, (double)step);
    a->b1 = (float)b1;
    a->b2 = (float)b2;
    a->omb1 = (float)(1.0 - b1);
    a->omb2 = (float)(1.0 - b2);
    a->step_size = (float)(lr / bc1);
    a->bc2_sqrt = (float)std::sqrt(bc2);
    a->inv_bc2_sqrt = (float)(1.0 / std::sqrt(bc2));
    a->eps = (float)eps;
    a->dev_consts = nullptr;
    return IGS_OK;
}

igs_status igs_project_bwd_adam(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                                const igs_frame* frame, const float* g2d, float* m_means_sigma, float* m_opacity,
                                float* m_color, float* v_means_sigma, float* v_opacity, float* v_color, double lr,
                                double b1, double b2, double eps, int64_t step, void* stream) {
    igs_status st;
    if ((st = check_scene(scene)) || (st = check_camera(cam)) || (st = check_opts(opts)) || (st = check_frame(frame)) ||
        (st = frame_matches(frame, scene, cam, opts)))
        return st;
    if (!g2d || !m_means_sigma || !m_opacity || !m_color || !v_means_sigma || !v_opacity || !v_color)
        return fail(IGS_ERR_INVALID_ARG, "g2d or an Adam moment buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(g2d) | reinterpret_cast<uintptr_t>(m_means_sigma) |
         reinterpret_cast<uintptr_t>(v_means_sigma) | reinterpret_cast<uintptr_t>(m_color) |
         reinterpret_cast<uintptr_t>(v_color)) & 15)
        return fail(IGS_ERR_INVALID_ARG, "g2d, means_sigma and color moments must be 16-byte aligned");
    igs::AdamParams a;
    if ((st = adam_params(lr, b1, b2, eps, step, &a))) return st;
    const igs::ViewParams vp = view_params(cam, opts, frame);
    return cuda_status(igs::launch_project_bwd_adam(*scene, vp, *frame, g2d, m_means_sigma, m_opacity, m_color,
                                                    v_means_sigma, v_opacity, v_color, a, (cudaStream_t)stream),
                       "igs_project_bwd_adam");
}

static igs_status project_bwd_adam_dev(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                                       const igs_frame* frame, const float* g2d, float* m_means_sigma,
                                       float* m_opacity, float* m_color, float* v_means_sigma, float* v_opacity,
                                       float* v_color, double lr, double b1, double b2, double eps, int32_t* d_state,
                                       const igs_camera* next_cam, const igs_frame* next_frame, void* stream,
                                       const char* name) {
    if (!d_state || (reinterpret_cast<uintptr_t>(d_state) & 15))
        return fail(IGS_ERR_INVALID_ARG, "d_state must be a 16-byte aligned device buffer of 4 words");
    igs_status st;
    if ((st = check_scene(scene)) || (st = check_camera(cam)) || (st = check_opts(opts)) || (st = check_frame(frame)) ||
        (st = frame_matches(frame, scene, cam, opts)))
        return st;
    if (next_cam && ((st = check_camera(next_cam)) || (st = check_frame(next_frame)) ||
                     (st = frame_matches(next_frame, scene, next_cam, opts))))
        return st;
    if (!g2d || !m_means_sigma || !m_opacity || !m_color || !v_means_sigma || !v_opacity || !v_color)
        return fail(IGS_ERR_INVALID_ARG, "g2d or an Adam moment buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(g2d) | reinterpret_cast<uintptr_t>(m_means_sigma) |
         reinterpret_cast<uintptr_t>(v_means_sigma) | reinterpret_cast<uintptr_t>(m_color) |
         reinterpret_cast<uintptr_t>(v_color)) & 15)
        return fail(IGS_ERR_INVALID_ARG, "g2d, means_sigma and color moments must be 16-byte aligned");
    igs::AdamParams a;
    if ((st = adam_params(lr, b1, b2, eps, 1, &a))) return st;  // b1, b2, eps; the step's constants come from d_state
    a.dev_consts = reinterpret_cast<const float*>(d_state + 1);
    const igs::ViewParams vp = view_params(cam, opts, frame);
    const igs::ViewParams vp_next = next_cam ? view_params(next_cam, opts, next_frame) : vp;
    cudaError_t e = igs::launch_adam_advance(d_state, lr, b1, b2, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e, name);
    return cuda_status(igs::launch_project_bwd_adam(*scene, vp, *frame, g2d, m_means_sigma, m_opacity, m_color,
                                                    v_means_sigma, v_opacity, v_color, a, (cudaStream_t)stream,
                                                    next_cam ? &vp_next : nullptr, next_cam ? next_frame : nullptr),
                       name);
}

igs_status igs_project_bwd_adam_dev(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                                    const igs_frame* frame, const float* g2d, float* m_means_sigma, float* m_opacity,
                                    float* m_color, float* v_means_sigma, float* v_opacity, float* v_color, double lr,
                                    double b1, double b2, double eps, int32_t* d_state, void* stream) {
    return project_bwd_adam_dev(scene, cam, opts, frame, g2d, m_means_sigma, m_opacity, m_color, v_means_sigma,
                                v_opacity, v_color, lr, b1, b2, eps, d_state, nullptr, nullptr, stream,
                                "igs_project_bwd_adam_dev");
}

igs_status igs_project_bwd_adam_next(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts,
                                     const igs_frame* frame, const float* g2d, float* m_means_sigma,
                                     float* m_opacity, float* m_color, float* v_means_sigma, float* v_opacity,
                                     float* v_color, double lr, double b1, double b2, double eps, int32_t* d_state,
                                     const igs_camera* next_cam, const igs_frame* next_frame, void* stream) {
    if (!next_cam || !next_frame) return fail(IGS_ERR_INVALID_ARG, "next_cam or next_frame is NULL");
    return project_bwd_adam_dev(scene, cam, opts, frame, g2d, m_means_sigma, m_opacity, m_color, v_means_sigma,
                                v_opacity, v_color, lr, b1, b2, eps, d_state, next_cam, next_frame, stream,
                                "igs_project_bwd_adam_next");
}

igs_status igs_render_bwd(const igs_scene* scene, const igs_camera* cam, const igs_opts* opts, const igs_frame* frame,
                          const float* dL_dimg, float* g2d, float* d_means_sigma, float* d_opacity, float* d_color,
                          void* stream) {
    igs_status st;
    if ((st = check_scene(scene)) || (st = check_camera(cam)) || (st = check_opts(opts)) || (st = check_frame(frame)) ||
        (st = frame_matches(frame, scene, cam, opts)))
        return st;
    if (!dL_dimg || !g2d || !d_means_sigma || !d_opacity || !d_color)
        return fail(IGS_ERR_INVALID_ARG, "gradient buffer is NULL");
    if ((st = igs_blend_bwd(frame, opts, dL_dimg, g2d, stream))) return st;
    return igs_project_bwd(scene, cam, opts, frame, g2d, d_means_sigma, d_opacity, d_color, stream);
}

igs_status igs_l1_loss(const float* img, const float* target, int64_t count, float* loss, float* dL_dimg,
                       void* stream) {
    if (!img || !target || !loss || !dL_dimg || count < 0) return fail(IGS_ERR_INVALID_ARG, "bad l1 arguments");
    return cuda_status(igs::launch_l1(img, target, count, loss, dL_dimg, (cudaStream_t)stream), "igs_l1_loss");
}

size_t igs_ssim_work_bytes(int32_t channels, int32_t height, int32_t width) {
    if (channels < 1 || height < 1 || width < 1) return 0;
    return igs::ssim_work_floats(channels, height, width) * sizeof(float);
}

igs_status igs_l1_ssim_loss(const float* img, const float* target, int32_t channels, int32_t height, int32_t width,
                            float lambda, float* loss, float* ssim, float* dL_dimg, void* work, void* stream) {
    if (!img || !target || !loss || !dL_dimg || !work) return fail(IGS_ERR_INVALID_ARG, "l1_ssim: NULL buffer");
    if (channels < 1 || channels > 65535 || height < 1 || width < 1)
        return fail(IGS_ERR_INVALID_ARG, "l1_ssim: channels must be 1..65535, height and width positive");
    if ((int64_t)channels * height * width >= ((int64_t)1 << 40))
        return fail(IGS_ERR_INVALID_ARG, "l1_ssim: image too large");
    if (!(lambda >= 0.f && lambda <= 1.f)) return fail(IGS_ERR_INVALID_ARG, "l1_ssim: lambda must be in [0, 1]");
    if (reinterpret_cast<uintptr_t>(work) & 15) return fail(IGS_ERR_INVALID_ARG, "l1_ssim: work not 16-byte aligned");
    return cuda_status(igs::launch_l1_ssim(img, target, channels, height, width, lambda, loss, ssim, dL_dimg,
                                           static_cast<float*>(work), (cudaStream_t)stream),
                       "igs_l1_ssim_loss");
}

// ------------------------------------------------------------ 2D fitting --

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

static igs_status check_fit2d(const float* particles, int32_t k, float D, int32_t width, int32_t height) {
    if (!particles && k > 0) return fail(IGS_ERR_INVALID_ARG, "fit2d: particles is NULL");
    if (!aligned16(particles)) return fail(IGS_ERR_INVALID_ARG, "fit2d: particles not 16-byte aligned");
    if (k < 0 || k > (1 << 27)) return fail(IGS_ERR_INVALID_ARG, "fit2d: k must be 0..2^27");
    if (width < 1 || height < 1 || width > (1 << 20) || height > (1 << 20))
        return fail(IGS_ERR_INVALID_ARG, "fit2d: width and height must be 1..2^20");
    if (!(D > 0.f)) return fail(IGS_ERR_INVALID_ARG, "fit2d: D must be positive");
    return IGS_OK;
}

igs_status igs_fit2d_render(const float* particles, int32_t k, float D, int32_t width, int32_t height, float* img,
                            void* stream) {
    igs_status st;
    if ((st = check_fit2d(particles, k, D, width, height))) return st;
    if (!img) return fail(IGS_ERR_INVALID_ARG, "fit2d_render: img is NULL");
    return cuda_status(igs::launch_fit2d_render(particles, k, D, width, height, img, (cudaStream_t)stream),
                       "igs_fit2d_render");
}

igs_status igs_fit2d_backward(const float* particles, int32_t k, float D, int32_t width, int32_t height,
                              const float* dL_dimg, float* d_particles, void* stream) {
    igs_status st;
    if ((st = check_fit2d(particles, k, D, width, height))) return st;
    if (!dL_dimg || (!d_particles && k > 0)) return fail(IGS_ERR_INVALID_ARG, "fit2d_backward: NULL buffer");
    return cuda_status(igs::launch_fit2d_backward(particles, k, D, width, height, dL_dimg, d_particles,
                                                  (cudaStream_t)stream),
                       "igs_fit2d_backward");
}

igs_status igs_fit2d_adam(float* particles, const float* d_particles, float* m, float* v, int32_t k,
                          const float* lr, double b1, double b2, double eps, int32_t* d_state, void* stream) {
    if (k < 0 || k > (1 << 27)) return fail(IGS_ERR_INVALID_ARG, "fit2d_adam: k must be 0..2^27");
    if (!lr || !d_state) return fail(IGS_ERR_INVALID_ARG, "fit2d_adam: lr or d_state is NULL");
    if (k > 0 && (!particles || !d_particles || !m || !v))
        return fail(IGS_ERR_INVALID_ARG, "fit2d_adam: NULL buffer");
    if (!aligned16(particles) || !aligned16(d_particles) || !aligned16(m) || !aligned16(v))
        return fail(IGS_ERR_INVALID_ARG, "fit2d_adam: buffers must be 16-byte aligned");
    if (!(b1 >= 0.0 && b1 < 1.0 && b2 >= 0.0 && b2 < 1.0 && eps > 0.0))
        return fail(IGS_ERR_INVALID_ARG, "fit2d_adam: need 0 <= b1, b2 < 1 and eps > 0");
    igs::Fit2dAdam a;
    for (int j = 0; j < 8; ++j) {
        if (!std::isfinite(lr[j]) || lr[j] < 0.f) return fail(IGS_ERR_INVALID_ARG, "fit2d_adam: lr must be >= 0");
        a.lr[j] = lr[j];
    }
    a.b1 = (float)b1;
    a.b2 = (float)b2;
    a.omb1 = (float)(1.0 - b1);
    a.omb2 = (float)(1.0 - b2);
    a.eps = (float)eps;
    a.b1d = b1;
    a.b2d = b2;
    return cuda_status(igs::launch_fit2d_adam(particles, d_particles, m, v, k, a, d_state, (cudaStream_t)stream),
                       "igs_fit2d_adam");
}

igs_status igs_fit2d_grad_accum(const float* d_particles, int32_t k, float* accum, void* stream) {
    if (k < 0 || k > (1 << 27)) return fail(IGS_ERR_INVALID_ARG, "fit2d_grad_accum: k must be 0..2^27");
    if (k > 0 && (!d_particles || !accum)) return fail(IGS_ERR_INVALID_ARG, "fit2d_grad_accum: NULL buffer");
    if (!aligned16(d_particles)) return fail(IGS_ERR_INVALID_ARG, "fit2d_grad_accum: d_particles must be 16-byte aligned");
    return cuda_status(igs::launch_fit2d_grad_accum(d_particles, k, accum, (cudaStream_t)stream),
                       "igs_fit2d_grad_accum");
}

igs_status igs_fit2d_densify(const float* particles, const float* m, const float* v, const float* accum, int32_t k,
                             int32_t n_iters, float tau_a, float tau_g, float log_sigma_min, int32_t capacity,
                             float* out, float* out_m, float* out_v, int32_t* d_count, void* stream) {
    if (k < 0 || k > (1 << 27)) return fail(IGS_ERR_INVALID_ARG, "fit2d_densify: k must be 0..2^27");
    if (capacity < 0 || capacity > (1 << 27)) return fail(IGS_ERR_INVALID_ARG, "fit2d_densify: capacity must be 0..2^27");
    if (n_iters < 1) return fail(IGS_ERR_INVALID_ARG, "fit2d_densify: n_iters must be >= 1");
    if (std::isnan(tau_a) || std::isnan(tau_g) || std::isnan(log_sigma_min))
        return fail(IGS_ERR_INVALID_ARG, "fit2d_densify: NaN threshold");
    if (!d_count) return fail(IGS_ERR_INVALID_ARG, "fit2d_densify: d_count is NULL");
    if (k > 0 && (!particles || !m || !v || !accum)) return fail(IGS_ERR_INVALID_ARG, "fit2d_densify: NULL input");
    if (capacity > 0 && (!out || !out_m || !out_v)) return fail(IGS_ERR_INVALID_ARG, "fit2d_densify: NULL output");
    if (!aligned16(particles) || !aligned16(m) || !aligned16(v) || !aligned16(out) || !aligned16(out_m) ||
        !aligned16(out_v))
        return fail(IGS_ERR_INVALID_ARG, "fit2d_densify: particle buffers must be 16-byte aligned");
    const auto overlaps = [](const float* a, int64_t na, const float* b, int64_t nb) {
        return a && b && na > 0 && nb > 0 && a < b + nb && b < a + na;
    };
    const int64_t ni = 8 * (int64_t)k, no = 8 * (int64_t)capacity;
    for (const float* o : {(const float*)out, (const float*)out_m, (const float*)out_v})
        for (const float* in : {particles, m, v})
            if (overlaps(o, no, in, ni)) return fail(IGS_ERR_INVALID_ARG, "fit2d_densify: outputs overlap inputs");
    const float thr = tau_g * (float)n_iters;  // one FP32 rounding
    return cuda_status(igs::launch_fit2d_densify(particles, m, v, accum, k, thr, tau_a, log_sigma_min, capacity, out,
                                                 out_m, out_v, d_count, (cudaStream_t)stream),
                       "igs_fit2d_densify");
}

igs_status igs_grad_accum(const float* g2d, const uint32_t* count, int64_t n, float* accum, uint32_t* vis,
                          void* stream) {
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(IGS_ERR_INVALID_ARG, "grad_accum: n out of range");
    if (n > 0 && (!g2d || !count || !accum || !vis)) return fail(IGS_ERR_INVALID_ARG, "grad_accum: NULL buffer");
    if (!aligned16(g2d)) return fail(IGS_ERR_INVALID_ARG, "grad_accum: g2d must be 16-byte aligned");
    return cuda_status(igs::launch_grad_accum3d(g2d, count, n, accum, vis, (cudaStream_t)stream), "igs_grad_accum");
}

size_t igs_densify_work_bytes(int64_t n) {
    if (n < 0 || n >= ((int64_t)1 << 31)) return 0;
    return igs::densify_work_bytes(n);
}

igs_status igs_densify(const igs_scene* scene, const igs_params* m, const igs_params* v, int32_t sh_degree,
                       int32_t param_mode, const float* accum, const uint32_t* vis, float op_min, float tau_g,
                       float scale_min, int64_t capacity, const igs_params* out, const igs_params* out_m,
                       const igs_params* out_v, int64_t* d_count, void* work, void* stream) {
    igs_status st;
    if ((st = check_scene(scene))) return st;
    if (!m || !v || !out || !out_m || !out_v || !d_count || !work)
        return fail(IGS_ERR_INVALID_ARG, "densify: NULL argument");
    if (sh_degree < -1 || sh_degree > 3) return fail(IGS_ERR_INVALID_ARG, "densify: sh_degree must be -1..3");
    if (param_mode != 0 && param_mode != 1) return fail(IGS_ERR_INVALID_ARG, "densify: param_mode must be 0 or 1");
    if (capacity < 0 || capacity >= ((int64_t)1 << 31)) return fail(IGS_ERR_INVALID_ARG, "densify: capacity out of range");
    if (std::isnan(op_min) || std::isnan(tau_g) || std::isnan(scale_min))
        return fail(IGS_ERR_INVALID_ARG, "densify: NaN threshold");
    const int64_t n = scene->n;
    const int C = sh_degree < 0 ? 3 : 3 * (sh_degree + 1) * (sh_degree + 1);
    if (n > 0 && (!accum || !vis || !m->means_sigma || !m->opacity || !m->color || !v->means_sigma || !v->opacity ||
                  !v->color))
        return fail(IGS_ERR_INVALID_ARG, "densify: NULL input array");
    const igs_params* outs[3] = {out, out_m, out_v};
    if (capacity > 0)
        for (const igs_params* o : outs)
            if (!o->means_sigma || !o->opacity || !o->color)
                return fail(IGS_ERR_INVALID_ARG, "densify: NULL output array");
    if (!aligned16(work)) return fail(IGS_ERR_INVALID_ARG, "densify: work must be 16-byte aligned");
    for (const igs_params* o : {m, v, out, out_m, out_v})
        if (!aligned16(o->means_sigma) || !aligned16(o->color))
            return fail(IGS_ERR_INVALID_ARG, "densify: means_sigma and color arrays must be 16-byte aligned");
    // no output array may overlap an input array
    struct Span { const void* p; size_t bytes; };
    const Span ins[] = {{scene->means_sigma, 16 * (size_t)n}, {scene->opacity, 4 * (size_t)n},
                        {scene->color, 4 * (size_t)C * n},    {m->means_sigma, 16 * (size_t)n},
                        {m->opacity, 4 * (size_t)n},          {m->color, 4 * (size_t)C * n},
                        {v->means_sigma, 16 * (size_t)n},     {v->opacity, 4 * (size_t)n},
                        {v->color, 4 * (size_t)C * n},        {accum, 4 * (size_t)n},
                        {vis, 4 * (size_t)n}};
    for (const igs_params* o : outs) {
        const Span os[] = {{o->means_sigma, 16 * (size_t)capacity}, {o->opacity, 4 * (size_t)capacity},
                           {o->color, 4 * (size_t)C * capacity}};
        for (const Span& a : os)
            for (const Span& b : ins) {
                const char *pa = (const char*)a.p, *pb = (const char*)b.p;
                if (pa && pb && a.bytes && b.bytes && pa < pb + b.bytes && pb < pa + a.bytes)
                    return fail(IGS_ERR_INVALID_ARG, "densify: an output overlaps an input");
            }
    }
    const float* in_p[3] = {scene->means_sigma, scene->opacity, scene->color};
    const float* in_m[3] = {m->means_sigma, m->opacity, m->color};
    const float* in_v[3] = {v->means_sigma, v->opacity, v->color};
    float* out_p[3] = {out->means_sigma, out->opacity, out->color};
    float* o_m[3] = {out_m->means_sigma, out_m->opacity, out_m->color};
    float* o_v[3] = {out_v->means_sigma, out_v->opacity, out_v->color};
    return cuda_status(igs::launch_densify(in_p, in_m, in_v, accum, vis, n, C, param_mode, op_min, tau_g, scale_min,
                                           capacity, out_p, o_m, o_v, d_count, work, (cudaStream_t)stream),
                       "igs_densify");
}

size_t igs_merge_work_bytes(int64_t n) {
    if (n < 0 || n >= ((int64_t)1 << 30)) return 0;
    return igs::merge_work_bytes(n);
}

igs_status igs_merge(const igs_scene* scene, const igs_params* m, const igs_params* v, int32_t sh_degree,
                     int32_t param_mode, const float* lo, float cell, float scale_max, const igs_params* out,
                     const igs_params* out_m, const igs_params* out_v, int64_t* d_count, void* work, void* stream) {
    igs_status st;
    if ((st = check_scene(scene))) return st;
    if (!m || !v || !out || !out_m || !out_v || !d_count || !work || !lo)
        return fail(IGS_ERR_INVALID_ARG, "merge: NULL argument");
    const int64_t n = scene->n;
    if (n >= ((int64_t)1 << 30)) return fail(IGS_ERR_INVALID_ARG, "merge: n must be below 2^30");
    if (sh_degree < -1 || sh_degree > 3) return fail(IGS_ERR_INVALID_ARG, "merge: sh_degree must be -1..3");
    if (param_mode != 0 && param_mode != 1) return fail(IGS_ERR_INVALID_ARG, "merge: param_mode must be 0 or 1");
    if (!(std::isfinite(cell) && cell > 0.f)) return fail(IGS_ERR_INVALID_ARG, "merge: cell must be finite and > 0");
    if (std::isnan(scale_max)) return fail(IGS_ERR_INVALID_ARG, "merge: NaN scale_max");
    if (!std::isfinite(lo[0]) || !std::isfinite(lo[1]) || !std::isfinite(lo[2]))
        return fail(IGS_ERR_INVALID_ARG, "merge: lo must be finite");
    const int C = sh_degree < 0 ? 3 : 3 * (sh_degree + 1) * (sh_degree + 1);
    const igs_params* arrays[5] = {m, v, out, out_m, out_v};
    if (n > 0)
        for (const igs_params* o : arrays)
            if (!o->means_sigma || !o->opacity || !o->color) return fail(IGS_ERR_INVALID_ARG, "merge: NULL array");
    if (!aligned16(work)) return fail(IGS_ERR_INVALID_ARG, "merge: work must be 16-byte aligned");
    for (const igs_params* o : arrays)
        if (!aligned16(o->means_sigma) || !aligned16(o->color))
            return fail(IGS_ERR_INVALID_ARG, "merge: means_sigma and color arrays must be 16-byte aligned");
    // no output array may overlap an input array or the scratch
    struct Span { const void* p; size_t bytes; };
    const size_t n_ = (size_t)n;
    const Span ins[] = {{scene->means_sigma, 16 * n_}, {scene->opacity, 4 * n_}, {scene->color, 4 * (size_t)C * n_},
                        {m->means_sigma, 16 * n_},     {m->opacity, 4 * n_},     {m->color, 4 * (size_t)C * n_},
                        {v->means_sigma, 16 * n_},     {v->opacity, 4 * n_},     {v->color, 4 * (size_t)C * n_},
                        {work, igs::merge_work_bytes(n)}};
    for (const igs_params* o : {out, out_m, out_v}) {
        const Span os[] = {{o->means_sigma, 16 * n_}, {o->opacity, 4 * n_}, {o->color, 4 * (size_t)C * n_}};
        for (const Span& a : os)
            for (const Span& b : ins) {
                const char *pa = (const char*)a.p, *pb = (const char*)b.p;
                if (pa && pb && a.bytes && b.bytes && pa < pb + b.bytes && pb < pa + a.bytes)
                    return fail(IGS_ERR_INVALID_ARG, "merge: an output overlaps an input or the scratch");
            }
    }
    const float* in_p[3] = {scene->means_sigma, scene->opacity, scene->color};
    const float* in_m[3] = {m->means_sigma, m->opacity, m->color};
    const float* in_v[3] = {v->means_sigma, v->opacity, v->color};
    float* out_p[3] = {out->means_sigma, out->opacity, out->color};
    float* o_m[3] = {out_m->means_sigma, out_m->opacity, out_m->color};
    float* o_v[3] = {out_v->means_sigma, out_v->opacity, out_v->color};
    return cuda_status(igs::launch_merge(in_p, in_m, in_v, n, C, param_mode, lo, cell, scale_max, out_p, o_m, o_v,
                                         d_count, work, (cudaStream_t)stream),
                       "igs_merge");
}

size_t igs_octree_work_bytes(int32_t levels) { return igs::octree_work_bytes(levels); }

igs_status igs_octree_init(const float* points, const float* colors, int64_t n, const float* lo, float side,
                           int32_t levels, int32_t k_max, float opacity, int32_t sh_degree, int32_t param_mode,
                           float* means_sigma, float* opacity_out, float* color, int32_t* d_count, void* work,
                           void* stream) {
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(IGS_ERR_INVALID_ARG, "octree_init: n out of range");
    if (levels < 0 || levels > 7) return fail(IGS_ERR_INVALID_ARG, "octree_init: levels must be 0..7");
    if (k_max < 1 || k_max > (1 << 27)) return fail(IGS_ERR_INVALID_ARG, "octree_init: k_max must be 1..2^27");
    if (!(side > 0.f) || !std::isfinite(side)) return fail(IGS_ERR_INVALID_ARG, "octree_init: side must be > 0");
    if (!(opacity > 0.f && opacity < 1.f)) return fail(IGS_ERR_INVALID_ARG, "octree_init: opacity must be in (0, 1)");
    if (sh_degree < -1 || sh_degree > 3 || (param_mode != 0 && param_mode != 1))
        return fail(IGS_ERR_INVALID_ARG, "octree_init: bad sh_degree or param_mode");
    if (!lo || !std::isfinite(lo[0]) || !std::isfinite(lo[1]) || !std::isfinite(lo[2]))
        return fail(IGS_ERR_INVALID_ARG, "octree_init: lo must be 3 finite floats");
    if ((n > 0 && (!points || !colors)) || !means_sigma || !opacity_out || !color || !d_count || !work)
        return fail(IGS_ERR_INVALID_ARG, "octree_init: NULL buffer");
    if (!aligned16(means_sigma) || !aligned16(work))
        return fail(IGS_ERR_INVALID_ARG, "octree_init: means_sigma and work must be 16-byte aligned");
    return cuda_status(igs::launch_octree_init(points, colors, n, lo, side, levels, k_max, opacity, sh_degree,
                                               param_mode, means_sigma, opacity_out, color, d_count, work,
                                               (cudaStream_t)stream),
                       "igs_octree_init");
}

size_t igs_quadtree_work_bytes(int32_t side, int32_t min_cell) {
    if (side < 1 || side > 512 || (side & (side - 1)) || min_cell < 1) return 0;
    return igs::quadtree_work_bytes(side, min_cell);
}

igs_status igs_quadtree_init(const float* img, int32_t side, int32_t k_max, int32_t min_cell, float* particles,
                             int32_t* d_count, void* work, void* stream) {
    if (side < 1 || side > 512 || (side & (side - 1)))
        return fail(IGS_ERR_INVALID_ARG, "quadtree_init: side must be a power of two <= 512");
    if (k_max < 1 || k_max > (1 << 27) || min_cell < 1)
        return fail(IGS_ERR_INVALID_ARG, "quadtree_init: need 1 <= k_max <= 2^27 and min_cell >= 1");
    if (!img || !particles || !d_count || !work) return fail(IGS_ERR_INVALID_ARG, "quadtree_init: NULL buffer");
    if (!aligned16(particles) || !aligned16(work))
        return fail(IGS_ERR_INVALID_ARG, "quadtree_init: particles and work must be 16-byte aligned");
    return cuda_status(igs::launch_quadtree_init(img, side, k_max, min_cell, particles, d_count, work,
                                                 (cudaStream_t)stream),
                       "igs_quadtree_init");
}

igs_status igs_adam(float* p, const float* g, float* m, float* v, int64_t count, double lr, double b1, double b2,
                    double eps, int64_t step, void* stream) {
    if (!p || !g || !m || !v || count < 0) return fail(IGS_ERR_INVALID_ARG, "bad adam arguments");
    igs::AdamParams a;
    igs_status st;
    if ((st = adam_params(lr, b1, b2, eps, step, &a))) return st;
    return cuda_status(igs::launch_adam(p, g, m, v, count, a, (cudaStream_t)stream), "igs_adam");
}

// ------------------------------------------------------------------- batch --

// View v's frame inside a batch workspace (the layout igs_frame_layout gives a
// view of that size with view_capacity[v] entries, at frame_offset[v]).
static igs_status batch_frame(const igs_batch* b, const igs_opts* opts, int v, igs_frame* f) {
    igs_camera cam;
    std::memset(&cam, 0, sizeof cam);
    cam.R[0] = cam.R[4] = cam.R[8] = 1.f;
    cam.fx = cam.fy = 1.f;
    cam.znear = 0.01f;
    cam.width = b->width[v];
    cam.height = b->height[v];
    size_t bytes = 0;
    return igs_frame_layout(b->n, b->view_capacity[v], &cam, opts, b->workspace + b->frame_offset[v], &bytes, f);
}

igs_status igs_batch_layout(int64_t n, int32_t views, const igs_camera* cams, const igs_opts* opts,
                            const int64_t* capacities, int32_t blend_batch, void* workspace, size_t* bytes,
                            igs_batch* batch) {
    igs_status st;
    if ((st = check_opts(opts))) return st;
    if (!bytes || !cams || !capacities) return fail(IGS_ERR_INVALID_ARG, "bytes, cams or capacities is NULL");
    if (views < 1 || views > IGS_MAX_VIEWS) return fail(IGS_ERR_INVALID_ARG, "views must be 1..%d", IGS_MAX_VIEWS);
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(IGS_ERR_INVALID_ARG, "n out of range");
    const int bb = blend_batch == 0 ? opts->tile * opts->tile : blend_batch;
    if (!igs::batch_blend_variant_ok(opts->tile, bb))
        return fail(IGS_ERR_INVALID_ARG, "unsupported blend batch %d for tile %d", bb, opts->tile);
    igs_batch b;
    std::memset(&b, 0, sizeof b);
    b.n = n;
    b.views = views;
    b.tile = opts->tile;
    b.blend_batch = bb;
    int64_t tiles = 0, floats = 0, cap = 0;
    size_t off = align256(4 * ((size_t)igs::kBatchCtrlWords + (size_t)views));  // status, work counter, entries
    const size_t o_table = off;
    off += align256(igs::batch_table_bytes(views));
    for (int v = 0; v < views; ++v) {
        if ((st = check_camera(&cams[v]))) return st;
        if (capacities[v] < 0 || capacities[v] >= ((int64_t)1 << 30))
            return fail(IGS_ERR_INVALID_ARG, "view %d: capacity must be in [0, 2^30)", v);
        const int64_t tx = (cams[v].width + opts->tile - 1) / opts->tile, ty = (cams[v].height + opts->tile - 1) / opts->tile;
        b.width[v] = cams[v].width;
        b.height[v] = cams[v].height;
        b.tile_base[v] = (uint32_t)tiles;
        b.image_offset[v] = floats;
        b.view_capacity[v] = capacities[v];
        tiles += tx * ty;
        floats += 3 * (int64_t)cams[v].width * cams[v].height;
        cap += capacities[v];
        size_t fb = 0;
        if ((st = igs_frame_layout(n, capacities[v], &cams[v], opts, nullptr, &fb, nullptr))) return st;
        b.frame_offset[v] = (int64_t)off;
        off += align256(fb);
    }
    if (tiles >= ((int64_t)1 << 31)) return fail(IGS_ERR_INVALID_ARG, "too many tiles");
    b.tiles_total = tiles;
    b.image_floats = floats;
    b.capacity = cap;
    *bytes = off;
    if (!workspace) return IGS_OK;
    if (!batch) return fail(IGS_ERR_INVALID_ARG, "batch is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return fail(IGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    char* w = static_cast<char*>(workspace);
    b.workspace = w;
    b.info = reinterpret_cast<uint32_t*>(w);
    b.view_entries = b.info + igs::kBatchCtrlWords;
    b.table = w + o_table;
    *batch = b;  // (no fan-out streams yet: igs_batch_set_views makes them)
    return IGS_OK;
}

igs_status igs_batch_set_views(igs_batch* batch, const igs_camera* cams, const igs_opts* opts, void* stream) {
    igs_status st;
    if (!batch || !batch->info || !cams) return fail(IGS_ERR_INVALID_ARG, "batch or cams is NULL");
    if ((st = check_opts(opts))) return st;
    if (opts->tile != batch->tile) return fail(IGS_ERR_INVALID_ARG, "batch laid out for another tile size");
    static thread_local igs::BatchView host[IGS_MAX_VIEWS];
    for (int v = 0; v < batch->views; ++v) {
        if ((st = check_camera(&cams[v]))) return st;
        if (cams[v].width != batch->width[v] || cams[v].height != batch->height[v])
            return fail(IGS_ERR_INVALID_ARG, "view %d: image size differs from the layout", v);
        igs_frame f;
        if ((st = batch_frame(batch, opts, v, &f))) return st;
        igs::BatchView& h = host[v];
        std::memset(&h, 0, sizeof h);
        h.vp = view_params(&cams[v], opts, &f);
        h.tile_base = batch->tile_base[v];
        h.img_off = batch->image_offset[v];
        h.rec = reinterpret_cast<float4*>(f.rec);
        h.rect = reinterpret_cast<uint2*>(f.rect);
        h.disc = reinterpret_cast<float4*>(f.disc);
        h.count = f.count;
        h.depth_key = f.depth_key;
        h.ranges = reinterpret_cast<const uint2*>(f.ranges);
        h.vals = f.vals;
        h.info = f.info;
    }
    cudaError_t e = igs::batch_fanout_make(*batch);
    if (e != cudaSuccess) return cuda_status(e, "igs_batch_set_views (fan-out streams)");
    const int pb = igs::batch_persistent_blocks(batch->tile, batch->blend_batch);
    if (pb <= 0) return fail(IGS_ERR_CUDA, "could not size the persistent blend");
    batch->persistent_blocks = pb;
    return cuda_status(cudaMemcpyAsync(batch->table, host, sizeof(igs::BatchView) * batch->views,
                                       cudaMemcpyHostToDevice, (cudaStream_t)stream),
                       "igs_batch_set_views");
}

igs_status igs_render_batch(igs_batch* batch, const igs_scene* scene, const igs_opts* opts, float* images,
                            void* stream) {
    igs_status st;
    if (!batch || !batch->info) return fail(IGS_ERR_INVALID_ARG, "batch is NULL or not laid out");
    if ((st = check_scene(scene)) || (st = check_opts(opts))) return st;
    if (scene->n != batch->n) return fail(IGS_ERR_INVALID_ARG, "batch laid out for another n");
    if (opts->tile != batch->tile) return fail(IGS_ERR_INVALID_ARG, "batch laid out for another tile size");
    if (!images) return fail(IGS_ERR_INVALID_ARG, "images is NULL");
    if (batch->persistent_blocks <= 0 || !batch->fanout) return fail(IGS_ERR_INVALID_ARG, "call igs_batch_set_views first");
    static thread_local igs_frame frames[IGS_MAX_VIEWS];
    for (int v = 0; v < batch->views; ++v)
        if ((st = batch_frame(batch, opts, v, &frames[v]))) return st;
    igs::BlendParams bp;
    bp.width = bp.height = bp.tiles_x = bp.tiles_y = 0;
    bp.alpha_min = opts->alpha_min; bp.alpha_max = opts->alpha_max; bp.t_min = opts->t_min;
    for (int i = 0; i < 3; ++i) bp.bg[i] = opts->bg[i];
    return cuda_status(igs::launch_render_batch(*batch, frames, *scene, bp, opts->sh_degree, images,
                                                (cudaStream_t)stream, opts->footprint),
                       "igs_render_batch");
}

void igs_batch_release(igs_batch* batch) {
    if (batch) igs::batch_fanout_free(*batch);
}

igs_status igs_batch_status(const igs_batch* batch, uint32_t* host_info, void* stream) {
    if (!batch || !batch->info || !host_info) return fail(IGS_ERR_INVALID_ARG, "batch or host_info is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(host_info, batch->info, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "igs_batch_status");
    if (host_info[igs::kInfoErr] != 0) {
        const igs_status d = (igs_status)host_info[igs::kInfoErr];
        return fail(d, "device reported: %s (entries needed = %u)", igs_status_string(d), host_info[igs::kInfoNeed]);
    }
    return IGS_OK;
}

void igs_debug_silence_lookback_once(void) { igs::g_silence_next.store(1); }

igs_status igs_frame_status(const igs_frame* frame, uint32_t* host_info, void* stream) {
    igs_status st;
    if ((st = check_frame(frame))) return st;
    if (!host_info) return fail(IGS_ERR_INVALID_ARG, "host_info is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(host_info, frame->info, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "igs_frame_status");
    if (host_info[igs::kInfoErr] != 0) {
        const igs_status d = (igs_status)host_info[igs::kInfoErr];
        return fail(d, "device reported: %s (M needed = %u)", igs_status_string(d), host_info[igs::kInfoNeed]);
    }
    return IGS_OK;
}

igs_status igs_frame_walk_segments(const igs_frame* frame, int64_t* host_count, void* stream) {
    igs_status st;
    if ((st = check_frame(frame))) return st;
    if (!host_count) return fail(IGS_ERR_INVALID_ARG, "host_count is NULL");
    const uint32_t* used = igs::blend_segments_used(*frame);
    if (!used) {
        *host_count = -1;
        return IGS_OK;
    }
    uint32_t v = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&v, used, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "igs_frame_walk_segments");
    *host_count = (int64_t)v;
    return IGS_OK;
}

igs_status igs_frame_reset_status(igs_frame* frame, void* stream) {
    igs_status st;
    if ((st = check_frame(frame))) return st;
    return cuda_status(cudaMemsetAsync(frame->info, 0, igs::kInfoWords * 4, (cudaStream_t)stream),
                       "igs_frame_reset_status");
}

}  // extern "C"
