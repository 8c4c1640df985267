"""Python binding of libigs (include/igs.h): argument marshalling only.

Every step of the splatting path runs in the library's CUDA kernels; this
module converts torch tensors to device pointers, passes torch's current
stream, and raises on any non-OK status. There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.

Functions keep the C names without the ``igs_`` prefix: ``project``,
``bin_sort``, ``render_fwd``, ``render_bwd``, ``l1_loss``, ``l1_ssim_loss``, ``adam``,
``export_keys``, ``frame_status``. ``Frame`` owns one view's workspace.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import _build

ABI_VERSION = 3
_lock = threading.Lock()
_lib = None


class IgsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_CAPACITY, ERR_NOT_READY, ERR_DEVICE_TIMEOUT, ERR_UNSUPPORTED = range(8)


class IgsCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("znear", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32)]


class IgsOpts(C.Structure):
    _fields_ = [("tile", C.c_int32), ("sh_degree", C.c_int32), ("param_mode", C.c_int32),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_min", C.c_float), ("bg", C.c_float * 3),
                ("footprint", C.c_int32)]


class IgsScene(C.Structure):
    _fields_ = [("means_sigma", C.c_void_p), ("opacity", C.c_void_p), ("color", C.c_void_p), ("n", C.c_int64)]


class IgsParams(C.Structure):
    _fields_ = [("means_sigma", C.c_void_p), ("opacity", C.c_void_p), ("color", C.c_void_p)]


class IgsFrame(C.Structure):
    _fields_ = [("n", C.c_int64), ("capacity", C.c_int64), ("width", C.c_int32), ("height", C.c_int32),
                ("tile", C.c_int32), ("tiles_x", C.c_int32), ("tiles_y", C.c_int32), ("sort_chunks", C.c_int32),
                ("rec", C.c_void_p), ("rect", C.c_void_p), ("disc", C.c_void_p), ("count", C.c_void_p),
                ("depth_key", C.c_void_p), ("order", C.c_void_p), ("offset", C.c_void_p), ("tile_key", C.c_void_p),
                ("vals", C.c_void_p),
                ("ranges", C.c_void_p), ("T_final", C.c_void_p), ("n_contrib", C.c_void_p), ("info", C.c_void_p),
                ("scratch", C.c_void_p), ("scratch_bytes", C.c_size_t)]


MAX_VIEWS = 256


class IgsBatch(C.Structure):
    _fields_ = [("n", C.c_int64), ("capacity", C.c_int64), ("views", C.c_int32), ("tile", C.c_int32),
                ("blend_batch", C.c_int32), ("persistent_blocks", C.c_int32), ("tiles_total", C.c_int64),
                ("image_floats", C.c_int64), ("image_offset", C.c_int64 * MAX_VIEWS),
                ("tile_base", C.c_uint32 * MAX_VIEWS), ("width", C.c_int32 * MAX_VIEWS),
                ("height", C.c_int32 * MAX_VIEWS), ("view_capacity", C.c_int64 * MAX_VIEWS),
                ("frame_offset", C.c_int64 * MAX_VIEWS), ("workspace", C.c_void_p), ("info", C.c_void_p),
                ("view_entries", C.c_void_p), ("table", C.c_void_p), ("fanout", C.c_void_p)]


class IgsTiming(C.Structure):
    _fields_ = [("arrival_ns", C.c_int64), ("admit_ns", C.c_int64), ("start_ns", C.c_int64), ("done_ns", C.c_int64),
                ("entries", C.c_uint32), ("status", C.c_int32), ("retries", C.c_int32), ("group", C.c_int32)]


SYMBOLS = {
    # name: (restype, argtypes)
    "igs_abi_version": (C.c_int32, []),
    "igs_launch_count": (C.c_uint64, []),
    "igs_last_error": (C.c_char_p, []),
    "igs_status_string": (C.c_char_p, [C.c_int]),
    "igs_frame_layout": (C.c_int, [C.c_int64, C.c_int64, C.POINTER(IgsCamera), C.POINTER(IgsOpts), C.c_void_p,
                                   C.POINTER(C.c_size_t), C.POINTER(IgsFrame)]),
    "igs_project": (C.c_int, [C.POINTER(IgsScene), C.POINTER(IgsCamera), C.POINTER(IgsOpts), C.POINTER(IgsFrame),
                              C.c_void_p]),
    "igs_bin_sort": (C.c_int, [C.POINTER(IgsFrame), C.POINTER(IgsOpts), C.c_void_p]),
    "igs_export_keys": (C.c_int, [C.POINTER(IgsFrame), C.c_void_p, C.c_void_p]),
    "igs_render_fwd": (C.c_int, [C.POINTER(IgsFrame), C.POINTER(IgsOpts), C.c_void_p, C.c_void_p]),
    "igs_render_bwd": (C.c_int, [C.POINTER(IgsScene), C.POINTER(IgsCamera), C.POINTER(IgsOpts), C.POINTER(IgsFrame),
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "igs_blend_bwd": (C.c_int, [C.POINTER(IgsFrame), C.POINTER(IgsOpts), C.c_void_p, C.c_void_p, C.c_void_p]),
    "igs_render_fwd_clear": (C.c_int, [C.POINTER(IgsFrame), C.POINTER(IgsOpts), C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
    "igs_blend_bwd_acc": (C.c_int, [C.POINTER(IgsFrame), C.POINTER(IgsOpts), C.c_void_p, C.c_void_p, C.c_void_p]),
    "igs_project_bwd": (C.c_int, [C.POINTER(IgsScene), C.POINTER(IgsCamera), C.POINTER(IgsOpts),
                                  C.POINTER(IgsFrame), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "igs_project_bwd_adam": (C.c_int, [C.POINTER(IgsScene), C.POINTER(IgsCamera), C.POINTER(IgsOpts),
                                       C.POINTER(IgsFrame), C.c_void_p] + [C.c_void_p] * 6 +
                             [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64, C.c_void_p]),
    "igs_project_bwd_adam_dev": (C.c_int, [C.POINTER(IgsScene), C.POINTER(IgsCamera), C.POINTER(IgsOpts),
                                           C.POINTER(IgsFrame), C.c_void_p] + [C.c_void_p] * 6 +
                                 [C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p]),
    "igs_project_bwd_adam_next": (C.c_int, [C.POINTER(IgsScene), C.POINTER(IgsCamera), C.POINTER(IgsOpts),
                                            C.POINTER(IgsFrame), C.c_void_p] + [C.c_void_p] * 6 +
                                  [C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                   C.POINTER(IgsCamera), C.POINTER(IgsFrame), C.c_void_p]),
    "igs_l1_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "igs_ssim_work_bytes": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32]),
    "igs_l1_ssim_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_float,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "igs_fit2d_render": (C.c_int, [C.c_void_p, C.c_int32, C.c_float, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "igs_fit2d_backward": (C.c_int, [C.c_void_p, C.c_int32, C.c_float, C.c_int32, C.c_int32, C.c_void_p,
                                     C.c_void_p, C.c_void_p]),
    "igs_fit2d_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_float),
                                 C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p]),
    "igs_fit2d_grad_accum": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "igs_fit2d_densify": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_float,
                                    C.c_float, C.c_float, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "igs_grad_accum": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "igs_densify_work_bytes": (C.c_size_t, [C.c_int64]),
    "igs_densify": (C.c_int, [C.POINTER(IgsScene), C.POINTER(IgsParams), C.POINTER(IgsParams), C.c_int32, C.c_int32,
                              C.c_void_p, C.c_void_p, C.c_float, C.c_float, C.c_float, C.c_int64,
                              C.POINTER(IgsParams), C.POINTER(IgsParams), C.POINTER(IgsParams), C.c_void_p,
                              C.c_void_p, C.c_void_p]),
    "igs_merge_work_bytes": (C.c_size_t, [C.c_int64]),
    "igs_merge": (C.c_int, [C.POINTER(IgsScene), C.POINTER(IgsParams), C.POINTER(IgsParams), C.c_int32, C.c_int32,
                            C.POINTER(C.c_float), C.c_float, C.c_float, C.POINTER(IgsParams), C.POINTER(IgsParams),
                            C.POINTER(IgsParams), C.c_void_p, C.c_void_p, C.c_void_p]),
    "igs_octree_work_bytes": (C.c_size_t, [C.c_int32]),
    "igs_octree_init": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_float), C.c_float, C.c_int32,
                                  C.c_int32, C.c_float, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    "igs_quadtree_work_bytes": (C.c_size_t, [C.c_int32, C.c_int32]),
    "igs_quadtree_init": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "igs_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_double,
                           C.c_double, C.c_double, C.c_int64, C.c_void_p]),
    "igs_frame_status": (C.c_int, [C.POINTER(IgsFrame), C.POINTER(C.c_uint32), C.c_void_p]),
    "igs_frame_walk_segments": (C.c_int, [C.POINTER(IgsFrame), C.POINTER(C.c_int64), C.c_void_p]),
    "igs_frame_reset_status": (C.c_int, [C.POINTER(IgsFrame), C.c_void_p]),
    "igs_debug_silence_lookback_once": (None, []),
    "igs_sort_depth_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "igs_batch_layout": (C.c_int, [C.c_int64, C.c_int32, C.POINTER(IgsCamera), C.POINTER(IgsOpts),
                                   C.POINTER(C.c_int64), C.c_int32, C.c_void_p, C.POINTER(C.c_size_t),
                                   C.POINTER(IgsBatch)]),
    "igs_batch_release": (None, [C.POINTER(IgsBatch)]),
    "igs_batch_set_views": (C.c_int, [C.POINTER(IgsBatch), C.POINTER(IgsCamera), C.POINTER(IgsOpts), C.c_void_p]),
    "igs_render_batch": (C.c_int, [C.POINTER(IgsBatch), C.POINTER(IgsScene), C.POINTER(IgsOpts), C.c_void_p,
                                   C.c_void_p]),
    "igs_batch_status": (C.c_int, [C.POINTER(IgsBatch), C.POINTER(C.c_uint32), C.c_void_p]),
    "igs_serve_create": (C.c_int, [C.c_void_p, C.c_size_t, C.c_int32, C.POINTER(IgsOpts), C.POINTER(C.c_void_p)]),
    "igs_serve_set_grouping": (C.c_int, [C.c_void_p, C.c_int32]),
    "igs_serve_add_scene": (C.c_int, [C.c_void_p, C.POINTER(IgsScene), C.c_int32, C.c_int32,
                                      C.POINTER(C.c_int32)]),
    "igs_serve_submit": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(IgsCamera), C.c_void_p,
                                   C.POINTER(C.c_uint64)]),
    "igs_serve_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int64, C.POINTER(IgsTiming)]),
    "igs_serve_stats": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int64)] * 4),
    "igs_serve_destroy": (None, [C.c_void_p]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libigs.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libigs.so not found at {path}: build it with __graft_entry__.build()")
            lib = C.CDLL(path)
            for name, (res, args) in SYMBOLS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            if lib.igs_abi_version() != ABI_VERSION:
                raise RuntimeError("libigs ABI version mismatch")
            _lib = lib
    return _lib


def _check(status, what):
    if status != OK:
        msg = load().igs_last_error().decode(errors="replace")
        raise IgsError(status, f"{what}: {msg}")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


# ------------------------------------------------------------ structures ----

def camera(cam) -> IgsCamera:
    """igs_camera from an object with R (3x3), t (3), fx, fy, cx, cy, znear, width, height."""
    c = IgsCamera()
    R = [float(x) for x in torch.as_tensor(cam.R, dtype=torch.float32).reshape(9).tolist()]
    t = [float(x) for x in torch.as_tensor(cam.t, dtype=torch.float32).reshape(3).tolist()]
    c.R[:] = R
    c.t[:] = t
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.znear = float(getattr(cam, "znear", 0.01))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def opts(tile=16, sh_degree=-1, param_mode=0, alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=1e-4,
         bg=(0.0, 0.0, 0.0), footprint=0) -> IgsOpts:
    o = IgsOpts()
    o.tile, o.sh_degree, o.param_mode = int(tile), int(sh_degree), int(param_mode)
    o.alpha_min, o.alpha_max, o.t_min = alpha_min, alpha_max, t_min
    o.bg[:] = [float(x) for x in bg]
    o.footprint = int(footprint)
    return o


def _check_color_width(scene, sh_degree, where):
    """The colour rows must hold the coefficients the SH degree implies (3 for
    RGB, 3 (d + 1)^2 for degree d): the kernels read that many floats per row."""
    want = 3 if sh_degree < 0 else 3 * (sh_degree + 1) ** 2
    if int(scene.color.shape[1]) != want:
        raise ValueError(f"{where}: color has {int(scene.color.shape[1])} floats per Gaussian, "
                         f"sh_degree {sh_degree} needs {want}")


def _check_g2d(frame, g2d, where):
    """The 2D gradient that a call clears or accumulates into: a contiguous
    float32 tensor of at least 8 floats per Gaussian of the frame (the kernels
    write 2 n float4 there)."""
    if not isinstance(g2d, torch.Tensor) or g2d.dtype != torch.float32 or not g2d.is_contiguous():
        raise ValueError(f"{where}: g2d must be a contiguous float32 tensor")
    if g2d.numel() < 8 * frame.n:
        raise ValueError(f"{where}: g2d holds {g2d.numel()} floats, the frame needs {8 * frame.n}")


def _check_f32(t, need, where, name):
    """A contiguous float32 tensor of at least `need` elements (a kernel reads or
    writes that many floats through its pointer)."""
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{where}: {name} must be a contiguous float32 tensor")
    if t.numel() < need:
        raise ValueError(f"{where}: {name} holds {t.numel()} floats, {need} needed")


def _check_image(frame, t, where, name):
    """A planar [3][H][W] float32 image of the frame's size."""
    _check_f32(t, 3 * int(frame.width) * int(frame.height), where, name)


def _check_param_grads(scene, d_ms, d_op, d_col, where, names=("d_means_sigma", "d_opacity", "d_color")):
    """Per-Gaussian outputs shaped like the scene's arrays: [n][4], [n], [n][C]."""
    n, c = scene.n, int(scene.color.shape[1])
    for t, need, name in ((d_ms, 4 * n, names[0]), (d_op, n, names[1]), (d_col, c * n, names[2])):
        _check_f32(t, need, where, name)


class Scene:
    """Device scene: means_sigma [N,4], opacity [N], color [N,C] (FP32, CUDA)."""

    def __init__(self, means_sigma, opacity, color):
        for name, t in (("means_sigma", means_sigma), ("opacity", opacity), ("color", color)):
            if t.dtype != torch.float32:
                raise ValueError(f"Scene: {name} must be float32")
        n = int(means_sigma.shape[0]) if means_sigma.dim() == 2 else -1
        if n < 0 or means_sigma.shape[1] != 4:
            raise ValueError("Scene: means_sigma must be [N, 4]")
        if opacity.dim() != 1 or opacity.shape[0] != n:
            raise ValueError("Scene: opacity must be [N]")
        if color.dim() != 2 or color.shape[0] != n or color.shape[1] not in (3, 12, 27, 48):
            raise ValueError("Scene: color must be [N, C] with C = 3, 12, 27 or 48")
        self.means_sigma, self.opacity, self.color = means_sigma, opacity, color
        self.n = n
        s = IgsScene()
        s.means_sigma = _ptr(means_sigma).value if self.n else None
        s.opacity = _ptr(opacity).value if self.n else None
        s.color = _ptr(color).value if self.n else None
        s.n = self.n
        self.struct = s

    @staticmethod
    def from_numpy(sc, device="cuda"):
        return Scene(torch.from_numpy(sc.means_sigma).to(device), torch.from_numpy(sc.opacity).to(device),
                     torch.from_numpy(sc.color).to(device))


_DT = {"f32": torch.float32, "u32": torch.int32, "u64": torch.int64}


class Frame:
    """One view's workspace, carved by igs_frame_layout from one uint8 tensor."""

    def __init__(self, n, capacity, cam, o, device="cuda"):
        lib = load()
        self.cam = cam if isinstance(cam, IgsCamera) else camera(cam)
        self.opts = o
        nbytes = C.c_size_t(0)
        _check(lib.igs_frame_layout(int(n), int(capacity), C.byref(self.cam), C.byref(o), None, C.byref(nbytes),
                                    None), "igs_frame_layout")
        self.nbytes = int(nbytes.value)
        self.ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        self._shift = (-base) % 256
        self.struct = IgsFrame()
        _check(lib.igs_frame_layout(int(n), int(capacity), C.byref(self.cam), C.byref(o),
                                    C.c_void_p(base + self._shift), C.byref(nbytes), C.byref(self.struct)),
               "igs_frame_layout")
        self.n, self.capacity = int(n), int(capacity)
        self.width, self.height = self.struct.width, self.struct.height
        self.tiles_x, self.tiles_y = self.struct.tiles_x, self.struct.tiles_y
        self.tiles = self.tiles_x * self.tiles_y

    def view(self, field, count, dtype=torch.int32):
        """A tensor view of `count` elements of a frame buffer (for inspection)."""
        addr = getattr(self.struct, field)
        off = addr - self.ws.data_ptr()
        nb = count * torch.empty((), dtype=dtype).element_size()
        return self.ws[off:off + nb].view(dtype)

    # typed views of the documented buffers
    def rec(self):
        return self.view("rec", self.n * 8, torch.float32).view(self.n, 8)

    def count(self):
        return self.view("count", self.n)

    def depth_key(self):
        return self.view("depth_key", self.n)

    def disc(self):
        return self.view("disc", self.n * 4, torch.float32).view(self.n, 4)

    def rect(self):
        return self.view("rect", self.n * 2).view(self.n, 2)

    def order(self):
        return self.view("order", self.n)

    def tile_key(self, m):
        return self.view("tile_key", m)

    def vals(self, m):
        return self.view("vals", m)

    def ranges(self):
        return self.view("ranges", self.tiles * 2).view(self.tiles, 2)

    def T_final(self):
        return self.view("T_final", self.width * self.height, torch.float32).view(self.height, self.width)

    def n_contrib(self):
        return self.view("n_contrib", self.width * self.height).view(self.height, self.width)

    def info(self):
        return self.view("info", 16)


# ------------------------------------------------------------ entry points --

def project(scene: Scene, cam: IgsCamera, o: IgsOpts, frame: Frame, stream=None):
    _check_color_width(scene, o.sh_degree, "project")
    _check(load().igs_project(C.byref(scene.struct), C.byref(cam), C.byref(o), C.byref(frame.struct),
                              _stream(stream)), "igs_project")


def bin_sort(frame: Frame, o: IgsOpts, stream=None):
    _check(load().igs_bin_sort(C.byref(frame.struct), C.byref(o), _stream(stream)), "igs_bin_sort")


def export_keys(frame: Frame, stream=None):
    keys = torch.empty(max(frame.capacity, 1), dtype=torch.int64, device=frame.ws.device)
    _check(load().igs_export_keys(C.byref(frame.struct), _ptr(keys), _stream(stream)), "igs_export_keys")
    return keys


def render_fwd(frame: Frame, o: IgsOpts, img, stream=None):
    _check_image(frame, img, "render_fwd", "img")
    _check(load().igs_render_fwd(C.byref(frame.struct), C.byref(o), _ptr(img), _stream(stream)), "igs_render_fwd")


def render_bwd(scene: Scene, cam: IgsCamera, o: IgsOpts, frame: Frame, dL_dimg, g2d, d_means_sigma, d_opacity,
               d_color, stream=None):
    _check_color_width(scene, o.sh_degree, "render_bwd")
    _check_image(frame, dL_dimg, "render_bwd", "dL_dimg")
    _check_g2d(frame, g2d, "render_bwd")
    _check_param_grads(scene, d_means_sigma, d_opacity, d_color, "render_bwd")
    _check(load().igs_render_bwd(C.byref(scene.struct), C.byref(cam), C.byref(o), C.byref(frame.struct),
                                 _ptr(dL_dimg), _ptr(g2d), _ptr(d_means_sigma), _ptr(d_opacity), _ptr(d_color),
                                 _stream(stream)), "igs_render_bwd")


def blend_bwd(frame: Frame, o: IgsOpts, dL_dimg, g2d, stream=None):
    _check_image(frame, dL_dimg, "blend_bwd", "dL_dimg")
    _check_g2d(frame, g2d, "blend_bwd")
    _check(load().igs_blend_bwd(C.byref(frame.struct), C.byref(o), _ptr(dL_dimg), _ptr(g2d), _stream(stream)),
           "igs_blend_bwd")


def render_fwd_clear(frame: Frame, o: IgsOpts, img, g2d, stream=None):
    """render_fwd that also zeroes g2d ([n][8] float32) for blend_bwd_acc."""
    _check_image(frame, img, "render_fwd_clear", "img")
    _check_g2d(frame, g2d, "render_fwd_clear")
    _check(load().igs_render_fwd_clear(C.byref(frame.struct), C.byref(o), _ptr(img), _ptr(g2d), _stream(stream)),
           "igs_render_fwd_clear")


def blend_bwd_acc(frame: Frame, o: IgsOpts, dL_dimg, g2d, stream=None):
    """blend_bwd into a g2d that render_fwd_clear zeroed (no clearing here)."""
    _check_image(frame, dL_dimg, "blend_bwd_acc", "dL_dimg")
    _check_g2d(frame, g2d, "blend_bwd_acc")
    _check(load().igs_blend_bwd_acc(C.byref(frame.struct), C.byref(o), _ptr(dL_dimg), _ptr(g2d), _stream(stream)),
           "igs_blend_bwd_acc")


def project_bwd(scene: Scene, cam: IgsCamera, o: IgsOpts, frame: Frame, g2d, d_means_sigma, d_opacity, d_color,
                stream=None):
    _check_color_width(scene, o.sh_degree, "project_bwd")
    _check_g2d(frame, g2d, "project_bwd")
    _check_param_grads(scene, d_means_sigma, d_opacity, d_color, "project_bwd")
    _check(load().igs_project_bwd(C.byref(scene.struct), C.byref(cam), C.byref(o), C.byref(frame.struct),
                                  _ptr(g2d), _ptr(d_means_sigma), _ptr(d_opacity), _ptr(d_color),
                                  _stream(stream)), "igs_project_bwd")


def project_bwd_adam(scene: Scene, cam: IgsCamera, o: IgsOpts, frame: Frame, g2d, m, v, step, lr=1e-3, b1=0.9,
                     b2=0.999, eps=1e-8, stream=None):
    """Projection backward fused with Adam: scene parameters and the moments
    m = (m_ms, m_op, m_col), v = (v_ms, v_op, v_col) are updated in place."""
    _check_color_width(scene, o.sh_degree, "project_bwd_adam")
    _check_g2d(frame, g2d, "project_bwd_adam")
    _check_param_grads(scene, *m, "project_bwd_adam", ("m[0]", "m[1]", "m[2]"))
    _check_param_grads(scene, *v, "project_bwd_adam", ("v[0]", "v[1]", "v[2]"))
    _check(load().igs_project_bwd_adam(C.byref(scene.struct), C.byref(cam), C.byref(o), C.byref(frame.struct),
                                       _ptr(g2d), *[_ptr(t) for t in m], *[_ptr(t) for t in v], lr, b1, b2, eps,
                                       int(step), _stream(stream)), "igs_project_bwd_adam")


def project_bwd_adam_dev(scene: Scene, cam: IgsCamera, o: IgsOpts, frame: Frame, g2d, m, v, state, lr=1e-3,
                         b1=0.9, b2=0.999, eps=1e-8, stream=None):
    """project_bwd_adam with the step count on the device: state is an int32[4]
    tensor (zero before the first step) that the call advances, so the step can
    be captured in a CUDA graph and replayed."""
    _check_color_width(scene, o.sh_degree, "project_bwd_adam_dev")
    _check_g2d(frame, g2d, "project_bwd_adam_dev")
    _check_param_grads(scene, *m, "project_bwd_adam_dev", ("m[0]", "m[1]", "m[2]"))
    _check_param_grads(scene, *v, "project_bwd_adam_dev", ("v[0]", "v[1]", "v[2]"))
    _check(load().igs_project_bwd_adam_dev(C.byref(scene.struct), C.byref(cam), C.byref(o), C.byref(frame.struct),
                                           _ptr(g2d), *[_ptr(t) for t in m], *[_ptr(t) for t in v], lr, b1, b2, eps,
                                           _ptr(state), _stream(stream)), "igs_project_bwd_adam_dev")


def project_bwd_adam_next(scene: Scene, cam: IgsCamera, o: IgsOpts, frame: Frame, g2d, m, v, state, next_cam,
                          next_frame: Frame, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    """project_bwd_adam_dev, then the projection of next_cam into next_frame from
    the updated parameters in the same pass (what project() would write)."""
    _check_color_width(scene, o.sh_degree, "project_bwd_adam_next")
    _check_g2d(frame, g2d, "project_bwd_adam_next")
    _check_param_grads(scene, *m, "project_bwd_adam_next", ("m[0]", "m[1]", "m[2]"))
    _check_param_grads(scene, *v, "project_bwd_adam_next", ("v[0]", "v[1]", "v[2]"))
    _check(load().igs_project_bwd_adam_next(C.byref(scene.struct), C.byref(cam), C.byref(o), C.byref(frame.struct),
                                            _ptr(g2d), *[_ptr(t) for t in m], *[_ptr(t) for t in v], lr, b1, b2,
                                            eps, _ptr(state), C.byref(next_cam), C.byref(next_frame.struct),
                                            _stream(stream)), "igs_project_bwd_adam_next")


def l1_loss(img, target, loss, dL_dimg, stream=None):
    for t, name in ((img, "img"), (target, "target"), (dL_dimg, "dL_dimg")):
        _check_f32(t, int(img.numel()), "l1_loss", name)
    _check_f32(loss, 1, "l1_loss", "loss")
    _check(load().igs_l1_loss(_ptr(img), _ptr(target), int(img.numel()), _ptr(loss), _ptr(dL_dimg),
                              _stream(stream)), "igs_l1_loss")


def ssim_work_bytes(channels, height, width):
    return int(load().igs_ssim_work_bytes(int(channels), int(height), int(width)))


def l1_ssim_loss(img, target, lam, loss, dL_dimg, work, ssim=None, stream=None):
    """(1 - lam) L1 + lam (1 - SSIM) of planar [C][H][W] (or [H][W]) images into
    loss (device float) and dL_dimg; ssim (device float) optional; work: a device
    buffer of at least ssim_work_bytes bytes."""
    shp = tuple(img.shape) if img.dim() == 3 else (1,) + tuple(img.shape)
    if tuple(target.shape) != tuple(img.shape) or tuple(dL_dimg.shape) != tuple(img.shape) or len(shp) != 3:
        raise ValueError("img, target and dL_dimg must share a [C][H][W] or [H][W] shape")
    need = ssim_work_bytes(*shp)
    if work.numel() * work.element_size() < need:
        raise ValueError(f"work holds {work.numel() * work.element_size()} bytes, needs {need}")
    _check(load().igs_l1_ssim_loss(_ptr(img), _ptr(target), shp[0], shp[1], shp[2], float(lam), _ptr(loss),
                                   _ptr(ssim) if ssim is not None else None, _ptr(dL_dimg), _ptr(work),
                                   _stream(stream)), "igs_l1_ssim_loss")


# ------------------------------------------------------------ 2D fitting --

def _particles(p):
    if p.dim() != 2 or p.shape[1] != 8 or p.dtype != torch.float32 or not p.is_contiguous():
        raise ValueError("particles must be a contiguous float32 [k][8] tensor")
    return p


def fit2d_render(particles, D, img, stream=None):
    """img ([3][H][W]) = sum of the particles' kernels within distance D."""
    _particles(particles)
    _check(load().igs_fit2d_render(_ptr(particles), particles.shape[0], float(D), img.shape[2], img.shape[1],
                                   _ptr(img), _stream(stream)), "igs_fit2d_render")


def fit2d_backward(particles, D, dL_dimg, d_particles, stream=None):
    _particles(particles)
    _check(load().igs_fit2d_backward(_ptr(particles), particles.shape[0], float(D), dL_dimg.shape[2],
                                     dL_dimg.shape[1], _ptr(dL_dimg), _ptr(d_particles), _stream(stream)),
           "igs_fit2d_backward")


def fit2d_adam(particles, d_particles, m, v, lr, state, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    """Adam over the particles with per-slot learning rates lr (8 floats); state:
    device int32[2] step counter, zero before the first step."""
    _particles(particles)
    lrs = (C.c_float * 8)(*[float(x) for x in lr])
    _check(load().igs_fit2d_adam(_ptr(particles), _ptr(d_particles), _ptr(m), _ptr(v), particles.shape[0], lrs,
                                 float(b1), float(b2), float(eps), _ptr(state), _stream(stream)), "igs_fit2d_adam")


def fit2d_grad_accum(d_particles, accum, stream=None):
    """accum ([k] float32, device) += the norm of each particle's position gradient."""
    _particles(d_particles)
    _check(load().igs_fit2d_grad_accum(_ptr(d_particles), d_particles.shape[0], _ptr(accum), _stream(stream)),
           "igs_fit2d_grad_accum")


def fit2d_densify(particles, m, v, accum, n_iters, tau_a, tau_g, log_sigma_min, out, out_m, out_v, count,
                  stream=None):
    """Delete (max |A| < tau_a), divide (accum > tau_g * n_iters and log sigma >=
    log_sigma_min: four half-scale children) or keep each particle into out,
    out_m, out_v ([capacity][8]); the new count goes to count (device int32)."""
    _particles(particles)
    _check(load().igs_fit2d_densify(_ptr(particles), _ptr(m), _ptr(v), _ptr(accum), particles.shape[0], int(n_iters),
                                    float(tau_a), float(tau_g), float(log_sigma_min), out.shape[0], _ptr(out),
                                    _ptr(out_m), _ptr(out_v), _ptr(count), _stream(stream)), "igs_fit2d_densify")


def _params(arrs):
    p = IgsParams()
    p.means_sigma, p.opacity, p.color = (_ptr(a).value if a.numel() else None for a in arrs)
    return p


def grad_accum(g2d, count, accum, vis, stream=None):
    """Densify statistic of one step: for Gaussians with count > 0 (the frame's
    per-Gaussian tile count), accum += |(du, dv)| from g2d [n][8] and vis += 1."""
    n = int(accum.shape[0])
    _check_f32(g2d, 8 * n, "grad_accum", "g2d")
    _check_f32(accum, n, "grad_accum", "accum")
    for t, name in ((count, "count"), (vis, "vis")):
        if (not isinstance(t, torch.Tensor) or t.element_size() != 4 or t.dtype.is_floating_point
                or not t.is_contiguous() or t.numel() < n):
            raise ValueError(f"grad_accum: {name} must be a contiguous 32-bit integer tensor of at least {n} elements")
    _check(load().igs_grad_accum(_ptr(g2d), _ptr(count), n, _ptr(accum), _ptr(vis), _stream(stream)),
           "igs_grad_accum")


def densify_work_bytes(n):
    return int(load().igs_densify_work_bytes(int(n)))


def densify(scene: Scene, m, v, sh_degree, param_mode, accum, vis, op_min, tau_g, scale_min, out, out_m, out_v,
            count, work, stream=None):
    """Delete / divide / keep every Gaussian of `scene` (stored parameters) with
    its Adam moments m, v = (means_sigma, opacity, color) tensors into out,
    out_m, out_v (same layout, capacity = out[0].shape[0]); the new count goes to
    count (device int64)."""
    _check_color_width(scene, sh_degree, "densify")
    _check(load().igs_densify(C.byref(scene.struct), C.byref(_params(m)), C.byref(_params(v)), int(sh_degree),
                              int(param_mode), _ptr(accum), _ptr(vis), float(op_min), float(tau_g),
                              float(scale_min), int(out[0].shape[0]), C.byref(_params(out)),
                              C.byref(_params(out_m)), C.byref(_params(out_v)), _ptr(count), _ptr(work),
                              _stream(stream)), "igs_densify")


def merge_work_bytes(n):
    return int(load().igs_merge_work_bytes(int(n)))


def merge(scene: Scene, m, v, sh_degree, param_mode, lo, cell, scale_max, out, out_m, out_v, count, work,
          stream=None):
    """Merge the eligible Gaussians of `scene` (stored parameters) that share a
    grid cell of side `cell` from the corner lo, with their Adam moments m, v =
    (means_sigma, opacity, color) tensors, into out, out_m, out_v (same layout,
    at least scene.n Gaussians); the new count goes to count (device int64, -1
    if the device sort gave up)."""
    _check_color_width(scene, sh_degree, "merge")
    for o in (out, out_m, out_v):
        if int(o[0].shape[0]) < scene.n or int(o[1].shape[0]) < scene.n or int(o[2].shape[0]) < scene.n:
            raise ValueError("merge: every output array needs room for scene.n Gaussians")
    lo3 = (C.c_float * 3)(*[float(x) for x in lo])
    _check(load().igs_merge(C.byref(scene.struct), C.byref(_params(m)), C.byref(_params(v)), int(sh_degree),
                            int(param_mode), lo3, float(cell), float(scale_max), C.byref(_params(out)),
                            C.byref(_params(out_m)), C.byref(_params(out_v)), _ptr(count), _ptr(work),
                            _stream(stream)), "igs_merge")


def octree_work_bytes(levels):
    return int(load().igs_octree_work_bytes(int(levels)))


def octree_init(points, colors, lo, side, levels, k_max, opacity=0.5, sh_degree=-1, param_mode=0, stream=None):
    """Octree initialisation of 3D Gaussians from a coloured point set (device
    [n][3] tensors); returns (means_sigma [K][4], opacity [K], color [K][C]) on
    the device (one synchronisation to read K)."""
    if points.dtype != torch.float32 or colors.dtype != torch.float32:
        raise ValueError("octree_init: points and colors must be float32")
    if points.dim() != 2 or points.shape[1] != 3 or tuple(colors.shape) != tuple(points.shape):
        raise ValueError("octree_init: points and colors must be [n, 3] tensors with the same n")
    dev = points.device
    nc = 3 if sh_degree < 0 else 3 * (sh_degree + 1) ** 2
    ms = torch.empty((k_max, 4), dtype=torch.float32, device=dev)
    op = torch.empty(k_max, dtype=torch.float32, device=dev)
    col = torch.empty((k_max, nc), dtype=torch.float32, device=dev)
    count = torch.zeros(1, dtype=torch.int32, device=dev)
    work = torch.empty(octree_work_bytes(levels), dtype=torch.uint8, device=dev)
    lo3 = (C.c_float * 3)(*[float(x) for x in lo])
    n = int(points.shape[0])
    _check(load().igs_octree_init(_ptr(points) if n else None, _ptr(colors) if n else None, n, lo3, float(side),
                                  int(levels), int(k_max), float(opacity), int(sh_degree), int(param_mode), _ptr(ms),
                                  _ptr(op), _ptr(col), _ptr(count), _ptr(work), _stream(stream)), "igs_octree_init")
    k = int(count.item())
    return ms[:k], op[:k], col[:k]


def quadtree_work_bytes(side, min_cell):
    return int(load().igs_quadtree_work_bytes(int(side), int(min_cell)))


def quadtree_init(img, k_max, min_cell, particles, count, work, stream=None):
    """QuadTree initialisation of a [3][S][S] image into particles (>= k_max x 8)
    and the particle count into count (device int32)."""
    if img.dim() != 3 or img.shape[0] != 3 or img.shape[1] != img.shape[2]:
        raise ValueError("img must be [3][S][S]")
    _check(load().igs_quadtree_init(_ptr(img), img.shape[1], int(k_max), int(min_cell), _ptr(particles),
                                    _ptr(count), _ptr(work), _stream(stream)), "igs_quadtree_init")


def adam(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _check(load().igs_adam(_ptr(p), _ptr(g), _ptr(m), _ptr(v), int(p.numel()), lr, b1, b2, eps, int(step),
                           _stream(stream)), "igs_adam")


def frame_status(frame: Frame, stream=None):
    """(status, [M, kept, error, M needed]); synchronises the stream."""
    info = (C.c_uint32 * 4)()
    st = load().igs_frame_status(C.byref(frame.struct), info, _stream(stream))
    if st not in (OK, ERR_CAPACITY, ERR_DEVICE_TIMEOUT):
        _check(st, "igs_frame_status")
    return st, list(info)


def frame_stats(frame: Frame, stream=None):
    """Counters of the frame's last binning and forward, read from its own
    buffers (synchronises the stream): Gaussians kept (visible), entries
    (Gaussian, tile) M, their mean and largest count per tile, the share of
    empty tiles, and the mean and largest number of list positions a pixel's
    walk reached (n_contrib: the last blended entry + 1)."""
    st, info = frame_status(frame, stream)
    if st != OK:
        raise IgsError(st, "frame_stats: the frame's last binning did not complete")
    r = frame.ranges().to(torch.int64)
    per_tile = (r[:, 1] - r[:, 0]).clamp(min=0)
    nc = frame.n_contrib().to(torch.int64)
    tiles = max(1, int(per_tile.numel()))
    return {"kept": int(info[1]), "entries": int(info[0]),
            "entries_per_tile_mean": float(per_tile.sum()) / tiles, "entries_per_tile_max": int(per_tile.max()),
            "empty_tiles": float((per_tile == 0).sum()) / tiles,
            "contrib_per_pixel_mean": float(nc.float().mean()), "contrib_per_pixel_max": int(nc.max())}


def frame_walk_segments(frame: Frame, stream=None):
    """Pool slots the frame's last forward blend took for walk segments (-1: the
    frame has none); synchronises the stream."""
    out = C.c_int64(0)
    _check(load().igs_frame_walk_segments(C.byref(frame.struct), C.byref(out), _stream(stream)),
           "igs_frame_walk_segments")
    return int(out.value)


_WORD_DTYPES = tuple(d for d in (torch.int32, getattr(torch, "uint32", None)) if d is not None)


def sort_depth_noalloc(depth_key, order, stream=None):
    """igs_sort_depth_noalloc: order = stable argsort of depth_key (int32 views of
    uint32 data, n <= 2^20), scratch from the library's static device array.
    Both tensors must be 1-D, contiguous, 4 bytes per element and of the same
    length (the kernels write n words to order)."""
    for name, t in (("depth_key", depth_key), ("order", order)):
        if t.dtype not in _WORD_DTYPES or t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"sort_depth_noalloc: {name} must be a contiguous 1-D int32 (or uint32) tensor")
    if order.numel() != depth_key.numel():
        raise ValueError("sort_depth_noalloc: order must have as many elements as depth_key")
    if order.device != depth_key.device:
        raise ValueError("sort_depth_noalloc: depth_key and order must be on the same device")
    _check(load().igs_sort_depth_noalloc(_ptr(depth_key), int(depth_key.numel()), _ptr(order), _stream(stream)),
           "igs_sort_depth_noalloc")


class Batch:
    """One multi-view batch: workspace from igs_batch_layout (a frame per view,
    `capacity` entries each: one number for every view, or one per view) and
    the packed image buffer."""

    def __init__(self, n, cams, o, capacity, blend_batch=0, device="cuda"):
        lib = load()
        self.cams = [c if isinstance(c, IgsCamera) else camera(c) for c in cams]
        self.opts = o
        V = len(self.cams)
        caps = [int(capacity)] * V if isinstance(capacity, int) else [int(c) for c in capacity]
        if len(caps) != V:
            raise ValueError("Batch: one capacity per view")
        arr = (IgsCamera * V)(*self.cams)
        carr = (C.c_int64 * V)(*caps)
        nbytes = C.c_size_t(0)
        _check(lib.igs_batch_layout(int(n), V, arr, C.byref(o), carr, int(blend_batch), None, C.byref(nbytes), None),
               "igs_batch_layout")
        self.nbytes = int(nbytes.value)
        self.ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        self.struct = IgsBatch()
        _check(lib.igs_batch_layout(int(n), V, arr, C.byref(o), carr, int(blend_batch),
                                    C.c_void_p(base + (-base) % 256), C.byref(nbytes), C.byref(self.struct)),
               "igs_batch_layout")
        self.images = torch.empty(int(self.struct.image_floats), dtype=torch.float32, device=device)
        self.n, self.capacities, self.capacity = int(n), caps, sum(caps)

    def set_views(self, cams=None, stream=None):
        if cams is not None:
            self.cams = [c if isinstance(c, IgsCamera) else camera(c) for c in cams]
        arr = (IgsCamera * len(self.cams))(*self.cams)
        _check(load().igs_batch_set_views(C.byref(self.struct), arr, C.byref(self.opts), _stream(stream)),
               "igs_batch_set_views")

    def render(self, scene: "Scene", stream=None):
        _check_color_width(scene, self.opts.sh_degree, "Batch.render")
        _check(load().igs_render_batch(C.byref(self.struct), C.byref(scene.struct), C.byref(self.opts),
                                       _ptr(self.images), _stream(stream)), "igs_render_batch")

    def status(self, stream=None):
        info = (C.c_uint32 * 4)()
        st = load().igs_batch_status(C.byref(self.struct), info, _stream(stream))
        if st not in (OK, ERR_CAPACITY, ERR_DEVICE_TIMEOUT):
            _check(st, "igs_batch_status")
        return st, list(info)

    def image(self, v):
        off = int(self.struct.image_offset[v])
        h, w = int(self.struct.height[v]), int(self.struct.width[v])
        return self.images[off:off + 3 * h * w].view(3, h, w)

    def view_entries(self):
        """Entries of each view in the last render (device int32 [V] view)."""
        V = int(self.struct.views)
        off = int(self.struct.view_entries) - self.ws.data_ptr()
        return self.ws[off:off + 4 * V].view(torch.int32)

    def release(self):
        """Free the fan-out streams (after the batch's work has finished)."""
        if getattr(self, "struct", None) is not None and self.struct.fanout:
            torch.cuda.synchronize(self.ws.device)
            load().igs_batch_release(C.byref(self.struct))

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Server:
    """Render server (igs_serve_*): resident scenes, continuous batching over
    `slots` streams, admission against a device pool of `pool_bytes`; with
    group > 1, up to `group` queued requests of one scene share one batched
    chain of launches."""

    def __init__(self, pool_bytes, slots=4, tile=16, bg=(0.0, 0.0, 0.0), device="cuda", group=1):
        self.pool = torch.empty(int(pool_bytes) + 256, dtype=torch.uint8, device=device)
        base = self.pool.data_ptr()
        self.opts = opts(tile=tile, bg=bg)
        h = C.c_void_p()
        _check(load().igs_serve_create(C.c_void_p(base + (-base) % 256), int(pool_bytes), int(slots),
                                       C.byref(self.opts), C.byref(h)), "igs_serve_create")
        self.handle = h
        self.scenes = []
        if group != 1:
            _check(load().igs_serve_set_grouping(self.handle, int(group)), "igs_serve_set_grouping")

    def add_scene(self, scene: Scene, sh_degree=-1, param_mode=0):
        _check_color_width(scene, sh_degree, "Server.add_scene")
        sid = C.c_int32()
        _check(load().igs_serve_add_scene(self.handle, C.byref(scene.struct), int(sh_degree), int(param_mode),
                                          C.byref(sid)), "igs_serve_add_scene")
        self.scenes.append(scene)  # keep the buffers alive
        return int(sid.value)

    def submit(self, scene_id, cam, img_out):
        c = cam if isinstance(cam, IgsCamera) else camera(cam)
        rid = C.c_uint64()
        _check(load().igs_serve_submit(self.handle, int(scene_id), C.byref(c), _ptr(img_out), C.byref(rid)),
               "igs_serve_submit")
        return int(rid.value)

    def poll(self, req_id, timeout_s=10.0):
        """(status, timing dict); status NOT_READY if still running after the timeout."""
        t = IgsTiming()
        st = load().igs_serve_poll(self.handle, C.c_uint64(req_id), int(timeout_s * 1e9), C.byref(t))
        return st, {k: getattr(t, k) for k, _ in IgsTiming._fields_}

    def stats(self):
        v = [C.c_int64() for _ in range(4)]
        _check(load().igs_serve_stats(self.handle, *[C.byref(x) for x in v]), "igs_serve_stats")
        return dict(zip(("pending", "in_flight", "pool_used", "pool_peak"), [x.value for x in v]))

    def close(self):
        if self.handle:
            load().igs_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels the library has launched in this process."""
    return int(load().igs_launch_count())


def debug_silence_lookback_once():
    """Failure-detection tests: the next bin_sort's first depth pass has one
    block that never publishes, so the later blocks' bounded waits run out and
    the frame reports ERR_DEVICE_TIMEOUT."""
    load().igs_debug_silence_lookback_once()


def frame_reset_status(frame: Frame, stream=None):
    _check(load().igs_frame_reset_status(C.byref(frame.struct), _stream(stream)), "igs_frame_reset_status")
