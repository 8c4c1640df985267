"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/igs.h declares; the host-only logic (frame
sizing, argument checks, status strings) behaves as documented."""
import ctypes as C
import os
import re

import pytest

from paper_2403_14244_gb300 import _build, igs, scenes

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "igs.h")


def _declared():
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^IGS_API\s+[\w\s\*]+?\b(igs_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for want in ("igs_project", "igs_bin_sort", "igs_render_fwd", "igs_render_bwd", "igs_l1_loss", "igs_adam",
                 "igs_frame_layout", "igs_frame_status"):
        assert want in names


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(_build.build())
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(igs.SYMBOLS)           # the binding covers the whole ABI


def test_abi_version_and_status_strings():
    lib = igs.load()
    assert lib.igs_abi_version() == igs.ABI_VERSION
    assert lib.igs_status_string(igs.OK) == b"ok"
    assert lib.igs_status_string(igs.ERR_CAPACITY) == b"entry capacity exceeded"


def test_frame_layout_sizes_without_gpu():
    lib = igs.load()
    sc, cam = scenes.workload_forward_4k()
    c = igs.camera(cam)
    nb = C.c_size_t(0)
    assert lib.igs_frame_layout(4096, 1 << 16, C.byref(c), C.byref(igs.opts(tile=16)), None, C.byref(nb), None) == 0
    small = nb.value
    assert small % 256 == 0
    assert lib.igs_frame_layout(4096, 1 << 20, C.byref(c), C.byref(igs.opts(tile=16)), None, C.byref(nb), None) == 0
    assert nb.value >= small + 8 * ((1 << 20) - (1 << 16))   # the entry buffers grow (8 or 16 bytes per entry)


@pytest.mark.parametrize("bad", ["tile", "fx", "capacity", "n", "sh"])
def test_frame_layout_rejects_bad_arguments(bad):
    lib = igs.load()
    sc, cam = scenes.workload_forward_4k()
    o = igs.opts(tile=16)
    n, cap = 4096, 1 << 16
    if bad == "tile":
        o = igs.opts(tile=12)
    elif bad == "fx":
        cam.fy = cam.fx + 1
    elif bad == "capacity":
        cap = 1 << 30
    elif bad == "n":
        n = -1
    elif bad == "sh":
        o = igs.opts(tile=16, sh_degree=4)
    nb = C.c_size_t(0)
    st = lib.igs_frame_layout(n, cap, C.byref(igs.camera(cam)), C.byref(o), None, C.byref(nb), None)
    assert st == igs.ERR_INVALID_ARG
    assert lib.igs_last_error()                             # a message for the caller


def test_null_arguments_rejected_before_any_launch():
    lib = igs.load()
    assert lib.igs_project(None, None, None, None, None) == igs.ERR_INVALID_ARG
    assert lib.igs_bin_sort(None, None, None) == igs.ERR_INVALID_ARG
    assert lib.igs_render_fwd(None, None, None, None) == igs.ERR_INVALID_ARG
    assert lib.igs_l1_loss(None, None, 0, None, None, None) == igs.ERR_INVALID_ARG
    assert lib.igs_adam(None, None, None, None, 0, 1e-3, 0.9, 0.999, 1e-8, 1, None) == igs.ERR_INVALID_ARG


def test_product_path_has_no_oracle_or_cpu_fallback():
    pkg = os.path.dirname(igs.__file__)
    for root, _, files in os.walk(pkg):
        for name in files:
            if name.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                with open(os.path.join(root, name)) as f:
                    text = f.read()
                assert "import oracle" not in text and "from oracle" not in text, name
                assert "liboracle" not in text, name


@pytest.mark.parametrize("pts,cols", [((5, 3, "f64"), (5, 3, "f32")), ((5, 4, "f32"), (5, 4, "f32")),
                                      ((5, 3, "f32"), (6, 3, "f32"))])
def test_octree_init_rejects_bad_tensors_before_any_launch(pts, cols):
    """float64 points, [n, 4] rows or colours of another n raise in the binding, before any
    allocation or launch."""
    import torch
    mk = lambda n, c, dt: torch.zeros((n, c), dtype=torch.float64 if dt == "f64" else torch.float32)  # noqa: E731
    with pytest.raises(ValueError, match="octree_init"):
        igs.octree_init(mk(*pts), mk(*cols), (-1, -1, -1), 2.0, 4, 100)


def test_scene_and_colour_width_checked_in_the_binding():
    """A scene of the wrong dtype or shape, or colour rows that do not match the SH degree (the
    kernels read 3 (d + 1)^2 floats per row), raise in the binding before any launch."""
    import types

    import torch
    z = torch.zeros
    for ms, op, col in ((z(4, 4, dtype=torch.float64), z(4), z(4, 3)), (z(4, 3), z(4), z(4, 3)),
                        (z(4, 4), z(5), z(4, 3)), (z(4, 4), z(4), z(4, 5)), (z(4, 4), z(4, 1), z(4, 3))):
        with pytest.raises(ValueError, match="Scene"):
            igs.Scene(ms, op, col)
    for C, ok in ((3, (-1, 0)), (12, (1,)), (27, (2,)), (48, (3,))):
        sc = types.SimpleNamespace(color=z(2, C))
        for d in (-1, 0, 1, 2, 3):
            if d in ok:
                igs._check_color_width(sc, d, "t")
            else:
                with pytest.raises(ValueError, match="sh_degree"):
                    igs._check_color_width(sc, d, "t")


@pytest.mark.parametrize("bad", ["short_order", "int16_order", "int64_key", "2d_key", "strided_order"])
def test_sort_depth_noalloc_binding_refuses_bad_buffers(bad):
    """The kernels write n 4-byte words to order: a shorter or narrower order,
    or keys that are not n 4-byte words, are refused before anything launches."""
    import torch
    n = 1000
    key = torch.zeros(n, dtype=torch.int32)
    order = torch.zeros(n, dtype=torch.int32)
    if bad == "short_order":
        order = order[: n - 1]
    elif bad == "int16_order":
        order = torch.zeros(n, dtype=torch.int16)
    elif bad == "int64_key":
        key = torch.zeros(n, dtype=torch.int64)
    elif bad == "2d_key":
        key = key.view(10, 100)
        order = order.view(10, 100)
    else:
        order = torch.zeros(2 * n, dtype=torch.int32)[::2]
    before = igs.launch_count()
    with pytest.raises(ValueError):
        igs.sort_depth_noalloc(key, order)
    assert igs.launch_count() == before


def _fake_frame_scene(n=10, w=8, h=6, c=3):
    """Host stand-ins carrying what the binding's size checks read (no device memory)."""
    import types

    import torch
    frame = types.SimpleNamespace(n=n, width=w, height=h)
    scene = types.SimpleNamespace(n=n, color=torch.zeros(n, c))
    return frame, scene


@pytest.mark.parametrize("bad", ["short_img", "f64_img", "short_g2d", "strided_g2d", "short_d_color"])
def test_gradient_and_image_bindings_refuse_bad_buffers(bad):
    """The kernels write whole images ([3][H][W]), 8 floats per Gaussian of g2d
    and per-Gaussian rows of the gradients: a buffer that is shorter, strided or
    not float32 is refused before anything launches."""
    import torch
    n, w, h = 10, 8, 6
    frame, scene = _fake_frame_scene(n, w, h)
    o = igs.opts(tile=16)
    img = torch.zeros(3, h, w)
    g2d = torch.zeros(n, 8)
    d_ms, d_op, d_col = torch.zeros(n, 4), torch.zeros(n), torch.zeros(n, 3)
    if bad == "short_img":
        img = img.view(-1)[:-1]
    elif bad == "f64_img":
        img = img.double()
    elif bad == "short_g2d":
        g2d = g2d[:-1]
    elif bad == "strided_g2d":
        g2d = torch.zeros(n, 16)[:, ::2]
    else:
        d_col = d_col[:-1]
    before = igs.launch_count()
    calls = [lambda: igs.render_bwd(scene, None, o, frame, img, g2d, d_ms, d_op, d_col)]
    if bad != "short_d_color":
        calls += [lambda: igs.render_fwd_clear(frame, o, img, g2d), lambda: igs.blend_bwd(frame, o, img, g2d),
                  lambda: igs.blend_bwd_acc(frame, o, img, g2d)]
    if bad in ("short_img", "f64_img"):
        calls.append(lambda: igs.render_fwd(frame, o, img))
    else:
        calls.append(lambda: igs.project_bwd(scene, None, o, frame, g2d, d_ms, d_op, d_col))
    for call in calls:
        with pytest.raises(ValueError):
            call()
    assert igs.launch_count() == before
