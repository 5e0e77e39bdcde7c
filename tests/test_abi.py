"""The C-ABI library loads, exports every symbol include/vg.h declares, and its
structs have the layout the Python binding marshals (no GPU needed: only
argument checks that return before any CUDA call are exercised)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2403_11247_b300 import build as B
from paper_2403_11247_b300 import vg as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vg.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return V.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(vg_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vg_scene_upload", "vg_render_fwd", "vg_render_bwd", "vg_pose_grad", "vg_rvq_decode"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", V.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (vg_\w+)", out))
    assert set(names) <= exported
    assert set(V.exported_symbols()) <= exported


def test_struct_layouts_match_the_c_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "vg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(vg_camera), sizeof(vg_attr_group), sizeof(vg_scene_desc),
         sizeof(vg_render_params), sizeof(vg_scene_grads), sizeof(vg_stats), sizeof(vg_adam_tensor));
  printf("%zu %zu %zu %zu\\n", offsetof(vg_scene_desc, rot), offsetof(vg_scene_desc, mask_eps),
         offsetof(vg_render_params, pose_dev), offsetof(vg_camera, near_plane));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    sizes, offs = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.strip().split("\n")
    assert [int(x) for x in sizes.split()] == [C.sizeof(t) for t in (V.vg_camera, V.vg_attr_group, V.vg_scene_desc,
                                                                      V.vg_render_params, V.vg_scene_grads,
                                                                      V.vg_stats, V.vg_adam_tensor)]
    assert [int(x) for x in offs.split()] == [V.vg_scene_desc.rot.offset, V.vg_scene_desc.mask_eps.offset,
                                              V.vg_render_params.pose_dev.offset, V.vg_camera.near_plane.offset]


def test_default_params_are_the_stated_readings(lib):
    p = lib.vg_default_params()
    assert p.tile == 16 and p.jacobian_clamp == 1
    assert abs(p.alpha_max - 0.99) < 1e-7 and abs(p.alpha_min - 1 / 255) < 1e-9 and abs(p.t_min - 1e-4) < 1e-10
    assert abs(p.dilation - 0.3) < 1e-7 and p.sigma_cull == 3.0 and abs(p.clamp_factor - 1.3) < 1e-7


def test_argument_errors_return_before_any_cuda_call(lib):
    out = C.c_void_p()
    assert lib.vg_scene_upload(None, 0, None, C.byref(out)) == V.VG_ERR_INVALID_ARG
    assert b"null" in lib.vg_last_error()
    d = V.vg_scene_desc()
    d.n_anchors, d.k = 10, 0
    assert lib.vg_scene_upload(C.byref(d), 0, None, C.byref(out)) == V.VG_ERR_INVALID_ARG
    d.k = 4
    d.anchor_xyz = d.anchor_l = d.offsets = 16  # never dereferenced: the group check fails first
    d.logscale.dim = 2
    assert lib.vg_scene_upload(C.byref(d), 0, None, C.byref(out)) == V.VG_ERR_INVALID_ARG
    assert b"dim" in lib.vg_last_error()
    assert lib.vg_render_fwd(None, None, 1, None, None, None, None, None, None) == V.VG_ERR_INVALID_ARG
    assert lib.vg_render_bwd(None, None, 1, None, None, None, None, None, None, None) == V.VG_ERR_INVALID_ARG
    assert lib.vg_pose_grad(None, 1, None, None, None, None, None) == V.VG_ERR_INVALID_ARG
    g = V.vg_attr_group(3, 2, 300, None, None, None)
    assert lib.vg_rvq_decode(C.byref(g), 10, C.c_void_p(16), None) == V.VG_ERR_INVALID_ARG
    assert lib.vg_ctx_create(-1, C.byref(out)) == V.VG_ERR_INVALID_ARG
    dev = C.c_void_p(256)  # never dereferenced: every call below fails its argument checks first
    assert lib.vg_frame_decode(1, 4, 4, None, dev, C.c_float(1000.0), dev, dev, None) == V.VG_ERR_INVALID_ARG
    assert lib.vg_frame_decode(0, 4, 4, dev, dev, C.c_float(1000.0), dev, dev, None) == V.VG_ERR_INVALID_ARG
    assert lib.vg_frame_decode(1, 4, 4, dev, dev, C.c_float(0.0), dev, dev, None) == V.VG_ERR_INVALID_ARG
    assert lib.vg_frame_decode(1, 4, 4, dev, dev, C.c_float(float("nan")), dev, dev, None) == V.VG_ERR_INVALID_ARG
    assert lib.vg_loss_l1(0, 10, *([None] * 5), 0.5, -1.0, *([None] * 6)) == V.VG_ERR_INVALID_ARG


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2403_11247_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle|liboracle|vg_oracle|orc_", text, flags=re.M), f


def test_host_stage_copies_like_memcpy_at_any_alignment_and_size(lib):
    """The streaming-store staging copy is host only: it runs without a GPU."""
    import torch
    rng = np.random.default_rng(3)
    for n in (0, 1, 15, 16, 63, 64, 65, 1000, 4099):
        for off in (0, 1, 7, 16):
            src = rng.integers(0, 256, size=n).astype(np.uint8)
            dst = torch.zeros(n + off, dtype=torch.uint8)
            V.vg_host_stage(dst[off:], src)
            assert np.array_equal(dst.numpy()[off:], src) and not dst.numpy()[:off].any()
    with pytest.raises(ValueError):
        V.vg_host_stage(torch.zeros(3), np.zeros(4, np.float32))
