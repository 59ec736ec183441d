"""C-ABI checks that need no GPU: the library builds, loads and exports every entry
point the headers under include/ declare; the ctypes structures match the C layout;
host-only helpers and argument validation behave as documented."""
import ctypes
import glob
import json
import math
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1904_06017_gb300 as sg
from paper_1904_06017_gb300 import build as sgbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


@pytest.fixture(scope="module")
def lib():
    sgbuild.build()
    return sg.load_library()


def declared_functions():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(stereo_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(HEADERS) >= 2 and len(names) >= 25
    assert "stereo_softargmin_bwd" in names and "stereo_dt_refine_roll" in names
    out = subprocess.run(["nm", "-D", "--defined-only", sg.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (stereo_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_every_declared_function_has_a_ctypes_signature(lib):
    """Without argtypes ctypes would pass device pointers as 32-bit ints: every entry point the
    headers declare must have its argument and return types set by the binding."""
    untyped = [n for n in declared_functions() if getattr(lib, n).argtypes is None]
    assert not untyped, untyped
    # each signature has as many arguments as the header's declaration
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for name, params in re.findall(r"\b(stereo_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
            n = 0 if params.strip() in ("", "void") else params.count(",") + 1
            assert len(getattr(lib, name).argtypes) == n, (name, n)


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "stereo.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(stereo_params), offsetof(stereo_params, lambda0),
         offsetof(stereo_params, max_iters), sizeof(stereo_dt_result), offsetof(stereo_dt_result, n),
         sizeof(stereo_pair_desc), offsetof(stereo_pair_desc, psi_init), offsetof(stereo_pair_desc, delta_t),
         offsetof(stereo_pair_desc, wta_dev));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [ctypes.sizeof(sg.stereo_params), sg.stereo_params.lambda0.offset,
                    sg.stereo_params.max_iters.offset, ctypes.sizeof(sg.stereo_dt_result),
                    sg.stereo_dt_result.n.offset, ctypes.sizeof(sg.stereo_pair_desc),
                    sg.stereo_pair_desc.psi_init.offset, sg.stereo_pair_desc.delta_t.offset,
                    sg.stereo_pair_desc.wta_dev.offset]


def test_defaults_are_the_paper_constants(lib):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    p = sg.stereo_params_default()
    assert p.sigma0 == pytest.approx(g["sigma0"]["value"])
    assert p.sigma1 == pytest.approx(g["sigma1"]["value"])
    assert p.bil == g["bilateral_window"]["value"]
    assert p.bil * p.bil - 1 == g["neighbourhood_size"]["value"]
    assert p.lambda0 == g["lambda0"]["value"]
    assert p.delta_psi == pytest.approx(g["delta_psi_rad"]["value"], rel=1e-15)
    assert p.delta_psi == pytest.approx(math.pi / 1.8e6, rel=1e-15)


def test_row_shift_affine(lib):
    s = sg.stereo_row_shift_affine(5, 2.0, 0.5, 1.0)
    assert np.allclose(s, [1.0, 1.5, 2.0, 2.5, 3.0])
    with pytest.raises(sg.StereoError) as e:
        sg.stereo_row_shift_affine(0, 0, 0, 0)
    assert e.value.code == sg.STEREO_EINVAL


@pytest.mark.parametrize("field,value", [("width", 0), ("height", -3), ("pitch", 100),
                                         ("max_disp", 0), ("max_disp", 1000), ("win", 4),
                                         ("win", 13), ("bil", 17), ("bil", 2), ("sigma0", 0.0),
                                         ("sigma1", float("nan")), ("cost_dtype", 7),
                                         ("lambda0", -1.0), ("max_iters", 0)])
def test_create_rejects_bad_parameters(lib, field, value):
    p = sg.stereo_params_default(width=320, height=240, pitch=320, max_disp=64)
    setattr(p, field, value)
    with pytest.raises(sg.StereoError) as e:
        sg.stereo_create(p)
    assert e.value.code == sg.STEREO_EINVAL
    assert "stereo_create" in sg.stereo_last_error()


def test_null_pointers_rejected(lib):
    rc = lib.stereo_create(None, None)
    assert rc == sg.STEREO_EINVAL
    assert lib.stereo_warp_target(None, None, None, None, None) == sg.STEREO_EINVAL
    assert lib.stereo_cost_aggregate_wta(None, None, None, None, None, None, None, None) == sg.STEREO_EINVAL
    assert lib.stereo_cost_aggregate_wta_ex(None, None, None, None, None, None, None, None, None) == sg.STEREO_EINVAL
    assert lib.stereo_disparity_transform(None, None, None, 0.0, 0.0, None, None, None) == sg.STEREO_EINVAL
    assert lib.stereo_destroy(None) == sg.STEREO_OK
    assert lib.stereo_lr_check(None, None, None, None, None, None, None, 1.0, None) == sg.STEREO_EINVAL


def test_version(lib):
    assert "sm_103a" in sg.stereo_version()


def test_diff_struct_layout_matches_header(tmp_path):
    from paper_1904_06017_gb300 import diff as sgd
    prog = tmp_path / "layout_diff.c"
    prog.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "stereo_diff.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(stereo_diff_params), offsetof(stereo_diff_params, sigma0),
         offsetof(stereo_diff_params, temperature), offsetof(stereo_diff_params, warp_mode));
  return 0;
}''')
    exe = tmp_path / "layout_diff"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [ctypes.sizeof(sgd.stereo_diff_params), sgd.stereo_diff_params.sigma0.offset,
                    sgd.stereo_diff_params.temperature.offset, sgd.stereo_diff_params.warp_mode.offset]


def test_diff_defaults_and_workspace_size(lib):
    from paper_1904_06017_gb300 import diff as sgd
    p = sgd.stereo_diff_params_default()
    assert (p.win, p.bil, p.batch) == (9, 11, 1)
    assert p.sigma0 == pytest.approx(1.5) and p.sigma1 == pytest.approx(5.5)
    assert p.temperature == pytest.approx(0.1)
    p = sgd.stereo_diff_params_default(width=960, height=540, batch=8, max_disp=64)
    n = sgd.stereo_softargmin_workspace_bytes(p)
    W, H, B, D, rw = 960, 540, 8, 64, 4
    vol = B * D * H * W * 4
    # three volumes (c, h, dS/dc) and per-pixel arrays; the cost adjoint's Gamma(X, d) is summed
    # along its diagonals inside the kernel, so no fourth volume
    assert 3 * vol <= n <= 3.3 * vol
    assert n % 256 == 0
    # grows linearly in the batch
    p1 = sgd.stereo_diff_params_default(width=960, height=540, batch=1, max_disp=64)
    assert abs(n - 8 * sgd.stereo_softargmin_workspace_bytes(p1)) < 8 * 16 * 256
    assert sgd.stereo_dt_energy_workspace_bytes(8) >= 8 * 64 * 10 * 8


@pytest.mark.parametrize("field,value", [("width", 0), ("height", 9000), ("batch", 0), ("batch", 65),
                                         ("max_disp", 0), ("max_disp", 257), ("win", 4), ("win", 17),
                                         ("bil", 0), ("sigma0", -1.0), ("sigma1", float("inf")),
                                         ("temperature", 0.0)])
def test_diff_rejects_bad_parameters(lib, field, value):
    from paper_1904_06017_gb300 import diff as sgd
    p = sgd.stereo_diff_params_default(width=64, height=48, max_disp=16)
    setattr(p, field, value)
    with pytest.raises(sg.StereoError) as e:
        sgd.stereo_softargmin_workspace_bytes(p)
    assert e.value.code == sg.STEREO_EINVAL


def test_diff_rejects_null_and_small_workspaces(lib):
    from paper_1904_06017_gb300 import diff as sgd
    p = sgd.stereo_diff_params_default(width=64, height=48, max_disp=16)
    fake = 1 << 20          # never dereferenced: every check below fails before a launch
    assert lib.stereo_softargmin_fwd(ctypes.byref(p), fake, fake, fake, fake, None, 0, None) == sg.STEREO_EINVAL
    assert lib.stereo_softargmin_fwd(ctypes.byref(p), fake, fake, fake, fake, fake + 16, 1 << 30,
                                     None) == sg.STEREO_EINVAL
    assert "aligned" in sg.stereo_last_error()
    assert lib.stereo_softargmin_fwd(ctypes.byref(p), fake, fake, fake, fake, fake, 256, None) == sg.STEREO_EINVAL
    assert "needed" in sg.stereo_last_error()
    assert lib.stereo_softargmin_bwd(ctypes.byref(p), fake, fake, fake, None, fake, fake, None, fake, 1 << 40,
                                     None) == sg.STEREO_EINVAL
    p.warp_mode = 2
    assert lib.stereo_softargmin_fwd(ctypes.byref(p), fake, fake, fake, fake, fake, 1 << 40, None) == sg.STEREO_EINVAL
    assert "warp_mode" in sg.stereo_last_error()
    assert lib.stereo_dt_energy_fwd(64, 48, 1, fake, None, fake, fake, fake, 16, None) == sg.STEREO_EINVAL
    assert lib.stereo_dt_energy_bwd(0, 48, 1, fake, None, fake, fake, fake, fake, fake, 1 << 20,
                                    None) == sg.STEREO_EINVAL
    assert lib.stereo_dt_refine_roll(64, 48, 1, fake, None, 0.0, 1001, fake, fake, 1 << 20,
                                     None) == sg.STEREO_EINVAL
    assert lib.stereo_dt_refine_roll(64, 48, 1, fake, None, float("nan"), 5, fake, fake, 1 << 20,
                                     None) == sg.STEREO_EINVAL
