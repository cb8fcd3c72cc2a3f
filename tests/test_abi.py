"""The C-ABI library builds, loads without a GPU, and exports every function
include/gsreg.h declares; host-side logic that needs no device."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsreg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gs_status_t|void|const char \*|size_t|int)\s*\*?\s*(gs_\w+)\s*\(", text,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2408_10154_gb300 import build, gsreg
    build.build()
    return gsreg.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("gs_project", "gs_render", "gs_render_backward", "gs_register", "gs_loss", "gs_fuse",
              "gs_pose_step", "gs_bin", "gs_transform", "gs_ctx_create", "gs_ctx_destroy", "gs_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2408_10154_gb300 import gsreg
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(gsreg.EXPORTS) == set(declared_functions())


def test_default_options_match_the_oracle(lib):
    from paper_2408_10154_gb300 import gsreg
    o = gsreg.default_options()
    assert o.tile == int(O.DEFAULT_OPT[0])
    np.testing.assert_array_equal(np.float32([o.z_near, o.dilation, o.alpha_min, o.alpha_max, o.t_min]),
                                  O.DEFAULT_OPT[1:6])
    np.testing.assert_allclose([o.lr_rot, o.lr_trans, o.beta1, o.beta2, o.adam_eps, o.lr_final], O.DEFAULT_HYPER,
                               rtol=1e-6)
    assert o.tracking_loss == 0 and np.float32(o.lambda_c) == np.float32(O.TRACK_LAMBDA_C)
    assert o.exposure == 0 and np.float32(o.lr_exposure) == np.float32(0.1) and o.tile_schedule == 0 and o.tight_lists == 1
    assert np.float32(o.list_headroom) == np.float32(1.5)


def test_structs_match_the_library(lib):
    from paper_2408_10154_gb300 import gsreg
    structs = gsreg.abi_structs()
    sizes = (ctypes.c_size_t * len(structs))()
    assert lib.gs_abi_sizes(sizes, len(structs)) == len(structs)
    for st, sz in zip(structs, sizes):
        assert ctypes.sizeof(st) == sz, st.__name__
    assert ctypes.sizeof(gsreg.gs_camera_t) == 72 and ctypes.sizeof(gsreg.gs_options_t) == 4 * 25


def test_context_without_device_is_rejected(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    assert lib.gs_ctx_create(0, 0, ctypes.byref(h)) == 1  # GS_ERR_INVALID_ARG
    assert lib.gs_last_error(None) == b"null context"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no fallback path: without the compiled library the binding raises
    # before any work, for the loader and for a context alike
    from paper_2408_10154_gb300 import build, gsreg
    monkeypatch.setattr(build, "LIB", str(tmp_path / "libgsreg.so"))
    monkeypatch.setattr(gsreg, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        gsreg.load()
    with pytest.raises(RuntimeError, match="not built"):
        gsreg.Context(0)
