"""The C-ABI library loads and exports every entry point that
include/artemis.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "artemis.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(art_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._build_module().build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["art_create", "art_destroy", "art_load_octree", "art_load_skeleton", "art_set_pose",
                 "art_set_camera", "art_render_feature_maps", "art_load_shader", "art_shade", "art_sort_pairs"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (art_\w+)", out))
    assert set(declared_functions()) <= exported


def test_package_imports_and_fails_loudly_without_library(tmp_path):
    import paper_2202_05628_gb300 as art
    assert os.path.exists(art.LIB_PATH)
    with pytest.raises(ImportError):
        art.load_library(str(tmp_path / "missing.so"))


def test_flat_params_layout():
    import numpy as np
    import paper_2202_05628_gb300 as art
    import scenegen as sg
    layers = sg.tiny_net_weights(0, cin=4, mid=8)
    p = art.flat_params(layers)
    n = sum(w.size + b.size for w, b in layers)
    assert p.shape == (n,)
    np.testing.assert_array_equal(p[:layers[0][0].size], layers[0][0].ravel())


def test_no_gpu_means_no_context(lib_path):
    # the library has no CPU path: without a CUDA device art_create returns
    # ART_ERR_CUDA and no context, and the Python binding raises
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    lib = ctypes.CDLL(lib_path)
    lib.art_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.art_create(ctypes.byref(h), None) == 2 and h.value is None
    import paper_2202_05628_gb300 as art
    with pytest.raises((RuntimeError, art.ArtemisError)):
        art.Renderer()
