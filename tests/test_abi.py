"""The C-ABI library builds, loads and exports every symbol include/ddks.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os

import pytest

import paper_2106_13706_gb300 as pkg
from paper_2106_13706_gb300 import build as bld


@pytest.fixture(scope="module")
def lib():
    bld.build()
    return pkg.load()


def test_header_declares_the_boundary():
    names = pkg.declared_symbols()
    for n in ["ddks_ctx_create", "ddks_ctx_destroy", "ddks_distance", "ddks_distance_range",
              "ddks_permutation_test", "ddks_significance", "ddks_batch_distance", "ddks_submit",
              "ddks_poll", "ddks_strerror", "ddks_ctx_stats", "ddks_config_default", "ddks_vdks",
              "ddks_rdks", "ddks_rescale"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in pkg.declared_symbols():
        assert hasattr(lib, n), n
        assert isinstance(getattr(lib, n), ctypes._CFuncPtr)


def test_strerror_and_version(lib):
    assert pkg.ddks_strerror(0) == "ok"
    assert "NaN" in pkg.ddks_strerror(-2)
    assert pkg.ddks_version().count(".") == 2


def test_argument_errors_need_no_gpu(lib):
    # argument checks happen before any CUDA call
    r = pkg.binding.ddks_result()
    assert lib.ddks_distance(None, None, 1, None, 1, 3, 0, None, ctypes.byref(r)) == -1
    assert lib.ddks_ctx_destroy(None) == -1
    assert lib.ddks_vdks(None, None, 1, None, 1, 3, 0, 8, None, ctypes.byref(r)) == -1
    assert lib.ddks_rdks(None, None, 1, None, 1, 3, 0, None, ctypes.byref(r), None) == -1
    lib.ddks_rescale.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.ddks_rescale(None, None, 1, 0.0, 1.0, None, None) == -1


def test_library_is_in_tree():
    assert os.path.dirname(pkg.binding.LIB_PATH) == os.path.dirname(bld.__file__)


def test_config_defaults(lib):
    cfg = pkg.binding.ddks_config()
    cfg.radix_min_n = 123
    lib.ddks_config_default(ctypes.byref(cfg))
    assert cfg.radix_min_n == 0 and cfg.graphs == 1 and cfg.device == -1 and cfg.register_variant == 0
    # the binding's struct matches the header's field order and size
    names = [n for n, _ in pkg.binding.ddks_config._fields_]
    assert names[-3:] == ["radix_min_n", "register_variant", "rank_kernel"]
    assert names.index("graphs") == len(names) - 4
    assert ctypes.sizeof(pkg.binding.ddks_config) == 56


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the built library every entry point raises
    b = pkg.binding
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b, "LIB_PATH", str(tmp_path / "libddks.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        b.load()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        b.ddks_ctx_create(device=0)


def test_pointer_classification_refuses_other_devices(lib):
    # cudaMemoryType: 0 unregistered, 1 host, 2 device, 3 managed
    f = lib.ddks_classify_pointer
    assert f(2, 0, 0) == 1 and f(2, 3, 3) == 1      # device memory of the call's device: in place
    assert f(2, 1, 0) == -1 and f(2, 0, 1) == -1    # another GPU's memory: refused, never read
    assert f(3, 0, 1) == 1                          # managed memory: in place
    assert f(0, -2, 0) == 0 and f(1, 0, 5) == 0     # host memory: copied by the call
    assert f(7, 0, 0) == -1                         # unknown type
