"""CPU-only checks of the C-ABI library: it builds, loads, and exports every
symbol include/abfs.h declares.  No compute call is made without a GPU."""
import ctypes

import pytest

import paper_1906_03113_gb300 as abfs
from paper_1906_03113_gb300 import binding


@pytest.fixture(scope="module")
def lib():
    abfs.build()
    return abfs.load()


def test_exports_every_declared_symbol(lib):
    names = binding.declared_symbols()
    assert "abfs_run" in names and "abfs_graph_create" in names and "abfs_run_batch" in names
    for name in names:
        assert hasattr(lib, name), name


def test_strerror_and_version(lib):
    assert lib.abfs_strerror(0) == b"ok"
    assert b"timeout" in lib.abfs_strerror(5) or b"wait" in lib.abfs_strerror(5)
    assert lib.abfs_version() >= 10000


def test_default_params_are_valid(lib):
    p = abfs.default_params()
    assert p.mode == abfs.MODE_SUBMATRIX
    assert 32 <= p.tile <= 1024 and p.tile % 32 == 0
    assert p.unit_entries >= 256 and p.unit_entries & (p.unit_entries - 1) == 0
    assert p.timeout_ms > 0
    assert lib.abfs_check_params(ctypes.byref(p)) == 0


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    out = ctypes.c_void_p()
    # null arrays, n = 0
    assert lib.abfs_graph_create(None, None, 0, 0, 0, 0, None, ctypes.byref(out)) == binding.ERR_INVALID_ARG
    # n too large for this build
    colptr = (ctypes.c_uint32 * 2)(0, 0)
    assert lib.abfs_graph_create(colptr, None, 1 << 31, 0, 0, 0, None, ctypes.byref(out)) == binding.ERR_UNSUPPORTED
    # malformed CSC caught by host validation (colptr[n] != nnz)
    bad = (ctypes.c_uint32 * 3)(0, 1, 3)
    rows = (ctypes.c_uint32 * 2)(1, 0)
    assert lib.abfs_graph_create(bad, rows, 2, 2, 0, binding.VALIDATE, None,
                                 ctypes.byref(out)) == binding.ERR_INVALID_ARG
    # row index out of range
    cp = (ctypes.c_uint32 * 3)(0, 1, 2)
    rows = (ctypes.c_uint32 * 2)(5, 0)
    assert lib.abfs_graph_create(cp, rows, 2, 2, 0, binding.VALIDATE, None,
                                 ctypes.byref(out)) == binding.ERR_INVALID_ARG
    # asymmetric pattern declared undirected
    rows = (ctypes.c_uint32 * 2)(1, 1)
    assert lib.abfs_graph_create(cp, rows, 2, 2, 0, binding.VALIDATE, None,
                                 ctypes.byref(out)) == binding.ERR_NOT_SYMMETRIC
    # null handles
    assert lib.abfs_run(None, 0, None, None, None, None, None) == binding.ERR_INVALID_ARG
    assert lib.abfs_run_counts(None, 0, None, None, None, None, None, None) == binding.ERR_INVALID_ARG
    assert lib.abfs_run_host_many(None, None, 0, None, None, None, None, None) == binding.ERR_INVALID_ARG
    assert lib.abfs_graph_relabel(None) == binding.ERR_INVALID_ARG
    assert lib.abfs_batch_create_counts(None, None, 0, None, None, None, None, None,
                                        None) == binding.ERR_INVALID_ARG
    cal = binding.Calibration()
    assert lib.abfs_calibrate(9, ctypes.byref(cal), None) == binding.ERR_INVALID_ARG
    assert lib.abfs_calibrate(27, ctypes.byref(cal), None) == binding.ERR_INVALID_ARG
    assert lib.abfs_calibrate(16, None, None) == binding.ERR_INVALID_ARG
    assert lib.abfs_graph_destroy(None) == binding.ERR_INVALID_ARG
    assert lib.abfs_batch_destroy(None) == binding.ERR_INVALID_ARG


def test_parameter_validation(lib):
    p = abfs.default_params()
    size = ctypes.c_size_t()
    assert set(p.as_dict()) >= {"mode", "tile", "unit_entries", "narrow_max", "narrow_edges",
                                "ctas_per_sm", "shrink_theta", "shrink_max", "timeout_ms"}
    # footprint of a null graph is an argument error, not a crash
    assert lib.abfs_graph_footprint(None, ctypes.byref(p), ctypes.byref(size)) == binding.ERR_INVALID_ARG
    assert lib.abfs_check_params(None) == binding.ERR_INVALID_ARG

    def check(**kw):
        return lib.abfs_check_params(ctypes.byref(abfs.default_params(**kw)))

    ok, bad = 0, binding.ERR_INVALID_ARG
    for kw in (dict(tile=32), dict(tile=1024), dict(unit_entries=256), dict(unit_entries=65536),
               dict(mode=abfs.MODE_PLAIN), dict(ctas_per_sm=1), dict(shrink_theta=0.5, shrink_max=2),
               dict(narrow_resident=0), dict(claim_scan=0), dict(claim_scan=1),
               dict(narrow_max=0, narrow_edges=0), dict(bottom_up_alpha=5, bottom_up_beta=24),
               dict(bottom_up_alpha=0xFFFFFFFF, bottom_up_beta=0), dict(cluster_ctas=1),
               dict(cluster_ctas=16), dict(multi_source=0), dict(multi_source=64)):
        assert check(**kw) == ok, kw
    for kw in (dict(tile=16), dict(tile=1056), dict(tile=100), dict(unit_entries=128),
               dict(unit_entries=768), dict(unit_entries=131072), dict(mode=2), dict(ctas_per_sm=0),
               dict(ctas_per_sm=9), dict(shrink_theta=-0.1), dict(shrink_theta=1.5),
               dict(timeout_ms=0), dict(narrow_resident=2), dict(cluster_ctas=0),
               dict(cluster_ctas=17),
               # the hybrid reads the input columns: submatrix mode without shrink only
               dict(mode=abfs.MODE_PLAIN, bottom_up_alpha=5),
               dict(bottom_up_alpha=5, shrink_theta=0.5, shrink_max=1)):
        assert check(**kw) == bad, kw
