"""The C-ABI library loads and exports every symbol include/pgdto.h declares; host-side
argument checks answer without a GPU."""

import ctypes

import pytest

from paper_2511_13905_gb300 import binding


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = binding.declared_symbols()
    assert "pgdto_step" in names and "pgdto_project" in names and "pgdto_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_params_default_are_the_papers(lib):
    p = binding.params_default()
    assert p.C == 1e12 and p.alpha_max == 1e2 and p.tol_B == 1e-8 and p.tol_N == 1e-6
    assert p.alpha_fallback == 0.2 and p.eps_alpha == 1e-6 and p.t_warmup == 50 and p.omega == 1.0
    assert p.c1 == 1e-4 and p.c2 == 0.9
    assert p.stage1 == 0 and p.compaction == 0 and p.cluster_elems == 0
    assert lib.pgdto_params_default(None) == binding.PGDTO_ERR_ARG


@pytest.mark.parametrize("n,m,seg,lo,hi", [
    (0, 1, None, 0.0, 1.0),          # empty problem
    (10, 0, None, 0.0, 1.0),         # no rows
    (10, 5, None, 0.0, 1.0),         # more rows than supported
    (10, 1, None, 1.0, 1.0),         # lo == hi
    (10, 1, None, float("nan"), 1.0),
    (10, 2, [0, 5, 9], 0.0, 1.0),    # segments do not cover n
    (10, 2, [0, 0, 10], 0.0, 1.0),   # empty segment
    (10, 2, [0, 7, 5], 0.0, 1.0),    # non-monotone
])
def test_create_rejects_bad_arguments(lib, n, m, seg, lo, hi):
    h = ctypes.c_void_p()
    segarr = (ctypes.c_int64 * len(seg))(*seg) if seg is not None else None
    st = lib.pgdto_create(ctypes.byref(h), n, m, segarr, lo, hi, None, None)
    assert st == binding.PGDTO_ERR_ARG
    assert not h.value


def test_bad_params_rejected(lib):
    h = ctypes.c_void_p()
    p = binding.params_default(C=-1.0)
    assert lib.pgdto_create(ctypes.byref(h), 10, 1, None, 0.0, 1.0, ctypes.byref(p), None) == binding.PGDTO_ERR_ARG
    p = binding.params_default(max_passes=0)
    assert lib.pgdto_create(ctypes.byref(h), 10, 1, None, 0.0, 1.0, ctypes.byref(p), None) == binding.PGDTO_ERR_ARG
    p = binding.params_default(stage1=2)
    assert lib.pgdto_create(ctypes.byref(h), 10, 1, None, 0.0, 1.0, ctypes.byref(p), None) == binding.PGDTO_ERR_ARG


def test_null_handle_calls(lib):
    assert lib.pgdto_step(None, None, None, None, None, None, None) == binding.PGDTO_ERR_ARG
    assert lib.pgdto_project(None, None, None, None, None, None, None) == binding.PGDTO_ERR_ARG
    assert lib.pgdto_set_state(None, None, None, None, 0) == binding.PGDTO_ERR_ARG
    assert lib.pgdto_kernel_launches(None) == -1
    lib.pgdto_destroy(None)
    assert b"sm_103a" in lib.pgdto_version()


@pytest.mark.parametrize("n,count", [(0, 8), (131073, 8), (4096, 0), (4096, 4097)])
def test_autotune_rejects_sizes_outside_its_range(lib, n, count):
    best = ctypes.c_int(-1)
    assert lib.pgdto_autotune_batch(n, count, ctypes.byref(best), None, None) == binding.PGDTO_ERR_ARG
    assert best.value == -1
    lib.pgdto_autotune_reset()
