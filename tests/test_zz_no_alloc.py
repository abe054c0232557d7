"""pgdto_project_noalloc against pgdto_project and the FP64 oracle, through the C ABI.

The allocation-free entry point exists for callers that cannot call cudaMalloc: processes
whose device memory belongs to another allocator (a framework's caching allocator, or a
pool fixed at start-up) and loops that must not block in the driver's allocator.  It keeps
its workspace in one file-scope device array shared by every call, so this test makes two
calls in a row on different problems: the second must not be disturbed by what the first
left behind.  Each result is compared with a handle's pgdto_project and with the oracle
(lambda relative, x absolute and scaled row residual, each within 1e-6).  A wait that runs
out (made on the host: block 0 leaves before the first reduction) must come back as
PGDTO_ERR_TIMEOUT, never as the previous call's report.  This file is collected last so
that a run stopping at the first failure has run everything else.
"""

import numpy as np
import pytest

from paper_2511_13905_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-6
C = 1e12


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _problems():
    rng = np.random.default_rng(2024)
    n1 = 200003
    z1 = rng.uniform(-0.3, 1.3, n1).astype(np.float32)
    a1 = rng.lognormal(0.0, 1.0, n1).astype(np.float32)
    b1 = [0.6 * float(a1.astype(np.float64) @ np.clip(z1, 0, 1))]
    cfg = inputs.config3(dims=(24, 16, 16))
    n2 = cfg["n"]
    z2 = (cfg["x"].astype(np.float64) + 0.3 * rng.standard_normal(n2)).astype(np.float32)
    return [(z1, a1, b1, 1, None), (z2, cfg["A"], list(cfg["G"]), 4, [int(s) for s in cfg["seg"]])]


def _oracle(z, a, b, m, seg):
    from oracle import projection as P
    z64 = z.astype(np.float64)
    a64 = np.asarray(a, dtype=np.float64)
    if m == 1:
        lam = np.array([P.solve_single_exact(z64, a64, float(b[0]), 0.0, 1.0, C)])
        x = P.primal_from_dual(z64, a64[None, :], lam, 0.0, 1.0)
        return lam, x
    lam = P.solve_independent_exact(z64, a64, seg, np.asarray(b, np.float64), 0.0, 1.0, C)
    return lam, P.independent_primal(z64, a64, seg, lam, 0.0, 1.0)


def _dense_rows(a, m, seg):
    a64 = np.asarray(a, dtype=np.float64)
    if m == 1:
        return a64[None, :]
    A = np.zeros((m, a64.size))
    for j in range(m):
        A[j, seg[j]:seg[j + 1]] = a64[seg[j]:seg[j + 1]]
    return A


def test_noalloc_matches_project_and_oracle_on_two_calls_in_a_row(dev):
    import torch
    from oracle.checks import parity_errors
    from paper_2511_13905_gb300 import binding

    for z, a, b, m, seg in _problems():
        zt = torch.from_numpy(z).to(dev)
        at = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        x_ref = torch.empty_like(zt)
        h = binding.Handle(z.size, m, seg=seg, engine=1, compaction=0)
        st, lam_ref, _ = h.project(zt, at, b, x_ref)
        assert st == binding.PGDTO_OK
        h.close()
        x_na = torch.full_like(zt, float("nan"))
        st, lam_na, _ = binding.project_noalloc(zt, at, b, x_na, m=m, seg=seg)
        torch.cuda.synchronize()
        assert st == binding.PGDTO_OK, binding.STATUS_NAMES.get(st, st)
        x_na_h = x_na.cpu().numpy().astype(np.float64)
        lam_o, x_o = _oracle(z, a, b, m, seg)
        A = _dense_rows(a, m, seg)
        err = parity_errors(x_na_h, np.array(lam_na), x_o, lam_o, A, np.asarray(b, np.float64), C, 0.0, 1.0)
        err_h = parity_errors(x_ref.cpu().numpy().astype(np.float64), np.array(lam_ref), x_o, lam_o, A,
                              np.asarray(b, np.float64), C, 0.0, 1.0)
        print("no-alloc n=%d m=%d vs oracle: %s; pgdto_project vs oracle: %s" % (z.size, m, err, err_h))
        assert err["lam_rel"] <= TOL and err["x_abs"] <= TOL and err["viol_rel"] <= TOL, err
        # and against the handle's result, on the same tolerance
        lam_ref = np.array(lam_ref)
        floor = 1e-3
        assert np.all(np.abs(np.array(lam_na) - lam_ref) <= TOL * np.maximum(np.abs(lam_ref), floor))
        assert float(torch.max(torch.abs(x_na - x_ref)).item()) <= TOL


def test_noalloc_wait_that_runs_out_reports_timeout(dev):
    import torch
    from paper_2511_13905_gb300 import binding

    z, a, b, m, seg = _problems()[0]
    zt = torch.from_numpy(z).to(dev)
    at = torch.from_numpy(a).to(dev)
    x = torch.empty_like(zt)
    st, lam_good, _ = binding.project_noalloc(zt, at, b, x, m=m, seg=seg)
    assert st == binding.PGDTO_OK
    assert binding.noalloc_set_test_fault(1, 50) == binding.PGDTO_OK
    try:
        st, lam_bad, info = binding.project_noalloc(zt, at, b, x, m=m, seg=seg)
    finally:
        assert binding.noalloc_set_test_fault(0, 0) == binding.PGDTO_OK
    assert st == binding.PGDTO_ERR_TIMEOUT
    assert info.status == binding.PGDTO_ERR_TIMEOUT
    assert not np.isfinite(lam_bad[0])  # the unpublished report, not the previous call's lambda
    st, lam_again, _ = binding.project_noalloc(zt, at, b, x, m=m, seg=seg)
    torch.cuda.synchronize()
    assert st == binding.PGDTO_OK
    assert lam_again[0] == lam_good[0]


def test_noalloc_rejects_sizes_beyond_its_workspace(dev):
    import torch
    from paper_2511_13905_gb300 import binding
    z = torch.zeros(16, device=dev)
    st, _, _ = binding.project_noalloc(z, z, [0.0] * 5, z, m=5, seg=[0, 3, 6, 9, 12, 16])
    assert st == binding.PGDTO_ERR_ARG
