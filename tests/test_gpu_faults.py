"""Device-side failure detection without a GPU fault: a wait that nothing releases runs out
of a short budget, the call reports PGDTO_ERR_TIMEOUT, and the GPU and the handle keep
working.  The failure is made on the host (fault_inject makes block 0 leave before the
first grid reduction); nothing traps, faults or hangs."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _problem(dev, n=100000, m=1):
    import torch
    rng = np.random.default_rng(5)
    z = torch.from_numpy(rng.uniform(-0.2, 1.2, n).astype(np.float32)).to(dev)
    if m == 1:
        A = torch.from_numpy(rng.uniform(0.5, 1.5, n).astype(np.float32)).to(dev)
    else:
        A = torch.from_numpy(rng.uniform(0.5, 1.5, (m, n)).astype(np.float32)).to(dev)
    b = [0.4 * n] * m
    return z, A, b


@pytest.mark.parametrize("m", [1, 3])
def test_wait_that_runs_out_reports_timeout_and_recovers(dev, m):
    import torch
    from paper_2511_13905_gb300 import binding
    z, A, b = _problem(dev, m=m)
    n = z.numel()
    mode = "single" if m == 1 else "coupled"
    bad = binding.Handle(n, m, mode=mode, barrier_timeout_ms=50, fault_inject=1)
    x = torch.empty_like(z)
    st, lam, info = bad.project(z, A, b, x)
    assert st == binding.PGDTO_ERR_TIMEOUT
    # the error is reported once; a healthy handle on the same GPU works at once
    good = binding.Handle(n, m, mode=mode)
    st, lam, info = good.project(z, A, b, x)
    torch.cuda.synchronize()
    assert st == binding.PGDTO_OK
    assert lam[0] > 0
    # and the faulty handle reports the same condition again, not a stale success
    st, _, _ = bad.project(z, A, b, x)
    assert st == binding.PGDTO_ERR_TIMEOUT
    bad.close()
    good.close()


def test_fault_inject_rejects_unknown_values(dev):
    from paper_2511_13905_gb300 import binding
    with pytest.raises(binding.PgdtoError):
        binding.Handle(16, 1, fault_inject=2)
