"""pgdto_project_noalloc against pgdto_project, through the C ABI.

The allocation-free entry point exists for callers that cannot call cudaMalloc (code
running inside someone else's CUDA-graph capture, processes whose device memory belongs to
another allocator, loops that must not block in the allocator).  It keeps its workspace in
one file-scope device array shared by every call, so this test makes two calls in a row on
different problems: the second must not be disturbed by what the first left behind.  This
file is collected last so that a run stopping at the first failure has run everything else.
"""

import numpy as np
import pytest

from paper_2511_13905_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_X = 1e-6
TOL_LAM = 1e-6


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


def test_noalloc_matches_project_on_two_calls_in_a_row(dev):
    import torch
    from paper_2511_13905_gb300 import binding

    for z, a, b, m, seg in _problems():
        zt = torch.from_numpy(z).to(dev)
        at = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        x_ref = torch.empty_like(zt)
        # the allocation-free entry is the grid engine without compaction lists: compare
        # with a handle running the same form
        h = binding.Handle(z.size, m, seg=seg, engine=1, compaction=0)
        st, lam_ref, info_ref = h.project(zt, at, b, x_ref)
        assert st == binding.PGDTO_OK
        h.close()
        x_na = torch.full_like(zt, float("nan"))
        st, lam_na, info_na = binding.project_noalloc(zt, at, b, x_na, m=m, seg=seg)
        torch.cuda.synchronize()
        assert st == binding.PGDTO_OK, binding.STATUS_NAMES.get(st, st)
        lam_ref = np.array(lam_ref)
        lam_na = np.array(lam_na)
        floor = 1e-3
        assert np.all(np.abs(lam_na - lam_ref) <= TOL_LAM * np.maximum(np.abs(lam_ref), floor))
        assert float(torch.max(torch.abs(x_na - x_ref)).item()) <= TOL_X
        assert info_na.passes == info_ref.passes


def test_noalloc_rejects_sizes_beyond_its_workspace(dev):
    import torch
    from paper_2511_13905_gb300 import binding
    z = torch.zeros(16, device=dev)
    st, _, _ = binding.project_noalloc(z, z, [0.0] * 5, z, m=5, seg=[0, 3, 6, 9, 12, 16])
    assert st == binding.PGDTO_ERR_ARG
