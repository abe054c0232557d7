"""The batched form's autotuner (pgdto_autotune_batch) through the C ABI.

It times batched steps of synthetic problems for each candidate cluster-engine block share
and records the fastest for the device and n's power-of-two bucket; handles created
afterwards with cluster_elems = 0 take that share.  Whatever it picks, a problem's step
must stay bit-identical alone and in a batch (both handles created under the same table)
and within the parity tolerance of the oracle.  The table is cleared at the end so that
later tests see the built-in share.
"""

import numpy as np
import pytest

from oracle import oracle_step
from oracle.checks import parity_errors
from paper_2511_13905_gb300 import inputs

pytestmark = pytest.mark.gpu
C = 1e12
TOL = 1e-6
DIMS = (128, 64)  # n = 8192, the 2D volume row at a size the oracle runs in well under a second


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def T(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def test_autotuned_share_keeps_batch_equal_to_alone_and_the_oracle(dev):
    import torch
    from paper_2511_13905_gb300 import binding
    cfgs = [inputs.config1(dims=DIMS, seed_offset=k) for k in range(6)]
    n = cfgs[0]["n"]
    try:
        st, best, ms = binding.autotune_batch(n, 64)
        assert st == binding.PGDTO_OK, binding.STATUS_NAMES.get(st, st)
        assert best in (1024, 2048, 4096, 8192)
        assert ms > 0.0
        print("autotune n=%d x 64: cluster_elems=%d, %.4f ms per batched step" % (n, best, ms))

        def make(c):
            h = binding.Handle(c["n"], 1, engine=2)
            h.set_state(T(c["x_prev"], dev), T(c["g_prev"], dev), T(c["d_prev"], dev), c["t"])
            return h

        hs = [make(c) for c in cfgs]
        xs = [T(c["x"], dev) for c in cfgs]
        st, infos = binding.step_many(hs, xs, [T(c["g"], dev) for c in cfgs], [T(c["A"], dev) for c in cfgs],
                                      [c["gval"] for c in cfgs], [c["G"] for c in cfgs])
        torch.cuda.synchronize()
        assert st == binding.PGDTO_OK
        for c, h, x, info in zip(cfgs, hs, xs, infos):
            h.close()
            h1 = make(c)
            x1 = T(c["x"], dev)
            st1, info1 = h1.step(x1, T(c["g"], dev), T(c["A"], dev), c["gval"], c["G"])
            torch.cuda.synchronize()
            h1.close()
            assert st1 == binding.PGDTO_OK
            assert torch.equal(x, x1)
            assert info.lambda_[0] == info1.lambda_[0]
            ref = oracle_step(c["x"], c["x_prev"], c["g"], c["g_prev"], c["d_prev"], c["A"], c["gval"], c["G"],
                              c["t"], mode=c["mode"])
            err = parity_errors(x.cpu().numpy().astype(np.float64), np.array([info.lambda_[0]]), ref["x_new"],
                                ref["lam"], c["A"], ref["b"], C, 0.0, 1.0)
            assert err["lam_rel"] <= TOL and err["x_abs"] <= TOL and err["viol_rel"] <= TOL, err
    finally:
        binding.autotune_reset()
