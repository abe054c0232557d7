"""Free-set compaction (Sec. 4.2.1, params.compaction = 1) against the oracle on problems
whose CTA shares stream from global memory (where it applies): single rows, an equality
row on a negative bracket, the four-material step, and the 524,288-variable step; its lists
are used (a pass visits only part of the elements) and it gives the same answer to the
tolerance."""

import numpy as np
import pytest

from oracle import oracle_step
from oracle import projection as P
from oracle.checks import parity_errors
from paper_2511_13905_gb300 import inputs

pytestmark = pytest.mark.gpu
C = 1e12
TOL = {"lam_rel": 1e-6, "x_abs": 1e-6, "viol_rel": 1e-6}


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


def check(err, what=""):
    bad = {k: err[k] for k in TOL if not err[k] <= TOL[k]}
    assert not bad, "%s parity: %s (all: %s)" % (what, bad, {k: err[k] for k in TOL})


@pytest.mark.parametrize("n,seed,eq", [(1 << 22, 1, False), (3000017, 2, False), (1 << 22, 3, True)])
def test_compacted_projection(dev, n, seed, eq):
    import torch
    from paper_2511_13905_gb300 import binding
    rng = np.random.default_rng(seed)
    z = rng.uniform(-0.3, 1.3, n).astype(np.float32)
    a = rng.lognormal(0.0, 1.0, n).astype(np.float32)
    a64, z64 = a.astype(np.float64), z.astype(np.float64)
    b = float(a64 @ np.clip(z64, 0, 1)) * (1.2 if eq else 0.7)
    out = {}
    for cm in (0, 1):
        h = binding.Handle(n, 1, compaction=cm, eq_mask=int(eq), engine=1)
        xt = torch.empty(n, device=dev)
        st, lam, info = h.project(T(z, dev), T(a, dev), [b], xt)
        torch.cuda.synchronize()
        h.close()
        assert st == 0, info.as_dict(1)
        out[cm] = (np.array(lam), xt.cpu().numpy().astype(np.float64), info.visited)
    lr = P.solve_single_exact(z64, a64, b, 0.0, 1.0, C, equality=eq)
    if eq:
        assert lr < 0.0
    xr = np.clip(z64 - lr * a64, 0, 1)
    lam, x, vis = out[1]
    check(parity_errors(x, lam, xr, [lr], a[None, :], [b], C, 0.0, 1.0, eq=[eq]), "n=%d" % n)
    # the lists were in use: a later pass visited only part of the row, fewer in all
    assert vis % n != 0, vis
    assert vis < out[0][2], (vis, out[0][2])


def test_compacted_four_material_step(dev):
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config3()
    infos = {}
    for cm in (0, 1):
        h = binding.Handle(cfg["n"], 4, seg=cfg["seg"], compaction=cm)
        h.set_state(T(cfg["x_prev"], dev), T(cfg["g_prev"], dev), T(cfg["d_prev"], dev), cfg["t"])
        x = T(cfg["x"], dev)
        st, info = h.step(x, T(cfg["g"], dev), T(cfg["A"], dev), cfg["gval"], cfg["G"])
        torch.cuda.synchronize()
        h.close()
        assert st == 0
        infos[cm] = (info, x.cpu().numpy().astype(np.float64))
    ref = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"],
                      cfg["G"], cfg["t"], mode="independent", seg=cfg["seg"])
    seg = cfg["seg"]
    a = cfg["A"].astype(np.float64)

    def f(xv):
        ax = np.array([a[seg[j]:seg[j + 1]] @ xv[seg[j]:seg[j + 1]] for j in range(4)])
        aa = np.array([np.abs(a[seg[j]:seg[j + 1]]) @ np.abs(xv[seg[j]:seg[j + 1]]) for j in range(4)])
        return ax, aa
    info, x = infos[1]
    check(parity_errors(x, np.array(list(info.lambda_)[:4]), ref["x_new"], ref["lam"], f, ref["b"], C, 0.0, 1.0,
                        amax=np.ones(4)), "four materials")
    assert info.visited < infos[0][0].visited, (info.visited, infos[0][0].visited)


def test_compacted_single_cta_step_config2(dev):
    """The 524,288-variable step on one CTA (cluster engine, cluster_elems = n): the share is
    far beyond shared memory, so it streams from global memory and compaction runs (the
    cluster kernel's compaction variant)."""
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config2()
    n = cfg["n"]
    A, gval = inputs.config2_inputs(cfg, cfg["x"])
    # one CTA for half a million variables: the share cannot be resident, so compaction runs
    h = binding.Handle(n, 1, compaction=1, engine=2, cluster_elems=n)
    h.set_state(None, None, None, 0)
    x = T(cfg["x"], dev)
    st, info = h.step(x, T(cfg["g"], dev), T(A, dev), gval, cfg["G"])
    torch.cuda.synchronize()
    h.close()
    assert st == 0
    ref = oracle_step(cfg["x"], np.zeros(n), cfg["g"], np.zeros(n), np.zeros(n), A, gval, cfg["G"], 0)
    check(parity_errors(x.cpu().numpy(), [info.lambda_[0]], ref["x_new"], ref["lam"], A, ref["b"], C, 0.0, 1.0),
          "config2 single CTA")
