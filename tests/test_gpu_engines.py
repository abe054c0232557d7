"""Both execution engines against the oracle, and the batched form (many problems in one
launch) against the same problems run alone.

grid engine:    every SM on one problem, grid-wide reductions through global memory;
cluster engine: one thread-block cluster per problem, reductions in distributed shared
                memory; a list of problems runs in one launch."""

import numpy as np
import pytest

from oracle import oracle_step
from oracle import projection as P
from oracle.checks import parity_errors
from paper_2511_13905_gb300 import inputs

pytestmark = pytest.mark.gpu
C = 1e12
TOL = {"lam_rel": 1e-6, "x_abs": 1e-6, "viol_rel": 1e-6}
GRID, CLUSTER = 1, 2


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


def seg_fn(a, seg):
    a = np.asarray(a, dtype=np.float64)

    def f(x):
        ax = np.array([a[seg[j]:seg[j + 1]] @ x[seg[j]:seg[j + 1]] for j in range(len(seg) - 1)])
        aa = np.array([np.abs(a[seg[j]:seg[j + 1]]) @ np.abs(x[seg[j]:seg[j + 1]]) for j in range(len(seg) - 1)])
        return ax, aa
    return f


def oracle_for(cfg):
    return oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"],
                       cfg["G"], cfg["t"], mode=cfg["mode"], seg=cfg.get("seg"))


def errors(cfg, ref, x, lam):
    if cfg["mode"] == "independent":
        seg = cfg["seg"]
        amax = np.array([np.max(np.abs(cfg["A"][seg[j]:seg[j + 1]])) for j in range(len(seg) - 1)])
        return parity_errors(x, lam, ref["x_new"], ref["lam"], seg_fn(cfg["A"], seg), ref["b"], C, 0.0, 1.0,
                             amax=amax)
    return parity_errors(x, lam, ref["x_new"], ref["lam"], cfg["A"], ref["b"], C, 0.0, 1.0)


def step_one(dev, cfg, engine):
    import torch
    from paper_2511_13905_gb300 import binding
    h = binding.Handle(cfg["n"], cfg["m"], seg=cfg.get("seg"), engine=engine)
    h.set_state(T(cfg["x_prev"], dev), T(cfg["g_prev"], dev), T(cfg["d_prev"], dev), cfg["t"])
    x = T(cfg["x"], dev)
    st, info = h.step(x, T(cfg["g"], dev), T(cfg["A"], dev), cfg["gval"], cfg["G"])
    torch.cuda.synchronize()
    h.close()
    return st, info, x.cpu().numpy().astype(np.float64)


CFGS = [("wl1", lambda: inputs.config1()), ("wl1_small", lambda: inputs.config1(dims=(40, 25))),
        ("wl3_small", lambda: inputs.config3(dims=(24, 16, 12))),
        ("wl3_ragged", lambda: inputs.config3(dims=(13, 11, 7), materials=3))]


@pytest.mark.parametrize("engine", [GRID, CLUSTER])
@pytest.mark.parametrize("name,make", CFGS, ids=[c[0] for c in CFGS])
def test_step_both_engines(dev, engine, name, make):
    cfg = make()
    st, info, x = step_one(dev, cfg, engine)
    assert st == 0
    ref = oracle_for(cfg)
    assert info.alpha == pytest.approx(ref["alpha"], rel=1e-6)
    check(errors(cfg, ref, x, np.array(list(info.lambda_)[:cfg["m"]])), "%s engine %d" % (name, engine))


@pytest.mark.parametrize("engine", [GRID, CLUSTER])
def test_config2_full_size_both_engines(dev, engine):
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config2()
    n = cfg["n"]
    A, gval = inputs.config2_inputs(cfg, cfg["x"])
    h = binding.Handle(n, 1, engine=engine)
    h.set_state(None, None, None, 0)
    x = T(cfg["x"], dev)
    st, info = h.step(x, T(cfg["g"], dev), T(A, dev), gval, cfg["G"])
    torch.cuda.synchronize()
    assert st == 0
    ref = oracle_step(cfg["x"], np.zeros(n), cfg["g"], np.zeros(n), np.zeros(n), A, gval, cfg["G"], 0)
    check(parity_errors(x.cpu().numpy(), [info.lambda_[0]], ref["x_new"], ref["lam"], A, ref["b"], C, 0.0, 1.0),
          "wl2 engine %d" % engine)
    h.close()


def _mix():
    """Problems of uneven size and mode: single rows and independent rows."""
    out = [inputs.config1(dims=(64, 32)), inputs.config3(dims=(16, 12, 10)), inputs.config1(dims=(7, 5)),
           inputs.config3(dims=(21, 9, 8), materials=2), inputs.config1(dims=(300, 200)),
           inputs.config1(dims=(33, 17), seed_offset=5)]
    return out


def test_step_many_equals_each_alone_and_the_oracle(dev):
    import torch
    from paper_2511_13905_gb300 import binding
    cfgs = _mix()
    hs, xs, gs, As = [], [], [], []
    for c in cfgs:
        h = binding.Handle(c["n"], c["m"], seg=c.get("seg"), engine=CLUSTER)
        h.set_state(T(c["x_prev"], dev), T(c["g_prev"], dev), T(c["d_prev"], dev), c["t"])
        hs.append(h)
        xs.append(T(c["x"], dev))
        gs.append(T(c["g"], dev))
        As.append(T(c["A"], dev))
    st, infos = binding.step_many(hs, xs, gs, As, [c["gval"] for c in cfgs], [c["G"] for c in cfgs])
    torch.cuda.synchronize()
    assert st == 0
    for c, h, x, info in zip(cfgs, hs, xs, infos):
        st1, info1, x1 = step_one(dev, c, CLUSTER)
        assert st1 == 0
        xm = x.cpu().numpy().astype(np.float64)
        assert np.array_equal(xm, x1), c["name"]  # bit-identical alone and in the mix
        assert list(info.lambda_) == list(info1.lambda_)
        ref = oracle_for(c)
        check(errors(c, ref, xm, np.array(list(info.lambda_)[:c["m"]])), c["name"] + " in batch")
        assert h.get_state() == c["t"] + 1
        h.close()


def test_project_many(dev):
    import torch
    from paper_2511_13905_gb300 import binding
    rng = np.random.default_rng(9)
    sizes = [5, 1000, 77777, 4096, 31]
    hs, zs, As, bs, outs, probs = [], [], [], [], [], []
    for n in sizes:
        z = rng.uniform(-0.3, 1.3, n).astype(np.float32)
        a = rng.lognormal(0, 1, n).astype(np.float32)
        b = [0.6 * float(a.astype(np.float64) @ np.clip(z, 0, 1))]
        hs.append(binding.Handle(n, 1, engine=CLUSTER))
        zs.append(T(z, dev))
        As.append(T(a, dev))
        bs.append(b)
        outs.append(torch.empty(n, device=dev))
        probs.append((z, a, b))
    st, lams, infos = binding.project_many(hs, zs, As, bs, outs)
    torch.cuda.synchronize()
    assert st == 0
    for (z, a, b), lam, out in zip(probs, lams, outs):
        lr = P.solve_single_exact(z.astype(np.float64), a.astype(np.float64), b[0], 0.0, 1.0, C)
        xr = np.clip(z.astype(np.float64) - lr * a, 0, 1)
        check(parity_errors(out.cpu().numpy(), lam, xr, [lr], a[None, :], b, C, 0.0, 1.0), "n=%d" % z.size)
    for h in hs:
        h.close()


def test_step_many_rejects_bad_lists(dev):
    from paper_2511_13905_gb300 import binding
    cfg = inputs.config1(dims=(8, 8))
    h = binding.Handle(cfg["n"], 1)
    x = T(cfg["x"], dev)
    st, _ = binding.step_many([h, h], [x, x], [x, x], [x, x], [cfg["gval"]] * 2, [cfg["G"]] * 2)
    assert st == binding.PGDTO_ERR_ARG  # the same handle twice
    hc = binding.Handle(64, 2, mode="coupled")
    y = T(np.zeros(128, np.float32), dev)
    st, _ = binding.step_many([hc], [y], [y], [y], [[0, 0]], [[1, 1]])
    assert st == binding.PGDTO_ERR_ARG  # coupled rows are not served by the cluster engine
    h.close()
    hc.close()


@pytest.mark.parametrize("S", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("name,make", CFGS[:1] + CFGS[3:], ids=["wl1", "wl3_ragged"])
def test_cluster_sizes(dev, S, name, make):
    """The cluster engine at every cluster size (params.cluster_elems sets it from n)."""
    import torch
    from paper_2511_13905_gb300 import binding
    cfg = make()
    n = cfg["n"]
    h = binding.Handle(n, cfg["m"], seg=cfg.get("seg"), engine=CLUSTER, cluster_elems=-(-n // S))
    h.set_state(T(cfg["x_prev"], dev), T(cfg["g_prev"], dev), T(cfg["d_prev"], dev), cfg["t"])
    x = T(cfg["x"], dev)
    st, info = h.step(x, T(cfg["g"], dev), T(cfg["A"], dev), cfg["gval"], cfg["G"])
    torch.cuda.synchronize()
    h.close()
    assert st == 0
    ref = oracle_for(cfg)
    check(errors(cfg, ref, x.cpu().numpy().astype(np.float64), np.array(list(info.lambda_)[:cfg["m"]])),
          "%s S=%d" % (name, S))


def test_step_many_every_cluster_size(dev):
    """One batch whose problems need clusters of 1, 2, 4, 8 and 16 blocks (five launches on
    forked streams): each result equals the same problem run alone, and the oracle's."""
    import torch
    from paper_2511_13905_gb300 import binding
    cfgs = [inputs.config1(dims=d, seed_offset=k) for k, d in
            enumerate([(50, 40), (120, 100), (250, 120), (300, 200), (400, 300), (61, 29), (128, 64)])]
    hs, xs = [], []
    for c in cfgs:
        h = binding.Handle(c["n"], 1)
        h.set_state(T(c["x_prev"], dev), T(c["g_prev"], dev), T(c["d_prev"], dev), c["t"])
        hs.append(h)
        xs.append(T(c["x"], dev))
    st, infos = binding.step_many(hs, xs, [T(c["g"], dev) for c in cfgs], [T(c["A"], dev) for c in cfgs],
                                  [c["gval"] for c in cfgs], [c["G"] for c in cfgs])
    torch.cuda.synchronize()
    assert st == 0
    launches = sum(h.kernel_launches() for h in hs)
    assert launches == 5, launches
    for c, h, x, info in zip(cfgs, hs, xs, infos):
        st1, info1, x1 = step_one(dev, c, CLUSTER)
        assert st1 == 0
        xm = x.cpu().numpy().astype(np.float64)
        assert np.array_equal(xm, x1), c["name"]
        ref = oracle_for(c)
        check(errors(c, ref, xm, np.array(list(info.lambda_)[:1])), c["name"] + " in batch")
        h.close()
