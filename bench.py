"""Benchmark of the PGD-TO optimizer step on GB300.

Default workload (the one the metric is quoted on): min volume under the nonlinear
compliance row, 3D 128x64x64 hex mesh, n = 524288, m = 1, a 50-step trajectory from t = 0.
A "step" is one full optimizer step (step size, PR+ direction, trial point, projection,
x_{t+1}) through pgdto_step.  Between timed steps the synthetic sensitivities for the new
design are regenerated on the device (the stand-in for the finite-element solve, not timed)
and L2 is flushed by writing a 256 MiB buffer, so every step starts from HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload 1..4]

N > 1 (under torchrun): each rank runs its own independent replica (weak scaling, no data
collective); the job value is the steps of all ranks over the slowest rank's time.
--impl reference times the FP64 CPU oracle (paper's Alg. 1/2 projection) on the host cores.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    1: "volume_2d_256x128 (n=32768, m=1, one step from a prior step)",
    2: "min_volume_3d_128x64x64 (n=524288, m=1, 50-step trajectory)",
    3: "multimaterial_3d_192x96x96_x4 (n=7077888, m=4 independent)",
    4: "volume_com_3d_256x128x128 (n=4194304, m=4 coupled)",
}
KERNEL_SOURCES = ["paper_2511_13905_gb300/csrc/seg_kernels.cu", "paper_2511_13905_gb300/csrc/dev_common.cuh",
                  "paper_2511_13905_gb300/csrc/coupled_kernels.cu", "paper_2511_13905_gb300/csrc/step_common.cuh",
                  "paper_2511_13905_gb300/csrc/kernels.h"]


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_traffic(workload):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernel."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(str(workload))
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def combine_ranks(total_s, steps, world, device=None):
    """Job value over ranks: every rank ran `steps` independent steps in `total_s` seconds;
    the job's time is the slowest rank's (MAX all-reduce), its work the sum of all ranks'."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_s)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return world * steps / total_s, total_s


def algorithmic_bytes(n, m_eff, passes):
    """Streaming bytes of one step: 16 + (20 + 4 m_eff) + 4 (1 + m_eff) P + (12 + 4 m_eff) per element."""
    return n * (16 + (20 + 4 * m_eff) + 4 * (1 + m_eff) * passes + (12 + 4 * m_eff))


# --------------------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_13905_gb300 import binding, inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    wl = args.workload
    if wl == 2:
        cfg = inputs.config2()
    elif wl == 1:
        cfg = inputs.config1()
    elif wl == 3:
        cfg = inputs.config3()
    else:
        cfg = inputs.config4()
    n, m = cfg["n"], cfg["m"]
    m_eff = m if cfg["mode"] == "coupled" else 1

    def T(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    h = binding.Handle(n, m, seg=cfg.get("seg"))
    x0 = T(cfg["x"])
    x = x0.clone()
    g = T(cfg["g"])
    G = cfg["G"]
    if wl == 2:
        s_dev = T(cfg["s"]).double()

        def sensitivities(xc):
            # synthetic compliance surrogate g(x) = sum s (1 - x^3): row -3 x^2 s, value g(x)
            xd = xc.double()
            A = (-3.0 * xd * xd * s_dev).float().reshape(1, n)
            gval = [float(torch.sum(s_dev * (1.0 - xd * xd * xd)).item())]
            return A, gval
    else:
        A_fixed = T(cfg["A"])

        def sensitivities(xc):
            if cfg["mode"] == "independent":
                seg = cfg["seg"]
                xd = xc.double()
                return A_fixed, [float(xd[seg[j]:seg[j + 1]].sum().item()) for j in range(m)]
            Ad = A_fixed.reshape(m, n).double()
            return A_fixed, (Ad @ xc.double()).tolist()

    def reset():
        x.copy_(x0)
        if cfg["t"] > 0:
            h.set_state(T(cfg["x_prev"]), T(cfg["g_prev"]), T(cfg["d_prev"]), cfg["t"])
        else:
            h.set_state(None, None, None, 0)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    trajectory = wl == 2

    # warm-up (also checks that the step succeeds)
    reset()
    for _ in range(args.warmup):
        A, gval = sensitivities(x)
        st, info = h.step(x, g, A, gval, G)
        if st != 0:
            raise RuntimeError("pgdto_step failed: %s" % binding.STATUS_NAMES.get(st, st))
        if not trajectory:
            reset()
    torch.cuda.synchronize()

    # timed steps (device time, CUDA events on the launching stream)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    torch.cuda.synchronize()
    launches0 = h.kernel_launches()
    evs = []
    passes = []
    for k in range(args.steps):
        A, gval = sensitivities(x)
        flush.fill_(float(k))
        # a bounded spin (about 0.1 ms) keeps the device busy while the host enqueues the
        # step (about 50 us through the Python binding), so the events bracket device work;
        # the host path is what the end-to-end figure measures
        torch.cuda._sleep(200_000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, _ = h.step(x, g, A, gval, G, want_info=False)
        e1.record(stream)
        evs.append((e0, e1))
        st2, _, info = h.last_info()
        if st != 0 or st2 not in (0, binding.PGDTO_NOT_CONVERGED):
            raise RuntimeError("step %d failed: %s / %s" % (k, st, st2))
        passes.append(info.passes)
        if not trajectory:
            reset()
    torch.cuda.synchronize()
    launches = h.kernel_launches() - launches0
    clk = clocks.stop()
    times_ms = [a.elapsed_time(b) for a, b in evs]
    value, total_s = combine_ranks(sum(times_ms) / 1e3, args.steps, world, dev)

    # end to end through the host-buffer entry point (pinned memory, copies inside the timing)
    xh = torch.from_numpy(cfg["x"].copy()).pin_memory()
    gh = g.cpu().pin_memory()
    reset()
    e2e_times = []
    for k in range(args.warmup + args.steps):
        A, gval = sensitivities(xh.to(dev))
        Ah = A.cpu().pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = h.step_host(xh, gh, Ah, gval, G)
        t1 = time.perf_counter()
        if st not in (0, binding.PGDTO_NOT_CONVERGED):
            raise RuntimeError("step_host failed: %s" % st)
        if k >= args.warmup:
            e2e_times.append(t1 - t0)
        if not trajectory:
            xh.copy_(torch.from_numpy(cfg["x"]))
            reset()
    e2e_value, e2e_total = combine_ranks(sum(e2e_times), len(e2e_times), world, dev)
    a_bytes = 4 * (m * n if cfg["mode"] == "coupled" or wl in (1, 2) else n)
    h2d = 4 * n * 2 + a_bytes
    d2h = 4 * n

    avg_passes = sum(passes) / len(passes)
    step_s = total_s / args.steps
    alg_bytes = algorithmic_bytes(n, m_eff, avg_passes)
    peak, peak_kind = peaks()
    achieved = alg_bytes / step_s / 1e9
    result = {
        "metric": "PGD-TO optimizer steps/s",
        "value": value,
        "unit": "steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * step_s,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (compensated sums, f64 scalars)",
        "data": "synthetic",
        "config": {"workload": cfg["name"], "n": n, "m": m, "mode": cfg["mode"],
                   "trajectory": "50-step run from t=0" if trajectory else "one step from the seeded state",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "timing": "CUDA events on the launching stream; a bounded spin kernel ahead of the start "
                             "event keeps the device busy while the host enqueues the step",
                   "parallelism": "replicas" if world > 1
                   else "single GPU", "avg_projection_passes": avg_passes},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(wl),
                     "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                     else "fallback", "kernel": "pgdto::seg_kernel (fused step)",
                     "algorithmic_bytes_per_launch": alg_bytes},
        "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "api": "pgdto_step_host (pinned host buffers)"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    h.close()
    return result


# --------------------------------------------------------------------------- batched

def run_batched(args, local_rank=0):
    """B instances of the 256x128 single-row workload (n = 32,768 each, seeds 0..B-1), one
    step each from the seeded state: one pgdto_step_many launch (batched) against B
    pgdto_step launches back to back on the same stream (plain).  Device time by CUDA
    events around each form; state reset and an L2 flush between timed repetitions."""
    import numpy as np
    import torch

    from paper_2511_13905_gb300 import binding, inputs
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    B = args.batch_instances
    cfgs = [inputs.config1(seed_offset=k) for k in range(B)]
    n = cfgs[0]["n"]

    def T(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    hs = [binding.Handle(c["n"], 1) for c in cfgs]
    x0 = [T(c["x"]) for c in cfgs]
    xs = [t.clone() for t in x0]
    gs = [T(c["g"]) for c in cfgs]
    As = [T(c["A"]) for c in cfgs]
    prev = [(T(c["x_prev"]), T(c["g_prev"]), T(c["d_prev"])) for c in cfgs]
    gvals = [c["gval"] for c in cfgs]
    Gs = [c["G"] for c in cfgs]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def reset():
        for k in range(B):
            xs[k].copy_(x0[k])
            hs[k].set_state(prev[k][0], prev[k][1], prev[k][2], cfgs[k]["t"])

    def batched():
        st, _ = binding.step_many(hs, xs, gs, As, gvals, Gs, want_info=False)
        if st != binding.PGDTO_OK:
            raise RuntimeError("pgdto_step_many failed: %s" % st)

    def plain():
        for k in range(B):
            st, _ = hs[k].step(xs[k], gs[k], As[k], gvals[k], Gs[k], want_info=False)
            if st != binding.PGDTO_OK:
                raise RuntimeError("pgdto_step failed: %s" % st)

    def timed(fn, reps):
        out, passes = [], []
        for r in range(args.warmup + reps):
            reset()
            flush.fill_(float(r))
            l0 = sum(h.kernel_launches() for h in hs)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            # a bounded spin (about 2 ms) keeps the device busy while the host marshals the
            # B problems, so the events bracket device work only
            torch.cuda._sleep(4_000_000)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            launches = sum(h.kernel_launches() for h in hs) - l0
            infos = [h.last_info()[2] for h in hs]
            bad = [i.status for i in infos if i.status not in (0, binding.PGDTO_NOT_CONVERGED)]
            if bad:
                raise RuntimeError("batched workload step failed: %s" % bad[:4])
            if r >= args.warmup:
                out.append(e0.elapsed_time(e1))
                passes.append(sum(i.passes for i in infos))
        return float(np.median(out)), float(np.mean(passes)), launches, [h.last_info()[2] for h in hs]

    t_b, passes_b, launches_b, info_b = timed(batched, args.steps)
    x_b = [x.cpu().numpy() for x in xs]
    t_p, passes_p, launches_p, info_p = timed(plain, args.steps)
    diff = max(float(np.max(np.abs(a.astype(np.float64) - x.cpu().numpy()))) for a, x in zip(x_b, xs))
    bytes_b = sum(algorithmic_bytes(n, 1, i.passes) for i in info_b)
    peak, _ = peaks()
    for h in hs:
        h.close()
    return {"workload": "%d x volume_2d_256x128 (n=%d, m=1, one step each)" % (B, n),
            "batched": {"ms": t_b, "steps_per_s": B / (t_b / 1e3), "launches": launches_b,
                        "passes_per_instance": passes_b / B,
                        "roofline": {"bound": "hbm", "achieved": bytes_b / (t_b / 1e3) / 1e9, "peak": peak,
                                     "unit": "GB/s", "frac": bytes_b / (t_b / 1e3) / 1e9 / peak,
                                     "traffic": measured_traffic("batched") if B == 256 else None,
                                     "algorithmic_bytes_per_launch": bytes_b}},
            "plain": {"ms": t_p, "steps_per_s": B / (t_p / 1e3), "launches": launches_p,
                      "passes_per_instance": passes_p / B},
            "max_abs_diff_x_batched_vs_plain": diff,
            "timing": "median of %d CUDA-event-timed repetitions, L2 flushed (256 MiB write) before each; "
                      "the events bracket device work (the host marshals behind a spin kernel)" % args.steps}


# --------------------------------------------------------------------------- serving

def run_serving(args, local_rank=0):
    """Served (continuous batching) vs plain (one launch per request) on the same offered load.

    `sessions` design sessions from the serving workload recipe (n log-uniform in
    [4096, n_max], m in {1, 2, 4}, half of the m > 1 sessions independent, half coupled).
    In each of `waves` waves every session submits its next step at once; a request's
    latency runs from the wave's start to the moment its rho_{t+1} is in host memory.
    Plain: the same requests one after another, each its own launch (H2D of grad f and A,
    pgdto_step, D2H of x).  Both move the same bytes per request."""
    import numpy as np
    import torch

    from paper_2511_13905_gb300 import binding, inputs
    dev = torch.device("cuda", local_rank)
    reqs = inputs.serving_requests(count=args.serve_sessions, n_max=args.serve_nmax)
    probs = [inputs.request_problem(r) for r in reqs]
    rng = np.random.default_rng(inputs.SEED_BASE + 77)
    grads = [[(p["g"] * np.float32(1.0 + 0.05 * k)).astype(np.float32) for k in range(2)] for p in probs]
    waves = args.serve_waves

    def constraint_values(p, x):
        # g_j(x_t) at the session's current design (all rows are linear here), computed by
        # the client between waves, outside the timed region
        x = x.astype(np.float64)
        if p["mode"] == "independent":
            return np.add.reduceat(x, p["seg"][:-1])
        return np.atleast_2d(p["A"]).astype(np.float64) @ x

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]

    # served
    srv = binding.Server(budget_bytes=64 << 30, max_sessions=len(probs) + 1)
    outs = [np.empty(p["n"], np.float32) for p in probs]
    gvals = [np.asarray(p["gval"], np.float64) for p in probs]
    nc_served = 0
    lat = []
    warm = True
    t_total = 0.0
    for w in range(waves + 1):
        t0 = srv.clock_us()
        tickets = []
        for i, p in enumerate(probs):
            st, t = srv.submit(i, p["n"], p["m"], grads[i][w % 2], np.ascontiguousarray(p["A"]), gvals[i], p["G"],
                               outs[i], x0=p["x"] if w == 0 else None, seg=p.get("seg"))
            if st != binding.PGDTO_OK:
                raise RuntimeError("submit failed: %s" % st)
            tickets.append(t)
        done_at = {}
        for i in range(len(tickets)):
            # blocking waits; each completion time was stamped by the server when published
            st, d, _, t_done = srv.wait(tickets[i])
            if st != binding.PGDTO_OK or d not in (binding.PGDTO_OK, binding.PGDTO_NOT_CONVERGED):
                raise RuntimeError("served step failed: %s / %s" % (st, d))
            nc_served += int(d == binding.PGDTO_NOT_CONVERGED)
            done_at[i] = t_done
        t1 = max(done_at.values())
        if not warm:
            lat += [(done_at[i] - t0) * 1e-6 for i in range(len(probs))]
            t_total += (t1 - t0) * 1e-6
        warm = False
        gvals = [constraint_values(p, outs[i]) for i, p in enumerate(probs)]
    stats = srv.stats()
    srv.close()
    served_final = [o.copy() for o in outs]
    served = {"p50_ms": 1e3 * pct(lat, 0.5), "p99_ms": 1e3 * pct(lat, 0.99),
              "steps_per_s": len(lat) / t_total, "launches": stats["batches"], "not_converged": nc_served}

    # plain: one launch per request
    handles = [binding.Handle(p["n"], p["m"], seg=p.get("seg")) for p in probs]
    xd = [torch.from_numpy(p["x"].copy()).to(dev) for p in probs]
    gd = [torch.empty(p["n"], device=dev) for p in probs]
    Ad = [torch.empty(np.asarray(p["A"]).size, device=dev) for p in probs]
    # the same host arrays the served arm submits (pageable NumPy memory), copied by DMA
    # straight to and from the device as the server does
    ghost = [[torch.from_numpy(g) for g in gg] for gg in grads]
    Ahost = [torch.from_numpy(np.ascontiguousarray(p["A"]).ravel()) for p in probs]
    for h in handles:
        h.set_state(None, None, None, 0)
    gvals = [np.asarray(p["gval"], np.float64) for p in probs]
    nc_plain = 0
    lat_p = []
    t_total_p = 0.0
    warm = True
    for w in range(waves + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, p in enumerate(probs):
            gd[i].copy_(ghost[i][w % 2])
            Ad[i].copy_(Ahost[i])
            st, _ = handles[i].step(xd[i], gd[i], Ad[i], gvals[i], p["G"], want_info=True)
            if st not in (binding.PGDTO_OK, binding.PGDTO_NOT_CONVERGED):
                raise RuntimeError("plain step failed: %s" % st)
            nc_plain += int(st == binding.PGDTO_NOT_CONVERGED)
            torch.from_numpy(outs[i]).copy_(xd[i])
            if not warm:
                lat_p.append(time.perf_counter() - t0)
        t1 = time.perf_counter()
        if not warm:
            t_total_p += t1 - t0
        warm = False
        gvals = [constraint_values(p, outs[i]) for i, p in enumerate(probs)]
    for h in handles:
        h.close()
    plain = {"p50_ms": 1e3 * pct(lat_p, 0.5), "p99_ms": 1e3 * pct(lat_p, 0.99),
             "steps_per_s": len(lat_p) / t_total_p, "not_converged": nc_plain}
    # equal accuracy: both arms ran the same trajectories; the designs they end on
    diff = max(float(np.max(np.abs(a.astype(np.float64) - b.astype(np.float64)))) for a, b in zip(served_final, outs))
    return {"sessions": len(probs), "waves": waves, "requests_timed": len(lat),
            "n_range": [min(p["n"] for p in probs), max(p["n"] for p in probs)],
            "modes": {m: sum(1 for p in probs if p["mode"] == m) for m in ("single", "independent", "coupled")},
            "served": served, "plain": plain, "max_abs_diff_final_x": diff,
            "latency": "wave start to rho_{t+1} in host memory; every session submits one step per wave"}


# --------------------------------------------------------------------------- oracle

def oracle_workload(wl):
    from paper_2511_13905_gb300 import inputs
    if wl == 2:
        return inputs.config2()
    return {1: inputs.config1, 3: inputs.config3, 4: inputs.config4}[wl]()


def time_oracle_steps(wl, nsteps, budget_s):
    """Oracle steps ('paper' projector: Alg. 1 bisection / Alg. 2) on the workload; (steps, seconds)."""
    import numpy as np
    from oracle.step import oracle_step
    from paper_2511_13905_gb300 import inputs
    cfg = oracle_workload(wl)
    n = cfg["n"]
    x = cfg["x"].astype(np.float32)
    xp = cfg.get("x_prev", np.zeros(n, np.float32))
    gp = cfg.get("g_prev", np.zeros(n, np.float32))
    dp = cfg.get("d_prev", np.zeros(n, np.float32))
    t = cfg["t"]
    done, spent = 0, 0.0
    while done < nsteps and spent < budget_s:
        if wl == 2:
            A, gval = inputs.config2_inputs(cfg, x)
        else:
            A, gval = cfg["A"], cfg["gval"]
        t0 = time.perf_counter()
        ref = oracle_step(x, xp, cfg["g"], gp, dp, A, gval, cfg["G"], t, mode=cfg["mode"], seg=cfg.get("seg"),
                          projector="paper")
        spent += time.perf_counter() - t0
        done += 1
        if wl == 2:
            xp, gp, dp = x, cfg["g"], ref["d"].astype(np.float32)
            x = ref["x_new"].astype(np.float32)
            t += 1
    return done, spent


def cpu_baseline_subprocess(wl, nsteps, budget_s):
    """Run the oracle timing in a child pinned to one BLAS/OpenMP thread; returns the dict."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; d, s = bench.time_oracle_steps(%d, %d, %f); "
            "print(json.dumps([d, s]))" % (ROOT, wl, nsteps, budget_s))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    done, spent = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": done / spent, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": "%d oracle steps of the same workload (FP64 NumPy, Alg. 1 bisection / Alg. 2 as printed), "
                      "%.1f s of CPU time" % (done, spent)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    wl = args.workload
    # warm-up steps untimed, then K timed steps, each a full oracle step on the whole workload
    time_oracle_steps(wl, args.warmup, 60.0)
    done, spent = time_oracle_steps(wl, args.steps, 240.0)
    v = done / spent
    cfg_name = WORKLOADS[wl]
    return {
        "impl": "reference", "metric": "PGD-TO optimizer steps/s", "value": v, "unit": "steps/s",
        "n_gpus": 1, "steps": done, "warmup": args.warmup, "ms_per_step": 1e3 * spent / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg_name, "runs_on": "host CPU, 1 thread"},
        "cpu_baseline": {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
                         "sample": "%d full oracle steps (FP64 NumPy, Alg. 1 / Alg. 2 as printed)" % done},
        "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=2, choices=[1, 2, 3, 4])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--serve-sessions", type=int, default=48)
    ap.add_argument("--serve-waves", type=int, default=12)
    ap.add_argument("--serve-nmax", type=int, default=1 << 20)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_batched:
        res["batched"] = run_batched(args, local_rank)
    if rank == 0 and world == 1 and not args.no_serving:
        res["serving"] = run_serving(args, local_rank)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            res["cpu_baseline"] = cpu_baseline_subprocess(args.workload, 1000, 20.0)
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
