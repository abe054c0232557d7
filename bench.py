"""Benchmark of the PGD-TO optimizer step on GB300.

Headline (``value``, ``roofline``, ``e2e``, ``cpu_baseline``): the largest single-GPU
workload, four materials on a 3D 192x96x96 mesh, n = 7,077,888 variables in four
independent volume rows, one full optimizer step from the seeded state (t = 1).  A "step"
is one pgdto_step: step size, PR+ direction, trial point, projection, x_{t+1}.  Between
timed steps the handle's state is reset to the seeded one and L2 is flushed by writing a
256 MiB buffer, so every step starts from HBM.

``workloads`` carries the other configurations the same way: 1 (2D 256x128, n = 32768),
2 (the 50-step min-volume run on 3D 128x64x64, n = 524288; the timed steps continue the
run) and 4 (volume + centre of mass, 3D 256x128x128, n = 4194304, four coupled rows).
Every workload states its error against the FP64 oracle per result (lambda relative,
x absolute, scaled row residual), computed by the oracle leg in worker processes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload 1..4]

N > 1 (under torchrun): each rank runs its own independent replica (weak scaling, no data
collective); the job value is the steps of all ranks over the slowest rank's time.
--impl reference times the FP64 CPU oracle (the paper's Alg. 1/2 projection) on the host
cores, on the same workload, metric and unit.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HEADLINE = 3
WORKLOADS = {
    1: "volume_2d_256x128 (n=32768, m=1)",
    2: "min_volume_3d_128x64x64 (n=524288, m=1, 50-step run)",
    3: "multimaterial_3d_192x96x96_x4 (n=7077888, m=4 independent)",
    4: "volume_com_3d_256x128x128 (n=4194304, m=4 coupled)",
}
KERNEL_SOURCES = ["paper_2511_13905_gb300/csrc/seg_kernels.cu", "paper_2511_13905_gb300/csrc/dev_common.cuh",
                  "paper_2511_13905_gb300/csrc/coupled_kernels.cu", "paper_2511_13905_gb300/csrc/step_common.cuh",
                  "paper_2511_13905_gb300/csrc/kernels.h"]
DTYPE = ("f32 bulk streams; double-float (FP32 pairs) step scalars, brackets, roots, reductions and the "
         "coupled m x m Newton solve; f64 only in the report")
TOL = 1e-6
L2_BYTES = 126.5e6   # GB300 L2 (about 126 MB usable of the 129 MB quoted)


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


def measured_traffic(key):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(str(key))
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


def compulsory_bytes(n, m_eff):
    """Read x, x_prev, g, g_prev, d_prev and A once, write d and x_{t+1} once: 4 (5 + m_eff) + 8 per element."""
    return n * (4 * (5 + m_eff) + 8)


def pass_bytes(n, m_eff):
    """One projection pass reads the trial point and the coefficients: 4 (1 + m_eff) per element."""
    return n * 4 * (1 + m_eff)


def roofline(n, m_eff, passes, step_s, bw_hbm, bw_l2, traffic, kernel):
    """Both roofline readings of one step (bytes per launch over the event-timed launch):
    streaming = the streaming-byte count at the passes actually run, against the HBM peak;
    split = (compulsory bytes at the HBM rate + passes x pass bytes at the L2 read rate when
    a pass fits L2, else at the HBM rate) / step time; compulsory = compulsory bytes alone."""
    alg = algorithmic_bytes(n, m_eff, passes)
    comp = compulsory_bytes(n, m_eff)
    pb = pass_bytes(n, m_eff)
    bw_pass = bw_l2 if (bw_l2 and pb <= L2_BYTES) else bw_hbm
    t_floor = comp / (bw_hbm * 1e9) + passes * pb / (bw_pass * 1e9)
    achieved = alg / step_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": bw_hbm, "unit": "GB/s", "frac": achieved / bw_hbm,
            "traffic": traffic, "kernel": kernel, "algorithmic_bytes_per_launch": alg,
            "frac_split": t_floor / step_s, "split_floor_us": 1e6 * t_floor,
            "pass_bw_gbs": bw_pass, "pass_bytes": pb, "compulsory_bytes": comp,
            "frac_compulsory": comp / step_s / 1e9 / bw_hbm}


def kernel_name(n, mode):
    if mode == "coupled":
        return "pgdto::coupled_kernel (grid engine, one CTA per SM, cooperative)"
    if n <= (1 << 17):
        return "pgdto::seg_cluster_kernel (cluster engine, one thread-block cluster)"
    return "pgdto::seg_kernel (grid engine, one CTA per SM, cooperative)"


def make_cfg(wl):
    from paper_2511_13905_gb300 import inputs
    return {1: inputs.config1, 2: inputs.config2, 3: inputs.config3, 4: inputs.config4}[wl]()


# --------------------------------------------------------------------------- probes

def run_probes(dev, stream):
    """L2 and HBM read rates of a plain streaming read (pgdto_probe_read), CUDA-event timed:
    a 48 MiB buffer read 200 times in place (L2-resident after the first read), and a
    4 GiB buffer read 5 times (HBM)."""
    import torch
    from paper_2511_13905_gb300 import binding
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 4 * sms
    out = torch.empty(blocks, device=dev)
    res = {}
    for name, nbytes, reps in (("l2_read_gbs", 48 << 20, 200), ("hbm_read_gbs", 4 << 30, 5)):
        buf = torch.ones(nbytes // 4, device=dev)
        for _ in range(3):
            if binding.probe_read(buf, out, blocks) != 0:
                raise RuntimeError("pgdto_probe_read failed")
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            binding.probe_read(buf, out, blocks)
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = nbytes * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
        del buf
    res["how"] = ("pgdto_probe_read: 128-bit streaming reads, %d blocks x 512 threads; 48 MiB x 200 reads in place "
                  "(L2), 4 GiB x 5 reads (HBM); CUDA events around the repeated launches" % blocks)
    return res


# --------------------------------------------------------------------------- device-timed workloads

def time_workload(wl, args, dev, stream, flush, probes, world=1, local_rank=0, e2e=False):
    """Warm-up and K timed pgdto_step launches of workload `wl`; returns the result dict
    and the device outputs of the last timed step (for the oracle errors)."""
    import numpy as np
    import torch

    from paper_2511_13905_gb300 import binding, inputs

    cfg = make_cfg(wl)
    n, m = cfg["n"], cfg["m"]
    m_eff = m if cfg["mode"] == "coupled" else 1

    def T(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    # a problem small enough for one thread-block cluster: the library's autotuner picks
    # the cluster's block share for one problem of this n (synthetic problems of its own,
    # timed before this workload's timing); the handle is created under its choice
    tuned = None
    if cfg["mode"] != "coupled" and n <= (1 << 17):
        st, share, share_ms = binding.autotune_batch(n, 1)
        if st != binding.PGDTO_OK:
            raise RuntimeError("pgdto_autotune_batch failed: %s" % st)
        tuned = {"cluster_elems": share, "median_ms_synthetic": share_ms, "candidates": [1024, 2048, 4096, 8192],
                 "how": "pgdto_autotune_batch(n, 1): 3 + 5 steps of a synthetic problem per candidate share, "
                        "lowest median kept"}
    h = binding.Handle(n, m, seg=cfg.get("seg"))
    if tuned is not None:
        binding.autotune_reset()
    x0 = T(cfg["x"])
    x = x0.clone()
    g = T(cfg["g"])
    G = cfg["G"]
    trajectory = wl == 2
    if trajectory:
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
            return A_fixed, list(cfg["gval"])

    def reset():
        x.copy_(x0)
        if cfg["t"] > 0:
            h.set_state(T(cfg["x_prev"]), T(cfg["g_prev"]), T(cfg["d_prev"]), cfg["t"])
        else:
            h.set_state(None, None, None, 0)

    reset()
    for _ in range(args.warmup):
        A, gval = sensitivities(x)
        st, info = h.step(x, g, A, gval, G)
        if st not in (0, binding.PGDTO_NOT_CONVERGED):
            raise RuntimeError("pgdto_step failed: %s" % binding.STATUS_NAMES.get(st, st))
        if not trajectory:
            reset()
    torch.cuda.synchronize()

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    torch.cuda.synchronize()
    launches0 = h.kernel_launches()
    evs, passes, newton = [], [], []
    info = None
    for k in range(args.steps):
        A, gval = sensitivities(x)
        flush.fill_(float(k))
        # a bounded spin (about 0.1 ms) keeps the device busy while the host enqueues the
        # step (tens of microseconds through the Python binding), so the events bracket
        # device work; the host path is what the end-to-end figure measures
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
        newton.append(info.newton_iters)
        if not trajectory and k < args.steps - 1:
            reset()
    torch.cuda.synchronize()
    launches = h.kernel_launches() - launches0
    clk = clocks.stop()
    times_ms = [a.elapsed_time(b) for a, b in evs]
    value, total_s = combine_ranks(sum(times_ms) / 1e3, args.steps, world, dev)
    out_x = x.cpu().numpy()
    out_lam = list(info.lambda_)[:m]

    step_s = total_s / args.steps
    avg_passes = sum(passes) / len(passes)
    bw, peak_kind = peaks()
    res = {
        "workload": cfg["name"], "n": n, "m": m, "mode": cfg["mode"],
        "steps_per_s": value, "ms_per_step": 1e3 * step_s,
        "ms_per_step_median": statistics.median(times_ms), "ms_per_step_min": min(times_ms),
        "avg_projection_passes": avg_passes, "newton_iters": sum(newton) / len(newton),
        "trajectory": ("steps t = 0..%d of the run from t = 0; timed t = %d..%d" %
                       (args.warmup + args.steps - 1, args.warmup, args.warmup + args.steps - 1)) if trajectory
        else "one step from the seeded state (t = %d), the state reset before each timed step" % cfg["t"],
        "roofline": roofline(n, m_eff, avg_passes, step_s, bw, probes.get("l2_read_gbs"),
                             measured_traffic(wl), kernel_name(n, cfg["mode"])),
        "gpu_launches": launches,
        "clocks": clk,
    }
    if tuned is not None:
        res["autotune"] = tuned
    res["roofline"]["peak_source"] = ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                                      else "fallback")

    if e2e:
        # end to end through the host-buffer entry point: pinned host x, grad f and A copied in,
        # rho_{t+1} copied out, inside the timing
        xh = torch.from_numpy(cfg["x"].copy()).pin_memory()
        gh = torch.from_numpy(cfg["g"].copy()).pin_memory()
        reset()
        e2e_times = []
        for k in range(args.warmup + args.steps):
            A, gval = sensitivities(xh.to(dev))
            Ah = A.cpu().pin_memory()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, info_h = h.step_host(xh, gh, Ah, gval, G)
            t1 = time.perf_counter()
            if st not in (0, binding.PGDTO_NOT_CONVERGED):
                raise RuntimeError("step_host failed: %s" % st)
            if k >= args.warmup:
                e2e_times.append(t1 - t0)
            if not trajectory:
                xh.copy_(torch.from_numpy(cfg["x"]))
                reset()
        e2e_value, _ = combine_ranks(sum(e2e_times), len(e2e_times), world, dev)
        a_bytes = 4 * int(np.asarray(cfg["A"]).size) if not trajectory else 4 * n
        res["e2e"] = {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": 8 * n + a_bytes,
                      "d2h_bytes_per_step": 4 * n, "api": "pgdto_step_host (pinned host buffers)"}

    # the GPU's steps from the oracle's own states for the trajectory workload (its timed
    # steps continue the device's run, whose states the oracle must not take as inputs)
    h.close()
    return res, {"x": out_x, "lam": out_lam}


def run_trajectory_from_states(states, dev):
    """Workload 2: one device step from each of the oracle's states (outside any timing)."""
    import numpy as np
    import torch

    from paper_2511_13905_gb300 import binding, inputs
    cfg = inputs.config2()
    n = cfg["n"]

    def T(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    h = binding.Handle(n, 1)
    g = T(cfg["g"])
    outs = []
    for s in states:
        x = T(s["x"])
        A, gval = inputs.config2_inputs(cfg, s["x"])
        if s["t"] > 0:
            h.set_state(T(s["x_prev"]), g, T(s["d_prev"]), s["t"])
        else:
            h.set_state(None, None, None, 0)
        st, info = h.step(x, g, T(A), gval, cfg["G"])
        if st not in (0, binding.PGDTO_NOT_CONVERGED):
            raise RuntimeError("workload 2 step t=%d failed: %s" % (s["t"], st))
        outs.append({"x": x.cpu().numpy(), "lam": [info.lambda_[0]]})
    h.close()
    return outs


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

    # the library's autotuner picks the cluster engine's block share for B problems of this
    # n (synthetic problems of its own, timed before and outside this workload's timing);
    # the handles below, batched and plain alike, are created under its choice
    st, tuned, tuned_ms = binding.autotune_batch(n, B)
    if st != binding.PGDTO_OK:
        raise RuntimeError("pgdto_autotune_batch failed: %s" % st)
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
    lam_b = [[i.lambda_[0]] for i in info_b]
    t_p, passes_p, launches_p, info_p = timed(plain, args.steps)
    diff = max(float(np.max(np.abs(a.astype(np.float64) - x.cpu().numpy()))) for a, x in zip(x_b, xs))
    bytes_b = sum(algorithmic_bytes(n, 1, i.passes) for i in info_b)
    peak, _ = peaks()
    for h in hs:
        h.close()
    binding.autotune_reset()
    res = {"workload": "%d x volume_2d_256x128 (n=%d, m=1, one step each)" % (B, n),
           "autotune": {"cluster_elems": tuned, "median_ms_synthetic": tuned_ms,
                        "candidates": [1024, 2048, 4096, 8192],
                        "how": "pgdto_autotune_batch(n, B): 3 + 5 batched steps of B synthetic problems per "
                               "candidate share, lowest median kept"},
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
    return res, {"x": x_b, "lam": lam_b}


# --------------------------------------------------------------------------- serving

def run_serving(args, local_rank=0):
    """The serving stream: `sessions` design sessions x `serve_steps` steps = 2048 requests by
    default, n log-uniform in [4096, n_max], m in {1, 2, 4} (half of the m > 1 sessions with
    independent rows, half coupled), inputs from each request's seed.  Requests arrive by a
    seeded Poisson process; request i is step i // sessions of session i % sessions (round
    robin), and a session's next step needs its previous result.

    Each step's constraint values g_j(x_t) = a_j^T x_t follow the session's own designs;
    they are recorded by an untimed dry run through plain handles (formed on the device)
    and replayed by both timed arms, so the clients do no arithmetic on the timed path.

    Plain: one worker takes the requests in arrival order, one launch each (H2D of grad f
    and A from the host arrays, pgdto_step, D2H of x_{t+1}).  Its capacity (steps/s with
    every request waiting from the start) sets the arrival rates: 0.5, 0.8 and 1.2 times it.
    Served: pgdto_submit at each arrival time, continuous batching in the server, latency
    from the arrival to the completion the server stamps.  Latency = completion - arrival,
    queueing included."""
    import numpy as np
    import torch

    from paper_2511_13905_gb300 import binding, inputs
    dev = torch.device("cuda", local_rank)
    S, K = args.serve_sessions, args.serve_steps
    reqs = inputs.serving_requests(count=S, n_max=args.serve_nmax)
    probs = [inputs.request_problem(r) for r in reqs]
    grads = [[np.ascontiguousarray((p["g"] * np.float32(1.0 + 0.05 * k)).astype(np.float32)) for k in range(2)]
             for p in probs]
    Ahost = [np.ascontiguousarray(p["A"]).ravel() for p in probs]
    order = [(i % S, i // S) for i in range(S * K)]

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]

    # ---- untimed dry run: each session's constraint values along its own trajectory
    gvals = [[None] * K for _ in range(S)]
    dry_final = []
    for s, p in enumerate(probs):
        n, m = p["n"], p["m"]
        h = binding.Handle(n, m, seg=p.get("seg"))
        h.set_state(None, None, None, 0)
        x = torch.from_numpy(p["x"].copy()).to(dev)
        A = torch.from_numpy(Ahost[s]).to(dev)
        for k in range(K):
            if p["mode"] == "independent":
                seg = p["seg"]
                gv = [float(x[seg[j]:seg[j + 1]].double().sum().item()) for j in range(m)]
            else:
                gv = (A.reshape(m, n).double() @ x.double()).tolist()
            gvals[s][k] = gv
            st, _ = h.step(x, torch.from_numpy(grads[s][k % 2]).to(dev), A, gv, p["G"], want_info=True)
            if st not in (binding.PGDTO_OK, binding.PGDTO_NOT_CONVERGED):
                raise RuntimeError("dry-run step failed: %s" % st)
        dry_final.append(x.cpu().numpy())
        h.close()
    torch.cuda.synchronize()

    # ---- plain arm: one worker, arrival order, one launch per request
    def run_plain(arrivals):
        handles = [binding.Handle(p["n"], p["m"], seg=p.get("seg")) for p in probs]
        for h in handles:
            h.set_state(None, None, None, 0)
        xd = [torch.from_numpy(p["x"].copy()).to(dev) for p in probs]
        gd = [torch.empty(p["n"], device=dev) for p in probs]
        Ad = [torch.empty(Ahost[s].size, device=dev) for s in range(S)]
        gh = [[torch.from_numpy(g) for g in gg] for gg in grads]
        Ah = [torch.from_numpy(a) for a in Ahost]
        outs = [np.empty(p["n"], np.float32) for p in probs]
        nc = 0
        lat = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        last = t0
        for i, (s, k) in enumerate(order):
            t_arr = t0 + arrivals[i]
            now = time.perf_counter()
            while now < t_arr:
                if t_arr - now > 2e-4:
                    time.sleep(t_arr - now - 1e-4)
                now = time.perf_counter()
            gd[s].copy_(gh[s][k % 2])
            Ad[s].copy_(Ah[s])
            st, _ = handles[s].step(xd[s], gd[s], Ad[s], gvals[s][k], probs[s]["G"], want_info=True)
            if st not in (binding.PGDTO_OK, binding.PGDTO_NOT_CONVERGED):
                raise RuntimeError("plain step failed: %s" % st)
            nc += int(st == binding.PGDTO_NOT_CONVERGED)
            torch.from_numpy(outs[s]).copy_(xd[s])
            last = time.perf_counter()
            lat.append(last - t_arr)
        for h in handles:
            h.close()
        return {"p50_ms": 1e3 * pct(lat, 0.5), "p99_ms": 1e3 * pct(lat, 0.99),
                "steps_per_s": len(lat) / (last - t0), "not_converged": nc, "launches": len(lat)}, outs

    # ---- served arm: submit at each arrival time, the server batches what is ready
    def run_served(arrivals):
        srv = binding.Server(budget_bytes=64 << 30, max_sessions=S + 1)
        outs = [np.empty(p["n"], np.float32) for p in probs]
        last_ticket = [None] * S
        done_t = {}
        arr_t = []
        tickets = []
        nc = 0

        def collect(ticket):
            nonlocal nc
            st, d, _, t_done = srv.wait(ticket)
            if st != binding.PGDTO_OK or d not in (binding.PGDTO_OK, binding.PGDTO_NOT_CONVERGED):
                raise RuntimeError("served step failed: %s / %s" % (st, d))
            nc += int(d == binding.PGDTO_NOT_CONVERGED)
            done_t[ticket] = t_done

        # sessions open before the timed stream, as the plain arm creates its handles
        for s, p in enumerate(probs):
            st = srv.open(s, p["n"], p["m"], p["x"], seg=p.get("seg"))
            if st != binding.PGDTO_OK:
                raise RuntimeError("session open failed: %s" % st)
        t0 = srv.clock_us()
        for i, (s, k) in enumerate(order):
            t_arr = t0 + int(1e6 * arrivals[i])
            now = srv.clock_us()
            while now < t_arr:
                if t_arr - now > 200:
                    time.sleep((t_arr - now - 100) * 1e-6)
                now = srv.clock_us()
            p = probs[s]
            while True:
                st, t = srv.submit(s, p["n"], p["m"], grads[s][k % 2], Ahost[s], gvals[s][k], p["G"], outs[s],
                                   seg=p.get("seg"))
                if st == binding.PGDTO_OK:
                    break
                if st != binding.PGDTO_ERR_BUSY or last_ticket[s] is None or last_ticket[s] in done_t:
                    raise RuntimeError("submit failed: %s" % st)
                collect(last_ticket[s])  # the session's previous step is still running
            last_ticket[s] = t
            tickets.append(t)
            arr_t.append(t_arr)
        for t in tickets:
            if t not in done_t:
                collect(t)
        stats = srv.stats()
        srv.close()
        lat = [(done_t[t] - a) * 1e-6 for t, a in zip(tickets, arr_t)]
        span = (max(done_t.values()) - t0) * 1e-6
        return {"p50_ms": 1e3 * pct(lat, 0.5), "p99_ms": 1e3 * pct(lat, 0.99), "steps_per_s": len(lat) / span,
                "not_converged": nc, "launches": stats["batches"]}, outs

    def diff(a, b):
        return max(float(np.max(np.abs(x.astype(np.float64) - y.astype(np.float64)))) for x, y in zip(a, b))

    rng = np.random.default_rng(inputs.SEED_BASE + 5000)
    unit = rng.exponential(1.0, S * K)  # one exponential draw per request, scaled by each rate
    # plain capacity: every request waiting from the start
    plain_sat, _ = run_plain(np.zeros(S * K))
    cap = plain_sat["steps_per_s"]
    rates = []
    for f in (0.5, 0.8, 1.2):
        lam = f * cap
        arrivals = np.cumsum(unit) / lam
        pl, out_p = run_plain(arrivals)
        sv, out_s = run_served(arrivals)
        rates.append({"rate_vs_plain_capacity": f, "offered_steps_per_s": lam, "plain": pl, "served": sv,
                      "max_abs_diff_final_x_served_vs_plain": diff(out_s, out_p),
                      "max_abs_diff_final_x_served_vs_dry_run": diff(out_s, dry_final)})
    torch.cuda.synchronize()
    return {"requests": S * K, "sessions": S, "steps_per_session": K,
            "n_range": [min(p["n"] for p in probs), max(p["n"] for p in probs)],
            "n_total": int(sum(p["n"] for p in probs)),
            "modes": {m: sum(1 for p in probs if p["mode"] == m) for m in ("single", "independent", "coupled")},
            "plain_capacity_steps_per_s": cap, "rates": rates,
            "arrivals": "Poisson (seeded exponential gaps), request i = step i // %d of session i %% %d; a session's "
                        "next step waits for its previous result" % (S, S),
            "latency": "arrival to rho_{t+1} in host memory (queueing included)"}


# --------------------------------------------------------------------------- oracle leg
#
# Everything below that calls the FP64 oracle runs in worker processes (spawned before the
# first CUDA call): the CPU baseline (the oracle timed on the host cores) and, on the same
# inputs, the oracle's results that the device results are compared with.  Inputs come
# from the seeded generators only; the device results travel to the workers, never the
# other way round.

def _oracle_cfg(wl, seed_offset=0):
    from paper_2511_13905_gb300 import inputs
    return {1: inputs.config1, 2: inputs.config2, 3: inputs.config3, 4: inputs.config4}[wl](seed_offset=seed_offset)


def _errors(cfg, ref, dev_x, dev_lam):
    import numpy as np
    from oracle.checks import parity_errors
    lam = np.asarray(dev_lam, dtype=np.float64)
    if cfg["mode"] == "independent":
        seg = [int(s) for s in cfg["seg"]]
        a = np.asarray(cfg["A"], dtype=np.float64)

        def matvec(xv):
            return (np.array([a[seg[j]:seg[j + 1]] @ xv[seg[j]:seg[j + 1]] for j in range(len(seg) - 1)]),
                    np.array([np.abs(a[seg[j]:seg[j + 1]]) @ np.abs(xv[seg[j]:seg[j + 1]])
                              for j in range(len(seg) - 1)]))
        amax = [float(np.max(np.abs(a[seg[j]:seg[j + 1]]))) for j in range(len(seg) - 1)]
        err = parity_errors(dev_x, lam, ref["x_new"], ref["lam"], matvec, ref["b"], 1e12, 0.0, 1.0, amax=amax)
    else:
        err = parity_errors(dev_x, lam, ref["x_new"], ref["lam"], cfg["A"], ref["b"], 1e12, 0.0, 1.0)
    return {k: err[k] for k in ("lam_rel", "x_abs", "viol_rel")}


def oracle_errors_seeded(wl, dev_x, dev_lam, seed_offset=0):
    """The oracle's step on the seeded state of workload wl, and the device result's error."""
    from oracle.step import oracle_step
    cfg = _oracle_cfg(wl, seed_offset)
    t0 = time.perf_counter()
    ref = oracle_step(cfg["x"], cfg["x_prev"], cfg["g"], cfg["g_prev"], cfg["d_prev"], cfg["A"], cfg["gval"],
                      cfg["G"], cfg["t"], mode=cfg["mode"], seg=cfg.get("seg"))
    err = _errors(cfg, ref, dev_x, dev_lam)
    err["oracle_s"] = time.perf_counter() - t0
    return err


def oracle_errors_batch(seed_offsets, dev_xs, dev_lams):
    worst = {"lam_rel": 0.0, "x_abs": 0.0, "viol_rel": 0.0}
    for so, xv, lv in zip(seed_offsets, dev_xs, dev_lams):
        e = oracle_errors_seeded(1, xv, lv, so)
        for k in worst:
            worst[k] = max(worst[k], e[k])
    return worst


def oracle_trajectory_states(steps):
    """The oracle's own workload-2 run, t = 0..steps-1, as float32 states a caller would hold."""
    import numpy as np
    from oracle.step import oracle_step
    from paper_2511_13905_gb300 import inputs
    cfg = inputs.config2()
    n = cfg["n"]
    x = cfg["x"].astype(np.float32)
    x_prev = np.zeros(n, np.float32)
    d_prev = np.zeros(n, np.float32)
    g_prev = np.zeros(n, np.float32)
    out = []
    for t in range(steps):
        A, gval = inputs.config2_inputs(cfg, x)
        out.append({"t": t, "x": x.copy(), "x_prev": x_prev.copy(), "d_prev": d_prev.copy()})
        ref = oracle_step(x, x_prev, cfg["g"], g_prev, d_prev, A, gval, cfg["G"], t, mode="single")
        x_prev, g_prev, d_prev = x.copy(), cfg["g"].copy(), ref["d"].astype(np.float32)
        x = ref["x_new"].astype(np.float32)
    return out


def oracle_errors_trajectory(states, dev_outs):
    """Workload 2: the oracle's step from each state against the device step from it."""
    from oracle.step import oracle_step
    from paper_2511_13905_gb300 import inputs
    import numpy as np
    cfg = inputs.config2()
    worst = {"lam_rel": 0.0, "x_abs": 0.0, "viol_rel": 0.0}
    for s, o in zip(states, dev_outs):
        A, gval = inputs.config2_inputs(cfg, s["x"])
        g_prev = cfg["g"] if s["t"] > 0 else np.zeros(cfg["n"], np.float32)
        ref = oracle_step(s["x"], s["x_prev"], cfg["g"], g_prev, s["d_prev"], A, gval, cfg["G"], s["t"],
                          mode="single")
        c = dict(cfg)
        c["A"] = A
        e = _errors(c, ref, o["x"], o["lam"])
        for k in worst:
            worst[k] = max(worst[k], e[k])
    return worst


def time_oracle_steps(wl, nsteps, budget_s):
    """Oracle steps ('paper' projector: Alg. 1 bisection / Alg. 2 as printed) on the workload;
    returns (steps, seconds).  Workload 2 continues its run; the others repeat the seeded step."""
    import numpy as np
    from oracle.step import oracle_step
    from paper_2511_13905_gb300 import inputs
    cfg = _oracle_cfg(wl)
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


def _one_thread_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _pool(procs):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(processes=procs, initializer=_one_thread_env)


def host_identity():
    model = platform.processor() or platform.machine()
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"cpu_count": os.cpu_count(), "model": model, "machine": platform.machine()}


def cpu_baseline(wl, budget_s):
    """The oracle on one host thread, then on every host core at once (one process per core,
    each running whole steps of the same workload); value = steps per second of the whole
    host.  Each process holds one copy of the workload, so the process count is also capped
    by host memory (3 GB per process)."""
    ident = host_identity()
    pool = _pool(1)
    try:
        done, spent = pool.apply(time_oracle_steps, (wl, 100000, budget_s))
    finally:
        pool.close()
        pool.join()
    single = done / spent
    procs = os.cpu_count() or 1
    try:
        mem = os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        procs = max(1, min(procs, int(mem // (3 << 30))))
    except (ValueError, OSError, AttributeError):
        pass
    pool = _pool(procs)
    try:
        t0 = time.perf_counter()
        res = pool.starmap(time_oracle_steps, [(wl, 100000, budget_s)] * procs)
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    total = sum(d for d, _ in res)
    longest = max(s for _, s in res)
    return {"value": total / longest, "unit": "steps/s", "cores": procs, "kind": "oracle",
            "sample": "%d full oracle steps of the same workload (FP64 NumPy; Alg. 1 bisection / Alg. 2 as "
                      "printed), %d processes x %.0f s of CPU time each on the host cores (wall %.1f s)"
                      % (total, procs, budget_s, wall),
            "single_thread": {"value": single, "unit": "steps/s", "cores": 1,
                              "sample": "%d oracle steps, %.1f s on one thread" % (done, spent)},
            "host": ident}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    _one_thread_env()
    wl = args.workload
    # warm-up steps untimed, then K timed steps, each a full oracle step on the whole workload
    time_oracle_steps(wl, args.warmup, 120.0)
    done, spent = time_oracle_steps(wl, args.steps, 240.0)
    v = done / spent
    ident = host_identity()
    return {
        "impl": "reference", "metric": "PGD-TO optimizer steps/s", "value": v, "unit": "steps/s",
        "n_gpus": 1, "steps": done, "warmup": args.warmup, "ms_per_step": 1e3 * spent / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[wl], "runs_on": "host CPU, 1 thread (%s)" % ident["model"]},
        "cpu_baseline": {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
                         "sample": "%d full oracle steps (FP64 NumPy, Alg. 1 / Alg. 2 as printed)" % done},
        "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def profile_steps(which, steps):
    """Untimed steps of one workload, the driver of the ncu captures under profiles/: workloads
    1, 3 and 4 step from the seeded state (reset before each step), workload 2 runs its
    trajectory from t = 0, and "batched" runs the 256-instance batched step."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_13905_gb300 import binding, inputs
    dev = torch.device("cuda", 0)

    def T(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    if which == "batched":
        cfgs = [inputs.config1(seed_offset=k) for k in range(256)]
        hs = [binding.Handle(c["n"], 1) for c in cfgs]
        x0 = [T(c["x"]) for c in cfgs]
        xs = [t.clone() for t in x0]
        gs, As = [T(c["g"]) for c in cfgs], [T(c["A"]) for c in cfgs]
        prev = [(T(c["x_prev"]), T(c["g_prev"]), T(c["d_prev"])) for c in cfgs]
        for _ in range(steps):
            for k, c in enumerate(cfgs):
                xs[k].copy_(x0[k])
                hs[k].set_state(prev[k][0], prev[k][1], prev[k][2], c["t"])
            st, _ = binding.step_many(hs, xs, gs, As, [c["gval"] for c in cfgs], [c["G"] for c in cfgs],
                                      want_info=False)
            if st != binding.PGDTO_OK:
                raise RuntimeError("pgdto_step_many failed: %s" % st)
        torch.cuda.synchronize()
        print("profile-step batched: %d batched steps of 256 instances" % steps)
        return
    wl = int(which)
    cfg = make_cfg(wl)
    n, m = cfg["n"], cfg["m"]
    h = binding.Handle(n, m, seg=cfg.get("seg"))
    x = T(cfg["x"])
    g = T(cfg["g"])
    if wl == 2:
        s_dev = T(cfg["s"]).double()
        for _ in range(steps):
            xd = x.double()
            A = (-3.0 * xd * xd * s_dev).float().reshape(1, n)
            gval = [float(torch.sum(s_dev * (1.0 - xd * xd * xd)).item())]
            h.step(x, g, A, gval, cfg["G"], want_info=False)
            if h.last_info()[0] not in (0, binding.PGDTO_NOT_CONVERGED):
                raise RuntimeError("step failed")
    else:
        x0 = x.clone()
        A = T(cfg["A"])
        prev = (T(cfg["x_prev"]), T(cfg["g_prev"]), T(cfg["d_prev"]))
        for _ in range(steps):
            x.copy_(x0)
            h.set_state(prev[0], prev[1], prev[2], cfg["t"])
            h.step(x, g, A, cfg["gval"], cfg["G"], want_info=False)
            if h.last_info()[0] not in (0, binding.PGDTO_NOT_CONVERGED):
                raise RuntimeError("step failed")
    torch.cuda.synchronize()
    h.close()
    print("profile-step %d: %d steps" % (wl, steps))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=HEADLINE, choices=[1, 2, 3, 4])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-workloads", action="store_true", help="headline workload only")
    ap.add_argument("--no-errors", action="store_true", help="skip the oracle errors")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--serve-sessions", type=int, default=128)
    ap.add_argument("--serve-steps", type=int, default=16)
    ap.add_argument("--serve-nmax", type=int, default=4 << 20)
    ap.add_argument("--profile-step", default=None, choices=["1", "2", "3", "4", "batched"],
                    help="run --steps untimed steps of one workload (for an ncu capture) and print no bench line")
    args = ap.parse_args()
    if args.profile_step is not None:
        profile_steps(args.profile_step, args.steps)
        return
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

    lead = rank == 0 and world == 1
    errors = lead and not args.no_errors
    pool = _pool(min(8, os.cpu_count() or 1)) if errors else None  # spawned before any CUDA call
    pending = {}
    traj_steps = args.warmup + args.steps
    others = [w for w in (1, 2, 4) if w != args.workload] if lead and not args.no_workloads else []
    if errors and (2 in others or args.workload == 2):
        pending["traj_states"] = pool.apply_async(oracle_trajectory_states, (traj_steps,))

    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    probes = run_probes(dev, stream) if lead else {}

    head, head_out = time_workload(args.workload, args, dev, stream, flush, probes, world, local_rank, e2e=True)
    if errors and args.workload != 2:
        pending["err_%d" % args.workload] = pool.apply_async(
            oracle_errors_seeded, (args.workload, head_out["x"], head_out["lam"]))
    subs = {}
    for wl in others:
        r, o = time_workload(wl, args, dev, stream, flush, probes)
        subs[wl] = r
        if errors and wl != 2:
            pending["err_%d" % wl] = pool.apply_async(oracle_errors_seeded, (wl, o["x"], o["lam"]))
    if errors and "traj_states" in pending:
        states = pending.pop("traj_states").get()
        outs = run_trajectory_from_states(states, dev)
        pending["err_2"] = pool.apply_async(oracle_errors_trajectory, (states, outs))
        del states, outs
    batched = None
    if lead and not args.no_batched:
        batched, bouts = run_batched(args, local_rank)
        if errors:
            k = len(bouts["x"])
            chunks = [list(range(i, k, 8)) for i in range(8)]
            pending["err_batched"] = [pool.apply_async(oracle_errors_batch, ([i for i in c],
                                                                             [bouts["x"][i] for i in c],
                                                                             [bouts["lam"][i] for i in c]))
                                      for c in chunks]
    # the oracle results; host-timed measurements (serving, the CPU baseline) run after
    # them so that the worker processes do not compete for the host
    err = {}
    for key, fut in pending.items():
        if isinstance(fut, list):
            parts = [f.get() for f in fut]
            err[key] = {k: max(p[k] for p in parts) for k in parts[0]}
        else:
            err[key] = fut.get()
    if pool is not None:
        pool.close()
        pool.join()

    def attach(res, wl):
        e = err.get("err_%d" % wl)
        if e is not None:
            e = dict(e)
            e["tolerance"] = TOL
            e["within_tolerance"] = all(e[k] <= TOL for k in ("lam_rel", "x_abs", "viol_rel"))
            e["against"] = ("the oracle's step from its own state at each t = 0..%d" % (traj_steps - 1)
                            if wl == 2 else "the oracle's step on the timed step's inputs")
            res["oracle_errors"] = e

    attach(head, args.workload)
    for wl, r in subs.items():
        attach(r, wl)
    if batched is not None and "err_batched" in err:
        batched["oracle_errors"] = dict(err["err_batched"], tolerance=TOL,
                                        against="each instance against the oracle's step on its seeded state")

    result = {
        "metric": "PGD-TO optimizer steps/s",
        "value": head["steps_per_s"],
        "unit": "steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPE,
        "data": "synthetic",
        "config": {"workload": head["workload"], "n": head["n"], "m": head["m"], "mode": head["mode"],
                   "trajectory": head["trajectory"],
                   "l2": "flushed between timed steps (256 MiB write)",
                   "timing": "CUDA events on the launching stream around each pgdto_step launch; a bounded "
                             "spin kernel ahead of the start event keeps the device busy while the host enqueues",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "avg_projection_passes": head["avg_projection_passes"],
                   "ms_per_step_median": head["ms_per_step_median"]},
        "roofline": head["roofline"],
        "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
    }
    if "oracle_errors" in head:
        result["oracle_errors"] = head["oracle_errors"]
    if probes:
        result["probes"] = probes
    if subs:
        result["workloads"] = {str(wl): r for wl, r in subs.items()}
    if batched is not None:
        result["batched"] = batched
    if lead and not args.no_serving:
        result["serving"] = run_serving(args, local_rank)
    if lead and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_budget)
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
