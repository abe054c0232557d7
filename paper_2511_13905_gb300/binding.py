"""ctypes binding of libpgdto.so (include/pgdto.h), same names as the C ABI.

Argument marshalling only: tensors are passed as raw device (or host) pointers, the
CUDA stream as torch's current stream handle, and every computation runs in the
library's kernels.  There is no CPU path: if the library is missing, ``load`` raises.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpgdto.so")

PGDTO_OK = 0
PGDTO_ERR_ARG = 1
PGDTO_ERR_OOM = 2
PGDTO_ERR_CUDA = 3
PGDTO_ERR_NONFINITE = 4
PGDTO_ERR_TIMEOUT = 5
PGDTO_ERR_BUSY = 6
PGDTO_NOT_CONVERGED = 7
PGDTO_ERR_UNSUPPORTED = 8
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NONFINITE", 5: "ERR_TIMEOUT",
                6: "ERR_BUSY", 7: "NOT_CONVERGED", 8: "ERR_UNSUPPORTED"}

MODES = {"auto": 0, "single": 1, "independent": 2, "coupled": 3}


class Params(ctypes.Structure):
    _fields_ = [("C", ctypes.c_double), ("alpha_max", ctypes.c_double), ("alpha_fallback", ctypes.c_double),
                ("tol_B", ctypes.c_double), ("tol_N", ctypes.c_double), ("omega", ctypes.c_double),
                ("eps_alpha", ctypes.c_double), ("c1", ctypes.c_double), ("c2", ctypes.c_double),
                ("tol_lambda", ctypes.c_double), ("t_warmup", ctypes.c_int), ("maxiter_newton", ctypes.c_int),
                ("max_passes", ctypes.c_int), ("barrier_timeout_ms", ctypes.c_int), ("mode", ctypes.c_int),
                ("fault_inject", ctypes.c_int), ("engine", ctypes.c_int), ("cluster_elems", ctypes.c_int),
                ("eq_mask", ctypes.c_int), ("compaction", ctypes.c_int), ("stage1", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("lambda_", ctypes.c_double * 4),
                ("b", ctypes.c_double * 4), ("viol", ctypes.c_double * 4), ("rel_change", ctypes.c_double),
                ("phi_inf", ctypes.c_double), ("passes", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("stage", ctypes.c_int), ("branch", ctypes.c_int), ("status", ctypes.c_int), ("t", ctypes.c_int),
                ("visited", ctypes.c_double)]

    def as_dict(self, m=4):
        return {"alpha": self.alpha, "beta": self.beta, "lambda": list(self.lambda_)[:m], "b": list(self.b)[:m],
                "viol": list(self.viol)[:m], "rel_change": self.rel_change, "phi_inf": self.phi_inf,
                "passes": self.passes, "newton_iters": self.newton_iters, "stage": self.stage,
                "branch": self.branch, "status": self.status, "t": self.t, "visited": self.visited}


class Request(ctypes.Structure):
    _fields_ = [("session", ctypes.c_uint64), ("n", ctypes.c_int64), ("m", ctypes.c_int),
                ("seg_offsets", ctypes.POINTER(ctypes.c_int64)), ("lo", ctypes.c_float), ("hi", ctypes.c_float),
                ("x0", ctypes.c_void_p), ("grad_f", ctypes.c_void_p), ("A", ctypes.c_void_p),
                ("g_val", ctypes.c_double * 4), ("G", ctypes.c_double * 4), ("x_out", ctypes.c_void_p),
                ("close_session", ctypes.c_int), ("eq_mask", ctypes.c_int)]


class PgdtoError(RuntimeError):
    def __init__(self, status, where):
        super().__init__("%s returned %s" % (where, STATUS_NAMES.get(status, status)))
        self.status = status


_lib = None
P = ctypes.c_void_p
D = ctypes.POINTER(ctypes.c_double)


def load(path=None):
    """Load libpgdto.so once; raise if it is absent (build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libpgdto.so not found at %s: build it first (python -c 'import __graft_entry__ "
                           "as g; g.build()'); there is no fallback" % path)
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    sig = {
        "pgdto_params_default": (ctypes.c_int, [ctypes.POINTER(Params)]),
        "pgdto_create": (ctypes.c_int, [ctypes.POINTER(H), ctypes.c_int64, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int64), ctypes.c_float, ctypes.c_float,
                                        ctypes.POINTER(Params), P]),
        "pgdto_destroy": (None, [H]),
        "pgdto_set_stream": (ctypes.c_int, [H, P]),
        "pgdto_set_state": (ctypes.c_int, [H, P, P, P, ctypes.c_int]),
        "pgdto_get_state": (ctypes.c_int, [H, P, P, P, ctypes.POINTER(ctypes.c_int)]),
        "pgdto_step": (ctypes.c_int, [H, P, P, P, D, D, ctypes.POINTER(Info)]),
        "pgdto_step_host": (ctypes.c_int, [H, P, P, P, D, D, ctypes.POINTER(Info)]),
        "pgdto_project": (ctypes.c_int, [H, P, P, D, P, D, ctypes.POINTER(Info)]),
        "pgdto_last_info": (ctypes.c_int, [H, ctypes.POINTER(Info), D]),
        "pgdto_kernel_launches": (ctypes.c_int64, [H]),
        "pgdto_trace": (ctypes.c_int, [H, D, ctypes.c_int]),
        "pgdto_step_many": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(H), ctypes.POINTER(P), ctypes.POINTER(P),
                                           ctypes.POINTER(P), D, D, ctypes.POINTER(Info)]),
        "pgdto_project_many": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(H), ctypes.POINTER(P), ctypes.POINTER(P),
                                              D, ctypes.POINTER(P), D, ctypes.POINTER(Info)]),
        "pgdto_project_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                                 ctypes.c_float, ctypes.c_float, ctypes.c_double, P, P, D, P, D,
                                                 ctypes.POINTER(Info), P]),
        "pgdto_noalloc_set_test_fault": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
        "pgdto_probe_read": (ctypes.c_int, [P, ctypes.c_int64, P, ctypes.c_int, P]),
        "pgdto_autotune_batch": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                ctypes.POINTER(ctypes.c_double), P]),
        "pgdto_autotune_reset": (None, []),
        "pgdto_version": (ctypes.c_char_p, []),
        "pgdto_server_create": (ctypes.c_int, [ctypes.POINTER(H), ctypes.c_uint64, ctypes.c_int,
                                               ctypes.POINTER(Params), P]),
        "pgdto_submit": (ctypes.c_int, [H, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
        "pgdto_server_open": (ctypes.c_int, [H, ctypes.POINTER(Request)]),
        "pgdto_poll": (ctypes.c_int, [H, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Info)]),
        "pgdto_wait": (ctypes.c_int, [H, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Info),
                                      ctypes.POINTER(ctypes.c_int64)]),
        "pgdto_server_clock_us": (ctypes.c_int64, [H]),
        "pgdto_server_stats": (ctypes.c_int, [H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint64)]),
        "pgdto_server_destroy": (None, [H]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols():
    """Function names declared in include/pgdto.h (parsed from the header text)."""
    import re
    hdr = os.path.join(os.path.dirname(HERE), "include", "pgdto.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(pgdto_[a-z_0-9]+)\s*\(", text)))


def params_default(**overrides):
    p = Params()
    load().pgdto_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "mode" and isinstance(v, str):
            v = MODES[v]
        setattr(p, k, v)
    return p


def _dptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _darr(vals, m):
    arr = (ctypes.c_double * max(m, 1))()
    for j, v in enumerate(list(vals)[:m]):
        arr[j] = float(v)
    return arr


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Handle:
    """Owns a pgdto_handle (optimizer state + device workspace) for fixed n, m, mode."""

    def __init__(self, n, m, seg=None, lo=0.0, hi=1.0, params=None, stream=None, **param_overrides):
        self.lib = load()
        self.n, self.m = int(n), int(m)
        p = params if params is not None else params_default(**param_overrides)
        segarr = None
        if seg is not None:
            segarr = (ctypes.c_int64 * (self.m + 1))(*[int(s) for s in seg])
        h = ctypes.c_void_p()
        st = self.lib.pgdto_create(ctypes.byref(h), self.n, self.m, segarr, float(lo), float(hi),
                                   ctypes.byref(p), _stream_ptr(stream))
        if st != PGDTO_OK:
            raise PgdtoError(st, "pgdto_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.pgdto_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        return self.lib.pgdto_set_stream(self.h, _stream_ptr(stream))

    def set_state(self, x_prev=None, g_prev=None, d_prev=None, t=0):
        st = self.lib.pgdto_set_state(self.h, _dptr(x_prev), _dptr(g_prev), _dptr(d_prev), int(t))
        if st != PGDTO_OK:
            raise PgdtoError(st, "pgdto_set_state")

    def get_state(self, x_prev=None, g_prev=None, d_prev=None):
        t = ctypes.c_int()
        st = self.lib.pgdto_get_state(self.h, _dptr(x_prev), _dptr(g_prev), _dptr(d_prev), ctypes.byref(t))
        if st != PGDTO_OK:
            raise PgdtoError(st, "pgdto_get_state")
        return t.value

    def step(self, x, grad_f, A, g_val, G, want_info=True):
        """One optimizer step on device tensors; returns (status, Info or None)."""
        info = Info() if want_info else None
        st = self.lib.pgdto_step(self.h, _dptr(x), _dptr(grad_f), _dptr(A), _darr(g_val, self.m),
                                 _darr(G, self.m), ctypes.byref(info) if info is not None else None)
        return st, info

    def step_host(self, x, grad_f, A, g_val, G):
        """The step on host (CPU, ideally pinned) tensors; x is updated in place."""
        info = Info()
        st = self.lib.pgdto_step_host(self.h, _dptr(x), _dptr(grad_f), _dptr(A), _darr(g_val, self.m),
                                      _darr(G, self.m), ctypes.byref(info))
        return st, info

    def project(self, z, A, b, x_out, want_info=True):
        """Projection alone; returns (status, lambda list or None, Info or None)."""
        info = Info() if want_info else None
        lam = (ctypes.c_double * self.m)() if want_info else None
        st = self.lib.pgdto_project(self.h, _dptr(z), _dptr(A), _darr(b, self.m), _dptr(x_out), lam,
                                    ctypes.byref(info) if info is not None else None)
        return st, (list(lam) if lam is not None else None), info

    def last_info(self):
        info = Info()
        lam = (ctypes.c_double * self.m)()
        st = self.lib.pgdto_last_info(self.h, ctypes.byref(info), lam)
        return st, list(lam), info

    def trace(self, max_marks=62):
        """Phase timeline of the last call: microseconds since kernel start, one per grid reduction."""
        buf = (ctypes.c_double * max_marks)()
        k = self.lib.pgdto_trace(self.h, buf, max_marks)
        return list(buf)[:max(k, 0)]

    def kernel_launches(self):
        return int(self.lib.pgdto_kernel_launches(self.h))


def project_noalloc(z, A, b, x_out, m=1, seg=None, lo=0.0, hi=1.0, C=1e12, stream=None, want_info=True):
    """pgdto_project_noalloc: the projection without any device allocation (no handle).
    Returns (status, lambda list or None, Info or None)."""
    lib = load()
    n = int(z.numel())
    segarr = (ctypes.c_int64 * (m + 1))(*[int(s) for s in seg]) if seg is not None else None
    info = Info() if want_info else None
    lam = (ctypes.c_double * m)() if want_info else None
    st = lib.pgdto_project_noalloc(n, int(m), segarr, float(lo), float(hi), float(C), _dptr(z), _dptr(A),
                                   _darr(b, m), _dptr(x_out), lam, ctypes.byref(info) if info is not None else None,
                                   _stream_ptr(stream))
    return st, (list(lam) if lam is not None else None), info


def noalloc_set_test_fault(fault_inject, timeout_ms):
    """pgdto_noalloc_set_test_fault (tests only)."""
    return load().pgdto_noalloc_set_test_fault(int(fault_inject), int(timeout_ms))


def probe_read(buf, out, blocks, stream=None):
    """pgdto_probe_read: one streaming read of the device tensor buf (measurement tooling)."""
    return load().pgdto_probe_read(_dptr(buf), int(buf.numel()), _dptr(out), int(blocks), _stream_ptr(stream))


def autotune_batch(n, count, stream=None):
    """pgdto_autotune_batch: (status, chosen cluster_elems, its median batched-step ms)."""
    best = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    st = load().pgdto_autotune_batch(int(n), int(count), ctypes.byref(best), ctypes.byref(ms), _stream_ptr(stream))
    return st, best.value, ms.value


def autotune_reset():
    """pgdto_autotune_reset: forget the recorded shares on every device."""
    load().pgdto_autotune_reset()


def _ptrs(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr()
    return arr


def _rows4(vals_per_item):
    arr = (ctypes.c_double * (4 * len(vals_per_item)))()
    for k, vals in enumerate(vals_per_item):
        for j, v in enumerate(list(vals)[:4]):
            arr[4 * k + j] = float(v)
    return arr


def step_many(handles, xs, grads, As, g_vals, Gs, want_info=True):
    """pgdto_step_many: one launch, one step per handle.  Returns (status, [Info] or None)."""
    lib = load()
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.h for h in handles])
    infos = (Info * n)() if want_info else None
    st = lib.pgdto_step_many(n, hs, _ptrs(xs), _ptrs(grads), _ptrs(As), _rows4(g_vals), _rows4(Gs), infos)
    return st, (list(infos) if infos is not None else None)


def project_many(handles, zs, As, bs, x_outs, want_info=True):
    """pgdto_project_many: one launch, one projection per handle.  Returns (status, lambdas, infos)."""
    lib = load()
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.h for h in handles])
    infos = (Info * n)() if want_info else None
    lam = (ctypes.c_double * (4 * n))() if want_info else None
    st = lib.pgdto_project_many(n, hs, _ptrs(zs), _ptrs(As), _rows4(bs), _ptrs(x_outs), lam, infos)
    lams = [[lam[4 * k + j] for j in range(handles[k].m)] for k in range(n)] if want_info else None
    return st, lams, (list(infos) if infos is not None else None)


class Server:
    """pgdto_server: continuous batching of optimizer steps over device-resident design sessions.

    Host arrays are NumPy float32 (C-contiguous); the server copies grad_f and A during
    submit, and writes rho_{t+1} into the x_out array when the step completes (keep it
    alive until then)."""

    def __init__(self, budget_bytes, max_sessions=1024, params=None, stream=None, **param_overrides):
        self.lib = load()
        p = params if params is not None else params_default(**param_overrides)
        h = ctypes.c_void_p()
        st = self.lib.pgdto_server_create(ctypes.byref(h), int(budget_bytes), int(max_sessions), ctypes.byref(p),
                                          _stream_ptr(stream))
        if st != PGDTO_OK:
            raise PgdtoError(st, "pgdto_server_create")
        self.h = h
        self._keep = {}

    def submit(self, session, n, m, grad_f, A, g_val, G, x_out, x0=None, seg=None, lo=0.0, hi=1.0, close=False,
               eq_mask=0):
        r = Request()
        r.eq_mask = int(eq_mask)
        r.session, r.n, r.m, r.lo, r.hi = int(session), int(n), int(m), float(lo), float(hi)
        segarr = None
        if seg is not None:
            segarr = (ctypes.c_int64 * (m + 1))(*[int(v) for v in seg])
            r.seg_offsets = segarr
        r.x0 = x0.ctypes.data if x0 is not None else None
        r.grad_f = grad_f.ctypes.data
        r.A = A.ctypes.data
        for j in range(m):
            r.g_val[j] = float(g_val[j])
            r.G[j] = float(G[j])
        r.x_out = x_out.ctypes.data
        r.close_session = 1 if close else 0
        t = ctypes.c_uint64()
        st = self.lib.pgdto_submit(self.h, ctypes.byref(r), ctypes.byref(t))
        if st == PGDTO_OK:
            self._keep[t.value] = x_out
        return st, t.value

    def open(self, session, n, m, x0, seg=None, lo=0.0, hi=1.0, eq_mask=0):
        """pgdto_server_open: admit a session and upload its starting design (no step)."""
        r = Request()
        r.eq_mask = int(eq_mask)
        r.session, r.n, r.m, r.lo, r.hi = int(session), int(n), int(m), float(lo), float(hi)
        segarr = None
        if seg is not None:
            segarr = (ctypes.c_int64 * (m + 1))(*[int(v) for v in seg])
            r.seg_offsets = segarr
        r.x0 = x0.ctypes.data
        return self.lib.pgdto_server_open(self.h, ctypes.byref(r))

    def poll(self, ticket):
        """(call status, done status or PGDTO_ERR_BUSY, Info)."""
        d = ctypes.c_int()
        info = Info()
        st = self.lib.pgdto_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(d), ctypes.byref(info))
        if st == PGDTO_OK and d.value != PGDTO_ERR_BUSY:
            self._keep.pop(ticket, None)
        return st, d.value, info

    def wait(self, ticket, timeout_ms=60000):
        """Blocking poll: (call status, done status or PGDTO_ERR_BUSY, Info, completion time
        in microseconds on the server's clock)."""
        d = ctypes.c_int()
        info = Info()
        t = ctypes.c_int64()
        st = self.lib.pgdto_wait(self.h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(d), ctypes.byref(info),
                                 ctypes.byref(t))
        if st == PGDTO_OK and d.value != PGDTO_ERR_BUSY:
            self._keep.pop(ticket, None)
        return st, d.value, info, t.value

    def clock_us(self):
        """Microseconds since the server was created (the clock of wait's completion times)."""
        return int(self.lib.pgdto_server_clock_us(self.h))

    def stats(self):
        b, s_, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        u = ctypes.c_uint64()
        self.lib.pgdto_server_stats(self.h, ctypes.byref(b), ctypes.byref(s_), ctypes.byref(n), ctypes.byref(u))
        return {"batches": b.value, "steps": s_.value, "sessions": n.value, "bytes_in_use": u.value}

    def close(self):
        if getattr(self, "h", None):
            self.lib.pgdto_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
