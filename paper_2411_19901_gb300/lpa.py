"""Thin ctypes binding of the C ABI in ``include/lpa.h`` (``liblpa.so``).

Argument marshalling only: every step of label propagation runs in the CUDA library.
Functions carry the C names; pointer arguments accept a CUDA ``torch.Tensor`` (device
pointers), a numpy array (host pointers, for ``lpa_detect_host``), a raw integer address,
or None.  Streams default to PyTorch's current stream.  A missing library raises: there
is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblpa.so")

LPA_EXACT, LPA_MG, LPA_BM = 0, 1, 2
MODES = {"exact": LPA_EXACT, "mg": LPA_MG, "bm": LPA_BM}
LPA_VALIDATE = 0x1
LPA_TIMING = 0x2
LPA_MODULARITY = 0x4
LPA_PRUNE = 0x8
LPA_MG_UNCLAMPED = 0x10
LPA_RESCAN = 0x20
LPA_GRAPH = 0x40
LPA_MAX_ITER = 1024

STATUS = {0: "LPA_OK", -1: "LPA_EINVAL", -2: "LPA_ENOMEM", -3: "LPA_ECUDA",
          -4: "LPA_ETIMEOUT", -5: "LPA_EUNSUPPORTED", -6: "LPA_EINTERNAL"}


class LpaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class lpa_stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("changed", ctypes.c_int64 * LPA_MAX_ITER),
        ("edges_scanned", ctypes.c_int64),
        ("seconds", ctypes.c_double),
        ("sweep_ms", ctypes.c_double),
        ("setup_ms", ctypes.c_double),
        ("sweep_launches", ctypes.c_int64),
        ("device_bytes", ctypes.c_size_t),
        ("chunks", ctypes.c_int32),
        ("hubs", ctypes.c_int32),
        ("modularity", ctypes.c_double),
        ("sweep_ms_iter", ctypes.c_float * LPA_MAX_ITER),
        ("scanned_iter", ctypes.c_int64 * LPA_MAX_ITER),
    ]

    def to_dict(self) -> dict:
        it = int(self.iterations)
        return {
            "iterations": it,
            "converged": bool(self.converged),
            "changed": [int(x) for x in self.changed[:it]],
            "edges_scanned": int(self.edges_scanned),
            "seconds": float(self.seconds),
            "sweep_ms": float(self.sweep_ms),
            "setup_ms": float(self.setup_ms),
            "sweep_launches": int(self.sweep_launches),
            "device_bytes": int(self.device_bytes),
            "chunks": int(self.chunks),
            "hubs": int(self.hubs),
            "modularity": float(self.modularity),
            "sweep_ms_iter": [float(x) for x in self.sweep_ms_iter[:it]],
            "scanned": [int(x) for x in self.scanned_iter[:it]],
        }


class lpa_graph(ctypes.Structure):
    _fields_ = [
        ("offsets", ctypes.c_void_p),
        ("indices", ctypes.c_void_p),
        ("weights", ctypes.c_void_p),
        ("n", ctypes.c_int32),
        ("m", ctypes.c_int64),
        ("labels_out", ctypes.c_void_p),
    ]


class lpa_graph_stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("edges_scanned", ctypes.c_int64),
        ("modularity", ctypes.c_double),
    ]


class lpa_tuning(ctypes.Structure):
    """Launch choices that never change a result (zero = default); see include/lpa.h."""
    _fields_ = [
        ("window", ctypes.c_int32),
        ("lane_threads", ctypes.c_int32),
        ("serial_hubs", ctypes.c_int32),
    ]

    def to_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}

    @classmethod
    def from_dict(cls, d: dict) -> "lpa_tuning":
        return cls(**{f: int(d.get(f, 0)) for f, _ in cls._fields_})


class lpa_options(ctypes.Structure):
    _fields_ = [
        ("pl_period", ctypes.c_int32),
        ("leaf_e0", ctypes.c_int32),
        ("leaf_max", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("labels_in", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("tuning", ctypes.POINTER(lpa_tuning)),
    ]


_lib = None

_P = ctypes.c_void_p
_SIG = {
    "lpa_options_init": (None, [ctypes.POINTER(lpa_options)]),
    "lpa_detect": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int,
                                  ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _P, _P]),
    "lpa_detect_ex": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _P, _P,
                                     _P]),
    "lpa_detect_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _P, _P,
                                       _P]),
    "lpa_modularity": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64, _P, _P]),
    "lpa_modularity_ex": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64, _P, _P,
                                         _P]),
    "lpa_workspace_size": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int,
                                             ctypes.c_int32]),
    "lpa_workspace_size_ex": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int,
                                                ctypes.c_int32, _P]),
    "lpa_modularity_workspace_size": (ctypes.c_size_t, [ctypes.c_int32]),
    "lpa_batch_detect": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int, ctypes.c_int32,
                                        ctypes.c_double, ctypes.c_int32, _P, _P, _P]),
    "lpa_server_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_int32, ctypes.c_size_t, _P, _P]),
    "lpa_server_submit": (ctypes.c_int, [_P, _P, _P]),
    "lpa_server_step": (ctypes.c_int, [_P, _P]),
    "lpa_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, _P, _P]),
    "lpa_server_drain": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P]),
    "lpa_release_memory": (ctypes.c_int, []),
    "lpa_server_destroy": (ctypes.c_int, [_P]),
    "lpa_plan_create": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_void_p)]),
    "lpa_plan_sweep": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P]),
    "lpa_plan_run": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int32, _P, _P]),
    "lpa_plan_destroy": (ctypes.c_int, [_P]),
    "lpa_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lpa_last_error": (ctypes.c_char_p, []),
    "lpa_version": (ctypes.c_char_p, []),
    "lpa_launch_count": (ctypes.c_uint64, []),
    "lpa_modularity_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64, _P,
                                              _P, _P]),
}

EXPORTED = tuple(_SIG)


def load(path: str = LIB_PATH):
    """Load ``liblpa.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA library first "
            "(python -m paper_2411_19901_gb300.build); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIG.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        msg = load().lpa_last_error().decode(errors="replace")
        raise LpaError(status, msg)


def _ptr(x):
    """Device or host address of x (tensor, numpy array, int, None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("numpy arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream_handle(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _mode(mode):
    return MODES[mode] if isinstance(mode, str) else int(mode)


def lpa_options_init() -> lpa_options:
    o = lpa_options()
    load().lpa_options_init(ctypes.byref(o))
    return o


def make_options(pl_period=8, leaf_e0=64, leaf_max=256, validate=True, timing=False,
                 modularity=False, labels_in=None, stream=None, workspace=None,
                 workspace_bytes=0, prune=False, unclamped=False, rescan=False,
                 tuning=None, graph=False) -> lpa_options:
    """Options for the calls below.  ``tuning``: an lpa_tuning or a dict of its fields (the
    struct is kept alive by the returned options)."""
    o = lpa_options_init()
    if tuning is not None:
        t = tuning if isinstance(tuning, lpa_tuning) else lpa_tuning.from_dict(tuning)
        o._tuning_ref = t
        o.tuning = ctypes.pointer(t)
    o.pl_period = pl_period
    o.leaf_e0 = leaf_e0
    o.leaf_max = leaf_max
    o.flags = ((LPA_VALIDATE if validate else 0) | (LPA_TIMING if timing else 0)
               | (LPA_MODULARITY if modularity else 0) | (LPA_PRUNE if prune else 0)
               | (LPA_MG_UNCLAMPED if unclamped else 0) | (LPA_RESCAN if rescan else 0)
               | (LPA_GRAPH if graph else 0))
    o.labels_in = _ptr(labels_in)
    o.stream = _stream_handle(stream)
    if workspace is not None:
        o.workspace = _ptr(workspace)
        o.workspace_bytes = workspace_bytes or (workspace.numel() * workspace.element_size())
    return o


def lpa_detect(offsets, indices, weights, n, m, mode, k, tol, max_iter, labels_out,
               stats: lpa_stats | None = None):
    _check(load().lpa_detect(_ptr(offsets), _ptr(indices), _ptr(weights), n, m, _mode(mode),
                             k, tol, max_iter, _ptr(labels_out),
                             ctypes.byref(stats) if stats is not None else None))


def lpa_detect_ex(offsets, indices, weights, n, m, mode, k, tol, max_iter, labels_out,
                  stats: lpa_stats | None = None, opt: lpa_options | None = None):
    _check(load().lpa_detect_ex(_ptr(offsets), _ptr(indices), _ptr(weights), n, m,
                                _mode(mode), k, tol, max_iter, _ptr(labels_out),
                                ctypes.byref(stats) if stats is not None else None,
                                ctypes.byref(opt) if opt is not None else None))


def lpa_detect_host(offsets, indices, weights, n, m, mode, k, tol, max_iter, labels_out,
                    stats: lpa_stats | None = None, opt: lpa_options | None = None):
    _check(load().lpa_detect_host(_ptr(offsets), _ptr(indices), _ptr(weights), n, m,
                                  _mode(mode), k, tol, max_iter, _ptr(labels_out),
                                  ctypes.byref(stats) if stats is not None else None,
                                  ctypes.byref(opt) if opt is not None else None))


def lpa_modularity(offsets, indices, weights, n, m, labels) -> float:
    q = ctypes.c_double()
    _check(load().lpa_modularity(_ptr(offsets), _ptr(indices), _ptr(weights), n, m,
                                 _ptr(labels), ctypes.byref(q)))
    return float(q.value)


def lpa_modularity_ex(offsets, indices, weights, n, m, labels,
                      opt: lpa_options | None = None) -> float:
    q = ctypes.c_double()
    _check(load().lpa_modularity_ex(_ptr(offsets), _ptr(indices), _ptr(weights), n, m,
                                    _ptr(labels), ctypes.byref(q),
                                    ctypes.byref(opt) if opt is not None else None))
    return float(q.value)


LPA_NOALLOC_MAX_N = 1 << 20


def lpa_modularity_noalloc(offsets, indices, weights, n, m, labels,
                           opt: lpa_options | None = None) -> float:
    """Modularity computed in the library's fixed device scratch (no device allocation;
    n <= LPA_NOALLOC_MAX_N; concurrent calls race, see include/lpa.h)."""
    q = ctypes.c_double()
    _check(load().lpa_modularity_noalloc(_ptr(offsets), _ptr(indices), _ptr(weights), n, m,
                                         _ptr(labels), ctypes.byref(q),
                                         ctypes.byref(opt) if opt is not None else None))
    return float(q.value)


def lpa_workspace_size(n, m, mode, k=8) -> int:
    return int(load().lpa_workspace_size(n, m, _mode(mode), k))


def lpa_workspace_size_ex(n, m, mode, k=8, opt=None) -> int:
    """Workspace bound for the given options (their leaf_e0 sets the lane table's size)."""
    return int(load().lpa_workspace_size_ex(n, m, _mode(mode), k,
                                            ctypes.byref(opt) if opt is not None else None))


def lpa_modularity_workspace_size(n) -> int:
    return int(load().lpa_modularity_workspace_size(n))


def lpa_plan_create(offsets, indices, weights, n, m, mode, k, opt: lpa_options | None = None):
    h = ctypes.c_void_p()
    _check(load().lpa_plan_create(_ptr(offsets), _ptr(indices), _ptr(weights), n, m,
                                  _mode(mode), k,
                                  ctypes.byref(opt) if opt is not None else None,
                                  ctypes.byref(h)))
    return h.value


def lpa_plan_sweep(plan, c_prev, c_next, pick_less, want_dn=True):
    dn = ctypes.c_int64()
    _check(load().lpa_plan_sweep(plan, _ptr(c_prev), _ptr(c_next), int(bool(pick_less)),
                                 ctypes.byref(dn) if want_dn else None))
    return int(dn.value) if want_dn else None


def lpa_plan_run(plan, tol, max_iter, labels_out, stats: lpa_stats | None = None):
    _check(load().lpa_plan_run(plan, tol, max_iter, _ptr(labels_out),
                               ctypes.byref(stats) if stats is not None else None))


def lpa_plan_destroy(plan):
    _check(load().lpa_plan_destroy(plan))


def lpa_version() -> str:
    return load().lpa_version().decode()


def lpa_launch_count() -> int:
    return int(load().lpa_launch_count())


# ----------------------------------------------------------- tensor conveniences


class Plan:
    """A binned graph on the device (``lpa_plan_*``); use as a context manager."""

    def __init__(self, offsets, indices, weights=None, mode="mg", k=8, **opts):
        self.n = int(offsets.numel() - 1)
        self.m = int(indices.numel())
        self._keep = (offsets, indices, weights, opts.get("labels_in"))
        self.opt = make_options(**opts)
        self.handle = lpa_plan_create(offsets, indices, weights, self.n, self.m, mode, k,
                                      self.opt)

    def sweep(self, c_prev, c_next, pick_less=False, want_dn=True):
        return lpa_plan_sweep(self.handle, c_prev, c_next, pick_less, want_dn)

    def run(self, labels_out, tol=0.05, max_iter=20) -> dict:
        st = lpa_stats()
        lpa_plan_run(self.handle, tol, max_iter, labels_out, st)
        return st.to_dict()

    def close(self):
        if self.handle:
            lpa_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lpa_batch_detect(graphs, mode="mg", k=8, tol=0.05, max_iter=20,
                     opt: lpa_options | None = None):
    """Batched form.  ``graphs``: sequence of (offsets, indices, weights|None, labels_out)
    device tensors.  Returns (list of per-graph stat dicts, changed array [count, max_iter])."""
    import numpy as np

    count = len(graphs)
    arr = (lpa_graph * max(count, 1))()
    for g, (off, idx, w, out) in enumerate(graphs):
        arr[g] = lpa_graph(_ptr(off), _ptr(idx), _ptr(w), int(off.numel() - 1),
                           int(idx.numel()), _ptr(out))
    stats = (lpa_graph_stats * max(count, 1))()
    changed = np.zeros((max(count, 1), max(max_iter, 1)), dtype=np.int64)
    _check(load().lpa_batch_detect(ctypes.cast(arr, ctypes.c_void_p), count, _mode(mode), k,
                                   tol, max_iter,
                                   ctypes.byref(opt) if opt is not None else None,
                                   ctypes.cast(stats, ctypes.c_void_p),
                                   changed.ctypes.data))
    out = [{"iterations": int(stats[g].iterations), "converged": bool(stats[g].converged),
            "edges_scanned": int(stats[g].edges_scanned),
            "modularity": float(stats[g].modularity)} for g in range(count)]
    return out, changed[:count, :max_iter]


def lpa_release_memory() -> None:
    """Return the unused device memory of the library's pools to the driver."""
    _check(load().lpa_release_memory())


class Server:
    """Served form (``lpa_server_*``): submit device graphs, step, poll."""

    def __init__(self, mode="mg", k=8, tol=0.05, max_iter=20, hbm_budget_bytes=0, **opts):
        self.opt = make_options(**opts)
        h = ctypes.c_void_p()
        _check(load().lpa_server_create(_mode(mode), k, tol, max_iter, hbm_budget_bytes,
                                        ctypes.byref(self.opt), ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, offsets, indices, weights, labels_out) -> int:
        g = lpa_graph(_ptr(offsets), _ptr(indices), _ptr(weights), int(offsets.numel() - 1),
                      int(indices.numel()), _ptr(labels_out))
        t = ctypes.c_uint64()
        _check(load().lpa_server_submit(self.handle, ctypes.byref(g), ctypes.byref(t)))
        self._keep[t.value] = (offsets, indices, weights, labels_out)
        return int(t.value)

    def step(self) -> int:
        pending = ctypes.c_int32()
        _check(load().lpa_server_step(self.handle, ctypes.byref(pending)))
        return int(pending.value)

    def drain(self, cap: int = 4096) -> list:
        """Tickets finished since the last drain."""
        buf = (ctypes.c_uint64 * max(cap, 1))()
        cnt = ctypes.c_int32()
        _check(load().lpa_server_drain(self.handle, ctypes.cast(buf, ctypes.c_void_p), cap,
                                       ctypes.byref(cnt)))
        return [int(buf[i]) for i in range(cnt.value)]

    def poll(self, ticket: int):
        """None while running, else the request's stat dict (the ticket is then forgotten)."""
        done = ctypes.c_int32()
        st = lpa_graph_stats()
        _check(load().lpa_server_poll(self.handle, ticket, ctypes.byref(done), ctypes.byref(st)))
        if not done.value:
            return None
        self._keep.pop(ticket, None)
        return {"iterations": int(st.iterations), "converged": bool(st.converged),
                "edges_scanned": int(st.edges_scanned)}

    def close(self):
        if self.handle:
            load().lpa_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def detect(offsets, indices, weights=None, mode="mg", k=8, tol=0.05, max_iter=20,
           labels_out=None, **opts):
    """Run LPA on device tensors; returns (labels tensor, stats dict)."""
    import torch

    n = int(offsets.numel() - 1)
    if labels_out is None:
        labels_out = torch.empty(n, dtype=torch.int32, device=offsets.device)
    st = lpa_stats()
    lpa_detect_ex(offsets, indices, weights, n, int(indices.numel()), mode, k, tol, max_iter,
                  labels_out, st, make_options(**opts))
    return labels_out, st.to_dict()


def modularity(offsets, indices, weights, labels, **opts) -> float:
    """Modularity (Eq. 1) of device labels."""
    n = int(offsets.numel() - 1)
    return lpa_modularity_ex(offsets, indices, weights, n, int(indices.numel()), labels,
                             make_options(**opts))
