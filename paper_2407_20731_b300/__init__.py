"""paper_2407_20731_b300 -- in-situ reduction of spectral-element field
snapshots on one B300 GPU.

This module is the thin Python binding of ``libsemr.so``, the C ABI declared
in ``include/semr.h``: the same entry-point names, argument marshalling only.
Every step of the reduction runs in the library's CUDA kernels; PyTorch is
used only to hold device memory and to name CUDA streams.  There is no CPU
fallback: importing this module raises if the library has not been built.

The method is the GPU lossy compression of SEM fields in arXiv 2407.20731,
Sec. IV-B (spectral transform, energy-relative truncation, quantisation),
with the error check the paper calls "sufficient accuracy" and the
compression ratio of Eq. 1.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SEMR_BOUNDS=1 in the environment loads the checking build libsemr_bounds.so
# (compiled with -DSEMR_BOUNDS; the same ABI)
BOUNDS_BUILD = os.environ.get("SEMR_BOUNDS", "") == "1"
LIB_PATH = os.path.join(_HERE, "libsemr_bounds.so" if BOUNDS_BUILD else "libsemr.so")

# status codes (include/semr.h)
SEMR_OK, SEMR_EINVAL, SEMR_ENOMEM, SEMR_EBUDGET, SEMR_EAGAIN = 0, 1, 2, 3, 4
SEMR_ETIMEDOUT, SEMR_ECUDA, SEMR_ENOSPACE, SEMR_ENONFINITE, SEMR_EUNSUPPORTED = 5, 6, 7, 8, 9
SEMR_MAX_FIELDS, SEMR_LX_MIN, SEMR_LX_MAX = 16, 2, 12
SEMR_FP64, SEMR_FP32, SEMR_FP64_NATIVE = 0, 1, 2
SEMR_WRITE_RECON, SEMR_CUMULATIVE = 1, 2
SEMR_PAYLOAD_LOSSLESS, SEMR_PAYLOAD_CODE32, SEMR_PAYLOAD_FP32, SEMR_PAYLOAD_CUMULATIVE = 1, 2, 4, 8
SEMR_STATUS_OVERFLOW, SEMR_STATUS_TIMEOUT, SEMR_STATUS_NONFINITE, SEMR_STATUS_TINY = 1, 2, 4, 8
SEMR_STATUS_STAGE, SEMR_STATUS_BOUNDS = 16, 32
SEMR_BUILD_BOUNDS = 1


class semr_mesh(ctypes.Structure):
    _fields_ = [("lx", ctypes.c_int32), ("pad_", ctypes.c_int32), ("n_elem", ctypes.c_int64),
                ("jac", ctypes.c_void_p)]


class semr_fieldset(ctypes.Structure):
    _fields_ = [("n_fields", ctypes.c_int32), ("precision", ctypes.c_int32), ("tau", ctypes.c_double),
                ("flags", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("fields", ctypes.c_void_p * SEMR_MAX_FIELDS), ("recon", ctypes.c_void_p * SEMR_MAX_FIELDS)]


class semr_field_report(ctypes.Structure):
    _fields_ = [("l2_abs", ctypes.c_double), ("l2_rel", ctypes.c_double), ("linf_abs", ctypes.c_double),
                ("linf_rel", ctypes.c_double), ("sum_err2", ctypes.c_double), ("sum_energy", ctypes.c_double),
                ("umax", ctypes.c_double), ("kept", ctypes.c_uint64), ("bytes", ctypes.c_uint64),
                ("cr", ctypes.c_double)]


class semr_summary(ctypes.Structure):
    _fields_ = [("payload_bytes", ctypes.c_uint64), ("code_total", ctypes.c_uint64), ("status", ctypes.c_uint32),
                ("n_fields", ctypes.c_uint32), ("cr", ctypes.c_double), ("recomputed", ctypes.c_uint64),
                ("field", semr_field_report * SEMR_MAX_FIELDS)]


class semr_sizes(ctypes.Structure):
    _fields_ = [("header_bytes", ctypes.c_uint64), ("code_base", ctypes.c_uint64),
                ("payload_worst", ctypes.c_uint64), ("scratch_bytes", ctypes.c_uint64),
                ("elem_report_bytes", ctypes.c_uint64), ("code_width", ctypes.c_uint32),
                ("tiles", ctypes.c_uint32), ("scratch_min_bytes", ctypes.c_uint64)]


class semr_outputs(ctypes.Structure):
    _fields_ = [("payload", ctypes.c_void_p), ("payload_cap", ctypes.c_uint64), ("elem_report", ctypes.c_void_p),
                ("summary", ctypes.c_void_p), ("scratch", ctypes.c_void_p), ("scratch_bytes", ctypes.c_uint64)]


class semr_batch_item(ctypes.Structure):
    _fields_ = [("fs", semr_fieldset), ("mesh", semr_mesh), ("out", semr_outputs)]


SEMR_BATCH_AUTOTUNE = 1


class semr_request_info(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("slot", ctypes.c_int32), ("status", ctypes.c_int32), ("device_bytes", ctypes.c_uint64),
                ("summary", semr_summary)]

class semr_lattice(ctypes.Structure):
    _fields_ = [("lx", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("origin", ctypes.c_double * 3), ("h", ctypes.c_double * 3)]


SEMR_SLICE_MAX_CTRL, SEMR_SLICE_MAX_COMP, SEMR_SLICE_MAX_SIDE = 16, 3, 16384


class semr_slice(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("axis_u", ctypes.c_double * 3), ("axis_v", ctypes.c_double * 3),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("n_comp", ctypes.c_int32),
                ("n_ctrl", ctypes.c_int32), ("vmin", ctypes.c_double), ("vmax", ctypes.c_double),
                ("ctrl", (ctypes.c_double * 4) * SEMR_SLICE_MAX_CTRL), ("background", ctypes.c_uint32),
                ("pad_", ctypes.c_int32)]


# (name, restype, argtypes) of every exported entry point
_P = ctypes.c_void_p
EXPORTS = [
    ("semr_sizes_for", ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                      ctypes.POINTER(semr_sizes)]),
    ("semr_reduce_async", ctypes.c_int, [ctypes.POINTER(semr_fieldset), ctypes.POINTER(semr_mesh),
                                         ctypes.POINTER(semr_outputs), _P]),
    ("semr_reduce_async_timed", ctypes.c_int, [ctypes.POINTER(semr_fieldset), ctypes.POINTER(semr_mesh),
                                               ctypes.POINTER(semr_outputs), _P, _P, _P]),
    ("semr_open", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.c_uint64]),
    ("semr_submit", ctypes.c_int, [_P, ctypes.POINTER(semr_fieldset), ctypes.POINTER(semr_mesh),
                                   ctypes.POINTER(ctypes.c_uint64)]),
    ("semr_query", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("semr_fetch", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int, _P, ctypes.c_uint64,
                                  ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(semr_field_report), _P]),
    ("semr_close", None, [_P]),
    ("semr_decode", ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
    ("semr_gll", ctypes.c_int, [ctypes.c_int32, _P, _P]),
    ("semr_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("semr_batch_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(semr_batch_item), ctypes.c_int,
                                         ctypes.c_int, _P]),
    ("semr_batch_launch", ctypes.c_int, [_P, _P]),
    ("semr_batch_capture", ctypes.c_int, [_P, _P]),
    ("semr_batch_replay", ctypes.c_int, [_P, _P]),
    ("semr_batch_schedule", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("semr_batch_destroy", None, [_P]),
    ("semr_server_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64]),
    ("semr_server_submit", ctypes.c_int, [_P, ctypes.POINTER(semr_fieldset), ctypes.POINTER(semr_mesh),
                                          ctypes.POINTER(ctypes.c_uint64)]),
    ("semr_server_wait", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(semr_request_info)]),
    ("semr_server_release", ctypes.c_int, [_P, ctypes.c_uint64, _P, ctypes.c_uint64,
                                           ctypes.POINTER(ctypes.c_uint64)]),
    ("semr_server_stats", ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_uint64)] * 4 +
     [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]),
    ("semr_server_destroy", None, [_P]),
    ("semr_reduce_async_noalloc", ctypes.c_int, [ctypes.POINTER(semr_fieldset), ctypes.POINTER(semr_mesh), _P,
                                                 ctypes.c_uint64, _P, _P, _P]),
    ("semr_slice_rgba", ctypes.c_int, [ctypes.POINTER(semr_lattice), ctypes.POINTER(_P), ctypes.POINTER(semr_slice),
                                       _P, _P, _P]),
    ("semr_selftest_waits", ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
    ("semr_build_flags", ctypes.c_int, []),
    ("semr_bounds_status", ctypes.c_uint32, [ctypes.c_int]),
    ("semr_selftest_bounds", ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
]
SEMR_NOALLOC_SCRATCH_BYTES = 64 << 20

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python paper_2407_20731_b300/build.py")
_lib = ctypes.CDLL(LIB_PATH)
for _name, _res, _args in EXPORTS:
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class SemrError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {semr_strerror(code)} (status {code})")
        self.code = code


def _check(code: int, where: str) -> int:
    if code != SEMR_OK:
        raise SemrError(code, where)
    return code


# ---------------------------------------------------------------- raw ABI

def semr_strerror(code: int) -> str:
    return _lib.semr_strerror(code).decode()


def semr_build_flags() -> int:
    return _lib.semr_build_flags()


def semr_bounds_status(reset: bool = False) -> int:
    return _lib.semr_bounds_status(1 if reset else 0)


def semr_selftest_bounds() -> tuple[int, int]:
    """(return code, status word) of the checking build's self-test, in which
    every range test must fail (SEMR_EUNSUPPORTED in the default build)."""
    st = ctypes.c_uint32(0)
    rc = _lib.semr_selftest_bounds(ctypes.byref(st))
    return rc, int(st.value)


def semr_sizes_for(lx: int, n_elem: int, n_fields: int, tau: float) -> semr_sizes:
    s = semr_sizes()
    _check(_lib.semr_sizes_for(lx, n_elem, n_fields, tau, ctypes.byref(s)), "semr_sizes_for")
    return s


def semr_reduce_async(fs: semr_fieldset, mesh: semr_mesh, out: semr_outputs, stream: int) -> int:
    return _lib.semr_reduce_async(ctypes.byref(fs), ctypes.byref(mesh), ctypes.byref(out), stream)


def semr_reduce_async_timed(fs: semr_fieldset, mesh: semr_mesh, out: semr_outputs, stream: int,
                            ev_begin: int | None, ev_end: int | None) -> int:
    return _lib.semr_reduce_async_timed(ctypes.byref(fs), ctypes.byref(mesh), ctypes.byref(out), stream,
                                        ev_begin, ev_end)


def semr_reduce_async_noalloc(fs: semr_fieldset, mesh: semr_mesh, payload: int, payload_cap: int,
                              elem_report: int | None, summary: int, stream: int) -> int:
    """The reduction without any allocation: scratch comes from the library's
    fixed device array (see include/semr.h); calls must not overlap on the GPU."""
    return _lib.semr_reduce_async_noalloc(ctypes.byref(fs), ctypes.byref(mesh), payload, payload_cap,
                                          elem_report, summary, stream)


def semr_open(device: int = 0, stream: int = 0, mem_budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(_lib.semr_open(ctypes.byref(h), device, stream or None, mem_budget_bytes), "semr_open")
    return h.value


def semr_submit(handle: int, fs: semr_fieldset, mesh: semr_mesh) -> tuple[int, int]:
    t = ctypes.c_uint64(0)
    rc = _lib.semr_submit(handle, ctypes.byref(fs), ctypes.byref(mesh), ctypes.byref(t))
    return rc, t.value


def semr_query(handle: int, ticket: int) -> int:
    return _lib.semr_query(handle, ticket)


def semr_fetch(handle: int, ticket: int, wait: bool, payload: np.ndarray | None, n_fields: int,
               elem_report: np.ndarray | None = None):
    """Returns (status, payload_bytes, [semr_field_report] * n_fields)."""
    nbytes = ctypes.c_uint64(0)
    reps = (semr_field_report * max(n_fields, 1))()
    rc = _lib.semr_fetch(handle, ticket, 1 if wait else 0,
                         None if payload is None else payload.ctypes.data_as(_P),
                         0 if payload is None else payload.nbytes, ctypes.byref(nbytes), reps,
                         None if elem_report is None else elem_report.ctypes.data_as(_P))
    return rc, nbytes.value, list(reps)[:n_fields]


def semr_close(handle: int) -> None:
    _lib.semr_close(handle)


def semr_decode(payload: np.ndarray) -> np.ndarray:
    """Host decode of a payload to [n_fields, n_elem, lx^3] FP64."""
    payload = np.ascontiguousarray(payload, dtype=np.uint8)
    lx, nf, ne = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.semr_decode(payload.ctypes.data_as(_P), payload.nbytes, None, 0, ctypes.byref(lx),
                            ctypes.byref(nf), ctypes.byref(ne)), "semr_decode")
    out = np.zeros((nf.value, ne.value, lx.value ** 3))
    _check(_lib.semr_decode(payload.ctypes.data_as(_P), payload.nbytes, out.ctypes.data_as(_P), out.size,
                            None, None, None), "semr_decode")
    return out


def semr_selftest_waits() -> tuple[int, int]:
    """Status words of the look-back and mbarrier waits made to run out (both
    should be SEMR_STATUS_TIMEOUT)."""
    out = (ctypes.c_uint32 * 2)()
    _check(_lib.semr_selftest_waits(out), "semr_selftest_waits")
    return int(out[0]), int(out[1])


def semr_gll(lx: int) -> tuple[np.ndarray, np.ndarray]:
    x, w = np.zeros(lx), np.zeros(lx)
    _check(_lib.semr_gll(lx, x.ctypes.data_as(_P), w.ctypes.data_as(_P)), "semr_gll")
    return x, w


# ----------------------------------------------------- torch marshalling

def make_fieldset(fields, tau: float, precision: int = SEMR_FP64, recon=None,
                  cumulative: bool = False) -> semr_fieldset:
    """fields: sequence of CUDA FP64 tensors (contiguous, n_elem*lx^3 each).
    ``cumulative`` selects the cumulative-energy truncation (SEMR_CUMULATIVE)."""
    fs = semr_fieldset()
    fs.n_fields = len(fields)
    fs.precision = precision
    fs.tau = float(tau)
    fs.flags = (SEMR_WRITE_RECON if recon is not None else 0) | (SEMR_CUMULATIVE if cumulative else 0)
    for i, t in enumerate(fields):
        _require_cuda_f64(t)
        fs.fields[i] = t.data_ptr()
        if recon is not None:
            _require_cuda_f64(recon[i])
            fs.recon[i] = recon[i].data_ptr()
    return fs


def make_mesh(lx: int, jac) -> semr_mesh:
    _require_cuda_f64(jac)
    m = semr_mesh()
    m.lx = lx
    m.n_elem = jac.numel()
    m.jac = jac.data_ptr()
    return m


def _require_cuda_f64(t) -> None:
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")


@dataclass
class DeviceBuffers:
    """Caller-owned device buffers of one reduction (torch uint8 tensors)."""
    sizes: semr_sizes
    payload: object
    scratch: object
    summary: object
    elem_report: object | None
    outputs: semr_outputs


def alloc_buffers(lx: int, n_elem: int, n_fields: int, tau: float, device="cuda",
                  payload_cap: int | None = None, elem_report: bool = True) -> DeviceBuffers:
    import torch
    sz = semr_sizes_for(lx, n_elem, n_fields, tau)
    cap = int(sz.payload_worst if payload_cap is None else payload_cap)
    payload = torch.empty(cap, dtype=torch.uint8, device=device)
    scratch = torch.empty(int(sz.scratch_bytes) + 256, dtype=torch.uint8, device=device)
    summary = torch.zeros(ctypes.sizeof(semr_summary), dtype=torch.uint8, device=device)
    er = torch.empty(n_fields * n_elem * 3, dtype=torch.float64, device=device) if elem_report else None
    o = semr_outputs()
    o.payload = payload.data_ptr()
    o.payload_cap = cap
    o.elem_report = er.data_ptr() if er is not None else None
    o.summary = summary.data_ptr()
    sp = scratch.data_ptr()
    o.scratch = (sp + 255) // 256 * 256
    o.scratch_bytes = int(sz.scratch_bytes)
    return DeviceBuffers(sz, payload, scratch, summary, er, o)


def reduce_async(fields, jac, lx: int, tau: float, bufs: DeviceBuffers, precision: int = SEMR_FP64,
                 recon=None, stream=None, events=None, cumulative: bool = False) -> None:
    """Launch one reduction on ``stream`` (default: torch's current stream).
    ``events``: optional (begin, end) torch.cuda.Event pair recorded around the
    fused reduce kernel alone."""
    import torch
    fs = make_fieldset(fields, tau, precision, recon, cumulative)
    mesh = make_mesh(lx, jac)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    if events is None:
        _check(semr_reduce_async(fs, mesh, bufs.outputs, st), "semr_reduce_async")
    else:
        for ev in events:  # torch creates its events lazily, on the first record
            if not ev.cuda_event:
                ev.record(stream or torch.cuda.current_stream())
        _check(semr_reduce_async_timed(fs, mesh, bufs.outputs, st, events[0].cuda_event, events[1].cuda_event),
               "semr_reduce_async_timed")


def summary_from(bufs: DeviceBuffers) -> semr_summary:
    raw = bufs.summary.cpu().numpy().tobytes()
    return semr_summary.from_buffer_copy(raw)


@dataclass
class Result:
    payload: np.ndarray          # uint8
    summary: semr_summary
    elem_report: np.ndarray | None  # [F, E, 3]


def reduce(fields, jac, lx: int, tau: float, precision: int = SEMR_FP64, recon=None,
           elem_report: bool = True, cumulative: bool = False) -> Result:
    """Blocking convenience: reduce, then copy payload, summary and element
    report to the host."""
    import torch
    n_elem = jac.numel()
    bufs = alloc_buffers(lx, n_elem, len(fields), tau, fields[0].device, elem_report=elem_report)
    reduce_async(fields, jac, lx, tau, bufs, precision, recon, cumulative=cumulative)
    torch.cuda.current_stream().synchronize()
    sm = summary_from(bufs)
    payload = bufs.payload[: sm.payload_bytes].cpu().numpy()
    er = bufs.elem_report.view(len(fields), n_elem, 3).cpu().numpy() if elem_report else None
    return Result(payload, sm, er)


# ------------------------------------------------------------ batches

class Batch:
    """A planned batch of snapshot reductions (semr_batch_* entry points).

    ``snapshots``: list of (fields: list of CUDA FP64 tensors, jac, lx, tau,
    precision[, cumulative]).  Output buffers are allocated here (torch) and
    kept alive."""

    def __init__(self, snapshots, autotune: bool = True, stream=None):
        import torch
        self.snapshots = snapshots
        self.bufs = []
        items = (semr_batch_item * len(snapshots))()
        for i, snap in enumerate(snapshots):
            fields, jac, lx, tau, prec = snap[:5]
            cumulative = bool(snap[5]) if len(snap) > 5 else False
            b = alloc_buffers(lx, jac.numel(), len(fields), tau, fields[0].device)
            self.bufs.append(b)
            items[i].fs = make_fieldset(fields, tau, prec, cumulative=cumulative)
            items[i].mesh = make_mesh(lx, jac)
            items[i].out = b.outputs
        self._items = items
        st = (stream or torch.cuda.current_stream()).cuda_stream
        h = ctypes.c_void_p()
        _check(_lib.semr_batch_create(ctypes.byref(h), items, len(snapshots),
                                      SEMR_BATCH_AUTOTUNE if autotune else 0, st), "semr_batch_create")
        self.handle = h.value

    def launch(self, stream=None):
        import torch
        _check(_lib.semr_batch_launch(self.handle, (stream or torch.cuda.current_stream()).cuda_stream),
               "semr_batch_launch")

    def capture(self, stream=None):
        import torch
        _check(_lib.semr_batch_capture(self.handle, (stream or torch.cuda.current_stream()).cuda_stream),
               "semr_batch_capture")

    def replay(self, stream=None):
        import torch
        _check(_lib.semr_batch_replay(self.handle, (stream or torch.cuda.current_stream()).cuda_stream),
               "semr_batch_replay")

    def schedule(self):
        """[(lx, precision, tile, n_items, {tile: tuned_ms})] per group."""
        n = _lib.semr_batch_schedule(self.handle, -1, None, None, None, None, None, None, 0)
        out = []
        for g in range(n):
            lx, pr, tile, ni = (ctypes.c_int() for _ in range(4))
            ms = (ctypes.c_float * 4)()
            tl = (ctypes.c_int * 4)()
            _check(_lib.semr_batch_schedule(self.handle, g, ctypes.byref(lx), ctypes.byref(pr), ctypes.byref(tile),
                                            ctypes.byref(ni), ms, tl, 4), "semr_batch_schedule")
            out.append((lx.value, pr.value, tile.value, ni.value,
                        {tl[v]: ms[v] for v in range(4) if tl[v] > 0}))
        return out

    def results(self):
        """[(payload numpy, summary)] per snapshot (synchronises)."""
        import torch
        torch.cuda.synchronize()
        res = []
        for b in self.bufs:
            sm = summary_from(b)
            res.append((b.payload[: sm.payload_bytes].cpu().numpy(), sm))
        return res

    def close(self):
        if self.handle:
            _lib.semr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- serving

class Server:
    """Continuous-batching server (semr_server_* entry points)."""

    def __init__(self, device: int = 0, slots: int = 8, mem_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(_lib.semr_server_create(ctypes.byref(h), device, slots, mem_budget_bytes), "semr_server_create")
        self.handle = h.value
        self._keep = {}

    def submit(self, fields, jac, lx: int, tau: float, precision: int = SEMR_FP32, cumulative: bool = False) -> int:
        fs = make_fieldset(fields, tau, precision, cumulative=cumulative)
        mesh = make_mesh(lx, jac)
        rid = ctypes.c_uint64(0)
        _check(_lib.semr_server_submit(self.handle, ctypes.byref(fs), ctypes.byref(mesh), ctypes.byref(rid)),
               "semr_server_submit")
        self._keep[rid.value] = (fields, jac)  # inputs stay alive until release
        return rid.value

    def wait(self, rid: int, block: bool = True) -> tuple[int, semr_request_info]:
        info = semr_request_info()
        rc = _lib.semr_server_wait(self.handle, rid, 1 if block else 0, ctypes.byref(info))
        return rc, info

    def release(self, rid: int, payload: np.ndarray | None = None) -> tuple[int, int]:
        n = ctypes.c_uint64(0)
        rc = _lib.semr_server_release(self.handle, rid, None if payload is None else payload.ctypes.data_as(_P),
                                      0 if payload is None else payload.nbytes, ctypes.byref(n))
        self._keep.pop(rid, None)
        return rc, n.value

    def stats(self) -> dict:
        a, c, q, h, b = (ctypes.c_uint64() for _ in range(5))
        busy = ctypes.c_double()
        _check(_lib.semr_server_stats(self.handle, ctypes.byref(a), ctypes.byref(c), ctypes.byref(q),
                                      ctypes.byref(h), ctypes.byref(busy), ctypes.byref(b)), "semr_server_stats")
        return dict(admitted=a.value, completed=c.value, queued=q.value, held_bytes=h.value,
                    busy_seconds=busy.value, bytes_done=b.value)

    def close(self):
        if self.handle:
            _lib.semr_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ slice image

# A diverging blue - grey - red colour table (t, r, g, b).
COOL_WARM = [(0.0, 0.23, 0.30, 0.75), (0.5, 0.87, 0.87, 0.87), (1.0, 0.71, 0.02, 0.15)]


def make_lattice(lx: int, n, origin=(0.0, 0.0, 0.0), h=None) -> semr_lattice:
    """Lattice of n = (nx, ny, nz) affine elements; h defaults to the
    [0, 2 pi)^3 box of the synthetic snapshots."""
    m = semr_lattice()
    m.lx = lx
    m.nx, m.ny, m.nz = (int(v) for v in n)
    if h is None:
        h = tuple(2.0 * np.pi / int(v) for v in n)
    for d in range(3):
        m.origin[d] = float(origin[d])
        m.h[d] = float(h[d])
    return m


def make_slice(origin, axis_u, axis_v, width: int, height: int, vmin: float, vmax: float, n_comp: int = 1,
               ctrl=COOL_WARM, background: int = 0) -> semr_slice:
    s = semr_slice()
    for d in range(3):
        s.origin[d], s.axis_u[d], s.axis_v[d] = float(origin[d]), float(axis_u[d]), float(axis_v[d])
    s.width, s.height, s.n_comp = int(width), int(height), int(n_comp)
    s.vmin, s.vmax = float(vmin), float(vmax)
    s.n_ctrl = len(ctrl)
    for k, row in enumerate(ctrl):
        for c in range(4):
            s.ctrl[k][c] = float(row[c])
    s.background = int(background)
    return s


def semr_slice_rgba(mesh: semr_lattice, field_ptrs, sl: semr_slice, rgba: int, values: int | None,
                    stream: int) -> int:
    arr = (_P * SEMR_SLICE_MAX_COMP)(*[int(p) for p in field_ptrs])
    return _lib.semr_slice_rgba(ctypes.byref(mesh), arr, ctypes.byref(sl), rgba, values, stream)


def slice_rgba(fields, mesh: semr_lattice, sl: semr_slice, rgba=None, values=None, stream=None):
    """Render one slice image into device buffers (torch tensors): returns
    (rgba [H, W, 4] uint8, values [H, W] float32 or None).  ``fields``: the
    n_comp CUDA FP64 tensors (n_elem * lx^3 each)."""
    import torch
    for t in fields:
        _require_cuda_f64(t)
    dev = fields[0].device
    if rgba is None:
        rgba = torch.empty((sl.height, sl.width, 4), dtype=torch.uint8, device=dev)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(semr_slice_rgba(mesh, [t.data_ptr() for t in fields], sl, rgba.data_ptr(),
                           values.data_ptr() if values is not None else None, st), "semr_slice_rgba")
    return rgba, values


def write_ppm(path: str, rgba: np.ndarray) -> None:
    """Write an [H, W, 4] RGBA image as a binary PPM (RGB), row 0 of the
    array at the bottom (the rows run along axis_v, away from the origin)."""
    img = np.ascontiguousarray(np.asarray(rgba)[::-1, :, :3])
    with open(path, "wb") as f:
        f.write(b"P6\n%d %d\n255\n" % (img.shape[1], img.shape[0]))
        f.write(img.tobytes())
