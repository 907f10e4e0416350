"""Python binding of the C ABI in include/sbt.h (argument marshalling only).

Every computation happens in the CUDA library libsbt.so; this module checks
tensor types, passes raw pointers and allocates output tensors with PyTorch.
Importing it fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import torch

from .build import LIB

SBT_OK, SBT_ERR_ARG, SBT_ERR_CAPACITY, SBT_ERR_CUDA, SBT_ERR_TIMEOUT, SBT_ERR_STATE, SBT_EVENT_CUT = range(7)
_STATUS = {0: "SBT_OK", 1: "SBT_ERR_ARG", 2: "SBT_ERR_CAPACITY", 3: "SBT_ERR_CUDA",
           4: "SBT_ERR_TIMEOUT", 5: "SBT_ERR_STATE",
           6: "SBT_EVENT_CUT"}


class SbtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Geometry(ctypes.Structure):
    _fields_ = [("n_modules", ctypes.c_int32), ("module_z", ctypes.c_void_p),
                ("r_min", ctypes.c_float), ("r_max", ctypes.c_float),
                ("module_z2", ctypes.c_void_p)]


class Config(ctypes.Structure):
    _fields_ = [("k_doublets", ctypes.c_int32), ("max_scatter_seed", ctypes.c_float),
                ("max_scatter_follow", ctypes.c_float), ("max_chi2_tracklet", ctypes.c_float),
                ("hit_sigma", ctypes.c_float), ("max_hits_per_event", ctypes.c_int32),
                ("max_forming_tracks", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("gec_max_hits", ctypes.c_int32), ("fp16_hits", ctypes.c_int32)]


class TracksC(ctypes.Structure):
    _fields_ = [("track_offsets", ctypes.c_void_p), ("hit_offsets", ctypes.c_void_p),
                ("track_hits", ctypes.c_void_p), ("params", ctypes.c_void_p),
                ("chi2", ctypes.c_void_p), ("ndof", ctypes.c_void_p),
                ("event_status", ctypes.c_void_p), ("counts", ctypes.c_void_p),
                ("cap_tracks", ctypes.c_int32), ("cap_hits", ctypes.c_int32)]


class ResultC(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("status", ctypes.c_int32),
                ("n_tracks", ctypes.c_int32), ("hit_offsets", ctypes.c_void_p),
                ("track_hits", ctypes.c_void_p), ("params", ctypes.c_void_p),
                ("chi2", ctypes.c_void_p), ("latency_s", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"libsbt.so not built ({LIB}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB)
        sig = {
            "sbt_default_config": (_I32, [_P]),
            "sbt_create": (_I32, [_P, _P, _P]),
            "sbt_destroy": (_I32, [_P]),
            "sbt_last_error": (ctypes.c_char_p, [_P]),
            "sbt_reconstruct": (_I32, [_P, _P, _P, _P, _P, _P, _I32, _I32, _P, _P]),
            "sbt_reconstruct_batched": (_I32, [_P, _P, _P, _P, _P, _P, _I32, _I32, _P, _P]),
            "sbt_reconstruct_host": (_I32, [_P, _P, _P, _P, _P, _P, _I32, _I32, _P, _P]),
            "sbt_autotune": (_I32, [_P, _P, _P, _P, _P, _P, _I32, _I32, _P, _P, _P]),
            "sbt_tuned_shape": (_I32, [_P, _P, _P]),
            "sbt_set_launch_shape": (_I32, [_P, _I32, _I32]),
            "sbt_fit_adjoint": (_I32, [_P, _P, _P, _P, _P, _I32, _P, _P, _I32, _P, _P, _P, _P, _P]),
            "sbt_debug_sort": (_I32, [_P, _P, _P, _P, _P, _I32, _I32, _P, _P, _P, _P]),
            "sbt_debug_phi16": (_I32, [_P, _P, _I32, _P, _P]),
            "sbt_last_launch_count": (_I32, [_P]),
            "sbt_profile_batched": (_I32, [_P, _P, _P, _P, _P, _P, _I32, _I32, _P, _I32, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, h=None):
    if st != SBT_OK:
        msg = lib().sbt_last_error(h).decode() if h is not None or st != SBT_OK else ""
        raise SbtError(st, msg)


def _ptr(t: torch.Tensor | None, dtype: torch.dtype, name: str, device=True) -> int | None:
    if t is None:
        return None
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if device and not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if not device and t.is_cuda:
        raise ValueError(f"{name}: must be a host tensor")
    return t.data_ptr() if t.numel() > 0 else None


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def default_config(**overrides) -> Config:
    c = Config()
    _check(lib().sbt_default_config(ctypes.byref(c)))
    for k, v in overrides.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


@dataclasses.dataclass
class TrackOutput:
    """CSR tracks (see sbt_tracks in include/sbt.h)."""

    track_offsets: torch.Tensor
    hit_offsets: torch.Tensor
    track_hits: torch.Tensor
    params: torch.Tensor
    chi2: torch.Tensor
    ndof: torch.Tensor
    event_status: torch.Tensor
    counts: torch.Tensor

    @classmethod
    def allocate(cls, n_events: int, n_hits: int, device="cuda", cap_tracks=None, cap_hits=None,
                 pin_memory=False):
        cap_tracks = n_hits // 3 + 1 if cap_tracks is None else cap_tracks
        cap_hits = n_hits + 1 if cap_hits is None else cap_hits
        kw = dict(device=device)
        if pin_memory:
            kw = dict(device="cpu", pin_memory=True)
        i32 = dict(dtype=torch.int32, **kw)
        return cls(torch.zeros(n_events + 1, **i32), torch.zeros(cap_tracks + 1, **i32),
                   torch.zeros(cap_hits, **i32), torch.zeros(cap_tracks * 4, dtype=torch.float32, **kw),
                   torch.zeros(cap_tracks, dtype=torch.float32, **kw), torch.zeros(cap_tracks, **i32),
                   torch.zeros(n_events, **i32), torch.zeros(4, **i32))

    def c_struct(self, device=True) -> TracksC:
        f32, i32 = torch.float32, torch.int32
        return TracksC(_ptr(self.track_offsets, i32, "track_offsets", device),
                       _ptr(self.hit_offsets, i32, "hit_offsets", device),
                       _ptr(self.track_hits, i32, "track_hits", device),
                       _ptr(self.params, f32, "params", device), _ptr(self.chi2, f32, "chi2", device),
                       _ptr(self.ndof, i32, "ndof", device),
                       _ptr(self.event_status, i32, "event_status", device),
                       _ptr(self.counts, i32, "counts", device),
                       self.chi2.numel(), self.track_hits.numel())

    def compact(self) -> dict:
        """Host numpy copies trimmed to the produced sizes."""
        c = self.counts.cpu().numpy()
        T, H = int(c[0]), int(c[1])
        return dict(track_offsets=self.track_offsets.cpu().numpy(),
                    hit_offsets=self.hit_offsets[:T + 1].cpu().numpy(),
                    track_hits=self.track_hits[:H].cpu().numpy(),
                    params=self.params[:4 * T].cpu().numpy().reshape(T, 4),
                    chi2=self.chi2[:T].cpu().numpy(), ndof=self.ndof[:T].cpu().numpy(),
                    event_status=self.event_status.cpu().numpy(), counts=c)


class Handle:
    """Owns an sbt_handle (sbt_create / sbt_destroy)."""

    def __init__(self, module_z, config: Config | None = None, r_min=5.1, r_max=42.0,
                 module_z2=None):
        """module_z2: plane z of the x < 0 side of each module pair (None:
        one plane per module)."""
        import numpy as np
        self._mz = np.ascontiguousarray(np.asarray(module_z, dtype=np.float32))
        self._mz2 = (None if module_z2 is None
                     else np.ascontiguousarray(np.asarray(module_z2, dtype=np.float32)))
        if self._mz2 is not None and self._mz2.shape != self._mz.shape:
            raise ValueError("module_z2 must have one entry per module")
        g = Geometry(self._mz.shape[0], self._mz.ctypes.data, r_min, r_max,
                     self._mz2.ctypes.data if self._mz2 is not None else None)
        h = ctypes.c_void_p()
        st = lib().sbt_create(ctypes.byref(g), ctypes.byref(config) if config is not None else None,
                              ctypes.byref(h))
        if st != SBT_OK:
            raise SbtError(st, lib().sbt_last_error(None).decode())
        self.h = h
        self.n_modules = self._mz.shape[0]

    def close(self):
        if getattr(self, "h", None):
            lib().sbt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_launch_count(self) -> int:
        return int(lib().sbt_last_launch_count(self.h))


def sbt_create(module_z, config: Config | None = None, **kw) -> Handle:
    return Handle(module_z, config, **kw)


def sbt_destroy(h: Handle):
    h.close()


def _inputs(x, y, z, module, offsets):
    f32, i32 = torch.float32, torch.int32
    return (_ptr(x, f32, "x"), _ptr(y, f32, "y"), _ptr(z, f32, "z"), _ptr(module, i32, "module"),
            _ptr(offsets, i32, "event_offsets"), offsets.numel() - 1, x.numel())


def _reco(fn, h: Handle, x, y, z, module, event_offsets, out: TrackOutput | None, stream):
    px, py, pz, pm, po, E, H = _inputs(x, y, z, module, event_offsets)
    if out is None:
        out = TrackOutput.allocate(E, H, device=x.device)
    oc = out.c_struct()
    _check(fn(h.h, px, py, pz, pm, po, E, H, ctypes.byref(oc), _stream(stream)), h.h)
    return out


def sbt_reconstruct(h: Handle, x, y, z, module, event_offsets, out=None, stream=None) -> TrackOutput:
    """One block per event (plain launch)."""
    return _reco(lib().sbt_reconstruct, h, x, y, z, module, event_offsets, out, stream)


def sbt_reconstruct_batched(h: Handle, x, y, z, module, event_offsets, out=None,
                            stream=None) -> TrackOutput:
    """Persistent work-queue launch replayed from a CUDA graph."""
    return _reco(lib().sbt_reconstruct_batched, h, x, y, z, module, event_offsets, out, stream)


def sbt_reconstruct_host(h: Handle, x, y, z, module, event_offsets, out: TrackOutput | None = None,
                         stream=None) -> TrackOutput:
    """Host tensors in, host tensors out (copies inside the call)."""
    f32, i32 = torch.float32, torch.int32
    args = (_ptr(x, f32, "x", False), _ptr(y, f32, "y", False), _ptr(z, f32, "z", False),
            _ptr(module, i32, "module", False), _ptr(event_offsets, i32, "event_offsets", False))
    E, H = event_offsets.numel() - 1, x.numel()
    if out is None:
        out = TrackOutput.allocate(E, H, pin_memory=True)
    oc = out.c_struct(device=False)
    _check(lib().sbt_reconstruct_host(h.h, *args, E, H, ctypes.byref(oc), _stream(stream)), h.h)
    return out


def sbt_reconstruct_noalloc(h: Handle, x, y, z, module, event_offsets, out: TrackOutput,
                            stream=None) -> TrackOutput:
    """sbt_reconstruct for callers that must not allocate device memory: the
    library allocates nothing (its workspace is a fixed array in its device
    image, at most 524288 hits and 4096 events per call) and the caller passes
    preallocated outputs.  Calls that overlap on the GPU share that workspace
    and must be serialised."""
    f = lib().sbt_reconstruct_noalloc
    f.restype = _I32
    f.argtypes = [_P, _P, _P, _P, _P, _P, _I32, _I32, _P, _P]
    return _reco(f, h, x, y, z, module, event_offsets, out, stream)


def sbt_autotune(h: Handle, x, y, z, module, event_offsets, stream=None) -> tuple[int, int]:
    """Tunes the persistent launch on these events: (block size, resident blocks per SM)."""
    px, py, pz, pm, po, E, H = _inputs(x, y, z, module, event_offsets)
    chosen, per_sm = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().sbt_autotune(h.h, px, py, pz, pm, po, E, H, ctypes.byref(chosen), ctypes.byref(per_sm),
                              _stream(stream)), h.h)
    return int(chosen.value), int(per_sm.value)


def sbt_set_launch_shape(h: Handle, threads: int, blocks_per_sm: int):
    """Gives the handle a launch shape, e.g. one tuned on another handle."""
    _check(lib().sbt_set_launch_shape(h.h, int(threads), int(blocks_per_sm)), h.h)


def sbt_tuned_shape(h: Handle) -> tuple[int, int]:
    """(block size, resident blocks per SM) chosen by sbt_autotune; (0, 0) before it."""
    t, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().sbt_tuned_shape(h.h, ctypes.byref(t), ctypes.byref(b)), h.h)
    return int(t.value), int(b.value)


def sbt_profile_batched(h: Handle, x, y, z, module, event_offsets, out: TrackOutput, reps=3,
                        stream=None):
    """Mean ms per launch of (ordering, sort, persistent search, scan, output)."""
    px, py, pz, pm, po, E, H = _inputs(x, y, z, module, event_offsets)
    ms = (ctypes.c_float * 5)()
    oc = out.c_struct()
    _check(lib().sbt_profile_batched(h.h, px, py, pz, pm, po, E, H, ctypes.byref(oc), int(reps), ms,
                                     _stream(stream)), h.h)
    return [float(v) for v in ms]


def sbt_fit_adjoint(h: Handle, x, y, z, module, hit_offsets, track_hits, align,
                    want_grad=True, stream=None, with_skipped=False):
    """(chi2_sum [1] fp64, grad [n_modules, 6] fp64 or None) as CUDA tensors;
    with_skipped adds the number of tracks without a straight-line fit or
    with an index out of range ([1] int32), which contribute nothing."""
    f32, i32, f64 = torch.float32, torch.int32, torch.float64
    chi2 = torch.zeros(1, dtype=f64, device=x.device)
    grad = torch.zeros(h.n_modules * 6, dtype=f64, device=x.device) if want_grad else None
    skipped = torch.zeros(1, dtype=i32, device=x.device) if with_skipped else None
    st = lib().sbt_fit_adjoint(h.h, _ptr(x, f32, "x"), _ptr(y, f32, "y"), _ptr(z, f32, "z"),
                               _ptr(module, i32, "module"), x.numel(),
                               _ptr(hit_offsets, i32, "hit_offsets"),
                               _ptr(track_hits, i32, "track_hits"), hit_offsets.numel() - 1,
                               _ptr(align.contiguous(), f64, "align"), _ptr(chi2, f64, "chi2"),
                               _ptr(grad, f64, "grad") if grad is not None else None,
                               _ptr(skipped, i32, "skipped") if skipped is not None else None,
                               _stream(stream))
    _check(st, h.h)
    res = (chi2, (grad.view(h.n_modules, 6) if grad is not None else None))
    return res + (skipped,) if with_skipped else res


def sbt_debug_sort(h: Handle, x, y, module, event_offsets, stream=None):
    f32, i32 = torch.float32, torch.int32
    E, H = event_offsets.numel() - 1, x.numel()
    phi = torch.zeros(max(H, 1), dtype=torch.int16, device=x.device)
    perm = torch.zeros(max(H, 1), dtype=i32, device=x.device)
    mo = torch.zeros(max(E * (h.n_modules + 1), 1), dtype=i32, device=x.device)
    st = lib().sbt_debug_sort(h.h, _ptr(x, f32, "x"), _ptr(y, f32, "y"), _ptr(module, i32, "module"),
                              _ptr(event_offsets, i32, "event_offsets"), E, H, phi.data_ptr(),
                              perm.data_ptr(), mo.data_ptr(), _stream(stream))
    _check(st, h.h)
    return phi[:H], perm[:H], mo[:E * (h.n_modules + 1)].view(E, h.n_modules + 1)


def sbt_debug_phi16(x, y, stream=None) -> torch.Tensor:
    out = torch.zeros(max(x.numel(), 1), dtype=torch.int16, device=x.device)
    st = lib().sbt_debug_phi16(_ptr(x, torch.float32, "x"), _ptr(y, torch.float32, "y"), x.numel(),
                               out.data_ptr(), _stream(stream))
    _check(st)
    return out[:x.numel()]


class AlignmentChi2(torch.autograd.Function):
    """Summed track-fit chi2 as a function of the alignment parameters [M, 6]
    (fp64); the backward pass returns the gradient computed by the adjoint
    kernel in the same call."""

    @staticmethod
    def forward(ctx, align, handle, x, y, z, module, hit_offsets, track_hits):
        chi2, grad = sbt_fit_adjoint(handle, x, y, z, module, hit_offsets, track_hits,
                                     align.detach(), want_grad=True)
        ctx.save_for_backward(grad)
        return chi2[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None, None, None, None, None


def alignment_chi2(handle: Handle, x, y, z, module, hit_offsets, track_hits, align):
    return AlignmentChi2.apply(align, handle, x, y, z, module, hit_offsets, track_hits)


# ------------------------------------------------------------------ serving --


def _server_sigs():
    L = lib()
    sig = {
        "sbt_server_create": (_I32, [_P, _I64, _I32, _I32, _P]),
        "sbt_server_submit": (_I32, [_P, _I64, _P, _P, _P, _P, _I32]),
        "sbt_server_submit_schedule": (_I32, [_P, _P, _P, _P, _P, _P, _I32, _P, _I64]),
        "sbt_server_poll": (_I32, [_P, _P, _I32, _P, ctypes.c_double]),
        "sbt_server_drain": (_I32, [_P, _P, _P, _P, _I32, _P, ctypes.c_double]),
        "sbt_server_release": (_I32, [_P, _I64]),
        "sbt_server_stats": (_I32, [_P, _P]),
        "sbt_server_inject_failure": (_I32, [_P]),
        "sbt_server_destroy": (_I32, [_P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


@dataclasses.dataclass
class ServedResult:
    request_id: int
    status: int
    hit_offsets: "object"
    track_hits: "object"
    params: "object"
    chi2: "object"
    latency_s: float


class Server:
    """Continuous-batching request loop (sbt_server_* in include/sbt.h)."""

    def __init__(self, handle: Handle, memory_budget_bytes: int, max_streams: int = 4,
                 max_batch_events: int = 256):
        self.L = _server_sigs()
        s = ctypes.c_void_p()
        _check(self.L.sbt_server_create(handle.h, int(memory_budget_bytes), int(max_streams),
                                        int(max_batch_events), ctypes.byref(s)))
        self.s = s
        self._keep = []

    def submit(self, request_id: int, x, y, z, module):
        import numpy as np
        x, y, z = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, y, z))
        module = np.ascontiguousarray(module, dtype=np.int32)
        _check(self.L.sbt_server_submit(self.s, int(request_id), x.ctypes.data, y.ctypes.data,
                                        z.ctypes.data, module.ctypes.data, x.shape[0]))

    def submit_schedule(self, ev, arrival_s, first_id: int = 0):
        import numpy as np
        arrays = [np.ascontiguousarray(a) for a in (ev.x, ev.y, ev.z, ev.module, ev.event_offsets)]
        at = np.ascontiguousarray(arrival_s, dtype=np.float64)
        _check(self.L.sbt_server_submit_schedule(self.s, *[a.ctypes.data for a in arrays],
                                                 ev.n_events, at.ctypes.data, int(first_id)))

    def poll(self, max_results: int = 1024, timeout_s: float = 0.0):
        import numpy as np
        buf = (ResultC * max_results)()
        n = ctypes.c_int32()
        st = self.L.sbt_server_poll(self.s, buf, max_results, ctypes.byref(n), float(timeout_s))
        if st == SBT_ERR_TIMEOUT:
            return []
        _check(st)
        out = []
        for r in buf[:n.value]:
            T = r.n_tracks
            ho = np.ctypeslib.as_array((ctypes.c_int32 * (T + 1)).from_address(r.hit_offsets)).copy()
            H = int(ho[-1])
            th = (np.ctypeslib.as_array((ctypes.c_int32 * H).from_address(r.track_hits)).copy()
                  if H else np.zeros(0, np.int32))
            pr = (np.ctypeslib.as_array((ctypes.c_float * (4 * T)).from_address(r.params)).copy()
                  if T else np.zeros(0, np.float32))
            c2 = (np.ctypeslib.as_array((ctypes.c_float * T).from_address(r.chi2)).copy()
                  if T else np.zeros(0, np.float32))
            out.append(ServedResult(r.request_id, r.status, ho, th, pr.reshape(T, 4), c2, r.latency_s))
            self.L.sbt_server_release(self.s, r.request_id)
        return out

    def drain(self, max_results: int = 65536, timeout_s: float = 0.0):
        """(ids, status, latency_s) numpy arrays of finished requests; results released."""
        import numpy as np
        ids = np.empty(max_results, np.int64)
        st = np.empty(max_results, np.int32)
        lat = np.empty(max_results, np.float64)
        n = ctypes.c_int32()
        rc = self.L.sbt_server_drain(self.s, ids.ctypes.data, st.ctypes.data, lat.ctypes.data,
                                     max_results, ctypes.byref(n), float(timeout_s))
        if rc == SBT_ERR_TIMEOUT:
            n.value = 0
        else:
            _check(rc)
        k = n.value
        return ids[:k], st[:k], lat[:k]

    def stats(self) -> dict:
        v = (ctypes.c_double * 14)()
        _check(self.L.sbt_server_stats(self.s, v))
        return {"completed": v[0], "submitted": v[1], "batches": v[2], "mean_batch_events": v[3],
                "peak_bytes": v[4], "failed_batches": v[5], "feed_lag_s": v[6],
                "launch_busy_s": v[7], "upload_ms": v[8], "kernel_ms": v[9], "download_ms": v[10],
                "batch_wall_ms": v[11], "timed_batches": v[12], "allocations": v[13]}

    def inject_failure(self):
        _check(self.L.sbt_server_inject_failure(self.s))

    def close(self):
        if getattr(self, "s", None):
            self.L.sbt_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
