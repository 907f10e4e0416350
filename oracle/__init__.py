"""Plain CPU oracle of Search by triplet (arXiv 2207.03936).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use this package to check and time the CUDA library.  The
product path never imports it.  The C source (sbt_oracle.c) states the
algorithm and every reading of the paper it takes.

Parity pins live in tests/test_oracle_*.py (closed forms, library routines,
hand-built events with known answers, invariants, truth matching).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsbt_oracle.so")

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")


class Config(ctypes.Structure):
    """Tunable constants of the method (the paper calls them configurable)."""

    _fields_ = [("k_doublets", ctypes.c_int32),
                ("max_scatter_seed", ctypes.c_float),
                ("max_scatter_follow", ctypes.c_float),
                ("max_chi2_tracklet", ctypes.c_float),
                ("hit_sigma", ctypes.c_float)]


def config(k_doublets=4, max_scatter_seed=0.04, max_scatter_follow=0.04,
           max_chi2_tracklet=20.0, hit_sigma=0.012) -> Config:
    return Config(k_doublets, max_scatter_seed, max_scatter_follow, max_chi2_tracklet, hit_sigma)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction, no fast-math."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.sbt_oracle_atan2.restype = ctypes.c_float
        L.sbt_oracle_atan2.argtypes = [ctypes.c_float, ctypes.c_float]
        L.sbt_oracle_phi16.restype = ctypes.c_uint16
        L.sbt_oracle_phi16.argtypes = [ctypes.c_float, ctypes.c_float]
        L.sbt_oracle_phi16_array.restype = None
        L.sbt_oracle_phi16_array.argtypes = [_f32p, _f32p, ctypes.c_int32, _u16p]
        L.sbt_oracle_phi_distance.restype = ctypes.c_int32
        L.sbt_oracle_phi_distance.argtypes = [ctypes.c_uint16, ctypes.c_uint16]
        L.sbt_oracle_sort_event.restype = ctypes.c_int32
        L.sbt_oracle_sort_event.argtypes = [_f32p, _f32p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                            _i32p, _i32p, _u16p]
        L.sbt_oracle_fit.restype = None
        L.sbt_oracle_fit.argtypes = [_f32p, _f32p, _f32p, ctypes.c_int32, ctypes.c_float,
                                     _f32p, ctypes.POINTER(ctypes.c_float)]
        L.sbt_oracle_event.restype = ctypes.c_int32
        L.sbt_oracle_event.argtypes = [_f32p, _f32p, _f32p, _i32p, ctypes.c_int32, _f32p,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Config),
                                       _i32p, _i32p,
                                       _f32p, _f32p, _i32p, _i32p]
        L.sbt_oracle_batch.restype = ctypes.c_int32
        L.sbt_oracle_batch.argtypes = [_f32p, _f32p, _f32p, _i32p, _i32p, ctypes.c_int32, _f32p,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Config),
                                       ctypes.c_int32,
                                       _i32p, _i32p, _i32p, _i32p, _i32p, _f32p, _f32p, _i32p,
                                       _i32p]
        L.sbt_oracle_seed_step.restype = ctypes.c_int32
        L.sbt_oracle_seed_step.argtypes = [_f32p, _f32p, _f32p, _i32p, ctypes.c_int32, _f32p,
                                           ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Config),
                                           ctypes.c_int32,
                                           ctypes.c_void_p, _i32p, _i32p, _i32p]
        L.sbt_oracle_align_chi2.restype = ctypes.c_double
        L.sbt_oracle_align_chi2.argtypes = [_f32p, _f32p, _f32p, _i32p, ctypes.c_int32, _i32p, _i32p,
                                            ctypes.c_int32, _f32p, ctypes.c_int32, _f64p,
                                            ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _second_planes(module_z2, M: int):
    """(array kept alive, pointer) of the second plane positions of module
    pairs, or (None, None) for single planes."""
    if module_z2 is None:
        return None, None
    z2 = _f32(module_z2)
    if z2.shape != (M,):
        raise ValueError("module_z2 must have one entry per module")
    return z2, z2.ctypes.data


def atan2(y: float, x: float) -> float:
    return float(lib().sbt_oracle_atan2(float(y), float(x)))


def phi16(x, y) -> np.ndarray:
    x, y = _f32(x), _f32(y)
    out = np.empty(x.shape[0], dtype=np.uint16)
    lib().sbt_oracle_phi16_array(x, y, x.shape[0], out)
    return out


def phi_distance(u: int, v: int) -> int:
    return int(lib().sbt_oracle_phi_distance(u, v))


def sort_event(x, y, module, n_modules: int):
    """Returns (perm, module_offsets, phi16 in sorted order)."""
    x, y, module = _f32(x), _f32(y), _i32(module)
    n = x.shape[0]
    perm = np.empty(max(n, 1), np.int32)
    offs = np.empty(n_modules + 1, np.int32)
    phs = np.empty(max(n, 1), np.uint16)
    rc = lib().sbt_oracle_sort_event(x, y, module, n, n_modules, perm, offs, phs)
    if rc != 0:
        raise ValueError("invalid event")
    return perm[:n], offs, phs[:n]


def fit(x, y, z, sigma: float):
    """Straight-line least-squares fit: ((x0, y0, tx, ty), chi2)."""
    x, y, z = _f32(x), _f32(y), _f32(z)
    p = np.empty(4, np.float32)
    c = ctypes.c_float()
    lib().sbt_oracle_fit(x, y, z, x.shape[0], sigma, p, ctypes.byref(c))
    return p, np.float32(c.value)


@dataclasses.dataclass
class Tracks:
    """Reconstructed tracks in CSR form (batch-global hit indices)."""

    track_offsets: np.ndarray   # int32 [n_events + 1]
    hit_offsets: np.ndarray     # int32 [n_tracks + 1]
    track_hits: np.ndarray      # int32 [n_track_hits]
    params: np.ndarray          # float32 [n_tracks, 4]  (x0, y0, tx, ty)
    chi2: np.ndarray            # float32 [n_tracks]
    ndof: np.ndarray            # int32 [n_tracks]
    status: np.ndarray          # int32 [n_events]
    stats: np.ndarray           # int32 [n_events, 8]

    @property
    def n_tracks(self) -> int:
        return int(self.hit_offsets.shape[0] - 1)


def event(x, y, z, module, module_z, cfg: Config | None = None, module_z2=None):
    """Reconstruct one event; hit indices are local to the event.  module_z2:
    second plane of each module pair (hits with x < 0), None for single planes."""
    cfg = cfg or config()
    x, y, z, module, module_z = _f32(x), _f32(y), _f32(z), _i32(module), _f32(module_z)
    z2, z2p = _second_planes(module_z2, module_z.shape[0])
    n = x.shape[0]
    cap = max(n, 1)
    tl = np.empty(cap, np.int32)
    th = np.empty(cap, np.int32)
    pr = np.empty(4 * cap, np.float32)
    c2 = np.empty(cap, np.float32)
    nd = np.empty(cap, np.int32)
    st = np.zeros(8, np.int32)
    nt = lib().sbt_oracle_event(x, y, z, module, n, module_z, z2p, module_z.shape[0],
                                ctypes.byref(cfg), tl, th, pr, c2, nd, st)
    if nt < 0:
        raise ValueError("invalid event")
    h = int(tl[:nt].sum())
    ho = np.zeros(nt + 1, np.int32)
    np.cumsum(tl[:nt], out=ho[1:])
    return Tracks(np.array([0, nt], np.int32), ho, th[:h].copy(), pr[:4 * nt].reshape(nt, 4).copy(),
                  c2[:nt].copy(), nd[:nt].copy(), np.zeros(1, np.int32), st.reshape(1, 8))


def round_fp16(a) -> np.ndarray:
    """fp32 values rounded to the nearest fp16 (ties to even) and back: the
    coordinates of the fp16 hit-storage mode (the paper stores VELO hit
    coordinates in 16-bit floats; its optimisation table, 05-03-2020)."""
    return _f32(a).astype(np.float16).astype(np.float32)


def reconstruct(x, y, z, module, event_offsets, module_z, cfg: Config | None = None,
                n_threads: int | None = None, fp16_hits: bool = False, module_z2=None) -> Tracks:
    """Reconstruct a batch of events on host threads; returns CSR tracks.
    With fp16_hits the hit coordinates are first rounded to fp16, as the
    fp16 hit-storage mode keeps them; everything after is unchanged.
    module_z2: second plane of each module pair (hits with x < 0), None for
    single planes."""
    cfg = cfg or config()
    x, y, z, module = _f32(x), _f32(y), _f32(z), _i32(module)
    if fp16_hits:
        x, y, z = round_fp16(x), round_fp16(y), round_fp16(z)
    eo, module_z = _i32(event_offsets), _f32(module_z)
    z2, z2p = _second_planes(module_z2, module_z.shape[0])
    E = eo.shape[0] - 1
    H = int(eo[-1]) if E >= 0 else 0
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    tcap = H // 3 + E + 1
    ntr = np.zeros(max(E, 1), np.int32)
    nh = np.zeros(max(E, 1), np.int32)
    st = np.zeros(max(E, 1), np.int32)
    sl = np.zeros(tcap, np.int32)
    sh = np.zeros(max(H, 1), np.int32)
    sp = np.zeros(4 * tcap, np.float32)
    sc = np.zeros(tcap, np.float32)
    sn = np.zeros(tcap, np.int32)
    ss = np.zeros(8 * max(E, 1), np.int32)
    lib().sbt_oracle_batch(x, y, z, module, eo, E, module_z, z2p, module_z.shape[0],
                           ctypes.byref(cfg), int(n_threads), ntr, nh, st, sl, sh, sp, sc, sn, ss)
    ntr, nh, st = ntr[:E], nh[:E], st[:E]
    to = np.zeros(E + 1, np.int32)
    np.cumsum(ntr, out=to[1:])
    T = int(to[-1])
    # gather slots into CSR
    tslot = eo[:-1] // 3
    sel_t = (np.repeat(tslot - to[:-1], ntr) + np.arange(T)).astype(np.int64)
    lens = sl[sel_t]
    ho = np.zeros(T + 1, np.int32)
    np.cumsum(lens, out=ho[1:])
    hsel = (np.repeat(eo[:-1].astype(np.int64), nh)
            + np.arange(int(ho[-1])) - np.repeat(np.cumsum(nh) - nh, nh)).astype(np.int64)
    hits = sh[hsel] if ho[-1] > 0 else np.zeros(0, np.int32)
    params = sp.reshape(-1, 4)[sel_t]
    return Tracks(to, ho, hits.astype(np.int32), params.astype(np.float32), sc[sel_t], sn[sel_t],
                  st, ss[:8 * E].reshape(E, 8))


def seed_step(x, y, z, module, module_z, s: int, cfg: Config | None = None, flags=None,
              module_z2=None):
    """Seeds of seeding step s as (a, c, b) sorted positions, ordered by c."""
    cfg = cfg or config()
    x, y, z, module, module_z = _f32(x), _f32(y), _f32(z), _i32(module), _f32(module_z)
    z2, z2p = _second_planes(module_z2, module_z.shape[0])
    n = x.shape[0]
    cap = max(n, 1)
    oa, oc, ob = (np.empty(cap, np.int32) for _ in range(3))
    fl = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
    cnt = lib().sbt_oracle_seed_step(x, y, z, module, n, module_z, z2p, module_z.shape[0],
                                     ctypes.byref(cfg), int(s),
                                     fl.ctypes.data if fl is not None else None, oa, oc, ob)
    if cnt < 0:
        raise ValueError("invalid event or step")
    return np.stack([oa[:cnt], oc[:cnt], ob[:cnt]], axis=1)


def align_chi2(x, y, z, module, hit_offsets, track_hits, module_z, align, sigma: float,
               want_grad: bool = True, count_skipped: bool = False):
    """fp64 summed chi2 of fixed tracks after per-module alignment, and its
    gradient; with count_skipped also the number of tracks without a
    straight-line fit (fewer than two hits or modules, or an index out of
    range), which contribute nothing."""
    x, y, z, module = _f32(x), _f32(y), _f32(z), _i32(module)
    ho, th, module_z = _i32(hit_offsets), _i32(track_hits), _f32(module_z)
    align = np.ascontiguousarray(align, dtype=np.float64).reshape(-1)
    M = module_z.shape[0]
    g = np.zeros(6 * M, np.float64) if want_grad else None
    sk = np.zeros(1, np.int32)
    v = lib().sbt_oracle_align_chi2(x, y, z, module, x.shape[0], ho, th, ho.shape[0] - 1, module_z, M,
                                    align, float(sigma), g.ctypes.data if g is not None else None,
                                    sk.ctypes.data)
    res = (v, (g.reshape(M, 6) if g is not None else None))
    return res + (int(sk[0]),) if count_skipped else res
