"""Seeded synthetic VELO events with generator truth.

This module only draws inputs: it holds none of the reconstruction's
arithmetic, and both the CUDA path and the CPU oracle consume its arrays.

Geometry (Section 1 and Fig. 2 of the paper: 52 planar pixel modules around
the beam line).  Module planes sit at z = -290 + k * 1040/51 mm, k = 0..51,
with an active annulus 5.1 <= r <= 42 mm.  Module ids are given in traversal
order: id 0 is the plane furthest from the interaction point (z = 750 mm),
where occupancy is lowest, and ids increase towards smaller z.

Event recipe (the paper's upgrade Monte Carlo is not available, so these
stand in for it):

* primary vertices: z ~ N(0, 60 mm), x, y ~ N(0, 0.03 mm);
* per vertex Poisson(mu) forward tracks with eta ~ U(2, 5) and, where
  requested, Poisson(mu * backward_frac) backward tracks with
  eta ~ U(-5, -2); phi ~ U(0, 2 pi); straight lines from the vertex;
* optional multiple-scattering kinks: after every module plane a track
  crosses near the annulus, both slopes receive N(0, kink_sigma) kicks;
* a hit is recorded where the track crosses a plane inside the annulus,
  with probability hit_eff, smeared by N(0, 12 um) in x and y; hit z is the
  plane z;
* noise hits: Poisson(noise_frac * track hits) per event, uniform in the
  annulus area on uniformly drawn modules;
* hits are shuffled within each event (the reconstruction must not depend
  on input order beyond its stated tie-breaks).

Module-pair geometry (``pairs=True``; the paper's VELO has its modules on two
sides of the beam, Fig. 2, and the method works on module pairs, section
"Search by triplet").  The 52 planes stay where they are, but each covers one
side only: plane k (ascending z) records hits with x >= 0 when k is even and
x < 0 when k is odd (decided on the measured x; hits within 1 um of x = 0
are dropped so that the sign of a stored coordinate always names its plane).
Planes 2q and 2q + 1 form module pair q; the algorithm sees 26 modules (pair
ids in traversal order, 0 = the pair furthest from the interaction point)
and takes each pair's two plane positions, ``module_z`` for its x >= 0 plane
and ``module_z2`` for its x < 0 plane.  A straight track thus leaves one hit
per pair, about 41 mm apart.

Random numbers come from numpy's PCG64 with a fixed seed; events are drawn
in fixed chunks so the result does not depend on the machine.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_MODULES = 52
N_PAIRS = N_MODULES // 2
R_MIN = 5.1
R_MAX = 42.0
Z_FIRST = -290.0
Z_LAST = 750.0
PITCH = (Z_LAST - Z_FIRST) / (N_MODULES - 1)


def module_z_ascending() -> np.ndarray:
    """Plane z positions in ascending z (float64)."""
    return Z_FIRST + np.arange(N_MODULES, dtype=np.float64) * PITCH


def module_z_traversal() -> np.ndarray:
    """Plane z positions indexed by module id (traversal order, descending z), float32."""
    return module_z_ascending()[::-1].astype(np.float32).copy()


@dataclasses.dataclass
class Events:
    """Structure-of-arrays hits of a batch of events.

    x, y, z: float32 [n_hits]; module: int32 [n_hits] (traversal-order id);
    event_offsets: int32 [n_events + 1]; mc: int32 [n_hits] particle id of
    each hit (-1 for noise); particles are numbered globally over the batch.
    """

    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    module: np.ndarray
    event_offsets: np.ndarray
    mc: np.ndarray
    n_particles: int
    module_z: np.ndarray
    module_z2: np.ndarray | None = None   # second plane of each module pair (x < 0 side)

    @property
    def n_events(self) -> int:
        return int(self.event_offsets.shape[0] - 1)

    @property
    def n_hits(self) -> int:
        return int(self.event_offsets[-1])

    def hits_per_event(self) -> np.ndarray:
        return np.diff(self.event_offsets)

    def subset(self, first: int, count: int) -> "Events":
        """Events [first, first + count) as a new batch (offsets rebased)."""
        lo = int(self.event_offsets[first])
        hi = int(self.event_offsets[first + count])
        sl = slice(lo, hi)
        mc = self.mc[sl].copy()
        return Events(self.x[sl].copy(), self.y[sl].copy(), self.z[sl].copy(),
                      self.module[sl].copy(),
                      (self.event_offsets[first:first + count + 1] - lo).astype(np.int32),
                      mc, self.n_particles, self.module_z, self.module_z2)


@dataclasses.dataclass
class Recipe:
    n_events: int
    pv_mode: str = "fixed"          # "fixed" | "poisson" | "uniform"
    pv_mean: float = 1.0            # fixed count, Poisson mean, or (lo, hi) via pv_lo/pv_hi
    pv_lo: int = 1
    pv_hi: int = 20
    tracks_per_pv: float = 30.0
    backward_frac: float = 0.0
    kink_sigma: float = 0.0         # rad, per module plane
    hit_eff: float = 0.98
    smear: float = 0.012            # mm
    noise_frac: float = 0.01
    misalign: bool = False
    pairs: bool = False             # module-pair geometry (two one-sided planes per module)
    seed: int = 0


# The five workloads of this project (plain small, upgrade conditions,
# uneven-size batching, serving stream, alignment differentiation).
def recipe_for(config: int, n_events: int | None = None, seed: int = 0) -> Recipe:
    if config == 1:
        r = Recipe(n_events=16, pv_mode="fixed", pv_mean=1, tracks_per_pv=30.0)
    elif config in (2, 4):
        r = Recipe(n_events=1000, pv_mode="poisson", pv_mean=7.6, tracks_per_pv=25.0,
                   backward_frac=0.1, kink_sigma=0.5e-3)
    elif config == 3:
        r = Recipe(n_events=100_000, pv_mode="uniform", pv_lo=1, pv_hi=20, tracks_per_pv=25.0,
                   backward_frac=0.1, kink_sigma=0.5e-3)
    elif config == 5:
        r = Recipe(n_events=10_000, pv_mode="poisson", pv_mean=7.6, tracks_per_pv=25.0,
                   backward_frac=0.1, kink_sigma=0.5e-3, misalign=True)
    else:
        raise ValueError(f"unknown workload {config}")
    if n_events is not None:
        r.n_events = int(n_events)
    r.seed = seed
    return r


def misalignment(seed: int = 0) -> np.ndarray:
    """Per-module placement errors [52, 6] float64: (tx, ty, tz) ~ N(0, 10 um),
    (rx, ry, rz) ~ N(0, 0.1 mrad)."""
    rng = np.random.Generator(np.random.PCG64([seed, 0xA11])).normal
    t = rng(0.0, 0.010, size=(N_MODULES, 3))
    w = rng(0.0, 1.0e-4, size=(N_MODULES, 3))
    return np.concatenate([t, w], axis=1)


def _rot(ax, ay, az):
    """Rotation matrices Rz(az) @ Ry(ay) @ Rx(ax), vectorised over leading axis."""
    cx, sx = np.cos(ax), np.sin(ax)
    cy, sy = np.cos(ay), np.sin(ay)
    cz, sz = np.cos(az), np.sin(az)
    one, zero = np.ones_like(ax), np.zeros_like(ax)
    rx = np.stack([np.stack([one, zero, zero], -1), np.stack([zero, cx, -sx], -1),
                   np.stack([zero, sx, cx], -1)], -2)
    ry = np.stack([np.stack([cy, zero, sy], -1), np.stack([zero, one, zero], -1),
                   np.stack([-sy, zero, cy], -1)], -2)
    rz = np.stack([np.stack([cz, -sz, zero], -1), np.stack([sz, cz, zero], -1),
                   np.stack([zero, zero, one], -1)], -2)
    return rz @ ry @ rx


_CHUNK = 2000


def _chunk(rng: np.random.Generator, rec: Recipe, n_ev: int, zasc: np.ndarray):
    # primary vertices per event
    if rec.pv_mode == "fixed":
        npv = np.full(n_ev, int(rec.pv_mean), dtype=np.int64)
    elif rec.pv_mode == "poisson":
        npv = rng.poisson(rec.pv_mean, size=n_ev)
    else:
        npv = rng.integers(rec.pv_lo, rec.pv_hi + 1, size=n_ev)
    n_pv_tot = int(npv.sum())
    pv_ev = np.repeat(np.arange(n_ev), npv)
    pvz = rng.normal(0.0, 60.0, size=n_pv_tot)
    pvx = rng.normal(0.0, 0.03, size=n_pv_tot)
    pvy = rng.normal(0.0, 0.03, size=n_pv_tot)
    nf = rng.poisson(rec.tracks_per_pv, size=n_pv_tot)
    nb = (rng.poisson(rec.tracks_per_pv * rec.backward_frac, size=n_pv_tot)
          if rec.backward_frac > 0 else np.zeros(n_pv_tot, dtype=np.int64))
    ntr_pv = nf + nb
    trk_pv = np.repeat(np.arange(n_pv_tot), ntr_pv)
    n_trk = trk_pv.shape[0]
    # direction: first nf of each vertex forward, the rest backward
    first = np.repeat(np.cumsum(ntr_pv) - ntr_pv, ntr_pv)
    rank = np.arange(n_trk) - first
    fwd = rank < np.repeat(nf, ntr_pv)
    eta = rng.uniform(2.0, 5.0, size=n_trk)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n_trk)
    theta = 2.0 * np.arctan(np.exp(-eta))
    tant = np.tan(theta)
    sgn = np.where(fwd, 1.0, -1.0)
    tx0 = tant * np.cos(phi)
    ty0 = tant * np.sin(phi)
    z0 = pvz[trk_pv]
    x0 = pvx[trk_pv]
    y0 = pvy[trk_pv]
    # path length along |z| where the straight line sits in the annulus, widened
    u_lo = R_MIN / tant - 3.0 * PITCH
    u_hi = R_MAX / tant + 3.0 * PITCH
    # candidate planes: ascending index range for forward, descending for backward
    zf_lo = np.where(fwd, z0 + np.maximum(u_lo, 1e-6), z0 - u_hi)
    zf_hi = np.where(fwd, z0 + u_hi, z0 - np.maximum(u_lo, 1e-6))
    k_lo = np.clip(np.ceil((zf_lo - Z_FIRST) / PITCH), 0, N_MODULES).astype(np.int64)
    k_hi = np.clip(np.floor((zf_hi - Z_FIRST) / PITCH), -1, N_MODULES - 1).astype(np.int64)
    nk = np.maximum(k_hi - k_lo + 1, 0)
    tot = int(nk.sum())
    el_trk = np.repeat(np.arange(n_trk), nk)
    el_first = np.repeat(np.cumsum(nk) - nk, nk)
    el_rank = np.arange(tot) - el_first
    # travel order: forward ascending z, backward descending z
    k = np.where(fwd[el_trk], k_lo[el_trk] + el_rank, k_hi[el_trk] - el_rank)
    zk = zasc[k]
    u = sgn[el_trk] * (zk - z0[el_trk])
    crossed = u > 0.0
    if rec.kink_sigma > 0:
        kx = rng.normal(0.0, rec.kink_sigma, size=tot) * crossed
        ky = rng.normal(0.0, rec.kink_sigma, size=tot) * crossed

        def excl_segsum(v):
            c = np.cumsum(v)
            c_before = c - v
            base = c_before[el_first]
            return c_before - base

        c1x, c2x = excl_segsum(kx), excl_segsum(kx * u)
        c1y, c2y = excl_segsum(ky), excl_segsum(ky * u)
    else:
        c1x = c2x = c1y = c2y = 0.0
    xt = x0[el_trk] + tx0[el_trk] * u + (u * c1x - c2x)
    yt = y0[el_trk] + ty0[el_trk] * u + (u * c1y - c2y)
    r = np.sqrt(xt * xt + yt * yt)
    keep = crossed & (r >= R_MIN) & (r <= R_MAX)
    keep &= rng.uniform(size=tot) < rec.hit_eff
    sx = rng.normal(0.0, rec.smear, size=tot)
    sy = rng.normal(0.0, rec.smear, size=tot)
    if rec.pairs:
        # one-sided planes: even planes see x >= 0, odd planes x < 0 (measured x)
        mx = xt + sx
        keep &= np.where(k % 2 == 0, mx >= 1.0e-3, mx <= -1.0e-3)
    hx = (xt + sx)[keep]
    hy = (yt + sy)[keep]
    hz = zk[keep]
    hk = k[keep]
    htrk = el_trk[keep]
    hev = pv_ev[trk_pv[htrk]]
    # noise hits
    n_sig_ev = np.bincount(hev, minlength=n_ev)
    n_noise = rng.poisson(rec.noise_frac * n_sig_ev)
    nn = int(n_noise.sum())
    nev = np.repeat(np.arange(n_ev), n_noise)
    nk_ = rng.integers(0, N_MODULES, size=nn)
    nr = np.sqrt(rng.uniform(R_MIN * R_MIN, R_MAX * R_MAX, size=nn))
    nphi = rng.uniform(0.0, 2.0 * math.pi, size=nn)
    nx = nr * np.cos(nphi)
    if rec.pairs:
        # noise on a one-sided plane lies on its side
        nx = np.where(nk_ % 2 == 0, 1.0, -1.0) * np.maximum(np.abs(nx), 1.0e-3)
    ax = np.concatenate([hx, nx])
    ay = np.concatenate([hy, nr * np.sin(nphi)])
    az = np.concatenate([hz, zasc[nk_]])
    ak = np.concatenate([hk, nk_])
    amc = np.concatenate([htrk, np.full(nn, -1, dtype=np.int64)])
    aev = np.concatenate([hev, nev])
    # shuffle within events: sort by (event, random key)
    order = np.argsort(aev + rng.uniform(0.0, 0.5, size=aev.shape[0]))
    counts = np.bincount(aev, minlength=n_ev)
    return (ax[order], ay[order], az[order], ak[order], amc[order], counts, n_trk)


def _chunk_job(args):
    rec, ci, n_ev = args
    rng = np.random.Generator(np.random.PCG64([rec.seed, ci]))
    x, y, z, k, mc, counts, n_trk = _chunk(rng, rec, n_ev, module_z_ascending())
    if rec.misalign:
        return (x, y, z, k.astype(np.int32), mc.astype(np.int32), counts, n_trk)
    return (x.astype(np.float32), y.astype(np.float32), z.astype(np.float32),
            k.astype(np.int32), mc.astype(np.int32), counts, n_trk)


def generate(rec: Recipe, workers: int | None = None) -> Events:
    """Draw rec.n_events events (deterministic for a given recipe).

    Chunks of events are independent random streams, so large batches are
    drawn by a pool of spawned worker processes; the result does not depend
    on the number of workers.
    """
    zasc = module_z_ascending()
    n_chunks = (rec.n_events + _CHUNK - 1) // _CHUNK
    jobs = [(rec, ci, min(_CHUNK, rec.n_events - ci * _CHUNK)) for ci in range(n_chunks)]
    if workers is None:
        import os
        workers = min(n_chunks, os.cpu_count() or 1, 32)
    if workers > 1 and n_chunks > 1:
        import concurrent.futures
        import multiprocessing
        with concurrent.futures.ProcessPoolExecutor(
                max_workers=workers, mp_context=multiprocessing.get_context("spawn")) as ex:
            parts = list(ex.map(_chunk_job, jobs))
    else:
        parts = [_chunk_job(j) for j in jobs]
    xs, ys, zs, ks, mcs, cnts = [], [], [], [], [], []
    n_part = 0
    for (x, y, z, k, mc, counts, n_trk) in parts:
        mcs.append(np.where(mc >= 0, mc + n_part, -1).astype(np.int32))
        n_part += n_trk
        xs.append(x); ys.append(y); zs.append(z); ks.append(k); cnts.append(counts)
    x = np.concatenate(xs) if xs else np.zeros(0, np.float32)
    y = np.concatenate(ys) if ys else np.zeros(0, np.float32)
    z = np.concatenate(zs) if zs else np.zeros(0, np.float32)
    k = np.concatenate(ks) if ks else np.zeros(0, dtype=np.int32)
    mc = np.concatenate(mcs) if mcs else np.zeros(0, dtype=np.int32)
    counts = np.concatenate(cnts) if cnts else np.zeros(0, dtype=np.int64)
    if rec.misalign and rec.pairs:
        raise ValueError("misalignment is defined for single planes only")
    if rec.misalign:
        # measured position = placement error applied inversely about the plane centre
        th = misalignment(rec.seed)
        R = _rot(th[:, 3], th[:, 4], th[:, 5])
        c = np.stack([np.zeros(N_MODULES), np.zeros(N_MODULES), zasc], -1)
        p = np.stack([x, y, z], -1).astype(np.float64) - c[k] - th[k, :3]
        p = np.einsum("nji,nj->ni", R[k], p) + c[k]
        x, y, z = p[:, 0], p[:, 1], p[:, 2]
    offsets = np.zeros(rec.n_events + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    if offsets[-1] >= 2**31:
        raise ValueError("batch exceeds int32 hit indexing")
    if rec.pairs:
        module = (N_PAIRS - 1 - k // 2).astype(np.int32)
        zp = module_z_ascending().reshape(N_PAIRS, 2)[::-1].astype(np.float32)
        return Events(x.astype(np.float32), y.astype(np.float32), z.astype(np.float32), module,
                      offsets.astype(np.int32), mc, n_part, zp[:, 0].copy(), zp[:, 1].copy())
    module = (N_MODULES - 1 - k).astype(np.int32)
    return Events(x.astype(np.float32), y.astype(np.float32), z.astype(np.float32), module,
                  offsets.astype(np.int32), mc, n_part, module_z_traversal())


def make_events(config: int, n_events: int | None = None, seed: int = 0,
                workers: int | None = None, pairs: bool = False) -> Events:
    r = recipe_for(config, n_events, seed)
    r.pairs = pairs
    return generate(r, workers)


def reverse_traversal(ev: Events) -> Events:
    """The same hits traversed in the opposite direction (ascending z, from
    behind the interaction region outwards): module id m becomes M - 1 - m
    and the plane positions are reversed."""
    M = int(ev.module_z.shape[0])
    return Events(ev.x, ev.y, ev.z, (M - 1 - ev.module).astype(np.int32), ev.event_offsets, ev.mc,
                  ev.n_particles, ev.module_z[::-1].copy(),
                  None if ev.module_z2 is None else ev.module_z2[::-1].copy())


def poisson_arrivals(rate_hz: float, n: int, seed: int = 0) -> np.ndarray:
    """Open-loop arrival times (seconds from 0) of n requests at a mean rate."""
    rng = np.random.Generator(np.random.PCG64([seed, 0xA77]))
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
