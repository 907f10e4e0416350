"""Throughput benchmark of the GB300 Search-by-triplet library.

A step reconstructs one batch of synthetic events (100k uneven events, pileup
U(1, 20), 200-12600 hits each; inputs larger than L2) through the batched C
entry point (persistent work-queue kernel replayed from a CUDA graph).  The
line also reports the plain one-block-per-event launch on the same batch;
the same batch traversed in ascending z (module order reversed), with the
global event cut (busiest 10% of events rejected) and with fp16 hit storage;
the end-to-end host entry point (copies inside the timed region); the
continuous-batching server under open-loop arrivals; the alignment adjoint;
the dominant kernel's HBM and issue roofline fractions (DRAM bytes and
instruction counts from the committed full-size ncu capture); the SM clocks
seen during the timed region; and the CPU oracle timed on host cores over a
bounded sample, whose tracks are compared with the GPU's event by event.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank reconstructs its own batch (independent events, no
collective on the data path) and rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2207_03936_gb300 import synth  # noqa: E402  (numpy only; no CUDA)

METRIC = "VELO events/s on 1 GB300, batched vs plain; p99 latency; track-set match"
SERVE_STREAMS, SERVE_BATCH = 4, 2048   # serving slots and largest batch (measured best)
BUNCH_EVENTS, BUNCH_STREAMS = 500, 8   # the paper's mode: n events per bunch, several streams
WORKLOAD = "uneven batch: 100k events, pileup U(1,20), Poisson(25)+10% backward tracks per vertex"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--events", type=int, default=100_000)
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--threads", type=int, default=0, choices=[0, 64, 128, 256],
                   help="search block size; 0 = autotuned on the batch")
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-direction", action="store_true",
                   help="skip the ascending-z traversal of the same batch")
    p.add_argument("--no-fp16", action="store_true",
                   help="skip the fp16 hit-storage run of the same batch")
    p.add_argument("--no-gec", action="store_true",
                   help="skip the global-event-cut run (busiest 10% of events rejected)")
    p.add_argument("--no-pairs", action="store_true",
                   help="skip the module-pair geometry run (one-sided planes paired into 26 modules)")
    p.add_argument("--serving-sweep", action="store_true",
                   help="sweep arrival rate (0.1-1.5x of saturation) and memory budget (2-16 GB)")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def code_digest(path):
    """sha256 of a C/CUDA source with its comments and whitespace removed:
    changes to the code change it, changes to the comments do not."""
    import re
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256(" ".join(text.split()).encode()).hexdigest()


def profiled(kernel, hits):
    """Counters of one launch of `kernel` (name<threads>, or a tuple of names
    for a step made of several kernels: their sum) scaled to a batch of
    `hits` hits from the committed ncu capture (profiles/traffic.json, one
    kernel per capture on a batch of a few GB): DRAM bytes read and written,
    warp instructions and thread instructions issued, per hit of the captured
    batch times `hits`.  None when a kernel has no counters or its code
    differs from the one the counters were taken on (comments and whitespace
    aside)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if code_digest(os.path.join(ROOT, d["source"])) != d["source_code_sha256"]:
        return None
    names = (kernel,) if isinstance(kernel, str) else tuple(kernel)
    keys = ("dram_read_bytes", "dram_write_bytes", "warp_inst", "thread_inst")
    r = dict.fromkeys(keys, 0.0)
    for name in names:
        k = d["kernels"].get(name)
        if k is None:
            return None
        for key in keys:
            r[key] += k[key] * hits / k["hits"]
        r["captured_hits"], r["captured_events"] = k["hits"], k.get("events")
    return r


def profiled_traffic(kernel, hits):
    """DRAM bytes of one launch of `kernel` (dram__bytes_read.sum +
    dram__bytes_write.sum per hit of the committed capture, times hits), or None."""
    k = profiled(kernel, hits)
    return None if k is None else k["dram_read_bytes"] + k["dram_write_bytes"]


def issue_roofline(kernel, hits, kernel_ms, sm_mhz, sm_count):
    """Warp-instruction issue rate of `kernel` against the SMs' issue peak
    (4 schedulers per SM, one warp instruction per scheduler per cycle, at
    the SM clock sampled during the timed region), and its SIMT efficiency
    (threads per warp instruction / 32, the divergence figure)."""
    k = profiled(kernel, hits)
    if k is None or not sm_mhz:
        return None
    achieved = k["warp_inst"] / (kernel_ms / 1e3) / 1e9
    peak = 4 * sm_count * sm_mhz / 1e3
    return {"warp_inst": k["warp_inst"], "achieved_ginst_s": achieved, "peak_ginst_s": peak,
            "frac": achieved / peak, "sm_mhz": sm_mhz,
            "simt_efficiency": k["thread_inst"] / (32.0 * k["warp_inst"])}


# the output step: canonical order and CSR starts, then hit lists and fits
OUTPUT_KERNELS = ("k_output", "k_fit")


def roofline_entry(threads, hits, hbm_gbs, peak, peak_kind, kms, sm_mhz, sm_count, sort_gbs, out_gbs):
    """The dominant kernel's roofline.  The search waits on load latency, so
    the binding roof is instruction issue: warp instructions per second of the
    live launch against 4 schedulers x SMs x the sampled SM clock (counters
    from the committed capture, scaled per hit).  Its algorithmic HBM
    fraction, DRAM traffic and SIMT efficiency stand beside it; without
    counters for the current code the HBM fraction is the roofline."""
    kname = f"k_search_persistent<{threads}>"
    iss = issue_roofline(kname, hits, kms[2], sm_mhz, sm_count)
    traffic = profiled_traffic(kname, hits)
    common = {"kernel": "k_search_persistent", "kernel_ms": kms[2],
              "hbm_achieved_gbs": hbm_gbs, "hbm_peak_gbs": peak, "hbm_frac": hbm_gbs / peak,
              "peak_kind": peak_kind, "traffic": traffic,
              "traffic_source": "ncu capture of one launch on a smaller batch, scaled per hit (profiles/traffic.json)",
              "kernel_ms_all": {"order": kms[0], "sort": kms[1], "search": kms[2], "scan": kms[3], "output": kms[4]},
              "sort_kernel": {"achieved_gbs": sort_gbs, "frac": sort_gbs / peak,
                              "traffic": profiled_traffic("k_sort", hits),
                              "issue": issue_roofline("k_sort", hits, kms[1], sm_mhz, sm_count)},
              "output_kernel": {"kernels": list(OUTPUT_KERNELS), "achieved_gbs": out_gbs,
                                "frac": out_gbs / peak, "traffic": profiled_traffic(OUTPUT_KERNELS, hits),
                                "issue": issue_roofline(OUTPUT_KERNELS, hits, kms[4], sm_mhz, sm_count)}}
    if iss is not None:
        return {"bound": "issue", "achieved": iss["achieved_ginst_s"], "peak": iss["peak_ginst_s"],
                "unit": "G warp instructions/s", "frac": iss["frac"],
                "simt_efficiency": iss["simt_efficiency"], "warp_inst": iss["warp_inst"], **common}
    return {"bound": "hbm", "achieved": hbm_gbs, "peak": peak, "unit": "GB/s", "frac": hbm_gbs / peak,
            **common}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (read-only)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def serve(sbt, srv, ev, rate_hz, budget_bytes, timeout=120.0):
    """Open-loop Poisson arrivals at rate_hz into a running request loop.
    Latency runs from each event's scheduled arrival to its result on the
    host (both on the server's clock); events/s = completions over the span
    from the first arrival to the last completion on that clock.  The host
    loop that collects the results adds its own polling delay, so its wall
    span is reported beside it."""
    st0 = srv.stats()
    if rate_hz is None:
        arrival = np.zeros(ev.n_events)
    else:
        arrival = synth.poisson_arrivals(rate_hz, ev.n_events, seed=11)
    srv.submit_schedule(ev, arrival, first_id=0)  # copies the batch first; arrivals count from here
    t0 = time.perf_counter()
    ids, lat = [], []
    n_done = 0
    while n_done < ev.n_events and time.perf_counter() - t0 < timeout:
        i, _, l = srv.drain(65536, timeout_s=0.01)
        ids.append(i.copy())
        lat.append(l.copy())
        n_done += len(l)
    wall = time.perf_counter() - t0
    ids = np.concatenate(ids) if ids else np.zeros(0, np.int64)
    lat = np.concatenate(lat) if lat else np.zeros(0)
    st = srv.stats()
    span = float((arrival[ids] + lat).max() - arrival.min()) if len(lat) else 0.0
    nb = st["batches"] - st0["batches"]
    mean_batch = ((st["mean_batch_events"] * st["batches"] - st0["mean_batch_events"] * st0["batches"]) / nb
                  if nb > 0 else 0.0)
    pct = (lambda q: float(np.percentile(lat, q) * 1e3) if len(lat) else None)
    # where a batch's time went: uploads, kernels and downloads on its slot's
    # stream (CUDA events), and enqueue to harvest on the host clock
    nt = st.get("timed_batches", 0) - st0.get("timed_batches", 0)
    per_batch = ({k: (st[k] - st0[k]) / nt for k in ("upload_ms", "kernel_ms", "download_ms", "batch_wall_ms")}
                 if nt > 0 else None)
    return {"offered_hz": rate_hz, "events": int(len(lat)), "value": len(lat) / span if span > 0 else None,
            "unit": "events/s", "p50_ms": pct(50), "p99_ms": pct(99),
            "max_ms": float(lat.max() * 1e3) if len(lat) else None,
            "span_ms": span * 1e3, "host_wall_ms": wall * 1e3,
            "budget_gb": budget_bytes / 2**30, "mean_batch_events": mean_batch,
            "generator_max_lag_ms": st["feed_lag_s"] * 1e3,
            "launcher_busy_fraction": (st["launch_busy_s"] - st0["launch_busy_s"]) / span if span > 0 else None,
            "peak_inflight_gb_server_lifetime": st["peak_bytes"] / 2**30,
            "per_batch_ms": per_batch}


def cpu_baseline(ev, budget_s: float, gpu_out=None):
    """The oracle on all host cores over a bounded sample of the workload's
    events; optionally compares its tracks with the GPU's for those events."""
    import oracle
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(1)
    order = rng.permutation(ev.n_events)
    done, t_total, n_match, n_cmp = 0, 0.0, 0, 0
    chunk = 500
    while done < ev.n_events and t_total < budget_s:
        idx = np.sort(order[done:done + chunk])
        sub_off = [0]
        xs, ys, zs, ms = [], [], [], []
        for e in idx:
            lo, hi = ev.event_offsets[e], ev.event_offsets[e + 1]
            xs.append(ev.x[lo:hi]); ys.append(ev.y[lo:hi]); zs.append(ev.z[lo:hi]); ms.append(ev.module[lo:hi])
            sub_off.append(sub_off[-1] + hi - lo)
        x, y, z, m = (np.concatenate(a) for a in (xs, ys, zs, ms))
        sub_off = np.array(sub_off, np.int32)
        t0 = time.perf_counter()
        r = oracle.reconstruct(x, y, z, m, sub_off, ev.module_z, n_threads=cores, module_z2=ev.module_z2)
        t_total += time.perf_counter() - t0
        if gpu_out is not None:
            to, ho, th, prm = (gpu_out["track_offsets"], gpu_out["hit_offsets"], gpu_out["track_hits"],
                               gpu_out["params"])
            for j, e in enumerate(idx):
                g0, g1 = to[e], to[e + 1]
                o0, o1 = r.track_offsets[j], r.track_offsets[j + 1]
                gh = th[ho[g0]:ho[g1]] - ev.event_offsets[e]
                oh = r.track_hits[r.hit_offsets[o0]:r.hit_offsets[o1]] - sub_off[j]
                same = (g1 - g0 == o1 - o0 and np.array_equal(gh, oh)
                        and np.array_equal(prm[g0:g1].view(np.uint32), r.params[o0:o1].view(np.uint32)))
                n_match += int(same)
                n_cmp += 1
        done += len(idx)
    res = {"value": done / t_total, "unit": "events/s", "cores": cores, "kind": "oracle",
           "sample": f"{done} events drawn at random from the workload, {t_total:.1f} s wall on {cores} threads"}
    match = {"events_compared": n_cmp, "bit_exact_events": n_match} if gpu_out is not None else None
    return res, match


def per_event_launch(sbt, h, ev, a, b, stream):
    """One sbt_reconstruct call per event, back to back on one stream, timed
    with CUDA events; every event's tracks are compared with the batched
    result of the same events."""
    import torch
    dev = [torch.from_numpy(x).cuda() for x in (ev.x, ev.y, ev.z, ev.module)]
    offs = [torch.tensor([0, int(ev.event_offsets[e + 1] - ev.event_offsets[e])], dtype=torch.int32,
                         device="cuda") for e in range(ev.n_events)]
    sl = [slice(int(ev.event_offsets[e]), int(ev.event_offsets[e + 1])) for e in range(ev.n_events)]
    outs = [sbt.TrackOutput.allocate(1, sl[e].stop - sl[e].start) for e in range(ev.n_events)]

    def run():
        for e in range(ev.n_events):
            sbt.sbt_reconstruct(h, *(d[sl[e]] for d in dev), offs[e], out=outs[e])
    run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a.record(stream)
    run()
    b.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = a.elapsed_time(b)
    whole = sbt.sbt_reconstruct_batched(h, *dev, torch.from_numpy(ev.event_offsets).cuda()).compact()
    same = 0
    for e in range(ev.n_events):
        g = outs[e].compact()
        t0_, t1_ = whole["track_offsets"][e], whole["track_offsets"][e + 1]
        hits = whole["track_hits"][whole["hit_offsets"][t0_]:whole["hit_offsets"][t1_]] - ev.event_offsets[e]
        same += int(np.array_equal(g["track_hits"], hits)
                    and np.array_equal(g["params"].view(np.uint32), whole["params"][t0_:t1_].view(np.uint32)))
    return {"value": ev.n_events / (ms / 1e3), "unit": "events/s", "events": ev.n_events,
            "workload": "upgrade-condition events (config 2), one call per event", "device_ms": ms,
            "host_wall_ms": wall * 1e3, "identical_to_batched_events": same}


def bunched_launch(sbt, ev, dev, nmax, threads, ref):
    """Bunches of BUNCH_EVENTS consecutive events, one plain launch each,
    spread round-robin over BUNCH_STREAMS streams with a handle per stream;
    timed with CUDA events from the first launch to the last completion."""
    import torch
    hs = [sbt.sbt_create(ev.module_z, sbt.default_config(max_hits_per_event=nmax, threads_per_block=threads))
          for _ in range(BUNCH_STREAMS)]
    streams = [torch.cuda.Stream() for _ in range(BUNCH_STREAMS)]
    bun = []
    for b0 in range(0, ev.n_events, BUNCH_EVENTS):
        b1 = min(ev.n_events, b0 + BUNCH_EVENTS)
        lo, hi = int(ev.event_offsets[b0]), int(ev.event_offsets[b1])
        off = torch.from_numpy((ev.event_offsets[b0:b1 + 1] - lo).astype(np.int32)).cuda()
        bun.append((slice(lo, hi), off, sbt.TrackOutput.allocate(b1 - b0, hi - lo), b0, b1))
    main = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    done = [torch.cuda.Event() for _ in streams]

    def run(timed):
        if timed:
            start.record(main)
        for s in streams:
            s.wait_stream(main)
        for k, (sl, off, out, _, _) in enumerate(bun):
            i = k % BUNCH_STREAMS
            sbt.sbt_reconstruct(hs[i], *(d[sl] for d in dev[:4]), off, out=out, stream=streams[i])
        for s, d in zip(streams, done):
            d.record(s)
            main.wait_event(d)
        if timed:
            end.record(main)
    try:
        run(False)
        torch.cuda.synchronize()
        run(True)
        torch.cuda.synchronize()
        ms = start.elapsed_time(end)
        # a sample of bunches against the batched result
        same = 0
        for sl, off, out, b0, b1 in bun[::max(1, len(bun) // 8)]:
            g = out.compact()
            t0_, t1_ = ref["track_offsets"][b0], ref["track_offsets"][b1]
            h0, h1 = ref["hit_offsets"][t0_], ref["hit_offsets"][t1_]
            same += int(np.array_equal(g["track_hits"], ref["track_hits"][h0:h1] - sl.start))
        n_checked = len(bun[::max(1, len(bun) // 8)])
    finally:
        for x in hs:
            x.close()
    return {"value": ev.n_events / (ms / 1e3), "unit": "events/s", "ms_per_step": ms,
            "events_per_bunch": BUNCH_EVENTS, "streams": BUNCH_STREAMS, "bunches": len(bun),
            "bunches_checked": n_checked, "bunches_identical_to_batched": same}


def job_throughput(ms_local: float, events_local: int, ws: int, pg=None, device="cpu"):
    """Whole-job rate when every one of ws ranks reconstructs its own batch of
    events_local events: the step time is the maximum over the ranks (one
    all-reduce through pg when there is more than one), the value the events
    of all ranks over that time.  Returns (ms_max, events/s)."""
    import torch
    ms_max = float(ms_local)
    if pg is not None:
        t = torch.tensor([ms_max], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms_max = float(t.item())
    return ms_max, events_local * ws / (ms_max / 1e3)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    ev = synth.make_events(3, args.events)
    per_step, step_ms = [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res, _ = cpu_baseline(ev, args.cpu_seconds / max(args.steps, 1))
        if s >= args.warmup:
            per_step.append(res["value"])
            step_ms.append((time.perf_counter() - t0) * 1e3)
    v = float(np.mean(per_step))
    res["value"] = v
    # a step is one bounded sample of the workload (cpu_baseline.sample says how large)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "events/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "events": ev.n_events, "hits": ev.n_hits},
            "cpu_baseline": res,
            "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    # inputs are drawn before any CUDA call (the generator uses spawned workers)
    ev = synth.make_events(3, args.events, seed=rank)
    ev_adj = None if args.no_adjoint else synth.make_events(5)
    ev_srv = None if args.no_serving else synth.make_events(4, 40_000, seed=7)
    ev_pairs = None if args.no_pairs else synth.make_events(3, args.events, seed=rank, pairs=True)
    ev_pe = None if args.no_plain else synth.make_events(2, 1000, seed=rank)

    import torch
    from paper_2207_03936_gb300 import sbt
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()

    dev = [torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z, ev.module, ev.event_offsets)]
    # per-event capacity sized to the batch (shared memory per block scales with it)
    nmax = int(-(-int(np.diff(ev.event_offsets).max()) // 1024) * 1024)
    h = sbt.sbt_create(ev.module_z, sbt.default_config(max_hits_per_event=nmax))
    if args.threads:
        h.close()
        h = sbt.sbt_create(ev.module_z, sbt.default_config(max_hits_per_event=nmax,
                                                           threads_per_block=args.threads))
        threads = args.threads
        per_sm = 0
    else:
        threads, per_sm = sbt.sbt_autotune(h, *dev)
    out = sbt.TrackOutput.allocate(ev.n_events, ev.n_hits)
    stream = torch.cuda.current_stream()

    def tuned(handle):
        """Derived handles (other traversal, storage, cut or geometry) take the tuned shape."""
        if per_sm:
            sbt.sbt_set_launch_shape(handle, threads, per_sm)
        return handle
    for _ in range(args.warmup):
        sbt.sbt_reconstruct_batched(h, *dev, out=out)
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    launches = 0
    for _ in range(args.steps):
        sbt.sbt_reconstruct_batched(h, *dev, out=out)
        launches += h.last_launch_count()
    b.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = a.elapsed_time(b) / args.steps
    ms_max, value = job_throughput(ms, ev.n_events, ws, pg, "cuda")
    gpu_res = out.compact()
    counts = gpu_res["counts"]

    # per-kernel times (no graph, CUDA events on the launching stream)
    kms = sbt.sbt_profile_batched(h, *dev, out, reps=3)
    T, H = int(counts[0]), int(counts[1])
    # algorithmic bytes of the dominant kernel (the persistent search): sorted
    # hits in (float4 coordinates and phi16: 18 B per hit), module offsets and
    # event offsets; staged track hit records (16 B per track hit), per-track
    # smallest index and placement (8 B per track) and per-event counts out
    alg_bytes = (18 * ev.n_hits + 4 * (ev.n_events + 1) + 4 * 53 * ev.n_events
                 + 16 * H + 8 * T + 12 * ev.n_events)
    # the output step (output and fit kernels) reads the staged records and
    # per-track entries and writes the CSR arrays (track hits 4 B, offsets,
    # fits, chi2, ndof 28 B per track)
    out_bytes = 16 * H + 8 * T + 16 * ev.n_events + 4 * H + 28 * T
    out_gbs = out_bytes / (kms[4] / 1e3) / 1e9
    peak, peak_kind = peaks()
    achieved = alg_bytes / (kms[2] / 1e3) / 1e9
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz")
    # the sort kernel streams the inputs (16 B per hit) and writes the sorted hits (18 B per hit)
    sort_bytes = 16 * ev.n_hits + 4 * (ev.n_events + 1) + 18 * ev.n_hits + 4 * 54 * ev.n_events
    sort_gbs = sort_bytes / (kms[1] / 1e3) / 1e9

    # end to end through the host entry point (pinned host buffers)
    host_in = [torch.from_numpy(a).pin_memory() for a in (ev.x, ev.y, ev.z, ev.module, ev.event_offsets)]
    hout = sbt.TrackOutput.allocate(ev.n_events, ev.n_hits, pin_memory=True)
    for _ in range(2):
        sbt.sbt_reconstruct_host(h, *host_in, out=hout)
    n_e2e = max(1, min(args.steps, 5))   # mean over the calls (host-link stalls hit single calls)
    barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        sbt.sbt_reconstruct_host(h, *host_in, out=hout)
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e_ms_max, e2e_value = job_throughput(e2e_s * 1e3, ev.n_events, ws, pg, "cuda")
    h2d = 16 * ev.n_hits + 4 * (ev.n_events + 1)
    d2h = 16 + 4 * (ev.n_events + 1) + 4 * ev.n_events + 4 * (T + 1) + 4 * H + 24 * T
    e2e = {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms_max}
    del hout, host_in

    plain = None
    if not args.no_plain:
        pout = sbt.TrackOutput.allocate(ev.n_events, ev.n_hits)
        sbt.sbt_reconstruct(h, *dev, out=pout)
        torch.cuda.synchronize()
        a.record(stream)
        n_plain = max(1, min(args.steps, 3))
        for _ in range(n_plain):
            sbt.sbt_reconstruct(h, *dev, out=pout)
        b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b) / n_plain
        same = all(np.array_equal(v, pout.compact()[k]) for k, v in gpu_res.items())
        plain = {"value": ev.n_events / (pms / 1e3), "unit": "events/s", "ms_per_step": pms,
                 "identical_to_batched": bool(same)}
        del pout

    # the plain per-event launch: one sbt_reconstruct call per event of 1000
    # upgrade-condition events, back to back on one stream (what batching and
    # the persistent queue are measured against)
    per_event = None
    if ev_pe is not None:
        per_event = per_event_launch(sbt, h, ev_pe, a, b, stream)

    # bunches of BUNCH_EVENTS events of the same batch on BUNCH_STREAMS streams,
    # one handle per stream, one plain launch per bunch (the paper's n events
    # per bunch and several streams)
    bunches = None
    if not args.no_plain:
        bunches = bunched_launch(sbt, ev, dev, nmax, threads, gpu_res)
        torch.cuda.empty_cache()

    # the same batch traversed in ascending z: module ids and planes reversed
    ascending = None
    if not args.no_direction:
        M = len(ev.module_z)
        dev_asc = list(dev)
        dev_asc[3] = (M - 1 - dev[3]).to(torch.int32)
        ha = tuned(sbt.sbt_create(ev.module_z[::-1].copy(),
                                  sbt.default_config(max_hits_per_event=nmax, threads_per_block=threads)))
        aout = sbt.TrackOutput.allocate(ev.n_events, ev.n_hits)
        for _ in range(max(1, min(args.warmup, 2))):
            sbt.sbt_reconstruct_batched(ha, *dev_asc, out=aout)
        torch.cuda.synchronize()
        n_asc = max(1, min(args.steps, 3))
        a.record(stream)
        for _ in range(n_asc):
            sbt.sbt_reconstruct_batched(ha, *dev_asc, out=aout)
        b.record(stream)
        torch.cuda.synchronize()
        ams = a.elapsed_time(b) / n_asc
        ascending = {"value": ev.n_events / (ams / 1e3), "unit": "events/s", "ms_per_step": ams,
                     "tracks": int(aout.counts[0].item()), "tracks_descending": T}
        ha.close()
        del aout, dev_asc
        torch.cuda.empty_cache()

    # fp16 hit storage (x, y, z rounded to fp16, 8 bytes per sorted hit)
    fp16 = None
    if not args.no_fp16:
        hh = tuned(sbt.sbt_create(ev.module_z, sbt.default_config(max_hits_per_event=nmax,
                                                                  threads_per_block=threads, fp16_hits=1)))
        hout = sbt.TrackOutput.allocate(ev.n_events, ev.n_hits)
        for _ in range(max(1, min(args.warmup, 2))):
            sbt.sbt_reconstruct_batched(hh, *dev, out=hout)
        torch.cuda.synchronize()
        n_h = max(1, min(args.steps, 3))
        a.record(stream)
        for _ in range(n_h):
            sbt.sbt_reconstruct_batched(hh, *dev, out=hout)
        b.record(stream)
        torch.cuda.synchronize()
        hms = a.elapsed_time(b) / n_h
        hk = sbt.sbt_profile_batched(hh, *dev, hout, reps=2)
        fp16 = {"value": ev.n_events / (hms / 1e3), "unit": "events/s", "ms_per_step": hms,
                "speedup": ms / hms, "tracks": int(hout.counts[0].item()), "tracks_fp32": T,
                "kernel_ms": {"sort": hk[1], "search": hk[2]},
                "search_traffic": profiled_traffic(f"k_search_persistent_fp16<{threads}>", ev.n_hits)}
        hh.close()
        del hout
        torch.cuda.empty_cache()

    # module-pair geometry: the same pileup with one-sided planes paired into
    # 26 modules (half the hits per event); the oracle's pair reading checks
    # a sample of the events
    pairs, pairs_res = None, None
    if ev_pairs is not None:
        devp = [torch.from_numpy(a).cuda() for a in (ev_pairs.x, ev_pairs.y, ev_pairs.z,
                                                     ev_pairs.module, ev_pairs.event_offsets)]
        nmaxp = int(-(-int(np.diff(ev_pairs.event_offsets).max()) // 1024) * 1024)
        hp = tuned(sbt.sbt_create(ev_pairs.module_z,
                                  sbt.default_config(max_hits_per_event=nmaxp, threads_per_block=threads),
                                  module_z2=ev_pairs.module_z2))
        pout = sbt.TrackOutput.allocate(ev_pairs.n_events, ev_pairs.n_hits)
        for _ in range(max(1, min(args.warmup, 2))):
            sbt.sbt_reconstruct_batched(hp, *devp, out=pout)
        torch.cuda.synchronize()
        n_p = max(1, min(args.steps, 3))
        a.record(stream)
        for _ in range(n_p):
            sbt.sbt_reconstruct_batched(hp, *devp, out=pout)
        b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b) / n_p
        pk = sbt.sbt_profile_batched(hp, *devp, pout, reps=2)
        pairs_res = pout.compact()
        pairs = {"value": ev_pairs.n_events / (pms / 1e3), "unit": "events/s", "ms_per_step": pms,
                 "events": ev_pairs.n_events, "hits": ev_pairs.n_hits,
                 "tracks": int(pairs_res["counts"][0]), "kernel_ms": {"sort": pk[1], "search": pk[2]}}
        hp.close()
        del pout, devp
        torch.cuda.empty_cache()

    # global event cut: the busiest 10% of events rejected unreconstructed;
    # throughput over all input events, physics traded on a truth sample
    gec = None
    if not args.no_gec:
        from paper_2207_03936_gb300 import validation
        sizes = np.diff(ev.event_offsets)
        thr = int(np.quantile(sizes, 0.9))
        hg = tuned(sbt.sbt_create(ev.module_z, sbt.default_config(max_hits_per_event=nmax,
                                                                  threads_per_block=threads, gec_max_hits=thr)))
        gout = sbt.TrackOutput.allocate(ev.n_events, ev.n_hits)
        for _ in range(max(1, min(args.warmup, 2))):
            sbt.sbt_reconstruct_batched(hg, *dev, out=gout)
        torch.cuda.synchronize()
        n_gec = max(1, min(args.steps, 3))
        a.record(stream)
        for _ in range(n_gec):
            sbt.sbt_reconstruct_batched(hg, *dev, out=gout)
        b.record(stream)
        torch.cuda.synchronize()
        gms = a.elapsed_time(b) / n_gec
        K = min(2000, ev.n_events)

        def sample_indicators(res):
            to, ho = res["track_offsets"], res["hit_offsets"]
            tk = int(to[K])
            return validation.indicators(ho[:tk + 1], res["track_hits"][:int(ho[tk])],
                                         ev.mc[:int(ev.event_offsets[K])], ev.n_particles)
        gres = gout.compact()
        base_ind, cut_ind = sample_indicators(gpu_res), sample_indicators(gres)
        keep = sizes <= thr
        gec = {"max_hits": thr, "kept_events": int(keep.sum()),
               "kept_hits_fraction": float(sizes[keep].sum() / sizes.sum()),
               "value": ev.n_events / (gms / 1e3), "unit": "input events/s", "ms_per_step": gms,
               "speedup": ms / gms, "tracks": int(gres["counts"][0]),
               "sample": {"events": K, "efficiency_without_cut": base_ind["efficiency"],
                          "efficiency_with_cut": cut_ind["efficiency"],
                          "fake_fraction_with_cut": cut_ind["fake_fraction"],
                          "clone_fraction_with_cut": cut_ind["clone_fraction"]}}
        hg.close()
        del gout, gres
        torch.cuda.empty_cache()

    adj = None
    if ev_adj is not None:
        ad = [torch.from_numpy(a).cuda() for a in (ev_adj.x, ev_adj.y, ev_adj.z, ev_adj.module,
                                                     ev_adj.event_offsets)]
        r = sbt.sbt_reconstruct_batched(h, *ad)
        rc = r.compact()
        ho = torch.from_numpy(rc["hit_offsets"]).cuda()
        th = torch.from_numpy(rc["track_hits"]).cuda()
        align = torch.zeros(52, 6, dtype=torch.float64, device="cuda")
        sbt.sbt_fit_adjoint(h, ad[0], ad[1], ad[2], ad[3], ho, th, align)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            sbt.sbt_fit_adjoint(h, ad[0], ad[1], ad[2], ad[3], ho, th, align)
        b.record(stream)
        torch.cuda.synchronize()
        ams = a.elapsed_time(b) / args.steps
        adj = {"value": ev_adj.n_events / (ams / 1e3), "unit": "events/s", "ms_per_step": ams,
               "events": ev_adj.n_events, "tracks": int(rc["counts"][0]), "dtype": "f64"}
    serving = None
    if ev_srv is not None:
        # one long-lived server per memory budget (SERVE_STREAMS stream slots,
        # batches of at most SERVE_BATCH events), warmed up by one schedule
        # before anything is timed; offered rates are fractions of the
        # all-at-once rate at the 8 GB budget
        rates = [0.1, 0.5, 0.9, 1.3] if not args.serving_sweep else [0.1, 0.3, 0.5, 0.7, 0.9, 1.1, 1.3, 1.5]
        budgets = [2 << 30, 16 << 30] if not args.serving_sweep else [2 << 30, 4 << 30, 8 << 30, 16 << 30]
        servers = {}

        def server(b):
            if b not in servers:
                servers[b] = sbt.Server(h, b, SERVE_STREAMS, SERVE_BATCH)
                serve(sbt, servers[b], ev_srv, None, b)  # warm-up: buffers and pools reach size
            return servers[b]
        try:
            # all events at once, five times: the host-to-device copies share the
            # host with other work (slow in bursts), so the median run stands
            # for saturation
            sats = [serve(sbt, server(8 << 30), ev_srv, None, 8 << 30) for _ in range(5)]
            sat = sorted(sats, key=lambda r: r["value"])[2]
            at9 = serve(sbt, server(8 << 30), ev_srv, 0.9 * sat["value"], 8 << 30)
            runs = [serve(sbt, server(b), ev_srv, f * sat["value"], b) for b in budgets for f in rates]
        finally:
            for v in servers.values():
                v.close()
        serving = {"workload": "upgrade-condition events, open-loop Poisson arrivals",
                   "server": f"long-lived, {SERVE_STREAMS} stream slots, batches of at most {SERVE_BATCH} "
                             "events, warmed up by one schedule of the same events",
                   "saturation": sat, "at_0.9x": at9, "runs": runs,
                   "saturation_runs": [{"value": r["value"], "p99_ms": r["p99_ms"],
                                        "upload_ms_per_batch": (r["per_batch_ms"] or {}).get("upload_ms")}
                                       for r in sats],
                   "p99_ms_at_0.9x": at9["p99_ms"]}
    h.close()

    if rank == 0:
        cpu, match = cpu_baseline(ev, args.cpu_seconds, gpu_res)
        if pairs is not None:
            _, pairs["match"] = cpu_baseline(ev_pairs, min(args.cpu_seconds, 2.0), pairs_res)
        line = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "events": ev.n_events, "hits": ev.n_hits,
                       "hits_per_event_max": int(np.diff(ev.event_offsets).max()),
                       "tracks": T, "threads_per_block": threads, "blocks_per_sm": per_sm or None,
                       "l2": "inputs larger than L2 (no flush needed)"},
            "plain": plain,
            "plain_per_event": per_event,
            "batched_over_plain_per_event": (value / per_event["value"]) if per_event else None,
            "bunches": bunches,
            "ascending": ascending,
            "gec": gec,
            "fp16_hits": fp16,
            "module_pairs": pairs,
            "serving": serving,
            "match": match,
            "adjoint": adj,
            "e2e": e2e,
            "roofline": roofline_entry(threads, ev.n_hits, achieved, peak, peak_kind, kms, sm_mhz, sm_count,
                                       sort_gbs, out_gbs),
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
