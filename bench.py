"""Throughput benchmark of batched p-FHT-FSCL-L-P decoding on GB300.

One step = one rmdec_decode call over a batch of synthetic RM(2,9) frames (BPSK over AWGN at
Eb/N0 = 2.25 dB, where the P=20, L=4 decoder's FER is about 1e-4), with the LLRs resident in
HBM. Prints one JSON line (see the keys below). ``--impl reference`` times the CPU oracle on
the host cores instead (the reference arm of this method: there is no other implementation).

Under torchrun (N > 1 GPUs) every rank decodes its own batch (frames shard with no data-path
exchange: weak scaling); rank 0 prints the whole-job throughput from the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2108_12550_gb300 import inputs as I  # noqa: E402
from paper_2108_12550_gb300 import opcount  # noqa: E402
from paper_2108_12550_gb300 import replicas  # noqa: E402

WORKLOADS = {
    # name: (m, r, P, L, EbN0 dB, frames per step)
    "rm29_p20_l4": (9, 2, 20, 4, 2.25, 1 << 18),
    "rm27_p8_l4": (7, 2, 8, 4, 3.0, 1 << 20),
    "rm25_p4_l2": (5, 2, 4, 2, 3.0, 1 << 21),
    "rm39_p16_l8": (9, 3, 16, 8, 4.0, 1 << 16),
    "rm39_p20_l4": (9, 3, 20, 4, 3.0, 1 << 17),  # the serving mix's costliest code
    "rm28_p8_l4": (8, 2, 8, 4, 3.0, 1 << 19),  # a serving-mix code
}
METRIC = "frames/s RM(2,9) P=20 L=4 at FER~1e-4 Eb/N0; p50/p99 latency, mixed load"
# DRAM bytes per frame of one ncu capture per (workload, LLR type), valid only for the kernel
# that decodes the workload's launches and the code it was taken on (the prefix of
# kernel_fingerprint() of that kernel's source): pfht_kernel<9,2,4> on 16,384 FP32 frames
# (33,641,728 B read + 0 B written), ppt_kernel<7,2,4> on 65,536 INT8 frames (8,531,200 B read
# + 0 B written)
TRAFFIC = {
    ("rm29_p20_l4", "f32"): {"kernel": "warp", "source": "pfht_kernel.cuh",
                             "bytes_per_frame": (33641728 + 0) / 16384, "kernel_code_sha256": "4e5d0ffbfdf3aa35"},
    ("rm27_p8_l4", "i8"): {"kernel": "path", "source": "ppt_kernel.cuh",
                           "bytes_per_frame": (8531200 + 0) / 65536, "kernel_code_sha256": "91ef0b69b44bb38c"},
}
LANES_PER_SM = 128  # INT32/FP32 lanes per SM: one ALU operation per lane per clock


def kernel_fingerprint(source="pfht_kernel.cuh"):
    """sha256 of a kernel source with comments and blank lines removed: a capture stays
    valid across comment edits and goes stale on any code change."""
    import hashlib

    with open(os.path.join(ROOT, "paper_2108_12550_gb300", "csrc", source)) as fh:
        code = re.sub(r"//[^\n]*", "", fh.read())
    code = "\n".join(line.strip() for line in code.splitlines() if line.strip())
    return hashlib.sha256(code.encode()).hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def _frames(m, r, nf, ebn0, seed, chunk=1 << 16):
    """Seeded BPSK/AWGN frames (FP32 LLRs) and their messages, generated in chunks."""
    return I.make_frames_chunked(m, r, nf, ebn0, seed, chunk)


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def cpu_baseline(m, r, P, L, ebn0, n_frames, seed=3):
    """Times the CPU oracle (all host cores) on a bounded sample of the same workload."""
    import oracle

    llr, _ = _frames(m, r, n_frames, ebn0, seed)
    perms = I.perm_table(m, r, P, L, seed=1)
    cores = os.cpu_count() or 1
    oracle.decode(m, r, P, L, perms, llr[: min(64, n_frames)].astype(np.float64), want_margin=False)
    t0 = time.perf_counter()
    oracle.decode(m, r, P, L, perms, llr.astype(np.float64), n_threads=cores, want_margin=False)
    dt = time.perf_counter() - t0
    return {"value": n_frames / dt, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_frames} frames of the same workload (FP64 oracle, {cores} threads)"}


def run_reference(args, wl):
    m, r, P, L, ebn0, _ = wl
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = args.ref_frames
    import oracle

    llr, _ = _frames(m, r, per_step, ebn0, seed=5)
    perms = I.perm_table(m, r, P, L, seed=1)
    y = llr.astype(np.float64)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.decode(m, r, P, L, perms, y[: max(1, per_step // 8)], n_threads=cores, want_margin=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.decode(m, r, P, L, perms, y, n_threads=cores, want_margin=False)
    dt = time.perf_counter() - t0
    v = per_step * args.steps / dt
    line = {"metric": METRIC, "value": v, "unit": "frames/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "m": m, "r": r, "P": P, "L": L,
                                            "ebn0_db": ebn0, "frames_per_step": per_step},
            "cpu_baseline": {"value": v, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} frames per step, FP64 oracle on {cores} host threads"},
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class ServingMix:
    """The serving mix: Poisson arrivals (rate per second) of requests drawn uniformly over 16
    decoder configurations (RM(2,7), RM(2,8), RM(2,9), RM(3,9) x P in {8, 20} x INT8/FP32 LLRs,
    L = 4), each of 1-4096 frames (log-uniform) at an Eb/N0 drawn uniformly from 2-5 dB (four
    1-dB buckets of pre-generated frames per code, pinned host memory)."""

    POOL = 4096

    def __init__(self, n_req, rate, seed=7):
        import torch

        import paper_2108_12550_gb300 as pkg

        codes = [(7, 2), (8, 2), (9, 2), (9, 3)]
        self.cfgs = [(m, r, P, 4, dt) for (m, r) in codes for P in (8, 20) for dt in ("i8", "f32")]
        self.decs = [pkg.Decoder(m, r, P, L, perm_seed=1 + i, dtype=dt) for i, (m, r, P, L, dt) in enumerate(self.cfgs)]
        rng = np.random.default_rng(seed)
        pools = {}  # (code, dtype, Eb/N0 bucket) -> pinned LLRs
        for ci_code, (m, r) in enumerate(codes):
            for bi, eb in enumerate((2.0, 3.0, 4.0, 5.0)):
                llr, _ = _frames(m, r, self.POOL, eb, seed=1000 + ci_code * 10 + bi, chunk=self.POOL)
                pools[(m, r, "f32", bi)] = torch.from_numpy(np.ascontiguousarray(llr)).pin_memory()
                pools[(m, r, "i8", bi)] = torch.from_numpy(np.ascontiguousarray(I.quantize_i8(llr))).pin_memory()
        self.pools = pools
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
        self.trace = []
        for q in range(n_req):
            ci = int(rng.integers(len(self.cfgs)))
            m, r, _, _, dt = self.cfgs[ci]
            nf = int(np.exp(rng.uniform(0.0, np.log(4096))))
            bi = min(3, int(rng.uniform(2.0, 5.0) - 2.0))
            off = int(rng.integers(0, self.POOL - nf + 1))
            x = pools[(m, r, dt, bi)][off:off + nf]
            out = torch.zeros((nf, self.decs[ci].kw), dtype=torch.int32).pin_memory()
            self.trace.append((ci, x, out, float(arrivals[q])))
        self.frames = sum(t[1].shape[0] for t in self.trace)
        for ci, d in enumerate(self.decs):  # build device tables and grow staging to the largest request
            m, r, _, _, dt = self.cfgs[ci]
            d.decode_host(pools[(m, r, dt, 0)], torch.zeros((self.POOL, d.kw), dtype=torch.int32))
        torch.cuda.synchronize()

    def serve(self, fuse, streams=4):
        """Replays the trace through the continuous-batching server; fuse = one grouped launch
        per batch over all codes (else one launch per code). Returns (seconds, latencies in
        microseconds, server stats, the results)."""
        import paper_2108_12550_gb300 as pkg

        for t in self.trace:
            t[2].zero_()
        srv = pkg.Server(n_streams=streams, arena_bytes=2 << 30, max_batch_frames=1 << 15,
                         min_batch_frames=1024, max_wait_us=500, fuse_codes=fuse)
        ids = [srv.add_decoder(d) for d in self.decs]
        t0 = time.perf_counter()
        rids = []
        for ci, x, out, at in self.trace:
            while time.perf_counter() - t0 < at:
                pass
            rids.append(srv.submit(ids[ci], x, out))
        lat = []
        for rid in rids:
            st, l_us = srv.poll(rid, timeout_us=120_000_000)
            if st != pkg.OK:
                raise RuntimeError(f"serving request failed: {st}")
            lat.append(l_us)
        t_srv = time.perf_counter() - t0
        stats = srv.stats()
        srv.close()
        return t_srv, lat, stats, [t[2].clone() for t in self.trace]

    def plain(self):
        """The plain per-request form on the same trace: one synchronous host-to-host decode per
        request, in arrival order. Returns (seconds, latencies in microseconds)."""
        import torch

        s = torch.cuda.current_stream()
        t0 = time.perf_counter()
        plat = []
        for ci, x, out, at in self.trace:
            while time.perf_counter() - t0 < at:
                pass
            self.decs[ci].decode_host(x, out, s)
            plat.append((time.perf_counter() - t0 - at) * 1e6)
        return time.perf_counter() - t0, plat


def _pct(v):
    return {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99))}


def serving_leg(n_req, rate):
    """The latency half of the headline metric: the serving mix at a fixed offered load, the
    server (small requests of all codes fused into grouped launches) against the plain
    per-request launch on the same trace."""
    mix = ServingMix(n_req, rate)
    mix.serve(True)  # warm-up: first grouped launches, host page-in of the trace
    t_srv, lat, stats, served = mix.serve(True)
    t_plain, plat = mix.plain()
    same = all(a.equal(t[2]) for a, t in zip(served, mix.trace))
    return {"workload": "serving_mix", "offered_requests_per_s": rate, "requests": n_req, "frames": mix.frames,
            "server": {"frames_per_s": mix.frames / t_srv, "latency_us": _pct(lat), "batches": stats["batches"],
                       "form": "continuous batching, small requests of all codes in grouped launches"},
            "plain_per_request": {"frames_per_s": mix.frames / t_plain, "latency_us": _pct(plat),
                                  "form": "one synchronous rmdec_decode_host per request"},
            "results_identical_alone_and_in_mix": bool(same),
            "mix": "RM(2,7), RM(2,8), RM(2,9), RM(3,9) x P in {8,20} x INT8/FP32, L=4, 1-4096 frames "
                   "log-uniform, Eb/N0 2-5 dB, Poisson arrivals"}


def run_serving(args):
    """Serving mix: Poisson arrivals of requests over 16 decoder configurations; the
    continuous-batching server against a plain per-request launch on the same trace."""
    import torch

    n_req = args.requests
    mix = ServingMix(n_req, args.rate)
    trace, total_frames = mix.trace, mix.frames

    def serve(fuse):
        return mix.serve(fuse, args.streams)

    serve(True)  # warm-up: first grouped launches, host page-in of the trace
    t_fused, lat_f, stats_f, served_f = serve(True)
    t_srv, lat, stats, served = serve(False)

    # plain per-request launch: one synchronous host-to-host decode per request, in order
    t_plain, plat = mix.plain()
    same = all(torch.equal(a, t[2]) and torch.equal(b, t[2]) for a, b, t in zip(served, served_f, trace))
    line = {
        "metric": "frames/s serving mix (Poisson arrivals, mixed RM codes, P in {8,20}, L=4, INT8/FP32)",
        "value": total_frames / t_srv, "unit": "frames/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "mixed i8/f32", "data": "synthetic",
        "config": {"workload": "serving_mix", "requests": n_req, "rate_per_s": args.rate, "frames": total_frames,
                   "streams": args.streams, "codes": ["RM(2,7)", "RM(2,8)", "RM(2,9)", "RM(3,9)"]},
        "latency_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(np.max(lat))},
        "server": {"fuse_codes": False, **{k: stats[k] for k in ("batches", "completed", "frames_completed")}},
        "server_fused": {"value": total_frames / t_fused, "unit": "frames/s", "batches": stats_f["batches"],
                         "latency_us": {"p50": float(np.percentile(lat_f, 50)),
                                        "p99": float(np.percentile(lat_f, 99))},
                         "form": "small requests of all 16 codes share grouped launches"},
        "plain_per_request": {"value": total_frames / t_plain, "unit": "frames/s",
                              "latency_us": {"p50": float(np.percentile(plat, 50)),
                                             "p99": float(np.percentile(plat, 99))}},
        "results_identical_alone_and_in_mix": bool(same),
        "gpu_launches": int(stats["batches"]),  # one decode launch per batch
    }
    print(json.dumps(line), flush=True)


def run_grouped(args):
    """Grouped multi-code launches against one launch per code: RM(2,7) P=8 INT8, RM(2,8) P=8,
    RM(2,9) P=20, RM(3,9) P=8 INT8 (L = 4), at a few frames per code and at large segments
    (which the default split sends to their own launches). CUDA-event times, best of 5."""
    import torch

    import paper_2108_12550_gb300 as pkg

    specs = {"RM(2,9)": (9, 2, 20, "f32", 131072), "RM(2,7)": (7, 2, 8, "i8", 262144),
             "RM(3,9)": (9, 3, 8, "i8", 32768), "RM(2,8)": (8, 2, 8, "f32", 131072)}
    decs, xs = {}, {}
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    for i, (name, (m, r, P, dt, nf)) in enumerate(specs.items()):
        decs[name] = pkg.Decoder(m, r, P, 4, perm_seed=i + 1, dtype=dt)
        _, llr = I.make_frames_torch(m, r, nf, 2.5, gen)
        if dt == "i8":
            llr = torch.clamp(torch.round(llr / 0.25), -127, 127).to(torch.int8)
        xs[name] = llr.contiguous()
    torch.cuda.synchronize()

    def best_ms(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    cases, same = [], True
    mixes = {"four codes": ["RM(2,9)", "RM(2,7)", "RM(3,9)", "RM(2,8)"], "RM(2,.) codes": ["RM(2,9)", "RM(2,7)", "RM(2,8)"]}
    for label, keys in mixes.items():
        grp = pkg.Group([decs[k] for k in keys])
        for nf in (50, 200, 600, None):
            segs = [(i, xs[k][:nf] if nf else xs[k], None) for i, k in enumerate(keys)]
            t_sep = best_ms(lambda: [decs[k].decode(x) for k, (_, x, _) in zip(keys, segs)])
            t_grp = best_ms(lambda: grp.decode(segs))
            outs = grp.decode(segs)
            same = same and all(torch.equal(o, decs[k].decode(x)) for k, (_, x, _), o in zip(keys, segs, outs))
            cases.append({"mix": label, "frames_per_code": nf or "large (" + ", ".join(str(xs[k].shape[0]) for k in keys) + ")",
                          "grouped_ms": t_grp, "separate_ms": t_sep})
        grp.close()
    line = {"metric": "ms per decode of one segment per code: grouped launch vs one launch per code", "unit": "ms",
            "n_gpus": 1, "higher_is_better": False, "dtype": "mixed i8/f32", "data": "synthetic, 2.5 dB",
            "config": {"workload": "grouped_mix", "decoders": [f"{k} P={specs[k][2]} L=4 {specs[k][3]}" for k in specs]},
            "cases": cases, "results_identical_grouped_and_separate": bool(same)}
    print(json.dumps(line), flush=True)


# Frame error rates printed in the paper's Fig. 6 (RM(2,9) panel) for comparison
PAPER_FER = {"p-FHT-FSCL-4-20": {1.0: 9.80e-3, 1.5: 2.11e-3, 2.0: 2.99e-4, 2.5: 2.85e-5},
             "Aut-SSC-512": {1.0: 9.38e-3, 1.5: 2.14e-3, 2.0: 2.58e-4, 2.5: 2.76e-5}}


# FER sweeps of the paper's configurations: (m, r, P, L, [(run name, dtype, decoder kind)],
# default Eb/N0 points)
SWEEPS = {
    "rm29": (9, 2, 20, 4, [("p-FHT-FSCL-4-20", "f32", "pfht"), ("p-FHT-FSCL-4-20 FP16 LLRs", "f16", "pfht"),
                           ("p-FHT-FSCL-4-20 INT8 LLRs", "i8", "pfht"),
                           ("p-FHT-FSCL-4-20 FP16 LLRs tensor-core Hadamard", "f16", "pfht_tc"),
                           ("Aut-SSC-512", "f32", "autssc")],
             [1.0, 1.5, 2.0, 2.25, 2.5]),
    "rm27": (7, 2, 8, 4, [("p-FHT-FSCL-4-8", "f32", "pfht"), ("p-FHT-FSCL-4-8 INT8 LLRs", "i8", "pfht")],
             [1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 5.0]),
    "rm39": (9, 3, 16, 8, [("p-FHT-FSCL-8-16", "f32", "pfht"), ("p-FHT-FSCL-8-16 FP16 LLRs", "f16", "pfht"),
                           ("p-FHT-FSCL-8-16 FP16 LLRs tensor-core Hadamard", "f16", "pfht_tc")],
             [1.0, 1.5, 2.0, 2.5, 3.0]),  # no frame errors in 10^6 frames per point from 3 dB up
}


def run_fer_sweep(args):
    """FER of p-FHT-FSCL on the paper's configurations (RM(2,9) P=20 L=4 in FP32, FP16 and
    INT8 beside Aut-SSC-512; RM(2,7) P=8 L=4 in FP32 and INT8; RM(3,9) P=16 L=8 in FP32 and
    FP16), every decoder on the same frames, generated on the GPU in chunks, with decoding
    time per point and the rate of decisions differing from the FP32 decoder's."""
    import torch

    import paper_2108_12550_gb300 as pkg

    m, r, P, L, spec, default_eb = SWEEPS[args.sweep_code]
    k = I.rm_dims(m, r)[1]
    kw = (k + 31) // 32
    if args.ebn0 is None:
        args.ebn0 = default_eb

    def convert(dt):
        if dt == "f16":
            return lambda x: x.half()
        if dt == "i8":
            return lambda x: torch.clamp(torch.round(x / 0.25), -127, 127).to(torch.int8)
        return lambda x: x

    def make(dt, kind):
        if kind == "autssc":
            return pkg.Decoder(m, r, 512, algo="autssc", perm_seed=1)
        d = pkg.Decoder(m, r, P, L, perm_seed=1, dtype=dt)
        if kind == "pfht_tc":
            d.set_hadamard("tensor")
        return d

    runs = [(name, make(dt, kind), convert(dt)) for name, dt, kind in spec]
    fp32_name = spec[0][0]
    gen = torch.Generator(device="cuda")
    chunk = 1 << 18
    out = torch.empty((chunk, kw), dtype=torch.int32, device="cuda")
    ref_bits = torch.empty((chunk, kw), dtype=torch.int32, device="cuda")
    # Chunk c of point Eb/N0 draws its frames from its own seed, so chunks are independent and
    # a sweep can stop and resume: --checkpoint keeps one JSON line per finished chunk.
    done_chunks = {}
    if args.checkpoint and os.path.exists(args.checkpoint):
        with open(args.checkpoint) as fh:
            for line in fh:
                rec = json.loads(line)
                done_chunks[(rec.get("code", "rm29"), rec["ebn0_db"], rec["chunk"])] = rec
    ckpt = open(args.checkpoint, "a") if args.checkpoint else None
    points = []
    for eb in args.ebn0:
        n_pf = args.sweep_frames
        n_ssc = min(args.sweep_frames, args.ssc_frames)
        lims = {name: (n_ssc if name == "Aut-SSC-512" else n_pf) for name, _, _ in runs}
        err = {name: 0 for name, _, _ in runs}
        differ = {name: 0 for name, _, _ in runs}  # decisions other than the FP32 decoder's
        t_dec = {name: 0.0 for name, _, _ in runs}
        for ci, done in enumerate(range(0, n_pf, chunk)):
            f = min(chunk, n_pf - done)
            rec = done_chunks.get((args.sweep_code, eb, ci))
            if rec is None or rec["frames"] != f:
                gen.manual_seed(2108 * 1000003 + int(round(eb * 1000)) * 65537 + ci)
                u, llr = I.make_frames_torch(m, r, f, eb, gen)
                unpack = lambda w: ((w.view(-1, kw, 1) >> torch.arange(32, device="cuda")) & 1).view(-1, 32 * kw)[:, :k]
                rec = {"code": args.sweep_code, "ebn0_db": eb, "chunk": ci, "frames": f, "errors": {}, "differ": {},
                       "seconds": {}}
                for name, dec, conv in runs:
                    if done >= lims[name]:
                        continue
                    g = min(f, lims[name] - done)
                    xin = conv(llr[:g]).contiguous()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    dec.decode(xin, out[:g])
                    e1.record()
                    torch.cuda.synchronize()
                    rec["seconds"][name] = e0.elapsed_time(e1) * 1e-3
                    rec["errors"][name] = int(torch.any(unpack(out[:g]).to(torch.uint8) != u[:g], dim=1).sum().item())
                    if name == fp32_name:
                        ref_bits[:g].copy_(out[:g])
                    elif name.startswith("p-FHT"):
                        rec["differ"][name] = int(torch.any(out[:g] != ref_bits[:g], dim=1).sum().item())
                if ckpt:
                    ckpt.write(json.dumps(rec) + "\n")
                    ckpt.flush()
            for name in rec["errors"]:
                err[name] += rec["errors"][name]
                t_dec[name] += rec["seconds"][name]
                differ[name] += rec["differ"].get(name, 0)
        pt = {"ebn0_db": eb}
        for name, _, _ in runs:
            n = lims[name]
            pt[name] = {"frames": n, "errors": err[name], "fer": err[name] / n,
                        "frames_per_s": n / t_dec[name] if t_dec[name] else None}
            if name in PAPER_FER:
                pt[name]["paper_fer"] = PAPER_FER[name].get(eb)
            if name.startswith("p-FHT") and name != fp32_name:
                pt[name]["decisions_differing_from_fp32"] = differ[name] / n
        points.append(pt)
        print(json.dumps(pt), flush=True)
    if ckpt:
        ckpt.close()
    print(json.dumps({"metric": f"FER RM({r},{m}) P={P} L={L}: " + ", ".join(n for n, _, _ in spec) + " on the same frames",
                      "points": points, "data": "synthetic BPSK/AWGN frames generated on the GPU"}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="rm29_p20_l4", choices=sorted(WORKLOADS) + ["serving_mix", "fer_sweep", "grouped_mix"])
    ap.add_argument("--sweep-code", default="rm29", choices=sorted(SWEEPS), help="FER sweep: configuration")
    ap.add_argument("--ebn0", type=float, nargs="+", default=None,
                    help="FER sweep: Eb/N0 points (dB)")
    ap.add_argument("--sweep-frames", type=int, default=1 << 22, help="FER sweep: frames per point")
    ap.add_argument("--ssc-frames", type=int, default=1 << 20, help="FER sweep: Aut-SSC frames per point")
    ap.add_argument("--checkpoint", default=None, help="fer_sweep: JSON-lines file of finished chunks (resume)")
    ap.add_argument("--requests", type=int, default=2000, help="serving mix: requests in the trace")
    ap.add_argument("--rate", type=float, default=8000.0, help="serving mix: Poisson arrivals per second")
    ap.add_argument("--streams", type=int, default=4, help="serving mix: server CUDA streams")
    ap.add_argument("--frames", type=int, default=0, help="frames per step (default per workload)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "i8", "f16", "i16"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "warp", "path"],
                    help="decoder kernel: warp per decoder, thread per path (RM(2, m <= 8)), or auto")
    ap.add_argument("--hadamard", default="shuffle", choices=["shuffle", "tensor"],
                    help="FHT of the FHTL nodes: FP32 butterflies or FP16 tensor-core products")
    ap.add_argument("--cpu-frames", type=int, default=1500, help="CPU-baseline sample size")
    ap.add_argument("--ref-frames", type=int, default=1000, help="frames per reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=8000,
                    help="requests of the serving-mix latency leg of the default run (0: skip)")
    args = ap.parse_args()
    if args.workload == "serving_mix":
        return run_serving(args)
    if args.workload == "fer_sweep":
        return run_fer_sweep(args)
    if args.workload == "grouped_mix":
        return run_grouped(args)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    import torch.distributed as dist

    import paper_2108_12550_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)  # before the process group, so NCCL binds each rank to its GPU
    if world > 1:
        dist.init_process_group("nccl")
    m, r, P, L, ebn0, nf_default = wl
    nf = args.frames or nf_default
    n, k = I.rm_dims(m, r)
    llr_np, u_np = _frames(m, r, nf, ebn0, seed=100 + rank)
    if args.dtype == "i8":
        llr_np = I.quantize_i8(llr_np)
    elif args.dtype == "i16":
        llr_np = np.clip(np.rint(llr_np * 256), -32767, 32767).astype(np.int16)
    elif args.dtype == "f16":
        llr_np = I.to_f16(llr_np)
    dec = pkg.Decoder(m, r, P, L, perm_seed=1, dtype=args.dtype)
    if args.hadamard != "shuffle":
        dec.set_hadamard(args.hadamard)
    if args.kernel != "auto":
        dec.set_kernel(args.kernel)
    x = torch.from_numpy(llr_np).cuda()
    out = torch.empty((nf, dec.kw), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (also builds device tables)
    for _ in range(args.warmup):
        dec.decode(x, out, stream)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            dec.decode(x, out, stream)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = replicas.allreduce_max(ms, device="cuda")  # the job is as slow as its slowest rank
    value = nf * world / (ms_max * 1e-3)

    # correctness side-channel: frame error rate of the timed batches vs the transmitted messages
    got = pkg.unpack_bits(out.cpu().numpy(), k)
    errs, frames = replicas.allreduce_sum([int(np.sum(np.any(got != u_np, axis=1))), nf], device="cuda")
    fer = errs / frames

    # end to end through the host entry point: pinned host LLRs in, information bits out
    host_in = torch.from_numpy(llr_np).pin_memory()
    host_out = torch.empty((nf, dec.kw), dtype=torch.int32).pin_memory()
    dec.decode_host(host_in, host_out, stream)
    barrier()
    e0 = time.perf_counter()
    e_steps = args.steps
    for _ in range(e_steps):
        dec.decode_host(host_in, host_out, stream)
    barrier()
    e_ms = (time.perf_counter() - e0) / e_steps * 1e3
    e_value = nf * world / (replicas.allreduce_max(e_ms, device="cuda") * 1e-3)

    # plain per-frame form: one decode launch per frame, LLRs resident on the device
    n1 = min(nf, 512)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dec.decode(x[:1], out[:1], stream)
    p0.record(stream)
    for i in range(n1):
        dec.decode(x[i:i + 1], out[i:i + 1], stream)
    p1.record(stream)
    torch.cuda.synchronize()
    per_frame_value = n1 / (p0.elapsed_time(p1) * 1e-3)

    # roofline: the slower of the ALU side (algorithmic operations at one per lane per clock)
    # and the HBM side (LLRs read once, information bits written once)
    pk, src = _peaks()
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    ops = opcount.ops_per_frame(m, r, P, L)
    peak_ops = sms * LANES_PER_SM * sm_mhz * 1e6
    hbm_bw = float(pk.get("hbm_gbs", 6800.0)) * 1e9
    bytes_frame = llr_np.nbytes / nf + dec.kw * 4
    t_launch = ms * 1e-3
    t_alu, t_hbm = ops * nf / peak_ops, bytes_frame * nf / hbm_bw
    if t_alu >= t_hbm:
        bound, achieved, peak, unit = "alu", ops * nf / t_launch / 1e12, peak_ops / 1e12, "Tops/s"
    else:
        bound, achieved, peak, unit = "hbm", bytes_frame * nf / t_launch / 1e9, hbm_bw / 1e9, "GB/s"
    traffic = None
    tr = TRAFFIC.get((args.workload, args.dtype))
    if (tr and args.hadamard == "shuffle" and dec.kernel_for(nf) == tr["kernel"]
            and kernel_fingerprint(tr["source"]).startswith(tr["kernel_code_sha256"])):
        traffic = tr["bytes_per_frame"] * nf  # scaled from the captured case by frames
    line = {
        "metric": METRIC if args.workload == "rm29_p20_l4" else f"frames/s {args.workload}",
        "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": args.workload, "m": m, "r": r, "P": P, "L": L, "n": n, "k": k,
                   "ebn0_db": ebn0, "frames_per_step": nf, "l2": "inputs larger than L2 "
                   f"({llr_np.nbytes / 2**20:.0f} MiB of LLRs per step)", "parallelism": f"replicas{world}",
                   "launch": dict(zip(("warps_per_cta", "ctas_per_sm"), dec.get_tuning())),
                   "hadamard": args.hadamard, "kernel": args.kernel},
        "info_gbit_s": value * k / 1e9,
        "fer_of_timed_batch": fer,
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                     "frac": max(t_alu, t_hbm) / t_launch, "traffic": traffic, "traffic_unit": "bytes per launch",
                     "ops_per_frame": ops, "bytes_per_frame": bytes_frame,
                     "sides": {"alu": {"seconds": t_alu, "peak_tops": peak_ops / 1e12,
                                       "peak_source": f"{sms} SMs x {LANES_PER_SM} lanes x {sm_mhz:.0f} MHz "
                                                      f"({src} max SM clock)"},
                               "hbm": {"seconds": t_hbm, "peak_gbs": hbm_bw / 1e9,
                                       "peak_source": f"{src} copy bandwidth"}},
                     "launch_seconds": t_launch},
        "e2e": {"value": e_value, "unit": "frames/s", "h2d_bytes_per_step": int(llr_np.nbytes),
                "d2h_bytes_per_step": int(nf * dec.kw * 4)},
        "plain_per_frame": {"value": per_frame_value, "unit": "frames/s",
                            "form": "one rmdec_decode launch per frame, device-resident LLRs"},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(m, r, P, L, ebn0, args.cpu_frames)
    if rank == 0 and world == 1 and args.workload == "rm29_p20_l4" and args.serving_requests > 0:
        line["serving"] = serving_leg(args.serving_requests, args.rate)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
