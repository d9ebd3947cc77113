#!/usr/bin/env python3
"""Decoded information bits/s of SOGRAND block-turbo decoding of the
eBCH(64,57)^2 product code on GB300 (arXiv 2310.10737, Sec. VI workload).

One step = one product_decode of the whole batch: 100,000 frames of
eBCH(64,57)^2 (n = 4096, k = 3249), BPSK over AWGN with Eb/N0 swept
2.5..4.0 dB in 0.25 dB steps (frame f at point f mod 7), FP32 channel LLRs,
list size L = 4, query cap 10^4 per component decoding, alpha = 0.5, at most
20 iterations with per-frame early stop.  Inputs (1.64 GB of LLRs) are larger
than L2 and resident in HBM before timing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the method has no other implementation).
Under torchrun (N > 1) every rank decodes its own batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CODE = "ebch_64_57"
FRAMES = 100_000
EBN0 = [2.5 + 0.25 * i for i in range(7)]
L_LIST, CAP, ALPHA, MAX_ITER, SEED = 4, 10**4, 0.5, 20, 2310
SMS, INT32_LANES = 152, 128  # GB300: 152 SMs x 128 INT32/FP32 lanes per SM
METRIC = "decoded info bits/s, eBCH(64,57)^2 product code"

# DRAM bytes (read + write) per frame of k_product_persistent, from one ncu
# capture of a 10,000-frame decode of this workload (traffic grows with the
# frame count at a fixed Eb/N0 mix), valid only for the kernel sources whose
# digest is recorded with it: `traffic` is null once they change.
TRAFFIC = {"csrc_digest": "f6a931810f509a673668d4db930d62b4cc9f7661ce62958ec9f7ce4da77631f4",
           "bytes_per_frame": 280960.5,
           "source": "profiles/k_product_persistent_ebch64_57sq_10k_frames.md",
           # pipe activity of the same capture (percent of peak sustained over active cycles)
           "ncu": {"issue_active_pct": 68.8, "alu_pipe_pct": 45.6, "fma_pipe_pct": 25.8,
                   "tensor_pipe_pct": 0.0, "dram_throughput_pct": 1.5}}


KERNEL_SOURCES = ("kernels.cuh", "launch.h", "sg_common.h", "siso_warp.cuh")  # what k_product_persistent compiles from


def measured_hbm_gbs():
    """The machine's measured copy bandwidth (GB/s), or None without the peaks file."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = json.load(fh).get("hbm_gbs")
        return float(v) if v is not None else None
    except (OSError, ValueError, TypeError):
        return None


def csrc_digest():
    """SHA-256 of the measured kernel's sources (profiling-only #ifdef SG_PHASE_PROFILE blocks left out)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2310_10737_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name not in KERNEL_SOURCES:
            continue
        keep, depth = [], 0
        for line in open(os.path.join(d, name)):
            t = line.strip()
            if depth == 0 and t == "#ifdef SG_PHASE_PROFILE":
                depth = 1
                continue
            if depth:
                if t.startswith("#if"):
                    depth += 1
                elif t == "#endif":
                    depth -= 1
                continue
            keep.append(line)
        h.update(name.encode() + b"\0" + "".join(keep).encode())
    return h.hexdigest()


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def workload_config(frames):
    return {"workload": f"eBCH(64,57)^2 product code, {frames} frames, BPSK/AWGN Eb/N0 2.5:0.25:4.0 dB "
                        "(frame f at point f mod 7), L=4, query cap 1e4, alpha 0.5, max 20 iterations, early stop",
            "frames": frames, "n": 64, "k": 57, "info_bits_per_frame": 57 * 57, "L": L_LIST, "query_cap": CAP,
            "max_iter": MAX_ITER, "alpha": ALPHA, "ebn0_db": EBN0, "seed": SEED,
            "l2": "inputs larger than L2 (4 n^2 bytes per frame = 1.64 GB per 100k-frame step)"}


def make_inputs(code, frames, seed, threads):
    from workloads import awgn_frames
    snr = np.array(EBN0)[np.arange(frames) % len(EBN0)]
    return awgn_frames(code, frames, snr, seed=seed, threads=threads)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        self.skip = 0

    def mark(self):
        """Start of the timed region: wait for nvidia-smi to come up (its start-up
        must not overlap the timed work), then count only later samples."""
        if self.p is None:
            return
        t = time.time()
        while time.time() - t < 5.0 and self._rows() < 2:
            time.sleep(0.05)
        self.skip = self._rows()

    def _rows(self):
        self.f.flush()
        try:
            return sum(1 for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8)
        except OSError:
            return 0

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(", ") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        rows = rows[self.skip:] or rows[-1:]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({nm for r in rows for nm, v in zip(names, r[5:9]) if v.strip() == "Active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def rank_seed(rank):
    """Each rank decodes its own seeded batch (weak scaling: frames are independent)."""
    return SEED + rank


def max_over_ranks(x, dist, dev):
    """The slowest rank's figure (the timed region ends when every rank is done)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, frames, info_bits_per_frame, steps, ms):
    """Whole-job information bits/s: every rank's frames over the slowest rank's time."""
    return world * frames * info_bits_per_frame * steps / (ms / 1000)


SERVE_CODES = ["ebch_32_26", "ebch_64_57", "ebch_64_51", "ebch_128_120"]


def serving_bench(sg, torch, n_req, loads, seed, epoch_halves=16):
    """Poisson arrivals of decode requests (code uniform over four eBCH product
    codes, 1..64 frames, Eb/N0 uniform in 2.5..4 dB per request) into the
    continuous-batching server, at several offered loads; and the same arrivals
    decoded one request at a time (per-request launches of the plain form).
    Latency = submission (arrival) to outputs in host memory."""
    import threading
    from workloads import awgn_frames, ebch
    rng = np.random.default_rng(seed)
    lin = [ebch(nm) for nm in SERVE_CODES]
    codes = [sg.Code.from_linear_code(c) for c in lin]
    t0 = time.perf_counter()
    spec = [(int(rng.integers(0, len(lin))), int(rng.integers(1, 65)), float(rng.uniform(2.5, 4.0)))
            for _ in range(n_req)]
    # per code, every frame its requests need in one seeded batch (per-frame Eb/N0), then sliced
    frames = {}
    for ci, lc in enumerate(lin):
        snr = np.concatenate([[e] * F for c, F, e in spec if c == ci] or [[3.0]])
        frames[ci] = awgn_frames(lc, len(snr), snr, seed=seed, stream=100 + ci, threads=16)[2]
    pos = [0] * len(lin)
    reqs = []
    for ci, F, _ in spec:
        n = lin[ci].n
        llr = torch.from_numpy(np.ascontiguousarray(frames[ci][pos[ci]:pos[ci] + F])).pin_memory()
        pos[ci] += F
        out = dict(bits=torch.empty((F, n * n // 8), dtype=torch.uint8, pin_memory=True),
                   half_iters=torch.empty(F, dtype=torch.int32, pin_memory=True),
                   status=torch.empty(F, dtype=torch.uint8, pin_memory=True),
                   queries=torch.empty(F, dtype=torch.int64, pin_memory=True))
        reqs.append((ci, llr, out, F * lin[ci].k ** 2))
    del frames
    log(f"serving: {n_req} requests ({sum(F for _, F, _ in spec)} frames) generated in {time.perf_counter() - t0:.1f} s")
    for c, lc in zip(codes, lin):  # schedules tuned on a sample of that code's frames
        _, _, smp = awgn_frames(lc, 2000, 3.0, seed=seed + 7)
        c.tune(torch.from_numpy(smp).cuda(), L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=MAX_ITER)
    slots = [8192, 4096, 4096, 2048]
    bits = sum(b for *_, b in reqs)
    res = {"workload": "requests: code uniform over eBCH(32,26)^2, (64,57)^2, (64,51)^2, (128,120)^2; frames "
                       "uniform 1..64; Eb/N0 uniform 2.5..4.0 dB per request; Poisson arrivals; L=4, cap 1e4, "
                       "alpha 0.5, max 20 iterations",
           "requests": n_req, "info_bits": bits, "epoch_halves": epoch_halves,
           "slots": dict(zip(SERVE_CODES, slots)), "latency": "submission to outputs in host memory",
           "server": [], "per_request_plain": [], "per_request_batched": []}

    def pct(v, q):
        return float(np.percentile(np.array(v), q)) if v else None

    for lam in loads:
        gaps = rng.exponential(1.0 / lam, n_req)
        arrive = np.cumsum(gaps) - gaps[0]
        srv = sg.Server(codes, slots, L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=MAX_ITER,
                        epoch_halves=epoch_halves)
        tickets = [None] * n_req

        def client():
            start = time.perf_counter()
            for i, (ci, llr, out, _) in enumerate(reqs):
                d = start + arrive[i] - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets[i] = srv.submit(ci, llr, out)[0]

        t_start = time.perf_counter()
        th = threading.Thread(target=client)
        th.start()
        th.join()
        lat = [srv.wait(t, timeout_ms=600000)[1] for t in tickets]
        span = time.perf_counter() - t_start
        st = srv.stats()
        srv.close()
        res["server"].append({"offered_rps": lam, "achieved_rps": n_req / span, "p50_ms": pct(lat, 50),
                              "p99_ms": pct(lat, 99), "bits_per_s": bits / span, "launches": st["launches"]})
        log(f"serving: server at {lam:g} req/s: p50 {pct(lat, 50):.2f} ms p99 {pct(lat, 99):.2f} ms, "
            f"{bits / span:.3e} bits/s, {st['launches']} launches")
        # the same arrivals served one request at a time: the plain form (one
        # launch per half) and the batched form (one persistent launch per request)
        for form, pers in (("per_request_plain", False), ("per_request_batched", True)):
            lat = []
            start = time.perf_counter()
            for i, (ci, llr, _, _) in enumerate(reqs):
                a = start + arrive[i]
                d = a - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                o = sg.product_decode(codes[ci], llr.cuda(non_blocking=True), L=L_LIST, query_cap=CAP, alpha=ALPHA,
                                      max_iter=MAX_ITER, persistent=pers, stats=False)
                o["bits"].cpu()
                lat.append(1000 * (time.perf_counter() - a))
            span = time.perf_counter() - start
            res[form].append({"offered_rps": lam, "achieved_rps": n_req / span, "p50_ms": pct(lat, 50),
                              "p99_ms": pct(lat, 99), "bits_per_s": bits / span})
            log(f"serving: {form.replace('_', ' ')} at {lam:g} req/s: p50 {pct(lat, 50):.2f} ms "
                f"p99 {pct(lat, 99):.2f} ms, {bits / span:.3e} bits/s")
    for c in codes:
        c.close()
    return res


def _events_ms(torch, fn, reps):
    """Device time of `reps` calls of fn (CUDA events on the current stream,
    synchronised on both sides), after one untimed call."""
    fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _frame_errors(bits_dev, X):
    """Frames whose decoded (packed, LSB first) bits differ from the transmitted X [F, n, n]."""
    ref = np.packbits(X.reshape(X.shape[0], -1), axis=1, bitorder="little")
    return (bits_dev.cpu().numpy() != ref).any(axis=1)


def other_configs(sg, torch, cores, reps=2):
    """The other workloads of the method, measured beside the headline (each
    a separate figure, not part of `value`):
    C1  plain method: eBCH(32,26)^2, 200 frames at 3.0 dB, L=4, cap 1e4, 4 iterations;
    C2  component SISO: 10^6 eBCH(64,57) and 10^6 eBCH(32,26) words, Eb/N0 2/3/4/5 dB
        (word w at point w mod 4), L in {1, 2, 4}, cap 1e5, one launch per code and L;
    C4  mixed batch: 200,000 frames of eBCH(32,26)^2, (64,51)^2, (128,120)^2 in 4:2:1,
        Eb/N0 uniform in 2.5..4.0 dB per frame, L=4, cap 1e4, 20 iterations: one mixed
        launch vs the batched form per code vs the plain form per code;
    order_source: the order table against the lanes enumerating the order (order_source_ab)."""
    from workloads import awgn_frames, awgn_words, ebch
    res = {}
    dev = torch.device("cuda")
    # C1
    code = ebch("ebch_32_26")
    U, X, lch = awgn_frames(code, 200, 3.0, seed=1, threads=cores)
    c = sg.Code.from_linear_code(code)
    d = torch.from_numpy(lch).to(dev)
    kw = dict(L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=4, stats=False)
    c1 = {"workload": "eBCH(32,26)^2, 200 frames, 3.0 dB, L=4, cap 1e4, alpha 0.5, 4 iterations", "frames": 200}
    for form, pers in (("plain", False), ("persistent", True)):
        box = {}
        ms = _events_ms(torch, lambda: box.update(o=sg.product_decode(c, d, persistent=pers, **kw)), reps + 3)
        c1[form] = {"ms": ms, "bits_per_s": 200 * 26 * 26 / (ms / 1000),
                    "bler": float(_frame_errors(box["o"]["bits"], X).mean())}
    c.close()
    res["C1"] = c1
    log(f"C1: plain {c1['plain']['ms']:.2f} ms, persistent {c1['persistent']['ms']:.2f} ms")
    # C2
    W = 10**6
    snr = np.array([2.0, 3.0, 4.0, 5.0])[np.arange(W) % 4]
    c2 = {"workload": "10^6 words per code, Eb/N0 2/3/4/5 dB (word w at point w mod 4), component rate, "
                      "L in {1,2,4}, cap 1e5, one sogrand_decode launch per code and L", "words": W}
    for name in ("ebch_64_57", "ebch_32_26"):
        code = ebch(name)
        _, _, lw = awgn_words(code, W, snr, seed=2, threads=cores)
        c = sg.Code.from_linear_code(code)
        c.reserve(10**5)
        cap_t, tbytes = c.tables()
        d = torch.from_numpy(lw).to(dev)
        row = {"table_bytes": tbytes, "table_cap": cap_t}
        for L in (1, 2, 4):
            box = {}
            ms = _events_ms(torch, lambda: box.update(o=sg.sogrand_decode(c, d, L=L, query_cap=10**5, lists=False)),
                            reps)
            q = int(box["o"]["queries"].sum())
            row[f"L{L}"] = {"ms": ms, "words_per_s": W / (ms / 1000), "queries_per_s": q / (ms / 1000),
                            "info_bits_per_s": W * code.k / (ms / 1000), "queries_per_word": q / W}
        c2[name] = row
        c.close()
        del d
        log(f"C2 {name}: " + ", ".join(f"L={L} {row[f'L{L}']['ms']:.1f} ms" for L in (1, 2, 4)))
    res["C2"] = c2
    # C4
    names = ["ebch_32_26", "ebch_64_51", "ebch_128_120"]
    total = 200_000
    counts = [total * 4 // 7, total * 2 // 7]
    counts.append(total - sum(counts))
    rng = np.random.default_rng(SEED + 4)
    groups, refs, codes = [], [], []
    info = 0
    for i, (name, F) in enumerate(zip(names, counts)):
        code = ebch(name)
        snr = rng.uniform(2.5, 4.0, F)
        U, X, lf = awgn_frames(code, F, snr, seed=SEED + 40 + i, threads=cores)
        c = sg.Code.from_linear_code(code)
        d = torch.from_numpy(lf).to(dev)
        del lf
        c.tune(d[:4000], L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=MAX_ITER)
        groups.append((c, d))
        refs.append(X)
        codes.append(code)
        info += F * code.k * code.k
    kw = dict(L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=MAX_ITER)
    c4 = {"workload": f"{total} frames, eBCH(32,26)^2 : (64,51)^2 : (128,120)^2 = 4:2:1 "
                      f"({counts[0]} + {counts[1]} + {counts[2]}), Eb/N0 uniform 2.5..4.0 dB per frame, L=4, "
                      "cap 1e4, alpha 0.5, max 20 iterations", "frames": total, "info_bits": info,
          "schedules": {nm: (c.schedule(), "global" if c.dp_area() else "shared") for nm, (c, _) in zip(names, groups)}}
    box = {}
    ms = _events_ms(torch, lambda: box.update(o=sg.product_decode_mixed(groups, stats=False, **kw)[0]), reps)
    c4["mixed"] = {"ms": ms, "bits_per_s": info / (ms / 1000), "launches": 1,
                   "graph_kernels": 2 * len(groups),
                   "bler": {nm: float(_frame_errors(o["bits"], X).mean()) for nm, o, X in zip(names, box["o"], refs)}}
    for form, pers in (("batched_per_code", True), ("plain_per_code", False)):
        box = {}

        def per_code():
            box["o"] = [sg.product_decode(c, d, persistent=pers, stats=False, **kw) for c, d in groups]

        ms = _events_ms(torch, per_code, reps)
        c4[form] = {"ms": ms, "bits_per_s": info / (ms / 1000),
                    "bler": {nm: float(_frame_errors(o["bits"], X).mean()) for nm, o, X in zip(names, box["o"], refs)}}
    log("C4: " + ", ".join(f"{f} {c4[f]['ms']:.1f} ms" for f in ("mixed", "batched_per_code", "plain_per_code")))
    for c, _ in groups:
        c.close()
    res["C4"] = c4
    res["order_source"] = order_source_ab(sg, torch, cores, reps)
    return res


def order_source_ab(sg, torch, cores, reps):
    """Where the query loop takes its patterns (sogrand_code_order_source): the
    precomputed order table (the default) against the lanes enumerating the
    1-line ORBGRAND order themselves (unranking distinct-part partitions), on
    the first 20,000 frames of the headline workload (batched form, tuned
    schedule) and on the C2 eBCH(64,57) words at L=4, cap 1e5.  Both sources
    give identical outputs (checked here on the decoded bits and the query
    counts)."""
    from workloads import awgn_words, ebch
    dev = torch.device("cuda")
    code = ebch(CODE)
    F = 20_000
    _, _, lch = make_inputs(code, F, rank_seed(0), cores)
    d = torch.from_numpy(lch).to(dev)
    del lch
    c = sg.Code.from_linear_code(code)
    c.tune(d[:10_000], L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=MAX_ITER)
    kw = dict(L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=MAX_ITER, persistent=True, stats=False)
    r = {"workload": f"{F} frames of the headline workload (eBCH(64,57)^2, 2.5..4.0 dB), L=4, cap 1e4, "
                     "20 iterations, batched form; C2 eBCH(64,57) 10^6 words, L=4, cap 1e5",
         "schedule": [c.schedule(), "global" if c.dp_area() else "shared"]}
    outs = {}
    for name, src in (("table", 0), ("lanes", 1)):
        c.order_source(src)
        box = {}
        ms = _events_ms(torch, lambda: box.update(o=sg.product_decode(c, d, **kw)), reps + 1)
        outs[name] = (box["o"]["bits"].cpu().numpy(), box["o"]["queries"].cpu().numpy())
        r[name] = {"ms": ms, "info_bits_per_s": F * code.k * code.k / (ms / 1000)}
    c.order_source(0)
    r["identical"] = bool((outs["table"][0] == outs["lanes"][0]).all() and (outs["table"][1] == outs["lanes"][1]).all())
    c.close()
    del d
    W = 10**6
    snr = np.array([2.0, 3.0, 4.0, 5.0])[np.arange(W) % 4]
    _, _, lw = awgn_words(code, W, snr, seed=2, threads=cores)
    c = sg.Code.from_linear_code(code)
    c.reserve(10**5)
    d = torch.from_numpy(lw).to(dev)
    del lw
    for name, src in (("c2_table", 0), ("c2_lanes", 1)):
        c.order_source(src)
        box = {}
        ms = _events_ms(torch, lambda: box.update(o=sg.sogrand_decode(c, d, L=4, query_cap=10**5, lists=False)), reps)
        q = int(box["o"]["queries"].sum())
        r[name] = {"ms": ms, "words_per_s": W / (ms / 1000), "queries_per_s": q / (ms / 1000)}
    c.close()
    log(f"order source: table {r['table']['ms']:.1f} ms, lanes {r['lanes']['ms']:.1f} ms (identical: "
        f"{r['identical']}); C2 L=4 table {r['c2_table']['ms']:.2f} ms, lanes {r['c2_lanes']['ms']:.2f} ms")
    return r


def cpu_oracle_rate(code, lch, threads):
    """The oracle (FP64, plain C, all host cores) on a bounded sample: info bits/s."""
    import oracle
    oc = oracle.OracleCode(code)
    t = time.perf_counter()
    oracle.product_batch(oc, lch, L=L_LIST, cap=CAP, alpha=ALPHA, max_iter=MAX_ITER, threads=threads)
    dt = time.perf_counter() - t
    return lch.shape[0] * code.k * code.k / dt, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from workloads import ebch
    code = ebch(CODE)
    cores = os.cpu_count() or 1
    sample = args.ref_frames
    _, _, lch = make_inputs(code, sample, SEED, cores)
    for _ in range(args.warmup):
        cpu_oracle_rate(code, lch[: max(cores, 7)], cores)
    times = []
    for _ in range(args.steps):
        _, dt = cpu_oracle_rate(code, lch, cores)
        times.append(dt)
    ms = 1000 * sum(times) / len(times)
    value = sample * code.k * code.k / (ms / 1000)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "bits/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(FRAMES),
            "cpu_baseline": {"value": value, "unit": "bits/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {sample} frames of the workload per step (all 7 Eb/N0 points)"},
            "e2e": {"value": value, "unit": "bits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=FRAMES, help="frames per rank per step (default: the workload)")
    ap.add_argument("--ref-frames", type=int, default=700, help="oracle sample per reference step")
    ap.add_argument("--cpu-frames", type=int, default=3500, help="oracle sample for cpu_baseline")
    ap.add_argument("--e2e-steps", type=int, default=3, help="timed end-to-end calls (after one warm-up call)")
    ap.add_argument("--form", default="persistent", choices=["persistent", "plain"],
                    help="persistent: one kernel per decode with a device-side frame queue; plain: one launch per half")
    ap.add_argument("--plain-steps", type=int, default=3, help="steps of the other form, timed for comparison (0: off)")
    ap.add_argument("--serve-requests", type=int, default=1200, help="requests per offered load in the serving run (0: off)")
    ap.add_argument("--serve-loads", default="250,500,1000,2000,3000", help="offered loads, requests/s")
    ap.add_argument("--other-configs", type=int, default=1, help="1: also measure the C1, C2 and C4 workloads")
    ap.add_argument("--order-source", default="table", choices=["table", "lanes"],
                    help="query order of the headline decode: read from the order table, or enumerated by the lanes")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_10737_gb300 as sg
    from workloads import ebch

    code = ebch(CODE)
    F = args.frames
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    U, X, lch = make_inputs(code, F, rank_seed(rank), cores)
    log(f"inputs: {F} frames in {time.perf_counter() - t0:.1f} s")
    host = torch.from_numpy(lch).pin_memory()
    d_in = host.to(dev)
    c = sg.Code.from_linear_code(code)
    c.order_source(1 if args.order_source == "lanes" else 0)
    log("inputs resident on the device, code tables built")
    # schedule autotuner (set-up, outside the timed region): blocks per SM on a 10,000-frame sample
    sched, sched_ms = c.tune(d_in[: min(F, 10_000)], L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=MAX_ITER)
    log(f"schedule: {sched} blocks/SM (sample ms at 8 / 12: {sched_ms[0]:.1f} / {sched_ms[1]:.1f})")
    n, k = code.n, code.k
    out = dict(bits=torch.empty((F, n * n // 8), dtype=torch.uint8, device=dev),
               half_iters=torch.empty(F, dtype=torch.int32, device=dev),
               status=torch.empty(F, dtype=torch.uint8, device=dev),
               queries=torch.empty(F, dtype=torch.int64, device=dev),
               par_queries=torch.empty(F, dtype=torch.int64, device=dev),
               weight_sum=torch.zeros(1, dtype=torch.int64, device=dev),
               xf_words=torch.zeros(1, dtype=torch.int32, device=dev))

    def step(persistent):
        return sg.product_decode(c, d_in, L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=MAX_ITER, out=out,
                                 persistent=persistent)

    def timed(persistent, steps, warmup, sample_clocks):
        # the clock sampler starts before the warm-up steps, and the warm-up steps
        # do the timed steps' work (the first per-step reduction loads torch's
        # kernel, about a second): nothing one-off stays in the timed region
        clocks = ClockSampler() if sample_clocks else None
        for i in range(warmup):
            t0 = time.perf_counter()
            step(persistent)
            int(out["queries"].sum().item())
            torch.cuda.synchronize()
            log(f"{'persistent' if persistent else 'plain'} warm-up step {i}: {1000 * (time.perf_counter() - t0):.1f} ms")
        out["weight_sum"].zero_()
        if clocks:
            clocks.mark()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        ev0.record(stream)
        t_kern = t_check = 0.0
        launches = kern_launches = 0
        walls = []
        for _ in range(steps):
            tw = time.perf_counter()
            o = step(persistent)
            t_kern += o["timing_ms"][0]
            t_check += o["timing_ms"][1]
            launches += o["launches"]
            kern_launches += 1 if persistent else o["launches"] // 2
            walls.append((round(1000 * (time.perf_counter() - tw), 1), round(o["timing_ms"][0], 1)))
        ev1.record(stream)
        # every step decodes the same batch (decoding is deterministic), so the
        # query total is read once, after the timed region
        qtot = steps * int(out["queries"].sum().item())
        log(f"{'persistent' if persistent else 'plain'} steps (wall ms, kernel ms): {walls}")
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        ms = ev0.elapsed_time(ev1)
        log(f"{'persistent' if persistent else 'plain'} timed: {steps} steps in {ms:.1f} ms")
        ms = max_over_ranks(ms, dist, dev)
        return dict(ms=ms, t_kern=t_kern, t_check=t_check, launches=launches, kern_launches=kern_launches, qtot=qtot,
                    clk=clk, wsum=int(out["weight_sum"].item()))

    int_peak, int_ms = sg.sogrand_int_peak(50_000)  # the integer-pipe ceiling of this GPU, measured
    log(f"integer pipe: {int_peak / 1e12:.2f} Tops/s ({int_ms:.1f} ms)")
    main_persistent = args.form == "persistent"
    other = None
    if args.plain_steps > 0:
        other = timed(not main_persistent, args.plain_steps, 1, False)
    r = timed(main_persistent, args.steps, args.warmup, True)
    ms, t_half, t_check, launches, half_launches, qtot, clk = (r["ms"], r["t_kern"], r["t_check"], r["launches"],
                                                                r["kern_launches"], r["qtot"], r["clk"])
    wsum = r["wsum"]
    value = job_rate(world, F, k * k, args.steps, ms)

    # roofline of the dominant kernel (the half-iteration SISO kernel): integer ALU
    ops = 2 * (qtot + wsum)  # per query: w syndrome XORs + 1 membership test, and w + 1 mass terms (Sec. IV)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    nominal = SMS * INT32_LANES * sm_max * 1e6 / 1e12  # Tops/s
    peak = int_peak / 1e12
    achieved = ops / (t_half / 1000) / 1e12 if t_half > 0 else 0.0
    traffic = None
    # the recorded capture is of the order-table kernel
    same_kernel = main_persistent and args.order_source == "table" and TRAFFIC["csrc_digest"] == csrc_digest()
    if same_kernel:
        traffic = TRAFFIC["bytes_per_frame"] * F
    # HBM side: the LLRs in and decided bits out (algorithmic) and, from the capture, DRAM bytes
    t_launch_s = t_half / 1000 / max(half_launches, 1)
    llr_bytes = F * (4 * n * n + n * n // 8)
    hbm = {"algorithmic_bytes_per_launch": llr_bytes,
           "algorithmic_gbs": llr_bytes / t_launch_s / 1e9 if t_launch_s > 0 else None,
           "dram_gbs": traffic / t_launch_s / 1e9 if traffic is not None and t_launch_s > 0 else None,
           "peak_gbs": measured_hbm_gbs()}
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak if peak else None, "traffic": traffic,
                "traffic_source": TRAFFIC["source"] if traffic is not None else None,
                "kernel": "k_product_persistent" if main_persistent else "k_product_half", "launches": half_launches,
                "avg_launch_ms": t_half / max(half_launches, 1),
                "ops_per_launch": ops / max(half_launches, 1),
                "ops_def": "2 x (queries + summed pattern weights)",
                "kernel_share": t_half / (t_half + t_check) if t_half + t_check else None,
                "peak_def": f"measured: 32-bit LOP3 + IADD lane-ops/s at full occupancy (sogrand_int_peak, "
                            f"{int_ms:.1f} ms kernel); nominal 152 SMs x 128 lanes x {sm_max:.0f} MHz = "
                            f"{nominal:.2f} Tops/s",
                "hbm": hbm,
                "ncu": dict(TRAFFIC["ncu"], source=TRAFFIC["source"]) if same_kernel else None}

    # end to end through the C ABI on host buffers (copies inside the timed region)
    hout = dict(bits=torch.empty((F, n * n // 8), dtype=torch.uint8, pin_memory=True),
                half_iters=torch.empty(F, dtype=torch.int32, pin_memory=True),
                status=torch.empty(F, dtype=torch.uint8, pin_memory=True),
                queries=torch.empty(F, dtype=torch.int64, pin_memory=True))
    sg.product_decode_host(c, host, L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=MAX_ITER, out=hout)  # warm-up
    e2e_ms = []
    for _ in range(max(args.e2e_steps, 1)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        sg.product_decode_host(c, host, L=L_LIST, query_cap=CAP, alpha=ALPHA, max_iter=MAX_ITER, out=hout)
        e2e_ms.append(1000 * (time.perf_counter() - t))
    e2e_t = sum(e2e_ms) / len(e2e_ms)
    log(f"end to end: {e2e_ms}")
    e2e_t = max_over_ranks(e2e_t, dist, dev)
    e2e = {"value": job_rate(world, F, k * k, 1, e2e_t), "unit": "bits/s",
           "h2d_bytes_per_step": int(F * n * n * 4), "d2h_bytes_per_step": int(F * (n * n // 8 + 4 + 1 + 8)),
           "api": "product_decode_host (C ABI, pinned host buffers)"}

    # decoding quality of the timed configuration (BLER/BER/iterations/queries per Eb/N0)
    frames = sg.unpack_bits(out["bits"], n)
    ferr = (frames != X).reshape(F, -1)
    info_err = (frames[:, :k, :k] != U).reshape(F, -1)
    hi = out["half_iters"].cpu().numpy()
    qf = out["queries"].cpu().numpy()
    pq = out["par_queries"].cpu().numpy()
    quality = {}
    for i, e in enumerate(EBN0):
        sel = np.arange(F) % len(EBN0) == i
        quality[f"{e:.2f}"] = {"bler": float(ferr[sel].any(axis=1).mean()), "ber": float(info_err[sel].mean()),
                               "iterations": float(hi[sel].mean() / 2), "queries_per_bit": float(qf[sel].mean() / (n * n)),
                               "par_queries_per_bit": float(pq[sel].mean() / (n * n))}

    serving = None
    if rank == 0 and args.serve_requests > 0:
        serving = serving_bench(sg, torch, args.serve_requests, [float(x) for x in args.serve_loads.split(",")],
                                SEED + 1000 + rank)

    others = None
    if rank == 0 and args.other_configs:
        others = other_configs(sg, torch, cores)

    cpu = None
    if rank == 0 and world == 1 and args.cpu_frames > 0:
        rate, dt = cpu_oracle_rate(code, lch[: args.cpu_frames], cores)
        log(f"cpu baseline: {args.cpu_frames} frames in {dt:.1f} s")
        cpu = {"value": rate, "unit": "bits/s", "cores": cores, "kind": "oracle",
               "sample": f"first {args.cpu_frames} frames of the workload ({args.cpu_frames // 7} per Eb/N0 point), "
                         f"{dt:.1f} s wall"}
        # the same oracle on one host core (a smaller sample of the same frames)
        n1 = min(args.cpu_frames, 140)
        rate1, dt1 = cpu_oracle_rate(code, lch[:n1], 1)
        log(f"cpu baseline, one core: {n1} frames in {dt1:.1f} s")
        cpu["single_core"] = {"value": rate1, "unit": "bits/s", "cores": 1,
                              "sample": f"first {n1} frames of the workload, {dt1:.1f} s wall"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "bits/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(F),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
                "queries_per_s": world * qtot / (ms / 1000), "xf_words": int(out["xf_words"].item()),
                "quality": quality, "serving": serving, "other_configs": others,
                "schedule": {"blocks_per_sm": sched, "remaining_mass_area": ("global" if c.dp_area() else "shared"),
                             "tuned_on": f"{min(F, 10_000)} frames",
                             "sample_ms": {"8": sched_ms[0], "12": sched_ms[1]}},
                "form": ("persistent (one kernel per decode, device-side frame queue)" if main_persistent
                         else "plain (one launch per half iteration)"),
                "order_source": args.order_source}
        if other is not None:
            line["other_form"] = {"form": "plain" if main_persistent else "persistent",
                                  "value": job_rate(world, F, k * k, args.plain_steps, other["ms"]),
                                  "ms_per_step": other["ms"] / args.plain_steps, "steps": args.plain_steps,
                                  "gpu_launches": other["launches"]}
        print(json.dumps(line), flush=True)
    c.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
