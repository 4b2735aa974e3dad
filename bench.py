#!/usr/bin/env python3
"""Benchmark of PEPSI's server evaluation on GB300.

Workload (the paper-shaped configuration): N = 8192 slots = bins, t = 65537,
four RNS primes of 55, 55, 54, 54 bits, constant-weight code ell = 600,
h = 4, mu = 526 server layers; 1024 client items against 2^20 server items
(uniform 64-bit, 102 planted).  Synthetic sets, seeded.

One step = one pepsi_eval (Algorithm 2 with the equality circuit of
Algorithm 1) from device-resident request ciphertexts to a device-resident
result ciphertext.  By default the last ciphertext products of all layers
are rounded once (lazy rescaling, --rescale all); --rescale layer rounds
every layer's product (textbook FV words).  Both are exact and decrypt to
the same result; the line reports the other mode's time too.  The resident server plaintext table (82.7 GB of
64-bit words) is read in full by every step, so the inputs of a step are larger than L2.

Prints one JSON line.  --impl reference times the CPU oracle instead (the
project's plain C reference on the host cores, on a bounded layer sample
scaled to the full 526 layers).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "server eval ms at 1024 x 2^20 items; ct-mult+relin/s; NTT % of HBM roofline"
WL = dict(N=8192, prime_bits=[55, 55, 54, 54], h=4, ell=600, lambda_bar=32, mu=526, m=1024, n=1 << 20, planted=102)
# small case of the same kernels for profiler captures (5.5 GB of resident plaintexts, > L2)
WL_SMALL = dict(WL, mu=35, n=1 << 14)
# large configuration: the 468 GB plaintext table is regenerated per layer chunk
WL_LARGE = dict(N=16384, prime_bits=[55] * 6 + [54] * 2, h=8, ell=128, lambda_bar=40, mu=3487, m=4096, n=1 << 24,
                planted=41)
# the paper's own parameters for its headline run (Section 7, Table 5): h = 8,
# ell = 24, effective bitlength 19, b = N = 8192, 32-bit elements; q per
# Table 3 for h = 5..8 (204 bits, four 51-bit primes)
WL_PAPER_EXACT = dict(N=8192, prime_bits=[51] * 4, h=8, ell=24, lambda_bar=19, mu=526, m=1024, n=1 << 20,
                      planted=102, bits=32)
# the batched and served configurations: server sets of several sizes on
# contexts of both ring sizes and three Hamming weights; mu is the 2^-40
# bin-load rule at each (n, b) (the paper's own value at 2^20 / 8192)
P4, P8 = [55, 55, 54, 54], [55] * 6 + [54] * 2
MIXED = [
    # name, N, prime_bits, h, lambda_bar, ell, log2 n, mu
    ("N=8192 h=2 n=2^16", 8192, P4, 2, 16, 363, 16, 74),
    ("N=8192 h=4 n=2^20", 8192, P4, 4, 32, 600, 20, 526),  # the paper-shaped context and set
    ("N=8192 h=8 n=2^22", 8192, P4, 8, 40, 128, 22, 1869),
    ("N=16384 h=8 n=2^18", 16384, P8, 8, 40, 128, 18, 100),
    ("N=16384 h=4 n=2^16", 16384, P8, 4, 32, 600, 16, 51),
]
SERVE_SETS = (1, 2, 3)  # resident sets of 2^20, 2^22 and 2^18 items, N = 8192 and 16384
HASH_KEY, KEY_SEED, ENC_SEED = 0x5EED, 3, 4
CT_MULT_BATCH = 256  # ciphertext pairs per pepsi_ct_mult call of the ct-mult + relin throughput
WORKLOAD_NAME = ("paper-shaped PSI: N=8192 bins, t=65537, q=4 RNS primes (55,55,54,54 bits), CW code ell=600 h=4, "
                 "mu=526 layers, 1024 client x 2^20 server uniform 64-bit items, 102 planted")
L2_NOTE = "inputs larger than L2: the %.1f GB resident plaintext table is streamed from HBM every step"
RESCALE_NOTE = {"all": "lazy: last ciphertext products of all layers summed exactly, rounded once",
                "layer": "per layer: every ciphertext product rounded (textbook FV)"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x):
    """The largest x over the ranks of the process group (x itself without
    one): the replicas' step time is that of the slowest."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle
def oracle_setup():
    import oracle
    from paper_2310_14565_gb300.workload import make_sets

    oc = oracle.Ctx(N=WL["N"], t=65537, prime_bits=WL["prime_bits"], h=WL["h"], ell=WL["ell"],
                    lambda_bar=WL["lambda_bar"], mu=WL["mu"], hash_key=HASH_KEY)
    sets = make_sets(WL["m"], WL["n"], WL["planted"], bits=64)
    s, rlk = oc.keygen(KEY_SEED)
    rc, Ts, _ = oc.server_table(sets.server)
    rc2, cts, _ = oc.query(s, sets.client, ENC_SEED)
    assert rc == 0 and rc2 == 0
    return oracle, oc, rlk, cts, Ts


RESCALE = {"all": 0xFFFFFFFF, "layer": 1}
# the response is switched to one prime: one ciphertext of 2 x N words (the
# size of the paper's reported response)
RESPONSE_PRIMES = 1


def oracle_sample(oracle, oc, rlk, cts, Ts, layers, layer0=0, lazy=True):
    t = time.perf_counter()
    out = oc.eval(rlk, cts, Ts, layer0=layer0, nlayers=layers, group=max(1, layers) if lazy else 1)
    oc.mod_switch(out, RESPONSE_PRIMES)
    return (time.perf_counter() - t) * 1e3


def cpu_baseline(lazy):
    """The oracle as it stands on the host cores, on a bounded sample: the
    fixed part (request NTT, final relinearisation) plus a layer sample,
    scaled to the workload's 526 layers, in the rounding mode of the run."""
    oracle, oc, rlk, cts, Ts = oracle_setup()
    cores = oracle.get_threads()
    layers = max(2, 2 * cores)
    fixed = oracle_sample(oracle, oc, rlk, cts, Ts, 0, lazy=lazy)
    total = oracle_sample(oracle, oc, rlk, cts, Ts, layers, lazy=lazy)
    est = fixed + (total - fixed) * WL["mu"] / layers
    # the same on one core: the fixed part and two layers
    oracle.set_threads(1)
    try:
        fixed1 = oracle_sample(oracle, oc, rlk, cts, Ts, 0, lazy=lazy)
        total1 = oracle_sample(oracle, oc, rlk, cts, Ts, 2, lazy=lazy)
    finally:
        oracle.set_threads(cores)
    est1 = fixed1 + (total1 - fixed1) * WL["mu"] / 2
    return {"value": round(est, 1), "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": "request NTT + relin/scale (%.0f ms) and %d of 526 layers (%.0f ms), layer part scaled to 526"
                      % (fixed, layers, total - fixed),
            "one_core": {"value": round(est1, 1), "unit": "ms", "cores": 1,
                         "sample": "request NTT + relin/scale (%.0f ms) and 2 of 526 layers (%.0f ms), scaled"
                                   % (fixed1, total1 - fixed1)}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    oracle, oc, rlk, cts, Ts = oracle_setup()
    cores = oracle.get_threads()
    fixed = oracle_sample(oracle, oc, rlk, cts, Ts, 0)
    layers = max(1, cores)
    times = []
    lazy = args.rescale == "all"
    for i in range(args.warmup + args.steps):
        t = oracle_sample(oracle, oc, rlk, cts, Ts, layers, layer0=(i * layers) % (WL["mu"] - layers), lazy=lazy)
        if i >= args.warmup:
            times.append(t)
    per = statistics.median(times)
    est = fixed + (per - fixed) * WL["mu"] / layers
    line = {
        "impl": "reference", "metric": METRIC, "value": round(est, 1), "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "l2": "CPU run", "rescale": RESCALE_NOTE[args.rescale]},
        "cpu_baseline": {"value": round(est, 1), "unit": "ms", "cores": cores, "kind": "oracle",
                         "sample": "each step: request NTT + %d of 526 layers; value scales the layer part to 526"
                                   % layers},
        "e2e": {"value": round(est, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------ batched and served forms
def mixed_contexts(pepsi, torch, main_ctx, main_sid):
    """Contexts, server sets and requests of the batched and served
    configurations (MIXED): every context rounds its layers once, switches
    its response to one prime and is autotuned on one of its requests; four
    distinct requests per set, client sizes log-uniform in [16, 4096] with a
    tenth of each planted, encrypted straight into device memory.  The
    paper-shaped context and set of the main measurement are reused."""
    import math

    import numpy as np

    from paper_2310_14565_gb300.workload import make_sets

    rng = np.random.default_rng(11)
    out = []
    for i, (name, N, bits, h, lb, ell, ln, mu) in enumerate(MIXED):
        seed_items = 1 if (N, h, ln) == (WL["N"], WL["h"], 20) else 200 + i
        if seed_items == 1:
            ctx, sid = main_ctx, main_sid
        else:
            ctx = pepsi.Context(N=N, t=65537, prime_bits=bits, h=h, ell=ell, lambda_bar=lb, mu=mu, hash_key=HASH_KEY,
                                key_seed=KEY_SEED, rescale_group=RESCALE["all"], response_primes=RESPONSE_PRIMES)
            sid = ctx.server_load(make_sets(16, 1 << ln, 0, bits=64, seed_items=seed_items).server)
        reqs, sizes = [], []
        for j in range(4):
            m = int(round(math.exp(rng.uniform(math.log(16), math.log(4096)))))
            sets = make_sets(m, 1 << ln, max(1, m // 10), bits=64, seed_items=seed_items, seed_plant=300 + 10 * i + j)
            cts = torch.empty((ell, 2, len(bits), N), dtype=torch.int64, device="cuda")
            ctx.query(sets.client, 5000 + 10 * i + j, out=cts)
            reqs.append(cts)
            sizes.append(m)
        if seed_items != 1:
            ctx.autotune(sid, reqs[0])
        out.append(dict(name=name, ctx=ctx, sid=sid, reqs=reqs, N=N, client_sizes=sizes,
                        schedule=ctx.schedule()))
    torch.cuda.synchronize()
    return out


def leg_batched(pepsi, torch, mixed, nq=64):
    """Configuration 3: nq queries over the mixed sets (set, request, mode and
    mask seed drawn at random), as nq sequential pepsi_eval calls on one
    stream, as one engine run (a lane of four slots per set, all queries
    submitted at once), and as that schedule captured into one CUDA graph
    and replayed.  Same outputs required; host wall clock for all three."""
    import numpy as np

    rng = np.random.default_rng(12)
    picks = [(int(rng.integers(len(mixed))), int(rng.integers(4)), int(rng.integers(2)), 50 + q) for q in range(nq)]

    def buf(a):
        return torch.zeros((2, RESPONSE_PRIMES, mixed[a]["N"]), dtype=torch.int64, device="cuda")

    outs_seq = [buf(a) for a, _, _, _ in picks]
    outs_eng = [buf(a) for a, _, _, _ in picks]
    eng = pepsi.Engine([(m["ctx"], m["sid"], 4) for m in mixed])

    def sequential():
        for q, (a, r, mode, seed) in enumerate(picks):
            m = mixed[a]
            m["ctx"].eval(m["sid"], m["reqs"][r], mode=mode, mask_seed=seed, out=outs_seq[q])
        torch.cuda.synchronize()

    def engine():
        tickets = [eng.submit(a, mixed[a]["reqs"][r], out=outs_eng[q], mode=mode, mask_seed=seed)[0]
                   for q, (a, r, mode, seed) in enumerate(picks)]
        eng.run()
        for t in tickets:
            eng.wait(t)

    sequential()
    engine()
    times = {}
    for name, f in (("sequential", sequential), ("engine", engine), ("sequential2", sequential), ("engine2", engine)):
        t0 = time.perf_counter()
        f()
        times[name] = time.perf_counter() - t0
    same = all(torch.equal(outs_seq[q], outs_eng[q]) for q in range(nq))
    t_seq = min(times["sequential"], times["sequential2"])
    t_eng = min(times["engine"], times["engine2"])
    # the same batch's whole schedule captured into one CUDA graph and replayed
    for q in range(nq):
        outs_eng[q].zero_()
    torch.cuda.synchronize()
    for q, (a, r, mode, seed) in enumerate(picks):
        eng.submit(a, mixed[a]["reqs"][r], out=outs_eng[q], mode=mode, mask_seed=seed)
    graph = eng.capture()
    graph.launch()
    same_graph = all(torch.equal(outs_seq[q], outs_eng[q]) for q in range(nq))
    t_graph = []
    for _ in range(2):
        t0 = time.perf_counter()
        graph.launch()
        t_graph.append(time.perf_counter() - t0)
    graph.close()
    st = eng.stats()
    eng.close()
    per_set = {m["name"]: sum(1 for a, _, _, _ in picks if a == i) for i, m in enumerate(mixed)}
    return {"queries": nq, "sets": per_set, "engine_queries_per_s": round(nq / t_eng, 2),
            "sequential_queries_per_s": round(nq / t_seq, 2), "speedup": round(t_seq / t_eng, 3),
            "engine_s": round(t_eng, 4), "sequential_s": round(t_seq, 4), "identical_outputs": bool(same),
            "graph_queries_per_s": round(nq / min(t_graph), 2), "graph_identical_outputs": bool(same_graph),
            "engine_peak_state_gb": round(st["bytes_peak"] / 1e9, 2), "lane_slots": 4,
            "client_sizes": {m["name"]: m["client_sizes"] for m in mixed},
            "schedules": {m["name"]: m["schedule"] for m in mixed},
            "timing": "host wall clock over the whole batch, GPU synchronised at its end; best of two"}


def leg_serve(pepsi, torch, mixed, total=120, loads=(0.5, 0.9, 1.5)):
    """Configuration 5: Poisson arrivals over the resident sets of 2^20, 2^22
    and 2^18 items (N = 8192, 8192, 16384; each arrival picks a set and one
    of its four requests at random), at fractions of the sequential
    capacity.  Sequential: one pepsi_eval at a time in arrival order,
    synchronised.  Engine: the engine's thread serves submissions made at
    the arrival times.  Latency = completion - scheduled arrival."""
    import numpy as np

    lanes = [mixed[a] for a in SERVE_SETS]
    svc = []
    for m in lanes:  # sequential service time per set
        o = torch.zeros((2, RESPONSE_PRIMES, m["N"]), dtype=torch.int64, device="cuda")
        m["ctx"].eval(m["sid"], m["reqs"][0], out=o)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in range(4):
            m["ctx"].eval(m["sid"], m["reqs"][r], out=o)
            torch.cuda.synchronize()
        svc.append((time.perf_counter() - t0) / 4)
    capacity = 1.0 / float(np.mean(svc))
    eng = pepsi.Engine([(m["ctx"], m["sid"], 4) for m in lanes])
    runs, identical = [], True
    for li, load in enumerate(loads):
        rng = np.random.default_rng(13 + li)
        arrivals = np.cumsum(rng.exponential(1.0 / (load * capacity), size=total))
        pick = rng.integers(len(lanes), size=total)
        reqi = rng.integers(4, size=total)
        seq_out = [torch.zeros((2, RESPONSE_PRIMES, lanes[pick[q]]["N"]), dtype=torch.int64, device="cuda")
                   for q in range(total)]
        eng_out = [torch.zeros_like(x) for x in seq_out]
        torch.cuda.synchronize()
        # sequential server
        lat, t0 = [], time.perf_counter()
        for q in range(total):
            now = time.perf_counter() - t0
            if arrivals[q] > now:
                time.sleep(arrivals[q] - now)
            m = lanes[pick[q]]
            m["ctx"].eval(m["sid"], m["reqs"][reqi[q]], mode=q % 2, mask_seed=q, out=seq_out[q])
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - t0 - arrivals[q])
        span_seq = time.perf_counter() - t0
        # the engine, continuous batching
        eng.start()
        tickets, late, t0 = [], [], time.perf_counter()
        for q in range(total):
            now = time.perf_counter() - t0
            if arrivals[q] > now:
                time.sleep(arrivals[q] - now)
            late.append(max(0.0, time.perf_counter() - t0 - arrivals[q]))
            m = lanes[pick[q]]
            tickets.append(eng.submit(int(pick[q]), m["reqs"][reqi[q]], out=eng_out[q], mode=q % 2, mask_seed=q)[0])
        lat_e = [late[q] + eng.wait(t) * 1e-3 for q, t in enumerate(tickets)]
        span_eng = time.perf_counter() - t0
        eng.stop()
        identical &= all(torch.equal(seq_out[q], eng_out[q]) for q in range(total))
        for policy, ls, span in (("sequential", lat, span_seq), ("engine", lat_e, span_eng)):
            ms = np.array(ls) * 1e3
            runs.append({"load": load, "policy": policy, "requests": total,
                         "p50_ms": round(float(np.percentile(ms, 50)), 2),
                         "p99_ms": round(float(np.percentile(ms, 99)), 2),
                         "queries_per_s": round(total / span, 2)})
    st = eng.stats()
    eng.close()
    return {"sets": [m["name"] for m in lanes], "sequential_service_ms": [round(x * 1e3, 3) for x in svc],
            "capacity_queries_per_s": round(capacity, 2), "runs": runs, "identical_outputs": bool(identical),
            "engine_peak_state_gb": round(st["bytes_peak"] / 1e9, 2),
            "engine_budget_gb": round(st["budget"] / 1e9, 1), "lane_slots": 4,
            "arrivals": "Poisson, rate = load x sequential capacity; set and request uniform; modes alternate"}


# HBM the large configuration leaves free of resident plaintexts: its evaluation
# scratch at chunk 128 (the regenerated chunk's 64-bit plaintexts, 17.2 GB; circuit
# buffers, 4.3 GB; h' of the resident layers, 2 MB each) and the four-request
# batch's h' of every resident layer (double-buffered, 16.8 MB per layer), with a
# margin: about 1930 of the 3487 layers stay resident.
LARGE_RESERVE_GB = 70


def leg_large(pepsi, torch, steps=3, chunk=128, reserve_gb=None):
    """Configuration 4 (large) in the default line: N = 16384, eight primes,
    h = 8, ell = 128, mu = 3487, 4096 client x 2^24 server items; the
    resident prefix of the 468 GB table in 7-byte words, the rest
    regenerated per chunk.  A few steps after one warm-up.  reserve_gb: HBM
    left free of resident plaintexts for the evaluation's scratch (None: the
    library's default budget, 0.6 of the free memory)."""
    from paper_2310_14565_gb300.workload import make_sets

    W = WL_LARGE
    N, k = W["N"], len(W["prime_bits"])
    resident = 0
    free, _ = torch.cuda.mem_get_info()
    if reserve_gb is not None:
        resident = max(1, int(free - reserve_gb * 1e9))
    # the longest prefix of layers that fits the budget stays resident
    layer_bytes = W["ell"] * k * N * 7
    resident_layers = min(W["mu"], int((resident or 0.6 * free) // layer_bytes))
    ctx = pepsi.Context(N=N, t=65537, prime_bits=W["prime_bits"], h=W["h"], ell=W["ell"],
                        lambda_bar=W["lambda_bar"], mu=W["mu"], hash_key=HASH_KEY, key_seed=KEY_SEED,
                        rescale_group=RESCALE["all"], response_primes=RESPONSE_PRIMES, plaintext_bytes=7,
                        resident_bytes=resident)
    ctx.set_schedule(chunk=chunk)
    sets = make_sets(W["m"], W["n"], W["planted"], bits=64)
    t0 = time.perf_counter()
    sid = ctx.server_load(sets.server)
    offline = time.perf_counter() - t0
    cts = torch.empty((W["ell"], 2, k, N), dtype=torch.int64, device="cuda")
    ctx.query(sets.client, ENC_SEED, out=cts)
    out = torch.zeros((2, RESPONSE_PRIMES, N), dtype=torch.int64, device="cuda")
    ctx.eval(sid, cts, out=out)
    torch.cuda.synchronize()
    slots, budget = ctx.decrypt(out)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.eval(sid, cts, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ctx.profile(True)
    ctx.eval(sid, cts, out=out)
    prof = ctx.profile_read()
    ctx.profile(False)
    total_ms = sum(v[1] for v in prof.values())
    # four requests in one pepsi_eval_batch call: each regenerated plaintext chunk
    # serves all four (one shared multiply-accumulate launch per chunk)
    ctx.set_schedule(batch_requests=4)
    reqs = [cts]
    for i in range(3):
        r = torch.empty_like(cts)
        ctx.query(sets.client, ENC_SEED + 1 + i, out=r)
        reqs.append(r)
    bout = [torch.zeros_like(out) for _ in reqs]
    sout = [torch.zeros_like(out) for _ in reqs]
    e0.record(stream)
    for i in range(4):
        ctx.eval(sid, reqs[i], out=sout[i])
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    e0.record(stream)
    ctx.eval_batch([sid] * 4, reqs, outs=bout)
    e1.record(stream)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1)
    same = all(torch.equal(bout[i], sout[i]) for i in range(4))
    res = {"workload": "N=16384, 8 primes (55x6, 54x2), h=8, ell=128, mu=3487, 4096 client x 2^24 server items, "
                       "41 planted; 7-byte resident prefix, the rest regenerated per chunk",
           "ms_per_step": round(ms, 1), "steps": steps, "layer_chunk": chunk,
           "resident_layers": resident_layers, "resident_gb": round(resident_layers * layer_bytes / 1e9, 1),
           "batched": {"requests": 4, "ms_per_request": round(batch_ms / 4, 1),
                       "sequential_ms_per_request": round(seq_ms / 4, 1), "speedup": round(seq_ms / batch_ms, 3),
                       "identical_outputs": bool(same),
                       "note": "pepsi_eval_batch with batch_requests = 4: one plaintext regeneration per chunk "
                               "for the four requests"},
           "correct": bool(int(slots.sum()) == W["planted"] and budget > 0), "noise_budget_bits": round(budget, 2),
           "offline_server_load_s": round(offline, 2),
           "ptgen_share": round(prof["ptgen"][1] / total_ms, 3) if total_ms else None,
           "kernel_ms_per_step": {n: round(v[1], 2) for n, v in prof.items() if v[0]}}
    ctx.close()
    return res


# --------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import paper_2310_14565_gb300 as pepsi
    from paper_2310_14565_gb300 import build as _build
    from paper_2310_14565_gb300.workload import make_sets

    if not os.path.exists(pepsi.LIB_PATH):
        _build.build()
    N, k = WL["N"], len(WL["prime_bits"])
    if args.chunk:
        os.environ["PEPSI_CHUNK"] = str(args.chunk)
    # the auxiliary base is sized for one rounding over all layers; the
    # rounding mode of each evaluation is then a context setting
    ctx = pepsi.Context(N=N, t=65537, prime_bits=WL["prime_bits"], h=WL["h"], ell=WL["ell"],
                        lambda_bar=WL["lambda_bar"], mu=WL["mu"], hash_key=HASH_KEY, key_seed=KEY_SEED,
                        rescale_group=RESCALE["all"], response_primes=RESPONSE_PRIMES,
                        plaintext_bytes=args.plaintext_bytes or (7 if args.case == "large" else 8))
    ctx.set_rescale_group(RESCALE[args.rescale])
    pbytes = ctx.plaintext_bytes
    sets = make_sets(WL["m"], WL["n"], WL["planted"], bits=WL.get("bits", 64))
    t0 = time.perf_counter()
    sid = ctx.server_load(sets.server)
    offline_ms = (time.perf_counter() - t0) * 1e3
    cts_np, where = ctx.query(sets.client, ENC_SEED)
    shape = cts_np.shape
    cts_pinned = torch.from_numpy(cts_np.view("int64")).pin_memory()
    cts_dev = cts_pinned.cuda()
    out_dev = torch.empty((2, RESPONSE_PRIMES, N), dtype=torch.int64, device="cuda")
    out_pinned = torch.empty((2, RESPONSE_PRIMES, N), dtype=torch.int64).pin_memory()
    stream = torch.cuda.current_stream()

    def step():
        ctx.eval(sid, cts_dev, out=out_dev)

    # the layer-chunk schedule, autotuned on this request unless --chunk fixes
    # it (words do not depend on it)
    chunk = args.chunk if args.chunk else ctx.autotune(sid, cts_dev)
    if args.ntt_threads:
        ctx.set_schedule(ntt_threads=args.ntt_threads)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness of the timed configuration (outside the timed region)
    slots, budget = ctx.decrypt(out_dev)
    # every planted item matches; at a short effective bitlength an H0
    # collision may add a match (about 0.75 per query at lambda_bar = 19)
    correct = (int(slots.sum()) == WL["planted"] or (WL["lambda_bar"] < 32 and int(slots.sum()) >= WL["planted"])) \
        and budget > 0

    ctx.profile(False)  # resets the launch counters
    clocks = Clocks(local)
    time.sleep(0.5)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    prof_counts = ctx.profile_read()
    launches = sum(v[0] for v in prof_counts.values())
    ms = max_over_ranks(ms)

    # per-kernel CUDA-event timing pass (same workload, events on the launching stream)
    ctx.profile(True)
    psteps = max(3, min(args.steps, 20))
    for _ in range(psteps):
        step()
    prof = ctx.profile_read()
    ctx.profile(False)
    mac_launches, mac_ms = prof["mac"]
    mac_launches_per_eval = mac_launches / psteps
    # algorithmic bytes of the MAC per evaluation: the plaintext table (mu*ell*k*N words of
    # pbytes = 7 or 8 bytes), the prepared request (ell*2*k*N words of 8 bytes and their
    # 4-byte half sums, read once by each launch) and h' (mu*2*k*N words of 8 bytes)
    mu, ell = WL["mu"], WL["ell"]
    mac_bytes_eval = (pbytes * mu * ell * k * N + 12 * mac_launches_per_eval * ell * 2 * k * N +
                      8 * mu * 2 * k * N)
    mac_launch_ms = mac_ms / mac_launches
    achieved = mac_bytes_eval / mac_launches_per_eval / (mac_launch_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = stored_traffic() if args.case == "paper" and pbytes == 8 else None

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    for _ in range(2):
        ctx.eval(sid, cts_pinned, out=out_pinned)
    e2e = []
    for _ in range(max(3, min(args.steps, 20))):
        t = time.perf_counter()
        ctx.eval(sid, cts_pinned, out=out_pinned)
        e2e.append((time.perf_counter() - t) * 1e3)
    e2e_ms = statistics.median(e2e)

    # the same evaluation captured once in a CUDA graph and replayed
    graph = torch.cuda.CUDAGraph()
    gstream = torch.cuda.Stream()
    gstream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(graph, stream=gstream, capture_error_mode="relaxed"):
        ctx.eval(sid, cts_dev, out=out_dev, stream=torch.cuda.current_stream())
    graph.replay()
    torch.cuda.synchronize()
    gsteps = max(3, min(args.steps, 10))
    e0.record(stream)
    for _ in range(gsteps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / gsteps
    gslots, _ = ctx.decrypt(out_dev)
    graph_line = {"ms_per_step": round(graph_ms, 3), "steps": gsteps, "same_decryption": bool((gslots == slots).all())}
    del graph

    # the other rounding mode on the same context and table (same outputs after decryption)
    other = "layer" if args.rescale == "all" else "all"
    ctx.set_rescale_group(RESCALE[other])
    for _ in range(2):
        step()
    oslots, obudget = ctx.decrypt(out_dev)
    osteps = max(3, min(args.steps, 10))
    e0.record(stream)
    for _ in range(osteps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    other_line = {"rescale": RESCALE_NOTE[other], "ms_per_step": round(e0.elapsed_time(e1) / osteps, 3),
                  "noise_budget_bits": round(obudget, 2),
                  "same_decryption": bool((oslots == slots).all()), "steps": osteps}
    ctx.set_rescale_group(RESCALE[args.rescale])

    if args.case in ("large", "paper-exact"):
        line = {"metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": WORKLOAD_NAME, "rescale": RESCALE_NOTE[args.rescale],
                           "l2": ("inputs larger than L2 (plaintext chunks of %.1f GB)" % (chunk * 0.134)
                                  if args.case == "large" else
                                  "inputs larger than L2: the %.1f GB resident plaintext table is read every step"
                                  % (WL["mu"] * WL["ell"] * k * N * pbytes / 1e9)),
                           "plaintext_bytes_per_word": pbytes},
                "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": int(cts_np.nbytes),
                        "d2h_bytes_per_step": int(out_pinned.numel() * 8)},
                "other_rounding": other_line, "cuda_graph": graph_line, "layer_chunk": chunk,
                "correct": correct, "noise_budget_bits": round(budget, 2),
                "offline_server_load_ms": round(offline_ms, 1),
                "kernel_ms_per_step": {name: round(v[1] / psteps, 3) for name, v in prof.items() if v[0]},
                "gpu_launches": int(launches), "clocks": clk}
        if rank == 0:
            print(json.dumps(line), flush=True)
        ctx.close()
        return 0

    # batched form: 4 requests on the same server set in one pepsi_eval_batch call,
    # against 4 sequential pepsi_eval calls (same outputs)
    nbq = 4
    reqs = [cts_dev] + [torch.from_numpy(ctx.query(sets.client, ENC_SEED + 1 + i)[0].view("int64")).cuda()
                        for i in range(nbq - 1)]
    bouts = [torch.empty((2, RESPONSE_PRIMES, N), dtype=torch.int64, device="cuda") for _ in range(nbq)]
    souts = [torch.empty((2, RESPONSE_PRIMES, N), dtype=torch.int64, device="cuda") for _ in range(nbq)]
    for _ in range(2):
        ctx.eval_batch([sid] * nbq, reqs, outs=bouts)
        for i in range(nbq):
            ctx.eval(sid, reqs[i], out=souts[i])
    torch.cuda.synchronize()
    same = all(torch.equal(bouts[i], souts[i]) for i in range(nbq))
    breps = max(2, min(args.steps // nbq, 8))
    e0.record(stream)
    for _ in range(breps):
        ctx.eval_batch([sid] * nbq, reqs, outs=bouts)
    e1.record(stream)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / breps
    e0.record(stream)
    for _ in range(breps):
        for i in range(nbq):
            ctx.eval(sid, reqs[i], out=souts[i])
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / breps
    ctx.profile(True)
    ctx.eval_batch([sid] * nbq, reqs, outs=bouts)
    bprof = ctx.profile_read()
    ctx.profile(False)
    batched = {"requests": nbq, "ms_per_request": round(batch_ms / nbq, 3),
               "kernel_ms_per_call": {n: round(v[1], 3) for n, v in bprof.items() if v[0]},
               "sequential_ms_per_request": round(seq_ms / nbq, 3), "speedup": round(seq_ms / batch_ms, 3),
               "queries_per_s": round(1e3 * nbq / batch_ms, 2), "identical_outputs": bool(same)}
    del reqs, bouts, souts

    # ct-mult + relin throughput: a batch of 256 pairs at the workload's parameters (about
    # the 263 layers of one circuit chunk; 64 pairs fill 1.1 waves of the transforms)
    nb = min(CT_MULT_BATCH, WL["ell"] // 2)
    a = torch.empty((nb, 2, k, N), dtype=torch.int64, device="cuda")
    a.copy_(cts_dev[:nb])
    b = cts_dev[nb:2 * nb].contiguous()
    o2 = torch.empty((nb, 2, k, N), dtype=torch.int64, device="cuda")
    for _ in range(2):
        ctx.ct_mult(a, b, nb, o2, relin=True)
    torch.cuda.synchronize()
    e0.record(stream)
    reps = 10
    for _ in range(reps):
        ctx.ct_mult(a, b, nb, o2, relin=True)
    e1.record(stream)
    torch.cuda.synchronize()
    mult_per_s = nb * reps / (e0.elapsed_time(e1) * 1e-3)

    # NTT bandwidth: forward + inverse over the whole request (1200 ciphertext components x 4 primes)
    polys = cts_dev.clone()
    count = shape[0] * 2
    for _ in range(2):
        ctx.ntt(polys, count)
        ctx.ntt(polys, count, inverse=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(5):
        ctx.ntt(polys, count)
        ctx.ntt(polys, count, inverse=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ntt_ms = e0.elapsed_time(e1) / 10
    ntt_gbs = 2 * 8 * N * k * count / (ntt_ms * 1e-3) / 1e9

    # integer-pipe peaks (measured here, multipliers that change every step) and the
    # MAC's use of the wide multiply-add: 2 components x 3 Karatsuba split products
    # per plaintext word and request
    wide_peak = pepsi.int_peak(pepsi.INT_MAD_WIDE)
    mul_peak = pepsi.int_peak(pepsi.INT_MUL_WIDE)
    mad32_peak = pepsi.int_peak(pepsi.INT_MAD_LO)
    mac_wide_rate = 6.0 * mu * ell * k * N / (mac_launch_ms * 1e-3)
    bmac_ms = batched["kernel_ms_per_call"].get("mac", 0.0)
    bmac_rate = 6.0 * nbq * mu * ell * k * N / (bmac_ms * 1e-3) if bmac_ms else 0.0
    # the circuit kernels' share of the heavy multiply-add pipe: busy SM-cycles per
    # evaluation (full-size ncu counters) over this run's CUDA-event time of the class
    cyc = stored_pipe_cycles() if pbytes == 8 and args.rescale == "all" else None
    circuits = None
    if cyc:
        clock_hz = (clk.get("sm_mhz") or 2070.0) * 1e6
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        circuits = {}
        for cls in ("ntt", "lift", "tensor", "scale_round", "relin", "mac"):
            launches_c, ms_c = prof.get(cls, (0, 0.0))
            if cls in cyc and ms_c > 0:
                per_eval_s = ms_c / psteps * 1e-3
                circuits[cls] = round(cyc[cls] / (per_eval_s * clock_hz * sms), 3)
    int_pipe = {"mad_wide_u32_per_s": round(wide_peak / 1e12, 3), "mul_wide_u32_per_s": round(mul_peak / 1e12, 3),
                "mad_u32_per_s": round(mad32_peak / 1e12, 3), "unit": "T ops/s",
                "mac_mad_wide_frac": round(mac_wide_rate / wide_peak, 4),
                "batched_mac_mad_wide_frac": round(bmac_rate / wide_peak, 4),
                "circuits_heavy_pipe_busy": circuits,
                "note": "the MACs issue 6 mad.wide.u32 per plaintext word and request (2 components x 3 Karatsuba "
                        "split products); peaks measured with multipliers that change every step; "
                        "circuits_heavy_pipe_busy: fraction of the SMs' heavy multiply-add pipe cycles each kernel "
                        "class keeps busy (profiles/circuit_pipes_paper.md counters / this run's event times)"}

    line = {
        "metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "l2": L2_NOTE % (mu * ell * k * N * pbytes / 1e9), "parallelism": "replicas" if ws > 1 else "1 GPU",
                   "resident_plaintexts_gb": round(mu * ell * k * N * pbytes / 1e9, 1),
                   "plaintext_bytes_per_word": pbytes,
                   "rescale": RESCALE_NOTE[args.rescale],
                   "response": "switched to one prime (2 x N words)"},
        "other_rounding": other_line,
        "cuda_graph": graph_line,
        "layer_chunk": chunk,
        "correct": correct, "noise_budget_bits": round(budget, 2),
        "offline_server_load_ms": round(offline_ms, 1),
        "ct_mult_relin_per_s": round(mult_per_s, 1), "ct_mult_relin_batch": nb,
        "ntt": {"gbs": round(ntt_gbs, 1), "hbm_frac": round(ntt_gbs / peak, 4),
                "note": "forward+inverse over 1200x4 polynomials of N=8192, 2*8*N bytes per polynomial"},
        "roofline": {"bound": "hbm", "kernel": "k_mac", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": peak_kind, "launches_per_step": mac_launches_per_eval,
                     "avg_launch_ms": round(mac_launch_ms, 4)},
        "kernel_ms_per_step": {name: round(v[1] / psteps, 3) for name, v in prof.items() if v[0]},
        "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": int(cts_np.nbytes),
                "d2h_bytes_per_step": int(out_pinned.numel() * 8)},
        "batched": batched,
        "int_pipe": int_pipe,
        "schedule": ctx.schedule(),
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    extra = args.case == "paper" and not args.no_extra_legs and ws == 1
    if extra:
        # configurations 3 and 5 (batched and served), then 4 (large) after
        # the paper-shaped tables are released
        mixed = mixed_contexts(pepsi, torch, ctx, sid)
        line["batched_mixed"] = leg_batched(pepsi, torch, mixed)
        line["serving"] = leg_serve(pepsi, torch, mixed)
        for m in mixed:
            if m["ctx"] is not ctx:
                m["ctx"].close()
        del mixed
    ctx.close()
    if extra:
        del cts_dev, cts_pinned, out_dev, out_pinned
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        line["large"] = leg_large(pepsi, torch, reserve_gb=LARGE_RESERVE_GB)
    if rank == 0 and args.gpus == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.rescale == "all")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_sweep_h(args):
    """GPU counterpart of the paper's Figure 5 (Section 6.2): runtime of the
    server computation for one client batch against one server batch
    (gamma = mu = 1) as a function of the Hamming weight h, for effective
    bitlengths 16, 32, 48.  (N, q) per Table 3 with q split evenly into
    primes of at most 60 bits, ell by Eq. 1; h in {1, 2, 4, 8} (the weights
    of the equality circuit); pairs whose code length exceeds the library's
    65535 (16-bit codeword positions) are skipped.  Also the communication-optimal h of the request model."""
    import torch

    import paper_2310_14565_gb300 as pepsi
    from paper_2310_14565_gb300 import build as _build
    from paper_2310_14565_gb300.workload import make_sets

    if not os.path.exists(pepsi.LIB_PATH):
        _build.build()
    torch.cuda.set_device(0)
    rows = []
    for lb in (16, 32, 48):
        for h in (1, 2, 4, 8):
            bits, ell, ln, lq = pepsi.request_bits(lb, h, 4096)
            row = {"lambda_bar": lb, "h": h, "ell": ell, "log2_n": ln, "log2_q": lq,
                   "request_mb": round(bits / 8e6, 3)}
            if ell > 65535:
                row["skipped"] = "code length above 65535"
                rows.append(row)
                continue
            N = 1 << ln
            k = -(-lq // 60)
            prime_bits = [lq // k + (1 if i < lq % k else 0) for i in range(k)]
            ctx = pepsi.Context(N=N, t=65537, prime_bits=prime_bits, h=h, ell=ell, lambda_bar=lb, mu=1,
                                hash_key=HASH_KEY, key_seed=KEY_SEED)
            for seed in range(100, 150):  # mu = 1: redraw until no two server items share a bin
                sets = make_sets(N // 2, 8, 4, bits=64, seed_items=seed, seed_plant=seed + 1)
                try:
                    sid = ctx.server_load(sets.server)
                    break
                except pepsi.PepsiError as err:
                    if err.code != pepsi.E_BIN_OVERFLOW:
                        raise
            cts_np, where = ctx.query(sets.client, ENC_SEED)
            cts = torch.from_numpy(cts_np.view("int64")).cuda()
            out = torch.empty((2, k, N), dtype=torch.int64, device="cuda")
            stream = torch.cuda.current_stream()
            for _ in range(3):
                ctx.eval(sid, cts, out=out)
            torch.cuda.synchronize()
            slots, budget = ctx.decrypt(out)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 10
            e0.record(stream)
            for _ in range(reps):
                ctx.eval(sid, cts, out=out)
            e1.record(stream)
            torch.cuda.synchronize()
            row.update({"prime_bits": prime_bits, "ms": round(e0.elapsed_time(e1) / reps, 3),
                        "noise_budget_bits": round(budget, 2), "correct": bool(int(slots.sum()) == 4 and budget > 0)})
            rows.append(row)
            ctx.close()
            del cts, out
    comp = {}
    for lb in (16, 32, 48):
        done = [r for r in rows if r["lambda_bar"] == lb and r.get("correct")]
        comp[lb] = min(done, key=lambda r: (r["ms"], r["h"]))["h"] if done else None
    line = {"metric": "server computation ms per (client batch, server batch) vs Hamming weight (Figure 5 on GB300)",
            "unit": "ms", "data": "synthetic", "n_gpus": 1,
            "config": {"workload": "gamma = mu = 1, b = N bins, N and q per Table 3, m = N/2 client items, "
                                   "8 server items (4 shared), per-layer rounding"},
            "rows": rows, "comp_optimal_h_of_1_2_4_8": comp,
            "comm_optimal_h": {lb: pepsi.comm_optimal_h(lb, 4096) for lb in (16, 32, 48)},
            "paper_comp_optimal_h": {"16": 4, "32": 8, "48": 8, "cite": "Figure 5 caption (CPU, SEAL, one thread)"}}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """The served form alone (configuration 5): the paper-shaped context and
    the other resident sets of the mixed configurations, Poisson arrivals at
    several fractions of the sequential capacity, the engine's thread
    against one pepsi_eval at a time; one JSON line."""
    import torch

    import paper_2310_14565_gb300 as pepsi
    from paper_2310_14565_gb300 import build as _build
    from paper_2310_14565_gb300.workload import make_sets

    if not os.path.exists(pepsi.LIB_PATH):
        _build.build()
    torch.cuda.set_device(0)
    ctx = pepsi.Context(N=WL["N"], t=65537, prime_bits=WL["prime_bits"], h=WL["h"], ell=WL["ell"],
                        lambda_bar=WL["lambda_bar"], mu=WL["mu"], hash_key=HASH_KEY, key_seed=KEY_SEED,
                        rescale_group=RESCALE["all"], response_primes=RESPONSE_PRIMES)
    sets = make_sets(WL["m"], WL["n"], WL["planted"], bits=64)
    sid = ctx.server_load(sets.server)
    cts = torch.from_numpy(ctx.query(sets.client, ENC_SEED)[0].view("int64")).cuda()
    ctx.autotune(sid, cts)
    mixed = mixed_contexts(pepsi, torch, ctx, sid)
    res = leg_serve(pepsi, torch, mixed, total=max(120, args.steps * 4), loads=(0.5, 0.9, 1.2, 1.5))
    line = {"metric": "serving latency and throughput under Poisson arrivals (configuration 5)", "unit": "ms",
            "n_gpus": 1, "data": "synthetic", "config": {"workload": "resident sets " + ", ".join(res["sets"])},
            **res}
    print(json.dumps(line), flush=True)
    for m in mixed:
        if m["ctx"] is not ctx:
            m["ctx"].close()
    ctx.close()
    return 0


def stored_traffic():
    """DRAM bytes of one full k_mac launch, from the committed small-case
    capture of the same kernel (35 layers) scaled by the layers it
    processes: the plaintext reads and h' writes grow with the layers, the
    request is read once per launch.  None unless the capture was taken on
    the current kernel source."""
    path = os.path.join(ROOT, "profiles", "k_mac_small_dram.md")
    if not os.path.exists(path) or WL["mu"] != 526:
        return None
    for line in open(path):
        if line.startswith("machine-readable:"):
            kv = dict(f.split("=") for f in line.split()[1:])
            if kv.get("kernel_rev") != prof_rev():
                return None
            per_layer = (int(kv["traffic_bytes_per_launch"]) - int(kv["request_bytes"])) / int(kv["layers"])
            return int(round(per_layer * WL["mu"] + int(kv["request_bytes"])))
    return None


def kernels_rev():
    """Identity of all device code (kernels.cu, ntt_block.cuh, common.cuh),
    comments and blank lines removed: stored pipe counters apply while it
    matches."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in ("kernels.cu", "ntt_block.cuh", "common.cuh"):
        text = open(os.path.join(ROOT, "paper_2310_14565_gb300", "csrc", f)).read()
        code = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in code if ln).encode())
    return h.hexdigest()[:16]


def stored_pipe_cycles():
    """Busy SM-cycles of the heavy multiply-add pipe per evaluation and kernel
    class, from the committed full-size ncu summary, if it was taken on the
    current device code (else None)."""
    path = os.path.join(ROOT, "profiles", "circuit_pipes_paper.md")
    if not os.path.exists(path) or WL["mu"] != 526:
        return None
    for line in open(path):
        if line.startswith("machine-readable:"):
            kv = dict(f.split("=") for f in line.split()[1:])
            if kv.pop("kernel_rev", None) != kernels_rev():
                return None
            return {c: int(v.split(",")[0]) for c, v in kv.items()}
    return None


def prof_rev():
    """Identity of the MAC kernel source, to tell whether stored counters are
    current: a hash of its code with comments and blank lines removed, so
    that edits of comments alone keep the counters."""
    import hashlib
    import re

    src = os.path.join(ROOT, "paper_2310_14565_gb300", "csrc", "kernels.cu")
    text = open(src).read()
    start = text.find("// ------------------------------------------------------- fused MAC")
    end = text.find("// ---------------------------------------------------- RNS conversions")
    code = [re.sub(r"//.*$", "", ln).rstrip() for ln in text[start:end].splitlines()]
    return hashlib.sha256("\n".join(ln for ln in code if ln).encode()).hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-legs", action="store_true",
                    help="skip the batched (64 mixed queries), serving and large legs of the default run")
    ap.add_argument("--plaintext-bytes", type=int, choices=[0, 7, 8], default=0,
                    help="storage of the resident plaintexts per word: 8 (64-bit words) or 7 (three planes); "
                         "0: 7 for the large case, whose table is only partly resident, else 8")
    ap.add_argument("--chunk", type=int, default=0,
                    help="circuit chunk in layers (default: autotuned on the request)")
    ap.add_argument("--ntt-threads", type=int, default=0,
                    help="threads per transform block (default: autotuned with the chunk, or the default for N "
                         "when --chunk fixes the chunk)")
    ap.add_argument("--rescale", choices=["all", "layer"], default="all",
                    help="all: one rounding of the layers' last products per evaluation (lazy rescaling); "
                         "layer: every product rounded (textbook FV words)")
    ap.add_argument("--case", choices=["paper", "small", "large", "paper-exact", "sweep-h", "serve"], default="paper",
                    help="small: the same kernels on 2^14 server items (mu=35), for profiler captures; "
                         "large: N=16384, 8 primes, h=8, 4096 x 2^24 items, streamed plaintexts")
    args = ap.parse_args()
    global WORKLOAD_NAME
    if args.case == "small":
        WL.update(WL_SMALL)
        WORKLOAD_NAME = WORKLOAD_NAME.replace("mu=526", "mu=35").replace("2^20", "2^14") + " (profiling case)"
        args.no_cpu_baseline = True
    elif args.case == "paper-exact":
        WL.update(WL_PAPER_EXACT)
        WORKLOAD_NAME = ("the paper's own headline parameters: N=b=8192, t=65537, q=4 RNS primes (51 bits each, "
                         "204 bits per Table 3), CW code ell=24 h=8, effective bitlength 19, mu=526, 1024 client x "
                         "2^20 server uniform 32-bit items, 102 planted (paper: 0.83 s online on an unstated CPU)")
        args.no_cpu_baseline = True
    elif args.case == "large":
        WL.update(WL_LARGE)
        WORKLOAD_NAME = ("large PSI: N=16384 bins, t=65537, q=8 RNS primes (55x6, 54x2 bits), CW code ell=128 h=8, "
                         "mu=3487 layers, 4096 client x 2^24 server uniform 64-bit items, 41 planted, plaintexts "
                         "regenerated per layer chunk")
        args.no_cpu_baseline = True
    if args.warmup < 3:
        args.warmup = 3
    if args.case == "sweep-h":
        return run_sweep_h(args)
    if args.case == "serve":
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
