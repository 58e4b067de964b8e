"""Benchmark of the FDSC hot path on GB300.

One step = one image through one convolution layer, every online stage of
Fig. 2 plus HomRec: NTT2D(x_A) -> encrypt -> NTT2D(x_B) -> HomRec ->
HomConv + HomShare -> decrypt -> INTT2D(s_A) -> INTT2D(s_B), on the
32x32x64 -> 64 CIFAR-shaped layer (batch 1, 3x3 filters, n = 2048,
p = 65537, 60-bit q).  Keys, filter spectra and HomShare masks are prepared
before timing (the paper's t_setup); the step is the paper's t_online.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The device number (`value`) replays the step as a CUDA graph with inputs
resident in HBM, K steps back to back between CUDA events; the steps rotate
over independent instances of the layer whose data together exceed 3x L2,
so no step finds its inputs in L2.  `e2e` runs single-image requests of the same
layer through the server's C ABI with host buffers, copies in and out
included.
`--impl reference` times the CPU oracle (single thread) on a bounded sample.
Under torchrun every rank runs an independent replica on its own GPU (the
path has no exchange step) and rank 0 prints one JSON line.
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

import fdsc_inputs as FI  # noqa: E402

METRIC = "HomConv layers/s & mod-q MAC/s at 32×32×64; p50/p99 served latency"
STAGE_STREAMS = (1, 2, 2)  # streams per stage of the pipelined schedule: producers, HomConv, decryption
GRAPH_STEPS = 220   # steps recorded in one graph of the timed loop (20 rotations of the instances)
WORKLOAD = "cifar_32x32x64_b1"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "homconv_traffic.json")
KERNEL_SOURCES = ["paper_2003_05328_gb300/csrc/homconv.cu", "paper_2003_05328_gb300/csrc/modarith.cuh",
                  "paper_2003_05328_gb300/csrc/fdsc_internal.h"]


def kernel_digest() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def aggregate(local_seconds: float, local_units: float, world: int):
    """Whole-job figures: total units over the slowest rank's time."""
    if world == 1:
        return local_seconds, local_units
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def layer_counts(ls, T, beta, GB, n, addends=2):
    """Algorithmic bytes and modular products of one HomConv launch (filter
    read once; per image group the input ciphertexts, the c1 addends, the
    output ciphertexts and the mask words)."""
    filt = 8 * ls.Co * T * beta * n
    per_group = 8 * ((2 + addends) * T * beta * n + 2 * ls.Co * beta * n + ls.Co * beta * n)
    macs = 2 * ls.Co * T * beta * n * GB
    return filt + GB * per_group, macs


# the HomConv kernel behind each variant number (fdsc_set_homconv_variant)
HOMCONV_KERNELS = {3: "homconv_kernel<1,false,2>", 4: "homconv3_kernel<0>", 10: "homconv5_kernel<8>",
                   11: "homconv6_kernel<16,1>", 12: "homconv6_kernel<8,1>", 13: "homconv6_kernel<8,2>",
                   14: "homconv6_kernel<8,4>"}


def variant_used(T, requested):
    """The variant the library runs for T input ciphertexts (0 = its default)."""
    if requested in (11, 12, 13, 14) and T <= 64:
        return requested
    if requested == 10 and T <= 128 and T % 4 == 0:
        return 10
    if requested in (3, 4):
        return requested if T <= 256 or requested == 3 else 3
    return 12 if T <= 64 else (4 if T <= 256 else 3)


def homconv_kernel_name(T, requested):
    return HOMCONV_KERNELS.get(variant_used(T, requested), "homconv variant %d" % variant_used(T, requested))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, out_dir: str):
        self.gpu, self.proc, self.path, self.out_dir = gpu_index, None, None, out_dir

    def start(self):
        try:
            os.makedirs(self.out_dir, exist_ok=True)
            self.path = os.path.join(self.out_dir, f"clocks_bench_{os.getpid()}.csv")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle (baseline leg only)
def oracle_online_sample(budget_s: float, co_sample: int = 8):
    """Time the oracle's online stages on the bench layer: the input side
    (NTT2D x2, encrypt, HomRec) once per round and the output side (HomConv,
    decrypt, INTT2D x2) for `co_sample` of the Co output channels, repeated
    until `budget_s` is spent.  The output side is independent per output
    channel, so one layer costs t_in + t_out * Co / co_sample."""
    from oracle import oracle as O

    c = FI.CONFIGS[WORKLOAD]
    ls = c.layers[0]
    P = O.params(ls.n, ls.p)
    g_c, g_b = FI.default_pack(ls, P.S)
    L = O.layer(P, ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
    Ls = O.layer(P, ls.B, ls.Ci, co_sample, ls.H, ls.W, g_c, g_b)
    xA, xB = FI.shares(ls, c.cid)
    w = FI.weights(ls, c.cid)
    ks, es, ss = FI.seeds(c.cid)
    _, t_hat = O.keygen(P, ks)
    Phat = O.filter_prepare(P, Ls, w[:co_sample])
    Mhat, sB = O.mask_prepare(P, Ls, ss)
    names = ["ntt2d_xA", "encrypt", "ntt2d_xB", "homrec", "homconv_homshare", "decrypt", "intt2d_sA", "intt2d_sB"]
    acc = dict.fromkeys(names, 0.0)
    rounds = 0
    t0 = time.perf_counter()
    while rounds < 1 or time.perf_counter() - t0 < budget_s:
        t = [time.perf_counter()]
        XA = O.ntt2d(xA, ls.p).reshape(ls.B, ls.Ci, -1)
        t.append(time.perf_counter())
        ct = O.encrypt(P, L, t_hat, XA, es)
        t.append(time.perf_counter())
        XB = O.ntt2d(xB, ls.p).reshape(ls.B, ls.Ci, -1)
        t.append(time.perf_counter())
        ct = O.homrec(P, L, ct, XB)
        t.append(time.perf_counter())
        out = O.homconv(P, Ls, ct, Phat, Mhat)
        t.append(time.perf_counter())
        SA, _ = O.decrypt(P, Ls, t_hat, out)
        t.append(time.perf_counter())
        O.ntt2d(SA.reshape(ls.B, co_sample, ls.H, ls.W), ls.p, inverse=True)
        t.append(time.perf_counter())
        O.ntt2d(sB.reshape(ls.B, co_sample, ls.H, ls.W), ls.p, inverse=True)
        t.append(time.perf_counter())
        for i, k in enumerate(names):
            acc[k] += (t[i + 1] - t[i]) * (ls.Co / co_sample if i >= 4 else 1.0)
        rounds += 1
    stages = {k: v / rounds for k, v in acc.items()}
    per_layer = sum(stages.values())
    oracle_online_sample.stages_ms = {k: v * 1e3 for k, v in stages.items()}
    sample = (f"{rounds} round(s) of the {WORKLOAD} layer's online stages: input side in full, output side "
              f"(HomConv+HomShare, decrypt, INTT2D x2) for {co_sample}/{ls.Co} output channels, scaled to the "
              f"full layer; single thread")
    return per_layer, sample


def _output_side_worker(args):
    """One worker of the all-cores sample: the oracle's output side (HomConv +
    HomShare, decrypt, INTT2D x2) for output channels [lo, hi) of the bench
    layer, `reps` times; returns the seconds per repetition.  Runs in a
    process of its own (spawn), the oracle unchanged."""
    lo, hi, reps = args
    sys.path.insert(0, ROOT)
    from oracle import oracle as O

    ls = FI.CONFIGS[WORKLOAD].layers[0]
    c = FI.CONFIGS[WORKLOAD]
    P = O.params(ls.n, ls.p)
    g_c, g_b = FI.default_pack(ls, P.S)
    L = O.layer(P, ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
    Ls = O.layer(P, ls.B, ls.Ci, hi - lo, ls.H, ls.W, g_c, g_b)
    xA, xB = FI.shares(ls, c.cid)
    w = FI.weights(ls, c.cid)
    ks, es, ss = FI.seeds(c.cid)
    _, t_hat = O.keygen(P, ks)
    XA = O.ntt2d(xA, ls.p).reshape(ls.B, ls.Ci, -1)
    ct = O.homrec(P, L, O.encrypt(P, L, t_hat, XA, es), O.ntt2d(xB, ls.p).reshape(ls.B, ls.Ci, -1))
    Phat = O.filter_prepare(P, Ls, w[lo:hi])
    Mhat, sB = O.mask_prepare(P, Ls, ss)
    t0 = time.perf_counter()
    for _ in range(reps):
        out = O.homconv(P, Ls, ct, Phat, Mhat)
        SA, _ = O.decrypt(P, Ls, t_hat, out)
        O.ntt2d(SA.reshape(ls.B, hi - lo, ls.H, ls.W), ls.p, inverse=True)
        O.ntt2d(sB.reshape(ls.B, hi - lo, ls.H, ls.W), ls.p, inverse=True)
    return (time.perf_counter() - t0) / reps


def oracle_all_cores_sample(t_in_s: float, reps: int = 2):
    """The bench layer on every host core: the output side is independent per
    output channel, so the Co channels are split evenly over one spawned
    process per core, each running the unchanged oracle on its slice; the
    layer takes the input side (single thread, t_in_s) plus the slowest
    slice."""
    import multiprocessing as mp

    ls = FI.CONFIGS[WORKLOAD].layers[0]
    cores = max(1, min(os.cpu_count() or 1, ls.Co))
    bounds = [(i * ls.Co // cores, (i + 1) * ls.Co // cores) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        per = pool.map(_output_side_worker, [(lo, hi, reps) for lo, hi in bounds if hi > lo])
    per_layer = t_in_s + max(per)
    return {"value": 1.0 / per_layer, "unit": "layers/s", "cores": cores, "kind": "oracle",
            "sample": "input side single-threaded (%.0f ms), output side split over %d spawned processes of "
                      "%d-%d output channels each, %d repetitions; slowest slice" %
                      (t_in_s * 1e3, cores, ls.Co // cores, -(-ls.Co // cores), reps)}


def oracle_slice_step():
    """One reference step: the oracle on a proportional slice of the bench
    layer -- the input side (NTT2D, encryption, HomRec) for Ci/8 input
    channels and the output side (HomConv + HomShare, decryption, INTT2D x2)
    for Co/8 output channels.  Both sides are linear in those counts, so the
    step is 1/8 of a layer's work.  Returns (measured wall seconds, the
    fraction of a layer processed)."""
    from oracle import oracle as O

    c = FI.CONFIGS[WORKLOAD]
    ls = c.layers[0]
    P = O.params(ls.n, ls.p)
    g_c, g_b = FI.default_pack(ls, P.S)
    ci, co = ls.Ci // 8, ls.Co // 8
    assert ci % g_c == 0 and ci * ls.Co == co * ls.Ci  # the same fraction of both sides
    Lin = O.layer(P, ls.B, ci, ls.Co, ls.H, ls.W, g_c, g_b)
    Lfull = O.layer(P, ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
    Lout = O.layer(P, ls.B, ls.Ci, co, ls.H, ls.W, g_c, g_b)
    key = (ls.n, ls.p, ci, co)
    cache = oracle_slice_step.__dict__.setdefault("cache", {})
    if key not in cache:  # setup (keys, filter spectra, masks) is not part of the online step
        xA, xB = FI.shares(ls, c.cid)
        w = FI.weights(ls, c.cid)
        ks, es, ss = FI.seeds(c.cid)
        _, t_hat = O.keygen(P, ks)
        XA = O.ntt2d(xA, ls.p).reshape(ls.B, ls.Ci, -1)
        ct_full = O.homrec(P, Lfull, O.encrypt(P, Lfull, t_hat, XA, es), O.ntt2d(xB, ls.p).reshape(ls.B, ls.Ci, -1))
        Mhat, sB = O.mask_prepare(P, Lout, ss)
        cache[key] = (xA[:, :ci], xB[:, :ci], t_hat, es, ct_full, O.filter_prepare(P, Lout, w[:co]), Mhat, sB)
    xA, xB, t_hat, es, ct_full, Phat, Mhat, sB = cache[key]
    a = time.perf_counter()
    XA = O.ntt2d(xA, ls.p).reshape(ls.B, ci, -1)
    ct = O.encrypt(P, Lin, t_hat, XA, es)
    O.homrec(P, Lin, ct, O.ntt2d(xB, ls.p).reshape(ls.B, ci, -1))
    out = O.homconv(P, Lout, ct_full, Phat, Mhat)
    SA, _ = O.decrypt(P, Lout, t_hat, out)
    O.ntt2d(SA.reshape(ls.B, co, ls.H, ls.W), ls.p, inverse=True)
    O.ntt2d(sB.reshape(ls.B, co, ls.H, ls.W), ls.p, inverse=True)
    return time.perf_counter() - a, ci / ls.Ci


def run_reference(args, rank, world):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_slice_step()
    t0 = time.perf_counter()
    fracs = [oracle_slice_step()[1] for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    sec = wall / max(1, args.steps)  # measured wall time of one step (a 1/8 slice of the layer)
    frac = fracs[0]
    ls = FI.CONFIGS[WORKLOAD].layers[0]
    value = frac / sec  # layers of work processed per second
    sample = ("each of the %d steps: the oracle on %d of %d input channels and %d of %d output channels of the %s "
              "layer (%.3f of a layer's work, both sides being linear in those counts); single thread; "
              "ms_per_step is the measured wall time of one such step" %
              (args.steps, ls.Ci // 8, ls.Ci, ls.Co // 8, ls.Co, WORKLOAD, frac))
    line = {"metric": METRIC, "value": value, "unit": "layers/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "layer": "32x32x64->64 3x3", "batch": ls.B, "n": ls.n, "p": ls.p,
                       "q_bits": 60, "l2": "cpu"},
            "layer_fraction_per_step": frac,
            "mac_per_s": value * 2 * ls.Co * ls.Ci * ls.H * ls.W,
            "cpu_baseline": {"value": value, "unit": "layers/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "layers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))



# ------------------------------------------------------------------ end to end, batched, served
def e2e_through_server(F, P, ls, g_c, w_dev, t_hat, xA1, xB1, n_req, window=256):
    """Single-image requests of the bench layer through the server's C ABI
    (host buffers in and out), submitted back to back with at most `window`
    outstanding; whole-job wall time from the first submit to the last
    completion."""
    S = F.Server(hbm_budget_bytes=120 * 10**9, max_batch=16, lanes=4)
    tid = S.add_type(P, F.LayerSpec(1, ls.Ci, ls.Co, ls.H, ls.W, g_c, 1), w_dev, t_hat)
    S.start()
    xA1 = np.ascontiguousarray(xA1, dtype=np.uint32)
    xB1 = np.ascontiguousarray(xB1, dtype=np.uint32)
    outs = [(np.empty((ls.Co, ls.H, ls.W), np.uint32), np.empty((ls.Co, ls.H, ls.W), np.uint32))
            for _ in range(window)]
    for i in range(32):  # warm-up
        S.wait(S.submit(tid, 0, i, i, xA1, xB1, *outs[i % window]))
    tickets = [None] * n_req
    t0 = time.perf_counter()
    for i in range(n_req):
        if i >= window:
            S.wait(tickets[i - window])
        tickets[i] = S.submit(tid, 0, 1000 + i, 2000 + i, xA1, xB1, *outs[i % window])
    for i in range(max(0, n_req - window), n_req):
        S.wait(tickets[i])
    t1 = time.perf_counter()
    st = S.stats()
    S.close()
    return {"seconds": t1 - t0, "requests": n_req, "h2d": 2 * xA1.nbytes + 16, "d2h": 2 * outs[0][0].nbytes,
            "p50_us": st.p50_us, "p99_us": st.p99_us, "mean_batch": st.mean_batch}


def run_batched(F, flush, sleep_cycles, args):
    """The uneven stack (16 images through 32x32x64->64, 16x16x128->128 and
    8x8x256->256) as one autotuned plan (one graph launch) against the plain
    per-layer path: every (layer, image) pair launched on its own."""
    import torch

    c = FI.CONFIGS["stack_16img_32x32x64_16x16x128_8x8x256"]
    params, specs, singles = {}, [], []
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    for li, ls in enumerate(c.layers):
        P = params.setdefault((ls.n, ls.p), F.Params(ls.n, ls.p, max_T=256))
        xA, xB = FI.shares(ls, c.cid, li)
        w = dev(FI.weights(ls, c.cid, li), np.int8)
        ks, es, ss = FI.seeds(c.cid, li)
        t_hat = F.keygen(P, ks)
        base = dict(params=P, w=w, t_hat=t_hat, enc_seed=es, mask_seed=ss)
        specs.append(dict(base, layer=F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, 0, 0), xA=dev(xA, np.int32),
                          xB=dev(xB, np.int32),
                          yA=torch.empty((ls.B, ls.Co, ls.H, ls.W), dtype=torch.int32, device="cuda"),
                          yB=torch.empty((ls.B, ls.Co, ls.H, ls.W), dtype=torch.int32, device="cuda")))
        for b in range(ls.B):
            singles.append(dict(base, layer=F.LayerSpec(1, ls.Ci, ls.Co, ls.H, ls.W, 0, 0),
                                xA=dev(xA[b:b + 1], np.int32), xB=dev(xB[b:b + 1], np.int32),
                                yA=torch.empty((1, ls.Co, ls.H, ls.W), dtype=torch.int32, device="cuda"),
                                yB=torch.empty((1, ls.Co, ls.H, ls.W), dtype=torch.int32, device="cuda")))
    t0 = time.perf_counter()
    plan = F.Plan(specs, tune=True)
    tune_s = time.perf_counter() - t0
    per_pair = [F.Plan([d]) for d in singles]

    def timed(fn, reps):
        for _ in range(3):
            flush.fill_(1)
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda._sleep(sleep_cycles)
        for i, (a, b) in enumerate(ev):
            flush.fill_(i & 0xFF)
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    reps = max(5, min(args.steps // 20, 100))
    ms_plan = timed(plan.launch, reps)
    ms_single = timed(lambda: [pp.launch() for pp in per_pair], max(3, reps // 5))
    units = sum(ls.B for ls in c.layers)
    info = [plan.info(i) for i in range(len(c.layers))]
    out = {"workload": "stack_16img_32x32x64_16x16x128_8x8x256", "layers": [f"{ls.H}x{ls.W}x{ls.Ci}->{ls.Co}, n={ls.n}" for ls in c.layers],
           "images": c.layers[0].B, "layers_per_s": units / (np.mean(ms_plan) * 1e-3),
           "ms_per_launch": float(np.mean(ms_plan)), "per_layer_path_layers_per_s": units / (np.mean(ms_single) * 1e-3),
           "per_layer_path_ms": float(np.mean(ms_single)), "speedup_vs_per_layer": float(np.mean(ms_single) / np.mean(ms_plan)),
           "tuning_s": tune_s,
           "tuned": [{"g_c": x.g_c, "g_b": x.g_b, "homconv_variant": x.homconv_variant, "candidates": x.candidates,
                      "step_us": x.tuned_step_us} for x in info],
           "l2": "flushed before every timed launch", "launches": "1 graph (plan) vs %d graphs" % len(per_pair)}
    plan.close()
    for pp in per_pair:
        pp.close()
    for P in params.values():
        P.close()
    return out


# HomConv shapes where the contraction is a dense product: the 16-image stack's
# three layers and the binarized 64x64x128 layer at batch 8
TENSOR_SHAPES = [("stack_16img_32x32x64_16x16x128_8x8x256", 0), ("stack_16img_32x32x64_16x16x128_8x8x256", 1), ("stack_16img_32x32x64_16x16x128_8x8x256", 2), ("binarized_64x64x128_b8", 0)]


def run_tensor_homconv(F, flush, args):
    """HomConv + HomShare (+ HomRec addends) of the batched shapes on the
    tensor cores (fdsc_homconv_tc, digit planes in fp16, exact fp32 sums)
    against the CUDA-core kernel on the same words: each call recorded in a
    CUDA graph, L2 flushed before every timed replay, median.  Bytes are those
    the tensor-core kernel moves (its filter is fp16 digit planes, 16 bytes a
    word); the tensor work counts the digit MMAs it issues."""
    import torch

    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs") or 6800.0
    tpk = peaks.get("bf16_tflops") or 1900.0  # fp16 and bf16 MMAs run at the same rate
    out = []

    def median_us(fn, reps):
        fn()
        torch.cuda.synchronize()
        gr = torch.cuda.CUDAGraph()
        s0 = torch.cuda.Stream()
        s0.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s0):
            with torch.cuda.graph(gr, stream=s0):
                fn()
        torch.cuda.current_stream().wait_stream(s0)
        ts = []
        for i in range(reps + 2):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            gr.replay()
            b.record()
            b.synchronize()
            if i >= 2:
                ts.append(a.elapsed_time(b) * 1e3)
        return float(np.median(ts))

    for cfg, li in TENSOR_SHAPES:
        ls = FI.CONFIGS[cfg].layers[li]
        info = F.params_query(ls.n, ls.p)
        g_c, g_b = FI.default_pack(ls, info.S)
        L = F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
        P = F.Params(ls.n, ls.p, max_T=256)
        lay = F.layout(P, L)
        g = torch.Generator(device="cuda").manual_seed(FI.SEED_BASE + li)
        rnd = lambda k: torch.randint(0, info.q, (k,), dtype=torch.int64, device="cuda", generator=g)
        ct, Ph, Mh = rnd(lay.ct_in_words), rnd(lay.filter_words), rnd(lay.mask_words)
        A1, A2 = rnd(lay.n_in * ls.n), rnd(lay.n_in * ls.n)
        Ptc = F.filter_tc(P, L, Ph)
        o1 = torch.empty(lay.ct_out_words, dtype=torch.int64, device="cuda")
        o2 = torch.empty_like(o1)
        reps = 9 if lay.filter_words < (64 << 20) else 5
        us_tc = median_us(lambda: F.homconv_tc(P, L, ct, A1, A2, Ptc, Mh, out=o1), reps)
        us_cc = median_us(lambda: F.homconv_sum(P, L, ct, A1, A2, Ph, Mh, out=o2), reps)
        torch.cuda.synchronize()
        same = bool(torch.equal(o1, o2))
        status = F.homconv_tc_status()
        macs = 2 * ls.Co * lay.T * lay.beta * ls.n * lay.GB
        # the kernel's items: the d indices sharing a filter word (d <= 8) and
        # up to 8 / d image groups, B columns nb = 2 x groups x d
        dj = info.d if info.d <= 8 else 1
        gbt = 1
        while 2 * gbt <= 8 // dj and 2 * gbt <= lay.GB:
            gbt *= 2
        nb = 2 * gbt * dj
        items = lay.beta * (ls.n // dj) * (-(-ls.Co // 128)) * (-(-lay.GB // gbt))
        mmas = items * (8 * (-(-lay.T // 16)) + 1)
        flops = mmas * 2 * 128 * 8 * nb * 16
        byts = 8 * (Ptc.numel() + lay.ct_in_words + 2 * lay.n_in * ls.n + lay.ct_out_words + lay.mask_words)
        out.append({"layer": "%s %dx%dx%d->%d, batch %d, n=%d, p=%d" % (cfg, ls.H, ls.W, ls.Ci, ls.Co, ls.B, ls.n,
                                                                       ls.p),
                    "T": lay.T, "image_groups": lay.GB, "tensor_us": us_tc, "cuda_core_us": us_cc,
                    "speedup": us_cc / us_tc, "words_identical": same, "status": status,
                    "mod_q_macs_per_s": macs / (us_tc * 1e-6), "bytes": byts,
                    "GB_per_s": byts / (us_tc * 1e-6) / 1e9, "hbm_frac": byts / (us_tc * 1e-6) / 1e9 / hbm,
                    "digit_mma_tflops": flops / (us_tc * 1e-6) / 1e12,
                    "tensor_frac": flops / (us_tc * 1e-6) / 1e12 / tpk})
        del ct, Ph, Mh, A1, A2, Ptc, o1, o2
        torch.cuda.empty_cache()
        P.close()
    return {"kernel": "homconv_tc_kernel (fdsc_homconv_tc)", "peaks": {"hbm_GB_per_s": hbm, "fp16_tflops": tpk},
            "l2": "flushed before every timed replay", "shapes": out}


def plain_conv_plane(p, x, w):
    """One output plane of the cyclic convolution mod p, computed directly
    with numpy (a property check of the GPU shares; the filter taps sit at
    the top-left of the padded plane): y[i][j] = sum_ci sum_{a,c}
    w[ci][a][c] x[ci][(i-a) mod H][(j-c) mod W]."""
    Ci, fh, fw = w.shape
    y = np.zeros(x.shape[1:], np.int64)
    for ci in range(Ci):
        for a in range(fh):
            for c in range(fw):
                y += int(w[ci, a, c]) * np.roll(np.roll(x[ci].astype(np.int64), a, axis=0), c, axis=1)
    return y % p


def run_binarized(F, sleep_cycles, args):
    """The binarized 64x64x128 -> 128 layer at batch 8 (n = 4096, p = 12289,
    two slot sets per ciphertext and each spectrum over two ciphertexts,
    weights in {-1, +1}) through the fused online path: producers in one
    launch, HomConv on the tensor cores, fused decryption, Bob's INTT2D on a
    side stream.  One instance holds about 2 GB, far above L2, so every step
    reads its operands from HBM.  Shares are checked against the plain
    convolution on sampled planes."""
    import torch

    c = FI.CONFIGS["binarized_64x64x128_b8"]
    ls = c.layers[0]
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm = peaks.get("hbm_gbs") or 6800.0
    P = F.Params(ls.n, ls.p, max_T=ls.Ci)
    L = F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, 1, 1)
    lay = F.layout(P, L)
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    xA_h, xB_h = FI.shares(ls, c.cid)
    w_h = FI.weights(ls, c.cid)
    ks, es, ss = FI.seeds(c.cid)
    t_hat = F.keygen(P, ks)
    Phat = F.filter_prepare(P, L, dev(w_h, np.int8))
    Ptc = F.filter_tc(P, L, Phat)
    Mhat, sB = F.mask_prepare(P, L, ss)
    xA, xB = dev(xA_h, np.int32), dev(xB_h, np.int32)
    ct = torch.empty(lay.ct_in_words, dtype=torch.int64, device="cuda")
    A = torch.empty(lay.n_in * ls.n, dtype=torch.int64, device="cuda")
    R = torch.empty_like(A)
    out = torch.empty(lay.ct_out_words, dtype=torch.int64, device="cuda")
    yA = torch.empty((ls.B, ls.Co, ls.H, ls.W), dtype=torch.int32, device="cuda")
    yB = torch.empty_like(yA)
    side = torch.cuda.Stream()

    def step(tensor=True):
        main = torch.cuda.current_stream()
        side.wait_stream(main)
        with torch.cuda.stream(side):
            F.intt2d(P, sB.view(ls.B, ls.Co, ls.H, ls.W), out=yB)
        F.online_produce(P, L, t_hat, es, xA, xB, ct, A, R)
        if tensor:
            F.homconv_tc(P, L, ct, A, R, Ptc, Mhat, out=out)
        else:
            F.homconv_sum(P, L, ct, A, R, Phat, Mhat, out=out)
        F.decrypt_share(P, L, t_hat, out, out=yA)
        main.wait_stream(side)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        gr = torch.cuda.CUDAGraph()
        s0 = torch.cuda.Stream()
        s0.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s0):
            with torch.cuda.graph(gr, stream=s0):
                fn()
        torch.cuda.current_stream().wait_stream(s0)
        for _ in range(2):
            gr.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(sleep_cycles)
        a.record()
        for _ in range(reps):
            gr.replay()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e3 / reps

    F.set_launch_overlap(True)
    reps = max(5, min(args.steps // 20, 40))
    step_us = timed(step, reps)
    F.set_launch_overlap(False)
    hc_tc_us = timed(lambda: F.homconv_tc(P, L, ct, A, R, Ptc, Mhat, out=out), reps)
    hc_cc_us = timed(lambda: F.homconv_sum(P, L, ct, A, R, Phat, Mhat, out=out), max(3, reps // 4))
    prod_us = timed(lambda: F.online_produce(P, L, t_hat, es, xA, xB, ct, A, R), reps)
    dec_us = timed(lambda: F.decrypt_share(P, L, t_hat, out, out=yA), reps)
    assert F.homconv_tc_status() == 0
    # property check of the shares on sampled planes
    step()
    torch.cuda.synchronize()
    yA_n = yA.cpu().numpy().view(np.uint32).astype(np.int64)
    yB_n = yB.cpu().numpy().view(np.uint32).astype(np.int64)
    x = (xA_h.astype(np.int64) + xB_h) % ls.p
    rng = np.random.default_rng(c.cid)
    checked = 0
    for _ in range(4):
        b, co = int(rng.integers(ls.B)), int(rng.integers(ls.Co))
        if not np.array_equal((yA_n[b, co] + yB_n[b, co]) % ls.p, plain_conv_plane(ls.p, x[b], w_h[co])):
            raise RuntimeError("binarized layer: shares do not reconstruct the convolution")
        checked += 1
    # algorithmic bytes of one HomConv launch (the method's 8-byte words, the
    # filter once per group of d indices) and the bytes the tensor-core kernel moves
    d = P.info.d
    filt = 8 * ls.Co * lay.T * lay.beta * ls.n // d
    per_groups = 8 * lay.GB * (4 * lay.T * lay.beta * ls.n + 3 * ls.Co * lay.beta * ls.n)
    alg = filt + per_groups
    moved = 8 * Ptc.numel() + per_groups
    macs = 2 * ls.Co * lay.T * lay.beta * ls.n * lay.GB
    res = {"workload": "binarized_64x64x128_b8", "layer": "64x64x128->128 3x3, binarized weights, batch 8", "n": ls.n, "p": ls.p,
           "d": d, "beta": lay.beta, "T": lay.T, "image_groups": lay.GB,
           "step_us": step_us, "layers_per_s": ls.B / (step_us * 1e-6),
           "stage_us": {"online_produce": prod_us, "homconv_tc": hc_tc_us, "homconv_cuda_cores": hc_cc_us,
                        "decrypt_share": dec_us},
           "roofline": {"kernel": "homconv_tc_kernel (fdsc_homconv_tc)", "bound": "hbm",
                        "alg_bytes_per_launch": alg, "achieved": alg / (hc_tc_us * 1e-6) / 1e9, "peak": hbm,
                        "unit": "GB/s", "frac": alg / (hc_tc_us * 1e-6) / 1e9 / hbm,
                        "bytes_moved_per_launch": moved,
                        "frac_of_moved": moved / (hc_tc_us * 1e-6) / 1e9 / hbm,
                        "note": "alg: 8-byte filter words once per group of d = 2 evaluation indices, input, "
                                "addend, output and mask words; moved: the fp16 digit-plane filter (16 bytes a "
                                "distinct word) plus the same per-group words"},
           "mod_q_macs_per_s": macs / (hc_tc_us * 1e-6),
           "shares_checked_planes": checked,
           "launches": 4 * (reps + 4) + 3 * (reps + 3) + (max(3, reps // 4) + 3),
           "timing": "one CUDA graph per measurement, %d replays back to back, CUDA events; the step with "
                     "programmatic dependent launch" % reps}
    for t in (Phat, Ptc, Mhat, sB, xA, xB, ct, A, R, out, yA, yB):
        del t
    torch.cuda.empty_cache()
    P.close()
    return res


# the appendix network (MiniONN's CIFAR-10 network, Fig. 13 there): its six
# convolution layers, (Ci, Co, H, filter, 2x2 pooling after); the
# fully-connected layer and the activations are not part of the path
APPENDIX_CONVS = [(3, 64, 32, 3, False), (64, 64, 32, 3, True), (64, 64, 16, 3, False), (64, 64, 16, 3, True),
                  (64, 64, 8, 3, False), (64, 64, 8, 1, False)]


def run_chain(F, flush, sleep_cycles, args):
    """One inference of the appendix network's convolution stack (batch 1)
    as a chained plan: each layer reads the shares the previous one wrote,
    sum-pooled where the network pools (activations left to their own
    protocol).  L2 flushed before every timed launch."""
    import torch

    P = F.Params(2048, 65537, max_T=64)
    g = np.random.default_rng(FI.SEED_BASE + 7)
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    Ci0, H0 = APPENDIX_CONVS[0][0], APPENDIX_CONVS[0][2]
    inA = dev(g.integers(0, 65537, (1, Ci0, H0, H0)), np.int32)
    inB = dev(g.integers(0, 65537, (1, Ci0, H0, H0)), np.int32)
    specs = []
    for i, (Ci, Co, H, fh, pool) in enumerate(APPENDIX_CONVS):
        d = dict(params=P, layer=F.LayerSpec(1, Ci, Co, H, H, 0, 0), w=dev(g.integers(-8, 8, (Co, Ci, fh, fh)), np.int8),
                 t_hat=F.keygen(P, 700 + i), enc_seed=710 + i, mask_seed=720 + i, xA=inA, xB=inB,
                 yA=torch.empty((1, Co, H, H), dtype=torch.int32, device="cuda"),
                 yB=torch.empty((1, Co, H, H), dtype=torch.int32, device="cuda"))
        if pool:
            d["pA"] = torch.empty((1, Co, H // 2, H // 2), dtype=torch.int32, device="cuda")
            d["pB"] = torch.empty_like(d["pA"])
        inA, inB = (d["pA"], d["pB"]) if pool else (d["yA"], d["yB"])
        specs.append(d)
    plan = F.Plan(specs, tune=True, chain=True)
    reps = max(5, min(args.steps // 10, 200))
    for _ in range(3):
        flush.fill_(1)
        plan.launch()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda._sleep(sleep_cycles)
    for i, (a, b) in enumerate(ev):
        flush.fill_(i & 0xFF)
        a.record()
        plan.launch()
        b.record()
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    info = [plan.info(i) for i in range(len(specs))]
    plan.close()
    P.close()
    return {"network": "appendix network (MiniONN CIFAR-10, Fig. 13 there): 6 convolution layers, 2 sum poolings",
            "layers": ["%dx%dx%d->%d %dx%d%s" % (H, H, Ci, Co, fh, fh, " +pool" if pl else "")
                       for Ci, Co, H, fh, pl in APPENDIX_CONVS],
            "inference_us_p50": float(np.percentile(ms, 50)) * 1e3, "inference_us_p99": float(np.percentile(ms, 99)) * 1e3,
            "conv_layers_per_s": len(APPENDIX_CONVS) / (float(np.mean(ms)) * 1e-3),
            "packing": [{"g_c": x.g_c, "homconv_variant": x.homconv_variant} for x in info],
            "launches": reps, "l2": "flushed before every timed launch",
            "path": "one chained plan (FDSC_PLAN_CHAIN), one graph launch per inference"}


def run_serving(F, args, rate=None, n_req=None):
    """The served mix: Poisson arrivals (mean 2000 requests/s, or `rate`) of
    single-image requests drawn uniformly from three layer types, each from
    one of a pool of client keys; continuous batching inside the library's
    server under a 120 GB HBM budget; latency from submit to completion."""
    import threading

    import torch

    c = FI.CONFIGS["served_mix_28x28x1_32x32x64_16x16x128"]
    rate = rate or c.extra["rate_per_s"]
    n_req = n_req or args.serve_requests
    P = F.Params(2048, 65537, max_T=64)
    t0 = time.perf_counter()
    keys = torch.stack([F.keygen(P, 5000 + k) for k in range(args.serve_keys)]).reshape(-1)
    torch.cuda.synchronize()
    keygen_us = (time.perf_counter() - t0) / args.serve_keys * 1e6
    S = F.Server(hbm_budget_bytes=c.extra["hbm_budget_bytes"], max_batch=16, lanes=4)
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    types, pools = [], []
    for ti, ls in enumerate(c.layers):
        g_c, g_b = FI.default_pack(ls, P.info.S)
        tid = S.add_type(P, F.LayerSpec(1, ls.Ci, ls.Co, ls.H, ls.W, g_c, 1), dev(FI.weights(ls, c.cid, ti), np.int8),
                         keys)
        xA, xB = FI.shares(ls, c.cid, ti)  # batch 1: reuse as a pool by rolling the plane
        ins = [(np.ascontiguousarray(np.roll(xA[0], k, axis=-1)), np.ascontiguousarray(np.roll(xB[0], k, axis=-1)))
               for k in range(16)]
        outs = [(np.empty((ls.Co, ls.H, ls.W), np.uint32), np.empty((ls.Co, ls.H, ls.W), np.uint32))
                for _ in range(512)]
        types.append(tid)
        pools.append((ins, outs))
    S.start()
    g = np.random.default_rng(FI.SEED_BASE + c.cid)
    kinds = g.integers(0, len(types), n_req)
    keyidx = g.integers(0, args.serve_keys, n_req)
    arrivals = np.cumsum(g.exponential(1.0 / rate, n_req))
    tickets = [None] * n_req
    slot_owner = {}
    progress = [0]  # requests known complete, in submission order

    def waiter():
        for i in range(n_req):
            while tickets[i] is None:
                time.sleep(0.0002)
            S.wait(tickets[i])
            progress[0] = i + 1

    th = threading.Thread(target=waiter)
    th.start()
    start = time.perf_counter()
    for i in range(n_req):
        while time.perf_counter() - start < arrivals[i]:
            pass
        t = int(kinds[i])
        ins, outs = pools[t]
        slot = i % len(outs)
        prev = slot_owner.get((t, slot))
        while prev is not None and progress[0] <= prev:  # the slot's previous request must be done
            time.sleep(0.0001)
        xa, xb = ins[i % len(ins)]
        tickets[i] = S.submit(types[t], int(keyidx[i]), 7000 + i, 9000 + i, xa, xb, *outs[slot])
        slot_owner[(t, slot)] = i
    th.join()
    wall = time.perf_counter() - start
    st = S.stats()
    S.close()
    P.close()
    return {"workload": "served_mix_28x28x1_32x32x64_16x16x128" if rate == c.extra["rate_per_s"] else "served mix at %g requests/s" % rate,
            "requests": n_req, "rate_per_s": rate, "completed": int(st.completed),
            "lanes": int(st.lanes), "lane_capacity": int(st.lane_capacity), "reserved_bytes": int(st.reserved_bytes),
            "throughput_req_per_s": st.completed / wall, "p50_us": st.p50_us, "p99_us": st.p99_us,
            "mean_us": st.mean_us, "max_us": st.max_us, "mean_batch": st.mean_batch, "batches": int(st.batches),
            "peak_inflight_bytes": int(st.peak_inflight_bytes), "client_keys": args.serve_keys,
            "keygen_us_per_key": keygen_us, "hbm_budget_bytes": c.extra["hbm_budget_bytes"],
            "types": ["28x28(pad 32)x1->16 5x5", "32x32x64->64 3x3", "16x16x128->128 3x3"]}

# ------------------------------------------------------------------ GPU arm
def ntt2d_sweep(F, P, ls, back_to_back, args):
    """Forward NTT2D of B images x Ci planes (H x W, uint32) for a sweep of B:
    consecutive launches read and write consecutive slices of a 2 x 512 MiB
    window, so a slice comes round again only after 1 GiB of traffic (no L2
    reuse).  Algorithmic bytes: 4 B read + 4 B written per element."""
    import torch

    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    peak = peaks.get("hbm_gbs") or 6800.0
    plane = ls.H * ls.W
    win = (512 << 20) // 4
    x = torch.randint(0, ls.p, (win,), dtype=torch.int32, device="cuda")
    X = torch.empty_like(x)
    pts = []
    s = torch.cuda.Stream()
    for B in (1, 4, 16, 64, 256, 1024, 2048):
        planes = B * ls.Ci
        elems = planes * plane
        if elems > win:
            break
        nslices = win // elems  # one graph = one launch per slice, in order
        views = [(x[i * elems:(i + 1) * elems].view(planes, ls.H, ls.W), X[i * elems:(i + 1) * elems].view(planes, ls.H, ls.W))
                 for i in range(nslices)]
        gr = torch.cuda.CUDAGraph()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for a, b in views:
                F.ntt2d(P, a, out=b)
            torch.cuda.synchronize()
            with torch.cuda.graph(gr, stream=s):
                for a, b in views:
                    F.ntt2d(P, a, out=b)
        torch.cuda.current_stream().wait_stream(s)
        reps = max(2, min(64, (4 * 1024) // nslices))
        gr.replay()
        ev = back_to_back([gr], reps)
        torch.cuda.synchronize()
        us = ev[0].elapsed_time(ev[-1]) * 1e3 / (reps * nslices)
        gbs = 8 * elems / (us * 1e-6) / 1e9
        pts.append({"images": B, "planes": planes, "us": us, "GB_per_s": gbs, "frac": gbs / peak,
                    "launches": reps * nslices})
        del gr
    first = next((p["images"] for p in pts if p["frac"] >= 0.6), None)
    return {"plane": "%dx%d" % (ls.H, ls.W), "planes_per_image": ls.Ci, "peak_GB_per_s": peak,
            "launch": "fdsc_ntt2d launches over consecutive slices, one CUDA graph per batch size, replayed back to "
                      "back between CUDA events", "points": pts,
            "images_at_60pct": first}


def run_kernel_only(args):
    """A few launches of one part of the path, for profiler captures (no
    timing, no JSON line): `homconv` (HomConv + HomShare of the 32x32x64
    layer on seeded random words), `homconv_b16` (the same layer at 16
    images, the first layer of the 16-image stack), `homconv_tc` (the tensor-core HomConv of
    the 16x16x128->128 layer at 16 images), `ntt2d` (forward NTT2D of
    --planes 32x32 planes), `step` (the fused online step of that layer,
    eager), `binarized` (the binarized 64x64x128 layer at batch 8 through
    the fused path, HomConv on the tensor cores) or `plan` (the 16-image
    stack as one autotuned plan; under a profiler the tuner's timings, and
    so its choices, can differ)."""
    import torch

    torch.cuda.set_device(0)
    from paper_2003_05328_gb300 import build as B

    B.build()
    from paper_2003_05328_gb300 import fdsc as F

    c = FI.CONFIGS[WORKLOAD]
    ls = c.layers[0]
    info = F.params_query(ls.n, ls.p)
    g_c, g_b = FI.default_pack(ls, info.S)
    L = F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
    P = F.Params(ls.n, ls.p, max_T=64)
    lay = F.layout(P, L)
    F.set_homconv_variant(args.homconv_variant)
    g = torch.Generator(device="cuda")
    g.manual_seed(FI.SEED_BASE)
    rnd = lambda hi, k: torch.randint(0, hi, (k,), dtype=torch.int64, device="cuda", generator=g)
    if args.kernel_only == "plan":
        # the 16-image uneven stack as one autotuned plan, launched --steps times
        P.close()
        c2 = FI.CONFIGS["stack_16img_32x32x64_16x16x128_8x8x256"]
        params, specs = {}, []
        dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
        for li, ls2 in enumerate(c2.layers):
            P2 = params.setdefault((ls2.n, ls2.p), F.Params(ls2.n, ls2.p, max_T=256))
            xA, xB = FI.shares(ls2, c2.cid, li)
            ks, es, ss = FI.seeds(c2.cid, li)
            specs.append(dict(params=P2, w=dev(FI.weights(ls2, c2.cid, li), np.int8), t_hat=F.keygen(P2, ks),
                              enc_seed=es, mask_seed=ss,
                              layer=F.LayerSpec(ls2.B, ls2.Ci, ls2.Co, ls2.H, ls2.W, 0, 0), xA=dev(xA, np.int32),
                              xB=dev(xB, np.int32),
                              yA=torch.empty((ls2.B, ls2.Co, ls2.H, ls2.W), dtype=torch.int32, device="cuda"),
                              yB=torch.empty((ls2.B, ls2.Co, ls2.H, ls2.W), dtype=torch.int32, device="cuda")))
        plan = F.Plan(specs, tune=True)
        torch.cuda.synchronize()
        for _ in range(args.steps):
            plan.launch()
        torch.cuda.synchronize()
        print("tuned variants:", [plan.info(i).homconv_variant for i in range(len(specs))])
        plan.close()
        for P2 in params.values():
            P2.close()
        print("ran %d x plan" % args.steps)
        return
    if args.kernel_only == "binarized":
        # the binarized 64x64x128 layer at batch 8 through the fused path
        P.close()
        c4 = FI.CONFIGS["binarized_64x64x128_b8"]
        ls4 = c4.layers[0]
        P = F.Params(ls4.n, ls4.p, max_T=ls4.Ci)
        L4 = F.LayerSpec(ls4.B, ls4.Ci, ls4.Co, ls4.H, ls4.W, 1, 1)
        dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
        xA_h, xB_h = FI.shares(ls4, c4.cid)
        ks, es, ss = FI.seeds(c4.cid)
        t_hat = F.keygen(P, ks)
        Phat = F.filter_prepare(P, L4, dev(FI.weights(ls4, c4.cid), np.int8))
        Ptc = F.filter_tc(P, L4, Phat)
        Mhat, sB = F.mask_prepare(P, L4, ss)
        xA, xB = dev(xA_h, np.int32), dev(xB_h, np.int32)
        for _ in range(args.steps):
            ct, A, R = F.online_produce(P, L4, t_hat, es, xA, xB)
            F.intt2d(P, sB.view(ls4.B, ls4.Co, ls4.H, ls4.W))
            F.decrypt_share(P, L4, t_hat, F.homconv_tc(P, L4, ct, A, R, Ptc, Mhat))
        torch.cuda.synchronize()
        assert F.homconv_tc_status() == 0
        print("ran %d x binarized" % args.steps)
        P.close()
        return
    if args.kernel_only == "homconv_tc":
        # the tensor-core HomConv on the 16x16x128->128 layer of the 16-image stack
        ls = FI.CONFIGS["stack_16img_32x32x64_16x16x128_8x8x256"].layers[1]
        info = F.params_query(ls.n, ls.p)
        g_c, g_b = FI.default_pack(ls, info.S)
        L = F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
        P.close()
        P = F.Params(ls.n, ls.p, max_T=64)
        lay = F.layout(P, L)
        ct, Ph, Mh = rnd(info.q, lay.ct_in_words), rnd(info.q, lay.filter_words), rnd(info.q, lay.mask_words)
        A1, A2 = rnd(info.q, lay.n_in * ls.n), rnd(info.q, lay.n_in * ls.n)
        Ptc = F.filter_tc(P, L, Ph)
        out = torch.empty(lay.ct_out_words, dtype=torch.int64, device="cuda")
        for _ in range(args.steps):
            F.homconv_tc(P, L, ct, A1, A2, Ptc, Mh, out=out)
        torch.cuda.synchronize()
        assert F.homconv_tc_status() == 0
    elif args.kernel_only in ("homconv", "homconv_b16"):
        if args.kernel_only == "homconv_b16":
            ls = FI.CONFIGS["stack_16img_32x32x64_16x16x128_8x8x256"].layers[0]
            g_c, g_b = FI.default_pack(ls, info.S)
            L = F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
            lay = F.layout(P, L)
        ct, Ph, Mh = rnd(info.q, lay.ct_in_words), rnd(info.q, lay.filter_words), rnd(info.q, lay.mask_words)
        A1, A2 = rnd(info.q, lay.n_in * ls.n), rnd(info.q, lay.n_in * ls.n)
        out = torch.empty(lay.ct_out_words, dtype=torch.int64, device="cuda")
        for _ in range(args.steps):
            F.homconv_sum(P, L, ct, A1, A2, Ph, Mh, out=out)
    elif args.kernel_only == "ntt2d":
        x = rnd(ls.p, args.planes * ls.H * ls.W).to(torch.int32).view(args.planes, ls.H, ls.W)
        X = torch.empty_like(x)
        for _ in range(args.steps):
            F.ntt2d(P, x, out=X)
    else:
        dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
        xA_h, xB_h = FI.shares(ls, c.cid)
        ks, es, ss = FI.seeds(c.cid)
        t_hat = F.keygen(P, ks)
        Phat = F.filter_prepare(P, L, dev(FI.weights(ls, c.cid), np.int8))
        Mhat, sB = F.mask_prepare(P, L, ss)
        xA, xB = dev(xA_h, np.int32), dev(xB_h, np.int32)
        for _ in range(args.steps):
            ct, A, R = F.online_produce(P, L, t_hat, es, xA, xB)
            F.intt2d(P, sB.view(ls.B, ls.Co, ls.H, ls.W))
            F.decrypt_share(P, L, t_hat, F.homconv_sum(P, L, ct, A, R, Phat, Mhat))
    torch.cuda.synchronize()
    print("ran %d x %s" % (args.steps, args.kernel_only))
    P.close()


def run_gpu(args, rank, local_rank, world):
    import torch

    torch.cuda.set_device(local_rank)
    from paper_2003_05328_gb300 import build as B

    B.build()
    from paper_2003_05328_gb300 import fdsc as F

    c = FI.CONFIGS[WORKLOAD]
    ls = c.layers[0]
    info = F.params_query(ls.n, ls.p)
    g_c, g_b = FI.default_pack(ls, info.S)
    L = F.LayerSpec(ls.B, ls.Ci, ls.Co, ls.H, ls.W, g_c, g_b)
    P = F.Params(ls.n, ls.p, max_T=64)
    F.set_homconv_variant(args.homconv_variant)
    lay = F.layout(P, L)
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    l2 = torch.cuda.get_device_properties(local_rank).L2_cache_size

    # R independent instances of the layer (own weights, masks, shares, key,
    # ciphertext buffers), rotated step by step: every step's filter spectra
    # were last read R - 1 steps earlier, with more than 3x L2 of other data
    # in between, so no step finds its inputs in L2 (no flush needed).
    inst_bytes = 8 * (lay.filter_words + lay.mask_words + lay.ct_in_words + 2 * lay.n_in * ls.n + lay.ct_out_words)
    R = int(min(32, max(4, -(-3 * l2 // inst_bytes))))
    insts = []
    for r in range(R):
        xA_h, xB_h = FI.shares(ls, c.cid, r)
        ks, es, ss = FI.seeds(c.cid, r)
        d = dict(es=es, t_hat=F.keygen(P, ks), Phat=F.filter_prepare(P, L, dev(FI.weights(ls, c.cid, r), np.int8)))
        d["Mhat"], d["sB"] = F.mask_prepare(P, L, ss)
        d["sB4"] = d["sB"].view(ls.B, ls.Co, ls.H, ls.W)
        d["xA"], d["xB"] = dev(xA_h, np.int32), dev(xB_h, np.int32)
        d["XA"], d["XB"] = torch.empty_like(d["xA"]), torch.empty_like(d["xB"])
        d["ct"] = torch.empty(lay.ct_in_words, dtype=torch.int64, device="cuda")
        d["ct_out"] = torch.empty(lay.ct_out_words, dtype=torch.int64, device="cuda")
        d["SA"] = torch.empty(lay.out_spectra_words, dtype=torch.int32, device="cuda")
        d["yA"] = torch.empty((ls.B, ls.Co, ls.H, ls.W), dtype=torch.int32, device="cuda")
        d["yB"] = torch.empty_like(d["yA"])
        d["A_msg"] = torch.empty(lay.n_in * ls.n, dtype=torch.int64, device="cuda")
        d["A_rec"] = torch.empty_like(d["A_msg"])
        d["c1"] = F.encrypt_constants_seeded(P, L, d["t_hat"], es)  # the seeded form: c1 alone
        insts.append(d)
    LAUNCHES_PER_STEP = 4  # producers, HomConv, decryption, Bob's INTT2D
    side = [torch.cuda.Stream() for _ in range(3)]
    s_prod = [torch.cuda.Stream() for _ in range(STAGE_STREAMS[0])]
    s_hc = [torch.cuda.Stream() for _ in range(STAGE_STREAMS[1])]
    s_dec = [torch.cuda.Stream() for _ in range(STAGE_STREAMS[2])]
    s_bob = torch.cuda.Stream()
    stage_streams = s_prod + s_hc + s_dec + [s_bob]

    def step(d):
        """One online layer on the current stream: Alice's encryption
        constants and both parties' share encodings in one launch
        (fdsc_online_produce), then HomConv (+ HomRec addends + HomShare) and
        Alice's fused decryption + INTT2D; Bob's INTT2D of his mask share runs
        on a side stream.  Returns an event recorded after the producers."""
        main = torch.cuda.current_stream()
        side[2].wait_stream(main)
        with torch.cuda.stream(side[2]):
            F.intt2d(P, d["sB4"], out=d["yB"])
        F.online_produce(P, L, d["t_hat"], d["es"], d["xA"], d["xB"], d["ct"], d["A_msg"], d["A_rec"])
        produced = torch.cuda.Event()
        produced.record(main)
        F.homconv_sum(P, L, d["ct"], d["A_msg"], d["A_rec"], d["Phat"], d["Mhat"], out=d["ct_out"])
        F.decrypt_share(P, L, d["t_hat"], d["ct_out"], out=d["yA"])
        main.wait_stream(side[2])
        return produced

    def steps_pipelined(seq):
        """Consecutive steps (independent layers) software-pipelined by stage:
        every step's producers run on a producer stream, its HomConv on a
        HomConv stream once they are done, its decryption on a decryption
        stream once that is done (and Bob's INTT2D on a stream of its own);
        step i takes stream i mod k of a stage with k streams (STAGE_STREAMS:
        two HomConvs and two decryptions of consecutive steps overlap), so
        producers of later steps, HomConvs and decryptions of earlier ones run
        at once.  Every step is the whole layer, in the paper's order.  seq
        holds (instance, buffers) pairs: a step reads its instance's inputs
        (rotated over the R instances) and writes only its own buffers (a set
        per step of the graph), so no stream can overwrite what another still
        reads, however far the producers run ahead."""
        main = torch.cuda.current_stream()
        for st in stage_streams:
            st.wait_stream(main)
        for i, (d, o) in enumerate(seq):
            sp, sh, sd = s_prod[i % len(s_prod)], s_hc[i % len(s_hc)], s_dec[i % len(s_dec)]
            with torch.cuda.stream(sp):
                F.online_produce(P, L, d["t_hat"], d["es"], d["xA"], d["xB"], o["ct"], o["A_msg"], o["A_rec"])
                produced = torch.cuda.Event()
                produced.record(sp)
            with torch.cuda.stream(s_bob):
                F.intt2d(P, d["sB4"], out=o["yB"])
            with torch.cuda.stream(sh):
                sh.wait_event(produced)
                F.homconv_sum(P, L, o["ct"], o["A_msg"], o["A_rec"], d["Phat"], d["Mhat"], out=o["ct_out"])
                convolved = torch.cuda.Event()
                convolved.record(sh)
            with torch.cuda.stream(sd):
                sd.wait_event(convolved)
                F.decrypt_share(P, L, d["t_hat"], o["ct_out"], out=o["yA"])
        for st in stage_streams:
            main.wait_stream(st)

    def step_4streams(d):
        """The previous form of the step: the four producers as separate
        launches on four streams, each step after the one before."""
        main = torch.cuda.current_stream()
        for st in side:
            st.wait_stream(main)
        F.encrypt_constants(P, L, d["t_hat"], d["es"], out=d["ct"])
        with torch.cuda.stream(side[0]):
            F.encode_share(P, L, d["xA"], out=d["A_msg"])
        with torch.cuda.stream(side[1]):
            F.encode_share(P, L, d["xB"], out=d["A_rec"])
        with torch.cuda.stream(side[2]):
            F.intt2d(P, d["sB4"], out=d["yB"])
        for st in side:
            main.wait_stream(st)
        F.homconv_sum(P, L, d["ct"], d["A_msg"], d["A_rec"], d["Phat"], d["Mhat"], out=d["ct_out"])
        F.decrypt_share(P, L, d["t_hat"], d["ct_out"], out=d["yA"])

    def step_unfused(d):
        """The same layer through the step-by-step entry points, one stream."""
        F.ntt2d(P, d["xA"], out=d["XA"])
        F.encrypt(P, L, d["t_hat"], d["XA"], d["es"], out=d["ct"])
        F.ntt2d(P, d["xB"], out=d["XB"])
        F.homrec(P, L, d["XB"], d["ct"])
        F.homconv(P, L, d["ct"], d["Phat"], d["Mhat"], out=d["ct_out"])
        F.decrypt(P, L, d["t_hat"], d["ct_out"], out=d["SA"])
        F.intt2d(P, d["SA"].view(ls.B, ls.Co, ls.H, ls.W), out=d["yA"])
        F.intt2d(P, d["sB4"], out=d["yB"])

    def homconv_only(d):
        F.homconv_sum(P, L, d["ct"], d["A_msg"], d["A_rec"], d["Phat"], d["Mhat"], out=d["ct_out"])

    def homconv_seeded_only(d):
        F.homconv_seeded(P, L, d["es"], d["c1"], d["A_msg"], d["A_rec"], d["Phat"], d["Mhat"], out=d["ct_out"])

    # programmatic dependent launch for the online kernels recorded below:
    # each may start while its predecessor in the stream drains
    F.set_launch_overlap(True)
    for _ in range(max(1, args.warmup)):
        for d in insts:
            step(d)
            step_unfused(d)
    torch.cuda.synchronize()
    # the pipelined graphs: G = min(K, GRAPH_STEPS) steps, each writing its own
    # buffer set (ciphertexts, HomConv output, both output shares)
    G = max(1, min(args.steps, GRAPH_STEPS))
    bufs = [dict(ct=torch.empty_like(insts[0]["ct"]), A_msg=torch.empty_like(insts[0]["A_msg"]),
                 A_rec=torch.empty_like(insts[0]["A_rec"]), ct_out=torch.empty_like(insts[0]["ct_out"]),
                 yA=torch.empty_like(insts[0]["yA"]), yB=torch.empty_like(insts[0]["yB"])) for _ in range(G)]
    pipe_seq = lambda k: [(insts[i % R], bufs[i]) for i in range(k)]
    # the pipelined schedule gives every step's words exactly (checked on the first 2 R steps of a graph)
    ref = [(d["yA"].clone(), d["yB"].clone()) for d in insts]
    n_chk = min(G, 2 * R)
    for o in bufs[:n_chk]:
        o["yA"].zero_()
        o["yB"].zero_()
    # the pipelined schedule decrypts each ciphertext with one CTA: the pair form
    # (two CTAs per ciphertext in a cluster) is faster alone but slower while
    # producers and HomConvs share the GPU (20.8 against 18.4 us per step)
    pair_prev = F.set_decrypt_pair(False)
    steps_pipelined(pipe_seq(n_chk))
    torch.cuda.synchronize()
    pipelined_ok = all(torch.equal(bufs[i]["yA"], ref[i % R][0]) and torch.equal(bufs[i]["yB"], ref[i % R][1])
                       for i in range(n_chk))
    if not pipelined_ok:
        raise RuntimeError("pipelined steps differ from single steps")
    s = torch.cuda.Stream()

    def capture(fn):
        gr = torch.cuda.CUDAGraph()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fn()
            torch.cuda.synchronize()
            with torch.cuda.graph(gr, stream=s):
                fn()
        torch.cuda.current_stream().wait_stream(s)
        return gr

    # exactly K steps: G consecutive steps (cycling over the R instances)
    # recorded in one pipelined graph, replayed K // G times, then a graph of
    # the remaining K mod G steps
    g_main = capture(lambda: steps_pipelined(pipe_seq(G)))
    rem = args.steps % G
    g_rem = capture(lambda: steps_pipelined(pipe_seq(rem))) if rem else None
    F.set_decrypt_pair(pair_prev)
    g_step_pdl = [capture(lambda d=d: step(d)) for d in insts]
    # each instance's producers alone, and followed by its HomConv (one graph
    # each): the difference is the time HomConv adds after the producers' join
    g_prod = [capture(lambda d=d: F.online_produce(P, L, d["t_hat"], d["es"], d["xA"], d["xB"], d["ct"], d["A_msg"],
                                                   d["A_rec"])) for d in insts]
    g_prod_hc = [capture(lambda d=d: (F.online_produce(P, L, d["t_hat"], d["es"], d["xA"], d["xB"], d["ct"],
                                                       d["A_msg"], d["A_rec"]), homconv_only(d))) for d in insts]
    # the rest is recorded without the early launch: kernels measured alone,
    # and one step alone (the early launch lengthens a lone chain of kernels:
    # the dependents' waiting CTAs hold SM room while the earlier kernel runs)
    F.set_launch_overlap(False)
    g_step = [capture(lambda d=d: step(d)) for d in insts]
    g_prod_n = [capture(lambda d=d: F.online_produce(P, L, d["t_hat"], d["es"], d["xA"], d["xB"], d["ct"],
                                                     d["A_msg"], d["A_rec"])) for d in insts]
    g_prod_hc_n = [capture(lambda d=d: (F.online_produce(P, L, d["t_hat"], d["es"], d["xA"], d["xB"], d["ct"],
                                                         d["A_msg"], d["A_rec"]), homconv_only(d))) for d in insts]
    # the four-stream step of the unpipelined form, R steps per graph, each after the one before
    g_4s = capture(lambda: [step_4streams(d) for d in insts])
    g_unfused = [capture(lambda d=d: step_unfused(d)) for d in insts]
    # HomConv alone: one graph of R launches, one per instance, back to back
    g_hc = capture(lambda: [homconv_only(d) for d in insts])
    g_hc_warm = capture(lambda: [homconv_only(insts[0]) for _ in insts])
    g_hc_seeded = capture(lambda: [homconv_seeded_only(d) for d in insts])
    # a reference point of the memory system, not part of the path: one
    # library reduction (torch.sum) over each instance's filter words, the
    # same rotation and graph layout as the HomConv launches
    read_sink = torch.empty((), dtype=torch.int64, device="cuda")
    g_read = capture(lambda: [torch.sum(d["Phat"].view(-1), 0, out=read_sink) for d in insts])
    for _ in range(args.warmup):
        g_main.replay()
        g_hc.replay()
    torch.cuda.synchronize()
    sleep_cycles = int(60e6)  # about 30 ms at 2 GHz

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    def back_to_back(graphs, k, every=0):
        """Replays graphs[i % len] for i < k back to back between two CUDA
        events (plus one at every step boundary when `every`); returns the
        events.  A short spin kernel first lets the host queue steps ahead,
        so no step waits for its launch."""
        ev = [torch.cuda.Event(enable_timing=True) for _ in range((k if every else 1) + 1)]
        torch.cuda._sleep(sleep_cycles)
        ev[0].record()
        for i in range(k):
            graphs[i % len(graphs)].replay()
            if every:
                ev[i + 1].record()
        ev[-1].record()
        return ev

    clocks = ClockSampler(local_rank, args.clocks_dir or tempfile.gettempdir())
    clocks.start()
    time.sleep(0.3)
    barrier()
    seq = [g_main] * (args.steps // G) + ([g_rem] if g_rem is not None else [])
    ev = back_to_back(seq, len(seq))
    barrier()
    total_ms = ev[0].elapsed_time(ev[-1])
    # per-step latency: one step alone per graph, an event at every boundary
    # (the events themselves add a few microseconds per step)
    ev_d = back_to_back(g_step, min(args.steps, 1000), every=1)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev_d[:-2], ev_d[1:-1])]
    ev_dp = back_to_back(g_step_pdl, min(args.steps, 1000), every=1)
    torch.cuda.synchronize()
    step_ms_pdl = [a.elapsed_time(b) for a, b in zip(ev_dp[:-2], ev_dp[1:-1])]
    # the unpipelined four-stream step, R steps per graph launch
    n_4s = max(1, min(args.steps, 2200) // R)
    ev_4 = back_to_back([g_4s], n_4s)
    torch.cuda.synchronize()
    four_stream_ms = ev_4[0].elapsed_time(ev_4[-1]) / (n_4s * R)
    # producers alone vs producers followed by HomConv, one instance per graph
    # launch (rotated: cold filters), an event at every boundary; the median
    # difference is the time HomConv adds after the producers' join
    n_pj = max(2 * R, min(args.steps, 1100))
    ev_p = back_to_back(g_prod, n_pj, every=1)
    ev_ph = back_to_back(g_prod_hc, n_pj, every=1)
    torch.cuda.synchronize()
    t_p = [a.elapsed_time(b) for a, b in zip(ev_p[:-2], ev_p[1:-1])]
    t_ph = [a.elapsed_time(b) for a, b in zip(ev_ph[:-2], ev_ph[1:-1])]
    prod_ms = float(np.median(t_p))
    post_join_ms = float(np.median(t_ph)) - prod_ms
    ev_pn = back_to_back(g_prod_n, n_pj, every=1)
    ev_phn = back_to_back(g_prod_hc_n, n_pj, every=1)
    torch.cuda.synchronize()
    prod_n_ms = float(np.median([a.elapsed_time(b) for a, b in zip(ev_pn[:-2], ev_pn[1:-1])]))
    post_join_n_ms = float(np.median([a.elapsed_time(b) for a, b in zip(ev_phn[:-2], ev_phn[1:-1])])) - prod_n_ms

    # the step-by-step path, for comparison
    n_unfused = min(args.steps, 600)
    ev_u = back_to_back(g_unfused, n_unfused)
    torch.cuda.synchronize()
    unfused_ms = ev_u[0].elapsed_time(ev_u[-1]) / n_unfused

    # HomConv launches alone: R per graph replay, cold (rotated) and warm
    hc_reps = max(4, min(args.steps, 4000) // R)
    ev_h = back_to_back([g_hc], hc_reps)
    ev_w = back_to_back([g_hc_warm], hc_reps)
    torch.cuda.synchronize()
    ev_s = back_to_back([g_hc_seeded], hc_reps)
    torch.cuda.synchronize()
    ev_r = back_to_back([g_read], hc_reps)
    torch.cuda.synchronize()
    read_ms = ev_r[0].elapsed_time(ev_r[-1]) / (hc_reps * R)
    hc_avg = ev_h[0].elapsed_time(ev_h[-1]) / (hc_reps * R)
    hc_warm_ms = ev_w[0].elapsed_time(ev_w[-1]) / (hc_reps * R)
    hc_seeded_ms = ev_s[0].elapsed_time(ev_s[-1]) / (hc_reps * R)

    # NTT2D over a batch sweep of 32x32 planes (64 per image)
    sweep = ntt2d_sweep(F, P, ls, back_to_back, args)
    # the ALU side of the roofline: measured rates of the exact primitives
    calib = {name: F.calibrate(P, i) for i, name in enumerate(("mac_60x60_128", "shoup_mulmod_q", "shoup_mulmod_p"))}
    clk = clocks.stop()

    # end to end through the C ABI with HOST buffers: the serving API, closed loop
    xA_h, xB_h = FI.shares(ls, c.cid, 0)
    e2e = e2e_through_server(F, P, ls, g_c, dev(FI.weights(ls, c.cid, 0), np.int8), insts[0]["t_hat"], xA_h[0],
                             xB_h[0], args.e2e_requests)
    flush = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.int32, device="cuda")
    batched = None if args.skip_batched else run_batched(F, flush, sleep_cycles, args)
    tensor = None if args.skip_batched else run_tensor_homconv(F, flush, args)
    chain = None if args.skip_batched else run_chain(F, flush, sleep_cycles, args)
    binarized = None if args.skip_batched else run_binarized(F, sleep_cycles, args)
    serving = None if args.skip_serving else run_serving(F, args)
    # the same mix at a load where batches form (arrivals faster than one-request batches retire)
    serving_high = None if args.skip_serving else run_serving(F, args, rate=args.serve_high_rate)

    local_sec = total_ms / 1e3
    tot_sec, tot_units = aggregate(local_sec, float(args.steps * ls.B), world)
    e2e_sec, e2e_units = aggregate(e2e["seconds"], float(e2e["requests"]), world)
    if rank != 0:
        return
    value = tot_units / tot_sec
    alg_bytes, macs = layer_counts(ls, lay.T, lay.beta, lay.GB, ls.n)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        tr = json.load(open(TRAFFIC_FILE))
        if tr.get("kernel_digest") == kernel_digest() and tr.get("workload") == WORKLOAD:
            traffic = tr.get("dram_bytes_per_launch")
    achieved = alg_bytes / (hc_avg * 1e-3) / 1e9
    mac_rate = calib["mac_60x60_128"][0]
    t_hbm_us, t_alu_us = alg_bytes / (peak * 1e9) * 1e6, macs / mac_rate * 1e6
    bound = "hbm" if t_hbm_us >= t_alu_us else "alu"
    achieved_mac = macs / (hc_avg * 1e-3)
    hbm_side = {"achieved": achieved, "peak": peak, "peak_source": peak_src + " (hbm_gbs, burst copy)",
                "unit": "GB/s", "frac": achieved / peak, "t_us": t_hbm_us}
    alu_side = {"achieved": achieved_mac / 1e12, "peak": mac_rate / 1e12, "unit": "TMAC/s",
                "frac": achieved_mac / mac_rate, "t_us": t_alu_us, "mac_per_clk_per_sm": calib["mac_60x60_128"][1],
                "peak_source": "measured here (fdsc_calibrate: register-resident loop-carried chains of HomConv's "
                               "exact 60x60->128-bit multiply-accumulate on every SM)"}
    main = hbm_side if bound == "hbm" else alu_side
    pj_us = post_join_ms * 1e3
    roofline = {"kernel": "%s (homconv_sum, variant %d: HomRec addends + HomConv + HomShare)"
                          % (homconv_kernel_name(lay.T, args.homconv_variant), variant_used(lay.T, args.homconv_variant)),
                "bound": bound,
                "achieved": main["achieved"], "peak": main["peak"], "peak_source": main["peak_source"],
                "unit": main["unit"], "frac": main["frac"], "traffic": traffic, "alg_bytes_per_launch": alg_bytes,
                "macs_per_launch": macs, "launch_us": hc_avg * 1e3,
                "timing": "%d launches back to back over the %d instances (cold), CUDA events" % (hc_reps * R, R),
                "hbm": hbm_side, "alu": alu_side,
                "plain_read_reference": {
                    "us": read_ms * 1e3, "bytes": 8 * insts[0]["Phat"].numel(),
                    "frac_of_hbm": 8 * insts[0]["Phat"].numel() / (read_ms * 1e-3) / 1e9 / peak,
                    "what": "torch.sum over one instance's filter words (33.5 MB) per launch, instances rotated "
                            "(cold), R launches per graph replay: what one cold launch of that size reads on "
                            "this part, for comparison with the HomConv launch"},
                "after_producers": {
                    "us": pj_us, "achieved_GB_per_s": alg_bytes / (pj_us * 1e-6) / 1e9,
                    "frac_of_hbm": alg_bytes / (pj_us * 1e-6) / 1e9 / peak,
                    "producers_us": prod_ms * 1e3,
                    "without_early_launch": {"us": post_join_n_ms * 1e3, "producers_us": prod_n_ms * 1e3,
                                             "frac_of_hbm": alg_bytes / (post_join_n_ms * 1e-3) / 1e9 / peak},
                    "definition": "time HomConv adds after the producers' join: median time of a one-instance "
                                  "[online_produce -> homconv_sum] graph minus that of an [online_produce] graph "
                                  "(programmatic dependent launch on, instances rotated: cold filters)"}}
    useful_macs = 2 * ls.Co * ls.Ci * ls.H * ls.W * ls.B
    cpu = cpu_all = None
    if not args.no_cpu_baseline and world == 1:  # the oracle baseline: rank 0 of a single-GPU run
        per_layer, sample = oracle_online_sample(args.cpu_seconds)
        st = oracle_online_sample.stages_ms
        cpu = {"value": 1.0 / per_layer, "unit": "layers/s", "cores": 1, "kind": "oracle", "sample": sample,
               "stages_ms": st}
        t_in = (st["ntt2d_xA"] + st["encrypt"] + st["ntt2d_xB"] + st["homrec"]) * 1e-3
        cpu_all = oracle_all_cores_sample(t_in)
    line = {
        "metric": METRIC, "value": value, "unit": "layers/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "layer": "32x32x64->64 3x3", "batch": ls.B, "n": ls.n, "p": ls.p,
                   "q_bits": 60, "packing": {"g_c": g_c, "g_b": g_b, "T": lay.T},
                   "l2": "inputs larger than L2: %d independent instances of the layer (%d MiB; L2 %d MiB) "
                         "rotated step by step, each step's inputs last read %d steps earlier"
                         % (R, R * inst_bytes >> 20, l2 >> 20, R - 1),
                   "step": "online_produce (encryption constants | encode_share(x_A) | encode_share(x_B), one "
                           "launch) -> homconv_sum (HomRec + HomConv + HomShare) -> decrypt_share, intt2d(s_B) on a "
                           "side stream, programmatic dependent launch; consecutive steps (independent layers) "
                           "pipelined by stage (%d / %d / %d streams for producers / HomConv / decryption, one "
                           "CTA per decrypted ciphertext; each step of a graph writes its own ciphertext and output "
                           "buffers, its inputs rotate over the instances); K steps timed back to back as %d-step graphs (K // %d of them, then one "
                           "of K mod %d); per-step p50/p99 from one step alone per graph with an event at every "
                           "boundary" % (STAGE_STREAMS + (G, G, G)),
                   "homconv_variant": variant_used(lay.T, args.homconv_variant)},
        "mac_per_s": value * 2 * ls.Co * ls.Ci * ls.H * ls.W,
        "homconv_layers_per_s": ls.B / (hc_avg * 1e-3),
        "homconv_mac_per_s": macs / (hc_avg * 1e-3),
        "homconv_warm_us": hc_warm_ms * 1e3,
        "homconv_seeded": {"us": hc_seeded_ms * 1e3, "alg_bytes_per_launch": alg_bytes - 8 * lay.n_in * ls.n,
                           "note": "seeded input ciphertexts: c1 read, c0 drawn again from the encryption seed"},
        "useful_macs_per_layer": useful_macs // ls.B,
        "step_ms_p50": float(np.percentile(step_ms, 50)), "step_ms_p99": float(np.percentile(step_ms, 99)),
        "step_ms_distribution": "%d single steps (not pipelined, without the early launch, the library's "
                                "default) with an event at every boundary" % len(step_ms),
        "step_ms_p50_early_launch": float(np.percentile(step_ms_pdl, 50)),
        "pipelined_words_checked": pipelined_ok,
        "step_by_step_ms": unfused_ms,
        "step_ms_unpipelined_four_streams": four_stream_ms,
        "roofline": roofline,
        "e2e": {"value": e2e_units / e2e_sec, "unit": "layers/s", "h2d_bytes_per_step": e2e["h2d"],
                "d2h_bytes_per_step": e2e["d2h"], "requests": e2e["requests"], "p50_us": e2e["p50_us"],
                "p99_us": e2e["p99_us"], "mean_batch": e2e["mean_batch"],
                "path": "fdsc_server_submit/wait (C ABI) with host buffers, closed loop of single-image requests; "
                        "copies in and out inside the timed region; host wall clock"},
        "batched": batched,
        "homconv_tensor": tensor,
        "chain": chain,
        "binarized": binarized,
        "serving": serving,
        "serving_high_load": serving_high,
        "ntt2d_sweep": sweep,
        "primitive_rates": {k: {"ops_per_s": v[0], "ops_per_clk_per_sm": v[1]} for k, v in calib.items()},
        "gpu_launches": LAUNCHES_PER_STEP * (args.steps + len(step_ms) + len(step_ms_pdl)) + 6 * n_4s * R + 8 * n_unfused
                        + 3 * hc_reps * R + 6 * n_pj + (binarized["launches"] if binarized else 0)
                        + sum(pt["launches"] for pt in sweep["points"]),
        "homconv_variant": args.homconv_variant,
        "clocks": clk,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
    }
    print(json.dumps(line))
    P.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="fdsc", choices=["fdsc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--homconv-variant", type=int, default=0)
    ap.add_argument("--e2e-requests", type=int, default=2000)
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--serve-high-rate", type=float, default=50000.0)
    ap.add_argument("--serve-keys", type=int, default=64)
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--clocks-dir", default="", help="where the raw nvidia-smi clock samples go (default: a temp dir)")
    ap.add_argument("--kernel-only", choices=["homconv", "homconv_b16", "homconv_tc", "ntt2d", "step", "plan",
                                              "binarized"],
                    help="only run --steps launches of one part of the path (for profiler captures)")
    ap.add_argument("--planes", type=int, default=65536, help="planes for --kernel-only ntt2d")
    args = ap.parse_args()
    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "fdsc" else "gloo"
        dist.init_process_group(backend)
    try:
        if args.kernel_only:
            run_kernel_only(args)
        elif args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gpu(args, rank, local_rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
