#!/usr/bin/env python
"""Throughput of batched TabNet inference (logits + per-step masks +
aggregated mask written to device memory) on B300.

Default workload: the 35-input model (26 numeric: 13 lognormal(0,1), 13
ordinal 1..5; 9 categorical with cardinalities 2..10), n_d = n_a = 32, 5
decision steps, 2 classes, 65,536 rows per batch, seeded synthetic data and
weights, split-bf16 tensor-core precision (the mode that meets the bf16
tolerances against the FP64 oracle).  One step = one forward over one batch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own batch on its own GPU (weak scaling, no
collective on the data path); rank 0 prints one JSON line.  The reference
arm (--impl reference) times the FP64 CPU oracle on bounded samples of the
same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TabNet rows/s (logits+masks) BF16 vs FP32 at stated tol"
UNIT = "rows/s"
L2_BYTES = 126 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "bf16", "bf16x6", "fp8", "fp32"])
    ap.add_argument("--no-extras", action="store_true", help="skip the comparison arms")
    ap.add_argument("--no-tune", action="store_true", help="keep the library's default launch shape")
    return ap.parse_args()


def describe(name):
    from paper_2510_19689_b300 import synth
    s = synth.SPECS[name]
    return (f"{name}: {synth.ROWS[name]:,} rows x {s.n_feat} inputs ({s.n_num} numeric, {s.n_cat} categorical, "
            f"embedding dim {s.cat_emb_dim[0]}), n_d=n_a={s.n_d}, {s.n_steps} steps, {s.n_classes} classes")


def mac_per_row(params):
    """Algorithmic multiply-adds of one row: every FC at its true width."""
    N = params["n_d"] + params["n_a"]
    de = params["n_num"] + sum(params["cat_emb_dim"])
    lpf = params["n_shared"] + params["n_indep"]
    ft = de * 2 * N + (lpf - 1) * N * 2 * N
    return ((params["n_steps"] + 1) * ft + params["n_steps"] * params["n_a"] * de
            + params["n_d"] * params["n_classes"])


def bytes_per_row(params):
    de = params["n_num"] + sum(params["cat_emb_dim"])
    d = params["n_num"] + len(params["cat_card"])
    inp = 4 * params["n_num"] + 4 * len(params["cat_card"])
    out = 4 * params["n_classes"] + 4 * params["n_steps"] * de + 4 * d
    return inp, out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            j = json.load(f)
        return dict(hbm=j["hbm_gbs"], bf16=j["bf16_tflops"], bf16_sus=j["bf16_tflops_sustained"], src="measured")
    return dict(hbm=6400.0, bf16=1800.0, bf16_sus=1400.0, src="fallback")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2510_19689_b300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.startswith("tc_"):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, precision):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"tc_forward_{workload}_{precision}.md")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as f:
        for line in f:
            if line.startswith("- ") and "=" in line:
                k, v = line[2:].split("=", 1)
                kv[k.strip()] = v.strip().strip("`")
    if kv.get("kernel_source_sha") != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_rows_per_s(params, x_num, x_cat):
    """The FP64 oracle as it stands on the host cores, on a bounded sample."""
    from oracle import tabnet_oracle as O
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    t0 = time.perf_counter()
    O.forward(params, x_num, x_cat)
    dt = time.perf_counter() - t0
    return x_num.shape[0] / dt, cores, dt


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2510_19689_b300 import synth
    name = args.workload
    params = synth.make_params(synth.SPECS[name], synth.weight_seed(name))
    # size each step's sample so that warm-up + timed steps take ~1 minute
    probe_rows = {"c1": 1024, "c2": 1024, "c3": 128}[name]
    xp, cp = synth.make_rows(name, probe_rows)
    rate, _, _ = oracle_rows_per_s(params, xp, cp)
    budget_rows = rate * 60.0 / max(1, args.steps + args.warmup)
    sample_rows = int(min({"c1": 4096, "c2": 2048, "c3": 512}[name], max(16, budget_rows)))
    x_num, x_cat = synth.make_rows(name, sample_rows)
    for _ in range(max(0, args.warmup)):
        oracle_rows_per_s(params, x_num, x_cat)
    ts = []
    cores = None
    for _ in range(args.steps):
        r, cores, dt = oracle_rows_per_s(params, x_num, x_cat)
        ts.append(dt)
    ms = 1e3 * sum(ts) / len(ts)
    value = sample_rows / (ms / 1e3)
    sample = f"{sample_rows} rows of the {name} workload per step (float64 numpy oracle)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe(name), "sample_rows": sample_rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def bench_batching(model, params, dev, stream, n_segs=4096, max_rows=4096, reps=20):
    """Uneven request batches: n_segs requests with log-uniform row counts in
    [1, max_rows], each with its own buffers, served by one segmented launch
    (device descriptors) captured in a CUDA graph and replayed."""
    import numpy as np
    import torch
    from paper_2510_19689_b300 import synth, tabnet
    sizes = synth.segment_rows(n_segs, max_rows, seed=2004)
    total = int(sizes.sum())
    x_num, x_cat = synth.make_rows("c2", total, seed=2005)
    d = model.dims
    xn = torch.from_numpy(x_num).to(dev)
    xc = torch.from_numpy(x_cat).to(dev)
    lg = torch.empty((total, d.n_classes), device=dev)
    mk = torch.empty((total, d.n_steps, d.d_emb), device=dev)
    ag = torch.empty((total, d.n_feat), device=dev)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    segs = [dict(rows=int(sizes[i]), x_num=xn[offs[i]:], x_cat=xc[offs[i]:], logits=lg[offs[i]:],
                 masks=mk[offs[i]:], agg=ag[offs[i]:]) for i in range(n_segs)]
    desc = torch.frombuffer(bytearray(bytes(tabnet.segment_array(segs))), dtype=torch.uint8).to(dev)
    model.reserve_segments(n_segs)
    model.forward_segments_device(desc, n_segs, stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream(dev)
    cs.wait_stream(stream)
    with torch.cuda.stream(cs):
        with torch.cuda.graph(g, stream=cs):
            model.forward_segments_device(desc, n_segs, stream=cs)
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"value": total / (ms / 1e3), "unit": UNIT, "segments": n_segs, "rows": total,
            "ms_per_launch": ms, "launch": "one persistent kernel per replay of a captured CUDA graph "
                                         "(prefix-sum scan + forward)"}


def fp8_gemm_peak(dev, n=8192, reps=10):
    """Dense E4M3 x E4M3 -> bf16 GEMM rate of this GPU through PyTorch's scaled
    matmul (cuBLASLt), n^3, best of `reps`: the FP8 tensor peak a fused FP8
    path would be measured against (no such path is offered; see the
    rounding study)."""
    import torch
    try:
        a = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn).t()
        one = torch.ones((), device=dev)
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return {"value": 2.0 * n ** 3 / (best / 1e3) / 1e12, "unit": "TFLOP/s",
                "how": f"torch._scaled_mm e4m3 {n}^3, best of {reps}"}
    except Exception as exc:  # an older PyTorch without the scaled matmul
        return {"value": None, "unavailable": str(exc)[:200]}


def bench_serving(dev_index, rates=(1000, 5000, 20000, 50000, 100000, 200000), seconds=1.0,
                  streams_per_model=8, max_inflight_batches=32):
    """Poisson arrivals at each rate for `seconds`, request sizes
    floor(exp(U(0, ln 513))) in [1, 512] rows, the three model shapes
    resident (split-bf16), model chosen uniformly; the server's latency
    (completion seen on the host - submission) and completed rows/s."""
    import numpy as np
    from paper_2510_19689_b300 import synth, tabnet
    names = ["c1", "c2", "c3"]
    models = [tabnet.Model(synth.to_blob(synth.make_params(synth.SPECS[n], synth.weight_seed(n))), "bf16x3",
                           device=dev_index) for n in names]
    pools = [synth.make_rows(n, 512, seed=5000 + i) for i, n in enumerate(names)]
    srv = tabnet.Server(models, device_bytes=2 << 30, streams_per_model=streams_per_model,
                        max_inflight_batches=max_inflight_batches)
    out = []
    for rate in rates:
        rng = np.random.default_rng(rate)
        n = int(rate * seconds)
        t = np.cumsum(rng.exponential(1.0 / rate, n))
        sizes = np.clip(np.floor(np.exp(rng.uniform(0, math.log(513), n))), 1, 512).astype(int)
        which = rng.integers(0, 3, n)
        reqs = [(int(which[k]), pools[which[k]][0][:sizes[k]], pools[which[k]][1][:sizes[k]], float(t[k]))
                for k in range(n)]
        prepared = srv.prepare_replay(reqs)  # marshalling stays outside the timed region
        srv.reset_stats()
        t0 = time.perf_counter()
        srv.replay_prepared(prepared)
        wall = time.perf_counter() - t0
        st = srv.stats()
        out.append({"offered_req_per_s": rate, "requests": n, "completed": st["completed"],
                    "achieved_req_per_s": st["completed"] / wall, "rows_per_s": st["rows_completed"] / wall,
                    "p50_ms": st["p50_ms"], "p95_ms": st["p95_ms"], "p99_ms": st["p99_ms"],
                    "mean_batch_rows": st["mean_batch_rows"], "batches": st["batches"]})
    srv.close()
    for m in models:
        m.close()
    return {"models": "14-, 35- and 100-input models resident, split-bf16", "request_rows": "log-uniform 1..512",
            "rates": out}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    from paper_2510_19689_b300 import autotune, replicas, synth, tabnet

    # one process per GPU; rows are independent, so each rank runs its own
    # replica on its own batch (weak scaling, no collective in the step)
    group = replicas.Group("nccl")
    world, rank, local = group.world, group.rank, group.local
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    name = args.workload
    params, blob, x_num_h, x_cat_h = synth.load_config(name)
    rows = x_num_h.shape[0]
    model = tabnet.Model(blob, args.precision, device=local)
    d = model.dims
    inp_b, out_b = bytes_per_row(params)
    set_bytes = rows * (inp_b + out_b)
    n_sets = max(2, math.ceil(2 * L2_BYTES / set_bytes))
    sets = []
    for _ in range(n_sets):
        sets.append(dict(
            xn=torch.from_numpy(x_num_h).to(dev), xc=torch.from_numpy(x_cat_h).to(dev),
            lg=torch.empty((rows, d.n_classes), device=dev),
            mk=torch.empty((rows, d.n_steps, d.d_emb), device=dev),
            ag=torch.empty((rows, d.n_feat), device=dev)))
    stream = torch.cuda.current_stream(dev)

    def step(k):
        s = sets[k % n_sets]
        model.forward(s["xn"], s["xc"], rows, s["lg"], s["mk"], s["ag"], stream=stream)

    tile = None
    if args.precision != "fp32":
        s0 = sets[0]
        if not args.no_tune:
            autotune.tune(model, s0["xn"], s0["xc"], rows, s0["lg"], s0["mk"], s0["ag"], stream=stream,
                          cache_path=None)
        tile = model.tile_config()

    # parity on a sample against the FP64 oracle (bench inputs, bench launch shape)
    step(0)
    torch.cuda.synchronize()
    status = model.poll_status()
    from oracle import tabnet_oracle as O
    idx = np.linspace(0, rows - 1, 256).astype(np.int64)
    rl, rm, ra = O.forward(params, x_num_h[idx], x_cat_h[idx])
    it = torch.from_numpy(idx).to(dev)
    lg = sets[0]["lg"][it].cpu().numpy()
    mk = sets[0]["mk"][it].cpu().numpy()
    ag = sets[0]["ag"][it].cpu().numpy()
    parity = {"sample_rows": len(idx), "logit_abs_max": float(np.abs(lg - rl).max()),
              "mask_l1_max": float(np.abs(mk - rm).sum((1, 2)).max()),
              "agg_l1_max": float(np.abs(ag - ra).sum(1).max()),
              "argmax_agreement": float((lg.argmax(1) == rl.argmax(1)).mean()), "status": status}

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    group.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # an event after every step (recorded on the stream, no synchronisation)
    # gives the per-step spread; the total is e0 -> e1 as always
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(args.steps):
            step(k)
            marks[k].record(stream)
        e1.record(stream)
        e1.synchronize()
    group.barrier()
    per_step = [e0.elapsed_time(marks[0])] + [marks[k - 1].elapsed_time(marks[k]) for k in range(1, args.steps)]
    step_stats = {"min": float(np.min(per_step)), "median": float(np.median(per_step)),
                  "max": float(np.max(per_step))}
    ms_total = group.max(e0.elapsed_time(e1))
    ms_step = ms_total / args.steps
    value = replicas.throughput(group.sum(rows * args.steps), ms_total)
    clocks = clk.summary()

    extras = {}
    if rank == 0:
        # end to end through the host-buffer entry point (pinned host memory)
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        xn_p, xc_p = pin(x_num_h), pin(x_cat_h)
        lg_p = torch.empty((rows, d.n_classes)).pin_memory().numpy()
        mk_p = torch.empty((rows, d.n_steps, d.d_emb)).pin_memory().numpy()
        ag_p = torch.empty((rows, d.n_feat)).pin_memory().numpy()
        host_args = [tabnet._ptr(xn_p), tabnet._ptr(xc_p), rows, tabnet._ptr(lg_p), tabnet._ptr(mk_p),
                     tabnet._ptr(ag_p), stream.cuda_stream]
        L = tabnet.lib()
        for _ in range(3):
            tabnet._check(L.tabnet_forward_host(model._h, *host_args), "tabnet_forward_host")
        e2e_steps = 20
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            tabnet._check(L.tabnet_forward_host(model._h, *host_args), "tabnet_forward_host")
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        extras["e2e"] = {"value": rows / e2e_s, "unit": UNIT, "h2d_bytes_per_step": rows * inp_b,
                         "d2h_bytes_per_step": rows * out_b}

    pk = peaks()
    flop_launch = 2.0 * mac_per_row(params) * rows
    achieved = flop_launch / (ms_step / 1e3) / 1e12
    sustained = ms_total > 1000.0
    peak = pk["bf16_sus"] if sustained else pk["bf16"]
    traffic = profiled_traffic(name, args.precision) if args.precision != "fp32" else None
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_kind": ("bf16 sustained" if sustained else "bf16 burst") + f", of {pk['src']}",
                "flop_per_launch": flop_launch,
                "hbm_frac": (rows * (inp_b + out_b)) / (ms_step / 1e3) / 1e9 / pk["hbm"]}

    if rank == 0 and not args.no_extras:
        # the FP64 oracle on the host cores: a bounded sample of about 10 s of
        # CPU work (the batch's first rows, the whole batch repeated when it
        # takes less), sized from a short probe
        from oracle import tabnet_oracle as O
        n_probe = {"c1": 256, "c2": 1024, "c3": 128}[name]
        rp, cores, _ = oracle_rows_per_s(params, x_num_h[:n_probe], x_cat_h[:n_probe])
        n_cpu = int(min(rows, max(n_probe, rp * 10.0)))
        _, _, t_one = oracle_rows_per_s(params, x_num_h[:n_cpu], x_cat_h[:n_cpu])  # one pass at full size
        reps = max(1, int(round(10.0 / t_one)))
        t0 = time.perf_counter()
        for _ in range(reps):
            O.forward(params, x_num_h[:n_cpu], x_cat_h[:n_cpu])
        dt = time.perf_counter() - t0
        extras["cpu_baseline"] = {"value": n_cpu * reps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": f"first {n_cpu} rows of the {name} batch x {reps} passes, "
                                            f"float64 numpy ({dt:.1f} s)"}
        # the same oracle held to one host thread (a child process whose BLAS
        # pools are limited by the environment before numpy loads), about 5 s
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = ("import sys, time, json; sys.path.insert(0, %r); from paper_2510_19689_b300 import synth; "
                "from oracle import tabnet_oracle as O; p, _, xn, xc = synth.load_config(%r); "
                "t = time.perf_counter(); O.forward(p, xn[:%d], xc[:%d]); r = %d / (time.perf_counter() - t); "
                "n = int(min(len(xn), max(%d, r * 5.0))); "
                "t = time.perf_counter(); O.forward(p, xn[:n], xc[:n]); k = max(1, int(round(5.0 / (time.perf_counter() - t)))); "
                "t = time.perf_counter(); [O.forward(p, xn[:n], xc[:n]) for _ in range(k)]; "
                "dt = time.perf_counter() - t; print(json.dumps([n * k / dt, n, k, dt]))"
                ) % (ROOT, name, n_probe, n_probe, n_probe, n_probe)
        try:
            out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
            r1, n1, k1, dt1 = json.loads(out.stdout.strip().splitlines()[-1])
            extras["cpu_baseline"]["one_core"] = {"value": r1,
                                                  "sample": f"first {n1} rows x {k1} passes ({dt1:.1f} s)"}
        except Exception as exc:
            extras["cpu_baseline"]["one_core"] = {"value": None, "unavailable": str(exc)[:200]}
        # plain FP32 unfused GPU forward (PyTorch eager, TF32 off): the 5x target's divisor
        from paper_2510_19689_b300.unfused import UnfusedTabNet
        un = UnfusedTabNet(params, dev)
        s0 = sets[0]
        for _ in range(3):
            un.forward(s0["xn"], s0["xc"])
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(10):
            un.forward(s0["xn"], s0["xc"])
        a1.record()
        a1.synchronize()
        un_ms = a0.elapsed_time(a1) / 10
        extras["fp32_unfused"] = {"value": rows / (un_ms / 1e3), "unit": UNIT, "ms_per_step": un_ms}
        extras["speedup_vs_fp32_unfused"] = value / world / extras["fp32_unfused"]["value"]
        # the other precisions of the fused library on the same batch (the
        # three-part split only where the model shape has it)
        for prec in ("bf16", "bf16x6", "fp32"):
            if prec == args.precision:
                continue
            try:
                m2 = tabnet.Model(blob, prec, device=local)
            except tabnet.TabnetError as exc:
                extras[f"fused_{prec}"] = {"value": None, "unavailable": str(exc)[:200]}
                continue
            if prec != "fp32" and not args.no_tune:
                autotune.tune(m2, s0["xn"], s0["xc"], rows, s0["lg"], s0["mk"], s0["ag"], stream=stream,
                              cache_path=None)
            reps = 20 if prec != "fp32" else 3
            for _ in range(2):
                m2.forward(s0["xn"], s0["xc"], rows, s0["lg"], s0["mk"], s0["ag"], stream=stream)
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            for k in range(reps):
                s = sets[k % n_sets]
                m2.forward(s["xn"], s["xc"], rows, s["lg"], s["mk"], s["ag"], stream=stream)
            b1.record(stream)
            b1.synchronize()
            # the same 256 sampled rows against the FP64 oracle
            m2.forward(s0["xn"], s0["xc"], rows, s0["lg"], s0["mk"], s0["ag"], stream=stream)
            torch.cuda.synchronize()
            lg2 = s0["lg"][it].cpu().numpy()
            mk2 = s0["mk"][it].cpu().numpy()
            ag2 = s0["ag"][it].cpu().numpy()
            extras[f"fused_{prec}"] = {
                "value": rows / (b0.elapsed_time(b1) / reps / 1e3), "unit": UNIT,
                "parity": {"logit_rel_max": float((np.abs(lg2 - rl) / np.maximum(np.abs(rl), 1)).max()),
                           "mask_l1_max": float(np.abs(mk2 - rm).sum((1, 2)).max()),
                           "agg_l1_max": float(np.abs(ag2 - ra).sum(1).max()), "status": m2.poll_status()}}
            m2.close()

    if rank == 0 and not args.no_extras and args.precision != "fp32":
        # audit statistics over the step's aggregate (mean, variance, top-5
        # frequency per feature): the aggregate read twice plus once per row
        ag0 = sets[0]["ag"]
        for _ in range(3):
            tabnet.mask_stats(ag0, 5, stream=stream)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(20):
            tabnet.mask_stats(ag0, 5, stream=stream)
        a1.record(stream)
        a1.synchronize()
        ms_stats = a0.elapsed_time(a1) / 20
        extras["mask_stats"] = {"ms": ms_stats, "rows_per_s": rows / (ms_stats / 1e3), "k": 5,
                                "aggregate_bytes": rows * d.n_feat * 4}

    if rank == 0 and not args.no_extras and name == "c2":
        # a fresh process's first call (the serverless cold start), on the
        # paper's model shape (14 inputs, n_d = n_a = 8, 3 steps)
        extras["cold_start"] = {}
        for mode in ("torch", "notorch"):
            try:
                out = subprocess.run([sys.executable, "-m", "paper_2510_19689_b300.cold_start", "c1", "1000",
                                      "bf16x3", mode], cwd=ROOT, capture_output=True, text=True, timeout=600)
                extras["cold_start"][mode] = json.loads(out.stdout.strip().splitlines()[-1])
            except Exception as exc:
                extras["cold_start"][mode] = {"unavailable": str(exc)[:200]}

    if rank == 0 and not args.no_extras and name == "c3":
        extras["fp8_gemm_peak"] = fp8_gemm_peak(dev)

    if rank == 0 and not args.no_extras and args.precision != "fp32" and name == "c2":
        extras["batching"] = bench_batching(model, params, dev, stream)
        extras["serving"] = bench_serving(local)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "ms_per_step_stats": step_stats,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if args.precision != "fp32" else "f32", "data": "synthetic",
            "config": {"workload": describe(name), "rows_per_gpu": rows, "precision": args.precision,
                       "parallelism": f"replicas x{world} (rows sharded per GPU, no collective)",
                       "l2": f"{n_sets} rotating input/output sets of {set_bytes / 1e6:.1f} MB "
                             f"({n_sets * set_bytes / 1e6:.0f} MB > L2)",
                       "tile": tile},
            "gpu_launches": args.steps,
            "clocks": clocks,
            "roofline": roofline,
            "parity": parity,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    model.close()
    group.close()


if __name__ == "__main__":
    main()
