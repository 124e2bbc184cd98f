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
    """SM clock, power and throttle reasons sampled while running: through
    NVML every `period_s` (0.25 ms by default, so that even a few-millisecond
    timed region is sampled several times), else through nvidia-smi every
    200 ms."""

    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4))

    def __init__(self, device, period_s=0.00025):
        self.device = device
        self.period_s = period_s
        self.samples = []  # (sm_mhz, max_sm_mhz, power_w, reason bits)
        self.proc = None
        self.thread = None
        self.how = None

    @staticmethod
    def _nvml():
        """The driver's NVML library through ctypes (documented C API)."""
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        return lib

    def _nvml_handle(self, lib):
        import ctypes
        import torch
        h = ctypes.c_void_p()
        props = torch.cuda.get_device_properties(self.device)
        bus = getattr(props, "pci_bus_id", None)
        if bus is not None:
            pci = f"{getattr(props, 'pci_domain_id', 0):08x}:{bus:02x}:{getattr(props, 'pci_device_id', 0):02x}.0"
            if lib.nvmlDeviceGetHandleByPciBusId_v2(pci.encode(), ctypes.byref(h)) == 0:
                return h
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.device), ctypes.byref(h)) != 0:
            raise OSError("no NVML handle")
        return h

    def __enter__(self):
        import ctypes
        import threading
        try:
            lib = self._nvml()
            h = self._nvml_handle(lib)
            mx, sm, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) != 0:  # 1 = NVML_CLOCK_SM
                raise OSError("NVML max clock")
            reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.stop = threading.Event()

            def run():
                # the clock and the reasons every period; the power reading
                # (a slower query) at most every 20 ms, so that a timed
                # region of a few milliseconds still gets several samples
                t_pw = -1.0
                while not self.stop.is_set():
                    now = time.perf_counter()
                    if now - t_pw >= 0.02 and lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw)) == 0:
                        t_pw = now
                    if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(sm)) == 0
                            and reasons(h, ctypes.byref(rs)) == 0):
                        self.samples.append((float(sm.value), float(mx.value), pw.value / 1000.0, int(rs.value)))
                    self.stop.wait(self.period_s)

            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            self.how = f"NVML every {self.period_s * 1e3:g} ms"
        except Exception:
            self.thread = None
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.device),
                     "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
                     "--format=csv,noheader,nounits", "-lms", "200"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.how = "nvidia-smi every 200 ms"
            except OSError:
                self.proc = None
        return self

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            for l in out.splitlines():
                f = [x.strip() for x in l.split(",")]
                try:
                    self.samples.append((float(f[0]), float(f[1]), float(f[2]), int(f[3], 16)))
                except (ValueError, IndexError):
                    continue

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "how": self.how}
        sm = [x[0] for x in self.samples]
        reasons = sorted({n for *_, bits in self.samples for n, b in self.REASONS if bits & b})
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm), "sm_max_mhz": max(x[1] for x in self.samples),
                "power_w_max": max(x[2] for x in self.samples), "reasons": reasons, "samples": len(sm),
                "how": self.how}


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
    world = int(os.environ.get("WORLD_SIZE", "1"))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(name, args.precision, world), "sample_rows_per_step": sample_rows,
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


def bench_serving(dev_index, rates=(1000, 5000, 20000, 50000, 100000, 200000), seconds=None,
                  streams_per_model=16, max_inflight_batches=32, batch_min_rows=2048, batch_wait_us=200,
                  clients=8, batch_busy=2):
    """Poisson arrivals at each rate for `seconds` (default: long enough
    for 100,000 requests, at least 1 s and at most 10 s; the first 10 % of
    the requests are warm-up, left out of the latency statistics), request sizes
    floor(exp(U(0, ln 513))) in [1, 512] rows, the three model shapes
    resident (split-bf16), model chosen uniformly, submitted by `clients`
    threads; the server's latency (completion seen on the host - scheduled
    arrival, so a late submission counts) and completed rows/s."""
    import numpy as np
    from paper_2510_19689_b300 import synth, tabnet
    names = ["c1", "c2", "c3"]
    models = [tabnet.Model(synth.to_blob(synth.make_params(synth.SPECS[n], synth.weight_seed(n))), "bf16x3",
                           device=dev_index) for n in names]
    pools = [synth.make_rows(n, 512, seed=5000 + i) for i, n in enumerate(names)]
    srv = tabnet.Server(models, device_bytes=2 << 30, streams_per_model=streams_per_model,
                        max_inflight_batches=max_inflight_batches, batch_min_rows=batch_min_rows,
                        batch_wait_us=batch_wait_us, batch_busy=batch_busy)
    out = []
    for rate in rates:
        rng = np.random.default_rng(rate)
        secs = seconds if seconds is not None else min(10.0, max(1.0, 1e5 / rate))
        n = int(rate * secs)
        warm = n // 10
        t = np.cumsum(rng.exponential(1.0 / rate, n))
        sizes = np.clip(np.floor(np.exp(rng.uniform(0, math.log(513), n))), 1, 512).astype(int)
        which = rng.integers(0, 3, n)
        reqs = [(int(which[k]), pools[which[k]][0][:sizes[k]], pools[which[k]][1][:sizes[k]], float(t[k]))
                for k in range(n)]
        prepared = srv.prepare_replay(reqs)  # marshalling stays outside the timed region
        srv.reset_stats()
        t0 = time.perf_counter()
        srv.replay_prepared(prepared, threads=clients, warmup=warm)
        wall = time.perf_counter() - t0
        st = srv.stats()
        out.append({"offered_req_per_s": rate, "seconds": secs, "requests": n, "warmup_requests": warm,
                    "completed": st["completed"],
                    "achieved_req_per_s": st["completed"] / wall, "rows_per_s": st["rows_completed"] / wall,
                    "p50_ms": st["p50_ms"], "p95_ms": st["p95_ms"], "p99_ms": st["p99_ms"],
                    "mean_batch_rows": st["mean_batch_rows"], "batches": st["batches"],
                    "engine_staged": st["engine_staged"], "p50_queue_ms": st["p50_queue_ms"],
                    "p99_queue_ms": st["p99_queue_ms"], "engine_busy": st["engine_busy"],
                    "engine_max_pass_ms": st["engine_max_pass_ms"], "replay_max_late_ms": st["replay_max_late_ms"],
                    "p50_from_submit_ms": st["p50_submit_ms"], "p99_from_submit_ms": st["p99_submit_ms"]})
    srv.close()
    for m in models:
        m.close()
    return {"models": "14-, 35- and 100-input models resident, split-bf16", "request_rows": "log-uniform 1..512",
            "clients": clients, "latency": "completion seen on the host - scheduled arrival",
            "server": {"streams_per_model": streams_per_model, "max_inflight_batches": max_inflight_batches,
                       "batch_min_rows": batch_min_rows, "batch_wait_us": batch_wait_us, "batch_busy": batch_busy,
                       "step_masks": "compact (count + column/value slots) for the 35- and 100-input models, "
                                     "dense for the 14-input one"},
            "rates": out}


def bench_latency(dev, calls=200, host_calls=100):
    """The 14-input model's 1,024-row call (n_d = n_a = 8, 3 steps): per-call
    device time back to back over rotating input sets, and the latency one
    synchronous call shows on the host (launch included), for the float32
    path (its warp-per-row kernel at this size) and split-bf16."""
    import numpy as np
    import torch
    out = {"workload": describe("c1"), "rows_per_call": None, "arms": {}}
    for prec in ("fp32", "bf16x3"):
        w = Workload("c1", prec, dev)
        w.tune()
        out["rows_per_call"] = w.rows
        ms, stats, clocks = w.time(calls, 10)
        # the same calls back to back with no event between them (the
        # per-call marks above add a little to every call)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(w.stream)
        for k in range(calls):
            w.step(k)
        e1.record(w.stream)
        e1.synchronize()
        ms_plain = e0.elapsed_time(e1)
        lat = []
        for k in range(host_calls):
            t0 = time.perf_counter()
            w.step(k)
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - t0)
        lat = np.array(lat) * 1e3
        out["arms"][prec] = {"ms_per_call": ms / calls, "ms_per_call_stats": stats,
                             "ms_per_call_unmarked": ms_plain / calls,
                             "rows_per_s": w.rows * calls / (ms / 1e3),
                             "host_latency_ms": {"p50": float(np.median(lat)), "p99": float(np.quantile(lat, 0.99))},
                             "tile": w.tile, "clocks": clocks, "parity": w.parity(256)}
        w.close()
        del w
        torch.cuda.empty_cache()
    return out


def spec_params(name):
    """The shape fields of workload ``name`` (what the MAC and byte counts read)."""
    from paper_2510_19689_b300 import synth
    sp = synth.SPECS[name]
    return dict(n_num=sp.n_num, cat_card=list(sp.cat_card), cat_emb_dim=list(sp.cat_emb_dim), n_d=sp.n_d,
                n_a=sp.n_a, n_steps=sp.n_steps, n_classes=sp.n_classes, n_shared=sp.n_shared, n_indep=sp.n_indep)


def n_sets_for(name):
    """Rotating input/output sets so that consecutive steps never find their
    buffers in L2 (at least twice L2 in all)."""
    from paper_2510_19689_b300 import synth
    inp_b, out_b = bytes_per_row(spec_params(name))
    set_bytes = synth.ROWS[name] * (inp_b + out_b)
    return max(2, math.ceil(2 * L2_BYTES / set_bytes)), set_bytes


def workload_config(name, precision, world):
    """The `config` object of the JSON line -- the same in both arms."""
    from paper_2510_19689_b300 import synth
    n_sets, set_bytes = n_sets_for(name)
    return {"workload": describe(name), "rows_per_gpu": synth.ROWS[name], "precision": precision,
            "parallelism": f"replicas x{world} (rows sharded per GPU, no collective)",
            "l2": f"{n_sets} rotating input/output sets of {set_bytes / 1e6:.1f} MB "
                  f"({n_sets * set_bytes / 1e6:.0f} MB > L2)"}


class Workload:
    """One workload resident on the device: its model at one precision and
    `n_sets` rotating input/output sets."""

    def __init__(self, name, precision, dev, data=None):
        import torch
        from paper_2510_19689_b300 import synth, tabnet
        self.name, self.precision, self.dev = name, precision, dev
        self.params, self.blob, self.x_num, self.x_cat = data if data is not None else synth.load_config(name)
        self.rows = self.x_num.shape[0]
        self.model = tabnet.Model(self.blob, precision, device=dev.index)
        d = self.model.dims
        self.n_sets, _ = n_sets_for(name)
        xn = torch.from_numpy(self.x_num).to(dev)
        xc = torch.from_numpy(self.x_cat).to(dev)
        self.sets = [dict(xn=xn if k == 0 else xn.clone(), xc=xc if k == 0 else xc.clone(),
                          lg=torch.empty((self.rows, d.n_classes), device=dev),
                          mk=torch.empty((self.rows, d.n_steps, d.d_emb), device=dev),
                          ag=torch.empty((self.rows, d.n_feat), device=dev)) for k in range(self.n_sets)]
        self.stream = torch.cuda.current_stream(dev)
        self.tile = None

    def step(self, k):
        s = self.sets[k % self.n_sets]
        self.model.forward(s["xn"], s["xc"], self.rows, s["lg"], s["mk"], s["ag"], stream=self.stream)

    def tune(self, enabled=True):
        from paper_2510_19689_b300 import autotune
        if self.precision != "fp32":
            if enabled:
                s0 = self.sets[0]
                autotune.tune(self.model, s0["xn"], s0["xc"], self.rows, s0["lg"], s0["mk"], s0["ag"],
                              stream=self.stream, cache_path=None)
            self.tile = self.model.tile_config()

    def time(self, steps, warmup, group=None):
        """Exactly `steps` steps between synchronised events (max over ranks);
        clocks sampled in the region."""
        import numpy as np
        import torch
        for k in range(warmup):
            self.step(k)
        torch.cuda.synchronize()
        if group:
            group.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        with ClockSampler(self.dev.index) as clk:
            torch.cuda.synchronize()
            e0.record(self.stream)
            for k in range(steps):
                self.step(k)
                marks[k].record(self.stream)
            e1.record(self.stream)
            e1.synchronize()
        if group:
            group.barrier()
        per = [e0.elapsed_time(marks[0])] + [marks[k - 1].elapsed_time(marks[k]) for k in range(1, steps)]
        ms_total = group.max(e0.elapsed_time(e1)) if group else e0.elapsed_time(e1)
        return ms_total, {"min": float(np.min(per)), "median": float(np.median(per)), "max": float(np.max(per))}, \
            clk.summary()

    def sustained(self, seconds=1.0, batch=50):
        """Steps back to back for at least `seconds` of device time, clocks
        sampled throughout: the rate under the power cap."""
        import torch
        done, ms = 0, 0.0
        with ClockSampler(self.dev.index, period_s=0.005) as clk:
            while ms < 1e3 * seconds:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                for k in range(batch):
                    self.step(done + k)
                e1.record(self.stream)
                e1.synchronize()
                ms += e0.elapsed_time(e1)
                done += batch
        return {"value": self.rows * done / (ms / 1e3), "unit": UNIT, "steps": done, "seconds": ms / 1e3,
                "ms_per_step": ms / done, "clocks": clk.summary()}

    def e2e(self, steps=20):
        """The same metric through the host-buffer entry point (pinned host
        memory, both copies inside the timed region)."""
        import torch
        from paper_2510_19689_b300 import tabnet
        d = self.model.dims
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        xn_p, xc_p = pin(self.x_num), pin(self.x_cat)
        lg_p = torch.empty((self.rows, d.n_classes)).pin_memory().numpy()
        mk_p = torch.empty((self.rows, d.n_steps, d.d_emb)).pin_memory().numpy()
        ag_p = torch.empty((self.rows, d.n_feat)).pin_memory().numpy()
        args = [tabnet._ptr(xn_p), tabnet._ptr(xc_p), self.rows, tabnet._ptr(lg_p), tabnet._ptr(mk_p),
                tabnet._ptr(ag_p), self.stream.cuda_stream]
        L = tabnet.lib()
        for _ in range(3):
            tabnet._check(L.tabnet_forward_host(self.model._h, *args), "tabnet_forward_host")
        t0 = time.perf_counter()
        for _ in range(steps):
            tabnet._check(L.tabnet_forward_host(self.model._h, *args), "tabnet_forward_host")
        sec = (time.perf_counter() - t0) / steps
        inp_b, out_b = bytes_per_row(self.params)
        return {"value": self.rows / sec, "unit": UNIT, "h2d_bytes_per_step": self.rows * inp_b,
                "d2h_bytes_per_step": self.rows * out_b}

    def parity(self, n=256):
        """256 rows spread over the batch against the FP64 oracle (and, for the
        single-rounding modes, the error the rounding itself causes)."""
        import numpy as np
        import torch
        from oracle import tabnet_oracle as O
        self.step(0)
        torch.cuda.synchronize()
        status = self.model.poll_status()
        idx = np.linspace(0, self.rows - 1, n).astype(np.int64)
        rl, rm, ra = O.forward(self.params, self.x_num[idx], self.x_cat[idx])
        it = torch.from_numpy(idx).to(self.dev)
        s0 = self.sets[0]
        lg, mk, ag = s0["lg"][it].cpu().numpy(), s0["mk"][it].cpu().numpy(), s0["ag"][it].cpu().numpy()
        l1 = np.abs(mk - rm).sum((1, 2))
        return {"sample_rows": n, "logit_abs_max": float(np.abs(lg - rl).max()),
                "logit_rel_max": float((np.abs(lg - rl) / np.maximum(np.abs(rl), 1)).max()),
                "mask_l1_max": float(l1.max()), "mask_l1_mean": float(l1.mean()),
                "agg_l1_max": float(np.abs(ag - ra).sum(1).max()),
                "argmax_agreement": float((lg.argmax(1) == rl.argmax(1)).mean()), "status": status}

    def cpu_baseline(self, seconds=10.0):
        """The FP64 oracle as it stands on the host cores: a bounded sample of
        about `seconds` of CPU work (the batch's first rows, repeated when the
        batch takes less)."""
        from oracle import tabnet_oracle as O
        n_probe = {"c1": 256, "c2": 1024, "c3": 128}[self.name]
        rp, cores, _ = oracle_rows_per_s(self.params, self.x_num[:n_probe], self.x_cat[:n_probe])
        n_cpu = int(min(self.rows, max(n_probe, rp * seconds)))
        _, _, t_one = oracle_rows_per_s(self.params, self.x_num[:n_cpu], self.x_cat[:n_cpu])
        reps = max(1, int(round(seconds / t_one)))
        t0 = time.perf_counter()
        for _ in range(reps):
            O.forward(self.params, self.x_num[:n_cpu], self.x_cat[:n_cpu])
        dt = time.perf_counter() - t0
        return {"value": n_cpu * reps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"first {n_cpu} rows of the {self.name} batch x {reps} passes, float64 numpy ({dt:.1f} s)"}

    def close(self):
        self.model.close()
        self.sets = []


def roofline_for(params, rows, ms_step, precision, sustained, fp8_peak=None, traffic=None):
    """Algorithmic FLOP per launch over the event-timed launch duration,
    against the measured peak of the operands' type (bf16 for every bf16
    mode -- the split modes' extra products are not algorithmic work -- and
    the measured E4M3 GEMM rate for FP8)."""
    pk = peaks()
    flop = 2.0 * mac_per_row(params) * rows
    achieved = flop / (ms_step / 1e3) / 1e12
    if precision == "fp8" and fp8_peak:
        peak = fp8_peak * (pk["bf16_sus"] / pk["bf16"] if sustained else 1.0)
        kind = ("fp8 e4m3 GEMM measured in this run" + (" x the bf16 sustained/burst ratio" if sustained else "")
                + f" (bf16 peaks of {pk['src']})")
    else:
        peak = pk["bf16_sus"] if sustained else pk["bf16"]
        kind = ("bf16 sustained" if sustained else "bf16 burst") + f", of {pk['src']}"
    inp_b, out_b = bytes_per_row(params)
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": kind, "flop_per_launch": flop,
            "hbm_frac": rows * (inp_b + out_b) / (ms_step / 1e3) / 1e9 / pk["hbm"]}


def other_precisions(w, prec_list, steps, extras, it_rows=256):
    """The other precisions of the fused library on the same batch: rate and
    parity on the same sampled rows."""
    import torch
    from paper_2510_19689_b300 import tabnet
    for prec in prec_list:
        if prec == w.precision:
            continue
        try:
            w2 = Workload(w.name, prec, w.dev, data=(w.params, w.blob, w.x_num, w.x_cat))
        except tabnet.TabnetError as exc:
            extras[f"fused_{prec}"] = {"value": None, "unavailable": str(exc)[:200]}
            continue
        w2.tune()
        ms, stats, clocks = w2.time(steps if prec != "fp32" else 3, 2)
        n = steps if prec != "fp32" else 3
        extras[f"fused_{prec}"] = {"value": w2.rows * n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / n,
                                   "tile": w2.tile, "parity": w2.parity(it_rows)}
        w2.close()
        del w2
        torch.cuda.empty_cache()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_2510_19689_b300 import replicas

    # one process per GPU; rows are independent, so each rank runs its own
    # replica on its own batch (weak scaling, no collective in the step)
    group = replicas.Group("nccl")
    world, rank, local = group.world, group.rank, group.local
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    name = args.workload
    w = Workload(name, args.precision, dev)
    w.tune(not args.no_tune)
    parity = w.parity()

    ms_total, step_stats, clocks = w.time(args.steps, args.warmup, group)
    ms_step = ms_total / args.steps
    value = replicas.throughput(group.sum(w.rows * args.steps), ms_total)
    traffic = profiled_traffic(name, args.precision) if args.precision != "fp32" else None

    extras = {}
    fp8_peak = None
    if rank == 0 and not args.no_extras and (args.precision == "fp8" or name == "c2"):
        extras["fp8_gemm_peak"] = fp8_gemm_peak(dev)
        fp8_peak = extras["fp8_gemm_peak"].get("value")
    roofline = roofline_for(w.params, w.rows, ms_step, args.precision, False, fp8_peak, traffic)
    if rank == 0:
        extras["e2e"] = w.e2e()
        # the same step back to back for >= 1 s under the power cap
        sus = w.sustained(1.0)
        sus["roofline"] = roofline_for(w.params, w.rows, sus["ms_per_step"], args.precision, True, fp8_peak, traffic)
        extras["sustained"] = sus

    if rank == 0 and not args.no_extras:
        extras["cpu_baseline"] = w.cpu_baseline()
        # the same oracle held to one host thread (a child process whose BLAS
        # pools are limited by the environment before numpy loads), about 5 s
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        n_probe = {"c1": 256, "c2": 1024, "c3": 128}[name]
        code = ("import sys, time, json; sys.path.insert(0, %r); from paper_2510_19689_b300 import synth; "
                "from oracle import tabnet_oracle as O; p, _, xn, xc = synth.load_config(%r, rows=%d); "
                "t = time.perf_counter(); O.forward(p, xn[:%d], xc[:%d]); r = %d / (time.perf_counter() - t); "
                "n = int(min(len(xn), max(%d, r * 5.0))); "
                "t = time.perf_counter(); O.forward(p, xn[:n], xc[:n]); k = max(1, int(round(5.0 / (time.perf_counter() - t)))); "
                "t = time.perf_counter(); [O.forward(p, xn[:n], xc[:n]) for _ in range(k)]; "
                "dt = time.perf_counter() - t; print(json.dumps([n * k / dt, n, k, dt]))"
                ) % (ROOT, name, min(w.rows, 65536), n_probe, n_probe, n_probe, n_probe)
        try:
            out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
            r1, n1, k1, dt1 = json.loads(out.stdout.strip().splitlines()[-1])
            extras["cpu_baseline"]["one_core"] = {"value": r1, "sample": f"first {n1} rows x {k1} passes ({dt1:.1f} s)"}
        except Exception as exc:
            extras["cpu_baseline"]["one_core"] = {"value": None, "unavailable": str(exc)[:200]}
        # plain FP32 unfused GPU forward (PyTorch eager, TF32 off): the 5x target's divisor
        from paper_2510_19689_b300.unfused import UnfusedTabNet
        un = UnfusedTabNet(w.params, dev)
        s0 = w.sets[0]
        for _ in range(3):
            un.forward(s0["xn"], s0["xc"])
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(10):
            un.forward(s0["xn"], s0["xc"])
        a1.record()
        a1.synchronize()
        un_ms = a0.elapsed_time(a1) / 10
        extras["fp32_unfused"] = {"value": w.rows / (un_ms / 1e3), "unit": UNIT, "ms_per_step": un_ms}
        extras["speedup_vs_fp32_unfused"] = value / world / extras["fp32_unfused"]["value"]
        del un
        other_precisions(w, ("bf16", "bf16x6", "fp8", "fp32"), 20, extras)

    if rank == 0 and not args.no_extras and args.precision != "fp32":
        from paper_2510_19689_b300 import tabnet
        # audit statistics over the step's aggregate (mean, variance, top-5
        # frequency per feature): the aggregate read twice plus once per row
        ag0 = w.sets[0]["ag"]
        for _ in range(3):
            tabnet.mask_stats(ag0, 5, stream=w.stream)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(w.stream)
        for _ in range(20):
            tabnet.mask_stats(ag0, 5, stream=w.stream)
        a1.record(w.stream)
        a1.synchronize()
        ms_stats = a0.elapsed_time(a1) / 20
        extras["mask_stats"] = {"ms": ms_stats, "rows_per_s": w.rows / (ms_stats / 1e3), "k": 5,
                                "aggregate_bytes": w.rows * w.model.dims.n_feat * 4}

    if rank == 0 and not args.no_extras and name == "c2":
        # the paper's model shape (14 inputs, n_d = n_a = 8, 3 steps): the
        # latency of one 1,024-row call, and a fresh process's first call
        # (the serverless cold start)
        extras["c1_latency"] = bench_latency(dev)
        extras["cold_start"] = {}
        for mode in ("torch", "notorch"):
            try:
                out = subprocess.run([sys.executable, "-m", "paper_2510_19689_b300.cold_start", "c1", "1000",
                                      "bf16x3", mode], cwd=ROOT, capture_output=True, text=True, timeout=600)
                extras["cold_start"][mode] = json.loads(out.stdout.strip().splitlines()[-1])
            except Exception as exc:
                extras["cold_start"][mode] = {"unavailable": str(exc)[:200]}

    if rank == 0 and not args.no_extras and args.precision != "fp32" and name == "c2":
        extras["batching"] = bench_batching(w.model, w.params, dev, w.stream)
        extras["serving"] = bench_serving(local)
        # the largest configuration (1,048,576 rows of the 100-input model) in
        # the same run: split-bf16 and FP8, each with its own roofline, clocks,
        # end-to-end rate and parity sample, and the oracle's host rate
        w.close()
        torch.cuda.empty_cache()
        extras["c3"] = bench_large("c3", dev, fp8_peak, args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "ms_per_step_stats": step_stats,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "fp8": "e4m3"}.get(args.precision, "bf16"),
            "data": "synthetic",
            "config": workload_config(name, args.precision, world),
            "launch_shape": w.tile,
            "gpu_launches": args.steps,
            "clocks": clocks,
            "roofline": roofline,
            "parity": parity,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if w.sets:
        w.close()
    group.close()


def bench_large(name, dev, fp8_peak, args):
    """Both fast tensor-core modes on one large workload (one input set per
    mode beside the first's data)."""
    import torch
    from paper_2510_19689_b300 import synth
    data = synth.load_config(name)
    out = {"config": workload_config(name, "bf16x3 | fp8", 1), "arms": {}}
    for prec in ("bf16x3", "fp8"):
        w = Workload(name, prec, dev, data=data)
        w.tune()
        par = w.parity()
        steps = 10
        ms, stats, clocks = w.time(steps, 3)
        ms_step = ms / steps
        arm = {"value": w.rows * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "ms_per_step": ms_step,
               "ms_per_step_stats": stats, "tile": w.tile, "clocks": clocks,
               "roofline": roofline_for(w.params, w.rows, ms_step, prec, False, fp8_peak,
                                        profiled_traffic(name, prec)),
               "parity": par, "e2e": w.e2e(steps=5)}
        if prec == "bf16x3" and not args.no_extras:
            out["cpu_baseline"] = w.cpu_baseline()
        out["arms"][prec] = arm
        w.close()
        del w
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
