"""Throughput of the VQ-NNF hot path on one GB300 (or N replicas, one per GPU).

One step = the whole hot path on one synthetic template-query pair of the headline
workload: k-means codebook of the template (10 Lloyd steps), template NNF, template filter
responses, query NNF, query integral image + filter responses + Eq. 2 heatmap + argmax.
Metric: query Mpixel/s (query pixels / step time); the template side is inside the step.

Default workload: 2048 x 2048 query, D = 512, k = 128, 128 x 128 template (rotated, scaled,
occluded, noisy resample of the query), F = 10 (full window + 3 x 3 sub-windows).
Inputs are generated on the device from fixed seeds and stay resident (8 GiB of features,
larger than L2, so no flush is needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16|fp32|fp8] [--impl reference]
                  [--query-size S] [--no-compare] [--no-e2e] [--no-cpu-baseline] [--cpu-budget SEC]
                  [--no-paper-bank] [--no-soft] [--soft-batch B] [--no-batch] [--batch-eager] [--no-small]
                  [--shard replicas|bands]

With N > 1 ranks (torchrun), ``--shard replicas`` (default) gives every rank its own query
(weak scaling); ``--shard bands`` splits the one query's window rows into N row bands, each rank
scoring its band from its label rows plus a th - 1 row halo, the argmax combined by one MAX
all-reduce (strong scaling; main leg only).

``--query-size`` shrinks the query to S x S (for profiler captures of the same kernels on a
smaller case); the bench line itself is quoted on the default 2048.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on bounded
samples of the same workload instead.
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

HEADLINE = dict(H=2048, W=2048, D=512, k=128, th=128, tw=128, grid=3, iters=10, M=128,
                n_sp=20000, q_seed=1001, t_seed=2001, fit_seed=3001)
METRIC = "query Mpix/s at 2048^2, D=512, k=128: BF16 vs FP32 path, % of roofline"
OP_ASSIGN, OP_SCORE = 1, 3

# DRAM traffic of one launch of the BF16 contraction kernel (dram__bytes_read.sum +
# dram__bytes_write.sum), from the ncu capture summarised in
# profiles/assign_tc_kernel_query1024.md (1024 x 1024 query: 2,147,861,248 + 4,904,960 bytes),
# scaled by the pixel count (traffic is proportional to it).  Valid only for the kernel source
# it was taken on: the SHA-256 of assign_tc.cu below; any other source reports null.
TC_TRAFFIC_PER_PX = (2147861248 + 4904960) / (1024 * 1024)
TC_TRAFFIC_SRC_SHA256 = "191d4f541bad2ed706a4d3b51baf91a22bee137e456ad990249fa00d01510926"



def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons (every 50 ms, timestamped) from before the
    warm-up to after the timed region; ``summary(t0, t1)`` keeps the samples taken inside the
    timed region [t0, t1] (host wall clock)."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _when(stamp):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(stamp, fmt).timestamp()
            except ValueError:
                pass
        return None

    def summary(self, t0=None, t1=None):
        if self.proc is None or self.tmp is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        inside = rows
        window = "whole run"
        if t0 is not None:
            sel = [r for r in rows if (w := self._when(r[0])) is not None and t0 - 0.05 <= w <= t1 + 0.05]
            if sel:
                inside, window = sel, "timed region"
        sm = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in inside if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(inside), "window": window}


def reduce_max_ms(ms: float, device="cpu") -> float:
    """The job's step time: the maximum of the ranks' step times (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ms: float, world: int, query_px: int) -> float:
    """Whole-job throughput in Mpix/s: every rank processes one query per step (weak scaling)."""
    return world * query_px / (ms * 1e-3) / 1e6


def make_workload(dev, cfg):
    import synth
    q = synth.query_map(cfg["H"], cfg["W"], cfg["D"], M=cfg["M"], n_sp=cfg["n_sp"],
                        seed=cfg["q_seed"], device=dev)
    T, info = synth.warped_template(q, cfg["th"], cfg["tw"], seed=cfg["t_seed"])
    bank = synth.grid_bank(cfg["th"], cfg["tw"], cfg["grid"])
    return q, T, info, bank


class Pipeline:
    """The hot path with every buffer allocated once (so a step can be graph-captured)."""

    def __init__(self, vq, X, T, cfg, bank, prec, stream):
        import torch
        self.vq, self.X, self.T, self.cfg, self.prec, self.s = vq, X, T, cfg, prec, stream
        self.bank = vq.Bank(bank)
        H, W, D, k = cfg["H"], cfg["W"], cfg["D"], cfg["k"]
        th, tw = cfg["th"], cfg["tw"]
        dev = X.device
        self.ws_fit = vq.Workspace(vq.vqnnf_workspace_bytes(0, th, tw, D, k, prec=prec), dev)
        self.ws_a = vq.Workspace(vq.vqnnf_workspace_bytes(1, H, W, D, k, prec=prec), dev)
        self.ws_t = vq.Workspace(vq.vqnnf_workspace_bytes(1, th, tw, D, k, prec=prec), dev)
        # the template's NNF and responses run on a second stream beside the query's NNF (both
        # need only the codebook; the score needs both)
        self.s2 = torch.cuda.Stream(device=dev)
        self.ev_fit = torch.cuda.Event()
        self.ev_tpl = torch.cuda.Event()
        self.ws_s = vq.Workspace(vq.vqnnf_workspace_bytes(3, H, W, 0, k, th, tw, self.bank.F), dev)
        self.C = torch.empty((k, D), device=dev)
        self.tl = torch.empty((th, tw), dtype=torch.uint8, device=dev)
        self.ql = torch.empty((H, W), dtype=torch.uint8, device=dev)
        self.tc = torch.empty((self.bank.F, k), dtype=torch.int32, device=dev)
        self.heat = torch.empty((H - th + 1, W - tw + 1), device=dev)
        self.am = torch.empty(2, dtype=torch.int32, device=dev)
        self.stats = torch.zeros(4, dtype=torch.int64, device=dev)

    def step(self, ev=None, kev=None):
        """One pass of the hot path.  ev: 4 events marking the segment boundaries (the template
        segment is the codebook fit; the template's NNF and responses overlap the query's NNF
        on the second stream); kev: 4 events recorded by the library immediately around the
        query's contraction kernel and the score kernel (vqnnf_set_kernel_events)."""
        vq, c, s = self.vq, self.cfg, self.s
        if ev is not None:
            ev[0].record(s)
        vq.vqnnf_fit_codebook(self.T, c["k"], c["iters"], c["fit_seed"], self.prec, C=self.C,
                              ws=self.ws_fit, stream=s)
        self.ev_fit.record(s)
        self.s2.wait_event(self.ev_fit)
        vq.vqnnf_assign(self.T, self.C, self.prec, labels=self.tl, ws=self.ws_t, stream=self.s2)
        vq.vqnnf_filter_responses(self.tl, c["k"], self.bank, counts=self.tc, stream=self.s2)
        self.ev_tpl.record(self.s2)
        if ev is not None:
            ev[1].record(s)
        if kev is not None:
            vq.vqnnf_set_kernel_events(OP_ASSIGN, kev[0], kev[1])
        vq.vqnnf_assign(self.X, self.C, self.prec, labels=self.ql, stats=self.stats,
                        ws=self.ws_a, stream=s)
        if kev is not None:
            vq.vqnnf_set_kernel_events(OP_ASSIGN, None, None)
        if ev is not None:
            ev[2].record(s)
        s.wait_event(self.ev_tpl)
        if kev is not None:
            vq.vqnnf_set_kernel_events(OP_SCORE, kev[2], kev[3])
        vq.vqnnf_score(self.ql, c["k"], c["th"], c["tw"], self.bank, self.tc, heatmap=self.heat,
                       argmax_yx=self.am, ws=self.ws_s, stream=s)
        if kev is not None:
            vq.vqnnf_set_kernel_events(OP_SCORE, None, None)
        if ev is not None:
            ev[3].record(s)


def kernels_per_step(cfg, prec):
    """Kernels of this library launched by one step (counted from the launch sequence)."""
    k = cfg["k"]
    assign = 2 + 1 + 1 + 1          # prep mean + prep centroids, contraction, rescore, stats
    # gather; per Lloyd step: prep centroids, contraction, rescore, two sort kernels, update; the
    # first step also forms the reference point (prep mean), which the later steps keep
    fit = 1 + cfg["iters"] * (3 + 3) + (1 if cfg["iters"] > 0 else 0)
    tpl = (assign - 1) + 1          # template NNF, template responses
    score = 4 + 1 + 1               # row carries, band sums, band prefix, write pass; score; argmax
    return fit + tpl + assign + score


def run_gpu(args, rank, world):
    import numpy as np
    import torch
    import paper_2306_15010_gb300 as vq
    from paper_2306_15010_gb300 import build as _b

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if local == 0:
        _b.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    cfg = dict(HEADLINE)
    if args.query_size != cfg["H"]:
        cfg["n_sp"] = max(64, cfg["n_sp"] * args.query_size ** 2 // cfg["H"] ** 2)
        cfg["H"] = cfg["W"] = args.query_size
    q, T, info, bank = make_workload(dev, cfg)
    X = q.X
    L = cfg["H"] * cfg["W"]
    band = None
    if args.shard == "bands":
        # row-band sharding of the one query: rank r scores the window rows of band r, reading
        # its label rows plus the th - 1 row halo; the template side is recomputed from the same
        # seed on every rank (identical codebook); the argmax is one MAX all-reduce afterwards
        from paper_2306_15010_gb300 import bands as _bands
        band = _bands.band_rows(cfg["H"] - cfg["th"] + 1, world)[rank]
        if band[1] == band[0]:
            raise SystemExit("more ranks than window rows")
        cfg = dict(cfg, H=band[1] - band[0] + cfg["th"] - 1)
        X = X[band[0]:band[1] + cfg["th"] - 1]
    s = torch.cuda.Stream(device=dev)
    pipe = Pipeline(vq, X, T, cfg, bank, args.prec, s)
    clk = Clocks(local).__enter__()
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            pipe.step()
    torch.cuda.synchronize()
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    kevs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    for kv in kevs:                      # create the CUDA events the library records into
        for e in kv:
            e.record(s)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    # the timed step: one replay of a CUDA graph that holds the whole hot path (every kernel
    # of the step, enqueued once at capture)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            pipe.step()
        for _ in range(2):
            graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t_on = time.time()
    start.record(s)
    with torch.cuda.stream(s):
        for i in range(K):
            graph.replay()
    stop.record(s)
    torch.cuda.synchronize()
    t_off = time.time()
    time.sleep(0.1)
    clk.__exit__()
    ms = start.elapsed_time(stop) / K
    # diagnostics, outside the timed region: the same K steps enqueued call by call, with
    # events at the segment boundaries and around the two main kernels
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    d0.record(s)
    with torch.cuda.stream(s):
        for i in range(K):
            pipe.step(evs[i], kevs[i])
    d1.record(s)
    torch.cuda.synchronize()
    ms_calls = d0.elapsed_time(d1) / K
    if world > 1:
        import torch.distributed as dist
        ms = reduce_max_ms(ms, dev)
        dist.barrier()
    seg = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])]
                    for e in evs]).mean(0)
    kern = np.array([[kv[0].elapsed_time(kv[1]), kv[2].elapsed_time(kv[3])] for kv in kevs]).mean(0)
    stats = pipe.stats.cpu().tolist()
    am = pipe.am.cpu().tolist()
    if band is not None:
        by, bx = am
        hv = float(pipe.heat[by, bx].item())
        WO = cfg["W"] - cfg["tw"] + 1
        am = list(_bands.allreduce_argmax(hv, by + band[0], bx, WO, device=dev) if world > 1
                  else (by + band[0], bx))
    clocks = clk.summary(t_on, t_off)

    # the other precisions on the same inputs, same GPU: the BF16-vs-FP32 comparison and the
    # FP8 e4m3 contraction (every path returns exact labels; the report says what each costs)
    others = {}
    if not args.no_compare:
        for other in [p for p in ("fp32", "bf16", "fp8") if p != args.prec]:
            pipe2 = Pipeline(vq, X, T, cfg, bank, other, s)
            with torch.cuda.stream(s):
                for _ in range(args.warmup):
                    pipe2.step()
            torch.cuda.synchronize()
            graph2 = torch.cuda.CUDAGraph()
            with torch.cuda.stream(s):
                with torch.cuda.graph(graph2, stream=s):
                    pipe2.step()
                graph2.replay()
            torch.cuda.synchronize()
            st2 = torch.cuda.Event(enable_timing=True)
            sp2 = torch.cuda.Event(enable_timing=True)
            st2.record(s)
            with torch.cuda.stream(s):
                for i in range(K):
                    graph2.replay()
            sp2.record(s)
            torch.cuda.synchronize()
            ms2 = st2.elapsed_time(sp2) / K
            # one call-by-call step with events around its segments and its contraction
            ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            kev2 = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            for e in kev2:
                e.record(s)
            with torch.cuda.stream(s):
                pipe2.step(ev2, kev2)
            torch.cuda.synchronize()
            st = pipe2.stats.cpu().tolist()
            ndiff = int((pipe.ql != pipe2.ql).sum().item())
            hd = float((pipe.heat - pipe2.heat).abs().max().item()) / max(float(pipe.heat.abs().max().item()), 1e-30)
            others[other] = {
                "value": round(world * cfg["H"] * cfg["W"] / (ms2 * 1e-3) / 1e6, 3), "unit": "Mpix/s",
                "ms_per_step": round(ms2, 4),
                "segments_ms": {"template_side": round(ev2[0].elapsed_time(ev2[1]), 4),
                                "query_assign": round(ev2[1].elapsed_time(ev2[2]), 4),
                                "query_score": round(ev2[2].elapsed_time(ev2[3]), 4)},
                "query_contraction_ms": round(kev2[0].elapsed_time(kev2[1]), 4),
                "assign_stats": {"n_flagged": st[0], "n_candidates": st[1], "n_deep": st[2],
                                 "flagged_pct": round(100.0 * st[0] / (cfg["H"] * cfg["W"]), 3)},
                "labels_identical": ndiff == 0, "query_labels_differing": ndiff,
                "heat_max_rel_diff_vs_main": hd,
            }
            del graph2
            others[other]["_pipe"] = pipe2
            del pipe2
    # end to end through the same API: pinned host inputs in, argmax + heatmap out, per step
    e2e = None if args.no_e2e else run_e2e(vq, pipe, X, T, cfg, args, s, dev, am_ref=am)
    paper = None if args.no_paper_bank else run_paper_bank(vq, pipe, cfg, s, dev)
    soft_vq = None if args.no_soft else run_soft(vq, dev, B=args.soft_batch)
    batch = None if args.no_batch else run_batch(vq, dev, eager=args.batch_eager)

    if rank != 0:
        return None
    value = job_value(ms, world, L) if band is None else L / (ms * 1e-3) / 1e6
    peaks, peak_src = _peaks()
    roof = roofline(cfg, args.prec, kern[0], peaks, peak_src)
    roof_score = roofline_score(cfg, kern[1], peaks, tcounts=pipe.tc)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mpix/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "execution": {"timed": "CUDA graph replay of one whole step per iteration",
                      "ms_per_step_call_by_call": round(ms_calls, 4)},
        "higher_is_better": True, "scaling": "weak" if band is None else "strong", "vs_baseline": None,
        "dtype": {"bf16": "bf16", "fp8": "fp8e4m3", "fp32": "f32"}[args.prec], "data": "synthetic",
        "config": {"workload": f"{cfg['H']}x{cfg['W']} query, D=512, k=128, 128x128 template, F=10 "
                               "(full + 3x3), 10 Lloyd steps; whole hot path per step",
                   "prec": args.prec, "query_px": L, "l2": "inputs larger than L2 (8 GiB features)",
                   "parallelism": f"replicas x{world}" if band is None else
                   f"row bands x{world} (rank 0: window rows {band[0]}..{band[1] - 1} + {cfg['th'] - 1}-row halo)"},
        "segments_ms": {"template_side": round(seg[0], 4), "query_assign": round(seg[1], 4),
                        "query_score": round(seg[2], 4)},
        "kernels_ms": {"query_contraction": round(float(kern[0]), 4), "score": round(float(kern[1]), 4)},
        "query_only": {"value": round((world * L if band is None else L) / ((seg[1] + seg[2]) * 1e-3) / 1e6, 3),
                       "unit": "Mpix/s",
                       "note": "query assign + integral image + score per query, template side amortised"},
        "assign_stats": {"n_flagged": stats[0], "n_candidates": stats[1], "n_deep": stats[2]},
        "argmax_yx": am, "planted_top_left": list(info["top_left"]),
        "roofline": roof, "roofline_score": roof_score, "clocks": clocks, "e2e": e2e,
        "paper_bank": paper, "soft_vq": soft_vq, "batch": batch,
        **{f"{o}_path": {kk: vv for kk, vv in d.items() if kk != "_pipe"}
           for o, d in others.items()},
        "gpu_launches": kernels_per_step(cfg, args.prec) * K,
    }
    if "fp32" in others and args.prec == "bf16":
        line["fp32_path"]["speedup_bf16_over_fp32"] = round(others["fp32"]["ms_per_step"] / ms, 3)
    if "fp8" in others:
        line["fp8_path"]["speedup_fp8_over_main"] = round(ms / others["fp8"]["ms_per_step"], 3)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(q, T, cfg, bank, budget_s=args.cpu_budget, pipe=pipe, one_thread=True,
                                            other_pipes={o: d["_pipe"] for o, d in others.items()})
    for d in others.values():
        d.pop("_pipe", None)
    others.clear()
    if not args.no_small:
        # last, after every other leg: a failure here leaves an error entry, not a missing line
        try:
            line["small_workload"] = run_small(vq, dev)
        except Exception as exc:                          # noqa: BLE001
            line["small_workload"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    return line


def _tc_traffic(L):
    import hashlib
    src = os.path.join(ROOT, "paper_2306_15010_gb300", "csrc", "assign_tc.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    return round(TC_TRAFFIC_PER_PX * L) if sha == TC_TRAFFIC_SRC_SHA256 else None


def roofline(cfg, prec, kernel_ms, peaks, src):
    """The dominant kernel, the query's distance contraction, timed alone (library events)."""
    L, D, k = cfg["H"] * cfg["W"], cfg["D"], cfg["k"]
    if prec == "bf16":
        # HBM-bound: the contraction must read every FP32 feature once and write a label
        bytes_ = L * (D * 4 + 1)
        ach = bytes_ / (kernel_ms * 1e-3) / 1e9
        peak = float(peaks["hbm_gbs"])
        return {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": _tc_traffic(L),
                "kernel": "assign_tc_kernel (tcgen05 BF16 contraction + interval test), query launch",
                "kernel_ms": round(float(kernel_ms), 4),
                "algorithmic_bytes_per_px": D * 4 + 1, "peak_source": src + " (burst copy)"}
    if prec == "fp8":
        # HBM-bound: the e4m3 features (D bytes), the row's scale and norm (8) and the label (1)
        bytes_ = L * (D + 8 + 1)
        ach = bytes_ / (kernel_ms * 1e-3) / 1e9
        peak = float(peaks["hbm_gbs"])
        return {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": None,
                "kernel": "assign_fp8_kernel (tcgen05 e4m3 contraction + interval test), query launch",
                "kernel_ms": round(float(kernel_ms), 4),
                "algorithmic_bytes_per_px": D + 9, "peak_source": src + " (burst copy)"}
    # FP32 SIMT: bound by the FP32 FMA pipes, 152 SMs x 128 lanes x 2 flop x max SM clock
    flops = 2.0 * L * D * k
    ach = flops / (kernel_ms * 1e-3) / 1e12
    peak = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    return {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 2), "unit": "TFLOP/s",
            "frac": round(ach / peak, 4), "traffic": None,
            "kernel": "assign_fp32_kernel (FP32 SIMT contraction), query launch",
            "kernel_ms": round(float(kernel_ms), 4),
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}


def roofline_score(cfg, kernel_ms, peaks, tcounts=None):
    """Score kernel: integer ALU work of Eq. 2 over the integral image, against an issue-rate
    bound.  The kernel uses L1_f = area_f + sum over clusters with t_fj > 0 of (|t_fj - n_fj| -
    n_fj), so only the (filter, cluster) pairs present in the template cost work: per pair 3
    adds for the box sum and 3 for the filter term, plus, per cluster, the distinct integral-
    image corners of its present boxes.  That count (from the template's counts `tcounts`, F x
    k in bank order) is the algorithmic work; the dense form of Eq. 2 (every filter and cluster:
    (g+1)^2 corner loads, 3 g^2 + 3 box adds, 3 per filter) is reported beside it."""
    import synth
    k, th, tw, g = cfg["k"], cfg["th"], cfg["tw"], cfg["grid"]
    F = g * g + 1
    V = (cfg["H"] - th + 1) * (cfg["W"] - tw + 1)
    peak = 152 * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    dense_per = (g + 1) ** 2 + 3 * g * g + 3 + 3 * F
    dense = float(V) * k * dense_per / (kernel_ms * 1e-3) / 1e12
    sparse_per = None
    if tcounts is not None:
        bank = synth.grid_bank(th, tw, g)
        corners = [{(x, y) for (x0, y0, x1, y1, _) in f["rects"] for x in (x0, x1) for y in (y0, y1)}
                   for f in bank]
        tcn = tcounts.cpu().numpy()
        tot = 0
        for j in range(k):
            pres = [f for f in range(F) if tcn[f, j] > 0]
            if pres:
                tot += len(set().union(*(corners[f] for f in pres))) + 6 * len(pres)
        sparse_per = tot / k
    ops_per = sparse_per if sparse_per is not None else dense_per
    ach = float(V) * k * ops_per / (kernel_ms * 1e-3) / 1e12
    # the same launch against HBM: the 16-bit integral image read once, the heatmap written
    tbytes = (cfg["H"] + 1) * (cfg["W"] + 1) * k * 2 + V * 4
    hbm = tbytes / (kernel_ms * 1e-3) / 1e9
    out = {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 2), "unit": "Tops/s",
           "frac": round(ach / peak, 4), "traffic": None, "kernel": "score_grid_kernel",
           "kernel_ms": round(float(kernel_ms), 4),
           "algorithmic_ops_per_window_cluster": round(ops_per, 2),
           "ops_counted": "only the (filter, cluster) pairs with a nonzero template count (the kernel's "
                          "formulation): 3 box adds + 3 for |t - n| - n per pair, plus the distinct corner "
                          "loads of the cluster's present boxes" if sparse_per is not None else
                          "dense Eq. 2: every filter and cluster",
           "peak_source": "derived issue-rate bound: 152 SMs x 128 lanes x max SM clock, one operation "
                          "(integer add or compare, or a shared-memory corner load) per lane and cycle",
           "dense_equivalent": {"ops_per_window_cluster": dense_per, "achieved": round(dense, 2),
                                "frac": round(dense / peak, 4)},
           "hbm": {"achieved": round(hbm, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                   "frac": round(hbm / peaks["hbm_gbs"], 4), "bytes_per_launch": tbytes,
                   "note": "16-bit integral image read once + heatmap written"}}
    return out


def run_paper_bank(vq, pipe, cfg, s, dev, reps=5):
    """The paper's own filter bank (F_{2,3-rect}: Gaussian + Haar 2x/2y/3x/3y, S = 3 sub-scales,
    15 multi-rectangle filters, equal-weight reading) scored on this step's query NNF; the
    score kernel (generic bank path) timed alone with library-recorded events."""
    import torch
    import synth
    th, tw, k, H, W = cfg["th"], cfg["tw"], cfg["k"], cfg["H"], cfg["W"]
    bank = vq.Bank(synth.paper_bank(th, tw, "2,3-rect", 3, "equal"))
    ws = vq.Workspace(vq.vqnnf_workspace_bytes(3, H, W, 0, k, th, tw, bank.F), dev)
    heat = torch.empty_like(pipe.heat)
    am = torch.empty(2, dtype=torch.int32, device=dev)
    with torch.cuda.stream(s):
        tc = vq.vqnnf_filter_responses(pipe.tl, k, bank, stream=s)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(reps + 1)]
    for e in ev:
        for x in e:
            x.record(s)
    torch.cuda.synchronize()
    for i in range(reps + 1):
        ev[i][0].record(s)
        vq.vqnnf_set_kernel_events(OP_SCORE, ev[i][1], ev[i][2])
        vq.vqnnf_score(pipe.ql, k, th, tw, bank, tc, heatmap=heat, argmax_yx=am, ws=ws, stream=s)
        vq.vqnnf_set_kernel_events(OP_SCORE, None, None)
        ev[i][3].record(s)
    torch.cuda.synchronize()
    call = sorted(e[0].elapsed_time(e[3]) for e in ev[1:])[reps // 2]
    kern = sorted(e[1].elapsed_time(e[2]) for e in ev[1:])[reps // 2]
    return {"bank": "F_{2,3-rect}, S=3 (15 filters, 33 rectangles), equal-weight Gaussian reading",
            "score_call_ms": round(call, 4), "score_kernel_ms": round(kern, 4),
            "argmax_yx": am.cpu().tolist(), "kernel": "score_wgrid_kernel (weighted 3 x 3 grids, one per sub-scale)"}


def run_soft(vq, dev, reps=3, B=8):
    """The training path: soft-VQ heatmap of 8 queries 512 x 512, D = 256, k = 64, 3 x 3 cell
    filters (learnable weights, 1 at start), tau = 0.1; forward and backward (gradients for the
    query features, the centroids and the weights of L = sum heat * N(0,1) weights)."""
    import torch
    import synth
    H, W, D, k, th, tw, G, tau = 512, 512, 256, 64, 64, 64, 3, 0.1
    Q = torch.stack([synth.query_map(H, W, D, M=64, n_sp=1250, seed=4000 + i, device=dev).X for i in range(B)])
    T, _ = synth.crop_template(synth.query_map(H, W, D, M=64, n_sp=1250, seed=4000, device=dev), th, tw, seed=4100)
    T = T.to(dev).contiguous()
    g = torch.Generator(device="cpu").manual_seed(4200)
    C = (torch.rand((k, D), generator=g) * 0.8 + 0.1).to(dev)
    Gw = torch.randn((B, H - th + 1, W - tw + 1), generator=g).to(dev)
    Q.requires_grad_(True)
    C.requires_grad_(True)
    wf = torch.ones(G * G, device=dev, requires_grad=True)
    fw, bw = [], []
    for r in range(reps + 1):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        heat = vq.soft_heatmap(Q, T, C, wf, tau, G)
        e[1].record()
        (heat * Gw).sum().backward()
        e[2].record()
        torch.cuda.synchronize()
        if r:
            fw.append(e[0].elapsed_time(e[1]))
            bw.append(e[1].elapsed_time(e[2]))
        Q.grad = C.grad = wf.grad = None
    f_ms, b_ms = sorted(fw)[reps // 2], sorted(bw)[reps // 2]
    return {"workload": f"{B} queries 512x512, D=256, k=64, 64x64 template, 3x3 cells (F=9), tau=0.1",
            "forward_ms": round(f_ms, 3), "backward_ms": round(b_ms, 3),
            "train_step_mpix_s": round(B * H * W / ((f_ms + b_ms) * 1e-3) / 1e6, 2),
            "note": "backward includes the autograd engine's elementwise product and sum of the loss"}


def run_batch(vq, dev, reps=2, eager=False):
    """Batching: 64 templates (sides ~U{16..192} per axis, k ~U{8, 16, 32, 64, 128, 256}, warped
    crops as in the headline workload) against 16 queries (sides ~U{512..2048} per axis), D = 256,
    FP32 features, BF16 contraction; one vqnnf_match_batch call (every template's codebook,
    NNF and responses, every query's NNFs, every pair's heatmap and maximum) captured in a
    CUDA graph, tile plan from vqnnf_batch_tune."""
    import numpy as np
    import torch
    import synth
    r = np.random.default_rng(6000)
    nq, nt, D, G, iters = 16, 64, 256, 3, 10
    qsz = r.integers(512, 2049, (nq, 2))
    tsz = r.integers(16, 193, (nt, 2))
    ks = [int(v) for v in r.choice([8, 16, 32, 64, 128, 256], nt)]
    Xs = []
    for i, (H, W) in enumerate(qsz):
        q = synth.query_map(int(H), int(W), D, M=128, n_sp=max(64, 20000 * int(H) * int(W) // 2048 ** 2),
                            seed=6100 + i, device=dev)
        Xs.append(q)
    Ts = [synth.warped_template(Xs[j % nq], int(h), int(w), seed=6300 + j)[0] for j, (h, w) in enumerate(tsz)]
    Xs = [q.X for q in Xs]
    plan = vq.vqnnf_batch_tune(Xs, Ts, ks, iters, 6500, G)
    heats = [torch.empty((X.shape[0] - T.shape[0] + 1, X.shape[1] - T.shape[1] + 1), device=dev)
             for X in Xs for T in Ts]
    am = torch.empty((nq, nt, 2), dtype=torch.int32, device=dev)
    ws = vq.Workspace(vq.vqnnf_batch_workspace_bytes(Xs, Ts, ks, G), dev)
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        vq.vqnnf_match_batch(Xs, Ts, ks, iters, 6500, G, plan, heat=heats, argmax_yx=am, ws=ws, stream=s)
    torch.cuda.synchronize()
    g = None
    if not eager:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                vq.vqnnf_match_batch(Xs, Ts, ks, iters, 6500, G, plan, heat=heats, argmax_yx=am, ws=ws, stream=s)
            g.replay()
        torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    with torch.cuda.stream(s):
        for _ in range(reps):
            if g is not None:
                g.replay()
            else:
                vq.vqnnf_match_batch(Xs, Ts, ks, iters, 6500, G, plan, heat=heats, argmax_yx=am, ws=ws, stream=s)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    px = sum(int(X.shape[0]) * int(X.shape[1]) for X in Xs)
    cols = sum((k + 31) // 32 * 32 for k in ks)
    out = {"workload": f"{nq} queries ~U{{512..2048}}^2, {nt} templates ~U{{16..192}}^2, "
                       f"k ~U{{8..256}}, D={D}, grid bank G={G}, {iters} Lloyd steps; all pairs",
           "ms_per_batch": round(ms, 2), "pairs_per_s": round(nq * nt / (ms * 1e-3), 1),
           "query_mpix_per_s": round(px / (ms * 1e-3) / 1e6, 2),
           "pair_mpix_per_s": round(px * nt / (ms * 1e-3) / 1e6, 1),
           "plan": {"stationary": plan.stationary, "group_cols": plan.group_cols, "sf": plan.sf, "pf": plan.pf},
           "codebook_columns": cols, "query_px": px,
           "execution": "one vqnnf_match_batch call per batch, " +
                        ("enqueued directly" if eager else "CUDA graph replay")}
    del g, heats, ws
    torch.cuda.empty_cache()
    return out


SMALL = dict(H=256, W=256, D=64, k=16, th=32, tw=32, grid=3, iters=10, M=32, n_sp=200,
             q_seed=1000, t_seed=2000, fit_seed=3000)


def run_small(vq, dev, reps=50):
    """The small plain workload: a 256 x 256 query, D = 64, k = 16, a 32 x 32 crop template,
    F = 10 and 10 Lloyd steps. It is latency-bound, so it is reported per call, in both
    precisions: the whole path as one CUDA-graph replay, and the same calls enqueued one by one
    from Python. The difference is the launch and host overhead that the graph removes."""
    import torch
    import synth
    cfg = dict(SMALL)
    q = synth.query_map(cfg["H"], cfg["W"], cfg["D"], M=cfg["M"], n_sp=cfg["n_sp"], seed=cfg["q_seed"],
                        device=dev)
    T, _ = synth.crop_template(q, cfg["th"], cfg["tw"], seed=cfg["t_seed"])
    bank = synth.grid_bank(cfg["th"], cfg["tw"], cfg["grid"])
    s = torch.cuda.Stream(device=dev)
    L = cfg["H"] * cfg["W"]
    out = {"workload": "256x256 query, D=64, k=16, 32x32 crop template, F=10 (full + 3x3), 10 Lloyd steps; "
                       "whole hot path per call", "launches_per_call": kernels_per_step(cfg, "fp32")}
    for prec in ("fp32", "bf16"):
        pipe = Pipeline(vq, q.X, T, cfg, bank, prec, s)
        with torch.cuda.stream(s):
            for _ in range(3):
                pipe.step()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                pipe.step()
            g.replay()
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(s)
        with torch.cuda.stream(s):
            for _ in range(reps):
                g.replay()
        e[1].record(s)
        with torch.cuda.stream(s):
            for _ in range(reps):
                pipe.step()
        e[2].record(s)
        torch.cuda.synchronize()
        t_graph = e[0].elapsed_time(e[1]) / reps
        t_calls = e[1].elapsed_time(e[2]) / reps
        out[prec] = {"us_per_call": round(1e3 * t_graph, 1), "value": round(L / (t_graph * 1e-3) / 1e6, 3),
                     "unit": "Mpix/s", "us_per_call_enqueued_one_by_one": round(1e3 * t_calls, 1),
                     "overhead_removed_by_graph_us": round(1e3 * (t_calls - t_graph), 1)}
        del g, pipe
    return out


def run_e2e(vq, pipe, X, T, cfg, args, s, dev, am_ref=None):
    """End to end through the C ABI with host buffers: vqnnf_match_host takes the pinned host
    feature maps and writes the host heatmap and maximum, every step.  The host link (~210 GB/s
    here) bounds it; inside the call the template goes first and its side runs on a second
    stream while the query arrives in row bands, each assigned as soon as it has landed."""
    import torch
    try:
        hX = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
        hT = torch.empty(T.shape, dtype=T.dtype, pin_memory=True)
        hX.copy_(X.cpu())
        hT.copy_(T.cpu())
        hheat = torch.empty(pipe.heat.shape, dtype=torch.float32, pin_memory=True)
        ham = torch.empty(2, dtype=torch.int32, pin_memory=True)
    except Exception as exc:  # pragma: no cover
        return {"value": None, "unit": "Mpix/s", "error": str(exc)}
    c = cfg
    H, W, D = X.shape
    ws = vq.Workspace(vq.vqnnf_match_host_workspace_bytes(H, W, D, c["k"], c["th"], c["tw"], pipe.bank.F,
                                                          pipe.prec), dev)
    s2 = torch.cuda.Stream(device=dev)

    def one_step():
        vq.vqnnf_match_host(hX, hT, c["k"], c["iters"], c["fit_seed"], pipe.bank, pipe.prec, heatmap=hheat,
                            argmax_yx=ham, ws=ws, stream=s, stream2=s2)

    one_step()                                # warm-up
    torch.cuda.synchronize()
    # the floor: the step's host-to-device bytes alone (the fastest of three copies)
    copy_ms = float("inf")
    for _ in range(3):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            c0.record(s)
            pipe.X.copy_(hX, non_blocking=True)
            pipe.T.copy_(hT, non_blocking=True)
            c1.record(s)
        torch.cuda.synchronize()
        copy_ms = min(copy_ms, c0.elapsed_time(c1))
    n = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(n):
        one_step()
    s.synchronize()
    dt = (time.perf_counter() - t0) / n
    L = H * W
    out = {"value": round(L / dt / 1e6, 3), "unit": "Mpix/s",
           "h2d_bytes_per_step": hX.numel() * 4 + hT.numel() * 4,
           "d2h_bytes_per_step": hheat.numel() * 4 + 8, "steps": n, "ms_per_step": round(dt * 1e3, 2),
           "h2d_copy_ms": round(copy_ms, 2),
           "call": "vqnnf_match_host (C ABI, pinned host buffers in and out, two streams)",
           "argmax_matches_device_run": None if am_ref is None else ham.tolist() == list(am_ref)}
    del ws
    return out


def cpu_baseline(q, T, cfg, bank, budget_s=20.0, steps=1, pipe=None, one_thread=False, other_pipes=None):
    """The FP64 oracle timed on bounded samples of the same workload, scaled to one step, on
    all of the oracle's threads (and, with ``one_thread``, again on one thread).  With ``pipe``
    (the timed BF16 pipeline), this run's own results are also checked against the oracle on
    the same samples."""
    import numpy as np
    import oracle
    oracle.build()
    Xh = q.X[: 8].cpu().numpy()                   # 8 query rows = 16384 pixels
    Th = T.cpu().numpy()
    k, D = cfg["k"], cfg["D"]
    L = cfg["H"] * cfg["W"]
    th, tw = cfg["th"], cfg["tw"]
    HO, WO = cfg["H"] - th + 1, cfg["W"] - tw + 1
    px_asg = Xh.shape[0] * Xh.shape[1]
    # score sample: windows of a synthetic label field of the same size (labels for the
    # whole query would need the full assignment)
    ql = (q.sp_id.cpu().numpy() * 7 % k).astype(np.int32)
    tl = ql[:th, :tw]
    tc = oracle.filter_counts(tl, k, bank)
    rng = np.random.default_rng(0)
    nwin = 1024
    win = np.stack([rng.integers(0, HO, nwin), rng.integers(0, WO, nwin)], 1)

    def phases():
        t0 = time.perf_counter()
        C = oracle.fit_codebook(Th, k, 1, cfg["fit_seed"])   # one Lloyd step
        t_fit1 = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.assign(Xh, C)
        t_asg = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.score_at(ql, k, bank, tc, win)
        t_sc = time.perf_counter() - t0
        t_step = (t_fit1 * cfg["iters"] + t_asg * (L + th * tw) / px_asg + t_sc * HO * WO / nwin)
        return t_step, {"fit_one_lloyd_step": round(t_fit1, 4), f"assign_{px_asg}_px": round(t_asg, 4),
                        f"score_{nwin}_windows": round(t_sc, 4)}

    threads = oracle.set_threads(0)                          # the count in effect, unchanged
    t_step, ph = phases()
    out = {"value": round(L / t_step / 1e6, 6), "unit": "Mpix/s",
           "cores": threads, "kind": "oracle",
           "sample": (f"1 Lloyd step (x{cfg['iters']}), {px_asg} query pixels assigned, "
                      f"{nwin} windows scored; scaled to one full step"),
           "step_s_estimate": round(t_step, 2), "phases_s": ph}
    if one_thread:
        prev = oracle.set_threads(1)
        try:
            t1, ph1 = phases()
        finally:
            oracle.set_threads(prev)
        out["one_thread"] = {"value": round(L / t1 / 1e6, 6), "step_s_estimate": round(t1, 2), "phases_s": ph1}
    if pipe is not None:
        # this run's results on the same samples: the labels of the first 8 query rows under the
        # run's codebook (equal outside the oracle's near-tie band, relative gap < 1e-6), and the
        # heatmap at the sampled windows recomputed in FP64 from the run's labels and counts
        Cg = pipe.C.cpu().numpy()
        ref, d1, d2 = oracle.assign(Xh, Cg, return_dist=True)
        band = (oracle.relative_gap(d1, d2) < 1e-6).reshape(-1)
        gl = pipe.ql[: 8].cpu().numpy().astype(np.int32).reshape(-1)
        mism = int(((gl != ref.reshape(-1)) & ~band).sum())
        href = oracle.score_at(pipe.ql.cpu().numpy().astype(np.int32), k, bank, pipe.tc.cpu().numpy(), win)
        hg = pipe.heat.cpu().numpy()[win[:, 0], win[:, 1]].astype(np.float64)
        rel = float(np.abs(hg - href).max() / max(float(np.abs(href).max()), 1e-30))
        out["oracle_check"] = {"labels_checked": int(gl.size), "label_mismatches_outside_band": mism,
                               "near_tie_band_pixels": int(band.sum()),
                               "heat_windows_checked": int(nwin), "heat_max_rel_err": rel,
                               "heat_bound": 1e-4}
        # the other precisions' labels and heatmaps on the same samples (their codebooks equal
        # the main path's: the fit is exact in every precision)
        for name, p2 in (other_pipes or {}).items():
            g2 = p2.ql[: 8].cpu().numpy().astype(np.int32).reshape(-1)
            diff = g2 != ref.reshape(-1)
            h2ref = oracle.score_at(p2.ql.cpu().numpy().astype(np.int32), k, bank, p2.tc.cpu().numpy(), win)
            h2 = p2.heat.cpu().numpy()[win[:, 0], win[:, 1]].astype(np.float64)
            out["oracle_check"][f"{name}_path"] = {
                "codebook_equal_to_main": bool(torch_equal(p2.C, pipe.C)),
                "label_mismatches_outside_band": int((diff & ~band).sum()),
                "label_mismatches_inside_band": int((diff & band).sum()),
                "heat_max_rel_err": float(np.abs(h2 - h2ref).max() / max(float(np.abs(h2ref).max()), 1e-30))}
    return out


def torch_equal(a, b):
    import torch
    return torch.equal(a, b)


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step runs the bounded sample of cpu_baseline
    (one Lloyd step, 16,384 query pixels assigned, 1,024 windows scored) on the host cores.
    ``steps`` and ``ms_per_step`` are what actually ran (the sample's wall time per step);
    ``value`` is the metric, the sample's per-phase times scaled to one whole step, and
    ``full_step_ms_estimate`` that scaled step time."""
    if rank != 0:
        return None
    import torch
    cfg = dict(HEADLINE)
    gen_dev = "cuda" if torch.cuda.is_available() else "cpu"   # input generation only
    q, T, info, bank = make_workload(gen_dev, cfg)
    for _ in range(args.warmup):
        cpu_baseline(q, T, cfg, bank)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(q, T, cfg, bank))
    wall = time.perf_counter() - t0
    v = statistics.median(x["value"] for x in vals)
    full_s = statistics.median(x["step_s_estimate"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    return {"metric": METRIC, "value": v, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * wall / max(1, args.steps), 1),
            "ms_per_step_basis": "wall time of the sampled step that ran (not the whole workload)",
            "full_step_ms_estimate": round(1e3 * full_s, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "2048x2048 query, D=512, k=128, 128x128 template, F=10 "
                                   "(full + 3x3), 10 Lloyd steps; whole hot path per step",
                       "sampled": True, "sample": cb["sample"], "wall_s": round(wall, 1),
                       "torch_threads": torch.get_num_threads()},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", choices=["bf16", "fp32", "fp8"], default="bf16")
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) leg")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--query-size", type=int, default=HEADLINE["H"],
                    help="query side (profiling captures on a smaller case)")
    ap.add_argument("--no-soft", action="store_true", help="skip the soft-VQ training-path timing")
    ap.add_argument("--soft-batch", type=int, default=8,
                    help="queries in the soft-VQ training step (8 is the workload; fewer for profiling captures)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched many-templates timing")
    ap.add_argument("--batch-eager", action="store_true",
                    help="time the batch call enqueued directly instead of replayed from a CUDA graph "
                         "(for profilers that do not follow the replay of a large graph)")
    ap.add_argument("--no-paper-bank", action="store_true",
                    help="skip scoring with the paper's own filter bank")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the small latency-bound workload (256^2, D=64, k=16)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the other precision on the same inputs")
    ap.add_argument("--shard", choices=["replicas", "bands"], default="replicas",
                    help="N > 1: one query per rank (replicas, weak scaling) or the one query's window "
                         "rows split into N row bands (strong scaling); bands runs the main leg only")
    args = ap.parse_args()
    if args.shard == "bands":
        args.no_compare = args.no_e2e = args.no_cpu_baseline = args.no_paper_bank = True
        args.no_soft = args.no_batch = args.no_small = True
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    if args.warmup < 3 and args.impl == "gpu":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_gpu(args, rank, world)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
