"""Benchmark of one hybrid iteration (Alg. 3: A half-iteration, B half-iteration,
flow update) on the 256 x 256 Gaussian-mixture workload, through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line. A step is one hybrid iteration whose half-iterations each
end with total L1 X-marginal error <= 1e-5 (every cell solve stops within its
share of that budget, the shares summing to it: time to 1e-5 L1 marginal error
per iteration), replayed from the captured CUDA graph; `value`
is the mean device time per step (ms, lower is better) with the learned warm
start, `plain_ms_per_step` the same with the method's own previous-iterate
duals, both on the same trajectory, with the state resident in device memory.
Inputs: seeded synthetic mixtures (5 components + 1e-4 floor, seeds 0 and 1)
and a Knothe-Rosenblatt initial coupling, standing in for the paper's
Gaussian-mixture test images; W warm-up steps are run first, so the timed
steps continue the same trajectory.

--impl reference times the FP64 CPU oracle (the correctness reference) on a
bounded sample of the same workload and prints the same line for it.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-5 L1 marginal err (plain vs warm-start), cell-LSE HBM GB/s"
WORKLOAD = "dd256"
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# exp-throughput peak of the cell kernel: #SM (read from the device) x ex2 per SM
# per clock x the SM clock. GB300's SMs issue 32 MUFU ex2 per clock (twice the
# 16 of earlier generations); the library's dd_probe_ex2_rate measures the rate
# in the same run and the line reports both
EX2_PER_CLK_SM = 32
SM_MAX_MHZ_DEFAULT = 2070.0
# DRAM bytes (read + write) of the cell region of one half-iteration (both k_sink
# classes + k_c2b), from one ncu capture of this bench in the launch configuration
# below (the step-kernel summary under profiles/). The bytes are those the cells read and
# write (the composite boxes, the basic boxes, the duals), which the CTA sizes do
# not change; the line names the configuration of the capture
TRAFFIC_CELL_REGION = 19.06e6
TRAFFIC_TUNING = dict(threads=[512, 64, 512], small_area=768, small_side=48, cl_size=2, cl_cells=8, sm_reserve=0)
# cell solver of every arm: Anderson acceleration of the X-dual iteration
# (memory 4; same fixed point, same stop; with it, eps-scaling inside each solve
# no longer pays and is off)
# and the batch error budget (cell budgets ~ 1e-5 mu(X) / #cells, weighted by
# the cell's previous iteration count relative to the mean and rescaled to sum
# to 1e-5 mu(X), so the half-iteration's total L1 X error stays <= 1e-5 mu(X),
# the paper's batch criterion); the line reports how many cell solves ended on a
# plateau or at the iteration cap
SOLVER = dict(eps_levels=0, tol_share=1.0, tol_gamma=1.0, anderson=4)


def peaks():
    try:
        with open(MEASURED) as fh:
            d = json.load(fh)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", SM_MAX_MHZ_DEFAULT)),
                    bf16_tflops=float(d.get("bf16_tflops", 1900.0)), src="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, sm_max_mhz=SM_MAX_MHZ_DEFAULT, bf16_tflops=1900.0, src="fallback")


def network_forward(dd, pk, rows=(1089, 16641), reps=50):
    """Forward pass of the warm-start network (four BF16 layer products) on
    random inputs: CUDA-event time per pass on the tcgen05 kernel and on the
    warp-level mma.sync kernel, for the cell counts of one 256^2 and one 1024^2
    half-iteration."""
    import torch

    from paper_2405_09400_gb300 import warmstart as ws

    flop_row = 2.0 * (dd.DD_MLP_NIN * dd.DD_MLP_NHID + 2 * dd.DD_MLP_NHID ** 2 + dd.DD_MLP_NHID * dd.DD_MLP_NOUT)
    net = dd.MLP(max(rows))
    net.set_params(ws.init_params(0))
    g = torch.Generator(device="cuda").manual_seed(0)
    out = {"flop_per_row": flop_row, "peak_tflops": pk["bf16_tflops"], "peak_src": pk["src"] + " bf16 burst"}
    st = torch.cuda.current_stream()
    for M in rows:
        x = torch.randn((M, dd.DD_MLP_NIN), generator=g, device="cuda").to(torch.bfloat16)
        r = {}
        for name, kind in (("umma", dd.DD_MLP_GEMM_UMMA), ("mma_sync", dd.DD_MLP_GEMM_MMA)):
            net.set_gemm(kind)
            for _ in range(5):
                net.forward(x)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(reps):
                net.forward(x)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            tf = flop_row * M / (ms * 1e-3) / 1e12
            r[name] = {"ms": round(ms, 4), "tflops": round(tf, 2), "frac": round(tf / pk["bf16_tflops"], 4)}
        out[str(M)] = r
    net.set_gemm(dd.DD_MLP_GEMM_UMMA)
    net.close()
    return out


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons)}


def load_workload():
    import numpy as np  # noqa: F401

    import synth

    mu, nu, eps, p = synth.workload(WORKLOAD, 0)
    boxes = synth.boxes_from_coupling(mu.shape, p["s"], *synth.knothe_rosenblatt(mu, nu))
    return mu, nu, eps, p, boxes


def _arm(dd, mu, nu, eps, p, boxes, warm, weights, args, flush, stream, tune=None, flags=0):
    """One arm: W warm-up then K timed hybrid iterations from the KR plan, every
    iteration replayed from the captured graph (the first, which fixes the
    buffer sizes, runs step by step). Returns timings and per-step stats."""
    import torch

    g = dd.DomDec(mu, nu, eps, p["s"], boxes=boxes, tol=p["tol"], max_iter=20000, warm=warm, weights=weights,
                  flags=flags, **SOLVER)
    if tune is not None:
        g.set_tuning(tune["threads"], tune["small_area"], tune["small_side"], tune["cl_size"], tune["cl_cells"],
                     tune.get("sm_reserve", 0))
    # the first hybrid iteration from the initial coupling (cold solves for the
    # plain arm): part of the warm-up, reported on its own
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(1, stats=False)
    e1.record(stream)
    e1.synchronize()
    first_ms = e0.elapsed_time(e1)
    for _ in range(args.warmup - 1):
        g.step(1, stats=False)
    torch.cuda.synchronize()
    n0 = g.counters()["launches"]
    out = dict(step_ms=[], cell_ms=[], terms=[], cells=0, hbm_bytes=[], iters_mean=[], iters_max=[], first_ms=first_ms,
               stalled=0, maxiter=0, l1x_max=0.0, mcf_ms=[], host_step_ms=[], pivots=[], c2b_ms=[], c2b_bytes=[],
               xch_ms=[],
               xch_bytes=[])
    for _ in range(args.steps):
        flush.zero_()  # evict the state from L2 between steps (outside the timed events)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        g.step(1, stats=False)  # the iteration (its statistics are read after the timed region)
        a1.record(stream)
        a1.synchronize()
        out["step_ms"].append(a0.elapsed_time(a1))
        sa, sb, sf = g.step_stats()
        out["mcf_ms"].append(sf["ms_solve"])
        out["host_step_ms"].append(sf["ms_host_step"])
        out["pivots"].append(sf["pivots"])
        out["xch_ms"].append(sf["ms_exchange"])
        out["xch_bytes"].append(sf["bytes_exchange"])
        for s_ in (sa, sb):
            out["cell_ms"].append(s_["ms_cells"])
            out["terms"].append(s_["lse_terms"])
            out["cells"] += s_["ncell"]
            out["iters_mean"].append(s_["iters_mean"])
            out["iters_max"].append(s_["iters_max"])
            out["stalled"] += s_["n_stalled"]
            out["l1x_max"] = max(out["l1x_max"], s_["l1_x"])
            out["maxiter"] += s_["n_maxiter"]
            out["c2b_ms"].append(s_["ms_c2b"])
            out["c2b_bytes"].append(s_["bytes_c2b"])
            # algorithmic bytes of the cell kernels: read the member boxes, write
            # nu_J, b and the member outputs (4 B each)
            out["hbm_bytes"].append(4.0 * (4 * s_["stored_entries"]))
    torch.cuda.synchronize()
    out["launches"] = g.counters()["launches"] - n0
    out["graph"] = g.graph_counters()
    out["E"] = g.objective()
    g.close()
    return out


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__ as ge

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("nccl")
    ge.build()
    import paper_2405_09400_gb300 as dd
    from paper_2405_09400_gb300 import warmstart as ws

    mu, nu, eps, p, boxes = load_workload()
    stream = torch.cuda.current_stream()
    weights, _ = ws.load_params()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    arms = set(args.arms.split(","))
    # autotune the cell-kernel launch configuration on this GPU and workload, on
    # the state in the middle of the timed trajectory (the composite boxes widen
    # and the slowest cells grow along it)
    tune = None
    if args.tuning:
        t = [int(x) for x in args.tuning.split(",")]
        t += [1, 0, 0][len(t) - 5:] if len(t) < 8 else []
        tune = dict(threads=t[:3], small_area=t[3], small_side=t[4], cl_size=t[5], cl_cells=t[6], sm_reserve=t[7],
                    ms_default=None, ms_best=None, trials=0)
    elif not args.no_tune:
        tctx = dd.DomDec(mu, nu, eps, p["s"], boxes=boxes, tol=p["tol"], max_iter=20000, warm=dd.DD_WARM_MLP,
                         weights=weights, **SOLVER)
        tctx.step(args.warmup + args.steps // 2, stats=False)
        tune = tctx.autotune()
        tctx.close()

        def make_ctx():
            return dd.DomDec(mu, nu, eps, p["s"], boxes=boxes, tol=p["tol"], max_iter=20000, warm=dd.DD_WARM_MLP,
                             weights=weights, **SOLVER)

        tune = rerank_by_replay(make_ctx, tune, args.warmup + args.steps // 2)
    if world > 1:
        torch.distributed.barrier()
    none = None
    with ClockSampler(local) as clk:
        plain = _arm(dd, mu, nu, eps, p, boxes, dd.DD_WARM_PREV, None, args, flush, stream, tune) \
            if "plain" in arms else none
        warm = _arm(dd, mu, nu, eps, p, boxes, dd.DD_WARM_MLP, weights, args, flush, stream, tune)
    affine = _arm(dd, mu, nu, eps, p, boxes, dd.DD_WARM_AFFINE, None, args, flush, stream, tune) \
        if "affine" in arms else none
    eager = _arm(dd, mu, nu, eps, p, boxes, dd.DD_WARM_MLP, weights, args, flush, stream, tune,
                 dd.DD_FLAG_NO_GRAPH) if "eager" in arms else none

    def total(x):
        if x is None:
            return float("nan")
        t = sum(x["step_ms"])
        if world > 1:
            tt = torch.tensor([t], device="cuda")
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            t = float(tt.item())
        return t

    ms_plain = total(plain) / args.steps
    ms_warm = total(warm) / args.steps
    ms_aff = total(affine) / args.steps
    ms_eager = total(eager) / args.steps
    # dominant kernel: the persistent cell Sinkhorn kernel (learned-warm-start arm)
    k_ms = sum(warm["cell_ms"]) / len(warm["cell_ms"])
    k_terms = sum(warm["terms"]) / len(warm["terms"])
    pk = peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    clocks = clk.summary()
    sm_max = clocks.get("sm_max_mhz") or pk.get("sm_max_mhz") or SM_MAX_MHZ_DEFAULT
    ex2_peak = n_sm * EX2_PER_CLK_SM * sm_max * 1e6  # terms (ex2) per second
    ex2_meas, ex2_ms = dd.dd_probe_ex2_rate()
    achieved = k_terms / (k_ms * 1e-3)
    hbm_gbs = (sum(warm["hbm_bytes"]) / len(warm["hbm_bytes"])) / (k_ms * 1e-3) / 1e9

    # cell-LSE microbenchmark (the paper's Fig. 10 setting adapted): every cell of
    # the bench state solved with a fixed iteration count, so the cell kernels'
    # exp throughput is measured without the tail of slow cells
    micro = None
    if not args.no_micro:
        gm = dd.DomDec(mu, nu, eps, p["s"], boxes=boxes, tol=p["tol"], max_iter=20000, warm=dd.DD_WARM_PREV,
                       **SOLVER)
        gm.set_tuning(tune["threads"], tune["small_area"], tune["small_side"], tune["cl_size"], tune["cl_cells"],
                     tune.get("sm_reserve", 0))
        gm.step(args.warmup, stats=False)
        hdr_m, data_m = dd.dd_get_plan(gm.ctx, gm.nbasic)
        gm.close()
        K = 100
        gm = dd.DomDec(mu, nu, eps, p["s"], boxes=(hdr_m, data_m), fixed_iters=K, plan_tol=1e-5, warm=dd.DD_WARM_COLD,
                       flags=dd.DD_FLAG_NO_GRAPH)
        gm.set_tuning(tune["threads"], tune["small_area"], tune["small_side"], tune["cl_size"], tune["cl_cells"],
                     tune.get("sm_reserve", 0))
        gm.iterate(0)  # warm-up (sizes, allocation)
        rs = []
        for part in (0, 1, 0, 1):
            st = gm.iterate(part)
            rs.append((st["lse_terms"], st["ms_cells"], st["ncell"]))
        gm.close()
        terms = sum(r[0] for r in rs)
        ms = sum(r[1] for r in rs)
        ach = terms / (ms * 1e-3)
        micro = {"iterations_per_cell": K, "half_iterations": len(rs), "ms_per_half_iteration": round(ms / len(rs), 4),
                 "us_per_sinkhorn_iteration_all_cells": round(1e3 * ms / len(rs) / K, 3),
                 "achieved_texp2_s": round(ach / 1e12, 4), "peak_texp2_s": round(ex2_peak / 1e12, 4),
                 "frac": round(ach / ex2_peak, 5), "box_sweep": box_sweep(tune, ex2_peak)}

    # end to end through the C ABI with host buffers: H2D of the plan, one
    # hybrid iteration (graph replay), D2H of the plan, every step (pinned host memory)
    e2e = None
    if not args.no_e2e:
        ge2 = dd.DomDec(mu, nu, eps, p["s"], boxes=boxes, tol=p["tol"], max_iter=20000, plan_tol=1e-5,
                        warm=dd.DD_WARM_MLP, weights=weights, **SOLVER)
        ge2.set_tuning(tune["threads"], tune["small_area"], tune["small_side"], tune["cl_size"], tune["cl_cells"],
                     tune.get("sm_reserve", 0))
        for _ in range(args.warmup):
            ge2.step(1, stats=False)
        hdr, data = dd.dd_get_plan(ge2.ctx, ge2.nbasic)
        hdr_p = torch.empty(hdr.shape, dtype=torch.int32).pin_memory().numpy()
        data_p = torch.empty(4 * data.size + (1 << 20), dtype=torch.float64).pin_memory().numpy()
        out_p = torch.empty(4 * data.size + (1 << 20), dtype=torch.float64).pin_memory().numpy()
        torch.cuda.synchronize()
        ts = []
        bi = bo = 0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            hdr_p[...] = hdr
            n = data.size
            data_p[:n] = data
            t0 = time.perf_counter()
            dd.dd_set_plan(ge2.ctx, hdr_p, data_p[:n])
            ge2.step(1, stats=False)
            hdr, data = dd.dd_get_plan(ge2.ctx, ge2.nbasic, out=out_p)
            ts.append(time.perf_counter() - t0)
            bi = hdr_p.nbytes + 8 * n
            bo = hdr.nbytes + data.nbytes
        e2e = {"value": round(1e3 * sum(ts) / len(ts), 4), "unit": "ms", "h2d_bytes_per_step": int(bi),
               "d2h_bytes_per_step": int(bo)}
        ge2.close()

    # HBM-bound streams of the step: CompositeToBasic + balancing + truncation
    # (k_c2b) and the flow exchange (k_plan_exchange + k_exchange), algorithmic
    # bytes / event time, against the measured copy bandwidth
    def stream_gbs(ms, by):
        ms, by = float(np.mean(ms)), float(np.mean(by))
        gbs = by / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        return {"ms": round(ms, 4), "bytes": int(by), "achieved_gbs": round(gbs, 1),
                "frac": round(gbs / pk["hbm_gbs"], 4)}

    streams = {"k_c2b": stream_gbs(warm["c2b_ms"], warm["c2b_bytes"]),
               "k_exchange": stream_gbs(warm["xch_ms"], warm["xch_bytes"]), "peak_gbs": pk["hbm_gbs"]}
    netfwd = None if args.no_micro else network_forward(dd, pk)
    ttt = None if args.no_ttt else time_to_tolerance(dd, mu, nu, eps, p, boxes, weights, tune, stream)
    cfgs = None if args.no_configs else large_configs(dd, weights, args)

    arm_map = {k: x for k, x in (("plain", plain), ("warm", warm), ("affine", affine)) if x is not None}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args, mu, nu, eps, p, boxes)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(ms_warm, 4), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_warm, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (LSE) + f64 (mass/error/objective)",
        "data": "synthetic", "impl": "ours",
        "config": {"workload": "dd256: 256x256 grid, 5-component Gaussian mixtures + 1e-4 floor (seeds 0/1), "
                               "eps=2/256^2, 4x4 basic cells, KR initial coupling, flow update every iteration, "
                               "cell tol 1e-5; a step = one hybrid iteration (A, B, flow) replayed from a CUDA "
                               "graph, every half-iteration solved to total L1 X error <= 1e-5 (per-cell "
                               "budgets summing to 1e-5 mu(X), weighted by previous iteration counts)",
                   "cells_per_half_iteration": [1024, 1089], "warm_start": "learned (value); plain = "
                   "previous-iterate duals (the paper's)", "tuning": tune, "cell_solver": SOLVER,
                   "l2": "512 MB buffer written between timed steps", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "plain_ms_per_step": round(ms_plain, 4) if plain else None, "warm_start_ms_per_step": round(ms_warm, 4),
        "affine_start_ms_per_step": round(ms_aff, 4) if affine else None,
        "warm_start_step_by_step_ms_per_step": round(ms_eager, 4) if eager else None,
        "speedup_warm_vs_plain": round(ms_plain / ms_warm, 3) if plain else None,
        "first_step_ms": {k: round(x["first_ms"], 3) for k, x in arm_map.items()},
        "sinkhorn_iters_mean": {k: round(float(np.mean(x["iters_mean"])), 2) for k, x in arm_map.items()},
        "sinkhorn_iters_max_mean": {k: round(float(np.mean(x["iters_max"])), 1) for k, x in arm_map.items()},
        "cell_solves_stalled_or_capped": {k: x["stalled"] + x["maxiter"] for k, x in arm_map.items()},
        "cell_solves_on_plateau": {k: x["stalled"] for k, x in arm_map.items()},
        "cell_solves_capped": {k: x["maxiter"] for k, x in arm_map.items()},
        "cell_solves": {k: x["cells"] for k, x in arm_map.items()},
        "step_breakdown_ms": {"cell_kernels_A_plus_B": round(2 * k_ms, 3),
                              "min_cost_flow_host": round(float(np.mean(warm["mcf_ms"])), 3),
                              # device time from the edge costs to the flow back on the device
                              # (copies, host solve, handover to and from the host)
                              "flow_host_step_device": round(float(np.mean(warm["host_step_ms"])), 3),
                              "rest": round(ms_warm - 2 * k_ms - float(np.mean(warm["mcf_ms"])), 3),
                              "mcf_pivots_mean": round(float(np.mean(warm["pivots"])), 1)},
        "half_iteration_l1x_max": {k: x["l1x_max"] for k, x in arm_map.items()},
        "iterations_per_s": round(1e3 / ms_warm, 3),
        "cells_per_s": round(warm["cells"] / (sum(warm["step_ms"]) * 1e-3), 1),
        "graph": warm["graph"],
        "cell_lse_hbm_gbs": {"achieved": round(hbm_gbs, 2), "peak": pk["hbm_gbs"], "frac": round(hbm_gbs / pk["hbm_gbs"], 5),
                             "peak_src": pk["src"]},
        "roofline": {"bound": "alu", "kernel": "k_sink (persistent cell Sinkhorn, + k_c2b)",
                     "achieved": round(achieved / 1e12, 4), "peak": round(ex2_peak / 1e12, 4), "unit": "Texp2/s",
                     "frac": round(achieved / ex2_peak, 5),
                     "traffic": TRAFFIC_CELL_REGION,
                     "traffic_src": "ncu dram__bytes of one capture at threads %s, small %d/%d, clusters of %d "
                                    "for %d cells (profiles/, dd256 step kernels)" % (
                                        TRAFFIC_TUNING["threads"], TRAFFIC_TUNING["small_area"],
                                        TRAFFIC_TUNING["small_side"], TRAFFIC_TUNING["cl_size"],
                                        TRAFFIC_TUNING["cl_cells"]),
                     "kernel_ms_mean": round(k_ms, 4),
                     "work_per_launch": k_terms,
                     "peak_src": f"{n_sm} SMs x {EX2_PER_CLK_SM} ex2/clk x {sm_max:.0f} MHz"},
        "ex2_probe": {"measured_tex2_s": round(ex2_meas / 1e12, 4), "ms": round(ex2_ms, 4),
                      "ex2_per_clk_sm_at_max_clock": round(ex2_meas / (n_sm * sm_max * 1e6), 2)},
        "cell_lse_fixed_iterations": micro,
        "hbm_streams": streams,
        "network_forward": netfwd,
        "time_to_tolerance": ttt,
        "configs": cfgs,
        "clocks": clocks,
        "gpu_launches": int(warm["launches"]),
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


_ORACLE = {}


def _oracle_init(mu, eps, p, boxes):
    """Worker set-up (spawned process): one BLAS thread, the workload's state."""
    try:
        from threadpoolctl import threadpool_limits

        _ORACLE["limit"] = threadpool_limits(1)
    except ImportError:
        pass
    from oracle.domdec import Box
    from oracle.geometry import Geometry

    N = mu.shape[0]
    geom = Geometry(N, N, p["s"])
    _ORACLE.update(mu=mu, eps=eps, p=p, geom=geom, m=geom.basic_masses(mu), cells=geom.partition(0),
                   bx=[Box(o1, o2, a) for o1, o2, a in boxes])


def _oracle_cells(js):
    """Whole FP64 oracle solves (solve, CompositeToBasic, balance, truncate) of cells js."""
    from oracle.domdec import balance, basic_to_composite, composite_to_basic, solve_cell, truncate_box

    o = _ORACLE
    N = o["mu"].shape[0]
    t0 = time.perf_counter()
    for J in js:
        members = o["cells"][J]
        nuJ = basic_to_composite(o["bx"], members)
        res = solve_cell(o["geom"], o["mu"], o["eps"], 1.0 / N, members, nuJ, None, o["p"]["tol"], 100000)
        arrs, _ = composite_to_basic(o["geom"], members, nuJ, res)
        bal = balance(arrs, [o["m"][i] for i in members])
        for k, i in enumerate(members):
            truncate_box(bal[k], nuJ.o1, nuJ.o2, 1e-15, o["m"][i])
    return len(js), time.perf_counter() - t0


def _oracle_sample(mu, nu, eps, p, boxes, seconds, workers):
    """Time the FP64 oracle on a bounded sample: whole-cell solves of the first A
    half-iteration (cold start from the KR plan) on `workers` processes (spawned,
    one thread each; the cells of a half-iteration are independent) for about
    `seconds` of wall time. Each process times its own solves while all run
    concurrently; the time per cell with `workers` processes is the summed solve
    time / cells / workers, scaled to all cells of a hybrid iteration. Plus one
    flow-update step (edge costs and the LP) in one process, as the oracle
    computes it."""
    import multiprocessing as mp

    import numpy as np

    from oracle.flow import edge_costs, min_cost_flow

    _oracle_init(mu, eps, p, boxes)
    geom, bx, m = _ORACLE["geom"], _ORACLE["bx"], _ORACLE["m"]
    order = [int(J) for J in np.random.default_rng(0).permutation(len(_ORACLE["cells"]))]
    chunk = 4
    n = 0
    busy = 0.0
    if workers <= 1:
        t0 = time.perf_counter()
        while n < len(order) and time.perf_counter() - t0 <= seconds:
            c, b = _oracle_cells(order[n:n + 1])
            n += c
            busy += b
    else:
        with mp.get_context("spawn").Pool(workers, initializer=_oracle_init, initargs=(mu, eps, p, boxes)) as pool:
            t0 = time.perf_counter()
            pending = []
            k = 0
            while True:
                while k < len(order) and len(pending) < 2 * workers and time.perf_counter() - t0 <= seconds:
                    pending.append(pool.apply_async(_oracle_cells, (order[k:k + chunk],)))
                    k += chunk
                if not pending:
                    break
                c, b = pending.pop(0).get()
                n += c
                busy += b
    t_cell = busy / n / max(1, workers)  # time per cell with `workers` concurrent processes
    D = np.zeros(geom.nb)
    t1 = time.perf_counter()
    cbar = edge_costs(geom, mu, bx, D, 1.0 / mu.shape[0])
    t_cost = time.perf_counter() - t1
    t2 = time.perf_counter()
    min_cost_flow(geom.neighbours(), cbar, m)
    t_lp = time.perf_counter() - t2
    ncell = len(geom.partition(0)) + len(geom.partition(1))
    ms = 1e3 * (t_cell * ncell + t_cost + t_lp)
    return ms, n, t_cell, t_cost, t_lp


def cpu_baseline(args, mu, nu, eps, p, boxes):
    workers = os.cpu_count() or 1
    ms, n, t_cell, t_cost, t_lp = _oracle_sample(mu, nu, eps, p, boxes, args.cpu_seconds, workers)
    return {"value": round(ms, 1), "unit": "ms", "cores": workers, "kind": "oracle",
            "sample": f"FP64 oracle on {workers} processes (one thread each): {n} whole cell solves of the first A "
                      f"half-iteration (cold start from the KR plan, dense LSE, tol 1e-5), "
                      f"{t_cell*1e3:.2f} ms of wall time per cell, scaled to 2113 cells; edge costs "
                      f"{t_cost*1e3:.0f} ms (explicit sums, all cells) and the min-cost flow LP {t_lp*1e3:.0f} ms "
                      f"(HiGHS, full size) in one process"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    mu, nu, eps, p, boxes = load_workload()
    t0 = time.perf_counter()
    vals = []
    workers = os.cpu_count() or 1
    for _ in range(max(1, args.steps)):
        ms, n, t_cell, t_cost, t_lp = _oracle_sample(mu, nu, eps, p, boxes, args.cpu_seconds / max(1, args.steps),
                                                     workers)
        vals.append(ms)
    v = sum(vals) / len(vals)
    cpu = {"value": round(v, 1), "unit": "ms", "cores": workers, "kind": "oracle",
           "sample": f"FP64 oracle on {workers} processes (one thread each), per step {n} whole cell solves of the "
                     "first A half-iteration (cold, KR plan) scaled to 2113 cells, plus the flow-update step"}
    line = {"metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "dd256 (same as --impl ours)"}, "cpu_baseline": cpu,
            "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(time.perf_counter() - t0, 2)}
    print(json.dumps(line), flush=True)


def time_to_tolerance(dd, mu, nu, eps, p, boxes, weights, tune, stream, n_ref=1200, gaps=(1e-3, 1e-4)):
    """End-to-end time to tolerance on the bench workload, plain vs learned warm
    start: device time of the hybrid run from the KR plan (first iteration step
    by step, then graph replays) until the objective E_k is within `gap` of E*
    (relative), every half-iteration at total L1 X error <= 1e-5. E* is the
    smallest objective of a reference run of n_ref iterations with the same
    solver. Iteration counts come from a run with per-step statistics; the time
    from a second run of exactly that many steps without them."""
    import numpy as np
    import torch

    def make(warm):
        g = dd.DomDec(mu, nu, eps, p["s"], boxes=boxes, tol=p["tol"], max_iter=20000, warm=warm,
                      weights=weights if warm == dd.DD_WARM_MLP else None, **SOLVER)
        g.set_tuning(tune["threads"], tune["small_area"], tune["small_side"], tune["cl_size"], tune["cl_cells"],
                     tune.get("sm_reserve", 0))
        return g

    ref = make(dd.DD_WARM_PREV)
    Es = []
    for _ in range(n_ref):
        sa, sb, sf = ref.step(1, stats=True)
        Es.append(sb["objective"])
    ref.close()
    Estar = float(min(Es))
    out = {"E_star": Estar, "E_star_from": f"min objective of {n_ref} hybrid iterations (plain start, same solver)",
           "l1x_per_half_iteration": "<= 1e-5 (batch budget)", "runs": {}}
    for name, warm in (("plain", dd.DD_WARM_PREV), ("warm", dd.DD_WARM_MLP)):
        g = make(warm)
        need = {}
        l1x = 0.0
        for k in range(1, n_ref + 1):
            sa, sb, sf = g.step(1, stats=True)
            l1x = max(l1x, sa["l1_x"], sb["l1_x"])
            for gap in gaps:
                if gap not in need and (sb["objective"] - Estar) <= gap * abs(Estar):
                    need[gap] = k
            if len(need) == len(gaps):
                break
        g.close()
        res = {}
        for gap in gaps:
            if gap not in need:
                res[str(gap)] = None
                continue
            g = make(warm)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.step(need[gap], stats=False)
            e1.record(stream)
            e1.synchronize()
            res[str(gap)] = {"iterations": need[gap], "ms": round(e0.elapsed_time(e1), 2)}
            g.close()
        out["runs"][name] = dict(res, l1x_max=l1x)
    return out


def large_configs(dd, weights, args):
    """Per-iteration figures of the larger configurations, same cell solver:
    uneven512 (512 x 512, uniform mu, 8 narrow Gaussians, eps = h^2, KR plan) and
    dd1024 (1024 x 1024, 6-component mixtures, eps = 2 h^2) from its configured
    initial plan: a 512 x 512 plan of the 2 x 2-coarsened measures after 100
    hybrid iterations from KR, prolongated with 1 % seeded noise projected onto
    exact marginals (synth.prolongate), learned warm start. Each: 3 warm-up
    iterations, then 3 timed (CUDA events, graph replay)."""
    import numpy as np
    import torch

    import synth

    res = {}

    def timed(g, n_warm=3, n=3):
        g.step(n_warm, stats=False)
        ms, l1x, stalls, capped, mcf, cells, itmax = [], 0.0, 0, 0, [], [], []
        for _ in range(n):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.step(1, stats=False)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            sa, sb, sf = g.step_stats()
            l1x = max(l1x, sa["l1_x"], sb["l1_x"])
            stalls += sa["n_stalled"] + sb["n_stalled"]
            capped += sa["n_maxiter"] + sb["n_maxiter"]
            mcf.append(sf["ms_solve"])
            cells.append(sa["ms_cells"] + sb["ms_cells"])
            itmax.append(max(sa["iters_max"], sb["iters_max"]))
        return {"ms_per_step": round(float(np.mean(ms)), 3), "cell_kernels_ms": round(float(np.mean(cells)), 3),
                "min_cost_flow_host_ms": round(float(np.mean(mcf)), 3), "half_iteration_l1x_max": l1x,
                "plateau_stops": stalls, "capped": capped, "sinkhorn_iters_max": int(max(itmax)),
                "cells_per_half_iteration": [g.ncell[0], g.ncell[1]]}

    mu, nu, eps, p = synth.workload("uneven512", 0)
    boxes = synth.boxes_from_coupling(mu.shape, 4, *synth.knothe_rosenblatt(mu, nu))
    g = dd.DomDec(mu, nu, eps, 4, boxes=boxes, tol=1e-5, max_iter=20000, warm=dd.DD_WARM_PREV, **SOLVER)
    res["uneven512"] = timed(g)
    g.close()

    mu, nu, eps, p = synth.workload("dd1024", 0)
    muc, nuc = synth.coarsen(mu), synth.coarsen(nu)
    bc = synth.boxes_from_coupling(muc.shape, 4, *synth.knothe_rosenblatt(muc, nuc))
    gc = dd.DomDec(muc, nuc, 4 * eps, 4, boxes=bc, tol=1e-5, max_iter=20000, warm=dd.DD_WARM_PREV, **SOLVER)
    gc.step(100, stats=False)
    coarse = [(o1, o2, a) for o1, o2, a in gc.plan()]
    gc.close()
    fine = synth.prolongate(coarse, mu, nu, 4, noise=0.01, seed=0)
    g = dd.DomDec(mu, nu, eps, 4, boxes=fine, tol=1e-5, max_iter=20000, plan_tol=1e-6, warm=dd.DD_WARM_MLP,
                  weights=weights, **SOLVER)
    res["dd1024_prolongated"] = timed(g)
    g.close()
    return res


# finalists of the replay ranking besides the autotuner's choice: the configurations
# that did best in earlier runs of this bench (clusters of 2 or 4 CTAs for the 8 cells
# of most expected work gave ~4 % less cell time than none in paired runs)
REPLAY_FINALISTS = (dict(threads=[512, 64, 512], small_area=768, small_side=48, cl_size=1, cl_cells=0, sm_reserve=0),
                    dict(threads=[512, 64, 512], small_area=768, small_side=48, cl_size=2, cl_cells=8, sm_reserve=0),
                    dict(threads=[512, 64, 512], small_area=768, small_side=48, cl_size=4, cl_cells=8, sm_reserve=0),
                    dict(threads=[512, 128, 512], small_area=768, small_side=48, cl_size=1, cl_cells=0, sm_reserve=32))


def rerank_by_replay(make_ctx, tune, n_pre, k=6):
    """The library's autotuner times its trials step by step; the timed arms replay
    CUDA graphs, where the size classes start together. Re-rank its choice and the
    REPLAY_FINALISTS by the cell time of graph replays, paired: one context per
    configuration from the same start, stepped in lockstep through n_pre steps and
    then k measured steps (the per-step cost varies along the trajectory more than
    between configurations). Returns the fastest, with the measured means."""
    import numpy as np

    key = lambda t: (tuple(t["threads"]), t["small_area"], t["small_side"], t["cl_size"],
                     t["cl_cells"] if t["cl_size"] > 1 else 0, t["sm_reserve"])
    uniq = []
    for t in [dict(tune)] + [dict(t) for t in REPLAY_FINALISTS]:
        if all(key(t) != key(u) for u in uniq):
            uniq.append(t)
    ctxs = []
    for t in uniq:
        g = make_ctx()
        g.set_tuning(list(t["threads"]), t["small_area"], t["small_side"], t["cl_size"], t["cl_cells"], t["sm_reserve"])
        ctxs.append(g)
    ms = [[] for _ in uniq]
    for step in range(n_pre + k):
        for i, g in enumerate(ctxs):
            g.step(1, stats=False)
            if step >= n_pre:
                sa, sb, _ = g.step_stats()
                ms[i].append(sa["ms_cells"] + sb["ms_cells"])
    for g in ctxs:
        g.close()
    means = [float(np.mean(m)) for m in ms]
    best = dict(uniq[int(np.argmin(means))])
    best.update(ms_default=tune.get("ms_default"), ms_best=tune.get("ms_best"), trials=tune.get("trials"),
                autotuner_choice={k_: tune[k_] for k_ in ("threads", "small_area", "small_side", "cl_size", "cl_cells",
                                                          "sm_reserve")},
                replay_cell_ms={str(key(t)): round(v, 4) for t, v in zip(uniq, means)})
    return best


def box_sweep(tune, ex2_peak, K=50):
    """Cell-LSE throughput per box size: (2048/m)^2 independent cells with 8 x 8 X
    blocks and m x m boxes (synth.cell_lse_sweep), K fixed iterations from a cold
    start, A half-iterations only. Per size, the CTA sizes of the large- and
    small-box classes are chosen among four pairs by timing (the library's
    autotuner times A and B together; here only A has m x m boxes); two timed
    half-iterations per pair, the plan reset before each; the best pair is
    reported."""
    import paper_2405_09400_gb300 as dd
    import synth

    pairs = ((512, 64), (512, 128), (512, 256), (256, 128))
    rows = []
    for m in synth.cellbench.SIDES:
        mu, nu, eps, s, (hdr, data) = synth.cell_lse_sweep(m, 0)
        g = dd.DomDec(mu, nu, eps, s, boxes=(hdr, data), fixed_iters=K, warm=dd.DD_WARM_COLD,
                      flags=dd.DD_FLAG_NO_GRAPH)
        g.iterate(0)  # sizes, allocation
        best = None
        for t0, t1 in pairs:
            g.set_tuning([t0, t1, t0], tune["small_area"], tune["small_side"], 1, 0)
            terms = ms = 0.0
            for _ in range(2):
                g.set_plan((hdr, data))
                st = g.iterate(0)
                terms += st["lse_terms"]
                ms += st["ms_cells"]
            if best is None or ms < best[0]:
                best = (ms, terms, t0, t1, st["ncell"])
        g.close()
        ms, terms, t0, t1, ncell = best
        ach = terms / (ms * 1e-3)
        rows.append({"box": m, "cells": ncell, "threads_large_small": [t0, t1],
                     "ms_per_half_iteration": round(ms / 2, 4),
                     "us_per_sinkhorn_iteration_all_cells": round(1e3 * ms / 2 / K, 3),
                     "achieved_texp2_s": round(ach / 1e12, 4), "frac": round(ach / ex2_peak, 5)})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="default launch configuration (no autotuning)")
    ap.add_argument("--no-micro", action="store_true", help="skip the fixed-iteration cell-LSE microbenchmark")
    ap.add_argument("--no-ttt", action="store_true", help="skip the end-to-end time-to-tolerance runs")
    ap.add_argument("--no-configs", action="store_true", help="skip the 512 x 512 and 1024 x 1024 configurations")
    ap.add_argument("--tuning", default="", help="fixed launch configuration t0,t1,t2,small_area,small_side"
                                               "[,cl_size,cl_cells[,sm_reserve]] instead of autotuning (profiling runs)")
    ap.add_argument("--arms", default="plain,warm,affine,eager",
                    help="comma list of arms to time besides the learned warm start (plain, affine, eager)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
