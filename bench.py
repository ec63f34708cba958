"""Benchmark: chemistry cell-steps/s of the bulk-sparse GPU integrator on one flow step.

Workload (one step = one chemistry sub-step of the whole field): a 128^3 reacting-sheet field
(2,097,152 cells, 5% of them in a curved reacting sheet at 1500-3000 K with Dirichlet(0.5)
composition, the rest cold premix at 300-400 K), the seeded H2-air-shaped mechanism (9 species,
21 reversible reactions), dt = 1e-8 s, FP32 state.  Each step restores the input state from a
pristine device copy, flushes L2 (256 MiB write) and advances every cell through the C ABI
(bulk kernel + stiff kernel).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

A second leg ("gated" in the JSON line) times the same steps with the learned surrogate in
front of the method (chem_advance_gated), after training it on pairs made by the plain integrator
(outside the timed region), and reports the accepted fraction and the sampled error vs the oracle.
A third leg ("paper_loop") times the paper's own method on the same steps: explicit first-order
substeps under the relative-change rule of Sec. 2.1, driven by Algorithm 3 (chem_advance_explicit),
with its sampled error vs the oracle.  Three more objects carry the other workloads: "config2" (the
400-box AMR hierarchy through the box table, graph-replayed), "config3" (a 16M-cell flat batch,
plain and gated) and "config4" (the 53-species sheet at 32x32x16, plain and gated); `--no-configs`
leaves them out, and `--config 3|4` makes either the line's own workload.

Under torchrun (N > 1) every rank advances its own field (seed = rank): weak scaling, no
collective on the data path; the step time is the max over ranks.  `--impl reference` times the
FP64 CPU oracle (the checker of this library) on bounded stratified samples of the same field.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_2510_23993_gb300.shard import max_over_ranks  # noqa: E402

METRIC = "chem cell-steps/s at rel err ≤1e-4 (gated surrogate vs plain GPU), % roofline"
UNIT = "cell-steps/s"
DT = 1e-8
N_EDGE = 128
# algorithmic FP64 flops of the stiff integrator per unit of work (ns species, of which the leading
# na take part in the linear algebra; the trailing inert ones have identity rows and zero updates):
#   per attempted step: iteration matrix I - g h J (2 na^2) + LU with partial pivoting of the
#       na x na block (sum_k 2 (na-k-1)^2 + (na-k-1), plus na reciprocals) + error filter
#       (5 na + solve 2 na^2 + norm 2 na)
#   per Newton iteration: T(e) (mixture 12 ns + 2 iterations x 21) + residual 3 na + solve 2 na^2
#       + update/norm 2 na, except that the first iteration of an attempt starts from the step's
#       initial state, whose temperature is known: one T(e) fewer per attempt
#   per accepted step: T(e) of the new state (12 ns + 42)


def f_factor(ns, na):
    """Forming I - g h J (na^2 products and additions) and its LU with partial pivoting."""
    lu = sum(2 * (na - k - 1) ** 2 + (na - k - 1) for k in range(na)) + na
    return 2 * na * na + lu


def f_attempt(ns, na):
    """An attempted step that factors: the factorisation, the error estimate and its filter."""
    return f_factor(ns, na) + 5 * na + 2 * na * na + 2 * na


def f_te(ns):
    """One FP64 T(e) inversion: the mixture sums and two Newton iterations on the polynomial."""
    return 12 * ns + 42


def f_newton(ns, na):
    return f_te(ns) + 3 * na + 2 * na * na + 2 * na


def f_accept(ns, na):
    return f_te(ns)


def active_species(mech):
    """Species before the trailing run of inert ones (no net stoichiometry in any reaction)."""
    d = np.asarray(mech["nu_r"], int) - np.asarray(mech["nu_f"], int)
    na = mech["ns"]
    while na > 1 and not d[:, na - 1].any():
        na -= 1
    return na


# FP64 peak from the unit count (152 SMs x 2 FP64 FMA lanes/clock x 2 flops x 2.07 GHz), reported
# beside the measured one
FP64_PEAK_UNITS_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def _config(n, args):
    if args.config == 3:
        return {"workload": f"flat batch of {n} cells drawn from the AMR shear-layer state distribution (400 boxes "
                            f"over 3 levels per draw, ~3% stiff), H2-air-shaped mechanism 9 species / 21 reactions, "
                            f"dt = {DT:g} s, FP32 state; plain bulk-sparse vs gated surrogate",
                "cells": n, "dt_s": DT, "rtol": args.rtol, "atol": args.atol,
                "l2": "flushed (256 MiB write) and state restored from a pristine copy inside every step",
                "mechanism_seed": 0, "field_seed": "rank"}
    if args.config == 4:
        e = args.edge
        return {"workload": f"reacting sheet {2 * e}x{2 * e}x{e} ({n} cells, 4% reacting), hydrocarbon-shaped "
                            f"mechanism 53 species / 325 reactions (30 third-body), dt = {DT:g} s, FP32 state, "
                            f"bulk-sparse, one warp per cell",
                "cells": n, "dt_s": DT, "rtol": args.rtol, "atol": args.atol,
                "l2": "flushed (256 MiB write) and state restored from a pristine copy inside every step",
                "mechanism_seed": 0, "field_seed": "rank"}
    return {"workload": f"reacting sheet {args.edge}^3 ({n} cells, 5% reacting), H2-air-shaped mechanism "
                        f"9 species / 21 reactions, dt = {DT:g} s, FP32 state, bulk-sparse",
            "cells": n, "dt_s": DT, "rtol": args.rtol, "atol": args.atol,
            "l2": "flushed (256 MiB write) and state restored from a pristine copy inside every step",
            "mechanism_seed": 0, "field_seed": "rank"}


def _field(seed, edge=N_EDGE, config=1, cells=16_000_000):
    if config == 3:   # flat batch of cells drawn from the AMR jet-in-crossflow-like state distribution
        mech = synth.h2_air_mechanism(0)
        Ts, ps, Ys, hs = [], [], [], []
        k = 0
        while sum(t.size for t in Ts) < cells:
            boxes = synth.amr_boxes(seed=2 * seed + k)
            for T, p, Y, hot in synth.helix_box_fields(mech, boxes, seed=2 * seed + k, stiff_frac=0.03):
                Ts.append(T), ps.append(p), Ys.append(Y), hs.append(hot)
            k += 1
        perm = np.random.default_rng(seed).permutation(sum(t.size for t in Ts))[:cells]
        T, p, hot = np.concatenate(Ts)[perm], np.concatenate(ps)[perm], np.concatenate(hs)[perm]
        Y = np.concatenate(Ys, axis=1)[:, perm]
        return mech, T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32), hot
    if config == 4:   # 2e x 2e x e sheet, 4% reacting, 53-species mechanism (256 x 256 x 128 at e = 128)
        mech = synth.hydrocarbon_mechanism(0)
        T, p, Y, hot = synth.sheet_field(mech, nx=2 * edge, ny=2 * edge, nz=edge, frac=0.04, seed=seed)
        return mech, T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32), hot
    mech = synth.h2_air_mechanism(0)
    T, p, Y, hot = synth.sheet_field(mech, n=edge, seed=seed)
    return mech, T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32), hot


def _oracle_sample(mech, T, p, Y, hot, n_sample, seed):
    import oracle
    idx = synth.stratified_sample(hot, n_sample, seed=seed)
    rho, e = oracle.state_from_TpY(mech, T[idx], p[idx], Y[:, idx])
    rho, e = rho.astype(np.float32), e.astype(np.float32)
    t0 = time.perf_counter()
    T1, _, Y1, steps = oracle.advance(mech, rho, e, T[idx], Y[:, idx], DT)
    wall = time.perf_counter() - t0
    return idx, rho, e, T1, Y1, wall, oracle.max_threads()


class ClockSampler:
    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_bench_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
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
        self.f.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if "Active" in r[5 + j] and "Not" not in r[5 + j]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def run_gpu(args, rank, world, local_rank, dist):
    import torch
    import paper_2510_23993_gb300 as chem
    chem.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    mech, T, p, Y, hot = _field(seed=rank, edge=args.edge, config=args.config, cells=args.cells)
    n = T.size
    ns = mech["ns"]
    flags = chem.CHEM_FLAG_TIMING | chem.CHEM_FLAG_ORDER_RATE | (chem.CHEM_FLAG_FP64_RATES if args.fp64_rates else 0) \
        | (chem.CHEM_FLAG_TWO_PASS if args.two_pass else 0)
    ctx = chem.Context(mech, max_cells=max(n, args.train_pairs), rtol=args.rtol, atol=args.atol, flags=flags)
    tT, tp, tY = (torch.from_numpy(a).to(dev) for a in (T, p, Y))
    rho, e = torch.empty_like(tT), torch.empty_like(tT)
    ctx.state_from_TpY(tT, tp, tY, rho, e)
    sub = torch.zeros(n, dtype=torch.int32, device=dev)
    tuned = None
    if args.tune:   # launch configuration picked by the library's autotuner (outside the timed region)
        tuned = ctx.tune(tT, tp, tY, rho, e, DT, sub, cache_path=args.tune_cache)
    T0, Y0 = tT.clone(), tY.clone()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(i):
        tT.copy_(T0)
        tY.copy_(Y0)
        flush.fill_(i & 0xFF)
        ctx.advance(tT, tp, tY, rho, e, DT, sub)
        return ctx.status()

    for i in range(args.warmup):
        step(i)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    stats = [step(i) for i in range(args.steps)]
    ev1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist)
    total_cells = n * world
    value = total_cells * args.steps / (ms / 1e3)
    for s in stats:
        assert s["status"] == 0, s
    # dominant kernel: the stiff kernel (FP64 pipe); its algorithmic FP64 work per launch
    na = active_species(mech)
    stiff_ms = float(np.mean([s["stiff_ms"] for s in stats]))
    bulk_ms = float(np.mean([s["bulk_ms"] for s in stats]))
    flops = float(np.mean([_stiff_flops(s, ns, na) for s in stats]))
    achieved = flops / (stiff_ms / 1e3) / 1e12
    fp64_peak = chem.chem_measure_fp64_peak(reps=5)   # FMA chains on this GPU, outside the timed region
    roof = {"kernel": "stiff_kernel" if ns <= 15 else "stiff_kernel_lg", "bound": "alu", "pipe": "fp64", "achieved": achieved,
            "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
            "traffic": _traffic() if args.config == 1 and args.edge == N_EDGE else None,
            "kernel_ms": stiff_ms, "bulk_kernel_ms": bulk_ms,
            "algorithmic_flops_per_launch": flops, "active_species": na,
            "peak_source": "measured: chem_measure_fp64_peak (independent FP64 FMA chains on every SM, best of 5)",
            "frac_of_unit_count_peak": achieved / FP64_PEAK_UNITS_TFLOPS,
            "unit_count_peak": FP64_PEAK_UNITS_TFLOPS}
    # end to end through the host entry point (pinned host buffers, copies inside the timing)
    e2e = None
    if args.e2e:
        hT, hp, hY = (torch.from_numpy(a).pin_memory() for a in (T, p, Y))
        hrho, he = rho.cpu().pin_memory(), e.cpu().pin_memory()
        hsub = torch.zeros(n, dtype=torch.int32).pin_memory()
        wall = 0.0
        for i in range(args.warmup + args.steps):
            hT.copy_(torch.from_numpy(T))
            hY.copy_(torch.from_numpy(Y))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.advance_host(hT, hp, hY, hrho, he, DT, hsub)
            if i >= args.warmup:
                wall += time.perf_counter() - t0
        wall = max_over_ranks(wall, dist)
        e2e = {"value": total_cells * args.steps / wall, "unit": UNIT,
               "h2d_bytes_per_step": int(n * 4 * (ns + 4)), "d2h_bytes_per_step": int(n * 4 * (ns + 3))}
    # kernels per step: bulk, queue order, stiff (two-pass: + continuation order + second stiff launch)
    per_step = 5 if ctx.params.flags & chem.CHEM_FLAG_TWO_PASS else 3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": _config(n, args), "roofline": roof, "e2e": e2e, "gpu_launches": per_step * args.steps * world,
            "clocks": clk, "tuned": tuned,
            "stiff": {"queued_cells": stats[-1]["nqueued"], "bulk_cells": stats[-1]["nbulk"],
                      "substeps_per_stiff_cell": stats[-1]["substeps"] / max(1, stats[-1]["nqueued"]),
                      "attempts_per_substep": stats[-1]["attempts"] / max(1, stats[-1]["substeps"]),
                      "newton_per_attempt": stats[-1]["newton"] / max(1, stats[-1]["attempts"]),
                      "factorizations_per_attempt": stats[-1]["factorizations"] / max(1, stats[-1]["attempts"])}}
    if args.gated:   # the surrogate is compiled for the 9- and the 53-species mechanisms
        line["gated"] = _gated_leg(args, ctx, chem, torch, dev, mech, step_inputs=(tT, tp, tY, rho, e, sub, T0, Y0, flush),
                                   plain_ms=ms / args.steps, n=n, world=world, dist=dist, rank=rank)
    if args.paper_loop and ns == 9:   # the paper's explicit scheme is compiled for the dense path
        line["paper_loop"] = _paper_loop_leg(args, ctx, chem, torch, step_inputs=(tT, tp, tY, rho, e, sub, T0, Y0, flush),
                                             plain_ms=ms / args.steps, n=n, world=world, dist=dist)
    if args.configs and args.config == 1:
        line["config2"] = _config2_leg(args, chem, torch, dev, ctx.params.flags, ctx.params.k_bulk, rank, world, dist,
                                       fp64_peak)
        line["config3"] = _config3_leg(args, chem, torch, dev, ctx, rank, world, dist, fp64_peak,
                                       gated="gated" in line)
        line["config4"] = _config4_leg(args, chem, torch, dev, rank, world, dist, fp64_peak)
    if rank == 0 and world == 1 and args.cpu_baseline:
        # the 53-species oracle costs ~15 s per stiff cell per core: a smaller sample for config 4
        n_sample = args.cpu_sample if args.config == 1 else min(args.cpu_sample, 256)
        idx, orho, oe, oT, oY, wall, cores = _oracle_sample(mech, T, p, Y, hot, n_sample, seed=0)
        line["cpu_baseline"] = {"value": len(idx) / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{len(idx)} cells stratified from the same field "
                                          f"({int(hot[idx].sum())} reacting), FP64 Radau IIA rtol 1e-10"}
        line["accuracy"] = _accuracy(ctx, torch, dev, T[idx], p[idx], Y[:, idx], orho, oe, oT, oY, mech=mech)
        if "gated" in line:
            line["gated"]["accuracy"] = _accuracy(ctx, torch, dev, T[idx], p[idx], Y[:, idx], orho, oe, oT, oY,
                                                  gate_tol=args.gate_tol, mech=mech)
        if "paper_loop" in line:
            plain_frac = ctx.params.bulk_frac
            ctx.set_params(bulk_frac=args.paper_frac)
            line["paper_loop"]["accuracy"] = _accuracy(ctx, torch, dev, T[idx], p[idx], Y[:, idx], orho, oe, oT, oY,
                                                       explicit=True)
            ctx.set_params(bulk_frac=plain_frac)
    return line


def _stiff_flops(st, ns, na):
    """Algorithmic FP64 flops of the stiff phase from the counters of one advance call (the
    factorisations counted as done: the large-mechanism kernel reuses some across steps)."""
    nf = st.get("factorizations", st["attempts"])
    return (st["attempts"] * (f_attempt(ns, na) - f_factor(ns, na) - f_te(ns)) + nf * f_factor(ns, na)
            + st["newton"] * f_newton(ns, na) + st["substeps"] * f_accept(ns, na))


def _sampled_reference(mech, T, p, Y, hot, dts, n_sample, seed):
    """The oracle's results on a stratified sample (half of it stiff cells) of the inputs T, p, Y
    with steps dts: (sample indices, T, Y)."""
    import oracle
    idx = synth.stratified_sample(hot, n_sample, seed=seed, hot_frac=0.5)
    rho, e = oracle.state_from_TpY(mech, T[idx], p[idx], Y[:, idx])
    rho, e = rho.astype(np.float32), e.astype(np.float32)
    T_ref = np.empty(len(idx))
    Y_ref = np.empty((Y.shape[0], len(idx)))
    for d in np.unique(dts[idx]):
        m = dts[idx] == d
        T_ref[m], _, Y_ref[:, m], _ = oracle.advance(mech, rho[m], e[m], T[idx][m], Y[:, idx][:, m], float(d))
    return idx, T_ref, Y_ref


def _sampled_accuracy(mech, T, p, Y, hot, out_T, out_Y, dts, n_sample, seed, ref=None):
    """Error against the oracle on a stratified sample (half of it stiff cells): T, p, Y the inputs,
    out_T, out_Y the GPU's results for the same cells, dts the cells' steps; ref a result of
    _sampled_reference to compare against instead of a new sample."""
    idx, T_ref, Y_ref = ref if ref is not None else _sampled_reference(mech, T, p, Y, hot, dts, n_sample, seed)
    Tg, Yg = out_T[idx].astype(np.float64), out_Y[:, idx].astype(np.float64)
    big = Y_ref >= 1e-6
    rel = np.where(big, np.abs(Yg - Y_ref) / np.maximum(Y_ref, 1e-300), 0.0)
    ab = np.where(~big, np.abs(Yg - Y_ref), 0.0)
    eT = np.abs(Tg - T_ref) / T_ref
    over = (rel.max(0) > 1e-4) | (ab.max(0) > 1e-10) | (eT > 1e-4)
    return {"cells": int(len(idx)), "stiff_cells": int(hot[idx].sum()), "max_rel_Y": float(rel.max()),
            "max_abs_small_Y": float(ab.max()), "max_rel_T": float(eT.max()), "cells_over_1e-4": int(over.sum())}


def _config2_leg(args, chem, torch, dev, flags, k_bulk, rank, world, dist, fp64_peak):
    """Config 2: an uneven AMR hierarchy (400 boxes over 3 levels, edges 8-64 per axis, ~8.1M
    cells, a helical reacting shear layer with ~3% stiff cells, per-box dt = 1e-8 / 2^level) in one
    bulk and one persistent stiff launch over the box table, captured once into a CUDA graph and
    replayed every step.  The state is restored from pristine copies and L2 flushed inside every
    timed step; the launch configuration is the one the tuner picked for the config-1 field."""
    mech = synth.h2_air_mechanism(0)
    boxes = synth.amr_boxes(seed=rank)
    fields = synth.helix_box_fields(mech, boxes, seed=rank, stiff_frac=0.03)
    d_boxes, host = [], []
    for bx, (T, p, Y, hot) in zip(boxes, fields):
        T, p, Y = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
        d = {"T": torch.from_numpy(T).to(dev), "p": torch.from_numpy(p).to(dev), "Y": torch.from_numpy(Y).to(dev)}
        d["rho"], d["e"] = torch.empty_like(d["T"]), torch.empty_like(d["T"])
        d["substeps"] = torch.zeros(T.size, dtype=torch.int32, device=dev)
        d["dt"], d["level"] = DT / 2 ** bx["level"], bx["level"]
        d_boxes.append(d)
        host.append((T, p, Y, hot))
    total = sum(h[0].size for h in host)
    ctx = chem.Context(mech, max_cells=total, rtol=args.rtol, atol=args.atol, k_bulk=k_bulk,
                       flags=flags & ~chem.CHEM_FLAG_TIMING)
    for d in d_boxes:
        ctx.state_from_TpY(d["T"], d["p"], d["Y"], d["rho"], d["e"])
    pristine = [(d["T"].clone(), d["Y"].clone()) for d in d_boxes]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream()
    ctx.set_boxes(d_boxes)
    with torch.cuda.stream(stream):
        ctx.capture_boxes(stream)
    torch.cuda.synchronize()

    def step(i):
        with torch.cuda.stream(stream):
            for d, (T0, Y0) in zip(d_boxes, pristine):
                d["T"].copy_(T0)
                d["Y"].copy_(Y0)
            flush.fill_(i & 0xFF)
            ctx.launch_boxes(stream)
        return ctx.status(stream)

    for i in range(args.warmup):
        step(i)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = [step(i) for i in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist)
    for st in stats:
        assert st["status"] == 0, st
    ns, na = mech["ns"], active_species(mech)
    flops = float(np.mean([_stiff_flops(st, ns, na) for st in stats]))
    achieved = flops / (ms / args.steps / 1e3) / 1e12
    # results of the last step, against the oracle on a stratified sample of cells
    cat = lambda xs: np.concatenate(xs, axis=-1)
    T_all, p_all, Y_all, hot_all = (cat([h[k] for h in host]) for k in range(4))
    dts = cat([np.full(h[0].size, d["dt"]) for h, d in zip(host, d_boxes)])
    out_T = cat([d["T"].cpu().numpy() for d in d_boxes])
    out_Y = cat([d["Y"].cpu().numpy() for d in d_boxes])
    acc = _sampled_accuracy(mech, T_all, p_all, Y_all, hot_all, out_T, out_Y, dts, 512, seed=rank)
    ctx.close()
    return {"workload": f"AMR hierarchy: {len(boxes)} boxes over 3 levels (ratio 2, edges 8-64 per axis), "
                        f"{total} cells, helical reacting shear layer ({int(hot_all.sum())} stiff cells), "
                        f"per-box dt = {DT:g} s / 2^level; one bulk + one stiff launch over the box table, "
                        f"replayed as a CUDA graph",
            "cells": int(total), "boxes": len(boxes), "value": total * world * args.steps / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "queued_cells": stats[-1]["nqueued"],
            "substeps_per_stiff_cell": stats[-1]["substeps"] / max(1, stats[-1]["nqueued"]),
            "roofline": {"kernel": "stiff_kernel (whole step timed)", "bound": "alu", "pipe": "fp64",
                         "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                         "note": "algorithmic FP64 flops of the stiff phase over the whole step time (bulk kernel "
                                 "and state restore included), a lower bound of the stiff kernel's rate"},
            "accuracy": acc, "gpu_launches": 3 * args.steps * world,
            "l2": "flushed (256 MiB write) and state restored from pristine copies inside every step"}


def _config3_leg(args, chem, torch, dev, ctx1, rank, world, dist, fp64_peak, gated):
    """Config 3: 16M cells drawn i.i.d. from the AMR shear-layer state distribution (~3% stiff), as a
    flat batch: the plain method against the gated surrogate trained for the config-1 leg (the
    same network, copied into this context)."""
    mech, T, p, Y, hot = _field(seed=rank, config=3, cells=args.cells)
    n = T.size
    ctx = chem.Context(mech, max_cells=n, rtol=args.rtol, atol=args.atol, k_bulk=ctx1.params.k_bulk,
                       flags=ctx1.params.flags & ~chem.CHEM_FLAG_TIMING)
    tT, tp, tY = (torch.from_numpy(a).to(dev) for a in (T, p, Y))
    rho, e = torch.empty_like(tT), torch.empty_like(tT)
    ctx.state_from_TpY(tT, tp, tY, rho, e)
    T0, Y0 = tT.clone(), tY.clone()
    sub = torch.zeros(n, dtype=torch.int32, device=dev)
    acc_mask = torch.zeros(n, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if gated:
        ctx.surrogate_load(ctx1.surrogate_save())

    def run(gate):
        def step(i):
            tT.copy_(T0)
            tY.copy_(Y0)
            flush.fill_(i & 0xFF)
            if gate:
                ctx.advance_gated(tT, tp, tY, rho, e, DT, args.gate_tol, acc_mask, sub)
            else:
                ctx.advance(tT, tp, tY, rho, e, DT, sub)
            return ctx.status()

        for i in range(1):
            step(i)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        stats = [step(i) for i in range(2)]
        ev1.record()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        for st in stats:
            assert st["status"] == 0, st
        return max_over_ranks(ev0.elapsed_time(ev1), dist) / 2, stats[-1]

    dts = np.full(n, DT)
    ms_plain, st_plain = run(False)
    ns, na = mech["ns"], active_species(mech)
    achieved = _stiff_flops(st_plain, ns, na) / (ms_plain / 1e3) / 1e12
    out = {"workload": f"flat batch of {n} cells from the AMR shear-layer state distribution ({int(hot.sum())} "
                       f"stiff), dt = {DT:g} s; plain bulk-sparse vs gated surrogate",
           "cells": n, "plain": {"value": n * world / (ms_plain / 1e3), "unit": UNIT, "ms_per_step": ms_plain,
                                 "queued_cells": st_plain["nqueued"],
                                 "roofline": {"kernel": "stiff_kernel (whole step timed)", "achieved": achieved,
                                              "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak},
                                 "accuracy": _sampled_accuracy(mech, T, p, Y, hot, tT.cpu().numpy(),
                                                               tY.cpu().numpy(), dts, 512, seed=rank)},
           "timing": "1 warm-up + 2 timed steps per leg, state restored and L2 flushed inside each step"}
    if gated:
        ms_g, st_g = run(True)
        out["gated"] = {"value": n * world / (ms_g / 1e3), "unit": UNIT, "ms_per_step": ms_g,
                        "vs_plain": ms_plain / ms_g, "accepted_frac": float(acc_mask.float().mean().item()),
                        "queued_cells": st_g["nqueued"],
                        "accuracy": _sampled_accuracy(mech, T, p, Y, hot, tT.cpu().numpy(), tY.cpu().numpy(), dts,
                                                      512, seed=rank)}
    ctx.close()
    return out


def _config4_leg(args, chem, torch, dev, rank, world, dist, fp64_peak, edge=16, n_sample=32):
    """Config 4 on a reduced sheet (2e x 2e x e cells, 4% reacting, e = 16: 16,384 cells) with the
    53-species mechanism: the plain method (one warp per stiff cell) and the gated surrogate
    (56 inputs, 54 outputs, trained here outside the timed region), each 1 warm-up + 2 timed
    steps, both checked against the oracle on one stratified sample."""
    mech, T, p, Y, hot = _field(seed=rank, edge=edge, config=4)
    n, ns = T.size, mech["ns"]
    ctx = chem.Context(mech, max_cells=max(n, 65536), rtol=args.rtol, atol=args.atol,
                       flags=chem.CHEM_FLAG_TIMING | chem.CHEM_FLAG_ORDER_RATE)
    tT, tp, tY = (torch.from_numpy(a).to(dev) for a in (T, p, Y))
    rho, e = torch.empty_like(tT), torch.empty_like(tT)
    ctx.state_from_TpY(tT, tp, tY, rho, e)
    T0, Y0 = tT.clone(), tY.clone()
    sub = torch.zeros(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(i):
        tT.copy_(T0)
        tY.copy_(Y0)
        flush.fill_(i & 0xFF)
        ctx.advance(tT, tp, tY, rho, e, DT, sub)
        return ctx.status()

    step(0)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    stats = [step(i) for i in range(2)]
    ev1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    for st in stats:
        assert st["status"] == 0, st
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist) / 2
    st = stats[-1]
    na = active_species(mech)
    stiff_ms = float(np.mean([x["stiff_ms"] for x in stats]))
    achieved = _stiff_flops(st, ns, na) / (stiff_ms / 1e3) / 1e12
    dts = np.full(n, DT)
    ref = _sampled_reference(mech, T, p, Y, hot, dts, n_sample, seed=rank)
    out = {"workload": f"reacting sheet {2 * edge}x{2 * edge}x{edge} ({n} cells, 4% reacting), hydrocarbon-shaped "
                       f"mechanism {ns} species / {mech['nr']} reactions, dt = {DT:g} s, one warp per stiff cell",
           "cells": n,
           "plain": {"value": n * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "queued_cells": st["nqueued"],
                     "substeps_per_stiff_cell": st["substeps"] / max(1, st["nqueued"]),
                     "factorizations_per_attempt": st["factorizations"] / max(1, st["attempts"]),
                     "roofline": {"kernel": "stiff_kernel_lg", "bound": "alu", "pipe": "fp64", "achieved": achieved,
                                  "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                                  "kernel_ms": stiff_ms},
                     "accuracy": _sampled_accuracy(mech, T, p, Y, hot, tT.cpu().numpy(), tY.cpu().numpy(), dts,
                                                   n_sample, rank, ref=ref)},
           "timing": "1 warm-up + 2 timed steps per leg, state restored and L2 flushed inside each step"}
    if args.gated:
        leg_args = argparse.Namespace(**{**vars(args), "steps": 2, "warmup": 1})
        g = _gated_leg(leg_args, ctx, chem, torch, dev, mech, step_inputs=(tT, tp, tY, rho, e, sub, T0, Y0, flush),
                       plain_ms=ms, n=n, world=world, dist=dist, rank=rank)
        g["accuracy"] = _sampled_accuracy(mech, T, p, Y, hot, tT.cpu().numpy(), tY.cpu().numpy(), dts,
                                          n_sample, rank, ref=ref)
        out["gated"] = g
    ctx.close()
    return out


def _gated_leg(args, ctx, chem, torch, dev, mech, step_inputs, plain_ms, n, world, dist, rank):
    """The same steps with the learned surrogate in front of the method (chem_advance_gated).  The
    surrogate is trained first, outside the timed region, on pairs that the plain integrator makes
    (FP64-rate mode) from samples over T 300-3200 K, p 1-50 atm, Dirichlet Y, dt 1e-9..1e-6 s."""
    from paper_2510_23993_gb300 import surrogate
    tT, tp, tY, rho, e, sub, T0, Y0, flush = step_inputs
    nbox = 256
    if mech["ns"] == 9:
        m = args.train_pairs // nbox
        recipe = dict(premix_frac=1 / 3, mixing_frac=1 / 3)
        dist_txt = ("T U[300,3200] K, p U[1,50] atm, Y from Dirichlet(0.5), a premix-centred Dirichlet or a fuel/air "
                    "mixing-line Dirichlet (a third each), dt log-U[1e-9,1e-6] s")
    else:
        # 53 species: the stiff integration of a hot sample costs ~1000x a 9-species one, so the
        # network is trained on the states it can take at this accuracy, cold ones (T <= 1200 K:
        # the premix and mixing-line families), around the bench's dt; the gate's training box
        # then keeps every hotter cell on the plain path
        m = min(args.train_pairs, 65536) // nbox
        recipe = dict(premix_frac=0.5, mixing_frac=0.5, T_range=(300.0, 1200.0),
                      log_dt=(np.log(1e-9), np.log(1e-7)))
        dist_txt = ("T U[300,1200] K, p U[1,50] atm, Y from a premix-centred or a fuel/air mixing-line Dirichlet "
                    "(half each), dt log-U[1e-9,1e-7] s")
    Ts, ps, Ys, dts = synth.surrogate_samples(mech, nbox * m, seed=1000 + rank, **recipe)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, Yt, keep = surrogate.make_pairs(ctx, torch.from_numpy(Ts.astype(np.float32)).to(dev),
                                       torch.from_numpy(ps.astype(np.float32)).to(dev),
                                       torch.from_numpy(np.ascontiguousarray(Ys, dtype=np.float32)).to(dev),
                                       dts[:nbox])
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    ctx.surrogate_init(1 + rank)
    t0 = time.perf_counter()
    losses = ctx.surrogate_train(X, Yt, epochs=args.train_epochs, batch=4096, lr=1e-3, err_weight=0.1, seed=rank)
    t_train = time.perf_counter() - t0
    del X, Yt
    acc = torch.zeros(n, dtype=torch.uint8, device=dev)

    def gstep(i):
        tT.copy_(T0)
        tY.copy_(Y0)
        flush.fill_(i & 0xFF)
        ctx.advance_gated(tT, tp, tY, rho, e, DT, args.gate_tol, acc, sub)
        return ctx.status()

    for i in range(args.warmup):
        gstep(i)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    stats = [gstep(i) for i in range(args.steps)]
    ev1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist)
    for s in stats:
        assert s["status"] == 0, s
    accepted = int(acc.sum().item())
    return {"value": n * world * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "vs_plain": plain_ms / (ms / args.steps), "gate_tol": args.gate_tol, "accepted_cells": accepted,
            "accepted_frac": accepted / n, "queued_cells": stats[-1]["nqueued"],
            "gpu_launches": (1 + (5 if ctx.params.flags & chem.CHEM_FLAG_TWO_PASS else 3)) * args.steps * world,
            "train": {"pairs": int(keep.sum().item()), "pairs_s": t_pairs, "epochs": args.train_epochs,
                      "train_s": t_train, "loss_first": losses[0] if losses else None,
                      "loss_last": losses[-1] if losses else None,
                      "distribution": dist_txt + "; targets by the plain integrator at rtol 1e-6 / atol 1e-11"
                                      + (" with FP64 rates" if mech["ns"] == 9 else "")}}


def _paper_loop_leg(args, ctx, chem, torch, step_inputs, plain_ms, n, world, dist):
    """The same steps with the paper's own method (chem_advance_explicit): explicit first-order
    substeps under the bulk_frac change rule (Sec. 2.1), bulk launches of 5 substeps while more
    than 1e4 cells are active, then one sparse launch (Algorithm 3).  The host reads the active
    count after every launch, as the paper does, so the step includes those synchronizations."""
    tT, tp, tY, rho, e, sub, T0, Y0, flush = step_inputs
    plain_frac = ctx.params.bulk_frac
    ctx.set_params(bulk_frac=args.paper_frac)
    launches = []

    def pstep(i):
        tT.copy_(T0)
        tY.copy_(Y0)
        flush.fill_(i & 0xFF)
        launches.append(ctx.advance_explicit(tT, tp, tY, rho, e, DT, sub, k_steps=5, n_star=10000))
        return ctx.status()

    for i in range(args.warmup):
        pstep(i)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches.clear()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    stats = [pstep(i) for i in range(args.steps)]
    ev1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist)
    ctx.set_params(bulk_frac=plain_frac)
    st = stats[-1]
    return {"method": "explicit first-order substeps, |dY_k| <= frac max(|Y_k|, y_floor) (Sec. 2.1), Algorithm 3 "
                      "control: bulk launches of K = 5 substeps while N_active > N* = 1e4, then one sparse launch "
                      "(k_max 1e5)",
            "frac": args.paper_frac, "value": n * world * args.steps / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "vs_plain": plain_ms / (ms / args.steps),
            "bulk_launches": launches[-1], "sparse_cells": st["nqueued"], "failed_cells": st["nfailed"],
            "explicit_substeps": st["substeps"],
            "gpu_launches": sum(2 + nl for nl in launches) * world}


def _accuracy(ctx, torch, dev, T, p, Y, rho, e, T_ref, Y_ref, gate_tol=None, explicit=False, mech=None):
    """Error of the GPU path (plain, gated when gate_tol is given, or the paper's explicit loop)
    against the oracle on the CPU-baseline sample (oracle inputs)."""
    n = T.size
    a = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (T, p, Y, rho, e)]
    s = torch.zeros(n, dtype=torch.int32, device=dev)
    nacc = None
    if explicit:
        ctx.advance_explicit(a[0], a[1], a[2], a[3], a[4], DT, s)
    elif gate_tol is None:
        ctx.advance(a[0], a[1], a[2], a[3], a[4], DT, s)
    else:
        acc = torch.zeros(n, dtype=torch.uint8, device=dev)
        nacc = ctx.advance_gated(a[0], a[1], a[2], a[3], a[4], DT, gate_tol, acc, s)
    ctx.status()
    Tg, Yg = a[0].cpu().numpy().astype(np.float64), a[2].cpu().numpy().astype(np.float64)
    big = Y_ref >= 1e-6
    rel = np.where(big, np.abs(Yg - Y_ref) / np.maximum(Y_ref, 1e-300), 0.0)
    ab = np.where(~big, np.abs(Yg - Y_ref), 0.0)
    eT = np.abs(Tg - T_ref) / T_ref
    over = (rel.max(0) > 1e-4) | (ab.max(0) > 1e-10) | (eT > 1e-4)
    out = {"cells": int(n), "max_rel_Y": float(rel.max()), "p999_rel_Y": float(np.percentile(rel.max(0), 99.9)),
           "max_abs_small_Y": float(ab.max()), "max_rel_T": float(eT.max()), "cells_over_1e-4": int(over.sum())}
    if over.any() and mech is not None:
        # cells over the strict bar: how far the exact solution itself moves when e changes by one
        # FP32 ulp (the FP32 inputs and rate tables perturb the model at that level); a cell whose
        # error stays within the bar plus 3x that response is an ill-conditioned one, not a miss
        import oracle
        idx = np.nonzero(over)[0]
        e_p = np.asarray(e[idx], np.float64) * (1.0 + 2.0 ** -23)
        T_p, _, Y_p, _ = oracle.advance(mech, np.asarray(rho[idx], np.float64), e_p, T[idx], Y[:, idx], DT)
        bigs = big[:, idx]
        dY = np.where(bigs, np.abs(Y_p - Y_ref[:, idx]) / np.maximum(Y_ref[:, idx], 1e-300), np.abs(Y_p - Y_ref[:, idx]))
        dT = np.abs(T_p - T_ref[idx]) / T_ref[idx]
        eY = np.where(bigs, rel[:, idx], ab[:, idx])
        beyond = np.any(eY > np.where(bigs, 1e-4, 1e-10) + 3 * dY, axis=0) | (eT[idx] > 1e-4 + 3 * dT)
        out["over_bar_cells"] = [{"error": float(np.max(eY[:, j])), "oracle_one_ulp_response": float(np.max(dY[:, j])),
                                  "T_out": float(Tg[idx[j]])} for j in range(min(len(idx), 8))]
        out["cells_over_1e-4_beyond_conditioning"] = int(beyond.sum())
    elif not over.any():
        out["cells_over_1e-4_beyond_conditioning"] = 0
    if nacc is not None:
        out["accepted_in_sample"] = int(nacc)
    return out


def _traffic():
    """DRAM bytes of the stiff phase per step (its one or two stiff-kernel launches) from the
    committed ncu summary, if that was taken on the current source of the kernel (else null)."""
    path = os.path.join(ROOT, "profiles", "stiff_phase_traffic_sheet128.txt")
    if not os.path.exists(path):
        return None
    rec = dict(line.split(":", 1) for line in open(path).read().splitlines() if ":" in line)
    src = os.path.join(ROOT, "paper_2510_23993_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("stiff.cu", "stiff_body.cuh", "chem_device.cuh", "kernel_abi.cuh"):
        h.update(open(os.path.join(src, f), "rb").read())
    if rec.get("source_sha256", "").strip() != h.hexdigest():
        return None
    return float(rec["dram_bytes_per_step"])


def run_reference(args, world):
    mech, T, p, Y, hot = _field(seed=0, edge=args.edge, config=args.config, cells=args.cells)
    walls, ncell = [], 0
    for i in range(args.warmup + args.steps):
        idx, _, _, _, _, wall, cores = _oracle_sample(mech, T, p, Y, hot,
                                                      args.ref_sample if args.config == 1 else min(args.ref_sample, 256),
                                                      seed=i)
        if i >= args.warmup:
            walls.append(wall)
            ncell += len(idx)
    total = sum(walls)
    value = ncell / total
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(T.size, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{ncell // max(1, args.steps)} cells per step, stratified "
                                       f"({int(hot.mean() * 100 + 0.5)}% reacting) from the field of "
                                       f"{T.size} cells; FP64 Radau IIA rtol 1e-10"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _time_ms(fn, reps, torch):
    """Median CUDA-event time of fn() over reps calls (after one warm-up call)."""
    fn()
    out = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return float(np.median(out))


def run_study(args):
    """Comparisons with the paper's baseline strategies (one JSON line per measurement):
      rates:  the multi-kernel cuBLAS rate evaluation (chem_mk_rates) against the fused kernel
              (chem_rates) and, for 53 species, the tensor-core kernel (chem_rates_tc), one grid
              of n cells (App. C) and 1M cells split into G grids, one launch sequence per grid
              (Sec. 3.2.1, App. E), for the 9- and 53-species mechanisms;
      fusion: one chemistry step of 1M cells split into G boxes, advanced box by box
              (chem_advance per box) against one fused launch over the box table (graph replay);
      layout: the state load (chem_pressure_layout) from ~1.5 GiB of records in each storage
              layout, in HBM GB/s."""
    import torch
    import paper_2510_23993_gb300 as chem
    chem.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    if args.study == "layout":
        peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
        hbm = json.load(open(peaks)).get("hbm_gbs") if os.path.exists(peaks) else None
        names = {chem.CHEM_LAYOUT_SOA: "SoA (component-major)", chem.CHEM_LAYOUT_AOS: "AoS (cell-major)",
                 chem.CHEM_LAYOUT_AOSOA: "AoSoA (32-cell tiles)", chem.CHEM_LAYOUT_AOS_STAGED: "AoS staged in shared memory"}
        for label, mech in (("9 species", synth.h2_air_mechanism(0)), ("53 species", synth.hydrocarbon_mechanism(0))):
            ns = mech["ns"]
            nv = ns + 2
            n = (1536 << 20) // (4 * nv) // 128 * 128      # ~1.5 GiB of records, far above L2
            X = torch.rand(n * nv, dtype=torch.float32, device=dev) + 0.5
            p = torch.empty(n, dtype=torch.float32, device=dev)
            for layout, nm in names.items():
                ms = _time_ms(lambda: chem.pressure_layout(mech["W"], layout, X, n, p, ld=n), args.steps, torch)
                gbs = n * (nv + 1) * 4 / (ms / 1e3) / 1e9
                print(json.dumps({"study": "layout", "mechanism": label, "layout": nm, "cells": n,
                                  "bytes_per_cell": (nv + 1) * 4, "ms": ms, "GB_s": gbs,
                                  "frac_of_measured_hbm": gbs / hbm if hbm else None}), flush=True)
            del X, p
        return
    if args.study == "tail":
        # the stiff phase's critical path: the distribution of substeps per stiff cell on the
        # benchmark sheet, then the cells with the most substeps integrated alone (--tail-top
        # sizes, 0 = none), so that the time of the longest cell can be set against the phase
        mech = synth.h2_air_mechanism(0)
        T, p, Y, hot = synth.sheet_field(mech, n=args.edge, seed=0)
        T, p, Y = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
        ctx = chem.Context(mech, max_cells=T.size)
        tT, tp, tY = (torch.from_numpy(a).to(dev) for a in (T, p, Y))
        trho, te = torch.empty_like(tT), torch.empty_like(tT)
        ctx.state_from_TpY(tT, tp, tY, trho, te)
        rho, e = trho.cpu().numpy(), te.cpu().numpy()

        def run(idx, flags):
            ctx.set_params(flags=chem.CHEM_FLAG_TIMING | flags)
            d = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (T[idx], p[idx], Y[:, idx], rho[idx], e[idx])]
            sub = torch.zeros(len(idx), dtype=torch.int32, device=dev)
            ctx.advance(d[0], d[1], d[2], d[3], d[4], 1e-8, sub)
            return sub.cpu().numpy(), ctx.status()

        order = chem.CHEM_FLAG_TWO_PASS | chem.CHEM_FLAG_ORDER_RATE
        sub, st = run(np.arange(T.size), order)
        q = sub[hot]
        print(json.dumps({"study": "tail", "cells": int(T.size), "stiff_cells": int(st["nqueued"]),
                          "stiff_ms": st["stiff_ms"], "substeps_pct_50_90_99_999": np.percentile(q, [50, 90, 99, 99.9]).tolist(),
                          "substeps_max": int(q.max())}), flush=True)
        top = np.argsort(-sub)
        for k in [int(x) for x in args.tail_top.split(",") if int(x) > 0]:
            idx = np.sort(top[:k])
            s2, st2 = run(idx, order if k > 1 else 0)
            print(json.dumps({"study": "tail_alone", "cells": k, "stiff_ms": st2["stiff_ms"],
                              "substeps_max": int(s2.max()),
                              "us_per_substep_of_longest": 1e3 * st2["stiff_ms"] / max(1, int(s2.max()))}), flush=True)
        ctx.close()
        return
    if args.study == "rates_tc":
        # one size (--cells) of the 53-species rates: tensor-core kernel, warp-per-cell kernel and
        # the cuBLAS sequence on the same inputs (inputs above L2 at the default size)
        mech = synth.hydrocarbon_mechanism(0)
        N = args.cells if args.cells != 16_000_000 else 1 << 20
        rng = np.random.default_rng(0)
        T = rng.uniform(800, 3000, N).astype(np.float32)
        p = (rng.uniform(1, 20, N) * synth.P_ATM).astype(np.float32)
        Y = np.ascontiguousarray(rng.dirichlet(np.full(mech["ns"], 0.3), size=N).T, dtype=np.float32)
        ctx = chem.Context(mech, max_cells=N)
        mk = chem.MultiKernelRates(mech, max_cells=N)
        tT, tp, tY = (torch.from_numpy(a).to(dev) for a in (T, p, Y))
        rho, e = torch.empty_like(tT), torch.empty_like(tT)
        ctx.state_from_TpY(tT, tp, tY, rho, e)
        f = torch.empty_like(tY)
        t_c = _time_ms(lambda: ctx.rates_tc(rho, tT, tY, f), args.steps, torch)
        t_f = _time_ms(lambda: ctx.rates(rho, tT, tY, f), args.steps, torch)
        t_m = _time_ms(lambda: mk.rates(rho, tT, tY, f), args.steps, torch)
        hbm = (2 * mech["ns"] + 2) * 4 * N      # Y read, dY/dt written, rho and T read
        # tensor-core work as issued: K padded to 64 species, N to 336 reactions, three BF16 parts
        # of each FP32 operand (six split pairs for the efficiencies)
        nrp, ntb = 336, 32
        issued = N * (2 * 64 * ntb * 6 + 2 * 3 * 2 * 64 * nrp + 3 * 2 * nrp * 64)
        peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
        pk = json.load(open(peaks)) if os.path.exists(peaks) else {}
        tf = issued / (t_c / 1e3) / 1e12
        gbs = hbm / (t_c / 1e3) / 1e9
        print(json.dumps({"study": "rates_tc", "mechanism": "53 species / 325 reactions", "cells": N,
                          "tensor_core_ms": t_c, "fused_ms": t_f, "multikernel_ms": t_m,
                          "tensor_core_cells_per_s": N / (t_c / 1e3), "fused_over_tensor_core": t_f / t_c,
                          "multikernel_over_tensor_core": t_m / t_c,
                          "tensor_issued_TFLOP_s": tf,
                          "frac_of_measured_bf16": tf / pk["bf16_tflops"] if pk.get("bf16_tflops") else None,
                          "tensor_core_hbm_GB_s": gbs,
                          "frac_of_measured_hbm": gbs / pk["hbm_gbs"] if pk.get("hbm_gbs") else None}), flush=True)
        mk.close()
        ctx.close()
        return
    if args.study == "rates":
        for name, mech in (("9 species / 21 reactions", synth.h2_air_mechanism(0)),
                           ("53 species / 325 reactions", synth.hydrocarbon_mechanism(0))):
            N = 1 << 20
            rng = np.random.default_rng(0)
            T = rng.uniform(800, 3000, N).astype(np.float32)
            p = (rng.uniform(1, 20, N) * synth.P_ATM).astype(np.float32)
            Y = np.ascontiguousarray(rng.dirichlet(np.full(mech["ns"], 0.3), size=N).T, dtype=np.float32)
            ctx = chem.Context(mech, max_cells=N)
            mk = chem.MultiKernelRates(mech, max_cells=N)
            tT, tp, tY = (torch.from_numpy(a).to(dev) for a in (T, p, Y))
            rho, e = torch.empty_like(tT), torch.empty_like(tT)
            ctx.state_from_TpY(tT, tp, tY, rho, e)
            f = torch.empty_like(tY)
            for n in (1000, 10000, 100000, N):
                Ys = tY[:, :n].contiguous()
                fs = f[:, :n].contiguous()
                t_f = _time_ms(lambda: ctx.rates(rho[:n], tT[:n], Ys, fs), args.steps, torch)
                t_m = _time_ms(lambda: mk.rates(rho[:n], tT[:n], Ys, fs), args.steps, torch)
                line = {"study": "rates_one_grid", "mechanism": name, "cells": n, "fused_ms": t_f,
                        "multikernel_ms": t_m, "multikernel_over_fused": t_m / t_f}
                if mech["ns"] == 53:   # the stoichiometric contractions on the tensor cores
                    t_c = _time_ms(lambda: ctx.rates_tc(rho[:n], tT[:n], Ys, fs), args.steps, torch)
                    line.update(tensor_core_ms=t_c, multikernel_over_tensor_core=t_m / t_c,
                                tensor_core_cells_per_s=n / (t_c / 1e3))
                print(json.dumps(line), flush=True)
            for G in (1, 15, 150, 1000):
                off = np.linspace(0, N, G + 1).astype(np.int64)

                def per_grid():
                    for g in range(G):
                        a, b = int(off[g]), int(off[g + 1])
                        mk.rates(rho[a:], tT[a:], tY[:, a:], f[:, a:], n=b - a)

                t_m = _time_ms(per_grid, args.steps, torch)
                t_f = _time_ms(lambda: chem.chem_rates(ctx.handle, rho, tT, tY, N, N, f), args.steps, torch)
                print(json.dumps({"study": "rates_grids", "mechanism": name, "cells": N, "grids": G,
                                  "fused_one_launch_ms": t_f, "multikernel_per_grid_ms": t_m,
                                  "launches_multikernel": G * (5 if mech["third_body"].any() else 4),
                                  "multikernel_over_fused": t_m / t_f}), flush=True)
            mk.close()
            ctx.close()
    else:   # fusion of the whole chemistry step across boxes
        mech = synth.h2_air_mechanism(0)
        T, p, Y, hot = synth.sheet_field(mech, n=100, seed=0)
        T, p, Y = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
        N = T.size
        ctx = chem.Context(mech, max_cells=N)
        tT, tp, tY = (torch.from_numpy(a).to(dev) for a in (T, p, Y))
        rho, e = torch.empty_like(tT), torch.empty_like(tT)
        ctx.state_from_TpY(tT, tp, tY, rho, e)
        T0, Y0 = tT.clone(), tY.clone()
        sub = torch.zeros(N, dtype=torch.int32, device=dev)
        stream = torch.cuda.Stream()
        for G in (1, 15, 150, 1000):
            off = np.linspace(0, N, G + 1).astype(np.int64)
            boxes = [dict(T=tT[a:b], p=tp[a:b], Y=tY[:, a:b], rho=rho[a:b], e=e[a:b], substeps=sub[a:b], dt=DT,
                          level=0) for a, b in zip(off[:-1], off[1:])]

            def per_box():
                tT.copy_(T0)
                tY.copy_(Y0)
                for bx in boxes:
                    n = bx["T"].shape[0]
                    chem._check(chem.chem_advance(ctx.handle, bx["T"], bx["p"], bx["Y"], N, bx["rho"], bx["e"], n, DT,
                                                  bx["substeps"]), "chem_advance")

            t_b = _time_ms(per_box, max(2, args.steps // 2), torch)
            ctx.set_boxes(boxes)
            with torch.cuda.stream(stream):
                tT.copy_(T0)
                tY.copy_(Y0)
                ctx.capture_boxes(stream)
            torch.cuda.synchronize()

            def fused():
                with torch.cuda.stream(stream):
                    tT.copy_(T0)
                    tY.copy_(Y0)
                    ctx.launch_boxes(stream)
                stream.synchronize()

            t_f = _time_ms(fused, max(2, args.steps // 2), torch)
            print(json.dumps({"study": "step_boxes", "cells": N, "boxes": G, "per_box_calls_ms": t_b,
                              "fused_graph_ms": t_f, "per_box_over_fused": t_b / t_f,
                              "field": "reacting sheet 100^3, 5% reacting, dt 1e-8 s, boxes = equal slabs"}),
                  flush=True)
        ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--edge", type=int, default=N_EDGE, help="field edge (cells); 128 is the benchmark size")
    ap.add_argument("--config", type=int, default=1, choices=[1, 3, 4],
                    help="1: 9-species sheet (the benchmark); 3: flat batch from the AMR state distribution "
                         "(--cells), plain vs gated; 4: 53-species sheet of 2e x 2e x e cells")
    ap.add_argument("--cells", type=int, default=16_000_000, help="cells of the --config 3 batch")
    ap.add_argument("--rtol", type=float, default=1e-5)
    ap.add_argument("--atol", type=float, default=1e-10)
    ap.add_argument("--cpu-sample", type=int, default=65536)
    ap.add_argument("--ref-sample", type=int, default=8192)
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--tune-cache", default=None)
    ap.add_argument("--fp64-rates", action="store_true", help="stiff-cell rates in FP64 (CHEM_FLAG_FP64_RATES)")
    ap.add_argument("--two-pass", action="store_true", help="two-pass stiff schedule without tuning (the tuner "
                                                              "chooses it otherwise)")
    ap.add_argument("--no-gated", dest="gated", action="store_false", help="skip the gated-surrogate leg")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the config-2 (AMR boxes, graph replay) and config-3 (16M-cell batch) objects")
    ap.add_argument("--gate-tol", type=float, default=1e-5)
    ap.add_argument("--no-paper-loop", dest="paper_loop", action="store_false",
                    help="skip the leg that times the paper's explicit scheme under Algorithm 3")
    ap.add_argument("--paper-frac", type=float, default=0.05, help="relative change limit of the explicit scheme")
    ap.add_argument("--train-pairs", type=int, default=262144)
    ap.add_argument("--train-epochs", type=int, default=40)
    ap.add_argument("--tail-top", default="1,256,19456", help="--study tail: sizes of the longest-cell sets run alone")
    ap.add_argument("--study", default=None, choices=["rates", "rates_tc", "tail", "fusion", "layout"],
                    help="instead of the benchmark line: the comparisons with the paper's baseline strategies")
    args = ap.parse_args()
    if args.study:
        run_study(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, world)), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    line = run_gpu(args, rank, world, local_rank, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
