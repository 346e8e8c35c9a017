#!/usr/bin/env python
"""Benchmark of the GRMHD block update on GB300: zone-cycles per second.

Workload (default): one 256 x 128 x 64 block of the magnetised Fishbone-Moncrief
torus (Kerr-Schild a = 0.9375, r = 1.2..50 r_g log-spaced, theta 0..pi,
phi 0..2pi, Gamma = 13/9, loop field with max p_g / max p_b = 100, 2% seeded
u_g perturbation, seed 10192), FP64, PPM + HLL + CT + Newton inversion,
midpoint step at the CFL time step (C0 = 0.8). A zone-cycle is one cell
advanced one full step, predictor plus corrector (the paper's Sec. 5.3
definition). The state (~1.4 GB with scratch) is far larger than the 129 MB
L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own copy of the block (the
single block does not shard; replicas, weak scaling); value = all ranks'
zone-cycles / the slowest rank's time. `--impl reference` times the CPU
oracle (the plain FP64 implementation the CUDA path is checked against) on
the host cores, rank 0 only.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N1, N2, N3 = 256, 128, 64
SEED = 10192
METRIC = "zone-cycles/sec on 1 GB300 (plain FP64 vs chosen form at stated L1 error), % HBM roofline"
WORKLOAD = "FM torus block 256x128x64, Kerr-Schild a=0.9375, r 1.2-50, loop field beta=100, seed 10192, FP64"

# Algorithmic FP64 operations per unit of work, from the flop-counting CPU
# oracle on the 64x32x16 torus (tests/golden/make_flop_counts.py writes them;
# tests/test_bench_constants.py checks these copies against it).
FLOPS_PER_FACE = 318.09          # one HLL face flux from given edge states
FLOPS_PER_RECON_CELL = 105.18    # one cell's edge values (and a third of its kappa), one direction
FLOPS_PER_UPDATE_CELL = 694.5    # one cell: U, div F, source, inversion, floors (per stage)
FLOPS_PER_ZONE_CYCLE = 4605.0    # one cell, one full step
# Peaks. FP64: nominal GB300 rate (the profiling recipe's 1.25 TFLOP/s); the
# FMA rate measured by hamr_measure_fp64_peak is reported beside it.
FP64_NOMINAL_TFLOPS = 1.25
# DRAM bytes per launch of the dominant kernel group, from one ncu capture
# of this build's x1-face flux kernel (the x2 and x3 kernels move the same
# field sizes): 312.5 MB read + 115.4 MB written.
NCU_TRAFFIC_PER_LAUNCH = 427.9e6


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x, dist, device="cuda"):
    """The slowest rank's value of x (the job's time): an all-reduce MAX over the ranks of the process
    group (x itself on one rank). Every rank gets the result."""
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds_max):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / seconds_max


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def torus_inputs(n1=N1, n2=N2, n3=N3, seed=SEED):
    from paper_1912_10192_gb300 import workloads as W
    geo = W.torus_geometry(n1, n2, n3)
    prim, bf = W.torus_block(geo, seed=seed)
    return geo, prim, bf


TORUS_BC = (3, 3, 2, 2, 1, 1)  # no-inflow radial, polar axis, periodic phi


def cpu_oracle_rate(n1, n2, n3, steps, warmup, seed=SEED):
    """Oracle zone-cycles/s on a torus block (single thread)."""
    import oracle as O
    geo, prim, bf = torus_inputs(n1, n2, n3, seed)
    d = O.make_desc(n1, n2, n3, geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3, metric=O.METRIC_KS,
                    a=0.9375, gam=13.0 / 9.0, cour=0.8, bc=TORUS_BC)
    g = O.Grid(d)
    g.set(prim, bf)
    for _ in range(warmup):
        g.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        g.step()
    t = time.perf_counter() - t0
    return n1 * n2 * n3 * steps / t, t


def _oracle_worker(n, steps, barrier, out, idx):
    """One process of the all-cores CPU baseline: its own copy of an n[0] x n[1] x n[2] torus block."""
    sys.path.insert(0, ROOT)
    import oracle as O
    geo, prim, bf = torus_inputs(*n)
    d = O.make_desc(n[0], n[1], n[2], geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3,
                    metric=O.METRIC_KS, a=0.9375, gam=13.0 / 9.0, cour=0.8, bc=TORUS_BC)
    g = O.Grid(d)
    g.set(prim, bf)
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        g.step()
    out[idx] = time.perf_counter() - t0


def host_cpu():
    """nproc and the lscpu lines that name the host's cores."""
    info = {"nproc": os.cpu_count()}
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Architecture", "Model name", "CPU(s)", "Thread(s) per core", "Core(s) per socket",
                             "Socket(s)", "CPU max MHz"):
                info[k.strip()] = v.strip()
    except (OSError, subprocess.SubprocessError):
        info["lscpu"] = "unavailable"
    return info


def cpu_oracle_all_cores(n=(128, 64, 32), steps=2, procs=None):
    """Whole-host oracle rate: one single-threaded oracle process per core, each stepping its own copy of
    a torus block (independent blocks, the way the paper's CPU code spreads blocks over cores), started
    together; zone-cycles of all processes / the slowest process's time. Processes are spawned (fresh
    interpreters, no CUDA state inherited)."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    out = ctx.Array("d", procs)
    ps = [ctx.Process(target=_oracle_worker, args=(n, steps, barrier, out, i)) for i in range(procs)]
    for q in ps:
        q.start()
    for q in ps:
        q.join()
    t = max(out[:])
    return procs * n[0] * n[1] * n[2] * steps / t, t, procs


def run_reference(args, rank, world):
    if rank != 0:
        return
    n1, n2, n3 = 64, 32, 16
    rate, t = cpu_oracle_rate(n1, n2, n3, args.steps, args.warmup)
    sample = ("CPU oracle (plain FP64 C++, 1 thread), torus block %dx%dx%d (the benchmark's setup at 1/64 of "
              "its cells), %d timed steps after %d warm-up" % (n1, n2, n3, args.steps, args.warmup))
    line = {"metric": METRIC, "value": rate, "unit": "zone-cycles/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "%dx%dx%d" % (n1, n2, n3)}, "impl": "reference",
            "cpu_baseline": {"value": rate, "unit": "zone-cycles/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": "zone-cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def field_l1(pa, ba, pr, br):
    """Relative L1 per primitive field over the interior (utilde and face B as one field each)."""
    ng = 3
    sl = (slice(ng, ng + N3), slice(ng, ng + N2), slice(ng, ng + N1))

    def l1(vs, a, r):
        return float(sum(np.abs(a[v][sl] - r[v][sl]).sum() for v in vs) / sum(np.abs(r[v][sl]).sum() for v in vs))
    fa = [ba[0][ng:ng + N3, ng:ng + N2, ng:ng + N1 + 1], ba[1][ng:ng + N3, ng:ng + N2 + 1, ng:ng + N1],
          ba[2][ng:ng + N3 + 1, ng:ng + N2, ng:ng + N1]]
    fr = [br[0][ng:ng + N3, ng:ng + N2, ng:ng + N1 + 1], br[1][ng:ng + N3, ng:ng + N2 + 1, ng:ng + N1],
          br[2][ng:ng + N3 + 1, ng:ng + N2, ng:ng + N1]]
    return {"rho": l1((0,), pa, pr), "u": l1((1,), pa, pr), "utilde": l1((2, 3, 4), pa, pr),
            "Bface": float(sum(np.abs(x - y).sum() for x, y in zip(fa, fr)) / sum(np.abs(y).sum() for y in fr))}


def mixed_leg(args, hamr, torch, blk, dprim, dbf, g64, stream, cells, world, dist, precision=None):
    """Times a mixed-precision form on the benchmark workload (same protocol as
    the FP64 leg) and states its relative L1 error per field against the FP64
    state after the same number of steps from the same initial state."""
    precision = hamr.PREC_MIXED if precision is None else precision
    gm = hamr.Grid([blk], precision=precision)
    gm.set_state(dprim, dbf, stream=stream)
    for _ in range(args.warmup):
        gm.step(stream=stream)
    torch.cuda.synchronize()
    gm.set_timing(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        gm.step(stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    timing = gm.timing()
    gm.set_timing(False)
    ms_max = max_over_ranks(ms, dist)
    pm, bm = gm.get_state()
    p64, b64 = g64.get_state()
    gm.close()
    form = ("mixed: FP32 reconstruction, face fluxes, edge EMFs and connection source; FP64 metric, U^n, "
            "update and CT curl; Newton iterates in FP32 until a step is below 1e-5 W, then in FP64"
            if precision == hamr.PREC_MIXED else
            "mixed, FP64 inversion: FP32 reconstruction, face fluxes and edge EMFs; FP64 metric, U^n, update, "
            "connection source, CT curl and every Newton iteration")
    return {"form": form, "precision": int(precision),
            "value": job_rate(cells * args.steps, world, ms_max * 1e-3), "unit": "zone-cycles/s",
            "ms_per_step": ms_max / args.steps, "dtype": "f32+f64",
            "l1_vs_fp64": dict(field_l1(pm, bm, p64, b64), steps=args.warmup + args.steps),
            "kernel_ms": {k: round(v[1], 3) for k, v in timing.items()},
            "gpu_launches": int(sum(v[0] for k, v in timing.items() if k != "load"))}


def train_network(hamr, torch, n=10_000_000, nspin=10, steps=6000, seed=5):
    """The learned inversion guess, trained on the device: n random states (rho log-uniform 1e-6..1,
    u/rho 1e-4..1e2, Lorentz factor 1..50, sigma 0..100, r 0.9 r_+..100; nspin spins drawn from
    0..0.99), conserved variables and inputs formed by the library, then Adam on the training kernels."""
    from paper_1912_10192_gb300 import workloads as W
    t0 = time.perf_counter()
    spins = 0.99 * W.uniform01(seed + 1000, np.arange(nspin))
    feats, targs = [], []
    for k in range(nspin):
        pr, x1, x2 = W.random_states(n // nspin, seed=seed * 100 + k, a=float(spins[k]))
        P = torch.from_numpy(np.ascontiguousarray(pr.T)).cuda()
        X1, X2 = torch.from_numpy(x1).cuda(), torch.from_numpy(x2).cuda()
        U = torch.empty((6, len(x1)), dtype=torch.float64, device="cuda")
        hamr.prim2cons(P, X1, X2, U, a=float(spins[k]), gam=13.0 / 9.0)
        f = torch.empty((10, len(x1)), dtype=torch.float32, device="cuda")
        t = torch.empty((2, len(x1)), dtype=torch.float32, device="cuda")
        hamr.Mlp.features(U, P[5:8].contiguous(), X1, X2, f, prim=P, targ=t, a=float(spins[k]), gam=13.0 / 9.0)
        feats.append(f)
        targs.append(t)
    feat, targ = torch.cat(feats, 1).contiguous(), torch.cat(targs, 1).contiguous()
    del feats, targs
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    m = hamr.Mlp(seed=7)
    m.fit_norm(feat, targ)
    loss = m.train(feat, targ, steps=steps, batch=8192)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    info = {"pairs": n, "spins": nspin, "steps": steps, "batch": 8192, "data_s": round(t1 - t0, 2),
            "train_s": round(t2 - t1, 2), "loss_first": float(loss[:20].mean()), "loss_last": float(loss[-20:].mean())}
    return m, info


def mlp_leg(args, hamr, torch, blk, dprim, dbf, cells, stream):
    """The benchmark workload with the network attached to the inversions, both modes, against the plain
    start: zone-cycles/s, Newton iterations per inversion, entropy inversions."""
    m, info = train_network(hamr, torch)
    out = {"training": info}
    for name, mode in (("plain", None), ("rescue", hamr.MLP_RESCUE), ("first", hamr.MLP_FIRST)):
        g = hamr.Grid([blk])
        g.set_state(dprim, dbf, stream=stream)
        if mode is not None:
            g.set_mlp(m, mode)
        for _ in range(args.warmup):
            g.step(stream=stream)
        torch.cuda.synchronize()
        steps = min(args.steps, 20)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            g.step(stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        tot = dict(c2p_ok=0, c2p_entropy=0, c2p_fail=0, newton_iters=0)
        for _ in range(2):  # counters of single steps (stats synchronise)
            st = g.step(stream=stream, stats=True)
            for k in tot:
                tot[k] += st[k]
        ninv = tot["c2p_ok"] + tot["c2p_entropy"] + tot["c2p_fail"]
        out[name] = {"value": cells / (ms * 1e-3), "ms_per_step": ms,
                     "newton_iters_per_inversion": tot["newton_iters"] / max(ninv, 1),
                     "entropy_per_step": tot["c2p_entropy"] / 2, "fail_per_step": tot["c2p_fail"] / 2}
        g.close()
    out["inversion_variants"] = inversion_variants(hamr, torch, m)
    out["network_error_flag"] = m.error_flag()
    m.close()
    return out


def inversion_variants(hamr, torch, m, n=1_000_000, seed=6):
    """The energy inversions side by side on n random states (the validation law of the network) from a
    warm start (the true state perturbed by 5%) and a cold one (rho at rest with u = 1e-3 rho): Newton,
    the Aitken-accelerated pressure iteration, and Newton from the network's start. Fractions of energy /
    entropy / failed inversions, iterations per energy inversion (map evaluations for Aitken), and the
    device time of the call."""
    from paper_1912_10192_gb300 import workloads as W
    pr, x1, x2 = W.random_states(n, seed=seed)
    P = torch.from_numpy(np.ascontiguousarray(pr.T)).cuda()
    X1, X2 = torch.from_numpy(x1).cuda(), torch.from_numpy(x2).cuda()
    U = torch.empty((6, n), dtype=torch.float64, device="cuda")
    hamr.prim2cons(P, X1, X2, U, a=0.9375, gam=13.0 / 9.0)
    B = P[5:8].contiguous()
    starts = {"warm": P.clone(), "cold": P.clone()}
    starts["warm"][0] *= 1.05
    starts["warm"][1] *= 0.95
    starts["warm"][2:5] *= 1.02
    starts["cold"][1] = 1e-3 * starts["cold"][0]
    starts["cold"][2:5] = 0.0
    out = {"states": n}
    # the start's distance from the answer at which the network's start begins to pay: the true state
    # perturbed by a relative eps (rho up, u_g down, velocity up), Newton from it against Newton from the
    # network (which does not see the start)
    sweep = {}
    for eps in (1e-4, 1e-3, 1e-2, 5e-2, 2e-1):
        guess = P.clone()
        guess[0] *= 1.0 + eps
        guess[1] *= 1.0 - eps
        guess[2:5] *= 1.0 + 0.4 * eps
        row = {}
        for vname, mlp in (("newton", None), ("network_first", m)):
            st = torch.zeros(n, dtype=torch.int32, device="cuda")
            it = torch.zeros(n, dtype=torch.int32, device="cuda")
            hamr.con2prim(U, B, X1, X2, guess.clone(), st, it, mlp=mlp)
            ok = st == 0
            row[vname] = {"iters_per_energy_inversion": float(it[ok].float().mean()) if bool(ok.any()) else None,
                          "not_energy": float((st != 0).float().mean())}
        sweep["%g" % eps] = row
    out["start_distance_sweep"] = sweep
    for sname, guess in starts.items():
        for vname, flags, mlp in (("newton", 0, None), ("aitken", hamr.C2P_AITKEN, None), ("network_first", 0, m)):
            st = torch.zeros(n, dtype=torch.int32, device="cuda")
            it = torch.zeros(n, dtype=torch.int32, device="cuda")
            hamr.con2prim(U, B, X1, X2, guess.clone(), st, it, flags=flags, mlp=mlp)  # warm-up
            work = guess.clone()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            hamr.con2prim(U, B, X1, X2, work, st, it, flags=flags, mlp=mlp)
            e1.record()
            torch.cuda.synchronize()
            ok = st == 0
            out["%s_%s" % (sname, vname)] = {
                "energy": float(ok.float().mean()), "entropy": float((st == 1).float().mean()),
                "failed": float((st == 2).float().mean()),
                "iters_per_energy_inversion": float(it[ok].float().mean()) if bool(ok.any()) else None,
                "ms": round(e0.elapsed_time(e1), 3)}
    return out


def options_leg(args, hamr, torch, blk, dprim, dbf, cells, stream):
    """The benchmark workload with each option of the step switched on alone (FP64): upwinded EMFs, the
    PPM shock flattener, the Aitken inversion, floors in the drift frame, two levels of internal SMR;
    zone-cycles/s, ms/step and the CFL step after the timed steps (internal SMR buys time step, not
    zone-cycles)."""
    out = {}
    for name, kw in (("plain", {}), ("emf_upwind", {"emf": hamr.EMF_UPWIND}), ("flatten", {"flatten": 1}),
                     ("aitken_inversion", {"inversion": hamr.INV_AITKEN}),
                     ("drift_floors", {"floor_frame": hamr.FLOOR_DRIFT}),
                     ("internal_smr_2", {"smr": 2})):
        g = hamr.Grid([blk], **kw)
        g.set_state(dprim, dbf, stream=stream)
        for _ in range(args.warmup):
            g.step(stream=stream)
        torch.cuda.synchronize()
        steps = min(args.steps, 20)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            g.step(stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        st = g.step(stream=stream, stats=True)
        out[name] = {"value": cells / (ms * 1e-3), "ms_per_step": round(ms, 3), "dt_next": st["dt_next"],
                     "entropy_per_step": st["c2p_entropy"], "floor_hits_per_step": st["floor_hits"],
                     "iters_per_inversion": st["newton_iters"] / max(st["c2p_ok"] + st["c2p_entropy"] +
                                                                       st["c2p_fail"], 1)}
        g.close()
    return out


SHAPE_KEYS = ("recon_seg", "recon_x1_sweep", "bs_recon", "bs_flux", "bs_update")


def amr_leg(hamr, torch, precision=0, tune=True, nper=3, reps=2, smr=0):
    """The 512-block C3 torus tree (two refinement levels, 6-way polar children, LAT levels 0..3),
    whole LAT periods replayed from one CUDA graph. Every timing starts from the same initial state
    (restored), runs one untimed period (graph capture) and times nper periods. With tune: the
    autotuner runs on a representative state, then the default and the tuned launch shapes are timed
    alternately, reps times each, from the same initial state; the tuned shapes are used only if their
    median beats the default's by more than the spread of the repetitions. tune=False times the
    default shapes only. smr > 0 adds that many levels of internal SMR in the polar rows (Sec. 3.3.2),
    which lifts the CFL step of the polar blocks; the simulated time per period (the CFL fine step
    of the last timed period x 2^lmax) and per wall-clock second show what that buys."""
    from paper_1912_10192_gb300 import workloads as W
    blocks = W.c3_tree(n=32, smr=smr)
    states = W.torus_blocks(blocks, seed=3)
    g = hamr.Grid([hamr.block_from_dict(b) for b in blocks], precision=precision, smr=smr)
    lmax = max(b["lat"] for b in blocks)
    per = 2 ** lmax

    def restore():
        for i, (p, bf) in enumerate(states):
            g.set_state(p, bf, block=i)

    def time_periods():
        restore()
        g.batch_step(per)  # capture (after any change of launch shapes) + one period
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        g.batch_step(per * nper)
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / nper
    summary = W.tree_summary(blocks)
    real = sum(b["n1"] * b["n2"] * b["n3"] * 2 ** (lmax - b["lat"]) for b in blocks)
    eff = summary["cells"] * per
    base = {"workload": "C3: 512-block torus tree (8x4x4 base of 32^3, 16 disk blocks to level 1, 16 of those "
                        "to level 2, 32 polar blocks split 6-way, polar rows derefined in phi), %d cells, "
                        "1024x512x512 effective, seed 3" % summary["cells"],
            "precision": "mixed" if precision else "fp64", "internal_smr_levels": smr, "tree": summary,
            "fine_substeps_per_period": per, "real_zone_cycles_per_period": real}

    def sim_time(ms):  # the CFL fine step of the last period timed
        t = g.stats()["dt_used"] * per
        return {"sim_time_per_period": t, "sim_time_per_s": t / (ms * 1e-3)}
    default = g.launch_shapes()
    default = {k: default[k] for k in SHAPE_KEYS}
    if not tune:
        ms = time_periods()
        st = sim_time(ms)
        g.close()
        return dict(base, ms_per_period_default_shapes=ms, real_zone_cycles_per_s=real / (ms * 1e-3),
                    lat_effective_zone_cycles_per_s=eff / (ms * 1e-3), **st)
    restore()
    g.batch_step(per)
    rep = g.autotune()
    tuned = {k: rep[k] for k in SHAPE_KEYS}
    found = dict(tuned)
    times = {"default": [], "tuned": []}
    for r in range(reps):
        for name in (("default", "tuned") if r % 2 == 0 else ("tuned", "default")):
            g.set_launch_shapes(**(default if name == "default" else tuned))
            times[name].append(time_periods())
    md, mt = statistics.median(times["default"]), statistics.median(times["tuned"])
    spread = max(max(v) - min(v) for v in times.values())
    use_tuned = mt < md - spread
    ms = mt if use_tuned else md
    g.set_launch_shapes(**(tuned if use_tuned else default))
    st = sim_time(ms)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.regrid([hamr.block_from_dict(b) for b in blocks])  # onto the same tree: allocation + device fill
    regrid_ms = (time.perf_counter() - t0) * 1e3
    g.close()
    return dict(base, ms_per_period=ms, ms_per_period_default_shapes=md, ms_per_period_tuned_shapes=mt,
                ms_repetitions=times, ms_noise=spread, shapes_used="tuned" if use_tuned else "default",
                launch_shapes_tuned=found, autotuner_kept_tuned=rep["kept_tuned"],
                autotuner_groups_ms={"default": round(rep["ms_default"], 3), "tuned": round(rep["ms_tuned"], 3),
                                     "spread": round(rep["ms_spread"], 3)},
                regrid_same_tree_ms=round(regrid_ms, 1),
                real_zone_cycles_per_s=real / (ms * 1e-3), lat_effective_zone_cycles_per_s=eff / (ms * 1e-3), **st)


def run_ours(args, rank, world, local):
    import torch
    from paper_1912_10192_gb300 import _build, hamr

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    geo, prim, bf = torus_inputs()
    blk = hamr.block(N1, N2, N3, geo.x1min, geo.x2min, geo.x3min, geo.dx1, geo.dx2, geo.dx3, TORUS_BC)
    g = hamr.Grid([blk])
    dprim = torch.from_numpy(prim).cuda()
    dbf = torch.from_numpy(bf).cuda()
    stream = torch.cuda.current_stream()
    g.set_state(dprim, dbf, stream=stream)
    cells = N1 * N2 * N3
    for _ in range(args.warmup):
        g.step(stream=stream)
    torch.cuda.synchronize()

    # ---- timed region: K steps, device events on the launching stream
    g.set_timing(True)
    sampler = ClockSampler(local) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        g.step(stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = ev0.elapsed_time(ev1)
    if dist:
        dist.barrier()
    timing = g.timing()
    g.set_timing(False)
    ms_max = max_over_ranks(ms, dist)
    stats = g.stats()
    value = job_rate(cells * args.steps, world, ms_max * 1e-3)

    # ---- chosen form: the same workload with FP32 reconstruction, fluxes and EMFs
    chosen = None
    if not args.fp64_only:
        forms = [mixed_leg(args, hamr, torch, blk, dprim, dbf, g, stream, cells, world, dist, precision=pr)
                 for pr in (hamr.PREC_MIXED, hamr.PREC_MIXED_FP64INV)]
        ok = [f for f in forms if f["l1_vs_fp64"]["rho"] <= 1e-6]
        best = max(ok or forms, key=lambda f: f["value"])
        chosen = {"value": best["value"], "unit": "zone-cycles/s", "ms_per_step": best["ms_per_step"],
                  "form": best["form"], "l1_vs_fp64": best["l1_vs_fp64"], "fp64_value": value,
                  "speedup_vs_fp64": best["value"] / value, "rho_l1_target": 1e-6,
                  "variants": [{k: f[k] for k in ("precision", "value", "ms_per_step", "l1_vs_fp64", "kernel_ms")}
                               for f in forms]}

    # ---- the learned inversion guess and the batched AMR/LAT tree (single GPU, rank 0 only)
    extra = {}
    if not args.no_extra and world == 1:
        extra["mlp"] = mlp_leg(args, hamr, torch, blk, dprim, dbf, cells, stream)
        extra["options"] = options_leg(args, hamr, torch, blk, dprim, dbf, cells, stream)
        extra["amr_lat"] = [amr_leg(hamr, torch, 0), amr_leg(hamr, torch, 1),
                            amr_leg(hamr, torch, 1, tune=False, smr=2)]

    # ---- end to end: host buffers through the C ABI, copies inside the timed region
    e2e_steps = min(args.steps, 10)
    hp = torch.from_numpy(prim).pin_memory().numpy()
    hb = torch.from_numpy(bf).pin_memory().numpy()
    op = torch.empty(prim.shape, dtype=torch.float64).pin_memory().numpy()
    ob = torch.empty(bf.shape, dtype=torch.float64).pin_memory().numpy()
    g2 = hamr.Grid([blk])
    g2.set_state(hp, hb)
    g2.step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g2.set_state(hp, hb)
        g2.step()
        g2.get_state(prim=op, bface=ob)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    e2e = {"value": job_rate(cells * e2e_steps, world, max_over_ranks(te, dist)), "unit": "zone-cycles/s",
           "h2d_bytes_per_step": int(hp.nbytes + hb.nbytes), "d2h_bytes_per_step": int(op.nbytes + ob.nbytes),
           "steps": e2e_steps,
           "path": "hamr_grid_set_state(host, pinned) + hamr_block_step + hamr_grid_get_state(host) per step"}
    g2.close()

    # ---- roofline of the dominant kernel group (FP64 pipe bound)
    fp64_meas = hamr.measure_fp64_peak() / 1e3  # TFLOP/s
    dom = max(((k, v) for k, v in timing.items() if k != "load"), key=lambda kv: kv[1][1])
    name, (launches, dom_ms) = dom
    steps = args.steps
    faces = ((N1 + 1) * (N2 + 2) * (N3 + 2) + (N1 + 2) * (N2 + 1) * (N3 + 2) + (N1 + 2) * (N2 + 2) * (N3 + 1))
    per_step_units = {"flux": FLOPS_PER_FACE * faces * 2,
                      "recon": FLOPS_PER_RECON_CELL * 3 * (N1 + 2) * (N2 + 2) * (N3 + 2) * 2,
                      "update": FLOPS_PER_UPDATE_CELL * cells * 2}
    roofline = None
    if name in per_step_units:
        flops_per_launch = per_step_units[name] * steps / launches
        avg_s = dom_ms * 1e-3 / launches
        achieved = flops_per_launch / avg_s / 1e12
        roofline = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP64_NOMINAL_TFLOPS,
                    "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (profiling recipe)",
                    "measured_fp64_fma_tflops": fp64_meas, "frac_of_measured": achieved / fp64_meas,
                    "traffic": NCU_TRAFFIC_PER_LAUNCH, "avg_launch_ms": dom_ms / launches,
                    "share_of_step": dom_ms / ms}
    whole = FLOPS_PER_ZONE_CYCLE * cells * args.steps / (ms * 1e-3) / 1e12
    launches_total = sum(v[0] for k, v in timing.items() if k != "load")

    line = {"metric": METRIC, "value": value, "unit": "zone-cycles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells_per_gpu": cells, "dt": "CFL (C0=0.8), reduced on device",
                       "l2": "state and scratch ~1.4 GB per GPU >> 129 MB L2 (no flush needed)",
                       "parallelism": "replicas" if world > 1 else "single block"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches_total), "roofline": roofline,
            "step_fp64_tflops": whole, "step_fp64_frac_nominal": whole / FP64_NOMINAL_TFLOPS,
            "kernel_ms": {k: round(v[1], 3) for k, v in timing.items()},
            "c2p": {k: stats[k] for k in ("c2p_ok", "c2p_entropy", "c2p_fail", "floor_hits")}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, t = cpu_oracle_rate(N1, N2, N3, 1, 0)
        line["cpu_baseline"] = {"value": rate, "unit": "zone-cycles/s", "cores": 1, "kind": "oracle",
                                "sample": "one oracle step of the full 256x128x64 torus block (%.1f s)" % t}
        arate, at, nproc = cpu_oracle_all_cores()
        line["cpu_baseline"]["all_cores"] = {
            "value": arate, "unit": "zone-cycles/s", "cores": nproc, "kind": "oracle",
            "sample": "%d single-threaded oracle processes, one per core, each 2 steps of its own 128x64x32 "
                      "torus block, started together (%.1f s)" % (nproc, at),
            "host": host_cpu()}
    line.update(extra)
    line["chosen_form"] = chosen   # last: a truncated tail of the line still shows it
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-only", action="store_true", help="skip the mixed-precision leg")
    ap.add_argument("--no-extra", action="store_true", help="skip the network and AMR/LAT legs")
    ap.add_argument("--amr-periods", type=int, default=0, metavar="P",
                    help="only time P LAT periods of the 512-block FP64 tree at the default launch shapes "
                         "(for launch lists) and print them")
    ap.add_argument("--amr-precision", type=int, default=0, choices=[0, 1, 2],
                    help="with --amr-periods: 0 FP64, 1 and 2 the mixed forms")
    ap.add_argument("--amr-smr", type=int, default=0, help="with --amr-periods: internal SMR levels")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = env_rank()
    if args.amr_periods > 0:
        import torch
        from paper_1912_10192_gb300 import _build, hamr
        _build.build()
        print(json.dumps(amr_leg(hamr, torch, args.amr_precision, tune=False, nper=args.amr_periods,
                                 smr=args.amr_smr)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
