#!/usr/bin/env python
"""Benchmark of the doubly-periodic FCM mobility product on GB300.

Workload (one "step" = one mobility product M [F; T] -> [U; Omega], every stage of the hot path):
a sedimented layer of N = 2^20 microrollers above one no-slip wall, box 2048 x 2048 x [0, 8],
heights max(|N(1.6, 0.3)|, 1.05), force (0, 0, -1) and torque (0, 1, 0) on every particle, grid
3072^2 x 65 (h = 2/3), ES kernels m = 5 with the Table I shape parameters.  Inputs are synthetic and
seeded (paper_2210_01837_gb300.workloads.rollers_1m).  The working set (15 GB of grid in mixed
precision) is far larger than L2, so no explicit flush is needed between steps.

Headline: products/s of the mixed-precision path (float transforms, FP64 banded solves); the
all-FP64 path is timed on the same GPU and reported beside it, with the relative L2 difference of
the two outputs.  Per-stage CUDA-event timings give the roofline of each kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) every rank runs its own replica (independent systems, no collective on the
data path: weak scaling); the max time over ranks is used and rank 0 prints one JSON line.
--impl reference times the CPU oracle (the FP64 restatement under oracle/) on a bounded tile of the
same workload, on the host cores, and extrapolates to products/s of the full workload.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "mobility products/s at N=1M single wall (mixed vs FP64, same GPU); p99 served"
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # SMs x DFMA/clk/SM x 2 flop x max SM clock


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------------
# algorithmic work per stage (bytes that must cross HBM once; FP64 flops of the banded solves)
# ---------------------------------------------------------------------------------------------
def algorithmic(params, n, zocc, tsize, rec_bytes, fields=6):
    """fields: grid fields spread and transformed (6 with the spectral-curl torque route, 3 with
    the kernel-derivative route, whose interpolation still returns U and Omega)."""
    nx, ny, nz = params["nx"], params["ny"], params["nz"]
    nkx = nx // 2 + 1
    F = fields
    real = F * zocc * ny * nx * tsize
    cpx = F * zocc * ny * nkx * 2 * tsize
    K = nkx * ny
    return {
        "records": n * 9 * 8 + n * rec_bytes,
        "spread": real + n * rec_bytes,
        "fft_x_fwd": real + cpx,
        "fft_y_fwd": 2 * cpx,
        "cheb_fwd": cpx + 3 * nz * K * 2 * tsize,
        "cheb_bwd": 3 * nz * K * 2 * tsize + cpx,
        "fft_y_inv": 2 * cpx,
        "fft_x_inv": cpx + real,
        "interp": real + n * rec_bytes + n * 6 * 8,
        # FP64 flops per wavenumber and Chebyshev row of the table-driven solve: 8 real right-hand
        # sides (pressure, then u, v, w; re and im) x one FMA each for the elimination, the boundary
        # fold, the back substitution and the boundary value; the factorisation is a plan-time table
        # and each row's pivot scales the right-hand side where it is formed (float); the B B map
        # runs in float
        "solve_fp64_flops": K * nz * (8 * 4 * 2),
    }


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            return int(json.load(f)[kernel]["bytes_per_launch"])
    except Exception:
        return None


def occupied_planes(params, pos, alpha):
    """Chebyshev planes within alpha of some particle or of its wall image (the planes the
    library transforms); computed here only to size the algorithmic byte counts."""
    nz = params["nz"]
    c = np.arange(nz)
    zc = params["zmin"] + 0.5 * (params["zmax"] - params["zmin"]) * (1 + np.cos(np.pi * c / (nz - 1)))
    lo = max(params["zmin"], pos[:, 2].min() - alpha)
    hi = min(params["zmax"], pos[:, 2].max() + alpha)
    return int(np.count_nonzero((zc >= lo - 1e-12) & (zc <= hi + 1e-12)))


# ---------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle samples of this GPU during the timed region."""

    FIELDS = ("uuid,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None, index=0):
        self.proc = None
        self.lines = []
        self.uuid = uuid
        self.index = index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [[p.strip() for p in line.split(",")] for line in self.lines]
        rows = [r for r in rows if len(r) >= 10]
        mine = [r for r in rows if self.uuid and r[0].lower() == self.uuid.lower()]
        if not mine:
            mine = [r for r in rows if r[1] == str(self.index)]
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in mine:
            try:
                sm.append(float(r[2]))
                smax.append(float(r[3]))
                power.append(float(r[4]))
            except ValueError:
                continue
            for nm, v in zip(names, r[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------------
def cpu_oracle_tile(div, seed_offset=3):
    """One oracle product on a 1/div^2-area tile of the roller workload; returns (seconds, n)."""
    from oracle import Params, mobility
    from paper_2210_01837_gb300.workloads import rollers_1m
    params, pos, F, T = rollers_1m(n=(1 << 20) // (div * div), nxy=3072 // div, L=2048.0 / div,
                                   seed_offset=seed_offset)
    t0 = time.perf_counter()
    mobility(Params(**params), pos, F, T)
    return time.perf_counter() - t0, len(pos), params["nx"]


def cpu_oracle_config(name, div=1, seed=0):
    """One oracle product of workload `name` ("bw_small": whole; "slit_16k": a 1/div^2-area
    tile with the same density, heights and h; "batch": system `seed` of the 256-system uneven
    population, whole); returns seconds."""
    from oracle import Params, mobility
    from paper_2210_01837_gb300.workloads import batch_systems, bw_small, slit_16k
    if name == "bw_small":
        params, pos, F, T = bw_small()
    elif name == "batch":
        params, pos, F, T = batch_systems(count=256)[seed]
    else:
        params, pos, F, T = slit_16k(n=16384 // (div * div), nxy=384 // div, L=256.0 / div, seed_offset=2 + 100 * seed)
    t0 = time.perf_counter()
    mobility(Params(**params), pos, F, T)
    return time.perf_counter() - t0


def _oracle_config_runs(name, div, procs, threads, seeds=None):
    """Wall seconds of `procs` concurrent oracle products of `name`, each in a fresh interpreter
    with `threads` BLAS/OpenMP threads, and the per-process times."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    t0 = time.perf_counter()
    kids = []
    for i in range(procs):
        seed = seeds[i] if seeds is not None else i
        code = ("import sys, json; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench.cpu_oracle_config(%r, %d, %d)))" % (ROOT, name, div, seed))
        kids.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                     text=True, env=env))
    per = [json.loads(k.communicate(timeout=1800)[0].strip().splitlines()[-1]) for k in kids]
    return time.perf_counter() - t0, per


def oracle_configs():
    """The oracle on the small workloads on the host's cores: the 100-sphere wall case (128^2 x 65)
    whole (one process with every core's BLAS threads, and one process on one core); the 16k-sphere
    slit (384^2 x 97) as one 1/16-area tile per core, all at once, and one tile on one core (times x
    16: work is linear in N and in grid nodes); and a sample of the 256-system uneven batch."""
    cores = host_cores()
    c1_all, _ = _oracle_config_runs("bw_small", 1, 1, cores)
    c1_one, _ = _oracle_config_runs("bw_small", 1, 1, 1)
    div = 4
    wall, per = _oracle_config_runs("slit_16k", div, cores, 1)
    t1, _ = _oracle_config_runs("slit_16k", div, 1, 1)
    # the 256-system batch: every 8th of the 128 smallest systems (the whole population would take
    # hours of oracle time), one per core at once; the batch's time extrapolated by nx ny nz^3 (the
    # oracle's dense LU per wavenumber dominates: the two small workloads scale so within 15 %)
    from paper_2210_01837_gb300.workloads import batch_systems
    pop = batch_systems(count=256)
    nodes = [p_["nx"] * p_["ny"] * float(p_["nz"]) ** 3 for p_, _, _, _ in pop]
    order = sorted(range(len(pop)), key=lambda i: len(pop[i][1]))
    sample = order[:128:8]
    wall4, per4 = _oracle_config_runs("batch", 1, len(sample), 1, seeds=sample)
    scale4 = sum(nodes) / sum(nodes[i] for i in sample)
    return {"cores": cores,
            "batch": {"sample": f"{len(sample)} of the 128 smallest systems (every 8th by N; N "
                                f"{len(pop[sample[0]][1])}-{len(pop[sample[-1]][1])}), one per core at once: "
                                f"{wall4:.1f} s wall, {sum(per4):.1f} s of oracle time",
                      "batch_oracle_s_extrapolated": sum(per4) * scale4,
                      "rule": "oracle time per system proportional to nx ny nz^3; the 256 systems have "
                              f"{scale4:.1f}x the sample's; one core"},
            "bw_small": {"wall_s_all_cores": c1_all, "wall_s_one_core": c1_one, "sample": "whole product, N=100"},
            "slit_16k": {"products_per_s_all_cores": cores / (wall * div * div),
                         "wall_s_one_core_extrapolated": t1 * div * div,
                         "sample": f"{cores} concurrent 1/{div * div}-area tiles (N={16384 // (div * div)}, "
                                   f"{384 // div}^2x97, one core each): {wall:.1f} s wall (per tile "
                                   f"{min(per):.1f}-{max(per):.1f} s); one tile on one core {t1:.1f} s, x {div * div}"}}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_tiles(div, procs):
    """Wall seconds for `procs` concurrent oracle products, one per child process (each with one
    BLAS/OpenMP thread, seed offsets 3 + i: independent tiles of the same layer), plus the tile's
    N and grid side.  Children are fresh interpreters: no CUDA state is inherited."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    t0 = time.perf_counter()
    kids = []
    for i in range(procs):
        code = ("import sys, json; sys.path.insert(0, %r); import bench; "
                "t, n, nx = bench.cpu_oracle_tile(%d, seed_offset=%d); print(json.dumps([t, n, nx]))"
                % (ROOT, div, 3 + i))
        kids.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                     text=True, env=env))
    res = []
    for k in kids:
        out, _ = k.communicate(timeout=900)
        res.append(json.loads(out.strip().splitlines()[-1]))
    wall = time.perf_counter() - t0
    return wall, res[0][1], res[0][2], [r[0] for r in res]


def cpu_baseline(div=16):
    """The oracle as it stands on the host's cores: one product per core on independent
    1/div^2-area tiles of the same workload, all cores at once (the throughput reported), and one
    product on one core; rates are extrapolated to the full product by the area ratio."""
    scale = div * div
    cores = host_cores()
    wall, n, nx, per = _oracle_tiles(div, cores)
    t1, _, _, _ = _oracle_tiles(div, 1)
    return {"value": cores / (wall * scale), "unit": "products/s", "cores": cores, "kind": "oracle",
            "threads_per_process": {"OMP_NUM_THREADS": 1, "OPENBLAS_NUM_THREADS": 1, "numpy.fft": 1},
            "sample": f"oracle (numpy FP64) on {cores} concurrent 1/{scale}-area tiles of the same workload "
                      f"(one per core; N={n}, {nx}^2x65 each, same density, heights, h, kernels): {wall:.1f} s wall "
                      f"(per tile {min(per):.1f}-{max(per):.1f} s); products/s = cores / (wall x {scale}) (work is "
                      f"linear in N and in grid nodes; the FFT log factor is ignored)",
            "single_core": {"value": 1.0 / (t1 * scale), "unit": "products/s", "cores": 1,
                            "sample": f"one tile on one core: {t1:.1f} s, time x {scale}"}}


def run_reference(args, rank):
    if rank != 0:
        return
    div = 32
    cores = host_cores()
    for _ in range(args.warmup):
        _oracle_tiles(div, cores)
    walls = []
    n = nx = 0
    for _ in range(args.steps):
        wall, n, nx, _ = _oracle_tiles(div, cores)
        walls.append(wall)
    # each step: one oracle product per core on independent 1/div^2-area tiles, all at once
    t = float(np.mean(walls)) * div * div / cores
    value = 1.0 / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "rollers_1m: N=1048576 above one wall, 3072^2x65, m=5 Table I",
                      "sample": f"{cores} concurrent 1/{div * div}-area tiles per step (N={n}, {nx}^2x65 each), "
                                f"extrapolated"},
           "cpu_baseline": {"value": value, "unit": "products/s", "cores": cores, "kind": "oracle",
                            "sample": f"one 1/{div * div}-area tile of the roller workload per core per step, all "
                                      f"cores at once; products/s = cores / (wall x {div * div})"},
           "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------------------------
# batched and served products (independent systems of uneven size)
# ---------------------------------------------------------------------------------------------
def batch_leg(binding, torch, dev, count, steps, warmup, wave=64):
    """Products/s of `count` uneven systems, run in waves of `wave` systems (all plans of a wave
    resident): one after another on one stream, as one batched apply per wave, and as a replayed
    CUDA graph of each wave's batch.  Returns the summary and the first wave's systems."""
    from paper_2210_01837_gb300.workloads import batch_systems
    systems = batch_systems(count=count)
    stream = torch.cuda.current_stream(dev)
    tdev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    def timed(fn, k):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 1e3 / k

    binding.dpstokes_batch_prepare()
    t_seq = t_bat = t_graph = t_plans = 0.0
    waves = 0
    for w0 in range(0, count, wave):
        chunk = systems[w0:w0 + wave]
        t0 = time.perf_counter()
        plans, items = [], []
        for params, pos, F, T in chunk:
            plan = binding.Plan.from_params(params, with_torque=True, precision="mixed", max_n=len(pos))
            U = torch.empty((len(pos), 3), dtype=torch.float64, device=dev)
            plans.append(plan)
            items.append((plan, tdev(pos), tdev(F), tdev(T), U, torch.empty_like(U)))
        t_plans += time.perf_counter() - t0

        def sequential():
            for plan, pos, F, T, U, W in items:
                plan.apply(pos, F, T, U, W)

        def batched():
            binding.apply_batch(items)

        t_seq += timed(sequential, steps)
        t_bat += timed(batched, steps)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            batched()
        t_graph += timed(graph.replay, steps)
        for plan in plans:
            plan.check()
        del graph, items
        for plan in plans:
            plan.close()
        torch.cuda.synchronize(dev)
        waves += 1
    particles = sum(len(s[1]) for s in systems)
    out = {"workload": f"batch_systems: {count} uneven systems (N log-uniform 100..50000, half bottom wall / "
                       f"half slit, nz in 33/65/97), forces+torques, mixed; {waves} waves of <= {wave} resident plans",
           "systems": count, "particles": particles, "waves": waves, "plan_create_s": round(t_plans, 2),
           "sequential_products_per_s": count / t_seq, "batched_products_per_s": count / t_bat,
           "graph_products_per_s": count / t_graph, "batched_vs_sequential": t_seq / t_bat,
           "ms_per_batch": {"sequential": t_seq * 1e3, "batched": t_bat * 1e3, "graph": t_graph * 1e3}}
    return out, systems[:wave]


def configs_leg(binding, torch, dev, steps=5, warmup=3):
    """Time per product of the other workloads, for context: the small FP64 case (bw_small), the
    slit with 16k particles (slit_16k, mixed and FP64), and the paper's largest force-only scaling
    system (663,552 particles, grid 2700^2 x 19, m = 4; 370 ms per solve on a V100 in the paper)."""
    from paper_2210_01837_gb300.workloads import bw_small, lanczos_layer, slit_16k
    tdev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    hbm, _ = peaks()
    fracs = {}

    def ms(params, pos, F, T, precision, with_torque, key=None):
        plan = binding.Plan.from_params(params, with_torque=with_torque, precision=precision, max_n=len(pos))
        d_pos, d_F = tdev(pos), tdev(F)
        d_T = tdev(T) if with_torque else None
        U = torch.empty((len(pos), 3), dtype=torch.float64, device=dev)
        W = torch.empty_like(U) if with_torque else None
        for _ in range(warmup):
            plan.apply(d_pos, d_F, d_T, U, W)
        plan.check()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.apply(d_pos, d_F, d_T, U, W)
        e1.record()
        torch.cuda.synchronize(dev)
        plan.check()
        if key:
            # fractions of the measured copy bandwidth of the HBM-bound stages (separate timed pass)
            plan.enable_timing(True)
            log = []
            for _ in range(3):
                plan.apply(d_pos, d_F, d_T, U, W)
                log.append(plan.stage_times())
            plan.enable_timing(False)
            info = plan.info()
            work = algorithmic(params, len(pos), occupied_planes(params, pos, info.alpha_M),
                               4 if precision == "mixed" else 8, info.record_words * 4, fields=info.nfields)
            st = {k: float(np.mean([l_[k] for l_ in log])) for k in log[0]}
            fracs[key] = {k: round(work[k] / (st[k] * 1e-3) / 1e9 / hbm, 3)
                          for k in ("spread", "fft_x_fwd", "fft_y_fwd", "fft_y_inv", "fft_x_inv", "interp")}
        plan.close()
        return round(e0.elapsed_time(e1) / steps, 4)

    out = {}
    p, pos, F, _ = bw_small()
    out["bw_small_fp64_ms"] = ms(p, pos, F, None, "fp64", False, "bw_small_fp64")
    p, pos, F, T = slit_16k()
    out["slit_16k_mixed_ms"] = ms(p, pos, F, T, "mixed", True, "slit_16k_mixed")
    out["slit_16k_fp64_ms"] = ms(p, pos, F, T, "fp64", True, "slit_16k_fp64")
    p, pos, W = lanczos_layer(18, H=9.1)
    out["fig9_forces_663552_mixed_ms"] = ms(p, pos, W, None, "mixed", False)
    out["fig9_forces_663552_fp64_ms"] = ms(p, pos, W, None, "fp64", False)
    out["stage_frac_hbm"] = fracs
    out["fig9_paper_v100_ms"] = 370.0
    out["note"] = ("CUDA events per product after 3 warm-up products; the paper's 370 ms is its V100 time for the "
                   "same-sized system (precision not stated), context only")
    return out


def served_capacity(binding, torch, dev, systems):
    """Requests/s of the served population when every system runs once per batched apply."""
    tdev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    plans, items = [], []
    for params, pos, F, T in systems:
        plan = binding.Plan.from_params(params, with_torque=True, precision="mixed", max_n=len(pos))
        U = torch.empty((len(pos), 3), dtype=torch.float64, device=dev)
        plans.append(plan)
        items.append((plan, tdev(pos), tdev(F), tdev(T), U, torch.empty_like(U)))
    binding.apply_batch(items)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(2):
        binding.apply_batch(items)
    torch.cuda.synchronize(dev)
    t = (time.perf_counter() - t0) / 2
    del items
    for plan in plans:
        plan.close()
    return len(systems) / t


def fp64_unbatched_leg(binding, torch, systems, count, budget=120e9, seed=20221010):
    """The unbatched FP64 path: `count` requests drawn from the population, each submitted when
    the previous one has completed to a one-slot server running the all-FP64 product (plans
    resident, host inputs and outputs pinned); per-request latency (submission to completion, no
    queueing) and the products/s this gives."""
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    rng = np.random.default_rng(seed)
    picks = rng.integers(0, len(systems), count)
    srv = binding.Server(int(budget), slots=1)
    lat = []
    t_all = 0.0
    for rep in range(2):  # first pass creates the plans
        for i in (picks if rep else np.unique(picks)):
            params, pos, F, T = systems[i]
            n = len(pos)
            U = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
            W = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
            t = srv.submit(params, True, "fp64", n, pin(pos), pin(F), pin(T), U, W)
            r, _, _ = srv.wait(t)
            if r.status != 0:
                raise RuntimeError(f"FP64 request failed: {r.status}")
            if rep:
                lat.append(r.t_done - r.t_submit)
    srv.close()
    lat = np.array(lat) * 1e3
    return {"requests": count, "products_per_s": 1e3 * count / lat.sum(), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "how": "one-slot server, FP64 plans resident, each request submitted after the previous completed"}


def served_leg(binding, torch, systems, rate, duration, slots=8, budget=120e9, seed=20221009, max_queued=64,
               precision="mixed"):
    """Poisson arrivals of requests drawn uniformly from `systems` (host inputs in pinned memory) at
    `rate` per second for `duration` seconds; latency = completion - submission of the accepted
    requests.  At most `max_queued` requests wait for admission; a submission that finds the
    queue full is refused (load shedding) and counted."""
    import queue as _queue
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    inputs = [(params, pin(pos), pin(F), pin(T)) for params, pos, F, T in systems]
    nmax = max(len(s[1]) for s in systems)
    ring = 128  # output buffers in flight
    outs = [(torch.empty((nmax, 3), dtype=torch.float64).pin_memory().numpy(),
             torch.empty((nmax, 3), dtype=torch.float64).pin_memory().numpy()) for _ in range(ring)]
    srv = binding.Server(int(budget), slots=slots)
    # plans of the population resident before the clock starts
    for i, (params, pos, F, T) in enumerate(inputs):
        n = len(pos)
        t = srv.submit(params, True, precision, n, pos, F, T, outs[i % ring][0][:n], outs[i % ring][1][:n])
        r, _, _ = srv.wait(t)
        if r.status != 0:
            raise RuntimeError(f"served warm-up request failed: {r.status}")
    if max_queued:
        binding.dpstokes_server_set_queue_limit(srv.handle, max_queued)
    rng = np.random.default_rng(seed)
    n_req = max(1, int(rate * duration))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    picks = rng.integers(0, len(inputs), n_req)
    tickets = _queue.Queue()

    def submitter():
        t0 = time.perf_counter()
        for i in range(n_req):
            dt = t0 + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            params, pos, F, T = inputs[picks[i]]
            n = len(pos)
            U, W = outs[i % ring]
            t = srv.submit(params, True, precision, n, pos, F, T, U[:n], W[:n])
            if t is None:
                refused[0] += 1
            else:
                tickets.put(t)
        tickets.put(None)

    refused = [0]

    th = threading.Thread(target=submitter)
    th.start()
    lat, first, last, bad = [], None, None, 0
    while True:
        t = tickets.get()
        if t is None:
            break
        r, _, _ = srv.wait(t, timeout_s=600.0)
        bad += r.status != 0
        lat.append(r.t_done - r.t_submit)
        first = r.t_submit if first is None else min(first, r.t_submit)
        last = r.t_done if last is None else max(last, r.t_done)
    th.join()
    stats = srv.stats()
    srv.close()
    lat = np.array(lat) * 1e3
    done = len(lat)
    return {"offered_req_per_s": rate, "duration_s": duration, "requests": n_req, "accepted": done,
            "refused": refused[0], "failed": int(bad), "precision": precision,
            "throughput_req_per_s": done / (last - first) if done else 0.0,
            "p50_ms": float(np.percentile(lat, 50)) if done else None,
            "p99_ms": float(np.percentile(lat, 99)) if done else None,
            "mean_ms": float(lat.mean()) if done else None, "slots": slots, "max_queued": max_queued,
            "budget_gb": budget / 1e9, "plans_resident": stats["plans_resident"],
            "plans_evicted": stats["plans_evicted"]}


# ---------------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--div", type=int, default=1, help="shrink the workload by div^2 in area (testing only)")
    ap.add_argument("--nz", type=int, default=0, help="Chebyshev nodes in z (profiling only; default 65)")
    ap.add_argument("--batch-systems", type=int, default=256, help="systems in the batched leg (0: skip batched and served legs)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shapes (no autotuner)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="duration of each served leg (0: skip serving); the serving workload asks for 60")
    ap.add_argument("--serve-population", type=int, default=64, help="systems in the served population")
    ap.add_argument("--no-deriv", action="store_true", help="skip the kernel-derivative torque-route leg")
    ap.add_argument("--no-lanczos", action="store_true", help="skip the Brownian-increment (Lanczos) leg")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads' timings")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="also time the oracle on the small workloads and a batch sample on the host cores (minutes)")
    args = ap.parse_args()

    from paper_2210_01837_gb300.replicas import Collective, rank_env, replica_seed_offset, whole_job_rate
    env = rank_env()
    rank, world, local = env.rank, env.world, env.local

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2210_01837_gb300 import binding, build
    from paper_2210_01837_gb300.workloads import rollers_1m
    build.build()
    binding.load()

    div = args.div
    params, pos, F, T = rollers_1m(n=(1 << 20) // (div * div), nxy=3072 // div, L=2048.0 / div, seed_offset=replica_seed_offset(rank))
    if args.nz:
        params["nz"] = args.nz
    n = len(pos)
    dev = torch.device("cuda", local)
    tdev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_pos, d_F, d_T = tdev(pos), tdev(F), tdev(T)
    U = torch.empty((n, 3), dtype=torch.float64, device=dev)
    W = torch.empty_like(U)
    stream = torch.cuda.current_stream(dev)

    coll = Collective(dist, dev)
    barrier, max_over_ranks = coll.barrier, coll.max

    def time_plan(plan, steps, warmup):
        """Seconds for `steps` back-to-back applies (CUDA events on the launching stream, no
        per-stage events and no host synchronisation inside the timed region)."""
        for _ in range(warmup):
            plan.apply(d_pos, d_F, d_T, U, W)
        plan.check()
        barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.apply(d_pos, d_F, d_T, U, W)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        plan.check()
        return e0.elapsed_time(e1) / 1e3

    def stage_pass(plan, steps):
        """Per-stage milliseconds (mean over `steps` applies), from per-launch event pairs in a
        separate pass after the headline timing."""
        plan.enable_timing(True)
        log = []
        for _ in range(steps):
            plan.apply(d_pos, d_F, d_T, U, W)
            log.append(plan.stage_times())
        plan.enable_timing(False)
        plan.check()
        return {k: float(np.mean([s_[k] for s_ in log])) for k in log[0]}

    # ---- mixed precision (headline) --------------------------------------------------------
    plan = binding.Plan.from_params(params, with_torque=True, precision="mixed", max_n=n)
    tuned_ms = plan.autotune(d_pos, d_F, d_T, U, W) if not args.no_tune else None
    info = plan.info()
    tuned = {"autotune_ms": tuned_ms, "fft_col_width": info.fft_col_width,
             "fft_register_staged": {"rows": info.fft_register_rows, "cols": info.fft_register_cols},
             "solve_blocks": info.solve_blocks,
             "wavenumber_chunks": info.nchunks}
    launches_per_apply = info.launches_per_apply
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid=uuid, index=local)
    t_mixed = time_plan(plan, args.steps, args.warmup)
    clocks = sampler.stop()
    t_mixed = max_over_ranks(t_mixed)
    ms_step = t_mixed / args.steps * 1e3
    value = whole_job_rate(world, args.steps, t_mixed)
    U_mixed = U.clone()
    W_mixed = W.clone()

    stages = stage_pass(plan, max(3, min(args.steps, 10)))
    zocc = occupied_planes(params, pos, info.alpha_M)
    hbm, peak_kind = peaks()
    work = algorithmic(params, n, zocc, 4, info.record_words * 4)
    stage_roof = {}
    for k, ms in stages.items():
        if k in work:
            gbs = work[k] / (ms * 1e-3) / 1e9
            stage_roof[k] = {"ms": round(ms, 4), "GB/s": round(gbs, 1), "frac_hbm": round(gbs / hbm, 3)}
    solve_tflops = work["solve_fp64_flops"] / (stages["solve"] * 1e-3) / 1e12
    stage_roof["solve"] = {"ms": round(stages["solve"], 4), "fp64_TFLOP/s": round(solve_tflops, 3),
                           "frac_fp64_nominal": round(solve_tflops / FP64_NOMINAL_TFLOPS, 3)}
    dom = max((k for k in stages if k in work or k == "solve"), key=stages.get)
    if dom == "solve":
        roofline = {"bound": "alu", "kernel": "solve_tab_kernel (FP64 banded solves)", "achieved": round(solve_tflops, 4),
                    "peak": round(FP64_NOMINAL_TFLOPS, 3), "unit": "TFLOP/s",
                    "frac": round(solve_tflops / FP64_NOMINAL_TFLOPS, 4),
                    "traffic": measured_traffic("solve_tab_kernel<float, 0>") if div == 1 and not args.nz else None,
                    "traffic_source": "profiles/traffic.json (ncu dram bytes, scaled by wavenumbers)",
                    "peak_kind": "FP64 nominal from unit counts x max clock"}
    else:
        gbs = work[dom] / (stages[dom] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(gbs / hbm, 4), "traffic": None, "peak_kind": peak_kind}
    roofline["timing"] = "stage events from a separate pass after the headline timing"

    # ---- end to end through the public API with host buffers -------------------------------
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    h_pos, h_F, h_T = pin(pos), pin(F), pin(T)
    h_U = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    h_W = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    plan.apply_host(h_pos, h_F, h_T, h_U, h_W)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(e2e_steps):
        plan.apply_host(h_pos, h_F, h_T, h_U, h_W)
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": whole_job_rate(world, e2e_steps, t_e2e), "unit": "products/s", "h2d_bytes_per_step": 3 * h_pos.nbytes,
           "d2h_bytes_per_step": 2 * h_U.nbytes, "steps": e2e_steps}
    plan.close()
    del plan

    # ---- the kernel-derivative torque route (second route of Sec. III.D), same workload --------
    deriv = None
    if not args.no_deriv:
        plan_d = binding.Plan.from_params(params, with_torque="kernel_derivative", precision="mixed", max_n=n)
        tuned_d_ms = plan_d.autotune(d_pos, d_F, d_T, U, W) if not args.no_tune else None
        info_d = plan_d.info()
        t_d = max_over_ranks(time_plan(plan_d, args.steps, args.warmup))
        st_d = stage_pass(plan_d, max(3, min(args.steps, 10)))
        work_d = algorithmic(params, n, zocc, 4, info_d.record_words * 4, fields=3)
        roof_d = {}
        for k, ms in st_d.items():
            if k in work_d:
                gbs = work_d[k] / (ms * 1e-3) / 1e9
                roof_d[k] = {"ms": round(ms, 4), "GB/s": round(gbs, 1), "frac_hbm": round(gbs / hbm, 3)}
        rl2 = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        value_d = whole_job_rate(world, args.steps, t_d)
        deriv = {"value": value_d, "unit": "products/s", "ms_per_step": t_d / args.steps * 1e3,
                 "speedup_vs_spectral_curl": value_d / value, "nfields": info_d.nfields,
                 "gpu_launches": info_d.launches_per_apply * args.steps,
                 "launch_shapes": {"autotune_ms": tuned_d_ms, "fft_col_width": info_d.fft_col_width,
                                   "solve_blocks": info_d.solve_blocks, "wavenumber_chunks": info_d.nchunks},
                 "stages_ms": {k: round(v, 4) for k, v in st_d.items()}, "stage_roofline": roof_d,
                 "vs_spectral_curl_rel_l2": {"U": rl2(U, U_mixed), "Omega": rl2(W, W_mixed)},
                 "note": "same workload and precision; the two routes differ by the kernel sampling error at m = 5"}
        plan_d.close()
        del plan_d

    # ---- Brownian increments g = M^{1/2} W by Lanczos (Sec. IV.C) on the paper's layer ---------
    lanczos = None
    if not args.no_lanczos:
        from paper_2210_01837_gb300.workloads import lanczos_layer
        reps = max(1, 8 // div)
        lp, lpos, lW = lanczos_layer(reps, seed_offset=5 + rank)
        lplan = binding.Plan.from_params(lp, with_torque=False, precision="mixed", max_n=len(lpos))
        lz = binding.Lanczos(lplan, max_iter=40)
        d_lpos, d_lW = tdev(lpos), tdev(lW.ravel())
        for _ in range(2):
            g_l, it_l, hist_l = lz.sample(d_lpos, d_lW, tol=1e-3)
        k_l = max(1, min(args.steps, 5))
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(k_l):
            g_l, it_l, hist_l = lz.sample(d_lpos, d_lW, tol=1e-3)
        torch.cuda.synchronize(dev)
        t_l = max_over_ranks(time.perf_counter() - t0)
        lplan.enable_timing(True)
        lplan.apply(d_lpos, tdev(lW), None)
        t_prod = sum(lplan.stage_times().values())
        lplan.enable_timing(False)
        lanczos = {"value": whole_job_rate(world, k_l, t_l), "unit": "samples/s", "ms_per_sample": t_l / k_l * 1e3,
                   "iterations": it_l, "eps_history": [float(f"{e:.3e}") for e in hist_l], "tol": 1e-3,
                   "n": len(lpos), "product_kernel_ms": round(t_prod, 4),
                   "workload": f"lanczos_layer reps={reps}: {len(lpos)} non-overlapping spheres in two layers above "
                               f"one wall, H = 7.5 R_h, grid {lp['nx']}^2 x {lp['nz']}, m = 4, forces only, mixed",
                   "timing": "host clock around whole samples (one synchronisation per iteration)"}
        lz.close()
        lplan.close()

    configs = None
    if not args.no_configs and div == 1:
        configs = configs_leg(binding, torch, dev)
    if args.oracle_configs and rank == 0:
        configs = dict(configs or {})
        configs["oracle"] = oracle_configs()

    # ---- all-FP64 path on the same GPU -------------------------------------------------------
    fp64 = None
    if not args.no_fp64:
        plan64 = binding.Plan.from_params(params, with_torque=True, precision="fp64", max_n=n)
        t64 = max_over_ranks(time_plan(plan64, args.fp64_steps, 1))
        d = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        fp64 = {"value": whole_job_rate(world, args.fp64_steps, t64), "unit": "products/s",
                "ms_per_step": t64 / args.fp64_steps * 1e3, "steps": args.fp64_steps,
                "mixed_speedup": (world * args.steps / t_mixed) / (world * args.fp64_steps / t64),
                "mixed_vs_fp64_rel_l2": {"U": d(U_mixed, U), "Omega": d(W_mixed, W)}}
        plan64.close()

    # ---- batched and served products (independent systems of uneven size) --------------------
    batch = served = None
    if args.batch_systems > 0:
        batch, _ = batch_leg(binding, torch, dev, args.batch_systems, max(1, min(args.steps, 3)), 1)
    if args.serve_seconds > 0:
        from paper_2210_01837_gb300.workloads import serving_systems
        population = serving_systems(count=args.serve_population)
        capacity = served_capacity(binding, torch, dev, population)
        legs = {}
        for name, rate in (("half_capacity", 0.5 * capacity), ("0.8_capacity", 0.8 * capacity),
                           ("specified_2000", 2000.0)):
            legs[name] = served_leg(binding, torch, population, rate=rate, duration=args.serve_seconds)
        served = {"population": f"serving_systems: {len(population)} systems drawn from the uneven-batch size "
                                f"distribution, wall mode cycling over free / bottom wall / slit, forces + torques, "
                                f"mixed; requests drawn uniformly from them",
                  "capacity_req_per_s": capacity,
                  "capacity_how": "the whole population as one batched apply, twice; population / time",
                  "legs": legs,
                  "fp64_unbatched": fp64_unbatched_leg(binding, torch, population, min(32, len(population)))}
        served["p99_ms"] = legs["0.8_capacity"]["p99_ms"]

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "products/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
               "config": {"workload": ("rollers_1m" if div == 1 else f"rollers_1m/{div * div}")
                          + (f" nz={args.nz}" if args.nz else ""),
                          "n": n, "grid": f"{params['nx']}x{params['ny']}x{params['nz']}", "wall": "bottom_wall",
                          "box": f"{params['Lx']:g}x{params['Ly']:g}x[0,8]",
                          "kernels": "ES m=5, beta_M=6.525, beta_D=11.16 (Table I)", "precision": "mixed",
                          "occupied_planes": zocc, "l2": "working set >> L2 (no flush needed)",
                          "launch_shapes": tuned,
                          "parallelism": "replicas" if world > 1 else "1 GPU"},
               "particles_per_s": value * n, "fp64": fp64, "stages_ms": {k: round(v, 4) for k, v in stages.items()},
               "stage_roofline": stage_roof, "roofline": roofline, "e2e": e2e,
               "gpu_launches": launches_per_apply * args.steps, "clocks": clocks,
               "batch": batch, "served": served, "kernel_derivative_route": deriv, "lanczos": lanczos,
               "other_configs": configs}
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
