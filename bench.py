#!/usr/bin/env python
"""Throughput of the coupled HCA step: lattice site-steps/s at 256^3.

Workload (one step = oxygen solve + two drug solves + cell ODEs + CA sweep):
256^3 lattice, FP32 fields with FP64 reductions, synthetic maps from seeded
Gaussian random fields (correlation length 8 sites, cell density 0.4, vessel
density 0.12), bolus every 21 steps, CG to 1e-8 relative residual (FP64-measured, defect correction),
each CG iteration preconditioned by one geometric-multigrid V-cycle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun), every rank advances its
own independent replicate (seed + rank): replicas only, no collective on the
data path; the barrier and the max over ranks time the job.

--impl reference times the CPU oracle (the comparison arm: there is no
reference GPU code) on a bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "lattice site-steps/s at 256^3 coupled"
N_EDGE = 256
SAMPLE_EDGE = 64          # CPU sample lattice
WORKLOAD = dict(precision="f32", n_drugs=2, seed=1, rtol_o2=1e-8, rtol_drug=1e-8, picard_tol=1e-6,
                dose_interval=21, preconditioner=1)     # 1 = HCA_PC_MG
CORR_LEN = 8.0
# algorithmic HBM bytes per site of each kernel class (FP32):
#   pass A reads z, p_old, d and writes p_new and q = A p_new; pass B reads p, q, x, r and
#   writes x, r;
#   defect-correction residual (later sweeps) reads x_hi, x_lo, d, a, b and writes z, dx, r;
#   multigrid on the lattice, four kernels per V-cycle: the two pre-sweeps read r, 1/d and
#   write the pre-smoothed iterate v (12 B); the restriction reads v, r, d and writes
#   v' = v + (W2/d)(r - A v) and the 1/8-size coarse right-hand side (16.5 B); the prolongation
#   + first post-sweep reads v', 1/d and the 1/8-size coarse correction and writes y (12.5 B);
#   the last post-sweep reads y, r, 1/d and writes z (16 B); ODE reads state, K and
#   updates phi, P, Vc
BYTES_PER_SITE = {"pass_a": 20, "pass_b": 24, "setup": 17, "residual": 24, "ode": 29,
                  "mg_pre0": 12, "mg_restrict0": 16.5, "mg_post0": 12.5, "mg_last0": 16}
# the method's minimum per site where this design moves more: CG pass A reads
# z, d, p_old and writes p (16 B); storing q = A p for pass B adds 4 B
BYTES_MIN_PER_SITE = {**BYTES_PER_SITE, "pass_a": 16}
# step-level algorithmic bytes per lattice site (FP32 storage): set-up and
# solve start-up, ODE and CA 70 B, 13 B per defect-correction residual sweep,
# 40 B per CG iteration (two-pass minimum), plus per V-cycle the lattice's
# smoothing and transfers (29 B: the pre-sweeps and restriction need r and
# 1/d and leave one iterate and the next level's rhs, the post-sweeps need
# that iterate, r, 1/d and the coarse correction and write z, whatever the
# number of sweeps when they are fused) and the coarse levels (33 B per
# coarse site, by the same count)
STEP_FIXED_B, STEP_DC_B, STEP_IT_B, VCYCLE_LATTICE_B, VCYCLE_COARSE_B = 70, 13, 40, 29, 33
# the bytes this design's kernels move per CG iteration (pass A also stores
# q: 44 B) and per V-cycle (the four lattice kernels: 57 B; per coarse site the
# four coarse kernels, fused pre-sweeps 16, restriction 12.5, fused first
# post-sweep 20.5, last sweep 20 B: 69 B)
STEP_IT_DESIGN_B, VCYCLE_LATTICE_DESIGN_B, VCYCLE_COARSE_DESIGN_B = 44, 57, 69


def metric_name(edge: int = N_EDGE) -> str:
    """The headline metric at 256^3; other edges (a hidden option) say theirs."""
    return METRIC if edge == N_EDGE else f"lattice site-steps/s at {edge}^3 coupled"


def workload_config(edge: int = N_EDGE):
    return {"workload": f"{edge}^3 coupled HCA step (O2 quasi-steady CG + 2 implicit-Euler drug CGs + "
                        f"per-cell ODEs + 27-colour stochastic CA)",
            "solver": "CG preconditioned by one geometric-multigrid V-cycle per iteration; FP32 inner solves "
                      "with float-float-residual defect correction (FP64 norms)",
            "lattice": [edge] * 3, "precision": "f32 fields, f64 reductions", "n_drugs": 2,
            "cg_rtol": WORKLOAD["rtol_o2"], "maps": f"seeded GRF, correlation length {CORR_LEN:g} sites",
            "l2": f"working set ~{0.9 * (edge / 256) ** 3:.1f} GB per replicate > 129 MB L2; no flush needed"}


# ------------------------------------------------------------- clocks ---
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


def measured_peak_bf16():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    except Exception:
        return 1900.0, "fallback"


# FLOPs of one forward pass of the warm-start network per level-0 site:
# 2 * 27 * C_in * C_out per output site of each 3x3x3 convolution, levels 0..3
NET_FLOPS_PER_SITE = 2 * 27 * (16 * 16 + 32 * 16 + (16 * 32 + 64 * 32) / 8 + (32 * 64 + 64 * 64) / 64
                               + 64 * 64 / 512) + 2 * 16


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record(kernel: str):
    """ncu DRAM bytes per site for a kernel, if captured for the current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[kernel]
    except Exception:
        return None
    if rec.get("source_sha") != kernel_source_sha():
        return None
    return rec.get("dram_bytes_per_site")


def code_lines(text: str):
    """Source lines without // comments, trailing blanks and empty lines
    (a fingerprint of the code that comment edits leave unchanged; no
    string literal in these files holds //)."""
    out = []
    for line in text.splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code:
            out.append(code)
    return out


def kernel_source_sha(root: str = ROOT) -> str:
    """Fingerprint of the hot kernels' code, matched against profiles/traffic.json."""
    h = hashlib.sha256()
    for name in ("hca_internal.cuh", "row_ops.cuh", "pcg.cu", "mg.cu"):
        with open(os.path.join(root, "paper_2105_00448_gb300", "csrc", name), encoding="utf-8") as f:
            h.update("\n".join(code_lines(f.read())).encode())
    return h.hexdigest()[:16]


# ------------------------------------------------------------ oracle ---
def oracle_sample(steps: int, edge: int = SAMPLE_EDGE, seed: int = WORKLOAD["seed"]):
    """Time `steps` oracle steps on an edge^3 sample of the workload (seconds)."""
    from oracle import params as Pm
    from oracle.model import OracleSim
    from synth import make_maps

    # the oracle's own solver (Jacobi-preconditioned textbook CG); the
    # library-only settings (preconditioner) have no oracle counterpart
    params = {k: v for k, v in WORKLOAD.items() if k in Pm.Config.__dataclass_fields__}
    params["seed"] = seed
    cfg = Pm.Config(nx=edge, ny=edge, nz=edge, **params)
    maps = make_maps(edge, edge, edge, corr_len=CORR_LEN, seed=seed)
    sim = OracleSim(cfg, maps.p_cell, maps.perf, maps.p_vessel)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        sim.step(1)
        times.append(time.perf_counter() - t0)
    return times


def cpu_cores_used() -> int:
    # numpy element-wise kernels and the oracle's Python loops run on one thread
    return 1


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_replicate(args):
    """One spawned process: `steps` oracle steps of replicate `seed` (seconds)."""
    steps, edge, seed = args
    return sum(oracle_sample(steps, edge, seed))


def oracle_all_cores(steps: int, edge: int = SAMPLE_EDGE):
    """The oracle on every host core: one independent replicate (seed + i) per
    core in spawned processes (a pool forked after CUDA initialisation would
    hang), timed by the wall clock around the pool.  Returns (site-steps/s,
    processes, wall seconds)."""
    import multiprocessing as mp

    n = host_cores()
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        pool.map(_oracle_replicate, [(0, 8, 0)] * n)   # start-up (imports) outside the timed region
        t0 = time.perf_counter()
        pool.map(_oracle_replicate, [(steps, edge, WORKLOAD["seed"] + i) for i in range(n)])
        wall = time.perf_counter() - t0
    return n * edge ** 3 * steps / wall, n, wall


def cpu_baseline_record(steps: int):
    """The oracle timed on one core and on all host cores (64^3 samples)."""
    times = oracle_sample(steps)
    one = SAMPLE_EDGE ** 3 * len(times) / sum(times)
    allv, n, wall = oracle_all_cores(steps)
    return {"value": one, "unit": "site-steps/s", "cores": cpu_cores_used(), "kind": "oracle",
            "sample": f"{len(times)} coupled steps of the FP64 oracle (Jacobi-PCG) on a {SAMPLE_EDGE}^3 lattice with "
                      f"the 256^3 workload's recipe and parameters, one process ({sum(times):.1f} s)",
            "all_cores": {"value": allv, "unit": "site-steps/s", "cores": n, "kind": "oracle",
                          "sample": f"{n} independent {SAMPLE_EDGE}^3 replicates (seeds {WORKLOAD['seed']}.."
                                    f"{WORKLOAD['seed'] + n - 1}), {steps} steps each, one spawned process per host "
                                    f"core, wall {wall:.1f} s"}}


def step_roofline(prof, steps: int, sites: int, ms_per_step: float, level_fraction: float):
    """Step-level HBM roofline: the method's algorithmic bytes of one step
    (counts of CG iterations, defect-correction sweeps and V-cycles from the
    profiled steps, whose host loops check for convergence before every
    iteration and so launch only V-cycles that run) over the measured step
    time."""
    peak, peak_kind = measured_peak_hbm()
    n_it = prof["pass_a"]["launches"] / steps
    n_dc = prof["residual"]["launches"] / steps
    n_vc = prof["mg_post0"]["launches"] / steps
    terms = {"fixed": STEP_FIXED_B, "defect_correction": STEP_DC_B * n_dc, "cg_iterations": STEP_IT_B * n_it,
             "vcycle_lattice": VCYCLE_LATTICE_B * n_vc, "vcycle_coarse": VCYCLE_COARSE_B * level_fraction * n_vc}
    per_site = sum(terms.values())
    achieved = per_site * sites / (ms_per_step * 1e-3) / 1e9
    design = (STEP_FIXED_B + STEP_DC_B * n_dc + STEP_IT_DESIGN_B * n_it
              + n_vc * (VCYCLE_LATTICE_DESIGN_B + VCYCLE_COARSE_DESIGN_B * level_fraction))
    cg_only = (terms["fixed"] + terms["defect_correction"] + terms["cg_iterations"]) * sites / (ms_per_step * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": achieved / peak, "bytes_per_site": per_site, "terms_bytes_per_site": terms,
            "counts_per_step": {"cg_iterations": n_it, "dc_sweeps": n_dc, "vcycles": n_vc},
            "frac_without_vcycle": cg_only / peak,
            "design_bytes_per_site": design,
            "frac_design_bytes": design * sites / (ms_per_step * 1e-3) / 1e9 / peak,
            "formula": "70 + 13 n_dc + 40 n_it + n_vc (29 + 33 f_coarse) B/site x sites / step time; f_coarse = "
                       "coarse-level sites per lattice site; 29 and 33 B are the V-cycle's minimum with its sweeps "
                       "fused; frac_design_bytes counts what the kernels move (44 B per iteration, "
                       "57 + 69 f_coarse B per V-cycle)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    times = oracle_sample(args.warmup + args.steps)
    timed = times[args.warmup:]
    sites = SAMPLE_EDGE ** 3
    total = sum(timed)
    value = sites * len(timed) / total
    sample = (f"{len(timed)} coupled steps (after {args.warmup} warm-up) of the FP64 oracle on a {SAMPLE_EDGE}^3 "
              f"lattice with the 256^3 workload's recipe and parameters")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "site-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {**workload_config(), "solver": "the FP64 oracle's Jacobi-preconditioned CG (no multigrid)",
                       "precision": "f64", "sample_lattice": [SAMPLE_EDGE] * 3,
                       "l2": "CPU run (host cores): no GPU caches involved"},
            "cpu_baseline": {"value": value, "unit": "site-steps/s", "cores": cpu_cores_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "site-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------- replicas ---
# N > 1: every rank advances its own replicate (seed + rank, its own maps);
# there is no collective on the data path, only the timing barrier and the
# max over ranks of the timed region.
def replica_seed(base: int, rank: int) -> int:
    return base + rank


def max_over_ranks(t_ms: float, dist, device: str) -> float:
    """The job's time: the slowest rank's (all_reduce MAX; identity for one rank)."""
    if dist is None:
        return t_ms
    import torch

    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, sites: int, steps: int, t_ms: float) -> float:
    """Whole-job site-steps/s: every rank's sites over the slowest rank's time."""
    return world * sites * steps / (t_ms / 1e3)


# --------------------------------------------------------------- GPU ---
def coarse_level_fraction(n: int) -> float:
    """Sites of the multigrid coarse levels per lattice site (edges halved,
    rounding up, until a level has at most 512 sites)."""
    tot, m = 0, n
    while m ** 3 > 512:
        m = (m + 1) // 2
        tot += m ** 3
    return tot / n ** 3


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2105_00448_gb300 import hca
    from synth import make_maps

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = args.edge
    sites = n ** 3
    seed = replica_seed(WORKLOAD["seed"], rank)
    params = {**WORKLOAD, "seed": seed}
    maps = make_maps(n, n, n, corr_len=CORR_LEN, seed=seed)
    stream = torch.cuda.Stream()
    cfg = hca.make_config(n, n, n, stream=stream.cuda_stream, **params)
    sim = hca.Sim(cfg, (maps.p_cell, maps.perf, maps.p_vessel))
    level_frac = coarse_level_fraction(n)
    if args.warmup:
        sim.step(args.warmup, allow_noconv=True)
    torch.cuda.synchronize()
    launches0 = sim.launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rc = sim.step(args.steps, allow_noconv=True)
    ev1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    t_ms = ev0.elapsed_time(ev1)
    launches = sim.launches() - launches0
    stats = sim.stats()
    t_ms = max_over_ranks(t_ms, dist, "cuda")
    # Per-kernel device time: the next steps of the same run, driven from the
    # host with CUDA events around every launch on the library's stream.
    hca.hca_profile_enable(sim.handle, True)
    sim.step(args.profile_steps, allow_noconv=True)
    prof = hca.hca_get_profile(sim.handle)
    hca.hca_profile_enable(sim.handle, False)
    sim.close()
    value = job_value(world, sites, args.steps, t_ms)

    # roofline of the dominant kernel class (by summed device time)
    peak, peak_kind = measured_peak_hbm()
    dom = max(BYTES_PER_SITE, key=lambda k: prof[k]["ms"])
    avg_ms = prof[dom]["ms"] / max(1, prof[dom]["launches"])
    bytes_per_launch = BYTES_MIN_PER_SITE[dom] * sites
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    design_bytes = BYTES_PER_SITE[dom] * sites
    tr = traffic_record(dom)
    kernel_names = {"pass_a": "k_pass_a<float>", "pass_b": "k_pass_b<float>", "setup": "k_setup<float>",
                    "residual": "k_dc_residual", "ode": "k_ode<float>", "mg_pre0": "k_mg_pre0<float>",
                    "mg_restrict0": "k_mg_restrict0_rows<float>", "mg_post0": "k_mg_post0<float, true>",
                    "mg_last0": "k_mg_post0<float, false>"}
    roofline = {"bound": "hbm", "kernel": kernel_names[dom], "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": tr * sites if tr is not None else None,
                "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
                "design_bytes_per_launch": design_bytes,
                "frac_design_bytes": design_bytes / (avg_ms * 1e-3) / 1e9 / peak,
                "timing": f"CUDA events around each launch over {args.profile_steps} profiled steps "
                          f"following the timed region"}
    # time share of each kernel class over the timed region
    total_prof = sum(v["ms"] for v in prof.values())
    kernel_share = {k: round(v["ms"] / total_prof, 4) for k, v in prof.items() if v["launches"]}
    line = None
    if rank == 0:
        e2e = run_e2e(args, hca, make_maps, np, torch) if not args.skip_e2e else None
        cpu = None
        if world == 1 and not args.skip_cpu:
            cpu = cpu_baseline_record(args.cpu_steps)
        line = {"metric": metric_name(args.edge), "value": value, "unit": "site-steps/s", "n_gpus": world,
                "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {**workload_config(args.edge), "parallelism": f"replicas{world}" if world > 1 else "single"},
                "roofline": roofline,
                "roofline_step": step_roofline(prof, args.profile_steps, sites, t_ms / args.steps, level_frac),
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks,
                "cg_iterations_per_step": prof["pass_a"]["launches"] / args.profile_steps,
                "last_step": {"o2_iterations": stats["o2_iterations"], "drug_iterations": stats["drug_iterations"][:2],
                              "o2_rel_residual": stats["o2_rel_residual"],
                              "drug_rel_residual": stats["drug_rel_residual"][:2], "counts": stats["counts"]},
                "kernel_time_share": kernel_share, "status": int(rc)}
        if not args.skip_ws and world == 1:
            ws = run_ws_learned(args, hca, make_maps, np, torch)
            line["warm_start_learned"] = ws
            prev, lrn = ws["previous_step_start"], ws["learned_start"]
            line["learned_vs_plain"] = {
                "workload": ws["workload"],
                "o2_iterations_per_step": {"plain": prev["o2_iterations_per_step"],
                                           "learned": lrn["o2_iterations_per_step"]},
                "ms_per_step": {"plain": prev["ms_per_step"], "learned": lrn["ms_per_step"]},
                "step_time_ratio": ws["step_time_ratio"], "net_forward_ms": ws["net_forward"]["ms"],
                "net_tensor_frac": ws["roofline"]["frac"]}
        if args.batch and world == 1:
            line["batched"] = run_batch(args, hca, torch)
        if args.paper_time and world == 1:
            line["paper_time_stepping"] = run_paper_time(args, hca, make_maps, np, torch)
        if args.biopsy2d and world == 1:
            line["biopsy_2d"] = run_biopsy2d(args, hca, torch)
        if args.nonlinear and world == 1:
            line["o2_nonlinear"] = run_nonlinear(args, hca, make_maps, np, torch)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_ws_learned(args, hca, make_maps, np, torch):
    """The learned oxygen warm start on the 256^3 workload at rtol 1e-6: train
    the network on the oxygen solves of two 128^3 runs (seeds 2000, 2001),
    then run the 256^3 workload (seed 1) from the previous-step guess and from
    the network's guess, and time the network's forward pass alone."""
    from paper_2105_00448_gb300 import warmstart

    dev = torch.device("cuda", torch.cuda.current_device())
    n, m = args.edge, args.edge // 2
    ev = {**WORKLOAD, "rtol_o2": 1e-6}
    t0 = time.perf_counter()
    samples = []
    for seed in (2000, 2001):
        mp = make_maps(m, m, m, corr_len=CORR_LEN, seed=seed)
        sim = hca.Sim(hca.make_config(m, m, m, **{**WORKLOAD, "seed": seed}), (mp.p_cell, mp.perf, mp.p_vessel))
        sim.step(1, allow_noconv=True)
        samples += warmstart.collect_samples(sim, args.ws_samples // 2, dev)
        sim.close()
    t_collect = time.perf_counter() - t0
    net_t = hca.Net(m, m, m, trainable=True)
    net_t.set_params(warmstart.init_params(0))
    t0 = time.perf_counter()
    losses = warmstart.train(net_t, hca.make_config(m, m, m), samples, args.ws_iters, 1e-3, seed=1, lr_final=5e-5,
                             w_res=0.03)
    t_train = time.perf_counter() - t0
    params = net_t.params()
    net_t.close()
    del samples
    stream = torch.cuda.Stream()
    net = hca.Net(n, n, n, stream=stream.cuda_stream)
    net.set_params(params)
    # forward alone (features already in place): CUDA events on the network's stream
    x = torch.zeros(n * n * n * 16, dtype=torch.bfloat16, device=dev)
    out = torch.empty(n * n * n, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(2):
            hca.hca_net_forward_x(net.handle, x, out)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            hca.hca_net_forward_x(net.handle, x, out)
        e1.record(stream)
    stream.synchronize()
    fwd_ms = e0.elapsed_time(e1) / reps
    del x, out
    runs = {}
    maps = make_maps(n, n, n, corr_len=CORR_LEN, seed=WORKLOAD["seed"])
    for mode in (hca.HCA_WS_PREV, hca.HCA_WS_LEARNED):
        cfg = hca.make_config(n, n, n, stream=stream.cuda_stream, warm_start=mode, **ev)
        sim = hca.Sim(cfg, (maps.p_cell, maps.perf, maps.p_vessel))
        if mode == hca.HCA_WS_LEARNED:
            sim.set_warm_start_net(net)
        sim.step(args.warmup, allow_noconv=True)
        its, used, ms, r0 = [], 0, 0.0, [0.0, 0.0]
        for _ in range(args.ws_steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(1, allow_noconv=True)
            b.record(stream)
            stream.synchronize()
            ms += a.elapsed_time(b)
            st = sim.stats()
            its.append(st["o2_iterations"])
            used += st["ws_used"]
            r0[0] += st["ws_r0_prev"] / args.ws_steps
            r0[1] += st["ws_r0_learned"] / args.ws_steps
        sim.close()
        runs[mode] = {"o2_iterations_per_step": sum(its) / len(its), "ms_per_step": ms / args.ws_steps,
                      "guess_used_steps": used}
        if mode == hca.HCA_WS_LEARNED:
            runs[mode]["mean_rel_r0"] = {"previous_field": r0[0], "network_guess": r0[1]}
    net.close()
    peak, kind = measured_peak_bf16()
    achieved = NET_FLOPS_PER_SITE * n ** 3 / (fwd_ms * 1e-3) / 1e12
    prev, lrn = runs[hca.HCA_WS_PREV], runs[hca.HCA_WS_LEARNED]
    return {"workload": f"{n}^3 workload, oxygen rtol 1e-6, {args.ws_steps} steps after {args.warmup} warm-up",
            "training": f"{args.ws_iters} Adam steps (MSE + 0.03 residual, lr 1e-3 -> 5e-5) on {args.ws_samples} oxygen solves of two {m}^3 runs "
                        f"(seeds 2000, 2001); collect {t_collect:.1f} s, train {t_train:.1f} s; "
                        f"loss {float(np.mean(losses[:20])):.2e} -> {float(np.mean(losses[-50:])):.2e}",
            "previous_step_start": prev, "learned_start": lrn,
            "o2_iteration_ratio": lrn["o2_iterations_per_step"] / max(1e-9, prev["o2_iterations_per_step"]),
            "step_time_ratio": lrn["ms_per_step"] / max(1e-9, prev["ms_per_step"]),
            "net_forward": {"ms": fwd_ms, "flops": NET_FLOPS_PER_SITE * n ** 3},
            "roofline": {"bound": "tensor", "kernel": "network forward (7 conv launches + pools)",
                         "achieved": achieved, "peak": peak, "peak_kind": kind, "unit": "TFLOP/s",
                         "frac": achieved / peak}}


def run_batch(args, hca, torch):
    """Batched replicates of uneven size in one handle (one launch per kernel
    for the whole batch): sizes drawn from {64, 96, 128, 192}^3, seeds 1000 + r,
    the workload's physics and solver (each replicate its own multigrid
    hierarchy)."""
    from synth import make_maps, replicate_sizes

    sizes = replicate_sizes(args.batch)
    stream = torch.cuda.Stream()
    params = dict(WORKLOAD)
    cfgs, maps = [], []
    for r, n in enumerate(sizes):
        m = make_maps(n, n, n, corr_len=CORR_LEN, seed=1000 + r)
        maps.append((m.p_cell, m.perf, m.p_vessel))
        cfgs.append(hca.make_config(n, n, n, stream=stream.cuda_stream, **{**params, "seed": 1000 + r}))
    sim = hca.Sim(cfgs, maps, batch=True)
    sim.step(args.warmup, allow_noconv=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.batch_steps, allow_noconv=True)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / args.batch_steps
    its = [sim.stats(r) for r in range(len(sizes))]
    sim.close()
    total = sum(n ** 3 for n in sizes)
    return {"workload": f"{len(sizes)} replicates, edges {sorted(set(sizes))} "
                        f"(counts {[sizes.count(v) for v in sorted(set(sizes))]}), one handle",
            "sites": total, "ms_per_step": ms, "value": total / (ms / 1e3), "unit": "site-steps/s",
            "per_replicate_site_steps_s": {str(n): n ** 3 / (ms / 1e3) for n in sorted(set(sizes))},
            "steps": args.batch_steps, "preconditioner": "multigrid",
            "max_cg_iterations_last_step": max(s["o2_iterations"] + sum(s["drug_iterations"]) for s in its)}


def run_paper_time(args, hca, make_maps, np, torch):
    """The paper's time stepping for the drugs (Section 2.4.1): Crank-Nicolson
    with a 1-minute step, i.e. 60 sub-steps per hourly CA step, against the
    workload's one implicit-Euler step; the rest of the step unchanged."""
    n = args.edge
    maps = make_maps(n, n, n, corr_len=CORR_LEN, seed=WORKLOAD["seed"])
    stream = torch.cuda.Stream()
    out = {}
    for name, extra in (("implicit_euler_1", {}), ("crank_nicolson_60", {"drug_scheme": 1, "drug_substeps": 60})):
        sim = hca.Sim(hca.make_config(n, n, n, stream=stream.cuda_stream, **{**WORKLOAD, **extra}),
                      (maps.p_cell, maps.perf, maps.p_vessel))
        sim.step(args.warmup, allow_noconv=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.paper_time_steps, allow_noconv=True)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / args.paper_time_steps
        st = sim.stats()
        sim.close()
        out[name] = {"ms_per_step": ms, "value": n ** 3 / (ms / 1e3), "unit": "site-steps/s",
                     "drug_cg_iterations_last_step": st["drug_iterations"][:2]}
    out["workload"] = (f"{n}^3 workload, {args.paper_time_steps} steps after {args.warmup} warm-up; drugs by one "
                       f"implicit-Euler step of 60 min vs Crank-Nicolson at 1 min (60 sub-steps)")
    return out


def run_biopsy2d(args, hca, torch):
    """The paper's 2-D digital biopsy (Section 3.4): 2 x 10 voxels of
    100 x 100 sites (a 200 x 1000 lattice, nz = 1), piecewise-constant voxel
    maps (synth.biopsy_maps), one week = 168 hourly steps, timed with CUDA
    events; both CA update rules, FP64 and FP32 storage, multigrid-PCG (the
    flat lattice coarsens in-plane)."""
    import numpy as np
    from synth import biopsy_maps

    m = biopsy_maps(seed=11)
    _, ny, nx = m.shape
    stream = torch.cuda.Stream()
    out = {}
    for prec in ("f64", "f32"):
        for mode in (0, 1):
            params = {**WORKLOAD, "precision": prec, "ca_mode": mode, "seed": 11}
            sim = hca.Sim(hca.make_config(nx, ny, 1, stream=stream.cuda_stream, **params), (m.p_cell, m.perf, m.p_vessel))
            c0 = np.bincount(sim.states().reshape(-1), minlength=6)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(args.biopsy_steps, allow_noconv=True)
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1)
            st = sim.stats()
            sim.close()
            out[f"{prec}_{'sync' if mode else 'colour'}"] = {
                "seconds": ms / 1e3, "ms_per_step": ms / args.biopsy_steps,
                "site_steps_per_s": nx * ny * args.biopsy_steps / (ms / 1e3),
                "cancer_cells_start": int(c0[1] + c0[2]), "cancer_cells_end": int(st["counts"][1] + st["counts"][2])}
    out["workload"] = (f"2-D digital biopsy {ny} x {nx} sites (2 x 10 voxels of 100 x 100), {args.biopsy_steps} hourly "
                       f"steps after creation (initial O2 fixed point not timed), O2 + 2 drugs, multigrid-PCG rtol 1e-8")
    out["paper_context"] = "the paper reports about 18 h on 80 CPU cores for one week of this problem (Section 3.4)"
    return out


def run_nonlinear(args, hca, make_maps, np, torch):
    """The linearisation of the oxygen equation (Section 2.4.1) against its
    nonlinear solution on the workload: each step, from the same lattice and
    previous K, one handle takes the lagged-linearised solve and a second
    handle (o2_nonlinear) iterates it to the fixed point; the relative L2
    difference of the two fields is the linearisation error the paper bounds
    by 0.03 %.  Both O2 solves are timed with CUDA events."""
    n = args.edge
    maps = make_maps(n, n, n, corr_len=CORR_LEN, seed=WORKLOAD["seed"])
    stream = torch.cuda.Stream()
    args3 = (n, n, n, maps.p_cell, maps.perf, maps.p_vessel)
    lin = hca.Sim(hca.make_config(n, n, n, stream=stream.cuda_stream, **WORKLOAD), args3[3:])
    nl = hca.Sim(hca.make_config(n, n, n, stream=stream.cuda_stream, **{**WORKLOAD, "o2_nonlinear": 1}), args3[3:])
    lin.step(args.warmup, allow_noconv=True)
    st = torch.empty((n, n, n), dtype=torch.uint8, device="cuda")
    K = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    Kn = torch.empty_like(K)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    rel, mx, t_lin, t_nl, picard = [], [], [], [], []
    for _ in range(args.nl_steps):
        hca.hca_read_states(lin.handle, 0, st)
        hca.hca_read_fields(lin.handle, 0, hca.FIELD_O2, K)
        torch.cuda.synchronize()
        hca.hca_write_states(nl.handle, 0, st)
        hca.hca_write_fields(nl.handle, 0, hca.FIELD_O2, K)
        ev[0].record(stream)
        nl.stage(hca.STAGE_O2, allow_noconv=True)
        ev[1].record(stream)
        lin.stage(hca.STAGE_O2, allow_noconv=True)
        ev[2].record(stream)
        stream.synchronize()
        t_nl.append(ev[0].elapsed_time(ev[1]))
        t_lin.append(ev[1].elapsed_time(ev[2]))
        picard.append(nl.stats()["picard_iterations"])
        hca.hca_read_fields(lin.handle, 0, hca.FIELD_O2, K)
        hca.hca_read_fields(nl.handle, 0, hca.FIELD_O2, Kn)
        torch.cuda.synchronize()
        d = (K.double() - Kn.double())
        rel.append(float(d.norm() / Kn.double().norm()))
        mx.append(float(d.abs().max() / Kn.double().abs().max()))
        lin.stage(hca.STAGE_DRUGS | hca.STAGE_ODE | hca.STAGE_CA | hca.STAGE_ADVANCE, allow_noconv=True)
    stream.synchronize()
    lin.close()
    nl.close()
    return {"workload": f"{n}^3 workload, {args.nl_steps} steps after {args.warmup} warm-up; nonlinear: Picard "
                        f"iteration of the linearisation to ||dK||/||K|| <= {WORKLOAD['picard_tol']:g} "
                        f"(FP32 fields)",
            "linearisation_rel_l2": {"max": max(rel), "mean": sum(rel) / len(rel)},
            "linearisation_rel_max_norm": max(mx), "paper_bound_rel": 3e-4,
            "o2_ms_linearised": sum(t_lin) / len(t_lin), "o2_ms_nonlinear": sum(t_nl) / len(t_nl),
            "picard_iterations_mean": sum(picard) / len(picard)}


def run_e2e(args, hca, make_maps, np, torch):
    """Same metric through the public C ABI with host buffers: create from
    pinned host maps, then per step one hca_step and a read of the states and
    the oxygen field back to pinned host memory, all inside the timed region."""
    n = args.edge
    sites = n ** 3
    maps = make_maps(n, n, n, corr_len=CORR_LEN, seed=WORKLOAD["seed"])
    pin = lambda a: torch.from_numpy(a).pin_memory()
    pc, pf, pv = pin(maps.p_cell), pin(maps.perf), pin(maps.p_vessel)
    states = torch.empty((n, n, n), dtype=torch.uint8).pin_memory()
    oxy = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
    steps = args.e2e_steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cfg = hca.make_config(n, n, n, **WORKLOAD)
    h = hca.hca_create(cfg, pc, pf, pv)
    for _ in range(steps):
        rc = hca.hca_step(h, 1)
        if rc not in (hca.HCA_OK, hca.HCA_ERR_NOCONV):
            raise hca.HcaError(rc, "hca_step")
        hca.hca_read_states(h, 0, states)
        hca.hca_read_fields(h, 0, hca.FIELD_O2, oxy)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    hca.hca_destroy(h)
    return {"value": sites * steps / elapsed, "unit": "site-steps/s",
            "h2d_bytes_per_step": 3 * 4 * sites / steps, "d2h_bytes_per_step": sites * (1 + 4),
            "steps": steps, "includes": "create (map upload + initial O2 fixed point) and per-step state/O2 readback"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--edge", type=int, default=N_EDGE, help=argparse.SUPPRESS)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-ws", action="store_true",
                    help="skip training and measuring the learned oxygen warm start (about a minute)")
    ap.add_argument("--ws-samples", type=int, default=48)
    ap.add_argument("--ws-iters", type=int, default=4000)
    ap.add_argument("--ws-steps", type=int, default=10)
    ap.add_argument("--batch", type=int, default=0,
                    help="also time N batched replicates of uneven size (e.g. 64)")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--nonlinear", action="store_true",
                    help="also measure the oxygen linearisation error against the nonlinear solve")
    ap.add_argument("--nl-steps", type=int, default=4)
    ap.add_argument("--paper-time", action="store_true",
                    help="also time the drugs with Crank-Nicolson at 1-minute sub-steps")
    ap.add_argument("--paper-time-steps", type=int, default=3)
    ap.add_argument("--biopsy2d", action="store_true",
                    help="also time one week of the 2-D digital biopsy (200 x 1000 lattice)")
    ap.add_argument("--biopsy-steps", type=int, default=168)
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        raise SystemExit("need --steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
