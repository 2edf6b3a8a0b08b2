#!/usr/bin/env python
"""Benchmark of the Magnus-Lanczos TDKS step on one GB300 (or N replicas).

A step is one predictor-corrector second-order Magnus step (two adaptive
Lanczos exponentials, two Poisson solves, densities, LDA, dipole) of the
16-orbital molecule workload: [-16,16]^3 bohr, 16^3 hexahedra, p = 6
(857,375 interior DoF), 8 erf-pseudopotential atoms, Hartree + LDA, dt = 0.1,
Krylov tolerance 1e-10.  Metric: orbital-steps/s (value) and H-psi GDoF/s.

  python bench.py [--gpus N --steps K --warmup W] [--prec fp64|fp32]
  python bench.py --impl reference ...    # the CPU oracle on a bounded sample
  python bench.py --horizon 500           # the molecule's full 500 steps per precision
  python bench.py --apply-only --prec df64  # standalone Hbar applications
  python bench.py --stage-only            # one contraction stage: CUDA cores vs tensor cores
  python bench.py --stage-study           # dipole error with single element-kernel stages in FP32

Inputs are synthetic and resident in HBM before the timed region; the working
set (Krylov basis, 16 x 64 x 857k complex128 = 14 GB) is far larger than L2.
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

METRIC = ("orbital-steps/s & HΨ GDoF/s, mixed/batched vs FP64 on 1 GB300 at dipole "
          "err≤1e-6")
WORKLOAD = ("molecule_erf8_16x16x16_p6: [-16,16]^3 bohr, 16^3 hexahedra, p=6, 857,375 DoF, "
            "16 orbitals, 8 erf atoms, Hartree+LDA, kick 1e-3 x, dt 0.1, Krylov tol 1e-10")
BF16_NOTE = ("bfloat16 operands with FP32 products and sums, emulated on the CUDA cores to "
             "measure the accuracy of a BF16 tensor-core contraction: the rate is not that of a "
             "tensor-core kernel")
MIXED_NOTE = ("relaxed precision inside each Lanczos exponential: double-float contractions "
              "until every active orbital's a-posteriori estimate (Eq. 38) is <= 1e8 x tol, FP32 "
              "contractions for the remaining products; double-float recombination and density")
PROFILES = {"fp64": os.path.join(ROOT, "profiles", "hbar_fp64_molecule.txt"),
            "df64": os.path.join(ROOT, "profiles", "hbar_df64_molecule.txt")}
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "df64", "bf16", "mixed"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", dest="mixed", action="store_false",
                    help="skip the FP32 / DF64 comparison runs")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 64-system batched runs")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--no-graded", dest="graded", action="store_false",
                    help="skip the graded p = 8 all-electron-like runs")
    ap.add_argument("--graded-steps", type=int, default=2)
    ap.add_argument("--no-nonlocal", dest="nonlocal_kb", action="store_false",
                    help="skip the molecule run with Kleinman-Bylander projectors")
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false",
                    help="skip the adjoint-gradient timing on the pulse workload")
    ap.add_argument("--horizon", type=int, default=0,
                    help="run the molecule workload for this many steps per contraction type "
                         "(its full horizon is 500) and report the dipole differences")
    ap.add_argument("--host-loop", action="store_true",
                    help="host-driven Lanczos loop (for ncu launch lists: ncu cannot profile the "
                         "kernel nodes of graphs with conditional nodes; the kernels are the same)")
    ap.add_argument("--stage-only", action="store_true",
                    help="time the contraction-stage probe (CUDA cores vs tensor cores) only")
    ap.add_argument("--batch-profile", action="store_true",
                    help="the 64-system batch (--prec fp64, df64 or mixed): one half-step "
                         "exponential re-run kernel by kernel inside the NVTX range "
                         "batch_profile_pass (for an ncu launch list)")
    ap.add_argument("--stage-study", action="store_true",
                    help="dipole error vs the oracle series with single stages of the double-float "
                         "element kernel in FP32 (which stages need compensation)")
    ap.add_argument("--apply-only", action="store_true",
                    help="time standalone Hbar applications (16 orbitals) instead of steps")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


# ----------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and reference arm)
# ----------------------------------------------------------------------------
# Jacobi-PCG iterations of one oracle Poisson solve on the molecule workload (tol
# 1e-10, warm-started from the previous solution; a cold start takes 550): measured
# once with the oracle's own solver, which takes ~80 s per solve on one core.
ORACLE_CG_ITERS_PER_SOLVE = 386
# batched runs: Krylov cap of the systems whose exponentials restart at k_max 64
BATCH_KCAP = 128
ORACLE_SAMPLE_DESC = (
    "oracle (numpy, 1 pinned thread), molecule workload, extrapolated: each sample step "
    "times 2 Lanczos iterations of one orbital (Hbar apply + recurrence), the density of one "
    "orbital and one Jacobi-PCG iteration of the Poisson solve (stiffness apply + vector "
    "updates) with the oracle's own functions; one orbital-step = (k_half + k_full) Lanczos "
    "iterations + 2 densities + (2 solves x %d PCG iterations + 2 x (load vector, "
    "interpolation, LDA)) / 16 orbitals; k_half, k_full of orbital 0 come from a set-up run "
    "of the oracle's exponentials" % ORACLE_CG_ITERS_PER_SOLVE)
ATOM_RUN_DESC = ("oracle (numpy, 1 pinned thread), atom workload (6^3 hexahedra, p = 4, 1 "
                 "orbital), all 100 steps from the oracle ground state after the 1e-3 kick, "
                 "Poisson and LDA included: measured, not extrapolated")


def _pin_one_core(k: int):
    try:
        cores = sorted(os.sched_getaffinity(0))
        os.sched_setaffinity(0, {cores[min(k, len(cores) - 1)]})
        return True
    except (AttributeError, OSError):
        return False


def host_info() -> dict:
    import platform
    info = {"machine": platform.machine(), "logical_cpus": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Vendor ID", "CPU max MHz"):
                info[k.strip()] = v.strip()
    except Exception:
        pass
    return info


def oracle_sample_main(spec: str):
    """Runs in a fresh single-threaded interpreter pinned to one core; prints JSON lines."""
    import numpy as np
    a = json.loads(spec)
    pinned = _pin_one_core(a.get("core", 1))
    import synth
    from oracle import hamiltonian as ham
    from oracle import xc
    from oracle.lanczos import expm_lanczos
    from oracle.mesh import Mesh
    from oracle.propagate import Propagator, kick
    if a["mode"] == "atom":
        cfg = synth.config1()
        mesh = Mesh.from_config(cfg)
        gs = np.load(os.path.join(ROOT, "tests", "golden", f"gs_{cfg.name}.npz"))
        prop = Propagator.from_config(cfg, mesh, cg_tol=1e-13)
        t0 = time.perf_counter()
        psi = kick(mesh, gs["psibar"].astype(complex), cfg.kick, cfg.kick_dir)
        prop.init(psi)
        for _ in range(cfg.n_steps):
            psi, _, _ = prop.magnus_step(psi, cfg.dt)
        wall = time.perf_counter() - t0
        print(json.dumps({"atom": True, "steps": cfg.n_steps, "wall_s": wall, "pinned": pinned,
                          "orbital_steps_per_s": cfg.n_orb * cfg.n_steps / wall}), flush=True)
        return
    cfg = synth.config2()
    mesh = Mesh.from_config(cfg)
    prop = Propagator.from_config(cfg, mesh)
    psi = synth.smooth_orbitals(tuple(mesh.Ni), cfg.n_orb, seed=a["seed"])
    psi = kick(mesh, psi, cfg.kick, cfg.kick_dir)
    rho = ham.density(mesh, psi, cfg.occ)
    v = prop.v_nuc + xc.v_xc(rho)
    f = lambda x: ham.apply_H(mesh, v, x)
    # set-up: Krylov dimensions of both exponentials for orbital 0
    _, i_half = expm_lanczos(f, psi[:1], 0.5 * cfg.dt, cfg.tol, cfg.k_max)
    _, i_full = expm_lanczos(f, psi[:1], cfg.dt, cfg.tol, cfg.k_max)
    k_half, k_full = sum(i_half["k"][0]), sum(i_full["k"][0])
    # per-solve field work shared by all orbitals: load vector, interpolation, LDA
    t0 = time.perf_counter()
    b = 4.0 * np.pi * ham.load_vector(mesh, rho)
    ham.interp_q(mesh, b)
    xc.v_xc(rho)
    t_fields = time.perf_counter() - t0
    diag = ham.stiffness_diag(mesh)
    print(json.dumps({"setup": True, "k_half": k_half, "k_full": k_full, "pinned": pinned}), flush=True)
    x = np.zeros_like(b)
    r = b.copy()
    z = r / diag
    pv = z.copy()
    rz = r @ z
    for s in range(a["steps"]):
        o = s % cfg.n_orb
        t0 = time.perf_counter()
        expm_lanczos(f, psi[o:o + 1], 0.5 * cfg.dt, cfg.tol, cfg.k_max, k_fixed=2)
        t1 = time.perf_counter()
        ham.density(mesh, psi[o:o + 1], cfg.occ[o:o + 1])
        t2 = time.perf_counter()
        # one iteration of the oracle's Jacobi PCG (oracle/poisson.py pcg), same operations
        Ap = ham.stiffness_apply(mesh, pv)
        alpha = rz / (pv @ Ap)
        x += alpha * pv
        r -= alpha * Ap
        np.linalg.norm(r)
        z = r / diag
        rz_new = r @ z
        pv = z + (rz_new / rz) * pv
        rz = rz_new
        t3 = time.perf_counter()
        t_lanczos = (t1 - t0) / 2
        t_orb_step = ((k_half + k_full) * t_lanczos + 2 * (t2 - t1)
                      + (2 * ORACLE_CG_ITERS_PER_SOLVE * (t3 - t2) + 2 * t_fields) / cfg.n_orb)
        print(json.dumps({"step": s, "t_sample": t3 - t0, "orbital_steps_per_s": 1.0 / t_orb_step,
                          "t_lanczos_iter": t_lanczos, "t_density": t2 - t1, "t_cg_iter": t3 - t2,
                          "k_half": k_half, "k_full": k_full}), flush=True)


def oracle_cmd(spec: dict):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               PYTHONPATH=ROOT)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-sample", json.dumps(spec)]
    return cmd, env


def run_oracle_sample(steps: int, seed: int = 1, core: int = 1):
    cmd, env = oracle_cmd({"mode": "molecule", "steps": steps, "seed": seed, "core": core})
    r = subprocess.run(cmd, env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-2000:])
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


class OracleBackground:
    """The CPU-baseline oracle runs (molecule sample, full atom run), started before the
    first GPU call as separate single-threaded processes pinned to their own cores, so
    that they run while the GPU sections do."""

    def __init__(self, sample_steps: int):
        self.procs = {}
        for name, spec in (("molecule", {"mode": "molecule", "steps": sample_steps, "seed": 1, "core": 2}),
                           ("atom", {"mode": "atom", "core": 3})):
            cmd, env = oracle_cmd(spec)
            self.procs[name] = subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE,
                                                stderr=subprocess.PIPE, text=True)

    def results(self):
        out = {}
        for name, p in self.procs.items():
            so, se = p.communicate()
            if p.returncode != 0:
                out[name] = {"error": se[-500:]}
                continue
            out[name] = [json.loads(l) for l in so.splitlines() if l.startswith("{")]
        return out


def reference_arm(args, rank: int):
    if rank != 0:
        return
    t0 = time.perf_counter()
    recs = run_oracle_sample(args.warmup + args.steps)
    wall = time.perf_counter() - t0
    timed = [r for r in recs if "step" in r][args.warmup:]
    rates = [r["orbital_steps_per_s"] for r in timed]
    value = statistics.mean(rates)
    tsum = sum(r["t_sample"] for r in timed)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "orbital-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # a step of this arm is one timed sample (see cpu_baseline.sample), not a full
        # 16-orbital Magnus step: ms_per_step is the sample's measured duration
        "ms_per_step": 1e3 * tsum / len(timed), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "contractions": "fp64", "parallelism": "1 host core",
                   "sample": "2 Lanczos iterations + 1 density + 1 PCG iteration per step, "
                             "orbital-step time extrapolated"},
        "ms_per_orbital_step_extrapolated": 1e3 / value,
        "cpu_baseline": {"value": value, "unit": "orbital-steps/s", "cores": 1, "kind": "oracle",
                         "how": "extrapolated from timed samples", "sample": ORACLE_SAMPLE_DESC,
                         "timed_sample_s": tsum, "wall_s_incl_setup": wall, "host": host_info()},
        "e2e": {"value": value, "unit": "orbital-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, device_index: int):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        self.f = os.fdopen(fd, "w")
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={SMI_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:      # the sampler this object started, by its PID
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.f.close()

    def summary(self):
        if self.proc is None:
            os.unlink(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def profile_traffic(prec: str):
    """dram bytes per Hbar launch from the committed ncu summary, if the kernel
    source has not changed since the capture."""
    path = PROFILES.get(prec)
    if not path or not os.path.exists(path):
        return None
    src = open(os.path.join(ROOT, "paper_1810_13130_gb300", "csrc", "elements.cu"), "rb").read()
    h = hashlib.sha256(src).hexdigest()[:16]
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("elements_cu_sha256_16") != h:
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def replica_throughput(units_local: float, t_local: float, dist=None, device: str = "cpu"):
    """Whole-job throughput of N replicas (one workload per rank, no data exchange):
    the units of all ranks over the slowest rank's time.  Returns (value, t_max).
    With dist=None (one process) it is units / t."""
    if dist is None:
        return units_local / t_local, t_local
    import torch
    world = dist.get_world_size()
    tt = torch.tensor([t_local], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    t = tt.item()
    return world * units_local / t, t


HOST_LOOP = False   # --host-loop


def _run_steps(tdks, torch, cfg, prec, steps, warmup, local_rank, psi0, dist=None, timing=True):
    """K timed Magnus steps of a fresh context from psi0 (kicked on the device)."""
    ctx = tdks.Context.from_config(cfg)
    ctx.set_cg(1e-10)
    if HOST_LOOP:
        ctx.set_device_loop(False)
    psi = torch.from_numpy(psi0).cuda()
    ctx.kick(psi, cfg.kick, cfg.kick_dir)
    ctx.d_init = ctx.init_propagation(psi)
    stream = torch.cuda.current_stream()

    def step():
        return ctx.magnus_step(psi, cfg.dt, tol=cfg.tol, k_max=cfg.k_max, prec=prec)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ctx.get_counters(reset=True)
    ctx.set_timing(timing)
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        for _ in range(steps):
            stats.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    t = ev0.elapsed_time(ev1) * 1e-3
    cnt = ctx.get_counters(reset=True)
    ctx.set_timing(False)
    return ctx, psi, t, stats, cnt, clk.summary()


GOLDEN_WORKLOADS = ("config1", "config_mid")


def _golden_dipoles(tdks, torch, cfg, prec, tile=0, f32_stages=0):
    """The CUDA path over a committed oracle dipole series (tests/golden): the same
    ground state, kick, steps and tolerances.  Returns (dipoles, oracle dipoles)."""
    import numpy as np
    s = np.load(os.path.join(ROOT, "tests", "golden", f"series_{cfg.name}.npz"))
    gs = np.load(os.path.join(ROOT, "tests", "golden", f"gs_{cfg.name}.npz"))
    ctx = tdks.Context.from_config(cfg)
    ctx.set_cg(float(s["cg_tol"]))
    if tile:
        ctx.set_apply_tile(tile)
    if f32_stages:
        ctx.set_f32_stages(f32_stages)
    g = torch.from_numpy(gs["psibar"].astype(complex)).cuda()
    ctx.kick(g, float(s["kappa"]), tuple(s["kick_dir"]))
    d = [ctx.init_propagation(g)]
    for _ in range(int(s["n_steps"])):
        d.append(ctx.magnus_step(g, float(s["dt"]), tol=float(s["tol"]), k_max=int(s["k_max"]),
                                 prec=prec)["dipole"])
    ctx.close()
    return np.array(d), s["dipole"]


def dipole_err(d, ref) -> float:
    """max_n |d(t_n) - d_ref(t_n)| / max_n |d_ref(t_n) - d_ref(0)| (Sec. V, Eq. 30)."""
    import numpy as np
    return float(np.abs(np.asarray(d) - ref).max() / np.abs(ref - ref[0]).max())


def err_vs_oracle(tdks, torch, prec) -> dict:
    """Dipole error against the oracle series of the atom (100 steps) and the 8-orbital
    molecule (50 steps, 8 orbitals per element-kernel CTA as in the benchmark)."""
    import synth
    out = {}
    for name in GOLDEN_WORKLOADS:
        cfg = getattr(synth, name)()
        if not os.path.exists(os.path.join(ROOT, "tests", "golden", f"series_{cfg.name}.npz")):
            continue
        d, ref = _golden_dipoles(tdks, torch, cfg, prec, tile=8 if cfg.n_orb > 1 else 0)
        out[cfg.name] = dipole_err(d, ref)
    out["max"] = max(out.values())
    return out


STAGE_NAMES = ("interp z", "interp y", "interp x", "kinetic x", "kinetic y", "kinetic z",
               "interp^T z", "interp^T y", "interp^T x", "pointwise V + kinetic", "gathered input",
               "element results")


def stage_study(tdks, torch) -> dict:
    """Dipole error against the oracle series (atom 100 steps, 8-orbital molecule 50
    steps) of the double-float step with one stage, or one group of stages, of the
    element kernel in FP32 arithmetic (tdks_set_f32_stages), beside plain DF64 and the
    FP32 kernel."""
    import synth
    cases = [("none (DF64)", 0)] + [(n, 1 << i) for i, n in enumerate(STAGE_NAMES)]
    cases += [("interp (forward)", 0x7), ("kinetic", 0x38), ("interp^T", 0x1c0),
              ("interp, both directions", 0x1c7), ("all contractions", 0x1ff), ("all", 0xfff)]
    rows = []
    for label, mask in cases:
        row = {"stages_fp32": label, "mask": mask}
        for name in GOLDEN_WORKLOADS:
            cfg = getattr(synth, name)()
            d, ref = _golden_dipoles(tdks, torch, cfg, tdks.DF64, tile=8 if cfg.n_orb > 1 else 0,
                                     f32_stages=mask)
            row[cfg.name] = float(f"{dipole_err(d, ref):.3g}")
        rows.append(row)
    row = {"stages_fp32": "FP32 kernel (TDKS_FP32)", "mask": None}
    for name in GOLDEN_WORKLOADS:
        cfg = getattr(synth, name)()
        d, ref = _golden_dipoles(tdks, torch, cfg, tdks.FP32, tile=8 if cfg.n_orb > 1 else 0)
        row[cfg.name] = float(f"{dipole_err(d, ref):.3g}")
    rows.append(row)
    return {"mode": "stage_study", "bound": 1e-6, "rows": rows}


def batch_profile(tdks, torch, prec_name: str) -> dict:
    """The 64-system batch after tuning, one step at k_max 64, the Krylov caps and one
    more step (graphs, not profiled), then the half-step exponential of the current state
    once more outside the graph, kernel group by kernel group, inside the NVTX range
    batch_profile_pass; with the phase times of the last step (CUDA events)."""
    import synth
    prec = {"fp64": tdks.FP64, "df64": tdks.DF64, "mixed": tdks.MIXED}[prec_name]
    cfgs, dts, dirs = synth.config5()
    b = tdks.Batch(cfgs, dts, prec=prec, tol=1e-10, k_max=64)
    for k, c in enumerate(cfgs):
        psi = synth.smooth_orbitals(tuple((len(c.X) - 1) * c.p - 1 for _ in range(3)), c.n_orb, seed=500 + k)
        b.set_orbitals(k, torch.from_numpy(psi).cuda())
    b.kick([c.kick for c in cfgs], dirs)
    b.init()
    b.tune(reps=2)
    b.steps(1)
    b.tune_kmax(BATCH_KCAP)
    b.set_timing(True)
    b.steps(1)
    phases = b.phase_ms()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("batch_profile_pass")
    groups = b.profile_pass()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    b.close()
    return {"mode": "batch_profile", "prec": prec_name, "phases_ms": phases,
            "half_step_groups_ms": groups}


def batched_err_vs_oracle(tdks, torch, prec) -> dict:
    """The batched engine on the two oracle-series workloads advanced together."""
    import numpy as np
    import synth
    cfgs = [c for c in (getattr(synth, n)() for n in GOLDEN_WORKLOADS)
            if os.path.exists(os.path.join(ROOT, "tests", "golden", f"series_{c.name}.npz"))]
    ser = [np.load(os.path.join(ROOT, "tests", "golden", f"series_{c.name}.npz")) for c in cfgs]
    n = min(int(s["n_steps"]) for s in ser)
    b = tdks.Batch(cfgs, [float(s["dt"]) for s in ser], prec=prec, tol=1e-10, k_max=64)
    for k, c in enumerate(cfgs):
        gs = np.load(os.path.join(ROOT, "tests", "golden", f"gs_{c.name}.npz"))
        b.set_orbitals(k, torch.from_numpy(gs["psibar"].astype(complex)).cuda())
    b.kick([float(s["kappa"]) for s in ser], [tuple(s["kick_dir"]) for s in ser])
    d0 = b.init()
    d1 = b.steps(1)
    b.tune_kmax(BATCH_KCAP)          # as in the timed runs (no system here restarts at 64)
    d = np.concatenate([d0[None], d1, b.steps(n - 1)])
    b.close()
    out = {c.name: dipole_err(d[:, k], ser[k]["dipole"][: n + 1]) for k, c in enumerate(cfgs)}
    out["max"] = max(out.values())
    out["steps"] = n
    return out


def measured_peaks(tdks, local_rank: int) -> dict:
    """FP64 and FP32 FMA rates of this GPU, measured now (tdks_fma_probe), with the SM
    clocks sampled while the probe runs."""
    out = {}
    for name, prec, iters in (("fp64", tdks.FP64, 8192), ("fp32", tdks.FP32, 262144)):
        tdks.fma_probe(prec, 8, iters // 8, 2)                 # warm-up
        with ClockSampler(local_rank) as clk:
            t_end = time.perf_counter() + 1.0
            best = 0.0
            while time.perf_counter() < t_end:
                tf, ms = tdks.fma_probe(prec, 8, iters, 5)
                best = max(best, tf)
        out[name] = {"tflops": best, "clocks": clk.summary()}
    out["how"] = ("tdks_fma_probe: 8 CTAs/SM x 256 threads x 8 independent FMA chains, 5 launches "
                  "per CUDA-event timing, best over ~1 s of repeats")
    return out


def ours(args, rank: int, world: int, local_rank: int):
    import numpy as np
    # the CPU-baseline oracle processes start before the first GPU call
    bg = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        bg = OracleBackground(sample_steps=3)
    import torch
    import synth
    from paper_1810_13130_gb300 import tdks

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    precs = {"fp64": tdks.FP64, "fp32": tdks.FP32, "df64": tdks.DF64, "bf16": tdks.BF16,
             "mixed": tdks.MIXED}
    prec = precs[args.prec]
    peaks = measured_peaks(tdks, local_rank)
    cfg = synth.config2()
    psi0 = synth.smooth_orbitals(tuple(n * cfg.p - 1 for n in (cfg.nx, cfg.ny, cfg.nz)),
                                 cfg.n_orb, seed=1)
    ctx, psi, t, stats, cnt, clocks = _run_steps(tdks, torch, cfg, prec, args.steps, args.warmup,
                                                 local_rank, psi0, dist)
    n_int = ctx.n_int
    d_init = ctx.d_init
    applies = sum(s["applies"] for s in stats)
    value, t = replica_throughput(cfg.n_orb * args.steps, t, dist, "cuda")
    hpsi = world * n_int * applies / t / 1e9
    # roofline of the dominant kernel (the Hbar element kernel, timed inside the region)
    P1 = cfg.p + 1
    flops_unit = 36 * P1 ** 4 + 24 * P1 ** 3
    apply_s = cnt["apply_ms"] * 1e-3
    achieved_tf = cnt["apply_elem_orb"] * flops_unit / apply_s / 1e12 if apply_s > 0 else None
    pk = peaks["fp64" if args.prec == "fp64" else "fp32"]["tflops"]
    n_apply_calls = cnt["apply_launches"]          # one element launch per Hbar application
    avg_launch_ms = cnt["apply_ms"] / max(cnt["apply_launches"], 1)
    hbm_bytes = applies * n_int * 32.0 + n_apply_calls * ctx.n_elem * P1 ** 3 * 8.0
    traffic = profile_traffic(args.prec)
    roofline = {"bound": "alu",
                "kernel": f"k_hbar<P1={P1},{args.prec}> element kernel (timed with its gather assembly "
                          "and the fused Lanczos update: achieved is a lower bound for the element kernel)",
                "achieved": achieved_tf, "peak": pk, "unit": "TFLOP/s",
                "frac": (achieved_tf / pk) if achieved_tf else None, "traffic": traffic,
                "peak_source": ("measured in this run: FP64 FMA rate (tdks_fma_probe)" if args.prec == "fp64"
                                else "measured in this run: FP32 FMA rate (tdks_fma_probe)"),
                "flops_per_elem_orbital": flops_unit,
                "avg_launch_ms": avg_launch_ms, "apply_share_of_step": apply_s / t,
                "hbm_GBps_algorithmic": hbm_bytes / apply_s / 1e9 if apply_s > 0 else None,
                "hbm_frac_of_measured_6790": (hbm_bytes / apply_s / 1e9 / 6790.0) if apply_s > 0 else None}
    line = {"metric": METRIC, "value": value, "unit": "orbital-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "contractions": args.prec, "parallelism": f"replicas x{world}",
                       "l2": "working set > L2 (Krylov basis 14 GB, orbitals 219 MB)"},
            "hpsi_gdofs": hpsi, "applies_per_step": applies / args.steps,
            "krylov": {"k_half_max": max(s["k_half_max"] for s in stats),
                       "k_full_max": max(s["k_full_max"] for s in stats),
                       "substeps": sum(s["substeps"] for s in stats),
                       "cg_iters_per_solve": statistics.mean(c for s in stats for c in s["cg_iters"])},
            "roofline": roofline, "peaks_measured": peaks, "gpu_launches": cnt["launches"],
            "clocks": clocks}
    # end to end through the public C-ABI with host buffers (pinned), every step:
    # H2D of the orbitals + field, the step, D2H of the orbitals + dipole
    if args.e2e_steps > 0:
        hin = psi.cpu().pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        E = np.zeros(6)
        # one untimed call: the first allocates the device copy of the orbitals and
        # captures the Lanczos-loop graphs for its address
        ctx.propagate_host(hin, hout, 1, cfg.dt, E, init=False, tol=cfg.tol, k_max=cfg.k_max, prec=prec)
        hin, hout = hout, hin
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx.propagate_host(hin, hout, 1, cfg.dt, E, init=False, tol=cfg.tol, k_max=cfg.k_max,
                               prec=prec)
            hin, hout = hout, hin
        te = time.perf_counter() - t0
        nb = cfg.n_orb * n_int * 16
        line["e2e"] = {"value": world * cfg.n_orb * args.e2e_steps / te, "unit": "orbital-steps/s",
                       "h2d_bytes_per_step": nb + 48, "d2h_bytes_per_step": nb + 24,
                       "steps": args.e2e_steps}
    ctx.close()
    speedups = {}
    # mixed precision: same workload and step count per contraction type; dipole error
    # against the committed FP64 oracle series (atom 100 steps, 8-orbital molecule 50
    # steps), relative to the induced dipole, and against the FP64 path over the timed
    # steps of this workload
    if args.mixed and args.prec == "fp64":
        dm64 = np.array([s["dipole"] for s in stats])
        ind_m = float(np.abs(dm64[:, 0] - d_init[0]).max())
        mixed = {"dipole_err_vs_oracle": "max over the oracle series (tests/golden: atom 100 steps, "
                                         "8-orbital molecule 50 steps) of max_n |d - d_oracle| / "
                                         "max_n |d_oracle - d_oracle(0)|",
                 "dipole_err_molecule": f"the {args.steps} timed steps of this workload (after "
                                        f"{args.warmup} warm-up steps): max |d_x - d_x,fp64| / "
                                        "max |d_x,fp64 - d_x,fp64(0)|",
                 "fp64": {"dipole_err_vs_oracle": err_vs_oracle(tdks, torch, tdks.FP64)}}
        for name in ("df64", "mixed", "fp32", "bf16"):
            try:
                c2, _, t2, st2, cnt2, _ = _run_steps(tdks, torch, cfg, precs[name], args.steps, args.warmup,
                                                     local_rank, psi0, dist, timing=False)
                c2.close()
                v2 = world * cfg.n_orb * args.steps / t2
                dmm = np.array([s["dipole"] for s in st2])
                mixed[name] = {"value": v2, "unit": "orbital-steps/s",
                               "ms_per_step": 1e3 * t2 / args.steps, "speedup_vs_fp64": v2 / value,
                               "dipole_err_vs_oracle": err_vs_oracle(tdks, torch, precs[name]),
                               "dipole_rel_err_molecule": float(np.abs(dmm[:, 0] - dm64[:, 0]).max() / ind_m)}
                if name == "mixed":
                    mixed[name]["fp32_share_of_applies"] = (cnt2["apply_launches_fp32"] /
                                                            max(cnt2["apply_launches"], 1))
                    mixed[name]["note"] = MIXED_NOTE
            except tdks.TDKSError as e:      # reported, not fatal: the bench line still prints
                mixed[name] = {"error": str(e)}
        mixed["bf16"]["note"] = BF16_NOTE
        line["mixed"] = mixed
        for name in ("df64", "mixed", "fp32"):
            if "speedup_vs_fp64" in mixed[name]:
                e = mixed[name]["dipole_err_vs_oracle"]["max"]
                speedups[name] = {"speedup_vs_fp64": round(mixed[name]["speedup_vs_fp64"], 3),
                                  "dipole_err_vs_oracle": float(f"{e:.3g}"), "meets_1e-6": e <= 1e-6}
    if args.graded and args.prec == "fp64":
        line["graded"] = graded_section(tdks, torch, args, local_rank, dist)
    if args.nonlocal_kb and args.prec == "fp64":
        line["nonlocal"] = nonlocal_section(tdks, torch, cfg, psi0, args, value)
    if args.nonlocal_kb and args.prec == "fp64":
        line["gll_collocation"] = gll_section(tdks, torch, cfg, args)
    if args.batched and args.prec == "fp64":
        bs = batched_section(tdks, torch, args, local_rank)
        line["batched"] = bs
        for name, pr in (("fp64", tdks.FP64), ("df64", tdks.DF64), ("mixed", tdks.MIXED)):
            ev = batched_err_vs_oracle(tdks, torch, pr)
            bs[name]["dipole_err_vs_oracle"] = ev
            speedups[f"batched_{name}"] = {
                "speedup_vs_fp64": round(bs[name]["speedup_vs_fp64_per_system"], 3),
                "speedup_same_caps": round(bs[name]["speedup_vs_fp64_per_system_same_caps"], 3),
                "dipole_err_vs_oracle": float(f"{ev['max']:.3g}"), "meets_1e-6": ev["max"] <= 1e-6,
                "baseline": "per-system FP64 path (k_max 64) on the same 64 systems; same_caps: "
                            "with the batch's per-system Krylov caps"}
    if args.adjoint and args.prec == "fp64":
        line["adjoint"] = adjoint_section(tdks, torch)
    if args.mixed and args.prec == "fp64":
        line["contraction_stage"] = contraction_stage_section(tdks, torch)
    if bg is not None:
        res = bg.results()
        mol = res.get("molecule")
        atom = res.get("atom")
        cb = {"unit": "orbital-steps/s", "cores": 1, "kind": "oracle", "host": host_info()}
        if isinstance(mol, list):
            st = [r for r in mol if "step" in r]
            cb.update(value=statistics.mean(r["orbital_steps_per_s"] for r in st),
                      how="extrapolated from timed samples", sample=ORACLE_SAMPLE_DESC,
                      timed_sample_s=sum(r["t_sample"] for r in st),
                      k_half=st[0]["k_half"], k_full=st[0]["k_full"])
        else:
            cb["error"] = str(mol)
        if isinstance(atom, list) and atom:
            a = atom[0]
            cb["atom_measured"] = {"value": a["orbital_steps_per_s"], "unit": "orbital-steps/s",
                                   "how": "measured", "sample": ATOM_RUN_DESC, "wall_s": a["wall_s"],
                                   "steps": a["steps"]}
        else:
            cb["atom_measured"] = {"error": str(atom)}
        line["cpu_baseline"] = cb
    line["speedups"] = speedups
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def graded_section(tdks, torch, args, local_rank: int, dist) -> dict:
    """All-electron-like workload (bare -Z/r nuclei of a CH4 stand-in, 24^3 hexahedra
    graded by 1.25 toward the nuclei, p = 8, 5 orbitals, dt 0.01): rate and dipole error
    per contraction type against the FP64 path over the same steps."""
    import numpy as np
    import synth
    cfg = synth.config3()
    Ni = tuple((len(b) - 1) * cfg.p - 1 for b in (cfg.X, cfg.Y, cfg.Z))
    psi0 = synth.smooth_orbitals(Ni, cfg.n_orb, seed=1)
    S, W = args.graded_steps, 1
    out = {"workload": "ch4_bare_graded24_p8: [-20,20]^3 bohr, 24^3 hexahedra graded 1.25 toward "
                       "C (Z 6) + 4 H (Z 1), bare -Z/r, p=8, 6,967,871 DoF, 5 orbitals (smooth, "
                       "orthonormal), kick 1e-3 x, dt 0.01, Krylov tol 1e-10, k_max 64",
           "steps": S, "warmup": W,
           "dipole_err": "max |d_x - d_x,fp64| / max |d_x,fp64 - d_x,fp64(0)| over the timed steps"}
    ref = None
    for name, prec in (("fp64", tdks.FP64), ("df64", tdks.DF64), ("mixed", tdks.MIXED), ("fp32", tdks.FP32),
                       ("bf16", tdks.BF16)):
        try:
            c, _, t, st, _, clk = _run_steps(tdks, torch, cfg, prec, S, W, local_rank, psi0, dist,
                                             timing=False)
        except tdks.TDKSError as e:
            if name == "fp64":
                raise
            out[name] = {"error": str(e)}
            continue
        d = np.array([s["dipole"] for s in st])
        if ref is None:
            ref = (d, c.d_init)
        c.close()
        r = {"value": cfg.n_orb * S / t, "unit": "orbital-steps/s", "ms_per_step": 1e3 * t / S,
             "substeps_per_step": sum(s["substeps"] for s in st) / S,
             "applies_per_step": sum(s["applies"] for s in st) / S, "clocks": clk}
        if name != "fp64":
            ind = float(np.abs(ref[0][:, 0] - ref[1][0]).max())
            r["speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / r["ms_per_step"]
            r["dipole_rel_err"] = float(np.abs(d[:, 0] - ref[0][:, 0]).max() / ind)
        if name == "bf16":
            r["note"] = BF16_NOTE
        out[name] = r
    return out


def nonlocal_section(tdks, torch, cfg, psi0, args, value_local: float) -> dict:
    """The molecule workload with Kleinman-Bylander projectors (l <= 1, 4 per atom) on
    its 8 atoms: FP64 step rate against the same steps without them."""
    import synth
    kp = synth.KBParams()
    ctx = tdks.Context.from_config(cfg)
    ctx.set_cg(1e-10)
    ctx.set_kb(cfg.atom_R, kp.a, kp.b, kp.c, kp.lmax)
    info = ctx.kb_info()
    psi = torch.from_numpy(psi0).cuda()
    ctx.kick(psi, cfg.kick, cfg.kick_dir)
    ctx.init_propagation(psi)
    K = max(3, args.steps // 2)
    for _ in range(args.warmup):
        ctx.magnus_step(psi, cfg.dt, tol=cfg.tol, k_max=cfg.k_max)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    st = [ctx.magnus_step(psi, cfg.dt, tol=cfg.tol, k_max=cfg.k_max) for _ in range(K)]
    ev1.record()
    torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) * 1e-3
    ctx.close()
    v = cfg.n_orb * K / t
    return {"workload": "molecule workload + Kleinman-Bylander projectors on its 8 atoms "
                        f"(a {kp.a}, b {kp.b}, c {list(kp.c)}, lmax {kp.lmax})",
            "n_proj": info["n_proj"], "covered_nodes": info["n_covered"],
            "stored_values": info["n_values"], "value": v, "unit": "orbital-steps/s",
            "ms_per_step": 1e3 * t / K, "steps": K,
            "k_full_max": max(s["k_full_max"] for s in st),
            "rate_vs_local_only": v / value_local}


def gll_section(tdks, torch, cfg, args) -> dict:
    """The GLL-collocation variant of Hbar against the paper's Gauss-rule operator on the
    molecule workload (16 orbitals, V = V_N): device time per 16-orbital application."""
    import synth
    ctx = tdks.Context.from_config(cfg)
    psi = torch.from_numpy(synth.random_psi(cfg.n_orb, ctx.n_int, seed=3)).cuda()
    ctx.set_potential(ctx.nuclear_potential())
    vn = ctx.nuclear_potential_nodes()
    out = torch.empty_like(psi)
    res = {}
    for name, fn in (("gauss", lambda: ctx.apply_H(psi, out)), ("gll", lambda: ctx.apply_H_gll(psi, vn, out))):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            fn()
        ev1.record()
        torch.cuda.synchronize()
        res[name] = ev0.elapsed_time(ev1) / args.steps
    ctx.close()
    return {"workload": "molecule workload, 16 random orbitals, V = V_N (Gauss points / nodes)",
            "ms_per_apply_gauss": res["gauss"], "ms_per_apply_gll": res["gll"],
            "speedup": res["gauss"] / res["gll"],
            "accuracy": "harmonic-oscillator ground energy on [-6,6]^3, 2^3 elements, p = 6: "
                        "Gauss form -3.6e-3, GLL collocation -1.44e-2 from the exact 3/2 (oracle)"}


def adjoint_section(tdks, torch) -> dict:
    """Gradient of J = int d_z(t)^2 dt with respect to the 8 parameters of four
    Gaussian pulses driving the atom workload (200 steps of dt 0.1, checkpoints every
    20 steps): forward and adjoint device time, and the gradient against central
    differences (h = 1e-5) of the same forward."""
    import numpy as np
    import synth
    sc, pc = synth.config4()
    gs = np.load(os.path.join(ROOT, "tests", "golden", "gs_atom_soft_Z2_6x6x6_p4.npz"))
    ctx = tdks.Context.from_config(sc)
    ctx.set_cg(1e-13)
    psi0 = torch.from_numpy(gs["psibar"].astype(complex)).cuda()
    w = pc.objective_weights()
    e = np.asarray(pc.direction)
    tol, kmax = 1e-12, 64
    params = torch.tensor(pc.params, dtype=torch.float64, requires_grad=True)
    E = synth.pulse_samples(params, pc)
    ctx.objective_forward(psi0, E.detach().numpy(), w, e, pc.dt, pc.ckpt_every, tol, kmax)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = tdks.DipoleObjective.apply(E, ctx, psi0, w, e, pc.dt, pc.ckpt_every, tol, kmax, tdks.FP64, 12)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = params.grad.numpy().copy()
    fd = np.zeros_like(g)
    for k in range(len(g)):
        pp, pm = pc.params.copy(), pc.params.copy()
        pp[k] += pc.fd_h
        pm[k] -= pc.fd_h
        Jp = ctx.objective_forward(psi0, synth.pulse_samples(pp, pc), w, e, pc.dt, pc.ckpt_every, tol, kmax)[0]
        Jm = ctx.objective_forward(psi0, synth.pulse_samples(pm, pc), w, e, pc.dt, pc.ckpt_every, tol, kmax)[0]
        fd[k] = (Jp - Jm) / (2 * pc.fd_h)
    ctx.close()
    return {"workload": "atom_soft_Z2_6x6x6_p4 driven by 4 Gaussian pulses (omega 0.3, sigma 5, "
                        "t_j = 4j), 200 steps dt 0.1, checkpoints every 20, Krylov tol 1e-12, "
                        "12-point Gauss-Legendre Frechet quadrature",
            "J": J.item(), "forward_s": t1 - t0, "backward_s": t2 - t1,
            "backward_over_forward": (t2 - t1) / (t1 - t0),
            "grad_vs_central_fd_max_rel": float(np.abs(g - fd).max() / np.abs(fd).max()),
            "grad": g.tolist()}


def contraction_stage_section(tdks, torch) -> dict:
    """One 1-D contraction stage of the p = 6 element kernel (a 7 x 7 operator on 622,592
    lines, 256 times in shared memory) in each arithmetic: CUDA-core FP32 and double-float,
    tensor-core BF16 operands and three-TF32 products (mma); useful multiply-adds per
    second and the error against an FP64 matrix power."""
    import numpy as np
    P1, n, reps = 7, 512 * 152 * 8, 256
    rng = np.random.default_rng(7)
    op, _ = np.linalg.qr(rng.standard_normal((P1, P1)))
    x = rng.standard_normal((n, P1))
    ref = x @ np.linalg.matrix_power(op, reps).T
    xd = torch.from_numpy(x).cuda()
    out = {"workload": "7x7 orthogonal operator, 622,592 lines, 256 applications in shared memory",
           "useful_macs_per_launch": n * reps * P1 * P1}
    names = {0: "fp32_cuda_cores", 1: "double_float_cuda_cores", 2: "bf16_tensor_cores",
             3: "tf32x3_tensor_cores"}
    for v, name in names.items():
        y, ms = tdks.contraction_probe(v, op, xd, reps)
        out[name] = {"ms": ms, "useful_tmac_per_s": n * reps * P1 * P1 / (ms * 1e-3) / 1e12,
                     "rel_err_vs_fp64": float(np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max())}
    out["mma_useful_fraction"] = {"bf16_m16n8k16": 49 / 128, "tf32x3_m16n8k8": 49 / (3 * 64)}
    return out


def batched_section(tdks, torch, args, local_rank: int) -> dict:
    """64 independent uneven systems (n^3 elements n in 4..12, p in 4..8, 1-8 orbitals,
    own dt and kick): the batched engine (one CUDA graph per step, device-side Krylov
    loops, autotuned tiles) in the relaxed schedule, DF64 and FP64 against the plain
    per-system FP64 path
    (tdks_magnus_step system after system) over the same steps from the same kicked
    orbitals.  Dipole error: max over systems and steps of |d - d_fp64| relative to
    the largest |d_fp64(t) - d_fp64(0)| of that system."""
    import numpy as np
    import synth
    cfgs, dts, dirs = synth.config5()
    W, K = args.warmup, args.batch_steps
    psi0 = [synth.smooth_orbitals(tuple((len(c.X) - 1) * c.p - 1 for _ in range(3)), c.n_orb,
                                  seed=500 + k) for k, c in enumerate(cfgs)]
    orb_steps = sum(c.n_orb for c in cfgs) * K
    out = {"workload": "64 systems, seeded: n^3 hexahedra (n 4..12, h = 2 bohr), p 4..8, 1-8 "
                       "orbitals, 1-4 soft-Coulomb nuclei (Z 1..4), dt in {0.02, 0.05, 0.1}, "
                       "kick 1e-3 along a seeded direction; smooth orthonormal initial orbitals",
           "orbital_dofs": int(sum(c.n_orb * ((len(c.X) - 1) * c.p - 1) ** 3 for c in cfgs)),
           "steps": K, "warmup": W}
    runs = {}
    W2 = max(W - 1, 1)       # warm-up steps after the Krylov caps are set (graph rebuilt)
    for name, prec in (("mixed", tdks.MIXED), ("df64", tdks.DF64), ("fp64", tdks.FP64)):
        b = tdks.Batch(cfgs, dts, prec=prec, tol=1e-10, k_max=64)
        for k, p in enumerate(psi0):
            b.set_orbitals(k, torch.from_numpy(p).cuda())
        b.kick([c.kick for c in cfgs], dirs)
        d0 = b.init()
        tiles = b.tune(reps=2)
        # first warm-up step at k_max 64; the systems whose exponentials restarted at
        # that cap get a 128-vector basis (tdks_batch_tune_kmax), then the rest of the
        # warm-up
        dw = b.steps(1)
        caps = b.tune_kmax(BATCH_KCAP) if BATCH_KCAP > 64 else [64] * len(cfgs)
        dw = np.concatenate([dw, b.steps(W2)])
        b.stats(reset=True)
        st = torch.cuda.ExternalStream(b.stream)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            ev0.record(st)
            dk = b.steps(K)
            ev1.record(st)
            torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) * 1e-3
        sts = b.stats()
        runs[name] = {"dip": np.concatenate([d0[None], dw, dk]), "t": t, "caps": caps}
        raised = [k for k, c in enumerate(caps) if c > 64]
        out[name] = {"value": orb_steps / t, "unit": "orbital-steps/s", "ms_per_step": 1e3 * t / K,
                     "hpsi_gdofs": sts["dof_applies"] / t / 1e9, "k_max_seen": sts["k_max_seen"],
                     "krylov_caps": {"raised_to": BATCH_KCAP, "systems": len(raised),
                                     "added_basis_gb": round(sum(
                                         cfgs[k].n_orb * ((len(cfgs[k].X) - 1) * cfgs[k].p - 1) ** 3
                                         * (caps[k] - 64) * 16 for k in raised) / 1e9, 2)},
                     "clocks": clk.summary()}
        if name == "df64":
            out["tiles"] = tiles
        b.close()
        del b
        torch.cuda.empty_cache()
    # plain per-system FP64 path, same steps: at k_max 64 throughout, and with the
    # batch's per-system caps after the first step
    def per_system(caps):
        dref = np.zeros((1 + W2 + 1 + K, len(cfgs), 3))
        t_plain = 0.0
        for k, c in enumerate(cfgs):
            ctx = tdks.Context.from_config(c)
            g = torch.from_numpy(psi0[k]).cuda()
            ctx.kick(g, c.kick, dirs[k])
            dref[0, k] = ctx.init_propagation(g)
            dref[1, k] = ctx.magnus_step(g, c.dt, tol=1e-10, k_max=64)["dipole"]
            for s in range(W2):
                dref[2 + s, k] = ctx.magnus_step(g, c.dt, tol=1e-10, k_max=caps[k])["dipole"]
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            for s in range(K):
                dref[2 + W2 + s, k] = ctx.magnus_step(g, c.dt, tol=1e-10, k_max=caps[k])["dipole"]
            ev1.record()
            torch.cuda.synchronize()
            t_plain += ev0.elapsed_time(ev1) * 1e-3
            ctx.close()
        return dref, t_plain

    dref, t_plain = per_system([64] * len(cfgs))
    out["fp64_per_system"] = {"value": orb_steps / t_plain, "unit": "orbital-steps/s",
                              "ms_per_step": 1e3 * t_plain / K, "k_max": 64}
    caps = runs["fp64"]["caps"]
    if any(c != 64 for c in caps):
        dref_c, t_c = per_system(caps)
        out["fp64_per_system_same_caps"] = {"value": orb_steps / t_c, "unit": "orbital-steps/s",
                                            "ms_per_step": 1e3 * t_c / K,
                                            "k_max": "the batch's per-system caps"}
    else:
        dref_c, t_c = dref, t_plain
    ind = np.maximum(np.abs(dref - dref[0:1]).max(axis=(0, 2)), 1e-300)     # per system
    for name in runs:
        ref = dref_c if runs[name]["caps"] == caps else dref
        err = np.abs(runs[name]["dip"] - ref).max(axis=(0, 2)) / ind
        out[name]["dipole_rel_err"] = float(err.max())
        out[name]["speedup_vs_fp64_per_system"] = out[name]["value"] / out["fp64_per_system"]["value"]
        out[name]["speedup_vs_fp64_per_system_same_caps"] = out[name]["value"] * t_c / orb_steps
    return out


def apply_only(args, local_rank: int):
    """Standalone Hbar psi on the benchmark workload (16 orbitals, random
    orbitals, V = V_N): the kernel in isolation, for the roofline and ncu."""
    import numpy as np
    import torch
    import synth
    from paper_1810_13130_gb300 import tdks
    torch.cuda.set_device(local_rank)
    prec = {"fp64": tdks.FP64, "fp32": tdks.FP32, "df64": tdks.DF64, "bf16": tdks.BF16,
            "mixed": tdks.MIXED}[args.prec]
    cfg = synth.config2()
    ctx = tdks.Context.from_config(cfg)
    psi = torch.from_numpy(synth.random_psi(cfg.n_orb, ctx.n_int, seed=3)).cuda()
    ctx.set_potential(ctx.nuclear_potential())
    out = torch.empty_like(psi)
    for _ in range(args.warmup):
        ctx.apply_H(psi, out, prec)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record()
        for _ in range(args.steps):
            ctx.apply_H(psi, out, prec)
        ev1.record()
        torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) * 1e-3 / args.steps
    P1 = cfg.p + 1
    units = cfg.n_orb * ctx.n_elem
    flops = units * (36 * P1 ** 4 + 24 * P1 ** 3)
    byts = cfg.n_orb * ctx.n_int * 32.0 + ctx.n_elem * P1 ** 3 * 8.0   # read psi, write Hpsi, V
    peaks = measured_peaks(tdks, local_rank)
    peak = peaks["fp64" if args.prec == "fp64" else "fp32"]["tflops"]
    print(json.dumps({"mode": "apply_only", "prec": args.prec, "ms_per_apply": t * 1e3,
                      "hpsi_gdofs": cfg.n_orb * ctx.n_int / t / 1e9,
                      "tflops": flops / t / 1e12, "frac_alu": flops / t / 1e12 / peak,
                      "hbm_GBps": byts / t / 1e9, "frac_hbm": byts / t / 1e9 / 6790.0,
                      "peak_tflops_measured": peak,
                      "clocks": clk.summary()}), flush=True)
    ctx.close()


def horizon(args, local_rank: int):
    """The molecule workload over a long horizon (500 steps = its full run) with each
    contraction type, from the same kicked orbitals: dipole difference from the FP64
    path relative to the FP64 path's induced dipole (no oracle series exists at this
    size: the oracle takes about 16 minutes per step on one core)."""
    import numpy as np
    import torch
    import synth
    from paper_1810_13130_gb300 import tdks
    torch.cuda.set_device(local_rank)
    cfg = synth.config2()
    psi0 = synth.smooth_orbitals(tuple(n * cfg.p - 1 for n in (cfg.nx, cfg.ny, cfg.nz)),
                                 cfg.n_orb, seed=1)
    res = {"mode": "horizon", "workload": WORKLOAD, "steps": args.horizon}
    dips = {}
    for name, prec in (("fp64", tdks.FP64), ("df64", tdks.DF64), ("mixed", tdks.MIXED),
                       ("fp32", tdks.FP32)):
        ctx = tdks.Context.from_config(cfg)
        ctx.set_cg(1e-10)
        g = torch.from_numpy(psi0).cuda()
        ctx.kick(g, cfg.kick, cfg.kick_dir)
        d = [ctx.init_propagation(g)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with ClockSampler(local_rank) as clk:
            for _ in range(args.horizon):
                d.append(ctx.magnus_step(g, cfg.dt, tol=cfg.tol, k_max=cfg.k_max, prec=prec)["dipole"])
        tw = time.perf_counter() - t0
        ctx.close()
        dips[name] = np.array(d)
        res[name] = {"s_per_step": tw / args.horizon, "clocks": clk.summary()}
    ref = dips["fp64"]
    ind = np.abs(ref - ref[0]).max(axis=0)
    res["induced_dipole_fp64"] = ind.tolist()
    for name in ("df64", "mixed", "fp32"):
        err = np.abs(dips[name] - ref).max(axis=0) / ind
        res[name]["dipole_rel_diff_vs_fp64"] = err.tolist()
        res[name]["dipole_rel_diff_vs_fp64_max"] = float(err.max())
        # growth: the same measure over the first 10, 50, 100, 200 steps
        res[name]["by_horizon"] = {str(n): float((np.abs(dips[name][:n + 1] - ref[:n + 1]).max(axis=0) /
                                                  np.abs(ref[:n + 1] - ref[0]).max(axis=0)).max())
                                   for n in (10, 50, 100, 200, args.horizon) if n <= args.horizon}
    print(json.dumps(res), flush=True)


def main():
    global HOST_LOOP
    args = parse()
    HOST_LOOP = args.host_loop
    if args.oracle_sample is not None:
        oracle_sample_main(args.oracle_sample)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if args.apply_only:
        apply_only(args, local_rank)
        return
    if args.horizon > 0:
        horizon(args, local_rank)
        return
    if args.batch_profile:
        import torch
        from paper_1810_13130_gb300 import tdks
        torch.cuda.set_device(local_rank)
        print(json.dumps(batch_profile(tdks, torch, args.prec)), flush=True)
        return
    if args.stage_study:
        import torch
        from paper_1810_13130_gb300 import tdks
        torch.cuda.set_device(local_rank)
        print(json.dumps(stage_study(tdks, torch)), flush=True)
        return
    if args.stage_only:
        import torch
        from paper_1810_13130_gb300 import tdks
        torch.cuda.set_device(local_rank)
        print(json.dumps({"mode": "stage_only", **contraction_stage_section(tdks, torch)}), flush=True)
        return
    ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
