#!/usr/bin/env python
"""Benchmark of the RHS evaluation F(t, alpha) of the pseudospectral
quadrature method (rotating-sphere Navier-Stokes) at truncation L = 511 on
the 768 x 1536 Gauss-rectangle grid, mixed precision.

One step = one RHS evaluation (coefficient prep, per-order Legendre
synthesis, per-latitude FFT + product + FFT, per-order Legendre analysis,
recombination and diagonal update) on device-resident synthetic inputs.
The Legendre tables (>= 200 MB) exceed the 129 MB L2, so every step streams
them from HBM; no extra L2 flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (the single
RHS does not shard without an all-to-all; replicas only) and rank 0 prints
the whole-job aggregate.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RHS evals/s at L=511 (768x1536 grid), mixed precision"
UNIT = "RHS/s"
WORKLOAD = "L511"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, help="fp32 | bf16x3 (default: best mixed path)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--only", default=None, choices=sorted(EXTRAS),
                    help="run this one extra workload alone and print its line (no headline)")
    ap.add_argument("--ensemble-cluster", type=int, default=0, choices=[0, 1, 2, 4],
                    help="ensemble BF16X3 synthesis: CTAs per cluster without the autotuner (0: autotuned)")
    return ap.parse_args()


# --------------------------------------------------------------------------
# clocks sampled with nvidia-smi during the timed region

class ClockSampler:
    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def result(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = []
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except Exception:
                continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        inside = [r for r in rows if self.t0 - 1 <= r[0] <= self.t1 + 1] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


# --------------------------------------------------------------------------
# algorithmic bytes / flops of the kernels (per launch)

def sizes(L, nlat):
    nh = (nlat + 1) // 2
    n_ext = (L + 2) * (L + 3) // 2 - 1
    return nh, n_ext, nh * n_ext


def algorithmic(stage, L, nlat, prec, entries=None):
    """(bytes, flops) one launch of a stage must move / execute at minimum.
    entries: table entries the kernel reads when it skips tiles of negligible
    entries (the tensor-core path), else every entry E."""
    nh, n_ext, E = sizes(L, nlat)
    if entries:
        E = int(entries)
    tb = {"fp64": 8, "fp32": 4, "bf16x3": 4}[prec]     # table bytes per entry (hi+lo for bf16)
    vb = 8 if prec == "fp64" else 4                     # intermediate real size
    g = nlat * (L + 1) * 2 * vb                         # one complex [nlat][L+1] field
    nc = (L + 1) * (L + 2) // 2 - 1                     # packed coefficients (complex128 state)
    if prec == "bf16x3":
        # the tensor-core RHS: the synthesis reads alpha itself (its coefficient
        # tiles are built in the kernel), the analysis reads alpha and writes F
        if stage == "synthesis":
            return E * tb + nc * 16 + 3 * g, 12 * E
        if stage == "analysis":
            return E * tb + 2 * g + 2 * nc * 16, 8 * E
    if stage == "synthesis":
        return E * tb + n_ext * 6 * vb + 3 * g, 12 * E
    if stage == "analysis":
        return E * tb + 2 * g + n_ext * 4 * vb, 8 * E
    if stage == "ring":
        return 5 * g, 0
    return 0, 0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel_key):
    """Bytes per launch from the committed ncu summary, or None when the
    kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e:
        return None
    src = os.path.join(ROOT, e["source"])
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    return e["bytes_per_launch"] if h == e["source_sha"] else None


# --------------------------------------------------------------------------

def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x, device="cuda"):
    """The slowest rank's value of x (a duration), on every rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world, units_per_rank, seconds):
    """Whole-job throughput of `world` independent replicas that each
    processed `units_per_rank` units, timed by the slowest rank."""
    return world * units_per_rank / seconds


def time_rhs(plan, a, out, steps, torch):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        plan.rhs(a, out=out)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _timed(fn, torch):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def extra_ndf_L511(torch, prec, nsteps=500):
    """Adaptive NDF steps at the L = 511 workload (500 steps, rtol 1e-6, mixed path)."""
    from paper_1009_3308_gb300 import Integrator, Plan
    from seeded_inputs import workload
    w = workload("L511")
    c = w["config"]
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"], precision=prec)
    plan.set("RTOL", c["rtol"])
    plan.set("ATOL", 1e-3 * c["rtol"] * float(abs(w["alpha0"]).max()))
    integ = Integrator(plan, torch.from_numpy(w["alpha0"]).cuda())
    integ.step()
    infos, el = _timed(lambda: integ.advance(nsteps), torch)
    rhs = sum(i["rhs_evals"] for i in infos)
    return {"steps_per_s": nsteps / el, "rhs_evals_per_step": rhs / nsteps, "steps": nsteps,
            "precision": prec, "t_reached": integ.t, "api": "sphnse_advance (one call for all steps)"}


def extra_mixed_errors(torch, prec, nsteps=500):
    """Error per field of the mixed path at L = 511 against the FP64 GPU path
    (itself pinned to the oracle at 1e-12): grid fields zeta, u_theta, u_phi,
    the projection of a tangential field, F, and the state after the 500-step
    sequence of an adaptive mixed run replayed in both precisions."""
    from paper_1009_3308_gb300 import Integrator, Plan
    from seeded_inputs import workload
    w = workload("L511")
    c = w["config"]
    a0 = torch.from_numpy(w["alpha0"]).cuda()
    rel = lambda x, y: float(((x - y).norm() / y.norm()).item())
    p64 = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"])
    pm = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"], precision=prec)
    out = {}
    g64, gm = p64.grid_fields(a0), pm.grid_fields(a0)
    for name, x, y in zip(("zeta", "u_theta", "u_phi"), gm, g64):
        out[name] = rel(x, y)
    out["projection"] = rel(pm.project(g64[1], g64[2]), p64.project(g64[1], g64[2]))
    out["F"] = rel(pm.rhs(a0), p64.rhs(a0))
    atol = 1e-3 * c["rtol"] * float(abs(w["alpha0"]).max())
    for p in (p64, pm):
        p.set("RTOL", c["rtol"])
        p.set("ATOL", atol)
    run = Integrator(pm, a0.clone())
    sched = []
    for _ in range(nsteps):
        i = run.step()
        sched.append((i["h"], i["order"]))
    fin = {}
    for name, p in (("mixed", pm), ("fp64", p64)):
        it = Integrator(p, a0.clone())
        for h, k in sched:
            it.replay_step(h, k)
        fin[name] = it.alpha
    out["state_after_replayed_steps"] = rel(fin["mixed"], fin["fp64"])
    out["steps"] = nsteps
    out["t_reached"] = sum(h for h, _ in sched)
    return out


def extra_fp64_L255(torch, nrhs=1000):
    """The FP64 workload at L = 255 (384 x 768): 1000 RHS evaluations on the
    GPU and the relative error of F against the FP64 oracle."""
    import numpy as np
    from paper_1009_3308_gb300 import Plan
    from oracle.rhs import Problem, rhs_separable
    from seeded_inputs import workload
    w = workload("L255")
    c = w["config"]
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"])
    a = torch.from_numpy(w["alpha0"]).cuda()
    out = plan.empty_coeff()
    ms = time_rhs(plan, a, out, 5, torch)
    ms = time_rhs(plan, a, out, nrhs, torch)
    ref = rhs_separable(Problem(c["L"], c["nlon"], c["nu"], c["Omega"]), w["alpha0"])
    got = plan.rhs(a).cpu().numpy()
    return {"rhs_per_s": 1e3 / ms, "ms_per_rhs": ms, "rhs": nrhs,
            "rel_err_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}


def extra_coriolis_split(torch, prec):
    """RHS/s at the L = 511 workload with the Coriolis term applied as its
    diagonal (no 2 Omega cos(theta) in the grid product), and its relative
    difference from the unsplit F in the same precision."""
    import numpy as np
    from paper_1009_3308_gb300 import Plan
    from seeded_inputs import workload
    w = workload("L511")
    c = w["config"]
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"], precision=prec)
    a = torch.from_numpy(w["alpha0"]).cuda()
    full = plan.rhs(a).cpu().numpy()
    plan.set("CORIOLIS_SPLIT", 1)
    out = plan.empty_coeff()
    time_rhs(plan, a, out, 20, torch)
    ms = time_rhs(plan, a, out, 1000, torch)
    split = plan.rhs(a).cpu().numpy()
    return {"rhs_per_s": 1e3 / ms, "ms_per_rhs": ms, "precision": prec,
            "rel_diff_vs_unsplit": float(np.linalg.norm(split - full) / np.linalg.norm(full))}


def extra_batched_L511(torch, n=4, reps=200):
    """n independent L = 511 states in one batched BF16X3 RHS (an ensemble
    bucket): one table stream per stage serves every state of the group.
    Context for the single-state headline, not a substitute for it."""
    from paper_1009_3308_gb300 import Ensemble
    from seeded_inputs import coefficients, workload
    w = workload("L511")
    c = w["config"]
    ens = Ensemble([c["L"]] * n, [c["nu"]] * n, c["Omega"], precision="bf16x3")
    for i in range(n):
        ens.set_alpha(i, torch.from_numpy(coefficients(c["L"], 3000 + i, 0.02)))
    for _ in range(5):
        ens.rhs()
    _, el = _timed(lambda: [ens.rhs() for _ in range(reps)], torch)
    return {"states": n, "rhs_per_s": n * reps / el, "us_per_batched_rhs": 1e6 * el / reps}


def run_example2(torch, t_out=(10, 20, 30, 40, 50, 60), N=100, N1=75, rtol=1e-3, precision="fp64"):
    """Sec. 5 Example 2 (N = 100, Omega = 1, nu = 1e-4, rtol 1e-3): the random
    initial state of degree <= 20 driven by fhat_{3,0}(t), integrated to
    t = 60; at each output time the spectrum E(L) of U_75 = P_75 u_N and of
    the approximate inertial manifold Phi_150(U_75) (Eq. (eq:p-p)).  The
    forcing of a step is fhat_{3,0} at the end of the step the controller
    plans (the step API holds it constant over a step)."""
    import numpy as np
    from paper_1009_3308_gb300 import Integrator, Plan
    from seeded_inputs import example2, example2_forcing_30
    nu = 1e-4
    plan = Plan(N, 162, 324, nu, 1.0, precision=precision)
    plan.set("RTOL", rtol)
    a0 = example2(N)
    plan.set("ATOL", 1e-3 * rtol * float(np.abs(a0).max()))
    p2 = Plan(2 * N1, 243, 486, nu, 1.0)
    f = torch.zeros(plan.n_coeff, dtype=torch.complex128, device="cuda")
    f2 = torch.zeros(p2.n_coeff, dtype=torch.complex128, device="cuda")
    f[2] = example2_forcing_30(0.0)       # packed index of (L = 3, m = 0)
    it = Integrator(plan, torch.from_numpy(a0).cuda(), forcing=f, t_end=t_out[0])
    out, steps, rhs = [], 0, 0

    def spectra(t):
        a = it.alpha
        E = plan.energy_spectrum(a).cpu().numpy()[: N1 + 1]
        f2[2] = example2_forcing_30(t)
        phi = p2.inertial_manifold(N1, p2.resize(a, N, L_max=N1), f2)
        Ep = p2.energy_spectrum(phi).cpu().numpy()
        return E, Ep

    E0, _ = spectra(0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for te in t_out:
        it.st.t_end = float(te)
        while it.t < te * (1 - 1e-12):
            f[2] = example2_forcing_30(min(te, it.t + it.st.h))
            info = it.step()
            steps += 1
            rhs += info["rhs_evals"]
        E, Ep = spectra(te)
        out.append((te, E, Ep))
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    return E0, out, steps, rhs, el


def extra_example2(torch):
    import numpy as np
    E0, out, steps, rhs, el = run_example2(torch)
    L = np.arange(len(E0))
    cen = lambda E: float((L[1:] * E[1:]).sum() / E[1:].sum())
    rows = []
    for te, E, Ep in out:
        Lp = np.arange(76, len(Ep))
        y = np.log(np.maximum(Lp ** 4 * Ep[76:], 1e-300))
        slope = float(np.polyfit(Lp, y, 1)[0])
        rows.append({"t": te, "energy_U75": float(E.sum()), "centroid_L": cen(E),
                     "L4E_phi_slope_per_L": slope, "E_phi_total": float(Ep.sum())})
    return {"steps": steps, "rhs_evals": rhs, "seconds": el, "steps_per_s": steps / el,
            "energy_t0": float(E0.sum()), "centroid_L_t0": cen(E0), "outputs": rows,
            "precision": "fp64", "N": 100, "N1": 75, "rtol": 1e-3}


def extra_L31(torch, nsteps=100):
    """The L = 31 workload: 100 adaptive FP64 steps, rtol 1e-8, steady forcing
    (in one sphnse_advance call, and again one sphnse_step call per step)."""
    from paper_1009_3308_gb300 import Integrator, Plan
    from seeded_inputs import workload
    w = workload("L31")
    c = w["config"]
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"])
    plan.set("RTOL", c["rtol"])
    plan.set("ATOL", 1e-3 * c["rtol"] * float(abs(w["alpha0"]).max()))
    integ = Integrator(plan, torch.from_numpy(w["alpha0"]).cuda(), forcing=torch.from_numpy(w["forcing"]).cuda())
    integ.step()
    infos, el = _timed(lambda: integ.advance(nsteps), torch)
    rhs = sum(i["rhs_evals"] for i in infos)
    _, el1 = _timed(lambda: [integ.step() for _ in range(nsteps)], torch)
    # latency-bound: one RHS back to back and with a host round trip, next to
    # the floor of one tiny kernel launch + synchronize on this stream
    a = torch.from_numpy(w["alpha0"]).cuda()
    out = plan.empty_coeff()
    ms_b2b = time_rhs(plan, a, out, 2000, torch)
    lat = []
    for _ in range(200):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.rhs(a, out=out)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0)
    x = torch.zeros(1, device="cuda")
    floor = []
    for _ in range(200):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x.add_(1.0)
        torch.cuda.synchronize()
        floor.append(time.perf_counter() - t0)
    lat.sort()
    floor.sort()
    return {"steps_per_s": nsteps / el, "rhs_per_s": rhs / el, "steps": nsteps, "t_reached": integ.t,
            "api": "sphnse_advance (one call for all steps)", "steps_per_s_one_step_per_call": nsteps / el1,
            "precision": "fp64", "rhs_us_back_to_back": 1e3 * ms_b2b, "rhs_us_with_sync_median": 1e6 * lat[100],
            "launch_sync_floor_us_median": 1e6 * floor[100]}


def extra_adjoint(torch, nsteps=200, checkpoint=20):
    """Adjoint workload at L = 255: band energy + misfit gradient w.r.t. alpha0
    and nu through frozen-controller NDF steps, FP32 contractions, FP64 state,
    checkpoints every 20 steps."""
    import math as _m
    from paper_1009_3308_gb300 import Plan
    from paper_1009_3308_gb300.adjoint import adaptive_schedule, objective, trajectory
    from seeded_inputs import workload
    w = workload("adjoint")
    c = w["config"]
    plan = Plan(c["L"], c["nlat"], c["nlon"], c["nu"], c["Omega"], precision="fp32")
    plan.set("RTOL", c["rtol"])
    plan.set("ATOL", 1e-3 * c["rtol"] * float(abs(w["alpha0"]).max()))
    a0 = torch.from_numpy(w["alpha0"]).cuda()
    tgt = torch.from_numpy(w["target"]).cuda()
    _, sched, h0 = adaptive_schedule(plan, a0, nsteps)
    for rep in range(2):   # the first pass loads every kernel of the adjoint path once
        a0r = torch.view_as_real(a0).clone().requires_grad_(True)
        nut = torch.tensor(c["nu"], dtype=torch.float64, requires_grad=True)
        J, tf = _timed(lambda: objective(plan, trajectory(plan, a0r, nut, sched, h0, checkpoint=checkpoint), tgt,
                                         _m.radians(30), _m.radians(60)), torch)
        _, tb = _timed(lambda: J.backward(), torch)
    return {"adjoint_steps_per_s": nsteps / tb, "forward_replay_steps_per_s": nsteps / tf, "steps": nsteps,
            "checkpoint": checkpoint, "precision": "fp32 contractions, fp64 state", "L": c["L"],
            "grad_norm": float(a0r.grad.norm()), "dJ_dnu": float(nut.grad)}


def extra_ensemble(torch, nsteps=200, n=256, precision="fp32", cluster=0):
    """Batched ensemble: 256 instances, L uniform over {63, 127, 255}, nu
    log-uniform in [1e-5, 1e-3], per-instance adaptive steps; "fp32"
    streaming contractions or "bf16x3" (instances of a truncation share every
    table tile on the tensor cores; cluster > 0 fixes the CTAs per cluster of
    the synthesis instead of autotuning its shape)."""
    from paper_1009_3308_gb300 import Ensemble
    from seeded_inputs import ensemble
    mem = ensemble(n)
    ens = Ensemble([m["L"] for m in mem], [m["nu"] for m in mem], 1.0, precision=precision,
                   autotune=cluster == 0, cluster=max(cluster, 1))
    for i, m in enumerate(mem):
        ens.set_alpha(i, torch.from_numpy(m["alpha0"]))
    ens.set("RTOL", 1e-6)
    ens.set("ATOL", 1e-12)
    ens.init(0.0)
    ens.advance(2)
    _, tr = _timed(lambda: [ens.rhs() for _ in range(3)], torch)
    infos, el = _timed(lambda: ens.advance(nsteps), torch)
    rounds = ens.get("ROUNDS")
    rhs = sum(i["rhs_evals"] for i in infos)
    return {"instance_steps_per_s": n * nsteps / el, "instance_rhs_per_s_in_steps": rhs / el,
            "batched_rhs_per_s": 3 / tr, "instance_rhs_per_s_batched": 3 * n / tr,
            "rounds": rounds, "ms_per_round": 1e3 * el / rounds if rounds else None,
            "mean_rhs_per_instance_step": rhs / (n * nsteps),
            "instances": n, "steps": nsteps, "seconds": el,
            "stepping": "asynchronous rounds (sphnse_ensemble_advance)",
            "buckets": sorted(set(m["L"] for m in mem)), "precision": precision,
            "synthesis_shapes": ens.buckets() if precision == "bf16x3" else None}


def cpu_baseline(w, target_s=15.0):
    """The FP64 oracle as it stands, on this host's cores: RHS evaluations at
    the benchmark workload (tables built first, not timed)."""
    from oracle.rhs import Problem, rhs_separable
    c = w["config"]
    prob = Problem(c["L"], c["nlon"], c["nu"], c["Omega"])
    prob.tables()
    t0 = time.perf_counter()
    n = 0
    while True:
        rhs_separable(prob, w["alpha0"])
        n += 1
        el = time.perf_counter() - t0
        if el >= target_s or n >= 50:
            break
    return {"value": n / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} full RHS evaluations at L=511 on 768x1536 (FP64 numpy oracle; "
                      f"Legendre tables built before timing), {el:.1f} s"}


def arm_config(c, prec, world):
    """The workload both arms report (the reference arm times the oracle on it)."""
    return {"workload": "L=511 RHS evaluation, 768x1536 Gauss-rectangle grid, "
                        "seeded spectrum exp(-0.02 L)/(L(L+1)), nu=5e-5, Omega=1",
            "L": c["L"], "nlat": c["nlat"], "nlon": c["nlon"], "precision": prec,
            "l2": "inputs larger than L2 (Legendre tables streamed every step)",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle.rhs import Problem, rhs_separable
    from seeded_inputs import workload
    w = workload(WORKLOAD)
    c = w["config"]
    prob = Problem(c["L"], c["nlon"], c["nu"], c["Omega"])
    prob.tables()
    # each step is one full oracle RHS (~2 s); the count is capped so that the
    # run stays within a few minutes
    steps = max(1, min(args.steps, 40))
    warm = max(0, min(args.warmup, 2))
    for _ in range(warm):
        rhs_separable(prob, w["alpha0"])
    t0 = time.perf_counter()
    for _ in range(steps):
        rhs_separable(prob, w["alpha0"])
    el = time.perf_counter() - t0
    v = steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(c, args.precision or _best_mixed(), world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{steps} full RHS evaluations at L=511 (numpy FP64 oracle)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# the extra workloads, in the order the full run takes them (prec: the headline's precision)
EXTRAS = {
    "ndf_L511": lambda torch, prec, args: extra_ndf_L511(torch, prec),
    "mixed_errors_L511": lambda torch, prec, args: extra_mixed_errors(torch, prec),
    "fp64_L255": lambda torch, prec, args: extra_fp64_L255(torch),
    "coriolis_split_L511": lambda torch, prec, args: extra_coriolis_split(torch, prec),
    "batched_L511_x4": lambda torch, prec, args: extra_batched_L511(torch),
    "adjoint_L255": lambda torch, prec, args: extra_adjoint(torch),
    "ensemble": lambda torch, prec, args: extra_ensemble(torch, nsteps=_ens_steps(args)),
    "ensemble_bf16x3": lambda torch, prec, args: extra_ensemble(torch, nsteps=_ens_steps(args), precision="bf16x3",
                                                                cluster=args.ensemble_cluster),
    "L31_fp64_steps": lambda torch, prec, args: extra_L31(torch),
    "example2_N100": lambda torch, prec, args: extra_example2(torch),
}


def _ens_steps(args):
    # the configuration's 200 steps; a shorter run with --only and --steps (profiling targets)
    return min(args.steps, 200) if args.only else 200


def run_only(args):
    """One extra workload alone (one GPU), e.g. as a profiling target."""
    import torch
    prec = args.precision or _best_mixed()
    out = EXTRAS[args.only](torch, prec, args)
    print(json.dumps({"workload": args.only, **out}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.only:
        run_only(args)
        return
    import numpy as np
    import torch

    from paper_1009_3308_gb300 import Plan, _capi
    from seeded_inputs import workload

    world, rank, local = dist_setup(args)
    w = workload(WORKLOAD)
    c = w["config"]
    L, nlat, nlon = c["L"], c["nlat"], c["nlon"]
    prec = args.precision or _best_mixed()
    plan = Plan(L, nlat, nlon, c["nu"], c["Omega"], precision=prec)
    a = torch.from_numpy(w["alpha0"]).cuda()
    out = plan.empty_coeff()
    lib = _capi.lib()

    for _ in range(max(args.warmup, 3)):
        plan.rhs(a, out=out)
    torch.cuda.synchronize()

    import ctypes
    # stage split: a separate short pass with an event pair around every
    # kernel (each pair costs stream time, so the timed region below keeps
    # only the pair of the kernel whose roofline it reports)
    n_split = 50
    lib.sphnse_stage_timing(plan.handle, -1)
    for _ in range(n_split):
        plan.rhs(a, out=out)
    st_ms = (ctypes.c_double * 7)()
    st_n = (ctypes.c_long * 7)()
    lib.sphnse_stage_times(plan.handle, st_ms, st_n)
    lib.sphnse_stage_timing(plan.handle, 0)
    split = {name: st_ms[i] / n_split * 1e3 for i, name in enumerate(_capi.STAGES) if st_n[i]}
    kernels_per_rhs = int(round(sum(st_n[i] for i in range(7)) / n_split))
    dom = max(("synthesis", "analysis", "ring"), key=lambda k: split.get(k, 0.0))
    dom_id = _capi.STAGES.index(dom)

    clk = ClockSampler(local)
    time.sleep(0.3)
    # the dominant kernel's duration: an event pair around it on every
    # SAMPLE-th RHS of the timed region (a pair keeps the kernel from starting
    # early under its predecessor, so pairs on every call would slow the loop)
    SAMPLE = 32   # ~94 samples in the default 3000 steps
    plan.set("TIMING_PERIOD", SAMPLE)
    lib.sphnse_stage_timing(plan.handle, 1 << dom_id)
    barrier(world)
    torch.cuda.synchronize()
    clk.mark_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        plan.rhs(a, out=out)
    e1.record()
    torch.cuda.synchronize()
    clk.mark_end()
    barrier(world)
    ms_total = e0.elapsed_time(e1)
    ms_total = max_over_ranks(world, ms_total)
    lib.sphnse_stage_times(plan.handle, st_ms, st_n)
    lib.sphnse_stage_timing(plan.handle, 0)
    plan.set("TIMING_PERIOD", 1)
    clocks = clk.result()
    stage = {name: {"ms": st_ms[i], "launches": st_n[i]} for i, name in enumerate(_capi.STAGES)}
    launches = kernels_per_rhs * args.steps

    value = replica_rate(world, args.steps, ms_total / 1e3)
    ms_per_step = ms_total / args.steps

    # dominant kernel and its roofline (live durations from the timed region)
    avg_ms = stage[dom]["ms"] / max(stage[dom]["launches"], 1)
    ent = None
    if prec == "bf16x3" and dom in ("synthesis", "analysis"):
        ent = plan.get("SYN_ENTRIES" if dom == "synthesis" else "ANA_ENTRIES")
    nbytes, _ = algorithmic(dom, L, nlat, prec, ent)
    peak, peak_kind = peaks()
    achieved = nbytes / (avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "algorithmic_bytes": nbytes,
                "table_entries": ent if ent else sizes(L, nlat)[2],
                "avg_launch_ms": avg_ms, "timed_launches": stage[dom]["launches"],
                "duration_sampling": f"CUDA events around one launch in every {SAMPLE} in the timed region",
                "traffic": ncu_traffic(f"{dom}:{prec}:L511")}

    # end to end through the C ABI with host buffers (sphnse_rhs_host): every
    # step uploads its alpha from pinned memory and its F reaches pinned
    # memory (written there by the analysis); the host reads each step's F
    # one step later (host_wait), so that step k + 1's transfers overlap step
    # k's RHS
    pin_in = [torch.from_numpy(w["alpha0"]).pin_memory() for _ in range(2)]
    pin_out = [torch.empty_like(pin_in[0]).pin_memory() for _ in range(2)]
    for i in range(4):
        plan.host_wait(plan.rhs_host(pin_in[i & 1], pin_out[i & 1]))
    k_e2e = min(args.steps, 2000)
    chk = 0.0
    t0 = time.perf_counter()
    prev = None
    for i in range(k_e2e):
        tk = plan.rhs_host(pin_in[i & 1], pin_out[i & 1])
        if prev is not None:
            plan.host_wait(prev)
            chk += float(pin_out[(i - 1) & 1][1].real)   # the step's result, read on the host
        prev = tk
    plan.host_wait(prev)
    chk += float(pin_out[(k_e2e - 1) & 1][1].real)
    el = time.perf_counter() - t0
    el = max_over_ranks(world, el)
    e2e = {"value": replica_rate(world, k_e2e, el), "unit": UNIT, "h2d_bytes_per_step": pin_in[0].numel() * 16,
           "d2h_bytes_per_step": pin_out[0].numel() * 16, "steps": k_e2e,
           "api": "sphnse_rhs_host (pinned host buffers: alpha copied up before the step's kernels, F written by the analysis into the page-locked output; both overlap the previous step's RHS)",
           "finite": bool(np.isfinite(chk))}

    extras = {}
    # the extra workloads run on a single GPU only: under torchrun the line
    # reports the replicated headline, and the other GPUs are not held for them
    if not args.no_extras and world == 1:
        for p2 in ("fp64", "fp32", "bf16x3"):
            if p2 == prec:
                continue
            plan.set_precision(p2)
            ms = time_rhs(plan, a, out, min(args.steps, 200 if p2 == "fp64" else 1000), torch)
            extras[p2] = {"rhs_per_s": 1e3 / ms, "ms_per_rhs": ms}
        # accuracy of the timed path against the FP64 GPU path at full size
        plan.set_precision("fp64")
        f64 = plan.rhs(a).cpu().numpy()
        plan.set_precision(prec)
        fm = plan.rhs(a).cpu().numpy()
        extras["rel_err_vs_fp64"] = float(np.linalg.norm(fm - f64) / np.linalg.norm(f64))
        if "fp64" in extras:
            extras["speedup_vs_fp64"] = value / world / extras["fp64"]["rhs_per_s"]
        for name, fn in EXTRAS.items():
            try:
                extras[name] = fn(torch, prec, args)
            except Exception as e:  # an extra must not hide the headline line
                extras[name] = {"error": f"{type(e).__name__}: {e}"[:300]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16x3": "bf16x3+f32acc", "fp64": "f64"}[prec],
                "data": "synthetic",
                "config": arm_config(c, prec, world),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "stage_us_per_rhs": split, **extras}
        # the mixed-vs-FP64 comparison last, so that a truncated copy of the
        # line (its tail) still carries it
        tail = {}
        if "fp64" in extras:
            tail["fp64_rhs_per_s"] = extras["fp64"]["rhs_per_s"]
        for k in ("speedup_vs_fp64", "rel_err_vs_fp64", "mixed_errors_L511"):
            if k in extras:
                tail[k] = line.pop(k)
        if tail:
            tail["headline_rhs_per_s"] = value
            line["mixed_vs_fp64"] = tail
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _best_mixed():
    # the workload's stated mixed path: BF16 hi + lo split contractions on
    # tensor cores with FP32 accumulation
    return "bf16x3"


if __name__ == "__main__":
    main()
