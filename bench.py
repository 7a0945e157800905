#!/usr/bin/env python
"""Throughput of the MPCD + rigid-body time step on GB300.

One step = stream + body MD, site thermalisation (Eq. 7), binning, cell sums,
SRD collision with the cell thermostat, momentum transfer - the whole method
of arXiv 2604.14307 Sec. II - for every solvent particle and surface site.

Workload at N=1: the large suspension, L=200 (8M cells), density 10 (80M FP32
solvent particles), phi=0.3 of radius-4 spheres (8952 colloids) discretised
by 642-site icosphere shells (5.75M sites), SRD 130 deg with the cell-level
thermostat, dt=0.1, in the P32 form (FP32 state, int64 fixed-point cell sums,
FP64 bodies).  Inputs are synthetic (uniform solvent, Maxwell-Boltzmann
velocities, RSA placement).  Under torchrun each rank simulates its own
replica (different seed): weak scaling, no data-path collective.

Metric: particle-updates/s = (N_solvent + N_sites) * steps / time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/s (solvent+sites), FP32-mixed vs FP64 plain; % HBM peak"
UNIT = "particle-updates/s"
WORKLOAD = "suspension_L200_phi0.3_r4_642sites_density10_SRD130_thermostat"
FALLBACK_HBM_GBS = 6800.0


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-p64", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner")
    ap.add_argument("--tuning", default="",
                    help="block,tile,ctas_per_sm,staged of the solvent pass instead of the autotuner "
                         "(staged: 0 direct, 1 CTA ring, 2 warp-specialised, 3 ring per warp)")
    ap.add_argument("--L", type=int, default=200, help="box edge (tests use smaller boxes)")
    ap.add_argument("--workload", default="suspension",
                    choices=["suspension", "single_sphere_L10", "suspension_L50", "batched_single_sphere",
                             "batched_mixed_shapes", "phi_sweep_L120", "solvent_L200"],
                    help="suspension: the benchmark (box --L, rule --rule); the others are the smaller and "
                         "batched workloads and the paper-shaped phi sweep (--phi), for the record")
    ap.add_argument("--phi", type=float, default=0.3, help="volume fraction of phi_sweep_L120")
    ap.add_argument("--n-rep", type=int, default=0, help="replicas of the batched workloads (0: their default)")
    ap.add_argument("--thermostat", type=int, default=2, choices=[1, 2],
                    help="cell thermostat of the SRD workloads: E' ~ Gamma(3(Nc-1)/2, kT) drawn by "
                         "Marsaglia-Tsang rejection (2, the default) or as a sum of exponentials (1)")
    ap.add_argument("--rule", default="srd", choices=["srd", "at"],
                    help="collision rule of the workload: SRD with the cell thermostat (the benchmark) or "
                         "MPCD-AT (for the ALU-side measurement of the Philox/Box-Muller path)")
    ap.add_argument("--angular", action="store_true",
                    help="angular-momentum-conserving variant of the rule (SRD+a / MPCD-AT+a) on the "
                         "suspension or the pure solvent (--workload solvent_L200)")
    ap.add_argument("--no-protocols", action="store_true",
                    help="skip the transport-protocol measurements (momentum exchange, sedimentation, VACF)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.f.read().splitlines():
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def recorded_traffic(kernel: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e:
        return None
    src = os.path.join(ROOT, "paper_2604_14307_gb300", "csrc", e["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return e if h == e.get("source_sha256") else None


def host_cpu():
    """(threads this process may use, CPU model) of the host."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return len(os.sched_getaffinity(0)), model or "unknown"


def cpu_baseline(Bd, thermostat: int, steps: int = 4, L: int = 80):
    """The plain FP64 oracle as it stands on a bounded sample of the workload:
    an L=80 box with the same density, volume fraction, colloid radius and
    642-site shells (5.5M particle-updates per step), timed on all the host's
    cores (its OpenMP loops; the results equal the one-thread run's) and on one
    core.  The first step also serves as the FP64 reference of one GPU step of
    the FP32 form from the same state (oracle.parity: the FP32 form's error
    against the FP64 method on this sample)."""
    import oracle as O
    from oracle import parity as OP
    from paper_2604_14307_gb300 import inputs as I
    s = I.suspension(L, 10.0, 0.3, 4.0, 3, 10.0, I.SRD, thermostat, I.P32, seed=1, name="sample")
    st = I.initial_state(s)
    n = s.n_solvent + s.n_sites
    cores, model = host_cpu()
    used = O.set_threads(cores)
    t0 = time.perf_counter()
    ref = OP.fp64_reference(s, st)          # one FP64 step: stream, then the collision with its trace
    times = [time.perf_counter() - t0]
    osys, _, _ = ref
    ost = O.OracleState(osys, st)
    O.step(osys, ost, 1)                    # the same step without the trace (not timed)
    for _ in range(steps - 1):
        t0 = time.perf_counter()
        O.step(osys, ost, 1)
        times.append(time.perf_counter() - t0)
    O.set_threads(1)
    ost1 = O.OracleState(osys, st)
    t1 = []
    for _ in range(2):
        t0 = time.perf_counter()
        O.step(osys, ost1, 1)
        t1.append(time.perf_counter() - t0)
    # the FP32 form on the GPU, one unpipelined step from the same state
    sim = Bd.Simulation(s, sort_period=-1)
    sim.set_debug(True)
    sim.set_state(st)
    sim.stream()
    sim.couple(Bd.MPCD_PRE)
    sim.collide()
    d = sim.debug_cells()
    sim.couple(Bd.MPCD_POST)
    g = sim.get_state()
    sim.close()
    par = OP.compare(s, st, g, d["site_cell"], d["shift"], ref=ref, params=d["params"])
    return {"value": n / float(np.median(times)), "unit": UNIT, "cores": used, "kind": "oracle",
            "mode": "plain FP64 (no float32 decision, no fixed-point word)",
            "host_threads": cores, "cpu_model": model,
            "sample": f"{steps} plain-FP64 oracle step(s) of an L={L} box with the workload's density, "
                      f"phi, radius and sites ({n} particle-updates per step) on {used} threads, median time",
            "single_thread": {"value": n / float(np.median(t1)), "unit": UNIT, "cores": 1,
                              "sample": f"2 steps of the same box on one thread, median time"},
            "seconds": float(sum(times) + sum(t1))}, par


def body_protocols(sim, stream, steps: int = 20):
    """On the benchmark suspension: the sedimentation protocol of Sec. III.B (a
    force of 0.5 along x on every colloid, balanced on the solvent, which then
    streams under a constant force) and the per-body velocity autocorrelations
    of Sec. III.A; step time with and without each."""
    import torch

    def timed_steps(k):
        sim.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    base = timed_steps(steps)
    sim.set_body_force([0.5, 0.0, 0.0])
    forced = timed_steps(steps)
    D = sim.body_displacements()
    sim.set_body_force([0.0, 0.0, 0.0])
    # per-body velocity autocorrelations (Sec. III.A), 50 lags, every step
    sim.set_vacf(50, 1)
    with_vacf = timed_steps(steps)
    ct, cr, cnt = sim.vacf()
    sim.set_vacf(0, 1)
    return {"sedimentation": {"force": [0.5, 0.0, 0.0], "steps": steps, "ms_per_step_without": base,
                              "ms_per_step_with": forced, "mean_body_displacement_x": float(np.mean(D[:, 0]))},
            "vacf": {"n_lags": 50, "every": 1, "steps": steps, "ms_per_step_without": base,
                     "ms_per_step_with": with_vacf, "mean_C_T0": float(np.mean(ct[:, 0]))}}


def rnemd_protocol(Bd, I, stream, hbm, steps: int = 20):
    """The viscosity protocol of Sec. III.B on the paper's box: L = 120 x 240 x
    120 cells of pure solvent at 5 particles per cell (17.28M particles, P32,
    SRD + cell thermostat), exchanging up to 100 pairs between the slabs at
    y = 0 and y = 120 every step.  Reports the exchange kernels' time (CUDA
    events inside mpcd_step), their algorithmic bytes (two passes reading y and
    v_x of every particle) against the HBM peak, the step time with and without
    the exchange, and the oracle's time for one exchange on the same state."""
    import torch
    import oracle as O
    L = (120, 240, 120)
    prm = I.Params(rule=I.SRD, thermostat=1, precision=I.P32, seed=7)
    system = I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [L], 5.0, [[]], "rnemd_solvent",
                            placement_seed=7)
    st = I.initial_state(system)
    n = system.n_solvent
    sim = Bd.Simulation(system)
    sim.set_state(st)

    def timed_steps(k):
        sim.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    base = timed_steps(steps)
    sim.set_rnemd(y_a=0.0, y_b=120.0, width=1.0, v_target=0.5, max_pairs=100, period=1)
    with_x = timed_steps(steps)
    sim.set_profiling(True)
    sim.reset_profile()
    sim.step(steps)
    prof = sim.profile()
    sim.set_profiling(False)
    p, npairs = sim.rnemd_totals()
    sim.close()
    pk = prof["rnemd"]
    ms_x = pk["total_ms"] / max(pk["launches"], 1)
    n_slab = 2 * L[0] * L[2] * 5
    alg = 4.0 * n + n_slab * (4.0 + 16.0 + 16.0)   # the candidates (a few hundred entries) are not counted
    osys = O.OracleSystem(system)
    ost = O.OracleState(osys, st, compute_forces=False)
    t0 = time.perf_counter()
    O.rnemd_exchange(osys, ost, 0.0, 120.0, 1.0, 0.5, 100)
    t_cpu = time.perf_counter() - t0
    return {"config": {"box": list(L), "n_solvent": n, "density": 5, "max_pairs": 100, "slab_width": 1.0,
                       "v_target": 0.5, "period_steps": 1, "form": "P32", "rule": "SRD alpha=130 + cell thermostat"},
            "ms_per_exchange": ms_x, "launches_per_exchange": 3,
            "roofline": {"bound": "hbm", "achieved": alg / (ms_x / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / (ms_x / 1e3) / 1e9 / hbm, "bytes_per_exchange": alg,
                         "bytes_note": ("y of every particle (4 B); v_x of the slab members, their 16-B list "
                                        "entries written and read back (36 B per member)")},
            "ms_per_step_without": base, "ms_per_step_with": with_x,
            "pairs_per_exchange": npairs / (2 * steps + 3),
            "cpu_baseline": {"value": 1.0 / t_cpu, "unit": "exchanges/s", "cores": 1, "kind": "oracle",
                             "sample": f"one oracle exchange on the same {n}-particle state"}}


def run_reference(a, ws, rank):
    if rank != 0:
        return
    import oracle as O
    from paper_2604_14307_gb300 import inputs as I
    L = 80
    s = I.suspension(L, 10.0, 0.3, 4.0, 3, 10.0, I.SRD, a.thermostat, I.P32, seed=1, name="sample")
    st = I.initial_state(s)
    cores, model = host_cpu()
    used = O.set_threads(cores)                  # all host cores (OpenMP loops; same results as one thread)
    osys = O.OracleSystem(s, precision=O.P64)   # the plain FP64 method
    ost = O.OracleState(osys, st)
    n = s.n_solvent + s.n_sites
    O.step(osys, ost, a.warmup)
    t0 = time.perf_counter()
    O.step(osys, ost, a.steps)
    dt = time.perf_counter() - t0
    v = n * a.steps / dt
    sample = (f"plain FP64 oracle on {used} host threads ({model}), each step one step of an L={L} box "
              f"with the workload's density, phi, radius and 642-site shells ({n} particle-updates)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_L": L},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                         "cpu_model": model},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def place_timed_call(step_call, steps: int, period: int) -> int:
    """Run `step_call` (one mpcd_step(steps) call) from the state right after a
    re-sort until the next call replays a recorded graph and holds its share of
    re-sorts; returns that share.

    mpcd_step(n) replays a CUDA graph keyed by (n, solvent buffer parity,
    passes since the last re-sort); a call of n steps runs n - 1 fused passes,
    each counting towards the next re-sort, so from `since` it re-sorts
    (since + n - 1) // period times (each flips the parity) and ends at
    (since + n - 1) % period.  First every key of the replay cycle is recorded;
    then, since the call right after the re-sort would hold none, the phase is
    moved within the cycle until the call holds ceil((n - 1) / period)."""
    since, par, seen = 0, 0, set()

    def advance():
        nonlocal since, par
        step_call()
        par ^= ((since + steps - 1) // period) & 1
        since = (since + steps - 1) % period

    while steps >= 2 and (since, par) not in seen:
        seen.add((since, par))
        advance()
    resorts = -(-(steps - 1) // period) if steps >= 2 else 0
    for _ in range(2 * period):   # the cycle reaches such a phase (since = period - gcd)
        if steps < 2 or (since + steps - 1) // period >= resorts:
            break
        advance()
    return resorts


def main():
    a = args_()
    ws, rank, local = dist_env()
    if a.impl == "reference":
        run_reference(a, ws, rank)
        return
    import torch
    import torch.distributed as dist

    from paper_2604_14307_gb300 import binding as Bd
    from paper_2604_14307_gb300 import build_lib
    from paper_2604_14307_gb300 import inputs as I

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build_lib.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    L = a.L
    rule, thermo = (I.SRD, a.thermostat) if a.rule == "srd" else (I.AT, 0)

    def make_system(precision):
        """The workload in the given arithmetic form (seeded per rank)."""
        seed = 1 + rank
        if a.workload == "single_sphere_L10":
            return I.single_sphere_L10(precision, seed=seed), "single_sphere_L10_162sites_density5_SRD130"
        if a.workload == "suspension_L50":
            return I.suspension_L50(precision, seed=seed), "suspension_L50_phi0.2_r3_642sites_density5_MPCD-AT"
        if a.workload == "batched_single_sphere":
            n = a.n_rep or 4096
            return (I.batched_single_sphere(n_rep=n, precision=precision, seed=seed),
                    f"batched_{n}x_single_sphere_L12-24_162sites_density5_SRD130")
        if a.workload == "batched_mixed_shapes":
            n = a.n_rep or 256
            return (I.batched_mixed_shapes(n_rep=n, precision=precision, seed=seed),
                    f"batched_{n}x_mixed_shapes_L20-40_MPCD-AT")
        if a.workload == "solvent_L200":
            prm = I.Params(rule=rule, thermostat=thermo, precision=precision, seed=seed, angular=int(a.angular))
            name = "solvent_L200_density10_" + ("SRD130_thermostat" if rule == I.SRD else "MPCD-AT") + \
                ("+a" if a.angular else "")
            return I.build_system(prm, [I.sphere_shape(2.0, 2, 5.0)], [(L, L, L)], 10.0, [[]], name,
                                  placement_seed=seed), name
        if a.workload == "phi_sweep_L120":
            name = f"suspension_L120_phi{a.phi:g}_d6_162sites_density5_SRD130_thermostat"
            return I.suspension(120, 5.0, a.phi, 3.0, 2, 5.0, I.SRD, 1, precision, seed=seed, name=name), name
        w = WORKLOAD if a.rule == "srd" else WORKLOAD.replace("SRD130_thermostat", "MPCD-AT")
        sysm = I.suspension(L, 10.0, 0.3, 4.0, 3, 10.0, rule, thermo, precision, seed=seed, name=w)
        if a.angular:
            sysm.params.angular = 1
            w += "+a"
        return sysm, w

    system, workload = make_system(I.P32)
    default_workload = a.workload == "suspension" and not a.angular
    state = I.initial_state(system)
    n_upd = system.n_solvent + system.n_sites

    sim = Bd.Simulation(system, device=local)
    sim.set_state(state)
    if a.tuning:
        tb, tt, tc, tsg = (int(v) for v in a.tuning.split(","))
        sim.set_tuning(block=tb, tile=tt, ctas_per_sm=tc, staged=tsg)
        tuning = sim.tuning()
    else:
        tuning = sim.tuning() if a.no_tune else sim.autotune(steps_per_trial=10)
    sim.step(a.warmup)
    # every graph of the replay cycle is recorded and the timed call placed so
    # that it replays graphs and holds its share of re-sorts
    sim.sort()
    period = max(1, int(tuning["sort_period"]))
    resorts = place_timed_call(lambda: sim.step(a.steps), a.steps, period)
    torch.cuda.synchronize()

    # ------------------------------------------------------- timed (graph)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(a.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = n_upd * a.steps * ws / (ms_max / 1e3)

    # ------------------------------------ profiled pass (per-kernel events)
    # the same number of steps launched kernel by kernel with CUDA events on
    # each kernel's stream (no graph); it gives the per-kernel times and the
    # roofline of the dominant kernel, and its own step time
    sim.set_profiling(True)
    sim.reset_profile()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    sim.step(a.steps)
    p1.record(stream)
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1)
    prof = sim.profile()
    sim.set_profiling(False)

    # roofline of the dominant kernel: the fused solvent pass (the site/body
    # kernels run beside it on a second stream, so their event spans overlap it)
    hbm, src = peaks()
    name = "solvent_fused" if "solvent_fused" in prof else max(prof.items(), key=lambda kv: kv[1]["total_ms"])[0]
    pk = prof[name]
    per_launch_ms = pk["total_ms"] / max(pk["launches"], 1)
    achieved = pk["bytes_per_launch"] / (per_launch_ms / 1e3) / 1e9
    tr = recorded_traffic(name) if (a.rule == "srd" and default_workload) else None   # the record is of the benchmark
    traffic = None
    if tr is not None:
        traffic = float(tr["bytes_per_launch_per_particle"]) * system.n_solvent
    roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs copy)",
            "bytes_per_launch": pk["bytes_per_launch"], "ms_per_launch": per_launch_ms,
            "share_of_step": pk["total_ms"] / ms_prof,
            "measured_in": "profiled pass (kernel-by-kernel launches with CUDA events, same step count)"}
    launches = a.steps + sum(v["launches"] * (6 if k == "sort" else 1) for k, v in prof.items())
    # whole-step effective bandwidth: algorithmic bytes of every kernel / step time
    step_bytes = sum(v["bytes_per_launch"] * v["launches"] for v in prof.values()) / a.steps
    hbm_eff = {"bytes_per_update": step_bytes / n_upd, "gbs": step_bytes / (ms / a.steps / 1e3) / 1e9}
    hbm_eff["frac"] = hbm_eff["gbs"] / hbm
    kernels = {k: {"launches": v["launches"], "ms_per_launch": v["total_ms"] / max(v["launches"], 1),
                   "share": v["total_ms"] / ms_prof} for k, v in prof.items()}
    profiled = {"ms_per_step": ms_prof / a.steps, "steps": a.steps,
                "note": "kernel-by-kernel launches with CUDA events (no graph); the headline is the graph replay"}

    # ------------------------------------------------ end to end (host buffers)
    hb = sim.host_buffers(pinned=True)
    step0 = sim.get_state_buffers(hb)
    state_bytes = sum(v.nbytes for v in hb.values())
    # one untimed pass of the same sequence (warm-up: first-use costs of the
    # pinned buffers and the state permutations, and the CUDA graph of
    # mpcd_step(steps), which the timed pass then replays)
    sim.set_state_buffers(hb, step0)
    sim.step(a.steps)
    sim.get_state_buffers(hb)
    sim.diagnostics()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_state_buffers(hb, step0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    sim.step(a.steps)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    sim.get_state_buffers(hb)
    diag = sim.diagnostics()
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    e2e_parts = {"set_state_ms": (t1 - t0) * 1e3, "steps_ms": (t2 - t1) * 1e3,
                 "get_state_and_diagnostics_ms": (time.perf_counter() - t2) * 1e3}
    te_t = torch.tensor([te], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(te_t, op=dist.ReduceOp.MAX)
    e2e = {"value": n_upd * a.steps * ws / float(te_t.item()), "unit": UNIT,
           "h2d_bytes_per_step": state_bytes / a.steps, "d2h_bytes_per_step": (state_bytes + 80) / a.steps,
           "how": "mpcd_set_state from pinned host + mpcd_step(steps) + mpcd_get_state to pinned host "
                  "+ mpcd_diagnostics, wall clock", "parts": e2e_parts}
    protocols_on = rank == 0 and not a.no_protocols and default_workload
    bodyp = body_protocols(sim, stream) if protocols_on else {}
    sim.close()
    del hb

    # ------------------------------------------------------ plain FP64 form
    p64 = None
    if not a.no_p64:
        s64, _ = make_system(I.P64)
        sim64 = Bd.Simulation(s64, device=local)
        sim64.set_state(state)
        k64 = max(3, a.steps // 5)
        sim64.step(2)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        sim64.step(k64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        p64 = {"value": n_upd * k64 * ws / (ms64 / 1e3), "unit": UNIT, "steps": k64,
               "ms_per_step": ms64 / k64, "dtype": "f64",
               "speedup_p32_over_p64": value / (n_upd * k64 * ws / (ms64 / 1e3))}
        sim64.close()
    del state

    protocols = None
    if protocols_on:
        protocols = {"rnemd": rnemd_protocol(Bd, I, stream, peaks()[0]), **bodyp}

    cpu, parity = None, None
    if rank == 0 and not a.no_cpu and default_workload:   # the oracle sample is of the benchmark composition
        cpu, parity = cpu_baseline(Bd, a.thermostat)
        cpu.pop("seconds", None)

    state_bytes_dev = system.n_solvent * 28 + system.n_cells * 56
    l2_note = ("no flush: state per GPU (%.1f GB) is larger than L2 (129 MB)" % (state_bytes_dev / 1e9)
               if state_bytes_dev > 129e6 else
               "no flush: the state fits in L2 (129 MB), so the bandwidth fraction is not meaningful")
    rule_note = ("SRD alpha=130" + ({1: " + cell-level thermostat (E' as a sum of exponentials)",
                                      2: " + cell-level thermostat (E' by Marsaglia-Tsang rejection)"}
                                     .get(system.params.thermostat, ""))
                 if system.params.rule == I.SRD else "MPCD-AT (Andersen thermostat rule)")
    if getattr(system.params, "angular", 0):
        rule_note += ", angular-momentum-conserving (+a, unfused step)"
    if a.workload == "suspension":
        config = {"workload": workload, "L": L, "density": 10, "phi": 0.3, "colloid_radius": 4.0}
    else:
        config = {"workload": workload, "n_replicas": system.n_rep}
        if a.workload == "phi_sweep_L120":
            config.update({"L": 120, "density": 5, "phi": a.phi, "colloid_radius": 3.0})
        if a.workload == "solvent_L200":
            config.update({"L": L, "density": 10})
    config.update({"n_solvent": system.n_solvent, "n_bodies": system.n_bodies, "n_sites": system.n_sites,
                   "n_cells": system.n_cells, "form": "P32: FP32 state, int64 fixed-point cell sums, FP64 bodies",
                   "rule": rule_note, "dt": 0.1, "l2": l2_note, "tuning": tuning,
                   "resorts_in_timed_call": resorts,
                   "parallelism": f"replicas x{ws} (one box per GPU)"})
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config,
            "roofline": roof, "hbm_effective": hbm_eff, "kernels": kernels, "profiled_pass": profiled,
            "kernels_note": ("sites_post, body_impulse, body_md, body_force and the next step's sites_pre run "
                             "on a second stream beside solvent_fused; their event spans include shared time"),
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
            "p64": p64, "protocols": protocols, "parity_vs_fp64": parity,
            "diag_check": {"ke_solvent_per_particle": diag["ke_solvent"] / system.n_solvent},
        }
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
