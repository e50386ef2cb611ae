#!/usr/bin/env python
"""Benchmark of the energy-DG / Galerkin-difference hot path on GB300.

Metric: DOF-steps/s = (elements x (N+1)^d) x RK4 steps / second (Section
3.3 counts DOF this way).  One benchmark step = R classic RK4 steps of the
whole semi-discretisation (traces, fluxes, lifts, stiffness, constrained
u_t solve, mass inversion, stage combination) through gdg_step.

Default workload: 2-D constant coefficient u_tt = Laplace u on [0,1]^2,
64 x 64 elements of 8 x 8 GD cells, p = 5, upwind flux, u = 0 on the
boundary, standing mode cos(sqrt2 pi t) sin(pi x) sin(pi y), dt = 0.15 h
(0.8 of the largest RK4-stable step for the upwind p = 5 operator).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gdg|reference]
Under torchrun (N > 1) the ranks advance one mesh of 64 x 64N elements
together: each owns a 64 x 64 band of element rows (weak scaling), and the
face traces along the band edges go to the neighbouring ranks (NCCL point
to point) before every RK stage; `value` counts the DOF of all bands.
"""
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

WORKLOAD = dict(dim=2, n=(64, 64), N=8, p=5, flux="upwind", T=1.0, cfl=0.15)
WORKLOAD_NAME = ("2-D constant-coefficient wave, 64x64 elements of 8x8 GD cells, p=5, upwind, "
                 "Dirichlet, standing mode; modified-basis diagonalised route")


def dof(w=WORKLOAD):
    nel = 1
    for k in w["n"]:
        nel *= k
    return nel * (w["N"] + 1) ** w["dim"]


def executed_flops_per_stage_launch(w=WORKLOAD):
    """FP64 flops the parity stage kernels execute per stage launch (FMA = 2,
    averaged over the four RK stages).  With the modes ordered even first,
    gR = +-gL and eR = +-eL, so per element 2-D: fluxes 2 directions x n1
    lines x (2 faces x 7 + 4 sums/differences); per modal entry 23.5: k_u with
    the lifts folded into the solve 4, r_v 5, the RK update 6.5 (stage 1: 4,
    stages 2-3: 8, stage 4: 6), the traces' split dots 8; + 8 n1 trace
    sums/differences.  (ncu on the persistent step: 2,339 per element and
    stage from its DFMA / DADD / DMUL counts, this count 2,300.)"""
    n1 = w["N"] + 1
    nel = w["n"][0] * w["n"][1]
    return nel * (44 * n1 + 23.5 * n1 * n1)


# FP64 peak derived from unit counts and clock: 152 SMs x 2070 MHz x 4 FP64
# flop/clk/SM (2 FP64 FMA lanes per SM per clock) = 1.259 TFLOP/s.  The bench
# also measures, in the same process, what an FMA-chain kernel sustains
# (gdg_probe_fp64) and reports every FP64 fraction against both.
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12
# FP32 peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# Algorithmic FP64 flops per DOF per RK stage of the constant-coefficient
# modal route (the method's own count for the modified basis: fluxes, rank-one
# lifts per line, diagonal solves, RK combination, traces), the figure the
# headline roofline uses.
ALG_FLOPS_PER_DOF_STAGE = 40.0


def hbm_peak_gbs():
    """Measured HBM copy bandwidth (MEASURED_PEAKS.json at the repository
    root, a STREAM-style copy measured on this GPU model), else 6.8 TB/s, one
    earlier copy measurement on a GB300."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s)"


def fp64_probe_tflops(iters=4000, reps=3):
    """FP64 rate the GPU sustains on independent FMA chains (gdg_probe_fp64,
    CUDA events on the launching stream, best of reps)."""
    import torch
    from paper_2105_01722_gb300 import gdg
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    best = 0.0
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        flops = gdg.probe_fp64(iters, sink)
        e1.record()
        torch.cuda.synchronize()
        if r:   # the first launch warms up
            best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def var_counts(n1, it_u, it_v, form, sweeps_u=0.0, sweeps_v=0.0):
    """Algorithmic work per element and RK stage of the variable-coefficient
    path (Section 7.1), NA = n1^2 nodes: (FP64 flops, FP32 flops, bytes).
      stiffness term of r_v: one NA x NA product, 2 NA^2;
      face terms: per face a 3 n1 x 6 n1 operator on the own and neighbour
        face lines, 4 faces: 144 n1^2; lift assembly 8 NA; RK combination 8 NA;
      PCG iteration: one NA x NA product (2 NA^2), the frozen-coefficient
        preconditioner (four n1 x n1 contractions, 8 n1^3) and the vector
        work (12 NA); each solve also applies the preconditioner once first;
      mixed: the iterations in FP32; in FP64 one residual product per
        refinement sweep (2 NA^2) and the first preconditioned step;
      inverse: the folded operators, 189 columns of NA (2 * 189 NA), no PCG;
    bytes: the FP64 element matrices (PCG: S_c2 and M_J, 2 NA^2 * 8; mixed:
    their FP32 copies plus the FP64 matrices once per sweep; inverse: the
    folded operators 189 NA * 8) plus the face operators (72 n1^2 * 8) and
    the state."""
    NA = n1 * n1
    face = 144 * n1 * n1 + 16 * NA
    it_cost = 2 * NA * NA + 8 * n1 ** 3 + 12 * NA
    state = 8 * NA * 8
    if form == "fp64":
        f64 = 2 * NA * NA + face + (it_u + it_v) * it_cost + 2 * 8 * n1 ** 3
        return f64, 0.0, 2 * NA * NA * 8 + 72 * n1 * n1 * 8 + state
    if form == "mixed":
        f64 = 2 * NA * NA + face + (1 + sweeps_u + 1 + sweeps_v) * 2 * NA * NA + 8 * n1 ** 3
        f32 = (it_u + it_v) * it_cost
        byt = 2 * NA * NA * 4 + (2 + sweeps_u + sweeps_v) * NA * NA * 8 + 72 * n1 * n1 * 8 + state
        return f64, f32, byt
    if form == "inverse":
        cols = 12 * n1 + NA
        return 2 * cols * NA + face, 0.0, cols * NA * 8 + 72 * n1 * n1 * 8 + state
    raise ValueError(form)


def alu_roofline(f64, f32, byt, seconds, probe):
    """Roofline block of a whole-step measurement: achieved FP64 (and FP32)
    rates and HBM bandwidth from the algorithmic counts over the measured
    time; bound = the resource with the largest fraction."""
    hbm, hbm_src = hbm_peak_gbs()
    a64 = f64 / seconds / 1e12
    a32 = f32 / seconds / 1e12
    gbs = byt / seconds / 1e9
    fr = {"fp64": a64 / FP64_PEAK_TFLOPS, "fp32": a32 / FP32_PEAK_TFLOPS, "hbm": gbs / hbm}
    top = max(fr, key=fr.get)
    out = {"bound": "alu" if top != "hbm" else "hbm",
           "achieved": a64 if top == "fp64" else (a32 if top == "fp32" else gbs),
           "peak": FP64_PEAK_TFLOPS if top == "fp64" else (FP32_PEAK_TFLOPS if top == "fp32" else hbm),
           "unit": "TFLOP/s" if top != "hbm" else "GB/s", "frac": fr[top], "resource": top,
           "fp64_tflops": a64, "frac_fp64": fr["fp64"], "frac_fp64_of_probe": a64 / probe if probe else None,
           "hbm_gbs": gbs, "frac_hbm": fr["hbm"], "hbm_peak_source": hbm_src}
    if f32:
        out.update(fp32_tflops=a32, frac_fp32=fr["fp32"])
    return out

# FP64 thread instructions (DFMA + DADD + DMUL) per element and RK stage of the
# persistent step, from the ncu capture of the current kernel (16.04 M + 4.81 M
# + 1.44 M per one-step launch of the 64x64 mesh): the FP64 pipe's share of a
# stage's time follows from it at 2 FP64 lanes per SM and clock.
STEP2R_FP64_INST_PER_ELEMENT_STAGE = 22.28e6 / (4 * 4096)

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per RK stage of
# this workload, from one ncu capture per stage kernel (None for a kernel
# without a capture of its current code):
#   k_stage2p: the mean over the four stage launches of one RK4 step
#   k_step2r: one persistent launch of one RK4 step, over its 4 stages
STAGE_TRAFFIC_BYTES = {0: None, 3: (7.772160e6 + 256) / 4}


PROBE = {}   # in-process measured peaks (filled by run_gdg)


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


_ORACLE_TIMER = r"""
import json, sys, time
sys.path.insert(0, %r)
import numpy as np
from oracle import dg_const as dc, timeint as ti
from paper_2105_01722_gb300 import inputs
w = %r
nsteps, target_s = %d, %f
prob = dc.Problem(dim=w["dim"], n=tuple(w["n"]), N=w["N"], p=w["p"], flux=w["flux"])
ops = dc.operators(prob)
X, Y = inputs.cartesian_nodes(tuple(w["n"]), w["N"])
U, V = inputs.standing_mode_2d(X, Y)
ne = w["n"][0] * w["n"][1]
U, V = U.reshape(ne, -1), V.reshape(ne, -1)
dt = w["cfl"] / (w["n"][0] * w["N"])
f = lambda t, U, V: dc.time_derivative(prob, U, V, ops)
t0 = time.perf_counter(); U, V = ti.rk4_step(f, U, V, 0.0, dt); t1 = time.perf_counter()
rk = max(1, int(target_s / max(t1 - t0, 1e-6)))
for k in range(nsteps):
    t0 = time.perf_counter()
    U, V = ti.integrate(f, U, V, dt, dt, rk)
    t1 = time.perf_counter()
    print(json.dumps({"rk_steps": rk, "seconds": t1 - t0}), flush=True)
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_steps(nsteps, target_s, threads=1):
    """Time the FP64 oracle (as it stands) on the host cores with `threads`
    BLAS/OpenMP threads: `nsteps` samples of about `target_s` seconds, each a
    number of RK4 steps of the full benchmark mesh.  Returns
    [(rk_steps, seconds)] or an error."""
    code = _ORACLE_TIMER % (ROOT, WORKLOAD, nsteps, target_s)
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t,
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        return None, (r.stderr.strip().splitlines() or ["failed"])[-1]
    rows = [json.loads(x) for x in r.stdout.strip().splitlines() if x.startswith("{")]
    return [(d["rk_steps"], d["seconds"]) for d in rows], None


def cpu_baseline(target_s=12.0):
    """Bounded samples (about target_s of CPU work each) of the oracle: with
    every host core as BLAS threads (the reported figure) and with one."""
    cores = host_cores()
    out = None
    for threads in (cores, 1):
        rows, err = _oracle_steps(1, target_s, threads)
        if rows is None:
            rec = {"value": None, "unit": "DOF-steps/s", "cores": threads, "kind": "oracle",
                   "sample": "failed: " + err}
        else:
            rk, sec = rows[0]
            rec = {"value": dof() * rk / sec, "unit": "DOF-steps/s", "cores": threads, "kind": "oracle",
                   "sample": "%d RK4 steps of the full 64x64 p=5 mesh (%.1f s, numpy FP64, %d BLAS threads)"
                             % (rk, sec, threads)}
        if out is None:
            out = rec
        else:
            out["single_thread"] = rec
    return out


def run_reference(args):
    """The oracle arm: W + K bounded samples in one process, the K timed."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    total = args.steps + args.warmup
    cores = host_cores()
    rows, err = _oracle_steps(total, max(0.5, 120.0 / total), cores)
    if rows is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + err}))
        return 0
    timed = rows[args.warmup:]
    rk_total = sum(r for r, _ in timed)
    sec_total = sum(s for _, s in timed)
    value = dof() * rk_total / sec_total
    sample = ("%d timed samples of %d RK4 steps each on the full 64x64 p=5 mesh (numpy FP64, %d BLAS threads)"
              % (len(timed), timed[0][0], cores))
    line = {"impl": "reference", "metric": "DOF-steps/s", "value": value, "unit": "DOF-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec_total / len(timed), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "elements": list(WORKLOAD["n"]), "N": WORKLOAD["N"],
                       "p": WORKLOAD["p"], "dof": dof()},
            "cpu_baseline": {"value": value, "unit": "DOF-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "DOF-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _timed_ms(fn):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def forms_variable(steps=16):
    """Mapped 128 x 128 elements, c^2 = 1 + 0.5 sin 2pi x cos 2pi y, p = 3 and 5,
    PCG to rtol 1e-10: FP64 against FP32-inner / FP64-refined PCG (same stopping
    test, so equal accuracy by construction) and against precomputed element
    inverses (exact solves); the trajectories are compared with the FP64 PCG's."""
    import numpy as np
    import torch
    from paper_2105_01722_gb300 import gdg, inputs
    out = {}
    for p in (3, 5):
        X, Y = inputs.mapped_nodes((128, 128), 8, 0.05)
        C2 = inputs.c2_sine(X, Y)
        U0 = inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.05)
        dt = 0.1 / 1024 / np.sqrt(1.5)
        states = {}
        for prec, solver, name in ((gdg.FP64, gdg.SOLVE_PCG, "fp64"), (gdg.MIXED, gdg.SOLVE_PCG, "mixed"),
                                   (gdg.FP64, gdg.SOLVE_INVERSE, "inverse")):
            ctx = gdg.Context(gdg.make_problem(2, (128, 128), 8, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y,
                                               c2_nodes=C2, pcg_rtol=1e-10, pcg_maxit=100, precision=prec,
                                               solver=solver))
            u = torch.tensor(U0.ravel(), device="cuda")
            v = torch.zeros_like(u)
            ctx.step(u, v, 0.0, dt, 8)
            ctx.step_stats()
            ms = _timed_ms(lambda: ctx.step(u, v, 0.0, dt, steps))
            su, sv = ctx.step_stats()
            states[name] = torch.cat([u, v]).cpu().numpy()
            f64, f32, byt = var_counts(9, su["mean_iters"], sv["mean_iters"], name,
                                       su["mean_sweeps"], sv["mean_sweeps"])
            stages = 128 * 128 * 4 * steps
            out["p%d_%s" % (p, name)] = {
                "dof_steps_per_s": 128 * 128 * 81 * steps / (ms / 1e3), "ms_per_step": ms / steps,
                "pcg_u_mean_iters": su["mean_iters"], "pcg_v_mean_iters": sv["mean_iters"],
                "refine_sweeps_u": su["mean_sweeps"], "refine_sweeps_v": sv["mean_sweeps"],
                "roofline": alu_roofline(f64 * stages, f32 * stages, byt * stages, ms / 1e3, PROBE.get("fp64")),
                "per_element_stage": {"fp64_flops": f64, "fp32_flops": f32, "bytes": byt}}
            ctx.close()
        b = states["fp64"]
        for name in ("mixed", "inverse"):
            a = states[name]
            out["p%d_%s_vs_fp64_rel_l2" % (p, name)] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    out["workload"] = ("2-D variable c^2 on the sine-mapped unit square, 128x128 elements of 8x8 cells, "
                       "Gaussian pulse, PCG rtol 1e-10, %d RK4 steps after 8 warm-up steps" % steps)
    return out


def coarse_in_fine(n, N):
    """Indices into a (2n x 2n elements, N) nodal array of the nodes of the
    (n x n, N) mesh: coarse node (ey, ex, j, i) sits at fine element
    (2 ey + (j > N/2), 2 ex + (i > N/2)), node (2 j - N [j > N/2], 2 i - N [i > N/2])."""
    import numpy as np
    n1 = N + 1
    ey, ex, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n1), np.arange(n1), indexing="ij")
    hy, hx = (j > N // 2).astype(int), (i > N // 2).astype(int)
    fy, fx = 2 * ey + hy, 2 * ex + hx
    fj, fi = 2 * j - N * hy, 2 * i - N * hx
    return (((fy * (2 * n) + fx) * n1 + fj) * n1 + fi).ravel()


def forms_equal_error(T=0.25, ps=(3, 5), n=128):
    """Equal final error for the variable-coefficient forms (mapped n x n mesh,
    c^2 = 1 + 0.5 sin 2pi x cos 2pi y, Gaussian pulse of width 0.05): u at
    time T of FP64 PCG, mixed PCG and element inverses, each against an FP64
    reference on the 2n x 2n mesh of the same map with the same N (cells of
    half the size; every coarse node is a fine node), advanced with element
    inverses (exact element solves) at half the step.  A form matches when its
    error is at most 1.05x the FP64 PCG's."""
    import numpy as np
    import torch
    from paper_2105_01722_gb300 import gdg, inputs
    N = 8
    out = {"T": T, "mesh": [n, n], "reference_mesh": [2 * n, 2 * n],
           "reference": "FP64 element inverses on the 2x refined mesh (h/2), dt/2"}
    dt0 = 0.1 / (n * N) / np.sqrt(1.5)
    for p in ps:
        res = {}
        Xf, Yf = inputs.mapped_nodes((2 * n, 2 * n), N, 0.05)
        X, Y = inputs.mapped_nodes((n, n), N, 0.05)
        idx = coarse_in_fine(n, N)
        assert np.abs(Xf.ravel()[idx] - X.ravel()).max() < 1e-13 and np.abs(Yf.ravel()[idx] - Y.ravel()).max() < 1e-13
        steps = int(round(T / dt0))
        dt = T / steps
        t0 = time.perf_counter()
        ctx = gdg.Context(gdg.make_problem(2, (2 * n, 2 * n), N, p, coef=gdg.COEF_NODAL, x_nodes=Xf, y_nodes=Yf,
                                           c2_nodes=inputs.c2_sine(Xf, Yf), solver=gdg.SOLVE_INVERSE))
        u = torch.tensor(inputs.gaussian_pulse(Xf, Yf, 0.5, 0.5, 0.05).ravel(), device="cuda")
        v = torch.zeros_like(u)
        ctx.step(u, v, 0.0, 0.5 * dt, 2 * steps)
        ref = u.cpu().numpy()[idx]
        ctx.close()
        del u, v
        torch.cuda.empty_cache()
        res["reference_s"] = time.perf_counter() - t0
        for prec, solver, name in ((gdg.FP64, gdg.SOLVE_PCG, "fp64"), (gdg.MIXED, gdg.SOLVE_PCG, "mixed"),
                                   (gdg.FP64, gdg.SOLVE_INVERSE, "inverse")):
            ctx = gdg.Context(gdg.make_problem(2, (n, n), N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y,
                                               c2_nodes=inputs.c2_sine(X, Y), pcg_rtol=1e-10, pcg_maxit=100,
                                               precision=prec, solver=solver))
            u = torch.tensor(inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.05).ravel(), device="cuda")
            v = torch.zeros_like(u)
            t1 = time.perf_counter()
            ctx.step(u, v, 0.0, dt, steps)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t1
            a = u.cpu().numpy()
            res[name] = {"rel_l2_error": float(np.linalg.norm(a - ref) / np.linalg.norm(ref)),
                         "steps": steps, "wall_s": wall, "dof_steps_per_s": n * n * 81 * steps / wall}
            ctx.close()
        e64 = res["fp64"]["rel_l2_error"]
        for name in ("mixed", "inverse"):
            res[name]["error_vs_fp64"] = res[name]["rel_l2_error"] / e64
            res[name]["matches"] = res[name]["rel_l2_error"] <= 1.05 * e64
        out["p%d" % p] = res
    return out


def forms_routes(steps=64):
    """The two states of the diagonalised route on the headline workload
    (64x64 elements, p=5, FP64): GDG_ROUTE_MODAL (modal coefficients from the
    first stage to the last; the timed stage kernel or the persistent step)
    against GDG_ROUTE_NODAL (nodal state; every stage transforms its input to
    the modified basis and its k back with n1 x n1 contractions per
    direction)."""
    import numpy as np
    import torch
    from paper_2105_01722_gb300 import gdg, inputs
    w = WORKLOAD
    X, Y = inputs.cartesian_nodes(w["n"], w["N"])
    U0, V0 = inputs.standing_mode_2d(X, Y)
    dt = w["cfl"] / (w["n"][0] * w["N"])
    out = {"workload": WORKLOAD_NAME, "steps_per_call": steps}
    res = {}
    for route, name in ((gdg.ROUTE_MODAL, "modal"), (gdg.ROUTE_NODAL, "nodal")):
        pb = gdg.make_problem(2, w["n"], w["N"], w["p"], flux=gdg.FLUX_UPWIND, c2=1.0, route=route)
        ctx = gdg.Context(pb)
        u = torch.tensor(U0.ravel(), device="cuda")
        v = torch.tensor(V0.ravel(), device="cuda")
        ctx.step(u, v, 0.0, dt, steps)
        ms = _timed_ms(lambda: ctx.step(u, v, 0.0, dt, steps))
        res[name] = torch.cat([u, v]).cpu().numpy()
        out[name] = {"dof_steps_per_s": dof() * steps / (ms / 1e3), "ms_per_step": ms / steps}
        ctx.close()
    out["nodal_vs_modal_rel_l2"] = float(np.linalg.norm(res["nodal"] - res["modal"]) / np.linalg.norm(res["modal"]))
    out["modal_over_nodal"] = out["modal"]["dof_steps_per_s"] / out["nodal"]["dof_steps_per_s"]
    return out


def executed_flops_per_element_stage_3d(n1):
    """FP64 flops the 3-D parity stage kernel executes per element (FMA = 2):
    fluxes 3 directions x n1^2 x (2 faces x 7 + 4 sums/differences), per
    modal entry 22 (lifts 5 + 7, diagonal solve 2, RK 8), traces one split
    dot per direction and field (12 per entry) + 12 n1^2 sums/differences."""
    return 66 * n1 ** 2 + 34 * n1 ** 3


def ocean_sound_speed(depth):
    """Depth-dependent sound speed of the ocean-channel application (Section 7.2),
    m/s, depth in m (positive down)."""
    import numpy as np
    return 1450.0 + 50.0 * (100.0 / (depth + 40.0) + np.tanh((depth - 300.0) / 50.0))


def forms_ocean(nx=500, ny=250, N=8, p=3, steps=16):
    """The ocean-channel workload of Section 7.2 (the paper shows it as pictures
    only): the channel [0, 4000] x [-2000, 0] m with the depth-dependent sound
    speed c(D), D = -y, and a point source sin(400 pi t) at x = 1004 m,
    D = 300 m (near the sound-channel axis; the centre of an element), u = 0
    on every side.  The paper's
    100 x 50 elements of 40 x 40 cells are taken as 500 x 250 elements of 8 x 8
    cells (the same 4000 x 2000 cells), p = 3; element inverses with face
    operators; dt = 0.2 h / max c."""
    import numpy as np
    import torch
    from paper_2105_01722_gb300 import gdg, inputs
    t_setup = time.perf_counter()
    X, Y = inputs.cartesian_nodes((nx, ny), N, lo=(0.0, -2000.0), hi=(4000.0, 0.0))
    C2 = ocean_sound_speed(-Y) ** 2
    pb = gdg.make_problem(2, (nx, ny), N, p, bc=(gdg.BC_DIRICHLET, gdg.BC_DIRICHLET), flux=gdg.FLUX_UPWIND,
                          coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2, solver=gdg.SOLVE_INVERSE)
    ctx = gdg.Context(pb)
    Hx, Hy = 4000.0 / nx, 2000.0 / ny
    xs, ys = 1004.0, -300.0
    ex, ey = int(xs // Hx), int((ys + 2000.0) // Hy)
    ctx.set_point_source(ey * nx + ex, xs / Hx - ex, (ys + 2000.0) / Hy - ey, 1.0, 400.0 * np.pi)
    setup_s = time.perf_counter() - t_setup
    u = torch.zeros(X.size, dtype=torch.float64, device="cuda")
    v = torch.zeros_like(u)
    h = min(Hx, Hy) / N
    dt = 0.2 * h / float(np.sqrt(C2.max()))
    ctx.step(u, v, 0.0, dt, 8)
    ms = _timed_ms(lambda: ctx.step(u, v, 8 * dt, dt, steps))
    finite = bool(torch.isfinite(u).all() and torch.isfinite(v).all())
    E = ctx.energy(u, v)
    ctx.close()
    dof = nx * ny * (N + 1) ** 2
    f64, _, byt = var_counts(N + 1, 0, 0, "inverse")
    stages = nx * ny * 4 * steps
    roof = alu_roofline(f64 * stages, 0.0, byt * stages, ms / 1e3, PROBE.get("fp64"))
    return {"roofline": roof,
            "workload": "ocean channel 4000 x 2000 m, c(depth), point source sin(400 pi t) at (1004 m, 300 m "
                        "deep), %d x %d elements of %d x %d cells, p=%d, element inverses" % (nx, ny, N, N, p),
            "dof": dof, "dof_steps_per_s": dof * steps / (ms / 1e3), "ms_per_step": ms / steps,
            "setup_s": setup_s, "dt": dt, "finite": finite, "energy_after": E}


def forms_three_d(n=32, N=8, p=5, steps=16):
    """3-D constant coefficient (Sections 2.1.2 and 3 for d = 3): n^3 elements
    of N^3 cells, upwind, Dirichlet, standing mode sin(pi x) sin(pi y) sin(pi z),
    dt = 0.1 h; DOF-steps/s and the FP64 rate of the whole step."""
    import numpy as np
    import torch
    from paper_2105_01722_gb300 import gdg, inputs
    pb = gdg.make_problem(3, (n, n, n), N, p, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                          bc=(gdg.BC_DIRICHLET,) * 3, flux=gdg.FLUX_UPWIND, c2=1.0)
    ctx = gdg.Context(pb)
    X, Y, Z = inputs.cartesian_nodes_3d((n, n, n), N)
    u = torch.tensor((np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)).ravel(), device="cuda")
    v = torch.zeros_like(u)
    dt = 0.1 / (n * N)
    E0 = ctx.energy(u, v)
    ctx.step(u, v, 0.0, dt, 4)
    ms = _timed_ms(lambda: ctx.step(u, v, 0.0, dt, steps))
    E1 = ctx.energy(u, v)
    ctx.close()
    dof = n ** 3 * (N + 1) ** 3
    f64 = executed_flops_per_element_stage_3d(N + 1) * n ** 3 * 4 * steps
    return {"workload": "3-D constant c^2, %d^3 elements of %d^3 cells, p=%d, upwind, Dirichlet" % (n, N, p),
            "dof": dof, "dof_steps_per_s": dof * steps / (ms / 1e3), "ms_per_step": ms / steps,
            "roofline": alu_roofline(f64, 0.0, 16.0 * dof * 4 * steps, ms / 1e3, PROBE.get("fp64")),
            "flops_note": "FP64 flops the 3-D parity stage kernel executes per element and stage "
                          "(66 n1^2 + 34 n1^3, FMA = 2) over the whole step's time (entry and exit "
                          "transforms included); bytes: one pass of the FP64 (u, v) state per stage",
            "energy_ratio_after_20_steps": E1 / E0}


def forms_batched(steps=8, nmin=16, nmax=128):
    """48 independent problems (seeds 20210501+i, n ~ U{nmin..nmax}, p in
    {3,5,7}, alternating constant / smooth random c^2): one batch (persistent
    launches, graph, tuned) against stepping each problem with its own
    gdg_step; the variable-coefficient problems by FP64 PCG, mixed PCG or
    element inverses."""
    import numpy as np
    import torch
    from paper_2105_01722_gb300 import gdg, inputs
    specs = inputs.batched_problems(48, nmin=nmin, nmax=nmax)
    cfl = {3: 0.2, 5: 0.15, 7: 0.12}
    dof = sum(sp["n"] ** 2 * 81 for sp in specs)
    out = {"problems": 48, "n_range": [nmin, nmax], "dof": dof}
    for prec, solver, name in ((gdg.FP64, gdg.SOLVE_PCG, "fp64"), (gdg.MIXED, gdg.SOLVE_PCG, "mixed"),
                               (gdg.FP64, gdg.SOLVE_INVERSE, "inverse")):
        built = []
        for sp in specs:
            n, p = sp["n"], sp["p"]
            X, Y = inputs.cartesian_nodes((n, n), 8)
            if sp["variable"]:
                C2 = inputs.smooth_random_c2(X, Y, sp["seed"])
                pb = gdg.make_problem(2, (n, n), 8, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                                      pcg_rtol=1e-10, pcg_maxit=100, precision=prec, solver=solver)
                cmax = float(np.sqrt(C2.max()))
            else:
                pb = gdg.make_problem(2, (n, n), 8, p, c2=1.0)
                cmax = 1.0
            built.append((pb, inputs.gaussian_pulse(X, Y, sp["x0"], sp["y0"], 0.05).ravel(), cfl[p] / (n * 8) / cmax))
        us = [torch.tensor(b[1], device="cuda") for b in built]
        vs = [torch.zeros_like(u) for u in us]
        dts = [b[2] for b in built]
        batch = gdg.Batch([b[0] for b in built])
        batch.step(us, vs, dts, 4)
        for i, sp in enumerate(specs):     # reset the PCG counters
            if sp["variable"] and name != "inverse":
                batch.stats(i)
        ms = _timed_ms(lambda: batch.step(us, vs, dts, steps))
        f64 = f32 = byt = 0.0
        for i, sp in enumerate(specs):
            stages = sp["n"] ** 2 * 4 * steps
            if sp["variable"]:
                su, sv = batch.stats(i) if name != "inverse" else ({"mean_iters": 0, "mean_sweeps": 0},) * 2
                a, b_, c = var_counts(9, su["mean_iters"], sv["mean_iters"], name, su["mean_sweeps"],
                                      sv["mean_sweeps"])
            else:
                a, b_, c = ALG_FLOPS_PER_DOF_STAGE * 81, 0.0, 16.0 * 81
            f64 += a * stages
            f32 += b_ * stages
            byt += c * stages
        out["batched_" + name] = {"dof_steps_per_s": dof * steps / (ms / 1e3), "ms_per_step": ms / steps,
                                  "tuning": batch.tuning(),
                                  "roofline": alu_roofline(f64, f32, byt, ms / 1e3, PROBE.get("fp64"))}
        batch.close()
        ctxs = [gdg.Context(b[0]) for b in built]
        for c, u, v, d in zip(ctxs, us, vs, dts):
            c.step(u, v, 0.0, d, 4)
        ms = _timed_ms(lambda: [c.step(u, v, 0.0, d, steps) for c, u, v, d in zip(ctxs, us, vs, dts)])
        out["sequential_" + name] = {"dof_steps_per_s": dof * steps / (ms / 1e3), "ms_per_step": ms / steps}
        for c in ctxs:
            c.close()
        del us, vs
        torch.cuda.empty_cache()
    return out


def forms_learned(rows=20000, epochs=30, steps=16):
    """Learned u_t initial guess: 20k rows generated by the method on 128 x 128
    meshes with random smooth c^2 in [1/2, 2] (p = 5, 8x8 cells; 2,500 random
    elements of one snapshot per c^2 field, so eight fields), trained with the library's kernels; u_t
    PCG iterations and DOF-steps/s on an unseen 128 x 128 mesh (the same
    element size: the constraint row of the u_t system scales with the element
    area) at rtol 1e-10, with and without the network (FP64 and mixed PCG)."""
    import time
    import torch
    from paper_2105_01722_gb300 import gdg, inputs, learned
    t0 = time.time()
    X, T = learned.generate(rows, n=128, seed0=2000, snapshots=1, substeps=12, per_snapshot=2500)
    t1 = time.time()
    ntr = int(0.9 * rows)
    net, hist = learned.train(X[:ntr], T[:ntr], epochs=epochs, batch=256, lr=2e-3)
    t2 = time.time()
    out = {"rows": rows, "train_rows": ntr, "epochs": epochs, "generate_s": t1 - t0, "train_s": t2 - t1,
           "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
           "test_mean_rel_err": learned.relative_error(net, X[ntr:], T[ntr:])}
    for prec, name in ((gdg.FP64, "fp64"), (gdg.MIXED, "mixed")):
        pb, Xn, Yn, dt = learned.problem(128, 8, 5, seed=31337, rtol=1e-10, precision=prec)
        for attach in (False, True):
            ctx = gdg.Context(pb)
            if attach:
                ctx.mlp_attach(net)
            u = torch.tensor(inputs.gaussian_pulse(Xn, Yn, 0.5, 0.5, 0.05).ravel(), device="cuda")
            v = torch.zeros_like(u)
            ctx.step(u, v, 0.0, dt, 8)
            ctx.step_stats()
            ms = _timed_ms(lambda: ctx.step(u, v, 0.0, dt, steps))
            su, sv = ctx.step_stats()
            f64, f32, byt = var_counts(9, su["mean_iters"], sv["mean_iters"], name, su["mean_sweeps"],
                                       sv["mean_sweeps"])
            stages = 128 * 128 * 4 * steps
            if attach:   # one forward pass per u_t solve (FP32), plus the guess's FP64 residual product
                f32 += 2.0 * (162 * 64 + 64 * 64 + 64 * 81)
                f64 += 2.0 * 81 * 81
            out[name + ("_learned" if attach else "_plain")] = {
                "roofline": alu_roofline(f64 * stages, f32 * stages, byt * stages, ms / 1e3, PROBE.get("fp64")),
                "dof_steps_per_s": 128 * 128 * 81 * steps / (ms / 1e3), "ms_per_step": ms / steps,
                "pcg_u_mean_iters": su["mean_iters"], "pcg_u_max_iters": su["max_iters"],
                "guess_fallbacks": su["fell_back"], "guessed": su["guessed"]}
            ctx.close()
    return out


def run_gdg(args):
    import numpy as np
    import torch
    from paper_2105_01722_gb300 import gdg, inputs, shard

    rank, world, local = _env_rank()
    if world > 1:
        import torch.distributed as dist
        # one GPU per rank over NCCL; with fewer GPUs than ranks (a functional
        # check of the banded path on one GPU) the ranks share GPUs and
        # exchange through gloo, with host copies
        ngpu = torch.cuda.device_count()
        local = local % ngpu
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if ngpu >= world else "gloo")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    w = WORKLOAD
    R = args.rk_steps
    h = 1.0 / (w["n"][0] * w["N"])
    dt = w["cfl"] * h
    if world == 1:
        pb = gdg.make_problem(2, w["n"], w["N"], w["p"], flux=gdg.FLUX_UPWIND, c2=1.0)
        ctx = gdg.Context(pb)
        X, Y = inputs.cartesian_nodes(w["n"], w["N"])
    else:
        # one mesh over the GPUs: nx x (ny * world) elements on [0,1] x [0,world],
        # a band of ny rows (the single-GPU workload's size) per rank, the
        # face traces of the band edges exchanged (NCCL) before every stage
        gn = (w["n"][0], w["n"][1] * world)
        pb, (r0, r1) = shard.band_problem(gdg.make_problem, rank, world, 2, gn, w["N"], w["p"],
                                          hi=(1.0, float(world)), flux=gdg.FLUX_UPWIND, c2=1.0)
        ctx = gdg.Context(pb)
        hn = ctx.halo_len()
        mk = lambda on: torch.zeros(hn, dtype=torch.float64, device=dev) if on else None
        halo_bufs = (mk(rank > 0), mk(rank < world - 1), mk(rank > 0), mk(rank < world - 1))
        ctx.set_halo(*halo_bufs, shard.HaloExchange(rank, world, *halo_bufs))
        X, Y = inputs.cartesian_nodes(w["n"], w["N"], lo=(0.0, float(r0) / w["n"][1]),
                                      hi=(1.0, float(r1) / w["n"][1]))
    U0, V0 = inputs.standing_mode_2d(X, Y)
    u = torch.tensor(U0.ravel(), device=dev)
    v = torch.tensor(V0.ravel(), device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        flush.fill_(1.0)
        ctx.step(u, v, 0.0, dt, R)
    torch.cuda.synchronize()
    PROBE["fp64"] = fp64_probe_tflops()

    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))                      # evict the state from L2 between timed steps
        evs[k][0].record(stream)
        ctx.step(u, v, 0.0, dt, R)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall1 = time.perf_counter()
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = shard.max_over_ranks(sum(ms))
    ms_per_step = total_ms / args.steps
    value = world * dof() * R * args.steps / (total_ms / 1e3)

    stage_variant = ctx.stage_variant()
    # kernel-level pass: events around every launch (no graph), same work
    ctx.profile(True)
    for k in range(max(2, min(args.steps, 5))):
        flush.fill_(float(k))
        ctx.step(u, v, 0.0, dt, R)
    prof = ctx.profile_read()
    ctx.profile(False)
    st_n, st_ms = prof.get("stage", (1, float("nan")))
    # the persistent step (variant 3) is one launch for all 4R stages of a call
    stages_per_launch = 4 * R if stage_variant == 3 else 1
    stage_ms_isolated = st_ms / (st_n * stages_per_launch)
    # stage kernel duration inside the timed (graph) region: the step's time
    # less its entry/exit launches (transform, traces; timed in the pass
    # above), over its 4R stage launches; includes the gaps between launches
    n_steps_prof = max(2, min(args.steps, 5))
    other_ms = sum(t for k, (n, t) in prof.items() if k != "stage") / n_steps_prof
    stage_ms = (ms_per_step - other_ms) / (4 * R)
    if world > 1:
        # the per-stage time of a banded mesh includes the halo exchanges; the
        # stage kernel's own duration is the one measured around each launch
        step_stage_ms, stage_ms = stage_ms, stage_ms_isolated
    achieved = ALG_FLOPS_PER_DOF_STAGE * dof() / (stage_ms / 1e3) / 1e12
    achieved_x = executed_flops_per_stage_launch() / (stage_ms / 1e3) / 1e12

    # end to end through the C ABI with host buffers (pinned), copies timed
    hu = torch.tensor(U0.ravel()).pin_memory()
    hv = torch.tensor(V0.ravel()).pin_memory()
    ctx.step_host(hu, hv, 0.0, dt, R)
    e2e_t = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.step_host(hu, hv, 0.0, dt, R)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = shard.max_over_ranks(sum(e2e_t))
    e2e_val = world * dof() * R * args.steps / e2e_s

    # accuracy of the FP64 form at T = 1: M-norm distance to the GD
    # interpolant of the exact solution, evaluated by the library's energy
    # kernel (single mesh; the banded multi-GPU mesh is not a unit square)
    nT = int(round(w["T"] / dt))
    l2 = None
    if world == 1:
        ua = torch.tensor(U0.ravel(), device=dev)
        va = torch.tensor(V0.ravel(), device=dev)
        ctx.step(ua, va, 0.0, dt, nT)
        ue, _ = inputs.standing_mode_2d(X, Y, nT * dt)
        diff = ua - torch.tensor(ue.ravel(), device=dev)
        l2 = float(np.sqrt(2.0 * ctx.energy(torch.zeros_like(diff), diff)))

    line = None
    if rank == 0:
        cpu = cpu_baseline() if (world == 1 and not args.no_cpu_baseline) else None
        forms = {}
        if not args.no_forms and world == 1:
            for key, fn in (("variable_mapped_128", forms_variable), ("batched_48", forms_batched),
                            ("batched_48_small", lambda: forms_batched(nmin=8, nmax=24)),
                            ("routes_64", forms_routes),
                            ("learned_guess", forms_learned), ("three_d_32", forms_three_d),
                            ("ocean_channel", forms_ocean)):
                try:
                    forms[key] = fn()
                except Exception as exc:    # report, do not lose the headline line
                    forms[key] = {"error": repr(exc)}
        if args.equal_error and world == 1:
            try:
                forms["equal_error_mapped_128"] = forms_equal_error()
            except Exception as exc:
                forms["equal_error_mapped_128"] = {"error": repr(exc)}
        line = {
            "metric": "DOF-steps/s", "value": value, "unit": "DOF-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "elements": list(w["n"]), "N": w["N"], "p": w["p"],
                       "dof": dof(), "rk4_steps_per_step": R, "dt": dt,
                       "form": "FP64 modal (modified basis)",
                       "parallelism": ("one GPU" if world == 1 else
                                       "one %dx%d mesh, a %dx%d band of element rows per GPU, face traces "
                                       "of the band edges exchanged (NCCL point to point) before every RK stage"
                                       % (w["n"][0], w["n"][1] * world, w["n"][0], w["n"][1])),
                       "l2": "flushed between timed steps (512 MB write; state is 5.3 MB)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                         "peak_probe": PROBE.get("fp64"),
                         "frac_of_probe": achieved / PROBE["fp64"] if PROBE.get("fp64") else None,
                         "flops_per_dof_stage": ALG_FLOPS_PER_DOF_STAGE,
                         "traffic": STAGE_TRAFFIC_BYTES.get(stage_variant),
                         "kernel": {1: "k_stage2h", 2: "k_stage2f", 3: "k_step2r"}.get(stage_variant, "k_stage2p")
                                   + " (fused RK4 stage, modal route; variant chosen by timing)",
                         "avg_launch_us": stage_ms * 1e3,
                         "avg_launch_us_isolated": stage_ms_isolated * 1e3,
                         "duration_source": ("timed region (CUDA events on the launching stream) less the step's "
                                             "entry/exit launches, over 4R stage launches; _isolated: events "
                                             "around each launch outside the graph") if stage_variant != 3 else
                                            ("timed region (CUDA events on the launching stream) less the step's "
                                             "entry/exit launches, over the 4R stages of its one persistent "
                                             "launch (per-stage figures); _isolated: events around that launch "
                                             "in a separate pass, over its 4R stages"),
                         "flops_per_stage": ALG_FLOPS_PER_DOF_STAGE * dof(),
                         "flops_per_stage_executed": executed_flops_per_stage_launch(),
                         "achieved_executed": achieved_x,
                         "frac_executed": achieved_x / FP64_PEAK_TFLOPS,
                         "fp64_pipe_frac": (STEP2R_FP64_INST_PER_ELEMENT_STAGE * w["n"][0] * w["n"][1]
                                            / (stage_ms / 1e3) / (152 * 2 * 2.070e9 * (clocks["sm_mhz"] or 2070.0)
                                                                   / 2070.0))
                                           if stage_variant == 3 else None,
                         "flops_note": "achieved: 40 algorithmic FP64 flops per DOF and stage (the modal "
                                       "route's per-DOF count) x DOF, per stage of the timed region; "
                                       "_executed: the flops the parity stage body performs (28.4 per DOF, "
                                       "FMA = 2; the r -> 1-r symmetry halves the lifts and trace dots); "
                                       "fp64_pipe_frac: the persistent step's FP64 instructions per stage "
                                       "(ncu count) over the stage time at 2 lanes per SM and clock, the "
                                       "figure ncu's FP64 pipe utilisation measures",
                         "peak_source": "FP64 derived from unit counts and the maximum SM clock: "
                                        "152 SM x 2070 MHz x 4 flop/clk; peak_probe: gdg_probe_fp64 "
                                        "(independent FMA chains) timed in this process"},
            "kernels": {k: {"launches": n, "ms": t} for k, (n, t) in prof.items()},
            "gpu_launches": ((4 * R if stage_variant != 3 else 1) * args.steps + 3 * args.steps
                             + (2 * (4 * R) * args.steps if world > 1 else 0)),
            "e2e": {"value": e2e_val, "unit": "DOF-steps/s", "h2d_bytes_per_step": 2 * dof() * 8,
                    "d2h_bytes_per_step": 2 * dof() * 8},
            "clocks": clocks,
            "accuracy": {"T": nT * dt, "l2_error_vs_interpolant": l2} if l2 is not None else None,
            "wall_s": wall1 - wall0,
            "cpu_baseline": cpu,
            "forms": forms,
        }
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gdg", "reference"], default="gdg")
    ap.add_argument("--rk-steps", type=int, default=256,
                    help="RK4 steps per benchmark step (one gdg_step call)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the extra forms (variable/mapped, batched, learned) after the headline")
    ap.add_argument("--equal-error", action="store_true",
                    help="also run the variable-coefficient forms to T = 0.25 against a 2x refined FP64 "
                         "reference (several minutes)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gdg(args)


if __name__ == "__main__":
    sys.exit(main())
