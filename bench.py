"""Benchmark of the matrix-free evaporation hot path on GB300.

Workload: the 64^3-cell four-sphere case (Q2 velocity, 6.44 M velocity DoFs, 275 k level-set DoFs, density ratio
1e3, random-Fourier velocity).  One step = one pass of the whole hot path:
  set_fields (material-law table + variant-2 transport velocity with closest-point projection)
  -> 100 back-to-back FP64 momentum applies with the divergence row (the 64^3 configuration's "100 repeated applies")
  -> 100 FP32 momentum applies -> 100 level-set advection applies -> reinitialization operator and right-hand side
  -> adjoint apply (all four gradients) -> mixed-precision GMRES solve to 1e-10.
value = FP64 momentum operator-apply GDoF/s (velocity DoFs x applies / time of the 100 back-to-back applies, CUDA
events, max over ranks); the FP32 apply, the adjoint and the level-set apply are first-class keys beside it, each
with its roofline fractions; the whole-step rate is an extra.  Inputs (~0.5 GB touched per apply) exceed the 129 MB
L2.  Denominators: HBM from MEASURED_PEAKS.json, FP64 and FP32 from FMA probes run in this process.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs an independent replica (weak scaling, no collective on the data path); rank 0 prints
one JSON line.  --impl reference times the CPU oracle (assembled CSR operator) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD = "spheres64"
METRIC = "operator-apply GDoF/s and %HBM roofline (FP64 vs FP32-inner) + adjoint GDoF/s"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# DRAM bytes (read + write) per launch of a kernel from an ncu capture of this bench, valid only while the kernel's
# sources are unchanged: {(kernel, workload): (bytes, sha256 prefix of the sources)}.
MEASURED_TRAFFIC = {
    ("k_momentum32", "spheres64"): (430_798_208, "41e4f85604ffe5de"),
    ("k_momentum_df", "spheres64"): (1_227_021_952, "cfa79905aa5f0c2d"),
}
TRAFFIC_SOURCES = {"k_momentum32": ("paper_2401_07805_gb300/csrc/momentum32.cu",
                                    "paper_2401_07805_gb300/csrc/basis_ct.cuh",
                                    "paper_2401_07805_gb300/csrc/evap_internal.cuh"),
                   "k_momentum_df": ("paper_2401_07805_gb300/csrc/momentum_df.cu",
                                     "paper_2401_07805_gb300/csrc/async_copy.cuh",
                                     "paper_2401_07805_gb300/csrc/dfloat.cuh",
                                     "paper_2401_07805_gb300/csrc/physics.cuh",
                                     "paper_2401_07805_gb300/csrc/evap_internal.cuh")}


def sources_digest(kernel):
    """sha256 prefix of what the kernel is compiled from: its .cu, the basis tables, and the device-side part of
    evap_internal.cuh (everything before the host-side mesh struct, which does not enter the kernel).  Line comments
    and blank lines are left out, so that a comment edit keeps a traffic record valid."""
    import hashlib
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES[kernel]:
        data = open(os.path.join(ROOT, rel), "rb").read()
        if rel.endswith("evap_internal.cuh"):
            data = data.split(b"struct evap_mesh {")[0]
        for line in data.splitlines():
            code = line.split(b"//")[0].rstrip()
            if code:
                h.update(code + b"\n")
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload):
    rec = MEASURED_TRAFFIC.get((kernel, workload))
    if rec is None or rec[1] != sources_digest(kernel):
        return None
    return rec[0]


# Nominal rates, quoted beside the probes' measurements: FP64 1.25 TFLOP/s (the profiling recipe's table); FP32
# 152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s (the recipe's unit counts and maximum SM clock).
FP64_NOMINAL_TFLOPS = 1.25
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Instructions of one double-float multiply-add (df_fma of dfloat.cuh: TwoProduct 2, cross terms 2, TwoSum 6, error
# sum 2), each issued at the FP32 FMA rate: the double-float kernel's peak in FP64-equivalent flops is the measured
# FP32 rate / DF_FMA_INSTR (an FMA counts 2 flops on both sides).
DF_FMA_INSTR = 12
REPS = 100  # back-to-back applies per operator and step (the 64^3 configuration's 100 repeated applies)


def algorithmic_counts(n: int, p: int):
    """Algorithmic bytes and flops per apply (minimal traffic: every nodal vector read/written once; sum
    factorization flop count of the kernels' arithmetic)."""
    M = p * n + 1
    Nu, Np, nc = M ** 3, (n + 1) ** 3, n ** 3
    Q = p + 1
    nq = Q ** 3
    sweep = Q * nq                        # multiply-adds of one 1D sweep over a cell
    # momentum apply with cached quadrature-point coefficients, per cell and velocity component: 3 value sweeps +
    # 3 collocation-gradient sweeps (interpolation), 3 transposed gradient sweeps + 3 transposed value sweeps
    # (testing); ~50 multiply-adds per point for the fluxes; an FMA counts 2 flops
    interp = 6 * sweep
    mom_flop = 2 * nc * (3 * interp + 3 * interp + 50 * nq)
    # adjoint: interpolation of x and w (6 components; the u0 terms come from the quadrature-point cache), testing
    # of g_x and g_u0 (6 components), ~80 multiply-adds per point for the adjoint fluxes (the material-law
    # derivatives of the interface-zone points are not counted: a lower bound)
    adj_flop = 2 * nc * (6 * interp + 6 * interp + 80 * nq)
    # FP32 line kernel per cell (Q^2 line threads): z-sweeps (S, D on 3 components), y-sweeps (S, D on S-output,
    # S on D-output), x-lines (4 outputs per point and component, ~50 multiply-adds of fluxes per point, x-line
    # testing 4 per point, node and component), backward y- (3 per pair) and z-sweeps (2 per pair) of 3 components
    L2 = Q * Q
    mom32_fma = L2 * (3 * Q * 2 * Q) + L2 * (3 * Q * 3 * Q) + L2 * Q * (3 * 4 * Q + 50 + 3 * 4 * Q) \
        + L2 * (3 * Q * 3 * Q) + L2 * (3 * Q * 2 * Q)
    mom32_flop = 2 * nc * mom32_fma
    return dict(
        Nu=Nu, Np=Np, ncell=nc,
        # algorithmic bytes of the method (every nodal vector read or written once, no quadrature data stored):
        # FP64 apply: x, u0 and y [3 N_u] plus phi and mdot [N_phi]; FP32 apply: x, u0, y in FP32, phi, mdot in FP64
        mom64_alg_bytes=8 * (9 * Nu + 2 * Np),
        mom32_alg_bytes=4 * 9 * Nu + 8 * 2 * Np,
        # bytes the kernels stream: FP64 apply x in, y and y_p out, the 19 cached FP64 coefficients per quadrature
        # point; FP32 apply x in, y out, 12 FP32 u0 coefficients per quadrature point, cell code and table index
        mom64_bytes=8 * (3 * Nu * 2 + Np) + 8 * nc * 19 * nq,
        mom32_bytes=4 * (3 * Nu * 2) + 4 * nc * 12 * nq + 5 * nc,
        mom_flop=mom_flop,
        mom32_flop=mom32_flop,
        ls_adv_bytes=8 * (Np + Np + 3 * Np),
        ls_reinit_bytes=8 * 3 * Np,
        adj_bytes=8 * (3 * Nu * 5 + 5 * Np),            # x, w, u0 in; g_x, g_u0 out; phi, mdot, w_p in; g_phi, g_mdot out
        adj_flop=adj_flop,
    )


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_info():
    cores = os.cpu_count()
    try:
        model = [l for l in open("/proc/cpuinfo") if l.lower().startswith(("model name", "cpu part"))][0].split(":")[1]
        model = model.strip()
    except Exception:
        model = "unknown"
    return cores, model


def _oracle_block(args):
    """One host core's share of the CPU baseline (runs in a spawned process): the oracle's assembled FP64 momentum
    operator with its divergence rows on an nb^3-cell sub-block of the workload (no Dirichlet faces; the workload's
    fields restricted to the block), CSR assembly timed once, then `reps` applies (y = A x, y_p = B x - g) each
    timed, after all workers reached the barrier.  Returns (assembly s, list of apply s, velocity DoFs)."""
    name, nb, corner, reps, barrier = args
    sys.path.insert(0, ROOT)
    import workloads as wlmod
    from oracle import fe, momentum
    wl = wlmod.make_workload(name)
    n, p = wl.n, wl.p
    M, m1, mb, m1b = p * n + 1, n + 1, p * nb + 1, nb + 1
    cx, cy, cz = corner
    iu = np.arange(mb)
    K, J, I = np.meshgrid(p * cz + iu, p * cy + iu, p * cx + iu, indexing="ij")
    gu = (I + M * (J + M * K)).ravel()
    i1 = np.arange(m1b)
    K1, J1, I1 = np.meshgrid(cz + i1, cy + i1, cx + i1, indexing="ij")
    g1 = (I1 + m1 * (J1 + m1 * K1)).ravel()
    sub = lambda v: np.concatenate([v.reshape(3, -1)[c][gu] for c in range(3)])
    prm = dict(wl.params, dirichlet_faces=0)
    pb = momentum.Problem(mesh=fe.Mesh(nb, p, nb * wl.L / n), params=prm, phi=wl.phi[g1].copy(),
                          u0=sub(wl.u0), mdot=wl.mdot[g1].copy())
    x = sub(wl.x)
    t0 = time.perf_counter()
    A = momentum.assemble(pb)
    B, g = momentum.divergence(pb)
    t_asm = time.perf_counter() - t0
    barrier.wait()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        y = A @ x
        yp = B @ x - g
        ts.append(time.perf_counter() - t0)
    del y, yp
    return t_asm, ts, 3 * pb.mesh.n_u


def oracle_baseline(name: str = "spheres64", nb: int = 12, reps: int = 10, workers: int | None = None):
    """The CPU oracle as it stands on all host cores: one spawned process per core, each assembling the oracle's
    CSR momentum operator (full Gauss quadrature) on its own nb^3-cell sub-block of the workload and timing `reps`
    applies with the divergence rows; the aggregate rate is the sum over workers of block DoFs / median apply time
    (the applies of all workers run at the same time, after a barrier).  Spawned, so no process inherits a GPU
    context."""
    import multiprocessing as mp
    workers = workers or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    wl = workloads.make_workload(name)
    per = max(1, wl.n // nb)
    corners = [((k % per) * nb, ((k // per) % per) * nb, ((k // (per * per)) % per) * nb) for k in range(workers)]
    # one thread per worker process (the spawned interpreters read these at import): cores = workers
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({k: "1" for k in saved})
    try:
        with ctx.Manager() as mgr:
            barrier = mgr.Barrier(workers)
            with ctx.Pool(workers) as pool:
                res = pool.map(_oracle_block, [(name, nb, c, reps, barrier) for c in corners])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    rate = sum(dofs / float(np.median(ts)) for _, ts, dofs in res)
    return dict(value=rate / 1e9, unit="GDoF/s", cores=workers, kind="oracle",
                assembly_s=float(np.median([r[0] for r in res])),
                apply_ms_median=1e3 * float(np.median([np.median(r[1]) for r in res])),
                sample=f"the oracle's assembled FP64 momentum operator with divergence rows (CSR, full Gauss "
                       f"quadrature) on {workers} disjoint {nb}^3-cell sub-blocks of the {name} workload, one process "
                       f"per host core; median of {reps} applies after CSR assembly (assembly reported separately)")


def solve_comparison(evap, torch, dev):
    """96^3 slab (21.6 M velocity DoFs): FP64 GMRES(16) + Jacobi vs FP32-inner GMRES(16) with FP64 iterative
    refinement, both to ||f - A x|| <= 1e-10 ||f||; error of each against an FP64 solve driven to 1e-13."""
    wl = workloads.make_workload("slab96")
    op = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    op.set_fields(cu(wl.phi), cu(wl.u0), cu(wl.mdot))
    f = cu(wl.x)
    ref, info_ref = op.solve(f, mixed=False, rtol=1e-13, max_iter=5000)
    out = {"workload": "slab96: 96^3 cells, Q2 (21.6 M DoFs), slab at z = 0.5, ratio 1e3, Fourier u0 (seed 3)",
           "reference": dict(rtol=1e-13, iters=info_ref["iters"], relres=info_ref["relres"])}
    stream = torch.cuda.current_stream()
    for name, mixed in (("fp64", False), ("mixed", True)):
        op.solve(f, mixed=mixed, rtol=1e-10, max_iter=5000)  # warm-up (workspace allocation)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        x, info = op.solve(f, mixed=mixed, rtol=1e-10, max_iter=5000)
        e1.record(stream)
        torch.cuda.synchronize()
        err = float((x - ref).norm() / ref.norm())
        out[name] = dict(ms=e0.elapsed_time(e1), iters=info["iters"], relres=info["relres"], err_vs_fp64_ref=err)
    out["speedup_mixed_over_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    op.close()
    return out


def job_time_ms(torch, dist, ms: float, device, world: int) -> float:
    """The job's time: the largest of the ranks' times (every rank receives it); the rank's own time at N = 1."""
    if world <= 1:
        return ms
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def aggregate_gdofs(world: int, dofs_per_rank: int, ms: float) -> float:
    """Whole-job throughput: all ranks' DoFs over the job's time (independent replicas, weak scaling)."""
    return world * dofs_per_rank / (ms * 1e-3) / 1e9


def back_to_back(torch, fn, reps, warm):
    """Mean time (ms) of `reps` back-to-back calls after `warm` untimed ones, CUDA events on the current stream."""
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def operator_applies(evap, torch, dev, op, d, counts, hbm):
    """Extras beside the step: the closest-point transport pass alone on the 64^3 workload (20 repeats: band nodes/s,
    point evaluations, flags), the applies and the adjoint in the deterministic mode (8 colour passes instead of
    atomic adds: 20 applies after 3 each), and the adjoint on the 48^3 sphere (2.74 M DoFs, 20 applies after 3)."""
    out = {}
    x, x32 = d["x"], d["x32"]
    y, yp = torch.empty_like(x), torch.empty(op.n_p, dtype=torch.float64, device=dev)
    det = {}
    for mode in (False, True):
        op.set_deterministic(mode)
        t64 = back_to_back(torch, lambda: op.apply_momentum(x, prec=64, with_divergence=True, out=y, out_p=yp), 20, 3)
        t32 = back_to_back(torch, lambda: op.apply_momentum(x32, prec=32), 20, 3)
        ta = back_to_back(torch, lambda: op.apply_adjoint(d["w"], x, d["wp"]), 20, 3)
        det["deterministic" if mode else "atomic"] = dict(momentum_fp64_ms=t64, momentum_fp32_ms=t32, adjoint_ms=ta)
    op.set_deterministic(False)
    out["accumulation"] = det
    t = back_to_back(torch, op.update_transport_velocity, 20, 2)
    st = op.transport_stats()
    out["transport_velocity"] = dict(ms=t, band_nodes=st["band_nodes"], band_nodes_per_s=st["band_nodes"] / t * 1e3,
                                     evaluations_per_node=st["evaluations"] / max(st["band_nodes"], 1),
                                     flagged=st["flagged"])
    wl = workloads.make_workload("sphere48")
    op4 = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    op4.set_fields(cu(wl.phi), cu(wl.u0), cu(wl.mdot))
    w, xx, wp = cu(wl.extra["w"]), cu(wl.x), cu(wl.extra["w_p"])
    t = back_to_back(torch, lambda: op4.apply_adjoint(w, xx, wp), 20, 3)
    c4 = algorithmic_counts(wl.n, wl.p)
    out["adjoint_sphere48"] = dict(ms=t, gdofs=3 * op4.n_u / t / 1e6, fp64_tflops=c4["adj_flop"] / t / 1e9)
    op4.close()
    return out


def geometry_subsolver(torch, op, phi):
    """Level-set sub-solver on the current fields (64^3 four spheres): projected normal (3 CG solves), curvature
    (1 CG solve), the surface-tension force from them, 5 reinitialization steps with the projected normal frozen,
    and the advection fixed point (3 passes of transport velocity + Crank-Nicolson GMRES solve); each timed with
    CUDA events after one untimed run."""
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    t_n, (n, info_n) = timed(op.projected_normal)
    t_k, (kappa, info_k) = timed(lambda: op.curvature(n))
    t_s, _ = timed(lambda: op.surface_tension(n, kappa, 0.0728))
    op.set_levelset_normal(n)
    t_r, (psi, info_r) = timed(lambda: op.reinitialize(phi, 5))
    op.set_levelset_normal(None)
    t_a, (_, info_a) = timed(lambda: op.advect_levelset(3))
    op.update_transport_velocity()  # the advection leaves the last pass's u_Gamma on the mesh
    return dict(projected_normal=dict(ms=t_n, cg_iters=info_n["iters"], relres=info_n["relres"]),
                curvature=dict(ms=t_k, cg_iters=info_k["iters"], relres=info_k["relres"]),
                surface_tension_force=dict(ms=t_s, velocity_dofs=3 * op.n_u),
                reinit_5_steps=dict(ms=t_r, cg_iters=info_r["iters"], last_change=info_r["last_change"]),
                advection_3_passes=dict(ms=t_a, gmres_applies=info_a["lin_iters"],
                                        last_change=info_a["last_change"]),
                level_set_dofs=op.n_phi)


def saddle_case(evap, torch, dev):
    """Velocity-pressure system on the 64^3 four-sphere workload with the top face open (walls on the other five):
    the FP64 saddle-point apply (20 back-to-back after 3) and flexible-GMRES solves of [A, -B^T; B, 0] [x; p] =
    [f; g] from zero, f the workload's random vector (Dirichlet entries 0), g from the evaporation, to the paper's
    relative tolerance 1e-4 of the Navier-Stokes solve and to 1e-8; each solve timed with CUDA events."""
    wl = workloads.make_workload(WORKLOAD, dirichlet_faces=0x1F)
    op = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    op.set_fields(cu(wl.phi), cu(wl.u0), cu(wl.mdot))
    stream = torch.cuda.current_stream()
    nu3 = 3 * op.n_u
    f = wl.x.copy()
    m = workloads.node_coords(wl.n, wl.p)
    M = wl.p * wl.n + 1
    idx = np.round(m * (M - 1)).astype(np.int64)
    cons = np.zeros(len(m), dtype=bool)
    for ax in range(3):
        cons |= idx[:, ax] == 0
        if ax < 2:
            cons |= idx[:, ax] == M - 1
    f[np.tile(cons, 3)] = 0.0
    f = cu(f)
    pr = cu(np.random.default_rng(3).uniform(-1, 1, op.n_phi))
    t_apply = back_to_back(torch, lambda: op.apply_saddle(f, pr), 20, 3)
    res = dict(workload=f"{WORKLOAD} with the face z = 1 open: {nu3 / 1e6:.2f} M velocity + {op.n_phi / 1e3:.0f} k "
                        "pressure DoFs", apply_ms=t_apply, apply_gdofs=(nu3 + op.n_phi) / t_apply / 1e6)
    for rtol in (1e-4, 1e-8):
        op.solve_saddle(f, rtol=rtol)  # warm-up (workspace allocation)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, info = op.solve_saddle(f, rtol=rtol)
        e1.record(stream)
        torch.cuda.synchronize()
        res[f"solve_rtol_{rtol:g}"] = dict(ms=e0.elapsed_time(e1), applies=info["iters"], relres=info["relres"],
                                           converged=info["converged"])
    op.close()
    # coupled time steps (BDF1, one Picard linearization) on the same fields
    prm = dict(wl.params, newton=0)
    prm["c_mass"] = 1.0 / prm["dt"]
    op = evap.Operator(wl.n, wl.p, wl.L, prm)
    phi, u = cu(wl.phi), cu(np.where(np.tile(cons, 3), 0.0, wl.u0))
    pr = torch.zeros(op.n_phi, dtype=torch.float64, device=dev)
    md = cu(wl.mdot)
    phi, u, pr, _ = op.time_step(phi, u, pr, md)  # warm-up (workspaces)
    torch.cuda.synchronize()
    ms, its = [], []
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        phi, u, pr, info = op.time_step(phi, u, pr, md)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        its.append(info["ns_iters"])
    res["time_steps"] = dict(ms=ms, ns_applies=its, ns_rtol=1e-8, fp_iters=2, reinit_steps=2,
                             note="consecutive steps after one untimed step: BDF1 Picard velocity-pressure solve + "
                                  "advection fixed point + projected normal + reinitialization")
    op.close()
    return res


def subdivided_case(evap, torch, dev):
    """The four-sphere workload with the level set on the twice-subdivided mesh (n_sub = 2: 64^3 velocity cells, Q2,
    6.44 M velocity DoFs; 129^3 = 2.15 M level-set DoFs): set_fields (with the closest-point transport velocity on
    the fine lattice), the FP64-accurate momentum apply with its divergence row, the level-set advection apply, the
    adjoint (20 back-to-back calls after 3 each), and one projected normal and curvature."""
    wl = workloads.make_workload(WORKLOAD, n_sub=2)
    op = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    phi, u0, md, x = cu(wl.phi), cu(wl.u0), cu(wl.mdot), cu(wl.x)
    rng = np.random.default_rng(7)
    w, wp = cu(rng.uniform(-1, 1, wl.x.shape)), cu(rng.uniform(-1, 1, op.n_p))
    ts = back_to_back(torch, lambda: op.set_fields(phi, u0, md), 3, 1)
    y, yp = torch.empty_like(x), torch.empty(op.n_p, dtype=torch.float64, device=dev)
    t64 = back_to_back(torch, lambda: op.apply_momentum(x, prec=64, with_divergence=True, out=y, out_p=yp), 20, 3)
    t_ls = back_to_back(torch, lambda: op.apply_levelset(phi, mode="advect"), 20, 3)
    t_adj = back_to_back(torch, lambda: op.apply_adjoint(w, x, wp), 20, 3)
    t_n = back_to_back(torch, op.projected_normal, 2, 1)
    nu3 = 3 * op.n_u
    out = dict(workload="spheres64 with n_sub = 2: 6.44 M velocity DoFs, 2.15 M level-set DoFs, 275 k pressure DoFs",
               set_fields_ms=ts, momentum_fp64=dict(ms=t64, gdofs=nu3 / t64 / 1e6),
               levelset_advect=dict(ms=t_ls, gdofs=op.n_phi / t_ls / 1e6),
               adjoint=dict(ms=t_adj, gdofs=nu3 / t_adj / 1e6), projected_normal_ms=t_n)
    op.close()
    return out


def large_case(evap, torch, dev, p: int):
    """deformed128: 128^3 cells, degree-p velocity (p = 2: 51 M DoFs, p = 3: 171 M DoFs), deformed sphere with
    spherical-harmonic noise up to l = 6 (seed 5), density ratio 1e4.  FP64 and FP32 applies, the adjoint apply, and
    the mixed-precision solve against the plain FP64 solve (both to 1e-10), each timed with CUDA events."""
    wl = workloads.make_workload("deformed128", p=p)
    op = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.current_stream()
    phi, u0, md, x = cu(wl.phi), cu(wl.u0), cu(wl.mdot), cu(wl.x)

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    nu3 = 3 * op.n_u
    res = {"workload": f"deformed128 Q{p}: 128^3 cells, {nu3 / 1e6:.1f} M velocity DoFs, deformed sphere (seed 5), "
                       "density ratio 1e4"}
    res["set_fields_ms"], _ = timed(lambda: op.set_fields(phi, u0, md))
    x32 = x.float()
    t64, _ = timed(lambda: op.apply_momentum(x, prec=64), reps=3)
    t32, _ = timed(lambda: op.apply_momentum(x32, prec=32), reps=5)
    w = cu(np.random.default_rng(7).uniform(-1, 1, nu3))
    tad, _ = timed(lambda: op.apply_adjoint(w, x, None), reps=2)
    res["momentum_fp64"] = dict(ms=t64, gdofs=nu3 / t64 / 1e6)
    c = algorithmic_counts(wl.n, p)
    res["momentum_fp32"] = dict(ms=t32, gdofs=nu3 / t32 / 1e6, hbm_gbs=c["mom32_bytes"] / t32 / 1e6)
    res["adjoint"] = dict(ms=tad, gdofs=nu3 / tad / 1e6)
    tm, (xm, im) = timed(lambda: op.solve(x, mixed=True, rtol=1e-10, max_iter=5000))
    tf, (xf, inf) = timed(lambda: op.solve(x, mixed=False, rtol=1e-10, max_iter=5000))
    res["solve_fp64"] = dict(ms=tf, iters=inf["iters"], relres=inf["relres"])
    res["solve_mixed"] = dict(ms=tm, iters=im["iters"], relres=im["relres"],
                              diff_vs_fp64_solve=float((xm - xf).norm() / xf.norm()))
    res["speedup_mixed_over_fp64"] = tf / tm
    op.close()
    del phi, u0, md, x, x32, w, xm, xf
    torch.cuda.empty_cache()
    return res


def run_reference(args):
    """--impl reference: the CPU oracle's FP64 momentum apply on all host cores (rank 0 only): every step is one
    apply on each core's sub-block (oracle_baseline), the warm-up steps untimed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    base = oracle_baseline(WORKLOAD, nb=12, reps=args.warmup + args.steps)
    value = base["value"]
    cores, model = cpu_info()
    out = dict(impl="reference", metric=METRIC, value=value, unit="GDoF/s", n_gpus=args.gpus, steps=args.steps,
               warmup=args.warmup, ms_per_step=base["apply_ms_median"], higher_is_better=True, scaling="weak",
               vs_baseline=None, dtype="f64", data="synthetic",
               config=dict(workload="spheres64: 64^3 cells, Q2 velocity, 4 random spheres, density ratio 1e3, "
                                    "random-Fourier velocity (seed 2)",
                           sample=f"{base['cores']} disjoint 12^3-cell sub-blocks, one per host core",
                           l2="CSR blocks of ~0.2 GB per core exceed the host caches"),
               cpu_baseline=dict(base, value=value, cpu=model),
               e2e=dict(value=value, unit="GDoF/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(out), flush=True)


def rates(t_ms, dofs, alg_bytes, stream_bytes, flop, hbm, alu_peak):
    """Per-apply figures of an operator: GDoF/s, %HBM against the algorithmic bytes of the method and against the
    bytes the kernel streams, and the arithmetic rate against the measured FMA peak of its pipe."""
    t = t_ms * 1e-3
    return dict(ms=t_ms, gdofs=dofs / t / 1e9, alg_bytes=alg_bytes, hbm_frac=alg_bytes / t / 1e9 / hbm,
                stream_bytes=stream_bytes, hbm_frac_streamed=stream_bytes / t / 1e9 / hbm,
                tflops=flop / t / 1e12, alu_frac=flop / t / 1e12 / alu_peak)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-solve-compare", action="store_true", help="skip the 96^3 FP64-vs-mixed solve comparison")
    ap.add_argument("--no-large", action="store_true", help="skip the 128^3 Q2/Q3 large case")
    ap.add_argument("--no-applies", action="store_true", help="skip the extra per-operator timings")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the CPU baseline's worker processes are spawned before this process touches the GPU
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_baseline(WORKLOAD)
        cores, model = cpu_info()
        cpu.update(cpu=model, host_cores=cores)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    import paper_2401_07805_gb300 as evap
    from paper_2401_07805_gb300 import build
    if not os.path.exists(evap.library_path()):
        build.build()

    wl = workloads.make_workload(WORKLOAD)
    counts = algorithmic_counts(wl.n, wl.p)
    dev = torch.device("cuda", local)
    op = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    rng = np.random.default_rng(100 + rank)
    host = dict(phi=wl.phi, u0=wl.u0, mdot=wl.mdot, x=wl.x, w=rng.uniform(-1, 1, wl.x.shape),
                wp=rng.uniform(-1, 1, wl.phi.shape), psi=wl.phi.copy(), f=rng.uniform(-1, 1, wl.x.shape))
    d = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    d["x32"] = d["x"].float()
    stream = torch.cuda.current_stream()
    nu3, nphi = 3 * op.n_u, op.n_phi
    y64 = torch.empty(nu3, dtype=torch.float64, device=dev)
    yp64 = torch.empty(nphi, dtype=torch.float64, device=dev)
    y32 = torch.empty(nu3, dtype=torch.float32, device=dev)
    yl = torch.empty(nphi, dtype=torch.float64, device=dev)
    names = ["set_fields", "mom64", "mom32", "ls_advect", "ls_reinit", "adjoint", "solve"]
    solve_info = {}

    # arithmetic peaks of this GPU at its current clocks (probes of the library, before the timed region)
    fp64_peak = evap.fma_probe(64)
    fp32_peak = evap.fma_probe(32)

    def step(dd, ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        op.set_fields(dd["phi"], dd["u0"], dd["mdot"])
        mark(1)
        for _ in range(REPS):
            op.apply_momentum(dd["x"], prec=64, with_divergence=True, out=y64, out_p=yp64)
        mark(2)
        for _ in range(REPS):
            op.apply_momentum(dd["x32"], prec=32, out=y32)
        mark(3)
        for _ in range(REPS):
            op.apply_levelset(dd["psi"], mode="advect", out=yl)
        mark(4)
        lr = op.apply_levelset(dd["psi"], mode="reinit")
        lh = op.apply_levelset(dd["psi"], mode="reinit_rhs")
        mark(5)
        g = op.apply_adjoint(dd["w"], dd["x"], dd["wp"])
        mark(6)
        xs, info = op.solve(dd["f"], mixed=True, restart=16, rtol=1e-10, max_iter=400)
        mark(7)
        solve_info.update(info)
        return dict(y=y64, yp=yp64, y32=y32, la=yl, lr=lr, lh=lh, gx=g["x"], gu=g["u0"], gphi=g["phi"], gm=g["mdot"],
                    xs=xs)

    for _ in range(args.warmup):
        step(d)
    torch.cuda.synchronize()
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = evap.launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(K):
        step(d, evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = evap.launch_count() - l0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms_step = job_time_ms(torch, dist, t_start.elapsed_time(t_end), dev, world) / K
    part = {nm: float(np.mean([evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(K)]))
            for i, nm in enumerate(names)}
    # the headline: FP64 momentum applies, the max over ranks of the 100-apply group's time
    ms_mom64 = job_time_ms(torch, dist, part["mom64"], dev, world) / REPS
    value = aggregate_gdofs(world, nu3, ms_mom64)

    # end to end through the public API with host buffers: every apply copies its input x from pinned host memory
    # in and its results y, y_p out inside the timed region (copy streams overlap the copies of neighbouring
    # applies with compute, as a streaming caller would)
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(wl.x).pin_memory()
        yh = [torch.empty(nu3, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        yph = [torch.empty(nphi, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        xd = [torch.empty(nu3, dtype=torch.float64, device=dev) for _ in range(2)]
        yd = [torch.empty(nu3, dtype=torch.float64, device=dev) for _ in range(2)]
        ypd = [torch.empty(nphi, dtype=torch.float64, device=dev) for _ in range(2)]
        cin, cout = torch.cuda.Stream(), torch.cuda.Stream()
        op.set_fields(d["phi"], d["u0"], d["mdot"])
        n_e2e = REPS * K
        in_ev = [None, None]
        out_ev = [None, None]

        def copy_in(i):
            with torch.cuda.stream(cin):
                if out_ev[i % 2] is not None:
                    cin.wait_event(out_ev[i % 2])  # the buffer's previous apply has been read out
                xd[i % 2].copy_(xh, non_blocking=True)
                in_ev[i % 2] = cin.record_event()

        def run(n):
            copy_in(0)
            for i in range(n):
                b = i % 2
                stream.wait_event(in_ev[b])
                if i + 1 < n:
                    copy_in(i + 1)
                op.apply_momentum(xd[b], prec=64, with_divergence=True, out=yd[b], out_p=ypd[b])
                done = stream.record_event()
                with torch.cuda.stream(cout):
                    cout.wait_event(done)
                    yh[b].copy_(yd[b], non_blocking=True)
                    yph[b].copy_(ypd[b], non_blocking=True)
                    out_ev[b] = cout.record_event()
            stream.wait_event(out_ev[(n - 1) % 2])

        run(10)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run(n_e2e)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = job_time_ms(torch, dist, e0.elapsed_time(e1), dev, world) / n_e2e
        e2e = dict(value=aggregate_gdofs(world, nu3, e_ms), unit="GDoF/s", ms_per_apply=e_ms,
                   h2d_bytes_per_step=int(8 * nu3 * REPS), d2h_bytes_per_step=int(8 * (nu3 + nphi) * REPS),
                   note="FP64 momentum applies through the C ABI with the input x copied in from pinned host memory "
                        "and y, y_p copied out for every apply (100 applies per step); copies of neighbouring "
                        "applies overlap with compute on two copy streams")
        del xd, yd, ypd

    peaks, peak_src = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    mom64 = rates(ms_mom64, nu3, counts["mom64_alg_bytes"], counts["mom64_bytes"], counts["mom_flop"], hbm,
                  fp64_peak)
    mom32 = rates(part["mom32"] / REPS, nu3, counts["mom32_alg_bytes"], counts["mom32_bytes"], counts["mom32_flop"],
                  hbm, fp32_peak)
    y32_err = float((y32.double() - y64).norm() / y64.norm())
    mom32["rel_err_vs_fp64"] = y32_err
    adj = rates(part["adjoint"], nu3, counts["adj_bytes"], counts["adj_bytes"] + counts["mom64_bytes"]
                - 8 * (3 * counts["Nu"] * 2 + counts["Np"]), counts["adj_flop"], hbm, fp64_peak)
    ls = dict(ms=part["ls_advect"] / REPS, gdofs=nphi / (part["ls_advect"] / REPS * 1e-3) / 1e9,
              alg_bytes=counts["ls_adv_bytes"],
              hbm_frac=counts["ls_adv_bytes"] / (part["ls_advect"] / REPS * 1e-3) / 1e9 / hbm,
              note="275 k Q1 DoFs: the 11 MB of vectors stay in L2 across back-to-back applies")
    # Dominant kernel of the step (largest share of its launch list): the FP64-accurate momentum apply, 100 launches
    # per step plus the FP64 residuals of the mixed solve, evaluated in double-float arithmetic on the FP32 pipe.  It
    # is bound by FP32 instruction issue: its roofline is the double-float FMA rate (the measured FP32 FMA rate /
    # DF_FMA_INSTR), against which the algorithmic flops are counted; the same flops against the measured FP64 FMA
    # rate (above 1: the FP64 pipe's ceiling no longer applies) and the HBM fractions (against the method's
    # algorithmic bytes and against the bytes streamed with the quadrature-point cache) are beside it.
    df_peak = fp32_peak / DF_FMA_INSTR
    roofline = dict(bound="alu",
                    kernel="k_momentum_df<2,4,0,8,false> (FP64-accurate momentum apply with divergence row in double-float "
                           "arithmetic, 100 per step)",
                    achieved=mom64["tflops"], peak=df_peak, unit="TFLOP/s", frac=mom64["tflops"] / df_peak,
                    traffic=measured_traffic("k_momentum_df", WORKLOAD), flop_per_launch=counts["mom_flop"],
                    peak_source=f"double-float FMA rate: FP32 FMA probe in this process ({fp32_peak:.1f} TFLOP/s, "
                                f"evap_fma_probe) / {DF_FMA_INSTR} FP32 instructions per double-float FMA",
                    fp64_pipe=dict(peak=fp64_peak, frac=mom64["alu_frac"],
                                   peak_source=f"FP64 FMA probe in this process, nominal {FP64_NOMINAL_TFLOPS} TFLOP/s"),
                    hbm=dict(achieved=mom64["alg_bytes"] / ms_mom64 / 1e6, peak=hbm, unit="GB/s",
                             frac=mom64["hbm_frac"], bytes_per_launch=counts["mom64_alg_bytes"],
                             frac_streamed=mom64["hbm_frac_streamed"], streamed_bytes=counts["mom64_bytes"],
                             peak_source=f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"),
                    fp32_kernel=dict(kernel="k_momentum32<2,32,3,false> (FP32 momentum apply)", bound="hbm",
                                     achieved=mom32["alg_bytes"] / (mom32["ms"] * 1e6), peak=hbm, unit="GB/s",
                                     frac=mom32["hbm_frac"], frac_streamed=mom32["hbm_frac_streamed"],
                                     traffic=measured_traffic("k_momentum32", WORKLOAD),
                                     fp32_tflops=mom32["tflops"], fp32_frac=mom32["alu_frac"]))
    whole = dict(ms=ms_step, gdofs=aggregate_gdofs(world, nu3, ms_step),
                 parts_ms=part, solve=dict(iters=solve_info.get("iters"), relres=solve_info.get("relres")),
                 note="velocity DoFs per whole step (set_fields, 100 FP64 + 100 FP32 momentum applies, 100 level-set "
                      "advections, reinitialization operators, adjoint, mixed solve)")
    applies = None
    if rank == 0 and not args.no_applies:
        applies = operator_applies(evap, torch, dev, op, d, counts, hbm)
        applies["geometry"] = geometry_subsolver(torch, op, d["phi"])
        applies["saddle"] = saddle_case(evap, torch, dev)
        applies["n_sub_2"] = subdivided_case(evap, torch, dev)
    solves = None
    if rank == 0 and not args.no_solve_compare:
        solves = solve_comparison(evap, torch, dev)
    large = None
    if rank == 0 and not args.no_large:
        op.close()
        large = {f"q{p}": large_case(evap, torch, dev, p) for p in (2, 3)}
    if rank == 0:
        out = dict(metric=METRIC, value=value, unit="GDoF/s", n_gpus=world, steps=K, warmup=args.warmup,
                   ms_per_step=ms_step, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                   data="synthetic",
                   config=dict(workload="spheres64: 64^3 cells, Q2 velocity (6.44 M DoFs), Q1 level set (275 k "
                                        "DoFs), 4 random spheres, density ratio 1e3, random-Fourier velocity",
                               value="FP64 momentum operator apply with divergence row, 100 back-to-back applies "
                                     "per step",
                               step="set_fields + 100 FP64 + 100 FP32 momentum applies + 100 level-set advections + "
                                    "reinitialization operators + adjoint + mixed solve",
                               l2="inputs larger than L2 (no flush)", parallelism=f"replicas x{world}"),
                   momentum_fp64=mom64, momentum_fp32=mom32, adjoint=adj, levelset_advect=ls,
                   peaks=dict(fp64_tflops_measured=fp64_peak, fp64_tflops_nominal=FP64_NOMINAL_TFLOPS,
                              fp32_tflops_measured=fp32_peak, fp32_tflops_nominal=FP32_NOMINAL_TFLOPS,
                              hbm_gbs=hbm, hbm_source=peak_src),
                   roofline=roofline, whole_step=whole, applies=applies, solve_comparison=solves, large_case=large,
                   cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches), clocks=clocks)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
