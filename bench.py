"""Benchmark of the matrix-free evaporation hot path on GB300.

One step = one pass of the whole hot path over the 64^3-cell four-sphere workload (Q2 velocity, 6.44 M velocity
DoFs, 275 k level-set DoFs, density ratio 1e3, random-Fourier velocity):
  set_fields (material law table + variant-2 transport velocity with closest-point projection)
  -> momentum apply FP64 with divergence row -> momentum apply FP32 -> level-set advect / reinit / reinit RHS (FP64)
  -> adjoint apply (all four gradients) -> mixed-precision GMRES(16) solve to 1e-10.
value = velocity DoFs per step / step time (GDoF/s of the whole pass); per-operator GDoF/s, bytes and the roofline
of the dominant kernel are reported beside it.  Inputs (~0.5 GB touched per step) exceed the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs an independent replica (weak scaling, no collective on the data path); rank 0 prints
one JSON line.  --impl reference times the CPU oracle on a bounded sample of the same workload instead.
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
# sources are unchanged: {(kernel, workload): (bytes, sha256 prefix of the sources, profile summary)}.
MEASURED_TRAFFIC = {
    ("k_momentum32", "spheres64"): (431_719_680, "a39b9c808096dfb6", "profiles/k_momentum32_spheres64.md"),
    ("k_momentum64", "spheres64"): (1_228_852_224, "9de9670fb8e2d3b1", "profiles/k_momentum64_spheres64.md"),
}
TRAFFIC_SOURCES = {"k_momentum32": ("paper_2401_07805_gb300/csrc/momentum32.cu",
                                    "paper_2401_07805_gb300/csrc/basis_ct.cuh",
                                    "paper_2401_07805_gb300/csrc/evap_internal.cuh"),
                   "k_momentum64": ("paper_2401_07805_gb300/csrc/momentum.cu",
                                    "paper_2401_07805_gb300/csrc/physics.cuh",
                                    "paper_2401_07805_gb300/csrc/basis_ct.cuh",
                                    "paper_2401_07805_gb300/csrc/evap_internal.cuh")}


def sources_digest(kernel):
    """sha256 prefix of what the kernel is compiled from: its .cu, the basis tables, and the device-side part of
    evap_internal.cuh (everything before the host-side mesh struct, which does not enter the kernel)."""
    import hashlib
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES[kernel]:
        data = open(os.path.join(ROOT, rel), "rb").read()
        if rel.endswith("evap_internal.cuh"):
            data = data.split(b"struct evap_mesh {")[0]
        h.update(data)
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload):
    rec = MEASURED_TRAFFIC.get((kernel, workload))
    if rec is None or rec[1] != sources_digest(kernel):
        return None
    return rec[0]


# Nominal FP64 rate of GB300 (profiling recipe table: 1.25 TFLOP/s); the FP64 FMA probe measured 1.19 TFLOP/s.
FP64_PEAK_TFLOPS = 1.25
# FP32 peak from the unit counts and clocks of the profiling recipe: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x
# 2.07 GHz maximum SM clock = 80.5 TFLOP/s (the FMA probe measured 73 TFLOP/s at the clocks it saw).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


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
        # FP64 apply: x in, y and y_p out, the 19 cached FP64 coefficients per quadrature point streamed in
        mom64_bytes=8 * (3 * Nu * 2 + Np) + 8 * nc * 19 * nq,
        # FP32 apply: x in, y out, 12 FP32 u0 coefficients per quadrature point, cell code and table index
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


def oracle_sample(wl, nb: int = 8, reps: int = 1):
    """Time the CPU oracle on a bounded sample: every hot-path row of an nb^3-cell sub-block of the workload
    (momentum element matrices and apply with divergence rows, transport velocity of the sub-block's band nodes,
    level-set advect/reinit/reinit-RHS, adjoint parameter gradients).  Returns (seconds, velocity DoFs covered)."""
    from oracle import adjoint, fe, levelset, momentum, transport
    n = wl.n
    mesh = fe.Mesh(n, wl.p, wl.L)
    pb = momentum.Problem.from_workload(wl)
    c0 = n // 2 - nb // 2
    r = np.arange(c0, c0 + nb)
    Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
    cells = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    du = np.unique(mesh.dofs_u(cells))
    d1 = np.unique(mesh.dofs_phi(cells))
    rng = np.random.default_rng(0)
    w = rng.uniform(-1, 1, wl.x.shape)
    t0 = time.perf_counter()
    for _ in range(reps):
        momentum.apply_rows(pb, wl.x, du)
        momentum.divergence_rows(pb, wl.x, d1)
        band = d1[(wl.phi[d1] > -workloads_tanh3()) & (wl.phi[d1] < np.tanh(1.5))]
        transport.transport_velocity(mesh, wl.phi, wl.u0, wl.mdot, wl.params, nodes=band[: max(1, len(band) // 4)])
        sub = fe.Mesh(nb, 1, nb * mesh.h)
        ug = np.zeros(3 * sub.n_phi)
        phis = rng.uniform(-1, 1, sub.n_phi)
        for mode in ("advect", "reinit", "reinit_rhs"):
            levelset.apply(sub, mode, phis, phis, ug, wl.params)
        sub_wl = workloads.random_workload(nb, p=wl.p, seed=1)
        sub_pb = momentum.Problem.from_workload(sub_wl)
        adjoint.param_gradients(sub_pb, sub_wl.x, sub_wl.x, np.ones(sub_pb.mesh.n_phi))
    dt = (time.perf_counter() - t0) / reps
    return dt, 3 * len(du)


def workloads_tanh3():
    return float.fromhex("0x1.fd77d111a0b00p-1")


def oracle_sample_subprocess(nb: int, reps: int = 1):
    """Run oracle_sample in a fresh single-threaded interpreter (BLAS/OpenMP pinned to 1 thread, so the reported
    core count is the number actually used; a new process is spawned, never forked from one that holds a GPU
    context).  Returns (seconds, velocity DoFs covered, cores)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json, sys; sys.path.insert(0, %r); import bench, workloads; "
            "wl = workloads.make_workload(bench.WORKLOAD); dt, dofs = bench.oracle_sample(wl, nb=%d, reps=%d); "
            "print(json.dumps([dt, dofs]))" % (ROOT, nb, reps))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    dt, dofs = json.loads(out.stdout.strip().splitlines()[-1])
    return dt, dofs, 1


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
    """Per-operator throughput on the 64^3 four-sphere workload: 100 back-to-back applies after 10 warm-ups each
    (momentum FP64 with the divergence row, momentum FP32, level-set advection FP64), the closest-point transport
    pass alone (20 repeats: band nodes/s, point evaluations, flags), and the adjoint on the 48^3 sphere
    (2.74 M DoFs, 20 applies).  Inputs are larger than the L2 for every operator except the level set."""
    nu3, nphi = 3 * op.n_u, op.n_phi
    x, x32, psi = d["x"], d["x32"], d["psi"]
    y64 = torch.empty(nu3, dtype=torch.float64, device=dev)
    yp64 = torch.empty(nphi, dtype=torch.float64, device=dev)
    y32 = torch.empty(nu3, dtype=torch.float32, device=dev)
    yl = torch.empty(nphi, dtype=torch.float64, device=dev)
    out = {}
    t = back_to_back(torch, lambda: op.apply_momentum(x, prec=64, with_divergence=True, out=y64, out_p=yp64), 100, 10)
    out["momentum_fp64"] = dict(ms=t, gdofs=nu3 / t / 1e6, gbs=counts["mom64_bytes"] / t / 1e6,
                                fp64_tflops=counts["mom_flop"] / t / 1e9)
    t = back_to_back(torch, lambda: op.apply_momentum(x32, prec=32, out=y32), 100, 10)
    out["momentum_fp32"] = dict(ms=t, gdofs=nu3 / t / 1e6, gbs=counts["mom32_bytes"] / t / 1e6,
                                hbm_frac=counts["mom32_bytes"] / t / 1e6 / hbm,
                                fp32_tflops=counts["mom32_flop"] / t / 1e9,
                                rel_err_vs_fp64=float((y32.double() - y64).norm() / y64.norm()))
    t = back_to_back(torch, lambda: op.apply_levelset(psi, mode="advect", out=yl), 100, 10)
    out["levelset_advect_fp64"] = dict(ms=t, gdofs=nphi / t / 1e6, gbs=counts["ls_adv_bytes"] / t / 1e6)
    t = back_to_back(torch, op.update_transport_velocity, 20, 2)
    st = op.transport_stats()
    out["transport_velocity"] = dict(ms=t, band_nodes=st["band_nodes"], band_nodes_per_s=st["band_nodes"] / t * 1e3,
                                     evaluations_per_node=st["evaluations"] / max(st["band_nodes"], 1),
                                     flagged=st["flagged"])
    # adjoint on the 48^3 sphere
    wl = workloads.make_workload("sphere48")
    op4 = evap.Operator(wl.n, wl.p, wl.L, dict(wl.params))
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    op4.set_fields(cu(wl.phi), cu(wl.u0), cu(wl.mdot))
    w, xx, wp = cu(wl.extra["w"]), cu(wl.x), cu(wl.extra["w_p"])
    t = back_to_back(torch, lambda: op4.apply_adjoint(w, xx, wp), 20, 3)
    c4 = algorithmic_counts(wl.n, wl.p)
    out["adjoint_sphere48"] = dict(ms=t, gdofs=3 * op4.n_u / t / 1e6, fp64_tflops=c4["adj_flop"] / t / 1e9)
    op4.close()
    out["note"] = "100 back-to-back applies after 10 warm-ups (transport 20 after 2, adjoint 20 after 3)"
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
    """--impl reference: the CPU oracle, timed on a bounded sample per step (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each step is a bounded sample of the workload (all hot-path rows of a 10^3-cell sub-block), timed in a
    # single-threaded interpreter; the whole --steps K --warmup W run stays within a few minutes
    oracle_sample_subprocess(nb=4, reps=max(1, args.warmup))
    dt, dofs, _ = oracle_sample_subprocess(nb=10, reps=args.steps)
    t = dt * args.steps
    value = dofs * args.steps / t / 1e9
    cores, model = cpu_info()
    out = dict(impl="reference", metric=METRIC, value=value, unit="GDoF/s", n_gpus=args.gpus, steps=args.steps,
               warmup=args.warmup, ms_per_step=1e3 * t / args.steps, higher_is_better=True, scaling="weak",
               vs_baseline=None, dtype="f64", data="synthetic",
               config=dict(workload="spheres64: 64^3 cells, Q2 velocity, 4 random spheres, density ratio 1e3, "
                                    "random-Fourier velocity (seed 2)", sample="10^3-cell sub-block per step",
                           l2="sample fits in host caches (CPU)"),
               cpu_baseline=dict(value=value, unit="GDoF/s", cores=1, kind="oracle",
                                 sample="all hot-path rows of a 10^3-cell sub-block of the 64^3 workload "
                                        "(single thread)", cpu=model),
               e2e=dict(value=value, unit="GDoF/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-solve-compare", action="store_true", help="skip the 96^3 FP64-vs-mixed solve comparison")
    ap.add_argument("--no-large", action="store_true", help="skip the 128^3 Q2/Q3 large case")
    ap.add_argument("--no-applies", action="store_true", help="skip the per-operator back-to-back apply timings")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
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
    names = ["set_fields", "mom64", "mom32", "ls_advect", "ls_reinit", "ls_rhs", "adjoint", "solve"]
    solve_info = {}

    def step(dd, ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        op.set_fields(dd["phi"], dd["u0"], dd["mdot"])
        mark(1)
        y, yp = op.apply_momentum(dd["x"], prec=64, with_divergence=True)
        mark(2)
        y32 = op.apply_momentum(dd["x32"], prec=32)
        mark(3)
        la = op.apply_levelset(dd["psi"], mode="advect")
        mark(4)
        lr = op.apply_levelset(dd["psi"], mode="reinit")
        mark(5)
        lh = op.apply_levelset(dd["psi"], mode="reinit_rhs")
        mark(6)
        g = op.apply_adjoint(dd["w"], dd["x"], dd["wp"])
        mark(7)
        xs, info = op.solve(dd["f"], mixed=True, restart=16, rtol=1e-10, max_iter=400)
        mark(8)
        solve_info.update(info)
        return dict(y=y, yp=yp, y32=y32, la=la, lr=lr, lh=lh, gx=g["x"], gu=g["u0"], gphi=g["phi"], gm=g["mdot"], xs=xs)

    for _ in range(args.warmup):
        step(d)
    torch.cuda.synchronize()
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(9)] for _ in range(K)]
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
    ms_total = job_time_ms(torch, dist, t_start.elapsed_time(t_end), dev, world)
    ms_step = ms_total / K
    part = {nm: float(np.mean([evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(K)])) for i, nm in enumerate(names)}
    Nu3 = 3 * counts["Nu"]
    value = aggregate_gdofs(world, Nu3, ms_step)

    # end to end: pinned host inputs copied in and all results copied out inside the timed region.  The copies run on
    # two copy streams (host-to-device for step k+1 while step k computes; device-to-host of step k's results after
    # its compute), as a streaming pipeline would; every step still moves all of its inputs and results.
    e2e = None
    if not args.no_e2e:
        pinned = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
        outs_host = None
        h2d = sum(v.numel() * v.element_size() for v in pinned.values())
        cin, cout = torch.cuda.Stream(), torch.cuda.Stream()

        def fetch_inputs():
            with torch.cuda.stream(cin):
                nxt = {k: v.to(dev, non_blocking=True) for k, v in pinned.items()}
                return nxt, cin.record_event()

        total = args.warmup + K
        nxt, ev_in = fetch_inputs()
        ev_out = None
        for it in range(total):
            if it == args.warmup:
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                nxt, ev_in = fetch_inputs()  # the timed steps copy their own inputs
            stream.wait_event(ev_in)
            dd = nxt
            for v in dd.values():
                v.record_stream(stream)
            if it + 1 < total and it + 1 != args.warmup:
                nxt, ev_in = fetch_inputs()
            dd["x32"] = dd["x"].float()
            outs = step(dd)
            if outs_host is None:
                outs_host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in outs.items()}
            done = stream.record_event()
            with torch.cuda.stream(cout):
                cout.wait_event(done)
                for k, v in outs.items():
                    v.record_stream(cout)
                    outs_host[k].copy_(v, non_blocking=True)
                ev_out = cout.record_event()
        stream.wait_event(ev_out)
        e1.record(stream)
        torch.cuda.synchronize()
        d2h = sum(v.numel() * v.element_size() for v in outs_host.values())
        e_ms = job_time_ms(torch, dist, e0.elapsed_time(e1) / K, dev, world)
        e2e = dict(value=aggregate_gdofs(world, Nu3, e_ms), unit="GDoF/s", ms_per_step=e_ms,
                   h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h),
                   note="inputs of step k+1 copied in while step k computes; results copied out after each step")

    peaks, peak_src = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    # FP64 momentum apply: FP64-pipe bound (its FP64-pipe roofline is reported beside the dominant kernel's)
    t_mom = part["mom64"] * 1e-3
    mom_tflops = counts["mom_flop"] / t_mom / 1e12
    breakdown = {
        "set_fields_ms": part["set_fields"],
        "momentum_fp64": dict(ms=part["mom64"], gdofs=Nu3 / (part["mom64"] * 1e-3) / 1e9,
                              gbs=counts["mom64_bytes"] / (part["mom64"] * 1e-3) / 1e9,
                              hbm_frac=counts["mom64_bytes"] / (part["mom64"] * 1e-3) / 1e9 / hbm,
                              fp64_tflops=mom_tflops),
        "momentum_fp32": dict(ms=part["mom32"], gdofs=Nu3 / (part["mom32"] * 1e-3) / 1e9,
                              fp32_tflops=counts["mom32_flop"] / (part["mom32"] * 1e-3) / 1e12,
                              gbs=counts["mom32_bytes"] / (part["mom32"] * 1e-3) / 1e9,
                              hbm_frac=counts["mom32_bytes"] / (part["mom32"] * 1e-3) / 1e9 / hbm),
        "levelset_advect": dict(ms=part["ls_advect"], gdofs=counts["Np"] / (part["ls_advect"] * 1e-3) / 1e9),
        "levelset_reinit": dict(ms=part["ls_reinit"], gdofs=counts["Np"] / (part["ls_reinit"] * 1e-3) / 1e9),
        "levelset_reinit_rhs": dict(ms=part["ls_rhs"], gdofs=counts["Np"] / (part["ls_rhs"] * 1e-3) / 1e9),
        "adjoint": dict(ms=part["adjoint"], gdofs=Nu3 / (part["adjoint"] * 1e-3) / 1e9,
                        fp64_tflops=counts["adj_flop"] / (part["adjoint"] * 1e-3) / 1e12),
        "solve_mixed": dict(ms=part["solve"], iters=solve_info.get("iters"), relres=solve_info.get("relres")),
    }
    # Dominant kernel of the step (largest share of the launch list): the FP64 momentum apply, launched three times
    # per step (the step's own apply and the two FP64 residuals of the mixed solve).  It is bound by the FP64 pipe
    # (~90 % active; its ~1.9 flop per algorithmic byte is ten times GB300's FP64 machine balance), so its roofline
    # is the FP64 rate; its HBM fraction is reported beside it.  The FP32 apply inside the mixed solve (HBM-bound:
    # its roof is the larger of bytes / HBM peak and flops / FP32 peak) follows as the second kernel.
    g64 = counts["mom64_bytes"] / t_mom / 1e9
    t32 = part["mom32"] * 1e-3
    f32 = counts["mom32_flop"] / t32 / 1e12
    g32 = counts["mom32_bytes"] / t32 / 1e9
    hbm_bound = counts["mom32_bytes"] / (hbm * 1e9) >= counts["mom32_flop"] / (FP32_PEAK_TFLOPS * 1e12)
    alu32 = dict(achieved=f32, peak=FP32_PEAK_TFLOPS, unit="TFLOP/s", frac=f32 / FP32_PEAK_TFLOPS,
                 flop_per_launch=counts["mom32_flop"],
                 peak_source="FP32 peak from the recipe's unit counts and max clock (152 SM x 128 lanes x 2 x 2.07 "
                             "GHz); the FMA probe measured 73 TFLOP/s")
    mem32 = dict(achieved=g32, peak=hbm, unit="GB/s", frac=g32 / hbm, bytes_per_launch=counts["mom32_bytes"],
                 peak_source=peak_src)
    main32, other32 = (mem32, alu32) if hbm_bound else (alu32, mem32)
    roofline = dict(bound="alu",
                    kernel="k_momentum<double,2,8> (FP64 momentum apply: the step's apply and the two FP64 residuals "
                           "of the mixed solve)",
                    achieved=mom_tflops, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s", frac=mom_tflops / FP64_PEAK_TFLOPS,
                    traffic=measured_traffic("k_momentum64", WORKLOAD), flop_per_launch=counts["mom_flop"],
                    peak_source="nominal FP64 rate of the profiling recipe's table; an FMA probe measured 1.19 TFLOP/s",
                    hbm=dict(achieved=g64, peak=hbm, unit="GB/s", frac=g64 / hbm,
                             bytes_per_launch=counts["mom64_bytes"], peak_source=peak_src),
                    fp32_kernel=dict(kernel="k_momentum32<2,32,3> (FP32 momentum apply inside the mixed solve)",
                                     bound="hbm" if hbm_bound else "alu",
                                     achieved=main32["achieved"], peak=main32["peak"], unit=main32["unit"],
                                     frac=main32["frac"], traffic=measured_traffic("k_momentum32", WORKLOAD),
                                     peak_source=main32["peak_source"],
                                     **{"alu" if hbm_bound else "hbm": other32}))
    applies = None
    if rank == 0 and not args.no_applies:
        applies = operator_applies(evap, torch, dev, op, d, counts, hbm)
        applies["geometry"] = geometry_subsolver(torch, op, d["phi"])
        applies["saddle"] = saddle_case(evap, torch, dev)
    solves = None
    if rank == 0 and not args.no_solve_compare:
        solves = solve_comparison(evap, torch, dev)
    large = None
    if rank == 0 and not args.no_large:
        op.close()
        large = {f"q{p}": large_case(evap, torch, dev, p) for p in (2, 3)}
    cpu = None
    if rank == 0 and not args.no_cpu:
        dt, dofs, used = oracle_sample_subprocess(nb=20)
        cores, model = cpu_info()
        cpu = dict(value=dofs / dt / 1e9, unit="GDoF/s", cores=used, kind="oracle",
                   sample="all hot-path rows (momentum + divergence rows, transport velocity of a quarter of the "
                          "band nodes, 3 level-set operators, adjoint gradients) of a 20^3-cell sub-block of the 64^3 "
                          "workload, numpy in a single-threaded process", seconds=dt, cpu=model, host_cores=cores)
    if rank == 0:
        out = dict(metric=METRIC, value=value, unit="GDoF/s", n_gpus=world, steps=K, warmup=args.warmup,
                   ms_per_step=ms_step, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                   data="synthetic",
                   config=dict(workload="spheres64: 64^3 cells, Q2 velocity (6.44 M DoFs), Q1 level set (275 k "
                                        "DoFs), 4 random spheres, density ratio 1e3, random-Fourier velocity",
                               step="set_fields + FP64/FP32 momentum + 3 level-set applies + adjoint + mixed solve",
                               l2="inputs larger than L2 (no flush)", parallelism=f"replicas x{world}"),
                   roofline=roofline, breakdown=breakdown, applies=applies, solve_comparison=solves, large_case=large,
                   cpu_baseline=cpu, e2e=e2e,
                   gpu_launches=int(launches), clocks=clocks)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
