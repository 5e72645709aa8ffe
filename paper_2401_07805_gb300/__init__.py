"""GB300 matrix-free operators of the diffuse-interface evaporation model (arXiv 2401.07805).

Thin Python binding of the C ABI in include/evap.h (ctypes): it checks tensor shapes/dtypes/devices, passes raw
device pointers and the current torch CUDA stream, and raises on a non-zero status.  Every step of every operator
runs in the CUDA library libevap.so; there is no CPU fallback: if the library is missing or no GPU is present the
calls raise.

    op = Operator(n=64, degree=2, params=dict(rho_l=1000.0, rho_g=1.0, ...))
    op.set_fields(phi, u, mdot)              # float64 CUDA (or CPU, copied) tensors
    y, y_p = op.apply_momentum(x, prec=64, with_divergence=True)
    y_ls = op.apply_levelset(psi, mode="advect")
    grads = op.apply_adjoint(w, x, w_p)
    x, info = op.solve(f, mixed=True)
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

__all__ = ["Operator", "EvapError", "MomentumFunction", "lib", "library_path", "launch_count", "DEFAULT_PARAMS",
           "LEVELSET_MODES"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()

LEVELSET_MODES = {"advect": 0, "reinit": 1, "reinit_rhs": 2}
STATUS = {0: "EVAP_OK", -1: "EVAP_EINVAL", -2: "EVAP_ECUDA", -3: "EVAP_ENOTCONV", -4: "EVAP_ENOFIELDS",
          -5: "EVAP_ENOMEM", -6: "EVAP_ENONFINITE", -7: "EVAP_ETIMEOUT"}

# Exported symbols of include/evap.h with their ctypes signatures.
_c_int, _c_dbl, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p


class EvapParams(ctypes.Structure):
    _fields_ = [("rho_l", _c_dbl), ("rho_g", _c_dbl), ("mu_l", _c_dbl), ("mu_g", _c_dbl), ("eps", _c_dbl),
                ("dt", _c_dbl), ("c_mass", _c_dbl), ("theta", _c_dbl), ("dtau", _c_dbl), ("variant", _c_int),
                ("stress", _c_int), ("corr_zone", _c_int), ("newton", _c_int), ("dirichlet_faces", ctypes.c_uint),
                ("cpp_tol", _c_dbl), ("cpp_kmax", _c_int), ("eta_n", _c_dbl), ("eta_kappa", _c_dbl), ("n_sub", _c_int)]


SIGNATURES = {
    "evap_create_mesh": (_c_int, [_c_int, _c_int, _c_dbl, ctypes.POINTER(EvapParams), ctypes.POINTER(_vp)]),
    "evap_destroy": (_c_int, [_vp]),
    "evap_sizes": (_c_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "evap_pressure_size": (_c_int, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "evap_set_fields": (_c_int, [_vp, _vp, _vp, _vp, _vp]),
    "evap_set_transport_velocity": (_c_int, [_vp, _vp, _vp]),
    "evap_get_transport_velocity": (_c_int, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int64), _vp]),
    "evap_get_closest_points": (_c_int, [_vp, _vp, _vp]),
    "evap_update_transport_velocity": (_c_int, [_vp, _vp]),
    "evap_transport_stats": (_c_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64), _vp]),
    "evap_projected_normal": (_c_int, [_vp, _vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_dbl), _vp]),
    "evap_curvature": (_c_int, [_vp, _vp, _vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_dbl), _vp]),
    "evap_set_levelset_normal": (_c_int, [_vp, _vp, _vp]),
    "evap_reinitialize": (_c_int, [_vp, _vp, _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_dbl), _vp]),
    "evap_advect_levelset": (_c_int, [_vp, _vp, _c_int, _c_dbl, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                      ctypes.POINTER(_c_dbl), _vp]),
    "evap_set_checks": (_c_int, [_vp, _c_int]),
    "evap_set_deterministic": (_c_int, [_vp, _c_int]),
    "evap_time_step": (_c_int, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_c_dbl), _c_dbl, _c_int, _c_dbl, _c_int,
                                _c_int, _c_dbl, ctypes.POINTER(_c_int), ctypes.POINTER(_c_dbl),
                                ctypes.POINTER(_c_dbl), _vp]),
    "evap_apply_saddle": (_c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "evap_apply_schur": (_c_int, [_vp, _vp, _vp, _vp]),
    "evap_solve_saddle": (_c_int, [_vp, _vp, _vp, _vp, _c_int, _c_dbl, _c_int, ctypes.POINTER(_c_int),
                                   ctypes.POINTER(_c_dbl), _vp]),
    "evap_surface_tension": (_c_int, [_vp, _vp, _vp, _c_dbl, _vp, _vp]),
    "evap_apply_momentum": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _vp]),
    "evap_apply_levelset": (_c_int, [_vp, _c_int, _c_int, _vp, _vp, _vp]),
    "evap_apply_adjoint": (_c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "evap_solve": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_dbl, _c_int, ctypes.POINTER(_c_int),
                            ctypes.POINTER(_c_dbl), _vp]),
    "evap_jacobi_diagonal": (_c_int, [_vp, _vp, _vp]),
    "evap_jacobi_diagonal_noalloc": (_c_int, [_vp, _vp, _vp]),
    "evap_status_string": (ctypes.c_char_p, [_c_int]),
    "evap_last_error": (ctypes.c_char_p, []),
    "evap_launch_count": (ctypes.c_int64, []),
    "evap_fma_probe": (_c_int, [_c_int, ctypes.POINTER(_c_dbl), _vp]),
}

DEFAULT_PARAMS = dict(rho_l=1000.0, rho_g=1.0, mu_l=1e-3, mu_g=1e-5, eps=None, dt=1e-4, c_mass=None, theta=0.5,
                      dtau=None, variant=2, stress=1, corr_zone=0, newton=1, dirichlet_faces=0x3F, cpp_tol=1e-10,
                      cpp_kmax=20, eta_n=2.0, eta_kappa=2.0, n_sub=1)


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libevap.so")


def lib() -> ctypes.CDLL:
    """Load libevap.so (built in-tree by paper_2401_07805_gb300.build); raise if it is absent."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with paper_2401_07805_gb300.build.build(); "
                                   "the operators exist only as CUDA kernels (no CPU fallback)")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


class EvapError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().evap_last_error().decode()
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def fma_probe(prec: int = 64) -> float:
    """Measured FMA throughput (TFLOP/s) of the current device in FP64 (prec 64) or FP32 (prec 32)."""
    t = ctypes.c_double()
    _check(lib().evap_fma_probe(int(prec), ctypes.byref(t), _stream()), "evap_fma_probe")
    return t.value


def launch_count() -> int:
    """Kernels launched by libevap.so in this process so far."""
    return int(lib().evap_launch_count())


def _check(rc: int, where: str, allow=()):
    if rc != 0 and rc not in allow:
        raise EvapError(rc, where)
    return rc


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_params(n: int, L: float = 1.0, **over) -> EvapParams:
    prm = dict(DEFAULT_PARAMS)
    prm.update({k: v for k, v in over.items() if k in DEFAULT_PARAMS})
    h = L / n
    if prm["eps"] is None:
        prm["eps"] = h
    if prm["c_mass"] is None:
        prm["c_mass"] = 1.0 / prm["dt"]
    if prm["dtau"] is None:
        prm["dtau"] = min(prm["eps"], prm["dt"])
    return EvapParams(**{k: prm[k] for k, _ in EvapParams._fields_})


class Operator:
    """One mesh + parameter set + coefficient fields; owns a library handle on the current CUDA device."""

    def __init__(self, n: int, degree: int = 2, L: float = 1.0, params: dict | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the operators run only as CUDA kernels)")
        self.n, self.degree, self.L = n, degree, L
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._params = make_params(n, L, **(params or {}))
        self._h = ctypes.c_void_p()
        _check(lib().evap_create_mesh(n, degree, L, ctypes.byref(self._params), ctypes.byref(self._h)),
               "evap_create_mesh")
        nu, nphi = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().evap_sizes(self._h, ctypes.byref(nu), ctypes.byref(nphi)), "evap_sizes")
        self.n_u, self.n_phi = nu.value, nphi.value  # velocity nodes, level-set nodes
        npr = ctypes.c_int64()
        _check(lib().evap_pressure_size(self._h, ctypes.byref(npr)), "evap_pressure_size")
        self.n_p = npr.value  # pressure nodes (the divergence row, p, w_p)
        self.fields_version = 0  # bumped by every call that replaces (or drops) the mesh's fields

    # ------------------------------------------------------------------------------------------------- helpers
    def close(self):
        if self._h:
            lib().evap_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, t: torch.Tensor, numel: int, dtype: torch.dtype, name: str) -> torch.Tensor:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if t.numel() != numel:
            raise ValueError(f"{name} has {t.numel()} entries, expected {numel}")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if t.device != self.device:
            t = t.to(self.device, non_blocking=True)  # host buffers are copied in (end-to-end path)
        return t.contiguous()

    def _out(self, out, numel, dtype):
        if out is None:
            return torch.empty(numel, dtype=dtype, device=self.device)
        if out.numel() != numel or out.dtype != dtype or out.device != self.device or not out.is_contiguous():
            raise ValueError("bad output tensor")
        return out

    # ------------------------------------------------------------------------------------------------ C ABI
    def set_fields(self, phi: torch.Tensor, u: torch.Tensor, mdot: torch.Tensor):
        phi = self._dev(phi, self.n_phi, torch.float64, "phi")
        u = self._dev(u, 3 * self.n_u, torch.float64, "u")
        mdot = self._dev(mdot, self.n_phi, torch.float64, "mdot")
        self.fields_version += 1
        _check(lib().evap_set_fields(self._h, _ptr(phi), _ptr(u), _ptr(mdot), _stream()), "evap_set_fields")

    def set_transport_velocity(self, u_gamma: torch.Tensor):
        ug = self._dev(u_gamma, 3 * self.n_phi, torch.float64, "u_gamma")
        _check(lib().evap_set_transport_velocity(self._h, _ptr(ug), _stream()), "evap_set_transport_velocity")

    def transport_velocity(self):
        ug = torch.empty(3 * self.n_phi, dtype=torch.float64, device=self.device)
        flags = torch.empty(self.n_phi, dtype=torch.int32, device=self.device)
        nf = ctypes.c_int64()
        _check(lib().evap_get_transport_velocity(self._h, _ptr(ug), _ptr(flags), ctypes.byref(nf), _stream()),
               "evap_get_transport_velocity")
        return ug, flags, nf.value

    def closest_points(self):
        """Points y [3, N_phi] (physical coordinates) whose velocity the last transport-velocity pass took: the
        closest point of each projection-band node (App. C), the node itself elsewhere."""
        y = torch.empty(3 * self.n_phi, dtype=torch.float64, device=self.device)
        _check(lib().evap_get_closest_points(self._h, _ptr(y), _stream()), "evap_get_closest_points")
        return y.view(3, self.n_phi)

    def update_transport_velocity(self):
        """Recompute u_Gamma from the current fields (the pass set_fields runs)."""
        _check(lib().evap_update_transport_velocity(self._h, _stream()), "evap_update_transport_velocity")

    def transport_stats(self):
        """(band nodes, point evaluations, flagged nodes) of the last closest-point pass."""
        b, e, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().evap_transport_stats(self._h, ctypes.byref(b), ctypes.byref(e), ctypes.byref(f), _stream()),
               "evap_transport_stats")
        return dict(band_nodes=b.value, evaluations=e.value, flagged=f.value)

    # ---------------------------------------------------------------------------- level-set geometry sub-solver
    def projected_normal(self, raise_on_notconv: bool = False):
        """Q1 projected normal [3 N_phi] of the current level set (Eq. normal_vector_regularized) and CG info."""
        n = torch.empty(3 * self.n_phi, dtype=torch.float64, device=self.device)
        its, rel = ctypes.c_int(), ctypes.c_double()
        rc = lib().evap_projected_normal(self._h, _ptr(n), ctypes.byref(its), ctypes.byref(rel), _stream())
        _check(rc, "evap_projected_normal", allow=() if raise_on_notconv else (-3,))
        return n, dict(iters=its.value, relres=rel.value, converged=rc == 0)

    def curvature(self, n: torch.Tensor, raise_on_notconv: bool = False):
        """Regularized curvature [N_phi] of the Q1 normal field n (Eq. curvature_regularized) and CG info."""
        n = self._dev(n, 3 * self.n_phi, torch.float64, "n")
        kappa = torch.empty(self.n_phi, dtype=torch.float64, device=self.device)
        its, rel = ctypes.c_int(), ctypes.c_double()
        rc = lib().evap_curvature(self._h, _ptr(n), _ptr(kappa), ctypes.byref(its), ctypes.byref(rel), _stream())
        _check(rc, "evap_curvature", allow=() if raise_on_notconv else (-3,))
        return kappa, dict(iters=its.value, relres=rel.value, converged=rc == 0)

    def set_levelset_normal(self, n: torch.Tensor | None):
        """Frozen normal of the reinitialization operators: nodal field n [3 N_phi], or None for grad phi/|grad phi|."""
        nn = None if n is None else self._dev(n, 3 * self.n_phi, torch.float64, "n")
        _check(lib().evap_set_levelset_normal(self._h, _ptr(nn), _stream()), "evap_set_levelset_normal")

    def reinitialize(self, psi: torch.Tensor, steps: int, raise_on_notconv: bool = False):
        """`steps` reinitialization pseudo-time steps from psi (Eq. reinitialization); returns (psi, info)."""
        out = self._dev(psi, self.n_phi, torch.float64, "psi").clone()
        its, ch = ctypes.c_int(), ctypes.c_double()
        rc = lib().evap_reinitialize(self._h, _ptr(out), int(steps), ctypes.byref(its), ctypes.byref(ch), _stream())
        _check(rc, "evap_reinitialize", allow=() if raise_on_notconv else (-3,))
        return out, dict(iters=its.value, last_change=ch.value, converged=rc == 0)

    def advect_levelset(self, max_iters: int, tol: float = 0.0, out=None, raise_on_notconv: bool = False):
        """Algorithm 2 step 1: fixed point of transport velocity and Crank-Nicolson advection from the fields' level
        set; returns (phi^(n+1) [N_phi], info)."""
        phi = self._out(out, self.n_phi, torch.float64)
        fp, lin, ch = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        rc = lib().evap_advect_levelset(self._h, _ptr(phi), int(max_iters), float(tol), ctypes.byref(fp),
                                        ctypes.byref(lin), ctypes.byref(ch), _stream())
        _check(rc, "evap_advect_levelset", allow=() if raise_on_notconv else (-3,))
        return phi, dict(fp_iters=fp.value, lin_iters=lin.value, last_change=ch.value, converged=rc == 0)

    def time_step(self, phi: torch.Tensor, u: torch.Tensor, p: torch.Tensor, mdot: torch.Tensor, gravity=None,
                  fp_iters: int = 2, reinit_steps: int = 2, ns_rtol: float = 1e-8, u_prev=None,
                  picard_iters: int = 1, picard_atol: float = 1e-10, alpha: float = 0.0,
                  raise_on_notconv: bool = False):
        """One coupled step (velocity-pressure solve with Picard iterations, or Newton iterations on a mesh created
        with newton = 1; BDF1, or BDF2 given u_prev = u^(n-1); then Algorithm 2) from (phi, u, p) at t^n; returns new
        tensors (phi, u, p) at t^(n+1) and info (picard_res: the last nonlinear residual)."""
        phi = self._dev(phi, self.n_phi, torch.float64, "phi").clone()
        u = self._dev(u, 3 * self.n_u, torch.float64, "u").clone()
        p = self._dev(p, self.n_p, torch.float64, "p").clone()
        mdot = self._dev(mdot, self.n_phi, torch.float64, "mdot")
        up = None if u_prev is None else self._dev(u_prev, 3 * self.n_u, torch.float64, "u_prev")
        g = None if gravity is None else (ctypes.c_double * 3)(*[float(v) for v in gravity])
        its, rel, nl = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        self.fields_version += 1  # the step leaves the mesh without fields
        rc = lib().evap_time_step(self._h, _ptr(phi), _ptr(u), _ptr(p), _ptr(mdot), _ptr(up), g, float(alpha),
                                  int(picard_iters), float(picard_atol), int(fp_iters), int(reinit_steps),
                                  float(ns_rtol),
                                  ctypes.byref(its), ctypes.byref(rel), ctypes.byref(nl), _stream())
        _check(rc, "evap_time_step", allow=() if raise_on_notconv else (-3,))
        return phi, u, p, dict(ns_iters=its.value, ns_relres=rel.value, picard_res=nl.value, converged=rc == 0)

    def set_checks(self, on: bool = True):
        """Count NaN / Inf entries of every later call's inputs first (EVAP_ENONFINITE if any)."""
        _check(lib().evap_set_checks(self._h, int(bool(on))), "evap_set_checks")

    def set_deterministic(self, on: bool = True):
        """Cells accumulated in 8 parity-class passes without atomics: bitwise reproducible applies and solves."""
        _check(lib().evap_set_deterministic(self._h, int(bool(on))), "evap_set_deterministic")

    def apply_saddle(self, x: torch.Tensor, p: torch.Tensor):
        """(A x - B^T p, B x): the velocity-pressure operator of Eq. (weakNavierStokes) with the Q1 pressure."""
        x = self._dev(x, 3 * self.n_u, torch.float64, "x")
        p = self._dev(p, self.n_p, torch.float64, "p")
        y = torch.empty(3 * self.n_u, dtype=torch.float64, device=self.device)
        yp = torch.empty(self.n_p, dtype=torch.float64, device=self.device)
        _check(lib().evap_apply_saddle(self._h, _ptr(x), _ptr(p), _ptr(y), _ptr(yp), _stream()), "evap_apply_saddle")
        return y, yp

    def apply_schur(self, x: torch.Tensor):
        """S~ x, S~ = B diag(A)^-1 B^T assembled on the pressure lattice (the velocity-pressure preconditioner's Schur
        approximation), in FP32 arithmetic."""
        x = self._dev(x, self.n_p, torch.float64, "x")
        y = torch.empty(self.n_p, dtype=torch.float64, device=self.device)
        _check(lib().evap_apply_schur(self._h, _ptr(x), _ptr(y), _stream()), "evap_apply_schur")
        return y

    def solve_saddle(self, f: torch.Tensor, x0=None, p0=None, restart: int = 30, rtol: float = 1e-8,
                     max_iter: int = 600, raise_on_notconv: bool = False):
        """Solve [A, -B^T; B, 0] [x; p] = [f; g] (g from the fields' dilation rate); returns (x, p, info)."""
        f = self._dev(f, 3 * self.n_u, torch.float64, "f")
        x = (torch.zeros(3 * self.n_u, dtype=torch.float64, device=self.device) if x0 is None
             else self._dev(x0, 3 * self.n_u, torch.float64, "x0").clone())
        p = (torch.zeros(self.n_p, dtype=torch.float64, device=self.device) if p0 is None
             else self._dev(p0, self.n_p, torch.float64, "p0").clone())
        its, rel = ctypes.c_int(), ctypes.c_double()
        rc = lib().evap_solve_saddle(self._h, _ptr(f), _ptr(x), _ptr(p), int(restart), float(rtol), int(max_iter),
                                     ctypes.byref(its), ctypes.byref(rel), _stream())
        _check(rc, "evap_solve_saddle", allow=() if raise_on_notconv else (-3,))
        return x, p, dict(iters=its.value, relres=rel.value, converged=rc == 0)

    def surface_tension(self, n: torch.Tensor, kappa: torch.Tensor, alpha: float, out=None):
        """Surface-tension force [3 N_u] (Eq. surfaceTension, density-scaled delta) from Q1 normal and curvature."""
        n = self._dev(n, 3 * self.n_phi, torch.float64, "n")
        kappa = self._dev(kappa, self.n_phi, torch.float64, "kappa")
        f = self._out(out, 3 * self.n_u, torch.float64)
        _check(lib().evap_surface_tension(self._h, _ptr(n), _ptr(kappa), float(alpha), _ptr(f), _stream()),
               "evap_surface_tension")
        return f

    def apply_momentum(self, x: torch.Tensor, prec: int = 64, with_divergence: bool = False, out=None, out_p=None):
        dt = torch.float64 if prec == 64 else torch.float32
        x = self._dev(x, 3 * self.n_u, dt, "x")
        y = self._out(out, 3 * self.n_u, dt)
        yp = self._out(out_p, self.n_p, dt) if with_divergence else None
        _check(lib().evap_apply_momentum(self._h, prec, _ptr(x), _ptr(y), _ptr(yp), _stream()), "evap_apply_momentum")
        return (y, yp) if with_divergence else y

    def apply_levelset(self, x: torch.Tensor, mode: str = "advect", prec: int = 64, out=None):
        dt = torch.float64 if prec == 64 else torch.float32
        x = self._dev(x, self.n_phi, dt, "x")
        y = self._out(out, self.n_phi, dt)
        _check(lib().evap_apply_levelset(self._h, LEVELSET_MODES[mode], prec, _ptr(x), _ptr(y), _stream()),
               "evap_apply_levelset")
        return y

    def apply_adjoint(self, w: torch.Tensor, x: torch.Tensor, w_p: torch.Tensor | None = None,
                      need=("x", "u0", "phi", "mdot")):
        w = self._dev(w, 3 * self.n_u, torch.float64, "w")
        x = self._dev(x, 3 * self.n_u, torch.float64, "x")
        wp = None if w_p is None else self._dev(w_p, self.n_p, torch.float64, "w_p")
        f64 = dict(dtype=torch.float64, device=self.device)
        out = {k: None for k in ("x", "u0", "phi", "mdot")}
        if "x" in need:
            out["x"] = torch.empty(3 * self.n_u, **f64)
        if "u0" in need:
            out["u0"] = torch.empty(3 * self.n_u, **f64)
        if "phi" in need:
            out["phi"] = torch.empty(self.n_phi, **f64)
        if "mdot" in need:
            out["mdot"] = torch.empty(self.n_phi, **f64)
        _check(lib().evap_apply_adjoint(self._h, _ptr(w), _ptr(wp), _ptr(x), _ptr(out["x"]), _ptr(out["u0"]),
                                        _ptr(out["phi"]), _ptr(out["mdot"]), _stream()), "evap_apply_adjoint")
        return out

    def jacobi_diagonal(self):
        d = torch.empty(3 * self.n_u, dtype=torch.float64, device=self.device)
        _check(lib().evap_jacobi_diagonal(self._h, _ptr(d), _stream()), "evap_jacobi_diagonal")
        return d

    def solve(self, f: torch.Tensor, x0: torch.Tensor | None = None, mixed: bool = True, restart: int = 16,
              rtol: float = 1e-10, max_iter: int = 5000, raise_on_notconv: bool = False):
        f = self._dev(f, 3 * self.n_u, torch.float64, "f")
        x = torch.zeros_like(f) if x0 is None else self._dev(x0, 3 * self.n_u, torch.float64, "x0").clone()
        its, rel = ctypes.c_int(), ctypes.c_double()
        rc = lib().evap_solve(self._h, _ptr(f), _ptr(x), int(bool(mixed)), restart, rtol, max_iter, ctypes.byref(its),
                              ctypes.byref(rel), _stream())
        _check(rc, "evap_solve", allow=() if raise_on_notconv else (-3,))
        return x, dict(iters=its.value, relres=rel.value, converged=rc == 0)


class MomentumFunction(torch.autograd.Function):
    """(y, y_p) = (A(phi, u0) x, B x - g(phi, mdot)) with gradients from the adjoint kernel.

    forward(op, x, phi, u0, mdot) sets the operator's fields, applies the FP64 momentum operator with the
    divergence row; backward calls evap_apply_adjoint with (w, w_p) = (grad_y, grad_y_p) at the fields of its own
    forward: if the operator's fields were replaced since (another forward or set_fields), backward sets the saved
    ones again first."""

    @staticmethod
    def forward(ctx, op: Operator, x, phi, u0, mdot):
        op.set_fields(phi.detach(), u0.detach(), mdot.detach())
        y, yp = op.apply_momentum(x.detach(), prec=64, with_divergence=True)
        ctx.op = op
        ctx.version = op.fields_version
        ctx.save_for_backward(x, phi, u0, mdot)
        return y, yp

    @staticmethod
    def backward(ctx, gy, gyp):
        x, phi, u0, mdot = ctx.saved_tensors
        op = ctx.op
        if op.fields_version != ctx.version:  # linearize about this forward's fields, not the latest ones
            op.set_fields(phi.detach(), u0.detach(), mdot.detach())
            ctx.version = op.fields_version
        gy = torch.zeros(3 * op.n_u, dtype=torch.float64, device=op.device) if gy is None else gy.contiguous()
        gyp = None if gyp is None else gyp.contiguous()
        g = op.apply_adjoint(gy, x.detach(), gyp)
        return None, g["x"], g["phi"], g["u0"], g["mdot"]
