// One time step of the coupled problem: the Navier-Stokes step, then Algorithm 2 (level-set solver).
//   1. velocity-pressure solve with Picard iterations (mesh newton = 0) or Newton's method (newton = 1: each
//      iteration solves J(u^(k)) [du; dp] = R^(k), the residual R of the Picard operator below, the Jacobian J the
//      operator with the Newton term, App. D): BDF1 (c_m = 1/dt, u* = u^n) or, given u^(n-1),
//      BDF2 (c_m = 3/(2 dt), u* = (4 u^n - u^(n-1)) / 3); iteration k solves
//        [A(u^(k)), -B^T; B, 0] [u^(k+1); p^(k+1)] = [f; g],  f = sum_q W N_i rho (c_m u* + g_body),  u^(0) = u^n,
//      with the Dirichlet data of u^n (f = u^n on the Dirichlet DoFs, lifted by the solve),
//      at most picard_iters times, stopping before a solve once |[f; g] - K(u^(k)) [u^(k); p^(k)]| <= picard_atol;
//      with alpha != 0 f also carries the surface-tension force (Eq. surfaceTension) of the projected normal and
//      regularized curvature of phi^n
//   2. advection fixed point with the transport velocity of u^(n+1) (Algorithm 2 step 1), the result clamped to
//      [-1, 1]; its projected normal (Eq. normal_vector_regularized); reinitialization steps with that normal frozen
//      (Algorithm 2 step 2), starting from the clamped field.
// Host orchestration of the library's kernels and solvers; every arithmetic step runs on the device.
#include "physics.cuh"

namespace evap {

__global__ void k_clamp_copy(const double* __restrict__ a, double* __restrict__ b, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = a[i];
        b[i] = v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v);
    }
}

// u* = (4 u - u_prev) / 3
__global__ void k_bdf2_star(const double* __restrict__ u, const double* __restrict__ up, double* __restrict__ us,
                            int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        us[i] = (4.0 * u[i] - up[i]) / 3.0;
}

// y += x
__global__ void k_axpy1(double* __restrict__ y, const double* __restrict__ x, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

// r = [f; g] - r (the residual of the nonlinear system from its operator part in r)
__global__ void k_residual_split(const double* __restrict__ f, const double* __restrict__ g, double* __restrict__ r,
                                 int64_t Nu3, int64_t Np) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nu3 + Np; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = (i < Nu3 ? f[i] : g[i - Nu3]) - r[i];
}

// *out += sum_i (b_i - a_i)^2, or sum_i b_i^2 with only_b (one atomic per block)
__global__ void __launch_bounds__(256) k_diff_sq(const double* __restrict__ a, const double* __restrict__ b,
                                                 int64_t N, double* out, bool only_b = false) {
    __shared__ double sh[8];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = only_b ? b[i] : b[i] - a[i];
        s += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        atomicAdd(out, t);
    }
}

// The mesh's mass coefficient set to the scheme's, and its Newton flag cleared (the residual's Picard operator), for
// the duration of a step.
struct StepCoefficients {
    evap_mesh* h;
    double saved_cm;
    int saved_newton;
    StepCoefficients(evap_mesh* hh, double cm) : h(hh), saved_cm(hh->m.c_mass), saved_newton(hh->m.newton) {
        h->m.c_mass = cm;
        h->m.newton = 0;
    }
    ~StepCoefficients() {
        h->m.c_mass = saved_cm;
        h->m.newton = saved_newton;
    }
};

// The quadrature-point coefficients of the current fields with the Newton term on or off (the material-law table and
// the continuity right-hand side do not depend on it); the Jacobi diagonal and its preconditioner follow them.
static int qp_coeffs_newton(evap_mesh* h, int newton, cudaStream_t s) {
    h->m.newton = newton;
    int rc = launch_qp_coeffs(h, s);
    h->diag_valid = false;
    h->tp_valid = false;
    h->tp64_valid = false;
    return rc;
}

// x += d (velocity and pressure parts)
__global__ void k_add2(double* __restrict__ u, const double* __restrict__ du, int64_t Nu3, double* __restrict__ p,
                       const double* __restrict__ dp, int64_t Np) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nu3 + Np; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < Nu3)
            u[i] += du[i];
        else
            p[i - Nu3] += dp[i - Nu3];
    }
}

int time_step(evap_mesh* h, double* phi, double* u, double* p, const double* mdot, const double* u_prev,
              const double g[3], double alpha, int picard_iters, double picard_atol, int fp_iters, int reinit_steps,
              double ns_rtol, int* ns_iters, double* ns_relres, double* picard_res, cudaStream_t s) {
    const int64_t Nu3 = 3 * h->m.Nu, Np = h->m.Np, Nl = h->m.Nphi;  // pressure, level-set nodes
    const bool newton = h->m.newton != 0;
    // workspace: f, u* [3 N_u]; residual [3 N_u + N_p]; Newton correction [3 N_u + N_p]; advected level set
    // [N_phi]; normal [3 N_phi]; scalar
    if (!h->step_ws) {
        EVAP_CUDA(cudaMalloc(&h->step_ws, (4 * Nu3 + 2 * Np + 4 * Nl + 1) * sizeof(double)));
    }
    double* f = h->step_ws;
    double* ustar = f + Nu3;
    double* res = ustar + Nu3;
    double* corr = res + Nu3 + Np;
    double* adv = corr + Nu3 + Np;
    double* nrm = adv + Nl;
    double* sq = nrm + 3 * Nl;
    StepCoefficients cm(h, (u_prev ? 1.5 : 1.0) / h->m.dt);
    int rc = set_fields_flow(h, phi, u, mdot, s);  // the advection computes its own transport velocities
    if (rc) return rc;
    int status = EVAP_OK;
    // 1. Navier-Stokes: the inertia load of u* (plus the body force), then Picard iterations from (u^n, p^n)
    const double* us = u;
    if (u_prev) {
        k_bdf2_star<<<blocks_for(Nu3, 256), 256, 0, s>>>(u, u_prev, ustar, Nu3);
        EVAP_CHECK_LAUNCH("bdf2_star");
        us = ustar;
    }
    if ((rc = launch_mass_load(h, us, g, f, s))) return rc;
    if (alpha != 0.0) {  // surface tension of phi^n: projected normal (nrm), curvature (adv), force (res)
        rc = geo_projected_normal(h, nrm, nullptr, nullptr, s);
        if (rc == EVAP_ENOTCONV) status = rc;
        else if (rc) return rc;
        rc = geo_curvature(h, nrm, adv, nullptr, nullptr, s);
        if (rc == EVAP_ENOTCONV) status = rc;
        else if (rc) return rc;
        if ((rc = launch_surface_tension(h, nrm, adv, alpha, res, s))) return rc;
        k_axpy1<<<blocks_for(Nu3, 256), 256, 0, s>>>(f, res, Nu3);
        EVAP_CHECK_LAUNCH("step_add_surface");
    }
    // Dirichlet data: the velocity on the Dirichlet faces keeps its value of u^n (walls at rest, or an inflow)
    if ((rc = launch_constrained_copy(h, u, f, s))) return rc;
    int applies = 0;
    double relres = 0.0, nl = -1.0;
    for (int it = 0; it < picard_iters; ++it) {
        if (it > 0 || newton) {  // the nonlinear residual R = [f; g] - K_D(u^(k)) [u^(k); p^(k)] (Picard operator)
            if (it > 0 && (rc = set_fields_flow(h, h->phi, u, h->mdot, s))) return rc;  // relinearize
            const double* gc = nullptr;
            if ((rc = continuity_rhs(h, &gc, s))) return rc;
            if ((rc = launch_saddle_apply(h, u, p, res, res + Nu3, s, true))) return rc;  // K_D (lifted data)
            k_residual_split<<<blocks_for(Nu3 + Np, 256), 256, 0, s>>>(f, gc, res, Nu3, Np);
            EVAP_CHECK_LAUNCH("nonlinear_residual");
            if (it > 0) {
                EVAP_CUDA(cudaMemsetAsync(sq, 0, sizeof(double), s));
                k_diff_sq<<<blocks_for(Nu3 + Np, 256, 152 * 8), 256, 0, s>>>(corr, res, Nu3 + Np, sq, true);
                EVAP_CHECK_LAUNCH("nonlinear_residual_norm");
                double hs = 0.0;
                EVAP_CUDA(cudaMemcpyAsync(&hs, sq, sizeof(double), cudaMemcpyDeviceToHost, s));
                EVAP_CUDA(cudaStreamSynchronize(s));
                nl = std::sqrt(hs);
                if (nl <= picard_atol) break;
            }
        }
        int its = 0;
        if (newton) {
            // J(u^(k)) [du; dp] = R with the Jacobian: the operator with the Newton term (App. D); the correction
            // has zero Dirichlet data (u^(k) carries the boundary values, R vanishes on the Dirichlet rows)
            if ((rc = qp_coeffs_newton(h, 1, s))) return rc;
            EVAP_CUDA(cudaMemsetAsync(corr, 0, (Nu3 + Np) * sizeof(double), s));
            rc = solve_saddle(h, res, corr, corr + Nu3, 30, ns_rtol, 2000, &its, &relres, s, res + Nu3);
            int rc2 = qp_coeffs_newton(h, 0, s);
            if (rc2) return rc2;
            k_add2<<<blocks_for(Nu3 + Np, 256), 256, 0, s>>>(u, corr, Nu3, p, corr + Nu3, Np);
            EVAP_CHECK_LAUNCH("newton_update");
        } else {
            rc = solve_saddle(h, f, u, p, 30, ns_rtol, 2000, &its, &relres, s);
        }
        applies += its;
        if (rc == EVAP_ENOTCONV) status = rc;
        else if (rc) return rc;
    }
    if (ns_iters) *ns_iters = applies;
    if (ns_relres) *ns_relres = relres;
    if (picard_res) *picard_res = nl;
    // 2. level set with the transport velocity of u^(n+1)
    EVAP_CUDA(cudaMemcpyAsync(h->u, u, Nu3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rc = geo_advect_levelset(h, adv, fp_iters, 0.0, nullptr, nullptr, nullptr, s);
    if (rc == EVAP_ENOTCONV) status = rc;
    else if (rc) return rc;
    k_clamp_copy<<<blocks_for(Nl, 256, 152 * 8), 256, 0, s>>>(adv, h->phi, Nl);
    EVAP_CHECK_LAUNCH("step_clamp");
    rc = geo_projected_normal(h, nrm, nullptr, nullptr, s);
    if (rc == EVAP_ENOTCONV) status = rc;
    else if (rc) return rc;
    if ((rc = evap_set_levelset_normal(h, nrm, s))) return rc;
    EVAP_CUDA(cudaMemcpyAsync(phi, h->phi, Nl * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rc = geo_reinitialize(h, phi, reinit_steps, nullptr, nullptr, s);
    if (rc == EVAP_ENOTCONV) status = rc;
    else if (rc) return rc;
    if ((rc = evap_set_levelset_normal(h, nullptr, s))) return rc;
    // the mesh's level set, velocity and their derived coefficients no longer belong together
    h->has_fields = false;
    EVAP_CUDA(cudaStreamSynchronize(s));
    return status;
}

}  // namespace evap
