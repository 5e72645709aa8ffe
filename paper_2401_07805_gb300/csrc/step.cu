// One time step of the coupled problem: the Navier-Stokes step, then Algorithm 2 (level-set solver).
//   1. velocity-pressure solve with one Picard linearization about u^n (newton = 0): BDF1 (c_m = 1/dt, u* = u^n) or,
//      given u^(n-1), BDF2 (c_m = 3/(2 dt), u* = (4 u^n - u^(n-1)) / 3):
//        [A(u^n), -B^T; B, 0] [u^(n+1); p^(n+1)] = [f; g],  f = sum_q W N_i rho (c_m u* + g_body)
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

// The mesh's mass coefficient set to the scheme's for the duration of a step.
struct MassCoefficient {
    evap_mesh* h;
    double saved;
    MassCoefficient(evap_mesh* hh, double cm) : h(hh), saved(hh->m.c_mass) { h->m.c_mass = cm; }
    ~MassCoefficient() { h->m.c_mass = saved; }
};

int time_step(evap_mesh* h, double* phi, double* u, double* p, const double* mdot, const double* u_prev,
              const double g[3], int fp_iters, int reinit_steps, double ns_rtol, int* ns_iters, double* ns_relres,
              cudaStream_t s) {
    const int64_t Nu3 = 3 * h->m.Nu, Np = h->m.Nphi;
    if (!h->step_ws) {
        EVAP_CUDA(cudaMalloc(&h->step_ws, (2 * Nu3 + 4 * Np) * sizeof(double)));
    }
    double* f = h->step_ws;
    double* ustar = f + Nu3;
    double* adv = ustar + Nu3;
    double* nrm = adv + Np;
    MassCoefficient cm(h, (u_prev ? 1.5 : 1.0) / h->m.dt);
    int rc = evap_set_fields(h, phi, u, mdot, s);
    if (rc) return rc;
    int status = EVAP_OK;
    // 1. Navier-Stokes: the inertia load of u* (plus the body force), then the saddle solve from (u^n, p^n)
    const double* us = u;
    if (u_prev) {
        k_bdf2_star<<<blocks_for(Nu3, 256), 256, 0, s>>>(u, u_prev, ustar, Nu3);
        EVAP_CHECK_LAUNCH("bdf2_star");
        us = ustar;
    }
    if ((rc = launch_mass_load(h, us, g, f, s))) return rc;
    rc = solve_saddle(h, f, u, p, 30, ns_rtol, 2000, ns_iters, ns_relres, s);
    if (rc == EVAP_ENOTCONV) status = rc;
    else if (rc) return rc;
    // 2. level set with the transport velocity of u^(n+1)
    EVAP_CUDA(cudaMemcpyAsync(h->u, u, Nu3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rc = geo_advect_levelset(h, adv, fp_iters, 0.0, nullptr, nullptr, nullptr, s);
    if (rc == EVAP_ENOTCONV) status = rc;
    else if (rc) return rc;
    k_clamp_copy<<<blocks_for(Np, 256, 152 * 8), 256, 0, s>>>(adv, h->phi, Np);
    EVAP_CHECK_LAUNCH("step_clamp");
    rc = geo_projected_normal(h, nrm, nullptr, nullptr, s);
    if (rc == EVAP_ENOTCONV) status = rc;
    else if (rc) return rc;
    if ((rc = evap_set_levelset_normal(h, nrm, s))) return rc;
    EVAP_CUDA(cudaMemcpyAsync(phi, h->phi, Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
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
