// One time step of the coupled problem: the Navier-Stokes step, then Algorithm 2 (level-set solver).
//   1. velocity-pressure solve, BDF1 with one Picard linearization about u^n (newton = 0, c_m = 1/dt):
//        [A(u^n), -B^T; B, 0] [u^(n+1); p^(n+1)] = [f; g],  f = sum_q W N_i rho (u^n / dt + g_body)
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

int time_step(evap_mesh* h, double* phi, double* u, double* p, const double* mdot, const double g[3], int fp_iters,
              int reinit_steps, double ns_rtol, int* ns_iters, double* ns_relres, cudaStream_t s) {
    const int64_t Nu3 = 3 * h->m.Nu, Np = h->m.Nphi;
    if (!h->step_ws) {
        EVAP_CUDA(cudaMalloc(&h->step_ws, (Nu3 + 4 * Np) * sizeof(double)));
    }
    double* f = h->step_ws;
    double* adv = f + Nu3;
    double* nrm = adv + Np;
    int rc = evap_set_fields(h, phi, u, mdot, s);
    if (rc) return rc;
    int status = EVAP_OK;
    // 1. Navier-Stokes: the inertia load of u^n (plus the body force), then the saddle solve from (u^n, p^n)
    if ((rc = launch_mass_load(h, u, g, f, s))) return rc;
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
