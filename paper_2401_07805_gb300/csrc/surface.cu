// Surface-tension force of Eq. (surfaceTension) as the right-hand side of the momentum equation, FP64:
//   b_(i,c) = sum_q W_q N_i(x_q) alpha kappa_h(x_q) n_c(x_q) delta(x_q) rho(x_q) c_rho,
//   c_rho = (rho_g - rho_l) / (rho_l rho_g ln(rho_g / rho_l))  (the density-scaled delta, same section),
// kappa_h and n_h the caller's Q1 curvature and normal fields on the level-set mesh (normalized at the point:
// n_h / |n_h|, zero where |n_h| <= 1e-4), delta (Eq. delta) and the reciprocal rho (Eq. rhoEff) from the level set at
// the point.  One thread
// per velocity quadrature point; the test with the Q_p shape functions runs as three transposed 1D sweeps
// (z, y, x) through shared memory.  Dirichlet-constrained entries stay zero.
#include <cmath>

#include "physics.cuh"

namespace evap {

template <int P, int CB>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1))
    k_surface_tension(MeshArgs<double> m, Basis<double> bas, const double* __restrict__ phi,
                      const double* __restrict__ nf, const double* __restrict__ kappa, double alpha_crho,
                      double* __restrict__ out) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    __shared__ double sS[Q][Q];
    __shared__ double buf[2][CB][3][NQ];
    const int tid = threadIdx.x;
    const int lc = tid / NQ, t = tid % NQ;
    const int64_t cell = (int64_t)blockIdx.x * CB + lc;
    const bool active = cell < m.ncell;
    if (tid < Q * Q) sS[tid / Q][tid % Q] = bas.S[tid / Q][tid % Q];
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    const int n = m.n;
    int cx = 0, cy = 0, cz = 0;
    if (active) {
        cx = (int)(cell % n);
        cy = (int)((cell / n) % n);
        cz = (int)(cell / ((int64_t)n * n));
        // level-set-space fields at the point (the Q1 interpolant of the level-set cell containing it)
        const double tx = bas.t[a], ty = bas.t[b], tz = bas.t[c];
        double ph, gp[3], kq, nh[3], gdum[3];
        ls_at(phi, m, cx, cy, cz, tx, ty, tz, ph, gp);
        ls_at(kappa, m, cx, cy, cz, tx, ty, tz, kq, gdum);
#pragma unroll
        for (int d = 0; d < 3; ++d) ls_at(nf + d * m.Nphi, m, cx, cy, cz, tx, ty, tz, nh[d], gdum);
        const Material mat = material(ph, gp[0], gp[1], gp[2], m);
        const double W = bas.w[a] * bas.w[b] * bas.w[c] * m.vol_w;
        const double nn = sqrt(nh[0] * nh[0] + nh[1] * nh[1] + nh[2] * nh[2]);
        const double s = nn > NODAL_NORMAL_TINY ? W * alpha_crho * kq * mat.delta * mat.rho / nn : 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) buf[0][lc][d][t] = s * nh[d];
    }
    __syncthreads();
    // test with N_i = l_a(x) l_b(y) l_c(z): transposed sweeps z, y, x
    if (active)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            double v = 0.0;
#pragma unroll
            for (int q = 0; q < Q; ++q) v += sS[q][c] * buf[0][lc][f][a + Q * (b + Q * q)];
            buf[1][lc][f][t] = v;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            double v = 0.0;
#pragma unroll
            for (int q = 0; q < Q; ++q) v += sS[q][b] * buf[1][lc][f][a + Q * (q + Q * c)];
            buf[0][lc][f][t] = v;
        }
    __syncthreads();
    if (!active) return;
    const int M = m.M;
    const int gx = P * cx + a, gy = P * cy + b, gz = P * cz + c;
    const unsigned fc = m.faces;
    const bool cons = ((fc & 1u) && gx == 0) || ((fc & 2u) && gx == M - 1) || ((fc & 4u) && gy == 0) ||
                      ((fc & 8u) && gy == M - 1) || ((fc & 16u) && gz == 0) || ((fc & 32u) && gz == M - 1);
    if (cons) return;
    const int64_t gidx = gx + (int64_t)M * (gy + (int64_t)M * gz);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < Q; ++q) v += sS[q][a] * buf[0][lc][f][q + Q * (b + Q * c)];
        atomicAdd(&out[f * m.Nu + gidx], v);
    }
}

int launch_surface_tension(evap_mesh* h, const double* nf, const double* kappa, double alpha, double* out,
                           cudaStream_t s) {
    const MeshArgs<double>& m = h->m;
    const double rl = m.rho_l, rg = m.rho_g;
    const double crho = (rg - rl) / (rl * rg * std::log(rg / rl));
    EVAP_CUDA(cudaMemsetAsync(out, 0, 3 * m.Nu * sizeof(double), s));
    if (m.P == 2) {
        constexpr int CB = 8;
        k_surface_tension<2, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 27, 0, s>>>(m, h->b, h->phi, nf, kappa,
                                                                                        alpha * crho, out);
    } else {
        constexpr int CB = 4;
        k_surface_tension<3, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 64, 0, s>>>(m, h->b, h->phi, nf, kappa,
                                                                                        alpha * crho, out);
    }
    EVAP_CHECK_LAUNCH("surface_tension");
    return EVAP_OK;
}

}  // namespace evap
