// Velocity-pressure coupling of Eq. (weakNavierStokes) with the Q1 pressure of Sec. 2.5 (k_p = 1), FP64:
//   pressure term of the momentum row   y_(c,i) += s sum_q W p_h(x_q) d_c N_i(x_q)      (s = -1: -(div v, p); the
//                                       saddle-point apply folds it into the momentum kernel's stress flux)
//   continuity right-hand side         g_j = sum_q W N1_j v_dil                           (Eq. continuity, evaporDil)
//   saddle-point apply                 [y; y_p] = [A x - B^T p; B x]
// with B the divergence row of the momentum apply (velocity Gauss rule, Dirichlet entries of x read as 0) and
// Dirichlet-constrained velocity rows left to the momentum apply (identity), so B^T p vanishes there.
#include "physics.cuh"

namespace evap {

// B^T p, scaled by s, added to y: one thread per velocity quadrature point, CB cells per block.  The pressure is
// interpolated at the point from the cell's 8 Q1 nodes; the test with d_c N_i is the transpose of the momentum
// apply's gradient (collocation derivative at the Gauss points along c, then S^T along z, y, x), so B^T here is
// the exact transpose of the divergence row.
template <typename T, int P, int CB>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1))
    k_pressure_gradient(MeshArgs<T> m, Basis<T> bas, const T* __restrict__ p, T s, T* __restrict__ y) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    __shared__ T sS[Q][Q], sDc[Q][Q], sN1[Q][2];
    __shared__ T val[CB][NQ];
    __shared__ T buf[2][CB][3][NQ];
    const int tid = threadIdx.x;
    const int lc = tid / NQ, t = tid % NQ;
    const int64_t cell = (int64_t)blockIdx.x * CB + lc;
    const bool active = cell < m.ncell;
    if (tid < Q * Q) {
        sS[tid / Q][tid % Q] = bas.S[tid / Q][tid % Q];
        sDc[tid / Q][tid % Q] = bas.Dc[tid / Q][tid % Q] * m.inv_h;
    }
    if (tid < 2 * Q) sN1[tid / 2][tid % 2] = bas.N1[tid / 2][tid % 2];
    __syncthreads();
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    const int n = m.n;
    int cx = 0, cy = 0, cz = 0;
    if (active) {
        cx = (int)(cell % n);
        cy = (int)((cell / n) % n);
        cz = (int)(cell / ((int64_t)n * n));
        const int64_t m1 = n + 1;
        T pq = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int ja = j & 1, jb = (j >> 1) & 1, jc = j >> 2;
            pq += sN1[a][ja] * sN1[b][jb] * sN1[c][jc] * p[(cx + ja) + m1 * ((cy + jb) + m1 * (cz + jc))];
        }
        val[lc][t] = s * bas.w[a] * bas.w[b] * bas.w[c] * m.vol_w * pq;
    }
    __syncthreads();
    if (active) {
        T d0 = 0, d1 = 0, d2 = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            d0 += sDc[r][a] * val[lc][r + Q * (b + Q * c)];
            d1 += sDc[r][b] * val[lc][a + Q * (r + Q * c)];
            d2 += sDc[r][c] * val[lc][a + Q * (b + Q * r)];
        }
        buf[0][lc][0][t] = d0;
        buf[0][lc][1][t] = d1;
        buf[0][lc][2][t] = d2;
    }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T v = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) v += sS[q][c] * buf[0][lc][f][a + Q * (b + Q * q)];
            buf[1][lc][f][t] = v;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T v = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) v += sS[q][b] * buf[1][lc][f][a + Q * (q + Q * c)];
            buf[0][lc][f][t] = v;
        }
    __syncthreads();
    if (!active) return;
    const int M = m.M;
    const int gx = P * cx + a, gy = P * cy + b, gz = P * cz + c;
    if (constrained_node(gx, gy, gz, M, m.faces)) return;
    const int64_t gidx = gx + (int64_t)M * (gy + (int64_t)M * gz);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        T v = 0;
#pragma unroll
        for (int q = 0; q < Q; ++q) v += sS[q][a] * buf[0][lc][f][q + Q * (b + Q * c)];
        atomicAdd(&y[f * m.Nu + gidx], v);
    }
}

// g_j += sum_q N1_j(x_q) (W v_dil)_q over the cell's velocity Gauss points, from the cached coefficient slot 18.
template <int P>
__global__ void __launch_bounds__(128) k_continuity_rhs(MeshArgs<double> m, Basis<double> bas,
                                                        const double* __restrict__ qc, double* __restrict__ g) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= m.ncell) return;
    const int n = m.n;
    const int cx = (int)(cell % n), cy = (int)((cell / n) % n), cz = (int)(cell / ((int64_t)n * n));
    const double* v = qc + cell * QC_K * NQ + 18 * NQ;
    double out[8] = {};
    for (int t = 0; t < NQ; ++t) {
        const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
        const double vt = v[t];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            out[j] += bas.N1[a][j & 1] * bas.N1[b][(j >> 1) & 1] * bas.N1[c][j >> 2] * vt;
    }
    const int64_t m1 = n + 1;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        atomicAdd(&g[(cx + (j & 1)) + m1 * ((cy + ((j >> 1) & 1)) + m1 * (cz + (j >> 2)))], out[j]);
}

// y_p += B D^(-1) x (D = diag when given, else the identity): the divergence row of the momentum apply without its
// source, sum_q W N1_j (div x)(x_q); values at the points by S sweeps (x, y, z), the divergence by the collocation
// derivative, the Q1 test by three sweeps of N1.
template <typename T, int P, int CB>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1))
    k_divergence(MeshArgs<T> m, Basis<T> bas, const T* __restrict__ x, const T* __restrict__ diag,
                 T* __restrict__ yp) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    __shared__ T sS[Q][Q], sDc[Q][Q], sN1[Q][2];
    __shared__ T buf[2][3][CB][NQ];
    __shared__ T rbuf[CB][NQ], q1a[CB][2 * Q * Q], q1b[CB][4 * Q];
    const int tid = threadIdx.x;
    const int lc = tid / NQ, t = tid % NQ;
    const int64_t cell = (int64_t)blockIdx.x * CB + lc;
    const bool active = cell < m.ncell;
    if (tid < Q * Q) {
        sS[tid / Q][tid % Q] = bas.S[tid / Q][tid % Q];
        sDc[tid / Q][tid % Q] = bas.Dc[tid / Q][tid % Q] * m.inv_h;
    }
    if (tid < 2 * Q) sN1[tid / 2][tid % 2] = bas.N1[tid / 2][tid % 2];
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    const int n = m.n, M = m.M;
    int cx = 0, cy = 0, cz = 0;
    if (active) {
        cx = (int)(cell % n);
        cy = (int)((cell / n) % n);
        cz = (int)(cell / ((int64_t)n * n));
        const int gx = P * cx + a, gy = P * cy + b, gz = P * cz + c;
        const int64_t gidx = gx + (int64_t)M * (gy + (int64_t)M * gz);
        const bool cons = constrained_node(gx, gy, gz, M, m.faces);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int64_t i = k * m.Nu + gidx;
            buf[0][k][lc][t] = cons ? T(0) : (diag ? x[i] / diag[i] : x[i]);
        }
    }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T v = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) v += sS[a][k] * buf[0][f][lc][k + Q * (b + Q * c)];
            buf[1][f][lc][t] = v;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T v = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) v += sS[b][k] * buf[1][f][lc][a + Q * (k + Q * c)];
            buf[0][f][lc][t] = v;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T v = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) v += sS[c][k] * buf[0][f][lc][a + Q * (b + Q * k)];
            buf[1][f][lc][t] = v;
        }
    __syncthreads();
    if (active) {
        T tr = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r)
            tr += sDc[a][r] * buf[1][0][lc][r + Q * (b + Q * c)] + sDc[b][r] * buf[1][1][lc][a + Q * (r + Q * c)] +
                  sDc[c][r] * buf[1][2][lc][a + Q * (b + Q * r)];
        rbuf[lc][t] = bas.w[a] * bas.w[b] * bas.w[c] * m.vol_w * tr;
    }
    __syncthreads();
    if (active && t < 2 * Q * Q) {  // x-sweep: [jx][qy][qz]
        const int jx = t & 1, qy = (t >> 1) % Q, qz = (t >> 1) / Q;
        T v = 0;
#pragma unroll
        for (int q = 0; q < Q; ++q) v += sN1[q][jx] * rbuf[lc][q + Q * (qy + Q * qz)];
        q1a[lc][t] = v;
    }
    __syncthreads();
    if (active && t < 4 * Q) {  // y-sweep: [jx][jy][qz]
        const int jx = t & 1, jy = (t >> 1) & 1, qz = t >> 2;
        T v = 0;
#pragma unroll
        for (int q = 0; q < Q; ++q) v += sN1[q][jy] * q1a[lc][jx + 2 * (q + Q * qz)];
        q1b[lc][t] = v;
    }
    __syncthreads();
    if (active && t < 8) {  // z-sweep: Q1 node (jx, jy, jz)
        const int jx = t & 1, jy = (t >> 1) & 1, jz = t >> 2;
        T v = 0;
#pragma unroll
        for (int q = 0; q < Q; ++q) v += sN1[q][jz] * q1b[lc][jx + 2 * (jy + 2 * q)];
        const int64_t m1 = n + 1;
        atomicAdd(&yp[(cx + jx) + m1 * ((cy + jy) + m1 * (cz + jz))], v);
    }
}

// f += sum_q W rho c_m N_i (u_c + g_c / c_m) at the velocity Gauss points (the BDF1 inertia load of the old velocity
// plus the body force), from the cached coefficient slot 0 (W rho c_m); Dirichlet entries of u are read as 0 and the
// constrained rows of f are left untouched (zero).
template <int P, int CB>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1))
    k_mass_load(MeshArgs<double> m, Basis<double> bas, const double* __restrict__ qc, const double* __restrict__ u,
                double g0, double g1, double g2, double* __restrict__ f) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    __shared__ double sS[Q][Q];
    __shared__ double buf[2][3][CB][NQ];
    const int tid = threadIdx.x;
    const int lc = tid / NQ, t = tid % NQ;
    const int64_t cell = (int64_t)blockIdx.x * CB + lc;
    const bool active = cell < m.ncell;
    if (tid < Q * Q) sS[tid / Q][tid % Q] = bas.S[tid / Q][tid % Q];
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    const int n = m.n, M = m.M;
    int64_t gidx = 0;
    bool cons = false;
    if (active) {
        const int cx = (int)(cell % n), cy = (int)((cell / n) % n), cz = (int)(cell / ((int64_t)n * n));
        const int gx = P * cx + a, gy = P * cy + b, gz = P * cz + c;
        gidx = gx + (int64_t)M * (gy + (int64_t)M * gz);
        cons = constrained_node(gx, gy, gz, M, m.faces);
#pragma unroll
        for (int k = 0; k < 3; ++k) buf[0][k][lc][t] = cons ? 0.0 : u[k * m.Nu + gidx];
    }
    __syncthreads();
    if (active)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double v = 0.0;
#pragma unroll
            for (int r = 0; r < Q; ++r) v += sS[a][r] * buf[0][k][lc][r + Q * (b + Q * c)];
            buf[1][k][lc][t] = v;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double v = 0.0;
#pragma unroll
            for (int r = 0; r < Q; ++r) v += sS[b][r] * buf[1][k][lc][a + Q * (r + Q * c)];
            buf[0][k][lc][t] = v;
        }
    __syncthreads();
    if (active) {
        const double cf0 = qc[cell * QC_K * NQ + t];  // W rho c_m
        const double gc[3] = {g0 / m.c_mass, g1 / m.c_mass, g2 / m.c_mass};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double v = 0.0;
#pragma unroll
            for (int r = 0; r < Q; ++r) v += sS[c][r] * buf[0][k][lc][a + Q * (b + Q * r)];
            buf[1][k][lc][t] = cf0 * (v + gc[k]);
        }
    }
    __syncthreads();
    // test with N_i: transposed sweeps z, y, x
    if (active)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double v = 0.0;
#pragma unroll
            for (int q = 0; q < Q; ++q) v += sS[q][c] * buf[1][k][lc][a + Q * (b + Q * q)];
            buf[0][k][lc][t] = v;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double v = 0.0;
#pragma unroll
            for (int q = 0; q < Q; ++q) v += sS[q][b] * buf[0][k][lc][a + Q * (q + Q * c)];
            buf[1][k][lc][t] = v;
        }
    __syncthreads();
    if (!active || cons) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < Q; ++q) v += sS[q][a] * buf[1][k][lc][q + Q * (b + Q * c)];
        atomicAdd(&f[k * m.Nu + gidx], v);
    }
}

int launch_mass_load(evap_mesh* h, const double* u, const double g[3], double* f, cudaStream_t st) {
    const MeshArgs<double>& m = h->m;
    EVAP_CUDA(cudaMemsetAsync(f, 0, 3 * m.Nu * sizeof(double), st));
    if (m.P == 2) {
        constexpr int CB = 8;
        k_mass_load<2, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 27, 0, st>>>(m, h->b, h->qc, u, g[0], g[1],
                                                                                   g[2], f);
    } else {
        constexpr int CB = 4;
        k_mass_load<3, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 64, 0, st>>>(m, h->b, h->qc, u, g[0], g[1],
                                                                                   g[2], f);
    }
    EVAP_CHECK_LAUNCH("mass_load");
    return EVAP_OK;
}

__global__ void k_add_vec(double* __restrict__ y, const double* __restrict__ g, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += g[i];
}

template <typename T>
int launch_pressure_gradient(evap_mesh* h, const T* p, T s, T* y, cudaStream_t st) {
    const MeshArgs<T> m = mesh_args<T>(h);
    const Basis<T> b = cast_basis<T>(h->b);
    if (m.P == 2) {
        constexpr int CB = 8;
        k_pressure_gradient<T, 2, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 27, 0, st>>>(m, b, p, s, y);
    } else {
        constexpr int CB = 4;
        k_pressure_gradient<T, 3, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 64, 0, st>>>(m, b, p, s, y);
    }
    EVAP_CHECK_LAUNCH("pressure_gradient");
    return EVAP_OK;
}
template int launch_pressure_gradient<float>(evap_mesh*, const float*, float, float*, cudaStream_t);

template <typename T>
int launch_divergence(evap_mesh* h, const T* x, const T* diag, T* yp, cudaStream_t st) {
    const MeshArgs<T> m = mesh_args<T>(h);
    const Basis<T> b = cast_basis<T>(h->b);
    if (m.P == 2) {
        constexpr int CB = 8;
        k_divergence<T, 2, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 27, 0, st>>>(m, b, x, diag, yp);
    } else {
        constexpr int CB = 4;
        k_divergence<T, 3, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 64, 0, st>>>(m, b, x, diag, yp);
    }
    EVAP_CHECK_LAUNCH("divergence");
    return EVAP_OK;
}
template int launch_divergence<float>(evap_mesh*, const float*, const float*, float*, cudaStream_t);

// z = S~^(-1) r, S~ = B diag(A)^(-1) B^T (a SIMPLE-type approximation of the Schur complement B A^(-1) B^T: it keeps
// the discrete B, so the pressure nodes of open faces are treated like every other node): at most cg_iters iterations
// of the FP32 single-launch CG on the assembled stencil (schur.cu), or |r| <= EVAP_SADDLE_SCHUR_RTOL |r0| (an inexact
// solve: the outer method is flexible).
#ifndef EVAP_SADDLE_SCHUR_RTOL
#define EVAP_SADDLE_SCHUR_RTOL 1e-6
#endif
int schur_apply(evap_mesh* h, const double* r, double* z, int cg_iters, cudaStream_t st) {
    return schur_solve(h, r, z, EVAP_SADDLE_SCHUR_RTOL, cg_iters, nullptr, st);
}

// g (the continuity right-hand side of the current fields), computed once per set_fields into h->cont_rhs.
int continuity_rhs(evap_mesh* h, const double** g, cudaStream_t st) {
    const MeshArgs<double>& m = h->m;
    if (!h->cont_rhs) EVAP_CUDA(cudaMalloc(&h->cont_rhs, m.Np * sizeof(double)));
    if (!h->cont_valid) {
        EVAP_CUDA(cudaMemsetAsync(h->cont_rhs, 0, m.Np * sizeof(double), st));
        const unsigned grid = (unsigned)blocks_for(m.ncell, 128, 1LL << 40);
        if (m.P == 2)
            k_continuity_rhs<2><<<grid, 128, 0, st>>>(m, h->b, h->qc, h->cont_rhs);
        else
            k_continuity_rhs<3><<<grid, 128, 0, st>>>(m, h->b, h->qc, h->cont_rhs);
        EVAP_CHECK_LAUNCH("continuity_rhs");
        h->cont_valid = true;
    }
    *g = h->cont_rhs;
    return EVAP_OK;
}

// [y; y_p] = [A x - B^T p; B x]: the momentum apply with the pressure term folded into its stress flux (whose
// divergence row is B x - g), followed by + g.
int launch_saddle_apply(evap_mesh* h, const double* x, const double* p, double* y, double* yp, cudaStream_t st,
                        bool lifted) {
    const double* g = nullptr;
    int rc = continuity_rhs(h, &g, st);
    if (rc) return rc;
    if ((rc = launch_momentum<double>(h, x, y, yp, st, true, p, lifted))) return rc;
    k_add_vec<<<blocks_for(h->m.Np, 256, 152 * 8), 256, 0, st>>>(yp, g, h->m.Np);
    EVAP_CHECK_LAUNCH("saddle_add_g");
    return EVAP_OK;
}

}  // namespace evap
