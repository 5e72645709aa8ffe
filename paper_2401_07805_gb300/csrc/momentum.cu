// Matrix-free momentum apply y = A x (velocity block of Eq. weakNavierStokes linearized about u0, App. D) with the
// divergence row y_p = B x - g (Eq. continuity with the dilation rate of Eq. evaporDil), by sum factorization.
//
// Per cell (Sec. 2.5: y = sum_i R_i^T A_i R_i x):
//   gather   x, u0 at the (P+1)^3 nodes (Dirichlet nodes of x read as 0)
//   values   3 sweeps of the 1D matrix S[q][a] = l_a(t_q) per component            -> x_c, u0_c at the Gauss points
//   grads    collocation derivative Dc at the Gauss points along each direction     -> d_b x_c, d_b u0_c
//   flux     F_c  = W rho (c_m x_c + u0 . grad x_c + newton (grad u0 x)_c)
//            T_cb = 2 W mu (eps_cb - tr(eps) (z n)_c (z n)_b),  eps = sym grad x          (Eq. modified_viscous_stress)
//            with the quadrature-point coefficients (W rho c_m, W rho u0, W rho grad u0, 2 W mu, z n, W, W v_dil)
//            evaluated once per set_fields in FP64 (k_qp_coeffs) and read per apply: on GB300 the FP64 pipe, not
//            HBM, bounds this operator, and re-interpolating u0 on every apply cost ~30 % of its FP64 work
//   test     w_c = F_c + sum_b Dc^T T_cb, then 3 transposed sweeps S^T            -> nodal contributions
//   scatter  atomic add into y (constrained rows hold y = x, written by the init kernel)
// Thread layout: one thread per quadrature point, CB cells per block; sweeps go through shared memory, each thread
// keeps its rows/columns of the 1D matrices in registers.
#include "physics.cuh"

namespace evap {

// y = x on Dirichlet DoFs, 0 elsewhere; y_p = 0.  Each warp walks whole x-lines (component c, gy, gz) of M nodes,
// so the line's position is split once per warp and the lanes only test their own gx.
template <typename T>
__global__ void __launch_bounds__(256) k_momentum_init(int M, int64_t Nu, unsigned faces, const T* __restrict__ x,
                                                       T* __restrict__ y, T* __restrict__ yp, int64_t Np) {
    const int lines = 3 * M * M;
    const int wpb = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int line = blockIdx.x * wpb + warp; line < lines; line += gridDim.x * wpb) {
        const int c = line / (M * M), rem = line - c * M * M, gz = rem / M, gy = rem - gz * M;
        const bool cyz = ((faces & 4u) && gy == 0) || ((faces & 8u) && gy == M - 1) || ((faces & 16u) && gz == 0) ||
                         ((faces & 32u) && gz == M - 1);
        const int64_t off = c * Nu + (int64_t)M * (gy + (int64_t)M * gz);
        for (int gx = lane; gx < M; gx += 32) {
            const bool cons = cyz || ((faces & 1u) && gx == 0) || ((faces & 2u) && gx == M - 1);
            y[off + gx] = cons ? x[off + gx] : T(0);
        }
    }
    if (yp) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Np; i += stride) yp[i] = T(0);
    }
}

// Quadrature-point coefficients of the FP64 momentum operator, evaluated once per set_fields from u0 and the
// material-law table (layout [cell][QC_K][nq]):
//   0: W rho c_m   1..3: W rho u0_b   4..12: newton W rho d_d u0_c (index 4 + 3c + d)   13: 2 W mu
//   14..16: z n_b (correction gate times normal)   17: W   18: W v_dil
// W = w_qx w_qy w_qz h^3.  One thread per quadrature point, CB cells per block (u0 interpolated by sum factorization).
// Slots 1..12 are also stored in FP32 for the FP32 apply (slots 1..3 divided by h: that kernel takes reference
// gradients), in its 32-cell block layout
// qc32[((blk * QC32_K + k) * NQ + pt) * 32 + lane], cell (32 xb + lane, row) in block blk = xb + ceil(n / 32) row.
template <int P, int CB>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1))
    k_qp_coeffs(MeshArgs<double> m, Basis<double> bas, const int8_t* __restrict__ code,
                const int32_t* __restrict__ tindex, const double* __restrict__ table, const double* __restrict__ u0,
                double* __restrict__ qc, float* __restrict__ qc32) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    __shared__ double sS[Q][Q], sDc[Q][Q];
    __shared__ double buf[2][CB][3][NQ];
    const int tid = threadIdx.x;
    const int lc = tid / NQ, t = tid % NQ;
    const int64_t cell = (int64_t)blockIdx.x * CB + lc;
    const bool active = cell < m.ncell;
    if (tid < Q * Q) {
        sS[tid / Q][tid % Q] = bas.S[tid / Q][tid % Q];
        sDc[tid / Q][tid % Q] = bas.Dc[tid / Q][tid % Q];
    }
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    const int n = m.n, M = m.M;
    if (active) {
        const int cx = (int)(cell % n), cy = (int)((cell / n) % n), cz = (int)(cell / ((int64_t)n * n));
        const int64_t gidx = (P * cx + a) + (int64_t)M * ((P * cy + b) + (int64_t)M * (P * cz + c));
#pragma unroll
        for (int k = 0; k < 3; ++k) buf[0][lc][k][t] = u0[k * m.Nu + gidx];
    }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            double s = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s += sS[a][k] * buf[0][lc][f][k + Q * (b + Q * c)];
            buf[1][lc][f][t] = s;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            double s = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s += sS[b][k] * buf[1][lc][f][a + Q * (k + Q * c)];
            buf[0][lc][f][t] = s;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            double s = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s += sS[c][k] * buf[0][lc][f][a + Q * (b + Q * k)];
            buf[1][lc][f][t] = s;
        }
    __syncthreads();
    if (!active) return;
    double U[3], GU[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        U[k] = buf[1][lc][k][t];
        double g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            g0 += sDc[a][r] * buf[1][lc][k][r + Q * (b + Q * c)];
            g1 += sDc[b][r] * buf[1][lc][k][a + Q * (r + Q * c)];
            g2 += sDc[c][r] * buf[1][lc][k][a + Q * (b + Q * r)];
        }
        GU[k][0] = g0 * m.inv_h; GU[k][1] = g1 * m.inv_h; GU[k][2] = g2 * m.inv_h;
    }
    double rho, mu, nz[3], vd;
    const int8_t cc = code[cell];
    if (cc == CELL_TABLE) {
        const double* tb = table + (int64_t)tindex[cell] * TAB_K * NQ + t;
        rho = tb[0]; mu = tb[NQ]; nz[0] = tb[2 * NQ]; nz[1] = tb[3 * NQ]; nz[2] = tb[4 * NQ]; vd = tb[5 * NQ];
    } else {
        const bool liq = cc == CELL_LIQUID;
        rho = liq ? m.rho_H1 : m.rho_H0;
        mu = liq ? m.mu_H1 : m.mu_H0;
        nz[0] = nz[1] = nz[2] = 0.0;
        vd = 0.0;
    }
    const double W = bas.w[a] * bas.w[b] * bas.w[c] * m.vol_w;
    const double wr = W * rho;
    double v[QC_K];
    v[0] = wr * m.c_mass;
#pragma unroll
    for (int k = 0; k < 3; ++k) v[1 + k] = wr * U[k];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int d = 0; d < 3; ++d) v[4 + 3 * k + d] = m.newton ? wr * GU[k][d] : 0.0;
    v[13] = 2.0 * W * mu;
    v[14] = nz[0]; v[15] = nz[1]; v[16] = nz[2];
    v[17] = W;
    v[18] = W * vd;
    const int64_t base = cell * QC_K * NQ + t;
#pragma unroll
    for (int k = 0; k < QC_K; ++k) qc[base + (int64_t)k * NQ] = v[k];
    const int64_t row = cell / n;
    const int cx = (int)(cell - row * n);
    const int64_t blk = cx / 32 + (int64_t)((n + 31) / 32) * row;
    float* dst = qc32 + (blk * QC32_K * NQ + t) * 32 + (cx % 32);
#pragma unroll
    for (int k = 0; k < QC32_K; ++k) dst[(int64_t)k * NQ * 32] = (float)(k < 3 ? v[1 + k] * m.inv_h : v[1 + k]);
}

// PRES: the velocity-pressure apply, with the pressure term -(div v, p) of Eq. (weakNavierStokes) for the Q1 pressure
// pin added to the gradient-tested flux (T_cc -= W p_h(x_q)).
template <typename T, int P, int CB, bool PRES>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1))
    k_momentum(MeshArgs<T> m, Basis<T> bas, const T* __restrict__ qc, const T* __restrict__ x, T* __restrict__ y,
               T* __restrict__ yp, const T* __restrict__ pin) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    __shared__ T sS[Q][Q], sDc[Q][Q], sN1[Q][2];
    __shared__ T buf[2][6][CB][NQ];  // [half][slot][cell][point]: conflict-free lanes
    __shared__ T q1a[CB][2 * Q * Q], q1b[CB][4 * Q];  // divergence-row test sweeps (Q1 nodes)
    const int tid = threadIdx.x;
    const int lc = tid / NQ, t = tid % NQ;
    const int64_t cell = (int64_t)blockIdx.x * CB + lc;
    const bool active = cell < m.ncell;
    if (tid < Q * Q) {
        sS[tid / Q][tid % Q] = bas.S[tid / Q][tid % Q];
        sDc[tid / Q][tid % Q] = bas.Dc[tid / Q][tid % Q] * m.inv_h;  // physical collocation derivative
    }
    if (tid < 2 * Q) sN1[tid / 2][tid % 2] = bas.N1[tid / 2][tid % 2];
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    const int n = m.n, M = m.M;
    int cx = 0, cy = 0, cz = 0;
    int64_t gidx = 0;
    bool cons = false;
    if (active) {
        cx = (int)(cell % n);
        cy = (int)((cell / n) % n);
        cz = (int)(cell / ((int64_t)n * n));
        const int gx = P * cx + a, gy = P * cy + b, gz = P * cz + c;
        gidx = gx + (int64_t)M * (gy + (int64_t)M * gz);
        cons = constrained_node(gx, gy, gz, M, m.faces);
#pragma unroll
        for (int k = 0; k < 3; ++k) buf[0][k][lc][t] = cons ? T(0) : x[k * m.Nu + gidx];
    }
    __syncthreads();
    // this thread's rows (forward) and columns (transposed) of S and Dc, kept in registers
    T Sa[Q], Sb[Q], Sc[Q], Da[Q], Db[Q], Dz[Q], Ta[Q], Tb[Q], Tc[Q], Ea[Q], Eb[Q], Ec[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        Sa[k] = sS[a][k]; Sb[k] = sS[b][k]; Sc[k] = sS[c][k];
        Da[k] = sDc[a][k]; Db[k] = sDc[b][k]; Dz[k] = sDc[c][k];
        Ta[k] = sS[k][a]; Tb[k] = sS[k][b]; Tc[k] = sS[k][c];
        Ea[k] = sDc[k][a]; Eb[k] = sDc[k][b]; Ec[k] = sDc[k][c];
    }
    // values at the Gauss points: x-, y-, z-sweeps of S
    if (active) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T s = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s += Sa[k] * buf[0][f][lc][k + Q * (b + Q * c)];
            buf[1][f][lc][t] = s;
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T s = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s += Sb[k] * buf[1][f][lc][a + Q * (k + Q * c)];
            buf[0][f][lc][t] = s;
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            T s = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s += Sc[k] * buf[0][f][lc][a + Q * (b + Q * k)];
            buf[1][f][lc][t] = s;
        }
    }
    __syncthreads();
    // quadrature-point fluxes from the cached coefficients
    T F[3] = {0, 0, 0}, Tf[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, rdiv = 0;
    if (active) {
        T X[3], G[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            X[k] = buf[1][k][lc][t];
            T g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                g0 += Da[r] * buf[1][k][lc][r + Q * (b + Q * c)];
                g1 += Db[r] * buf[1][k][lc][a + Q * (r + Q * c)];
                g2 += Dz[r] * buf[1][k][lc][a + Q * (b + Q * r)];
            }
            G[k][0] = g0; G[k][1] = g1; G[k][2] = g2;
        }
        const T* q = qc + cell * QC_K * NQ + t;
        T cf[QC_K];
#pragma unroll
        for (int k = 0; k < QC_K; ++k) cf[k] = q[k * NQ];
        const T tr = G[0][0] + G[1][1] + G[2][2];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T v = cf[0] * X[k];
#pragma unroll
            for (int d = 0; d < 3; ++d) v += cf[1 + d] * G[k][d] + cf[4 + 3 * k + d] * X[d];
            F[k] = v;
        }
        const T sm = cf[13] * tr, hm = T(0.5) * cf[13];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = k; l < 3; ++l) {  // symmetric: 6 distinct entries
                const T v = hm * (G[k][l] + G[l][k]) - sm * cf[14 + k] * cf[14 + l];
                Tf[k][l] = v;
                Tf[l][k] = v;
            }
        rdiv = cf[17] * tr - cf[18];
        if constexpr (PRES) {
            const int64_t m1 = n + 1;
            T pq = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int ja = j & 1, jb = (j >> 1) & 1, jc = j >> 2;
                pq += sN1[a][ja] * sN1[b][jb] * sN1[c][jc] * pin[(cx + ja) + m1 * ((cy + jb) + m1 * (cz + jc))];
            }
            const T wp = cf[17] * pq;
            Tf[0][0] -= wp;
            Tf[1][1] -= wp;
            Tf[2][2] -= wp;
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int s = 0; s < 9; ++s) buf[s / 6][s % 6][lc][t] = Tf[s / 3][s % 3];
        buf[1][3][lc][t] = rdiv;
    }
    __syncthreads();
    // test with gradients: w_c = F_c + sum_b Dc^T T_cb
    T wv[3];
    if (active) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                const int i0 = 3 * k + 0, i1 = 3 * k + 1, i2 = 3 * k + 2;
                s0 += Ea[r] * buf[i0 / 6][i0 % 6][lc][r + Q * (b + Q * c)];
                s1 += Eb[r] * buf[i1 / 6][i1 % 6][lc][a + Q * (r + Q * c)];
                s2 += Ec[r] * buf[i2 / 6][i2 % 6][lc][a + Q * (b + Q * r)];
            }
            wv[k] = F[k] + (s0 + s1 + s2);
        }
        // divergence row, Q1 test functions: sum_q N1_j(q) r_q by three sweeps; x-sweep here: [jx][qy][qz]
        if (yp && t < 2 * Q * Q) {
            const int jx = t & 1, qy = (t >> 1) % Q, qz = (t >> 1) / Q;
            T s = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) s += sN1[q][jx] * buf[1][3][lc][q + Q * (qy + Q * qz)];
            q1a[lc][t] = s;
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < 3; ++k) buf[0][k][lc][t] = wv[k];
        if (yp && t < 4 * Q) {  // y-sweep: [jx][jy][qz]
            const int jx = t & 1, jy = (t >> 1) & 1, qz = t >> 2;
            T s = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) s += sN1[q][jy] * q1a[lc][jx + 2 * (q + Q * qz)];
            q1b[lc][t] = s;
        }
    }
    __syncthreads();
    // transposed sweeps S^T: z, y, x
    if (active) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T s = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) s += Tc[q] * buf[0][k][lc][a + Q * (b + Q * q)];
            buf[1][k][lc][t] = s;
        }
        if (yp && t < 8) {  // z-sweep: Q1 node (jx, jy, jz)
            const int jx = t & 1, jy = (t >> 1) & 1, jz = t >> 2;
            T s = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) s += sN1[q][jz] * q1b[lc][jx + 2 * (jy + 2 * q)];
            const int64_t m1 = n + 1;
            atomicAdd(&yp[(cx + jx) + m1 * ((cy + jy) + m1 * (cz + jz))], s);
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T s = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) s += Tb[q] * buf[1][k][lc][a + Q * (q + Q * c)];
            buf[0][k][lc][t] = s;
        }
    }
    __syncthreads();
    if (active && !cons) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T s = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) s += Ta[q] * buf[0][k][lc][q + Q * (b + Q * c)];
            atomicAdd(&y[k * m.Nu + gidx], s);
        }
    }
}

int launch_qp_coeffs(evap_mesh* h, cudaStream_t s) {
    const MeshArgs<double>& m = h->m;
    const int nq = h->b.Q * h->b.Q * h->b.Q;
    const int64_t need = m.ncell * QC_K * nq;
    if (h->qc_len < need) {
        if (h->qc) cudaFree(h->qc);
        h->qc = nullptr;
        h->qc_len = 0;
        EVAP_CUDA(cudaMalloc(&h->qc, need * sizeof(double)));
        h->qc_len = need;
    }
    const int64_t need32 = (int64_t)((m.n + 31) / 32) * m.n * m.n * QC32_K * nq * 32;
    if (h->qc32_len < need32) {
        if (h->qc32) cudaFree(h->qc32);
        h->qc32 = nullptr;
        h->qc32_len = 0;
        EVAP_CUDA(cudaMalloc(&h->qc32, need32 * sizeof(float)));
        h->qc32_len = need32;
    }
    if (m.P == 2) {
        constexpr int CB = 8;
        k_qp_coeffs<2, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 27, 0, s>>>(m, h->b, h->cell_code, h->table_index,
                                                                                  h->table, h->u, h->qc, h->qc32);
    } else {
        constexpr int CB = 4;
        k_qp_coeffs<3, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 64, 0, s>>>(m, h->b, h->cell_code, h->table_index,
                                                                                  h->table, h->u, h->qc, h->qc32);
    }
    EVAP_CHECK_LAUNCH("qp_coeffs");
    return EVAP_OK;
}

// dst = src on the DoFs of the Dirichlet faces, one warp per x-line as k_momentum_init.
__global__ void __launch_bounds__(256) k_constrained_copy(int M, int64_t Nu, unsigned faces,
                                                          const double* __restrict__ src, double* __restrict__ dst) {
    const int lines = 3 * M * M;
    const int wpb = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int line = blockIdx.x * wpb + warp; line < lines; line += gridDim.x * wpb) {
        const int c = line / (M * M), rem = line - c * M * M, gz = rem / M, gy = rem - gz * M;
        const bool cyz = ((faces & 4u) && gy == 0) || ((faces & 8u) && gy == M - 1) || ((faces & 16u) && gz == 0) ||
                         ((faces & 32u) && gz == M - 1);
        const int64_t off = c * Nu + (int64_t)M * (gy + (int64_t)M * gz);
        for (int gx = lane; gx < M; gx += 32)
            if (cyz || ((faces & 1u) && gx == 0) || ((faces & 2u) && gx == M - 1)) dst[off + gx] = src[off + gx];
    }
}

// *flag = 1 if src is nonzero on a Dirichlet DoF.
__global__ void __launch_bounds__(256) k_constrained_nonzero(int M, int64_t Nu, unsigned faces,
                                                             const double* __restrict__ src, unsigned* flag) {
    const int lines = 3 * M * M;
    const int wpb = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    bool any = false;
    for (int line = blockIdx.x * wpb + warp; line < lines; line += gridDim.x * wpb) {
        const int c = line / (M * M), rem = line - c * M * M, gz = rem / M, gy = rem - gz * M;
        const bool cyz = ((faces & 4u) && gy == 0) || ((faces & 8u) && gy == M - 1) || ((faces & 16u) && gz == 0) ||
                         ((faces & 32u) && gz == M - 1);
        const int64_t off = c * Nu + (int64_t)M * (gy + (int64_t)M * gz);
        for (int gx = lane; gx < M; gx += 32)
            if ((cyz || ((faces & 1u) && gx == 0) || ((faces & 2u) && gx == M - 1)) && src[off + gx] != 0.0) any = true;
    }
    if (__any_sync(0xffffffffu, any) && lane == 0) atomicOr(flag, 1u);
}

static unsigned constrained_grid(const MeshArgs<double>& m) {
    const int64_t lines = 3 * (int64_t)m.M * m.M;
    return (unsigned)std::min<int64_t>((lines + 7) / 8, 152 * 16);
}

int launch_constrained_copy(evap_mesh* h, const double* src, double* dst, cudaStream_t s) {
    const MeshArgs<double>& m = h->m;
    if (!m.faces) return EVAP_OK;
    k_constrained_copy<<<constrained_grid(m), 256, 0, s>>>(m.M, m.Nu, m.faces, src, dst);
    EVAP_CHECK_LAUNCH("constrained_copy");
    return EVAP_OK;
}

int constrained_nonzero(evap_mesh* h, const double* src, bool* any, cudaStream_t s) {
    const MeshArgs<double>& m = h->m;
    *any = false;
    if (!m.faces) return EVAP_OK;
    // the input-check counter doubles as the flag (it is only read right after its own reduction)
    if (!h->nonfinite) EVAP_CUDA(cudaMalloc(&h->nonfinite, sizeof(unsigned long long)));
    unsigned* flag = reinterpret_cast<unsigned*>(h->nonfinite);
    EVAP_CUDA(cudaMemsetAsync(flag, 0, sizeof(unsigned), s));
    k_constrained_nonzero<<<constrained_grid(m), 256, 0, s>>>(m.M, m.Nu, m.faces, src, flag);
    EVAP_CHECK_LAUNCH("constrained_nonzero");
    unsigned hv = 0;
    EVAP_CUDA(cudaMemcpyAsync(&hv, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    EVAP_CUDA(cudaStreamSynchronize(s));
    *any = hv != 0;
    return EVAP_OK;
}

template <typename T>
int launch_momentum(evap_mesh* h, const T* x, T* y, T* yp, cudaStream_t s, bool init, const T* p, bool all_columns) {
    MeshArgs<T> m = mesh_args<T>(h);
    if (all_columns) {
        // the unconstrained operator (no face read as 0), then the identity rows of the real faces
        if (sizeof(T) != 8 || !init) return EVAP_EINVAL;
        m.faces = 0u;
    }
    const Basis<T> b = cast_basis<T>(h->b);
    const T* qc = (const T*)h->qc;  // FP64 only (the FP32 apply takes the line kernel)
    if (init) {
        const int64_t lines = 3 * (int64_t)m.M * m.M;
        const unsigned grid = (unsigned)std::min<int64_t>((lines + 7) / 8, 152 * 16);
        k_momentum_init<T><<<grid, 256, 0, s>>>(m.M, m.Nu, m.faces, x, y, yp, m.Nphi);
        EVAP_CHECK_LAUNCH("momentum_init");
    }
    if constexpr (sizeof(T) == 4) {  // FP32: line-oriented kernel with u0 interpolated on the fly (momentum32.cu)
        (void)b;
        (void)qc;
        if (p) return EVAP_EINVAL;  // the pressure term is FP64 only
        return launch_momentum32(h, x, y, yp, s);
    } else {
        if (m.P == 2) {
            constexpr int CB = 8;
            const unsigned grid = (unsigned)((m.ncell + CB - 1) / CB);
            if (p)
                k_momentum<T, 2, CB, true><<<grid, CB * 27, 0, s>>>(m, b, qc, x, y, yp, p);
            else
                k_momentum<T, 2, CB, false><<<grid, CB * 27, 0, s>>>(m, b, qc, x, y, yp, nullptr);
        } else {
            constexpr int CB = 4;
            const unsigned grid = (unsigned)((m.ncell + CB - 1) / CB);
            if (p)
                k_momentum<T, 3, CB, true><<<grid, CB * 64, 0, s>>>(m, b, qc, x, y, yp, p);
            else
                k_momentum<T, 3, CB, false><<<grid, CB * 64, 0, s>>>(m, b, qc, x, y, yp, nullptr);
        }
        EVAP_CHECK_LAUNCH("momentum");
        if (all_columns) return launch_constrained_copy(h, (const double*)x, (double*)y, s);
        return EVAP_OK;
    }
}
template int launch_momentum<double>(evap_mesh*, const double*, double*, double*, cudaStream_t, bool, const double*,
                                     bool);
template int launch_momentum<float>(evap_mesh*, const float*, float*, float*, cudaStream_t, bool, const float*, bool);

}  // namespace evap
