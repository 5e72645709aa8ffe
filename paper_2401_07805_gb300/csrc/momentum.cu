// Momentum apply y = A x (velocity block of Eq. weakNavierStokes linearized about u0, App. D) with the divergence row
// y_p = B x - g (Eq. continuity with the dilation rate of Eq. evaporDil): the pieces shared by its implementations.
//   k_momentum_init   y = x on the Dirichlet DoFs, 0 elsewhere (the scatter of the applies adds the free rows)
//   k_qp_coeffs       the quadrature-point coefficients of the operator (W rho c_m, W rho u0, W rho grad u0, 2 W mu,
//                     z n, W, W v_dil), evaluated once per set_fields in FP64 and stored in FP64 (adjoint, Jacobi
//                     diagonal, continuity right-hand side), as double-float pairs (the FP64-accurate apply of
//                     momentum_df.cu) and, for the u0 terms, in FP32 (the FP32 apply of momentum32.cu): on GB300 the
//                     arithmetic, not HBM, bounds these operators, and the material law and the u0 interpolation
//                     would otherwise be recomputed by every apply
//   launch_momentum   dispatch: FP64 -> double-float kernel, FP32 -> line kernel; the lifting variant (all columns)
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
                double* __restrict__ qc, float2* __restrict__ qcdf, float* __restrict__ qc32) {
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
    for (int k = 0; k < QC_K; ++k) {
        qc[base + (int64_t)k * NQ] = v[k];
        const float hi = (float)v[k];
        qcdf[base + (int64_t)k * NQ] = make_float2(hi, (float)(v[k] - (double)hi));
    }
    const int64_t row = cell / n;
    const int cx = (int)(cell - row * n);
    const int64_t blk = cx / 32 + (int64_t)((n + 31) / 32) * row;
    float* dst = qc32 + (blk * QC32_K * NQ + t) * 32 + (cx % 32);
#pragma unroll
    for (int k = 0; k < QC32_K; ++k) dst[(int64_t)k * NQ * 32] = (float)(k < 3 ? v[1 + k] * m.inv_h : v[1 + k]);
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
    if (h->qcdf_len < 2 * need) {
        if (h->qcdf) cudaFree(h->qcdf);
        h->qcdf = nullptr;
        h->qcdf_len = 0;
        EVAP_CUDA(cudaMalloc(&h->qcdf, 2 * need * sizeof(float)));
        h->qcdf_len = 2 * need;
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
                                                                                  h->table, h->u, h->qc, (float2*)h->qcdf, h->qc32);
    } else {
        constexpr int CB = 4;
        k_qp_coeffs<3, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 64, 0, s>>>(m, h->b, h->cell_code, h->table_index,
                                                                                  h->table, h->u, h->qc, (float2*)h->qcdf, h->qc32);
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
    MeshArgs<double> m = h->m;
    if (all_columns) {
        // the unconstrained operator (no face read as 0), then the identity rows of the real faces
        if (sizeof(T) != 8 || !init) return EVAP_EINVAL;
        m.faces = 0u;
    }
    if (init) {
        const int64_t lines = 3 * (int64_t)m.M * m.M;
        const unsigned grid = (unsigned)std::min<int64_t>((lines + 7) / 8, 152 * 16);
        k_momentum_init<T><<<grid, 256, 0, s>>>(m.M, m.Nu, m.faces, x, y, yp, m.Np);  // y_p: pressure space
        EVAP_CHECK_LAUNCH("momentum_init");
    }
    if constexpr (sizeof(T) == 4) {  // FP32: line-oriented kernel (momentum32.cu)
        if (p) return EVAP_EINVAL;  // the pressure term is FP64 only
        return launch_momentum32(h, x, y, yp, s);
    } else {  // FP64-accurate: double-float arithmetic on the FP32 pipe (momentum_df.cu)
        int rc = launch_momentum_df(h, m, x, y, yp, p, s);
        if (rc) return rc;
        if (all_columns) return launch_constrained_copy(h, x, y, s);
        return EVAP_OK;
    }
}
template int launch_momentum<double>(evap_mesh*, const double*, double*, double*, cudaStream_t, bool, const double*,
                                     bool);
template int launch_momentum<float>(evap_mesh*, const float*, float*, float*, cudaStream_t, bool, const float*, bool);

}  // namespace evap
