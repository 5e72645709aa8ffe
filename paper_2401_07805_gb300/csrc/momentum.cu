// Momentum apply y = A x (velocity block of Eq. weakNavierStokes linearized about u0, App. D) with the divergence row
// y_p = B x - g (Eq. continuity with the dilation rate of Eq. evaporDil): the pieces shared by its implementations.
//   k_momentum_init   y = x on the Dirichlet DoFs, 0 elsewhere (the scatter of the applies adds the free rows)
//   k_qp_coeffs       the quadrature-point coefficients of the operator (W rho c_m, W rho u0, W rho grad u0, 2 W mu,
//                     z n, W, W v_dil), evaluated once per set_fields in double-float arithmetic and stored as
//                     double-float pairs (the FP64-accurate apply of momentum_df.cu and the adjoint), in FP64 (Jacobi
//                     diagonal, continuity right-hand side, mass load) and, for the u0 terms, in FP32 (the FP32
//                     apply of momentum32.cu): on GB300 the
//                     arithmetic, not HBM, bounds these operators, and the material law and the u0 interpolation
//                     would otherwise be recomputed by every apply
//   launch_momentum   dispatch: FP64 -> double-float kernel, FP32 -> line kernel; the lifting variant (all columns)
#include "dfloat.cuh"
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
// The interpolation of u0 and every product run in double-float arithmetic (dfloat.cuh) on the FP32 pipe: the FP64
// pipe keeps the conversions (u0 in, the FP64 copy of each coefficient out) and the few scalar factors.  The
// double-float results are the pairs of the apply's cache as they stand; the FP64 copy is their sum (within 2^-48).
template <int P, int CB>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1))
    k_qp_coeffs(MeshArgs<double> m, Basis<double> bas, DfBasis dfb, dfl cm_df, dfl invh_df,
                const int8_t* __restrict__ code, const int32_t* __restrict__ tindex, const double* __restrict__ table,
                const double* __restrict__ u0, double* __restrict__ qc, float2* __restrict__ qcdf,
                float* __restrict__ qc32) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    __shared__ dfl sS[Q][Q], sDc[Q][Q];
    __shared__ dfl buf[2][CB][3][NQ];
    const int tid = threadIdx.x;
    const int lc = tid / NQ, t = tid % NQ;
    const int64_t cell = (int64_t)blockIdx.x * CB + lc;
    const bool active = cell < m.ncell;
    if (tid < Q * Q) {
        sS[tid / Q][tid % Q] = dfb.S[tid / Q][tid % Q];
        sDc[tid / Q][tid % Q] = dfb.Dc[tid / Q][tid % Q];  // physical: Dc / h
    }
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    const int n = m.n, M = m.M;
    if (active) {
        const int cx = (int)(cell % n), cy = (int)((cell / n) % n), cz = (int)(cell / ((int64_t)n * n));
        const int64_t gidx = (P * cx + a) + (int64_t)M * ((P * cy + b) + (int64_t)M * (P * cz + c));
#pragma unroll
        for (int k = 0; k < 3; ++k) buf[0][lc][k][t] = df_from_double(u0[k * m.Nu + gidx]);
    }
    __syncthreads();
    if (active) {
        dfl Sa[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Sa[k] = sS[a][k];
#pragma unroll
        for (int f = 0; f < 3; ++f) buf[1][lc][f][t] = df_dot<Q>(Sa, &buf[0][lc][f][Q * (b + Q * c)], 1);
    }
    __syncthreads();
    if (active) {
        dfl Sb[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Sb[k] = sS[b][k];
#pragma unroll
        for (int f = 0; f < 3; ++f) buf[0][lc][f][t] = df_dot<Q>(Sb, &buf[1][lc][f][a + Q * Q * c], Q);
    }
    __syncthreads();
    if (active) {
        dfl Sc[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Sc[k] = sS[c][k];
#pragma unroll
        for (int f = 0; f < 3; ++f) buf[1][lc][f][t] = df_dot<Q>(Sc, &buf[0][lc][f][a + Q * b], Q * Q);
    }
    __syncthreads();
    if (!active) return;
    dfl U[3], GU[3][3];
    {
        dfl Da[Q], Db[Q], Dz[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            Da[k] = sDc[a][k];
            Db[k] = sDc[b][k];
            Dz[k] = sDc[c][k];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            U[k] = buf[1][lc][k][t];
            GU[k][0] = df_dot<Q>(Da, &buf[1][lc][k][Q * (b + Q * c)], 1);
            GU[k][1] = df_dot<Q>(Db, &buf[1][lc][k][a + Q * Q * c], Q);
            GU[k][2] = df_dot<Q>(Dz, &buf[1][lc][k][a + Q * b], Q * Q);
        }
    }
    double rho, mu, nz[3], vd;
    const int8_t cc = code[cell];
    const bool tab = cc == CELL_TABLE;
    if (tab) {
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
    const dfl wr = df_from_double(W * rho);
    dfl v[QC_K];
    v[0] = df_mul(wr, cm_df);
#pragma unroll
    for (int k = 0; k < 3; ++k) v[1 + k] = df_mul(wr, U[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int d = 0; d < 3; ++d) v[4 + 3 * k + d] = m.newton ? df_mul(wr, GU[k][d]) : dfl{0.f, 0.f};
    v[13] = df_from_double(2.0 * W * mu);
    const dfl z0{0.f, 0.f};
    v[14] = tab ? df_from_double(nz[0]) : z0;
    v[15] = tab ? df_from_double(nz[1]) : z0;
    v[16] = tab ? df_from_double(nz[2]) : z0;
    v[17] = df_from_double(W);
    v[18] = tab ? df_from_double(W * vd) : z0;
    const int64_t base = cell * QC_K * NQ + t;
#pragma unroll
    for (int k = 0; k < QC_K; ++k) {
        qc[base + (int64_t)k * NQ] = df_to_double(v[k]);
        qcdf[base + (int64_t)k * NQ] = make_float2(v[k].hi, v[k].lo);
    }
    const int64_t row = cell / n;
    const int cx = (int)(cell - row * n);
    const int64_t blk = cx / 32 + (int64_t)((n + 31) / 32) * row;
    float* dst = qc32 + (blk * QC32_K * NQ + t) * 32 + (cx % 32);
#pragma unroll
    for (int k = 0; k < QC32_K; ++k) dst[(int64_t)k * NQ * 32] = k < 3 ? df_mul(v[1 + k], invh_df).hi : v[1 + k].hi;
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
    const DfBasis dfb = make_df_basis(h->b, m.inv_h);
    const dfl cm = df_from_double(m.c_mass), ih = df_from_double(m.inv_h);
    if (m.P == 2) {
        constexpr int CB = 8;
        k_qp_coeffs<2, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 27, 0, s>>>(
            m, h->b, dfb, cm, ih, h->cell_code, h->table_index, h->table, h->u, h->qc, (float2*)h->qcdf, h->qc32);
    } else {
        constexpr int CB = 4;
        k_qp_coeffs<3, CB><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 64, 0, s>>>(
            m, h->b, dfb, cm, ih, h->cell_code, h->table_index, h->table, h->u, h->qc, (float2*)h->qcdf, h->qc32);
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
