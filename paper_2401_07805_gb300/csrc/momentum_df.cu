// FP64-accurate momentum apply in double-float arithmetic: the velocity block of Eq. weakNavierStokes linearized
// about u0 (App. D) with the corrected stress of Eq. modified_viscous_stress, the divergence row of Eq. continuity and,
// for the velocity-pressure apply, the pressure term -(div v, p), y = sum_i R_i^T A_i R_i x (Sec. 2.5), with every
// sweep, flux and test evaluated on hi + lo pairs of FP32 numbers (dfloat.cuh):
//   gather   x, u0 at the (P+1)^3 nodes (Dirichlet nodes of x read as 0), converted to double-float
//   values   3 sweeps of the 1D matrix S[q][a] = l_a(t_q) per component            -> x_c at the Gauss points
//   grads    collocation derivative Dc at the Gauss points along each direction     -> d_b x_c
//   flux     F_c  = W rho (c_m x_c + u0 . grad x_c + newton (grad u0 x)_c)
//            T_cb = 2 W mu (eps_cb - tr(eps) (z n)_c (z n)_b),  eps = sym grad x
//   test     w_c = F_c + sum_b Dc^T T_cb, then 3 transposed sweeps S^T            -> nodal contributions
//   scatter  atomic FP64 add into y (constrained rows hold y = x, written by the init kernel)
//
// Why: on GB300 the FP64 pipe (~1.2 TFLOP/s measured) bounds the plain FP64 apply two orders of magnitude below the
// HBM roof, while the FP32 pipe issues ~60x as many FMAs.  A double-float multiply-add costs ~12 FP32 instructions, so
// the same Gauss sums at ~48-bit precision (relative rounding ~4e-15 per operation, below the 1e-12 parity bar by
// two orders of magnitude) leave the FP64 pipe with only the conversions of the nodal values (x in, y out).
//
// Layout: one thread per quadrature point, CB cells per block, sweeps through shared
// memory; the thread keeps its rows of the 1D matrices (S, the physical collocation derivative Dc/h, their
// transposes) in registers as double-float constants.  The quadrature-point coefficients are the FP64 values of
// k_qp_coeffs split into double-float pairs (qcdf, [cell][QC_K][nq] float2, written by the same kernel), 8 bytes per
// coefficient as in FP64; each thread copies its point's coefficients into shared memory with cp.async at the start,
// so that their HBM latency is hidden behind the interpolation sweeps (without it, waits on these loads were the top
// stall).  The correction term is skipped at points where its
// gate z n is zero (outside the interface zone), and the Newton terms on Picard meshes.
#include <algorithm>

#include "async_copy.cuh"
#include "dfloat.cuh"
#include "physics.cuh"

namespace evap {

template <int P, int CB>
constexpr size_t df_coeff_smem() {
    return sizeof(float2) * CB * QC_K * (P + 1) * (P + 1) * (P + 1);
}

// Block shape for Q2: CB cells per block (one thread per point), at least MINB blocks per SM (which caps the
// registers).  Measured at 64^3 on GB300, 100 back-to-back applies with the divergence row (ms per apply):
// CB 4 / MINB 8 (64 registers) 0.685; CB 4 / 6 0.699; CB 8 / 4 0.700; CB 8 without a minimum (72 registers) 0.691;
// CB 8 / 3 0.722; CB 4 / 1 (89 registers) 0.738; CB 8 / 1 0.848; CB 12 / 1 1.207.  Single- and two-warp blocks,
// on another box against CB 4 / 8 at 0.691 there: CB 1 / 28 (72 registers) 0.695, CB 1 / 20 0.728, CB 2 / 14 0.709,
// CB 3 / 10 0.720.
#ifndef EVAP_DF_CB2
#define EVAP_DF_CB2 4
#endif
#ifndef EVAP_DF_MINB2
#define EVAP_DF_MINB2 8
#endif
#ifndef EVAP_DF_MINB2_PRES
#define EVAP_DF_MINB2_PRES 8
#endif

// Normalization of the sweep results (the closing Fast2Sum of each dot product).  A result that is converted to FP64
// next (the last transposed sweep) or that only starts a new accumulation (the value flux F, whose hi and lo enter
// the test sum through TwoSum) loses nothing when left unnormalized (hi + lo stays exact).  A result that is then
// multiplied carries its larger lo part into the rounded cross terms.  EVAP_DF_LAZY: 0 normalize all; 3 skip only the
// free cases; 2 also the gradients; 1 every sweep result.  Measured at 64^3 (ms per apply; relative error of the
// smoke case against the oracle): 0 0.6925, 4.8e-15; 3 0.6812, 5.7e-15; 2 0.6767, 5.7e-15; 1 0.6639, 8.9e-15, and
// with 1 the coupled step's velocity-pressure solve no longer reaches its 1e-10 (its rounding floor rises to 1.2e-10).
#ifndef EVAP_DF_LAZY
#define EVAP_DF_LAZY 2
#endif
template <int Q, bool LAZY>
__device__ __forceinline__ dfl df_dot_lz(const dfl* c, const dfl* v, int stride) {
    if constexpr (LAZY) {
        dfl s = df_prod(c[0], v[0]);
#pragma unroll
        for (int k = 1; k < Q; ++k) df_fma(s, c[k], v[k * stride]);
        return s;
    } else {
        return df_dot<Q>(c, v, stride);
    }
}
constexpr bool LZ_SWEEP = EVAP_DF_LAZY == 1;                    // interpolation and transposed sweeps, w
constexpr bool LZ_GRAD = EVAP_DF_LAZY == 1 || EVAP_DF_LAZY == 2;  // gradients at the points
constexpr bool LZ_FREE = EVAP_DF_LAZY != 0;                      // the last sweep, the value flux

template <int P, int CB, bool PRES, int MINB, bool DET>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1), MINB)
    k_momentum_df(MeshArgs<double> m, DfBasis bas, const float2* __restrict__ qc, const double* __restrict__ x,
                  double* __restrict__ y, double* __restrict__ yp, const double* __restrict__ pin, int colour) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    __shared__ dfl sS[Q][Q], sDc[Q][Q], sN1[Q][2];
    __shared__ dfl buf[2][6][CB][NQ];  // [half][slot][cell][point]
    __shared__ dfl q1a[CB][2 * Q * Q], q1b[CB][4 * Q];
    extern __shared__ float2 sqc[];  // [cell][QC_K][point]: this block's coefficients, copied while the sweeps run
    const int tid = threadIdx.x;
    const int lc = tid / NQ, t = tid % NQ;
    int cx = 0, cy = 0, cz = 0;
    const bool active = colour_cell((int64_t)blockIdx.x * CB + lc, m.n, DET ? colour : -1, cx, cy, cz);
    const int64_t cell = cx + (int64_t)m.n * (cy + (int64_t)m.n * cz);
    constexpr bool plain = DET;  // a colour pass: no other cell of the launch touches this cell's nodes
    float2* myq = sqc + (int64_t)lc * QC_K * NQ + t;
    if (active) {  // each thread fetches (and later reads) only its own point's coefficients
        const float2* src = qc + cell * QC_K * NQ + t;
#pragma unroll
        for (int k = 0; k < QC_K; ++k)
            if (m.newton || k < 4 || k > 12) cp_async8(myq + k * NQ, src + k * NQ);
    }
    cp_async_commit();
    if (tid < Q * Q) {
        sS[tid / Q][tid % Q] = bas.S[tid / Q][tid % Q];
        sDc[tid / Q][tid % Q] = bas.Dc[tid / Q][tid % Q];
    }
    if (tid < 2 * Q) sN1[tid / 2][tid % 2] = bas.N1[tid / 2][tid % 2];
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    const int n = m.n, M = m.M;
    int64_t gidx = 0;
    bool cons = false;
    if (active) {
        const int gx = P * cx + a, gy = P * cy + b, gz = P * cz + c;
        gidx = gx + (int64_t)M * (gy + (int64_t)M * gz);
        cons = constrained_node(gx, gy, gz, M, m.faces);
#pragma unroll
        for (int k = 0; k < 3; ++k) buf[0][k][lc][t] = cons ? dfl{0.f, 0.f} : df_from_double(x[k * m.Nu + gidx]);
    }
    __syncthreads();
    // values at the Gauss points: x-, y-, z-sweeps of S
    if (active) {
        dfl Sa[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Sa[k] = sS[a][k];
#pragma unroll
        for (int f = 0; f < 3; ++f) buf[1][f][lc][t] = df_dot_lz<Q, LZ_SWEEP>(Sa, &buf[0][f][lc][Q * (b + Q * c)], 1);
    }
    __syncthreads();
    if (active) {
        dfl Sb[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Sb[k] = sS[b][k];
#pragma unroll
        for (int f = 0; f < 3; ++f) buf[0][f][lc][t] = df_dot_lz<Q, LZ_SWEEP>(Sb, &buf[1][f][lc][a + Q * Q * c], Q);
    }
    __syncthreads();
    if (active) {
        dfl Sc[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Sc[k] = sS[c][k];
#pragma unroll
        for (int f = 0; f < 3; ++f) buf[1][f][lc][t] = df_dot_lz<Q, LZ_SWEEP>(Sc, &buf[0][f][lc][a + Q * b], Q * Q);
    }
    __syncthreads();
    // quadrature-point fluxes from the cached coefficients
    dfl F[3], Tf[3][3], rdiv{0.f, 0.f};
    if (active) {
        dfl X[3], G[3][3];
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
                X[k] = buf[1][k][lc][t];
                G[k][0] = df_dot_lz<Q, LZ_GRAD>(Da, &buf[1][k][lc][Q * (b + Q * c)], 1);
                G[k][1] = df_dot_lz<Q, LZ_GRAD>(Db, &buf[1][k][lc][a + Q * Q * c], Q);
                G[k][2] = df_dot_lz<Q, LZ_GRAD>(Dz, &buf[1][k][lc][a + Q * b], Q * Q);
            }
        }
        cp_async_wait_all();
        const float2* q = myq;
        const dfl c0 = ld_df(q);
        const dfl cu[3] = {ld_df(q + NQ), ld_df(q + 2 * NQ), ld_df(q + 3 * NQ)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dfl v = df_prod(c0, X[k]);
#pragma unroll
            for (int d = 0; d < 3; ++d) df_fma(v, cu[d], G[k][d]);
            if (m.newton) {
#pragma unroll
                for (int d = 0; d < 3; ++d) df_fma(v, ld_df(q + (4 + 3 * k + d) * NQ), X[d]);
            }
            F[k] = LZ_FREE ? v : df_norm(v);
        }
        const dfl c13 = ld_df(q + 13 * NQ);
        const dfl tr = df_add(df_add(G[0][0], G[1][1]), G[2][2]);
        const dfl hm = df_scale2(c13, 0.5f);
        const dfl nz[3] = {ld_df(q + 14 * NQ), ld_df(q + 15 * NQ), ld_df(q + 16 * NQ)};
        const bool corr = (nz[0].hi != 0.f) || (nz[1].hi != 0.f) || (nz[2].hi != 0.f);
        const dfl sm = corr ? df_mul(c13, tr) : dfl{0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = k; l < 3; ++l) {  // symmetric: 6 distinct entries
                dfl v = k == l ? df_mul(c13, G[k][k]) : df_mul(hm, df_add(G[k][l], G[l][k]));
                if (corr) {
                    dfl w = v;
                    df_fma(w, df_neg(sm), df_mul(nz[k], nz[l]));
                    v = df_norm(w);
                }
                Tf[k][l] = v;
                Tf[l][k] = v;
            }
        {
            dfl r = df_prod(ld_df(q + 17 * NQ), tr);
            const dfl src = ld_df(q + 18 * NQ);
            const dfl s2 = two_sum(r.hi, -src.hi);
            r.hi = s2.hi;
            r.lo = __fadd_rn(r.lo, __fsub_rn(s2.lo, src.lo));
            rdiv = df_norm(r);
        }
        if constexpr (PRES) {  // p at the point: trilinear interpolation by successive linear ones, in FP64
            const int64_t m1 = n + 1;
            const double* p0 = pin + cx + m1 * (cy + m1 * cz);
            const double tx = bas.t[a], ty = bas.t[b], tz = bas.t[c];
            double e[2][2];
#pragma unroll
            for (int jc = 0; jc < 2; ++jc)
#pragma unroll
                for (int jb = 0; jb < 2; ++jb) {
                    const double* r = p0 + m1 * (jb + m1 * jc);
                    e[jc][jb] = fma(tx, r[1] - r[0], r[0]);
                }
            const double f0 = fma(ty, e[0][1] - e[0][0], e[0][0]), f1 = fma(ty, e[1][1] - e[1][0], e[1][0]);
            const dfl wp = df_mul(ld_df(q + 17 * NQ), df_from_double(fma(tz, f1 - f0, f0)));
#pragma unroll
            for (int k = 0; k < 3; ++k) Tf[k][k] = df_sub(Tf[k][k], wp);
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
    dfl wv[3];
    if (active) {
        dfl Ea[Q], Eb[Q], Ec[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            Ea[k] = sDc[k][a];
            Eb[k] = sDc[k][b];
            Ec[k] = sDc[k][c];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int i0 = 3 * k + 0, i1 = 3 * k + 1, i2 = 3 * k + 2;
            dfl s = F[k];
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                df_fma(s, Ea[r], buf[i0 / 6][i0 % 6][lc][r + Q * (b + Q * c)]);
                df_fma(s, Eb[r], buf[i1 / 6][i1 % 6][lc][a + Q * (r + Q * c)]);
                df_fma(s, Ec[r], buf[i2 / 6][i2 % 6][lc][a + Q * (b + Q * r)]);
            }
            wv[k] = LZ_SWEEP ? s : df_norm(s);
        }
        // divergence row, Q1 test functions: sum_q N1_j(q) r_q by three sweeps; x-sweep here: [jx][qy][qz]
        if (yp && t < 2 * Q * Q) {
            const int jx = t & 1, qy = (t >> 1) % Q, qz = (t >> 1) / Q;
            dfl s = df_prod(sN1[0][jx], buf[1][3][lc][Q * (qy + Q * qz)]);
#pragma unroll
            for (int qq = 1; qq < Q; ++qq) df_fma(s, sN1[qq][jx], buf[1][3][lc][qq + Q * (qy + Q * qz)]);
            q1a[lc][t] = df_norm(s);
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < 3; ++k) buf[0][k][lc][t] = wv[k];
        if (yp && t < 4 * Q) {  // y-sweep: [jx][jy][qz]
            const int jx = t & 1, jy = (t >> 1) & 1, qz = t >> 2;
            dfl s = df_prod(sN1[0][jy], q1a[lc][jx + 2 * (0 + Q * qz)]);
#pragma unroll
            for (int qq = 1; qq < Q; ++qq) df_fma(s, sN1[qq][jy], q1a[lc][jx + 2 * (qq + Q * qz)]);
            q1b[lc][t] = df_norm(s);
        }
    }
    __syncthreads();
    // transposed sweeps S^T: z, y, x
    if (active) {
        dfl Tc[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Tc[k] = sS[k][c];
#pragma unroll
        for (int k = 0; k < 3; ++k) buf[1][k][lc][t] = df_dot_lz<Q, LZ_SWEEP>(Tc, &buf[0][k][lc][a + Q * b], Q * Q);
        if (yp && t < 8) {  // z-sweep: Q1 node (jx, jy, jz)
            const int jx = t & 1, jy = (t >> 1) & 1, jz = t >> 2;
            dfl s = df_prod(sN1[0][jz], q1b[lc][jx + 2 * (jy + 2 * 0)]);
#pragma unroll
            for (int qq = 1; qq < Q; ++qq) df_fma(s, sN1[qq][jz], q1b[lc][jx + 2 * (jy + 2 * qq)]);
            const int64_t m1 = n + 1;
            acc_add(&yp[(cx + jx) + m1 * ((cy + jy) + m1 * (cz + jz))], df_to_double(df_norm(s)), plain);
        }
    }
    __syncthreads();
    if (active) {
        dfl Tb[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Tb[k] = sS[k][b];
#pragma unroll
        for (int k = 0; k < 3; ++k) buf[0][k][lc][t] = df_dot_lz<Q, LZ_SWEEP>(Tb, &buf[1][k][lc][a + Q * Q * c], Q);
    }
    __syncthreads();
    if (active && !cons) {
        dfl Ta[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Ta[k] = sS[k][a];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            acc_add(&y[k * m.Nu + gidx], df_to_double(df_dot_lz<Q, LZ_FREE>(Ta, &buf[0][k][lc][Q * (b + Q * c)], 1)), plain);
    }
}

DfBasis make_df_basis(const Basis<double>& b, double inv_h) {
    DfBasis d{};
    for (int q = 0; q < b.Q; ++q) {
        for (int k = 0; k < b.Q; ++k) {
            d.S[q][k] = df_from_double(b.S[q][k]);
            d.Dc[q][k] = df_from_double(b.Dc[q][k] * inv_h);
        }
        d.N1[q][0] = df_from_double(b.N1[q][0]);
        d.N1[q][1] = df_from_double(b.N1[q][1]);
        d.t[q] = b.t[q];
    }
    return d;
}

// y = A x (+ y_p = B x - g, + the pressure term when p is given); the init kernel has written y = x on the Dirichlet
// DoFs (faces of m) and zeros elsewhere.
int launch_momentum_df(evap_mesh* h, const MeshArgs<double>& m, const double* x, double* y, double* yp,
                       const double* p, cudaStream_t s) {
    const DfBasis b = make_df_basis(h->b, m.inv_h);
    const float2* qc = reinterpret_cast<const float2*>(h->qcdf);
    const int c0 = h->deterministic ? 0 : -1, c1 = h->deterministic ? 8 : 0;  // colour passes, or one atomic pass
    auto run = [&](auto kern, int CB, int threads, size_t dyn) -> int {
        EVAP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        for (int colour = c0; colour < std::max(c1, c0 + 1); ++colour) {
            const int64_t cells = colour_cells(m.n, colour);
            if (cells == 0) continue;
            const unsigned grid = (unsigned)((cells + CB - 1) / CB);
            kern<<<grid, threads, dyn, s>>>(m, b, qc, x, y, yp, p, colour);
            EVAP_CHECK_LAUNCH("momentum_df");
        }
        return EVAP_OK;
    };
    int rc;
    if (m.P == 2) {
        constexpr int CB = EVAP_DF_CB2, MINB = EVAP_DF_MINB2, MINBP = EVAP_DF_MINB2_PRES;
        constexpr size_t dyn = df_coeff_smem<2, CB>();
        const bool det = h->deterministic;
        rc = p ? run(det ? k_momentum_df<2, CB, true, MINBP, true> : k_momentum_df<2, CB, true, MINBP, false>, CB,
                     CB * 27, dyn)
               : run(det ? k_momentum_df<2, CB, false, MINB, true> : k_momentum_df<2, CB, false, MINB, false>, CB,
                     CB * 27, dyn);
    } else {
        constexpr int CB = 4;
        constexpr size_t dyn = df_coeff_smem<3, CB>();
        const bool det = h->deterministic;
        rc = p ? run(det ? k_momentum_df<3, CB, true, 1, true> : k_momentum_df<3, CB, true, 1, false>, CB, CB * 64,
                     dyn)
               : run(det ? k_momentum_df<3, CB, false, 1, true> : k_momentum_df<3, CB, false, 1, false>, CB, CB * 64,
                     dyn);
    }
    return rc;
}

}  // namespace evap
