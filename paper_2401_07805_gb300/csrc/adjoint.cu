// Adjoint of the momentum apply, FP64-accurate.  The u0 terms and the material coefficients come from the
// quadrature-point cache of set_fields (the double-float pairs the forward apply uses, so g_x is its transpose to
// rounding); the chain-rule factors that depend only on phi and mdot (H'(d) d'(phi), its phi-derivative, the normal,
// 1/|grad phi|, c_1 delta, ...) come from the adjoint table that set_fields fills in FP64 for the interface cells.
//
// L = w . A(phi, u0) x + w_p . (B x - g(phi, mdot))  (velocity block and divergence row of Eq. weakNavierStokes).
// Per quadrature point with W the weight, (X, G) values/gradients of x, (Om, OmG) of w, (U, GU) of u0, pi of w_p:
//   dL/dX_d     = W rho (c_m Om_d + newton sum_c Om_c GU_cd)
//   dL/dG_db    = W rho Om_d U_b + 2 W mu (sym(OmG)_db - z delta_db (n . OmG n)) + W pi delta_db
//   dL/dU_b     = W rho sum_c Om_c G_cb,           dL/dGU_cd = newton W rho Om_c X_d
//   dL/drho     = W Om . (c_m X + G U + newton GU X),  dL/dmu = 2 W OmG : eps_mod(X)
//   dL/dn       = -2 W mu z tr(G) (OmG + OmG^T) n,  dL/dv_dil = -W pi
//   chain rule through Eqs. (heaviside), (rhoEff), (muEff), (normal_vector), (delta), (evaporDil):
//     drho/dH = -rho^2 (1/rho_l - 1/rho_g), dmu/dH = mu_l - mu_g, dH/dphi = H'(d) d'(phi),
//     d delta/dphi = (H''(d) d'(phi)^2 + H'(d) d''(phi)) |grad phi|, d delta/d grad phi = H'(d) d'(phi) n,
//     dn/d grad phi = (I - n n^T)/|grad phi|; the zone gate is piecewise constant.
// The value/gradient sensitivities are tested like the forward operator (S^T and Dc^T sweeps); the Q1 sensitivities
// are integrated against the level-set shape functions N_j and grad N_j (Q1 on the level-set mesh: the velocity
// cell subdivided n_sub times per direction).
#include <algorithm>

#include "async_copy.cuh"
#include "dfloat.cuh"
#include "physics.cuh"

namespace evap {

__device__ __forceinline__ bool cons_node(int gx, int gy, int gz, int M, unsigned f) {
    return ((f & 1u) && gx == 0) || ((f & 2u) && gx == M - 1) || ((f & 4u) && gy == 0) ||
           ((f & 8u) && gy == M - 1) || ((f & 16u) && gz == 0) || ((f & 32u) && gz == M - 1);
}

__global__ void k_adjoint_init(int M, int64_t Nu, int64_t Np, unsigned faces, const double* __restrict__ w,
                               double* gx, double* gu, double* gphi, double* gm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * Nu; i += stride) {
        if (gx) {
            const int64_t node = i % Nu;
            const int a = (int)(node % M), b = (int)((node / M) % M), c = (int)(node / ((int64_t)M * M));
            gx[i] = cons_node(a, b, c, M, faces) ? w[i] : 0.0;
        }
        if (gu) gu[i] = 0.0;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Np; i += stride) {
        if (gphi) gphi[i] = 0.0;
        if (gm) gm[i] = 0.0;
    }
}

// K = n_sub + 1: level-set shape functions per direction on a velocity cell (Q1 on its n_sub sub-intervals).
// The interpolation of x and w, the value / gradient sensitivities and their testing run in double-float arithmetic
// (dfloat.cuh) on the FP32 pipe, with the coefficients of the double-float cache (the pairs of the FP64 values the
// forward apply uses); so do the material-law sensitivities of the interface-zone points, with the factors of the
// adjoint table.  The level-set test sweeps run in FP64 (only table cells carry them: blocks without a table cell skip
// the sweeps).
// Block shape for Q2 on the velocity mesh's level set: CB cells per block, at least MINB blocks per SM (a register
// cap).  Measured at 64^3 on GB300 (20 back-to-back adjoints, ms), with the zone sensitivities from the adjoint
// table: CB 7 / MINB 3 (96 registers, some spills) 1.962; 8 / 2 2.126; 7 / 2 2.150; 6 / 3 2.241; 4 / 4 2.301; with
// the cached coefficients copied into shared memory by cp.async during the interpolation sweeps, 7 / 3 1.853; with
// the lazy normalization below, 7 / 3 1.836, 8 / 2 1.974, 7 / 2 1.978.
// Before the table (zone work in FP64): 7 / 3 2.995; 8 / 2 3.158; 7 / 2 3.261; 4 / 4 3.403; 4 / 3 3.526.
// Normalization as in the forward double-float apply: the gradients at the points, the value sensitivities that
// start the test sums and the last transposed sweep (converted to FP64 next) are left unnormalized (0: normalize).
// Measured at 64^3: 1.856 -> 1.831 ms, the smoke case's gradients still within 5e-15 of the oracle's.
#ifndef EVAP_ADJ_LAZY
#define EVAP_ADJ_LAZY 1
#endif
template <int Q>
__device__ __forceinline__ dfl adj_dot_lazy(const dfl* c, const dfl* v, int stride) {
#if EVAP_ADJ_LAZY
    dfl s = df_prod(c[0], v[0]);
#pragma unroll
    for (int k = 1; k < Q; ++k) df_fma(s, c[k], v[k * stride]);
    return s;
#else
    return df_dot<Q>(c, v, stride);
#endif
}

#ifndef EVAP_ADJ_CB2
#define EVAP_ADJ_CB2 7
#endif
#ifndef EVAP_ADJ_MINB2
#define EVAP_ADJ_MINB2 3
#endif

template <int P, int CB, int K, int MINB = 2>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1), MINB)
    k_adjoint(MeshArgs<double> m, DfBasis dfb, Basis<double> bas, dfl rho_liq, dfl rho_gas,
              const int8_t* __restrict__ code, const int32_t* __restrict__ tindex, const float2* __restrict__ adjt,
              const float2* __restrict__ qcd, const double* __restrict__ w,
              const double* __restrict__ wp, const double* __restrict__ x, double* gx, double* gu, double* gphi,
              double* gm, int colour) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    static_assert(K * Q * Q <= NQ && K * K * K <= NQ, "one thread per entry of each level-set test sweep");
    __shared__ dfl sS[Q][Q], sDc[Q][Q];
    __shared__ double sNL[Q][K], sDL[Q][K];
    __shared__ dfl buf[2][CB][12][NQ];
    __shared__ double q1a[CB][5][K * Q * Q], q1b[CB][5][K * K * Q];  // level-set test sweeps (FP64)
    extern __shared__ float2 sqc[];  // [cell][QC_K][point]: this block's cached coefficients, copied during the sweeps
    const int tid = threadIdx.x;
    const int lc = tid / NQ, t = tid % NQ;
    int cx = 0, cy = 0, cz = 0;
    const bool active = colour_cell((int64_t)blockIdx.x * CB + lc, m.n, colour, cx, cy, cz);
    const int64_t cell = cx + (int64_t)m.n * (cy + (int64_t)m.n * cz);
    const bool plain = colour >= 0;  // a colour pass: no other cell of the launch touches this cell's nodes
    float2* myq = sqc + (int64_t)lc * QC_K * NQ + t;
    if (active) {  // each thread fetches (and later reads) only its own point's coefficients: 0..3, 13, 17, newton 4..12
        const float2* src = qcd + cell * QC_K * NQ + t;
#pragma unroll
        for (int k = 0; k < QC_K; ++k)
            if (k < 4 || k == 13 || k == 17 || (m.newton && k <= 12)) cp_async8(myq + k * NQ, src + k * NQ);
    }
    cp_async_commit();
    if (tid < Q * Q) {
        sS[tid / Q][tid % Q] = dfb.S[tid / Q][tid % Q];
        sDc[tid / Q][tid % Q] = dfb.Dc[tid / Q][tid % Q];
    }
    if (tid < K * Q) {
        sNL[tid / K][tid % K] = bas.NL[tid / K][tid % K];
        sDL[tid / K][tid % K] = bas.DL[tid / K][tid % K];
    }
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    const int n = m.n, M = m.M;
    const int64_t m1 = n + 1;     // pressure nodes per axis (w_p)
    const int64_t ml = m.nl + 1;  // level-set nodes per axis
    int64_t gidx = 0;
    bool cons = false, tcell = false;
    if (active) {
        const int gxi = P * cx + a, gyi = P * cy + b, gzi = P * cz + c;
        gidx = gxi + (int64_t)M * (gyi + (int64_t)M * gzi);
        cons = cons_node(gxi, gyi, gzi, M, m.faces);
        tcell = code[cell] == CELL_TABLE;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            buf[0][lc][k][t] = cons ? dfl{0.f, 0.f} : df_from_double(x[k * m.Nu + gidx]);
            buf[0][lc][3 + k][t] = cons ? dfl{0.f, 0.f} : df_from_double(w[k * m.Nu + gidx]);
        }
    }
    // whether any cell of the block carries level-set sensitivities (a table cell)
    const bool block_table = __syncthreads_or(tcell) != 0;
    if (active) {
        dfl Sa[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Sa[k] = sS[a][k];
#pragma unroll
        for (int f = 0; f < 6; ++f) buf[1][lc][f][t] = df_dot<Q>(Sa, &buf[0][lc][f][Q * (b + Q * c)], 1);
    }
    __syncthreads();
    if (active) {
        dfl Sb[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Sb[k] = sS[b][k];
#pragma unroll
        for (int f = 0; f < 6; ++f) buf[0][lc][f][t] = df_dot<Q>(Sb, &buf[1][lc][f][a + Q * Q * c], Q);
    }
    __syncthreads();
    if (active) {
        dfl Sc[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Sc[k] = sS[c][k];
#pragma unroll
        for (int f = 0; f < 6; ++f) buf[1][lc][f][t] = df_dot<Q>(Sc, &buf[0][lc][f][a + Q * b], Q * Q);
    }
    __syncthreads();
    dfl gxv[3], guv[3], gxg[3][3], gug[3][3];
    double dphi = 0.0, dg[3] = {0, 0, 0}, dm = 0.0;
    if (active) {
        dfl V[6], Gr[6][3];
        {
            dfl Da[Q], Db[Q], Dz[Q];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                Da[k] = sDc[a][k];
                Db[k] = sDc[b][k];
                Dz[k] = sDc[c][k];
            }
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                V[f] = buf[1][lc][f][t];
                Gr[f][0] = adj_dot_lazy<Q>(Da, &buf[1][lc][f][Q * (b + Q * c)], 1);
                Gr[f][1] = adj_dot_lazy<Q>(Db, &buf[1][lc][f][a + Q * Q * c], Q);
                Gr[f][2] = adj_dot_lazy<Q>(Dz, &buf[1][lc][f][a + Q * b], Q * Q);
            }
        }
        const dfl* X = &V[0];
        const dfl* Om = &V[3];
        dfl (*G)[3] = &Gr[0];
        dfl (*OmG)[3] = &Gr[3];
        // cached coefficients (k_qp_coeffs): 0 W rho c_m, 1..3 W rho u0, 4..12 newton W rho grad u0, 13 2 W mu, 17 W
        cp_async_wait_all();
        const float2* qp = myq;
        const dfl W = ld_df(qp + 17 * NQ);
        // this point's entries of the adjoint table (table cells only; k_fill_table)
        const float2* ap = tcell ? adjt + (int64_t)tindex[cell] * ADJ_K * NQ + t : nullptr;
        const dfl rho = tcell ? ld_df(ap + ADJ_RHO * NQ) : (code[cell] == CELL_LIQUID ? rho_liq : rho_gas);
        const dfl wr = df_mul(W, rho);  // the W rho of the forward apply
        // w_p (pressure space, Q1 on the cell) and the level set (its own mesh; only in table cells) at the point
        const double tx = bas.t[a], ty = bas.t[b], tz = bas.t[c];
        double pi = 0;
        if (wp) {  // trilinear interpolation by successive linear interpolation (14 FP64 operations, not 40)
            const double* w0 = wp + cx + m1 * (cy + m1 * cz);
            double e[2][2];
#pragma unroll
            for (int jc = 0; jc < 2; ++jc)
#pragma unroll
                for (int jb = 0; jb < 2; ++jb) {
                    const double* r = w0 + m1 * (jb + m1 * jc);
                    e[jc][jb] = fma(tx, r[1] - r[0], r[0]);
                }
            const double f0 = fma(ty, e[0][1] - e[0][0], e[0][0]), f1 = fma(ty, e[1][1] - e[1][0], e[1][0]);
            pi = fma(tz, f1 - f0, f0);
        }
        // the phi / mdot sensitivities and the normal are needed only in the interface zone (or with the correction
        // applied everywhere), which lies in table cells; elsewhere H is 0 or 1 and its derivatives vanish
        const bool full = tcell && (ap[ADJ_ZONE * NQ].x != 0.f || (m.stress != 0 && m.corr_zone != 0));
        const dfl wm = ld_df(qp + 13 * NQ);
        const dfl hwm = df_scale2(wm, 0.5f);
        const dfl Wpi = df_mul(W, df_from_double(pi));
        // value / gradient sensitivities of the velocity block and of B^T w_p (the correction term added below)
        const dfl c0 = ld_df(qp);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            dfl v = df_prod(c0, Om[d]);
            if (m.newton) {
#pragma unroll
                for (int k = 0; k < 3; ++k) df_fma(v, Om[k], ld_df(qp + (4 + 3 * k + d) * NQ));
            }
            gxv[d] = EVAP_ADJ_LAZY ? v : df_norm(v);
            dfl u = df_prod(Om[0], G[0][d]);
            df_fma(u, Om[1], G[1][d]);
            df_fma(u, Om[2], G[2][d]);
            guv[d] = df_mul(wr, df_norm(u));
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                dfl g = df_prod(Om[d], ld_df(qp + (1 + e) * NQ));
                df_fma(g, hwm, df_add(OmG[d][e], OmG[e][d]));
                gxg[d][e] = d == e ? df_add(df_norm(g), Wpi) : df_norm(g);
                gug[d][e] = m.newton ? df_mul(wr, df_mul(Om[d], X[e])) : dfl{0.f, 0.f};
            }
        }
        if (full) {  // material-law sensitivities (interface-zone points only), double-float arithmetic
            const dfl nv[3] = {ld_df(ap + (ADJ_N + 0) * NQ), ld_df(ap + (ADJ_N + 1) * NQ), ld_df(ap + (ADJ_N + 2) * NQ)};
            const bool zg = ap[ADJ_ZG * NQ].x != 0.f;
            const dfl tr = df_add(df_add(G[0][0], G[1][1]), G[2][2]);
            // OmG n, OmG^T n and n . OmG n
            dfl on[3], otn[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                dfl u = df_prod(OmG[i][0], nv[0]), v = df_prod(OmG[0][i], nv[0]);
#pragma unroll
                for (int j = 1; j < 3; ++j) {
                    df_fma(u, OmG[i][j], nv[j]);
                    df_fma(v, OmG[j][i], nv[j]);
                }
                on[i] = df_norm(u);
                otn[i] = df_norm(v);
            }
            dfl nOn = df_prod(nv[0], on[0]);
            df_fma(nOn, nv[1], on[1]);
            df_fma(nOn, nv[2], on[2]);
            nOn = df_norm(nOn);
            if (zg) {  // the corrected strain's term of g_x
                const dfl corr = df_mul(wm, nOn);
#pragma unroll
                for (int d = 0; d < 3; ++d) gxg[d][d] = df_sub(gxg[d][d], corr);
            }
            // dL/drho = W Om . (c_m X + G u0 + newton grad u0 X) = (1/rho) sum_k Om_k (cached W rho terms)_k
            const dfl U[3] = {ld_df(qp + 1 * NQ), ld_df(qp + 2 * NQ), ld_df(qp + 3 * NQ)};
            dfl sr{0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                dfl f = df_prod(c0, X[k]);
#pragma unroll
                for (int b2 = 0; b2 < 3; ++b2) df_fma(f, U[b2], G[k][b2]);
                if (m.newton) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) df_fma(f, ld_df(qp + (4 + 3 * k + d) * NQ), X[d]);
                }
                if (k == 0)
                    sr = df_prod(Om[0], df_norm(f));
                else
                    df_fma(sr, Om[k], df_norm(f));
            }
            const dfl dL_drho = df_mul(ld_df(ap + ADJ_IRHO * NQ), df_norm(sr));
            // dL/dmu = 2 W (OmG : sym G - z tr(G) n . OmG n)
            dfl smu = df_prod(OmG[0][0], G[0][0]);
            df_fma(smu, OmG[1][1], G[1][1]);
            df_fma(smu, OmG[2][2], G[2][2]);
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int l = k + 1; l < 3; ++l)
                    df_fma(smu, df_add(OmG[k][l], OmG[l][k]), df_scale2(df_add(G[k][l], G[l][k]), 0.5f));
            if (zg) df_fma(smu, df_neg(tr), nOn);
            const dfl dL_dmu = df_mul(df_scale2(W, 2.0f), df_norm(smu));
            // dL/dn = -2 W mu z tr(G) (OmG + OmG^T) n; its part normal to n drops out (dn/dgrad phi)
            dfl dLdn[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            if (zg) {
                const dfl wtr = df_neg(df_mul(wm, tr));
#pragma unroll
                for (int i = 0; i < 3; ++i) dLdn[i] = df_mul(wtr, df_add(on[i], otn[i]));
            }
            dfl dp = df_prod(dL_drho, ld_df(ap + ADJ_CRHO * NQ));
            df_fma(dp, dL_dmu, ld_df(ap + ADJ_CMU * NQ));
            dfl pn = df_prod(dLdn[0], nv[0]);
            df_fma(pn, dLdn[1], nv[1]);
            df_fma(pn, dLdn[2], nv[2]);
            pn = df_neg(df_norm(pn));
            const dfl ign = ld_df(ap + ADJ_IGN * NQ);
            dfl dgv[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                dfl u = dLdn[i];
                df_fma(u, pn, nv[i]);
                dgv[i] = df_mul(df_norm(u), ign);
            }
            if (wp) {  // through v_dil = mdot c_1 delta (Eq. evaporDil), dL/dv_dil = -W pi
                const dfl dLdv = df_neg(Wpi);
                dm = df_to_double(df_mul(dLdv, ld_df(ap + ADJ_KD1 * NQ)));
                df_fma(dp, dLdv, ld_df(ap + ADJ_KD2 * NQ));
                const dfl k3 = df_mul(dLdv, ld_df(ap + ADJ_KD3 * NQ));
#pragma unroll
                for (int i = 0; i < 3; ++i) dgv[i] = df_add(dgv[i], df_mul(k3, nv[i]));
            }
            dphi = df_to_double(df_norm(dp));
#pragma unroll
            for (int i = 0; i < 3; ++i) dg[i] = df_to_double(dgv[i]);
        }
    }
    __syncthreads();
    // level-set sensitivities (FP64) in the slots 6..10 of buf[1], stored as doubles (8 bytes like a dfl)
    auto lsv = [&](int f, int pt) -> double& { return *reinterpret_cast<double*>(&buf[1][lc][6 + f][pt]); };
    if (active) {
        for (int s = 0; s < 9; ++s) buf[0][lc][s][t] = gxg[s / 3][s % 3];
        for (int s = 0; s < 3; ++s) buf[0][lc][9 + s][t] = gug[0][s];
        for (int s = 0; s < 6; ++s) buf[1][lc][s][t] = gug[1 + s / 3][s % 3];
        lsv(0, t) = dphi;
        lsv(1, t) = dg[0];
        lsv(2, t) = dg[1];
        lsv(3, t) = dg[2];
        lsv(4, t) = dm;
    }
    __syncthreads();
    dfl tx3[3], tu3[3];
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
            const int ib = 3 * k;      // gxg[k][*] slots in buf[0]
            const int iu = 9 + 3 * k;  // gug[k][*] slots: 9..17 over buf[0][9..11], buf[1][0..5]
            dfl s = gxv[k], u = guv[k];
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                const int p0 = r + Q * (b + Q * c), p1 = a + Q * (r + Q * c), p2 = a + Q * (b + Q * r);
                df_fma(s, Ea[r], buf[0][lc][ib + 0][p0]);
                df_fma(s, Eb[r], buf[0][lc][ib + 1][p1]);
                df_fma(s, Ec[r], buf[0][lc][ib + 2][p2]);
                if (m.newton) {
                    const int j0 = iu + 0, j1 = iu + 1, j2 = iu + 2;
                    df_fma(u, Ea[r], j0 < 12 ? buf[0][lc][j0][p0] : buf[1][lc][j0 - 12][p0]);
                    df_fma(u, Eb[r], j1 < 12 ? buf[0][lc][j1][p1] : buf[1][lc][j1 - 12][p1]);
                    df_fma(u, Ec[r], j2 < 12 ? buf[0][lc][j2][p2] : buf[1][lc][j2 - 12][p2]);
                }
            }
            tx3[k] = df_norm(s);
            tu3[k] = df_norm(u);
        }
        // level-set sensitivities: g_phi[j] = sum_q N_j dL/dphi + grad N_j . dL/dgrad phi, g_mdot[j] = sum_q N_j
        // dL/dmdot with the level-set shape functions N_j of the cell (K per direction), by three sweeps; field f:
        // 0 dL/dphi, 1..3 dL/dgrad phi (x, y, z), 4 dL/dmdot.  Along direction d the 1D factor is the reference
        // derivative DL for field 1 + d, NL otherwise.  x-sweep: [jx][qy][qz].
        if (block_table && t < K * Q * Q) {
            const int jx = t % K, qy = (t / K) % Q, qz = (t / K) / Q;
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                double sacc = 0.0;
#pragma unroll
                for (int q = 0; q < Q; ++q) sacc += (f == 1 ? sDL[q][jx] : sNL[q][jx]) * lsv(f, q + Q * (qy + Q * qz));
                q1a[lc][f][t] = sacc;
            }
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            buf[0][lc][k][t] = tx3[k];
            buf[0][lc][3 + k][t] = tu3[k];
        }
        if (block_table && t < K * K * Q) {  // y-sweep: [jx][jy][qz]
            const int jx = t % K, jy = (t / K) % K, qz = t / (K * K);
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                double sacc = 0.0;
#pragma unroll
                for (int q = 0; q < Q; ++q)
                    sacc += (f == 2 ? sDL[q][jy] : sNL[q][jy]) * q1a[lc][f][jx + K * (q + Q * qz)];
                q1b[lc][f][t] = sacc;
            }
        }
    }
    __syncthreads();
    if (active && tcell && t < K * K * K) {  // z-sweep and scatter of level-set node (jx, jy, jz) of a table cell
        const int jx = t % K, jy = (t / K) % K, jz = t / (K * K);
        double r[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            double sacc = 0.0;
#pragma unroll
            for (int q = 0; q < Q; ++q) sacc += (f == 3 ? sDL[q][jz] : sNL[q][jz]) * q1b[lc][f][jx + K * (jy + K * q)];
            r[f] = sacc;
        }
        const int ks = K - 1;  // n_sub
        const int64_t nd = (ks * cx + jx) + ml * ((ks * cy + jy) + ml * (ks * cz + jz));
        if (gphi) acc_add(&gphi[nd], r[0] + m.inv_h * (r[1] + r[2] + r[3]), plain);
        if (gm) acc_add(&gm[nd], r[4], plain);
    }
    // transposed sweeps S^T of the 6 value fields (g_x, g_u0): z, y, x
    if (active) {
        dfl Tc[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Tc[k] = sS[k][c];
#pragma unroll
        for (int f = 0; f < 6; ++f) buf[1][lc][f][t] = df_dot<Q>(Tc, &buf[0][lc][f][a + Q * b], Q * Q);
    }
    __syncthreads();
    if (active) {
        dfl Tb[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Tb[k] = sS[k][b];
#pragma unroll
        for (int f = 0; f < 6; ++f) buf[0][lc][f][t] = df_dot<Q>(Tb, &buf[1][lc][f][a + Q * Q * c], Q);
    }
    __syncthreads();
    if (active) {
        dfl Ta[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) Ta[k] = sS[k][a];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const double s = df_to_double(adj_dot_lazy<Q>(Ta, &buf[0][lc][f][Q * (b + Q * c)], 1));
            if (f < 3) {
                if (gx && !cons) acc_add(&gx[f * m.Nu + gidx], s, plain);
            } else if (gu) {
                acc_add(&gu[(f - 3) * m.Nu + gidx], s, plain);
            }
        }
    }
}

int launch_adjoint(evap_mesh* h, const double* w, const double* wp, const double* x, double* gx, double* gu,
                   double* gphi, double* gm, cudaStream_t s) {
    const MeshArgs<double>& m = h->m;
    k_adjoint_init<<<blocks_for(3 * m.Nu, 256), 256, 0, s>>>(m.M, m.Nu, m.Nphi, m.faces, w, gx, gu, gphi, gm);  // level set
    EVAP_CHECK_LAUNCH("adjoint_init");
    const DfBasis dfb = make_df_basis(h->b, m.inv_h);
    const float2* qcd = reinterpret_cast<const float2*>(h->qcdf);
    const dfl rho_liq = df_from_double(m.rho_H1), rho_gas = df_from_double(m.rho_H0);  // rho outside table cells
    const int c0 = h->deterministic ? 0 : -1, c1 = h->deterministic ? 8 : 0;  // colour passes, or one atomic pass
    auto run = [&](auto kern, int CB, int threads) -> int {
        const size_t dyn = sizeof(float2) * QC_K * threads;  // the block's cached coefficients (threads = CB NQ)
        EVAP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        EVAP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared));
        for (int colour = c0; colour < std::max(c1, c0 + 1); ++colour) {
            const int64_t cells = colour_cells(m.n, colour);
            if (cells == 0) continue;
            kern<<<(unsigned)((cells + CB - 1) / CB), threads, dyn, s>>>(m, dfb, h->b, rho_liq, rho_gas, h->cell_code,
                                                                       h->table_index, h->adj_table, qcd, w, wp, x,
                                                                       gx, gu, gphi, gm, colour);
            EVAP_CHECK_LAUNCH("adjoint");
        }
        return EVAP_OK;
    };
    constexpr int CA = EVAP_ADJ_CB2, MA = EVAP_ADJ_MINB2;
    if (m.P == 2 && m.nsub == 1)  // 7 cells: 189 threads, 98 % of the lanes of 6 warps
        return run(k_adjoint<2, CA, 2, MA>, CA, CA * 27);
    if (m.P == 2)  // the subdivided level set's larger test-sweep buffers (static shared memory <= 48 KB)
        return run(k_adjoint<2, 6, 3>, 6, 6 * 27);
    if (m.nsub == 1) return run(k_adjoint<3, 2, 2>, 2, 2 * 64);
    return run(k_adjoint<3, 2, 3>, 2, 2 * 64);
}

}  // namespace evap
