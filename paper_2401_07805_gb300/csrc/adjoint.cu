// Adjoint of the momentum apply, FP64.  The u0 terms and the material coefficients come from the quadrature-point cache
// of set_fields (the same FP64 values the forward apply uses, so g_x is exactly its transpose); the material-law
// derivatives are recomputed from phi at the points of the interface zone.
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
template <int P, int CB, int K>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1), 2)
    k_adjoint(MeshArgs<double> m, Basis<double> bas, const double* __restrict__ phi, const double* __restrict__ mdot,
              const int8_t* __restrict__ code, const int32_t* __restrict__ tindex, const double* __restrict__ table,
              const double* __restrict__ qc, const double* __restrict__ w, const double* __restrict__ wp,
              const double* __restrict__ x, double* gx, double* gu, double* gphi, double* gm) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    static_assert(K * Q * Q <= NQ && K * K * K <= NQ, "one thread per entry of each level-set test sweep");
    __shared__ double sS[Q][Q], sDc[Q][Q], sN1[Q][2], sNL[Q][K], sDL[Q][K];
    __shared__ double buf[2][CB][12][NQ];
    __shared__ double q1a[CB][5][K * Q * Q], q1b[CB][5][K * K * Q];  // level-set test sweeps of the phi / mdot sensitivities
    const int tid = threadIdx.x;
    const int lc = tid / NQ, t = tid % NQ;
    const int64_t cell = (int64_t)blockIdx.x * CB + lc;
    const bool active = cell < m.ncell;
    if (tid < Q * Q) {
        sS[tid / Q][tid % Q] = bas.S[tid / Q][tid % Q];
        sDc[tid / Q][tid % Q] = bas.Dc[tid / Q][tid % Q] * m.inv_h;  // physical collocation derivative
    }
    if (tid < 2 * Q) sN1[tid / 2][tid % 2] = bas.N1[tid / 2][tid % 2];
    if (tid < K * Q) {
        sNL[tid / K][tid % K] = bas.NL[tid / K][tid % K];
        sDL[tid / K][tid % K] = bas.DL[tid / K][tid % K];
    }
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    const int n = m.n, M = m.M;
    const int64_t m1 = n + 1;       // pressure nodes per axis (w_p)
    const int64_t ml = m.nl + 1;    // level-set nodes per axis
    int cx = 0, cy = 0, cz = 0;
    int64_t gidx = 0;
    bool cons = false;
    if (active) {
        cx = (int)(cell % n);
        cy = (int)((cell / n) % n);
        cz = (int)(cell / ((int64_t)n * n));
        const int gxi = P * cx + a, gyi = P * cy + b, gzi = P * cz + c;
        gidx = gxi + (int64_t)M * (gyi + (int64_t)M * gzi);
        cons = cons_node(gxi, gyi, gzi, M, m.faces);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            buf[0][lc][k][t] = cons ? 0.0 : x[k * m.Nu + gidx];
            buf[0][lc][3 + k][t] = cons ? 0.0 : w[k * m.Nu + gidx];
        }
    }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            double s = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s += sS[a][k] * buf[0][lc][f][k + Q * (b + Q * c)];
            buf[1][lc][f][t] = s;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            double s = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s += sS[b][k] * buf[1][lc][f][a + Q * (k + Q * c)];
            buf[0][lc][f][t] = s;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            double s = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) s += sS[c][k] * buf[0][lc][f][a + Q * (b + Q * k)];
            buf[1][lc][f][t] = s;
        }
    __syncthreads();
    double gxv[3] = {0, 0, 0}, guv[3] = {0, 0, 0}, gxg[3][3] = {}, gug[3][3] = {};
    double dphi = 0.0, dg[3] = {0, 0, 0}, dm = 0.0;
    if (active) {
        double V[6], Gr[6][3];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            V[f] = buf[1][lc][f][t];
            double g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                g0 += sDc[a][r] * buf[1][lc][f][r + Q * (b + Q * c)];
                g1 += sDc[b][r] * buf[1][lc][f][a + Q * (r + Q * c)];
                g2 += sDc[c][r] * buf[1][lc][f][a + Q * (b + Q * r)];
            }
            Gr[f][0] = g0; Gr[f][1] = g1; Gr[f][2] = g2;  // sDc holds the physical derivative (1/h folded in)
        }
        const double* X = &V[0];
        const double* Om = &V[3];
        double (*G)[3] = &Gr[0];
        double (*OmG)[3] = &Gr[3];
        // cached coefficients (k_qp_coeffs): 0 W rho c_m, 1..3 W rho u0, 4..12 newton W rho grad u0, 13 2 W mu, 17 W
        double qv[QC_K];
        {
            const double* qp = qc + cell * QC_K * NQ + t;
#pragma unroll
            for (int k = 0; k < QC_K; ++k) qv[k] = (k >= 14 && k <= 16) || k == 18 ? 0.0 : qp[k * NQ];
        }
        const double W = qv[17];
        const int8_t cc = code[cell];
        const bool tcell = cc == CELL_TABLE;
        const double rho_c = tcell ? table[(int64_t)tindex[cell] * TAB_K * NQ + t]
                                   : (cc == CELL_LIQUID ? m.rho_H1 : m.rho_H0);
        const double wr = W * rho_c;  // the W rho of the forward apply
        // w_p (pressure space, Q1 on the cell) and the level set (its own, possibly subdivided, mesh; only in table
        // cells) at the point
        const double tx = bas.t[a], ty = bas.t[b], tz = bas.t[c];
        double ph = 0, pi = 0;
        if (wp) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int ja = j & 1, jb = (j >> 1) & 1, jc = j >> 2;
                const int64_t nd = (cx + ja) + m1 * ((cy + jb) + m1 * (cz + jc));
                pi += (ja ? tx : 1.0 - tx) * (jb ? ty : 1.0 - ty) * (jc ? tz : 1.0 - tz) * wp[nd];
            }
        }
        double gp[3] = {0, 0, 0}, md = 0.0;
        if (tcell) ls_at(phi, m, cx, cy, cz, tx, ty, tz, ph, gp);
        // the phi / mdot sensitivities and the normal are needed only in the interface zone (or with the correction
        // applied everywhere), which lies in table cells; elsewhere H is 0 or 1 and its derivatives vanish
        const bool zone = tcell && fabs(ph) < PHI_BAND;
        const bool full = zone || (tcell && m.stress != 0 && m.corr_zone != 0);
        const double nw = m.newton ? 1.0 : 0.0;
        Material mat;
        if (full) {
            double gm_[3];
            ls_at(mdot, m, cx, cy, cz, tx, ty, tz, md, gm_);
            mat = material(ph, gp[0], gp[1], gp[2], m);
        }
        const double wm = qv[13];
        // value / gradient sensitivities of the velocity block and of B^T w_p (the correction term added below)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            gxv[d] = qv[0] * Om[d] + Om[0] * qv[4 + d] + Om[1] * qv[7 + d] + Om[2] * qv[10 + d];
            guv[d] = wr * (Om[0] * G[0][d] + Om[1] * G[1][d] + Om[2] * G[2][d]);
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                gxg[d][e] = Om[d] * qv[1 + e] + wm * 0.5 * (OmG[d][e] + OmG[e][d]) + (d == e ? W * pi : 0.0);
                gug[d][e] = nw * wr * Om[d] * X[e];
            }
        }
        if (full) {
            const double rho = mat.rho;
            const double zg = correction_on(m, mat.zone) ? 1.0 : 0.0;
            const double* nv = mat.n;
            const double tr = G[0][0] + G[1][1] + G[2][2];
            double nOn = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) nOn += nv[i] * OmG[i][j] * nv[j];
#pragma unroll
            for (int d = 0; d < 3; ++d) gxg[d][d] -= wm * zg * nOn;
            double dH = 0.0, d2H = 0.0, dd = 0.0, d2d = 0.0;
            if (mat.zone) {
                const double dist = m.eps * log((1.0 + ph) / (1.0 - ph));
                double sn, cs;
                sincos(PI * dist / (3.0 * m.eps), &sn, &cs);
                dH = (1.0 + cs) / (6.0 * m.eps);
                d2H = -PI * sn / (18.0 * m.eps * m.eps);
                const double om = 1.0 - ph * ph;
                dd = 2.0 * m.eps / om;
                d2d = 4.0 * m.eps * ph / (om * om);
            }
            // coefficient sensitivities; u0 and newton grad u0 from the cached W rho u0 / (W rho)
            const double iwr = 1.0 / wr;
            double dL_drho = 0.0, dL_dmu = 0.0, dL_dn[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double Fk = m.c_mass * X[k] +
                                  (qv[1] * G[k][0] + qv[2] * G[k][1] + qv[3] * G[k][2] + qv[4 + 3 * k] * X[0] +
                                   qv[5 + 3 * k] * X[1] + qv[6 + 3 * k] * X[2]) * iwr;
                dL_drho += Om[k] * Fk;
#pragma unroll
                for (int l = 0; l < 3; ++l)
                    dL_dmu += OmG[k][l] * (0.5 * (G[k][l] + G[l][k]) - zg * tr * nv[k] * nv[l]);
            }
            dL_drho *= W;
            dL_dmu *= 2.0 * W;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                double sacc = 0.0;
#pragma unroll
                for (int j = 0; j < 3; ++j) sacc += (OmG[i][j] + OmG[j][i]) * nv[j];
                dL_dn[i] = -wm * zg * tr * sacc;
            }
            const double krho = 1.0 / m.rho_l - 1.0 / m.rho_g;  // d(1/rho)/dH, Eq. (rhoEff)
            const double drho_dH = -rho * rho * krho;
            const double dmu_dH = m.mu_l - m.mu_g;
            dphi = (dL_drho * drho_dH + dL_dmu * dmu_dH) * dH * dd;
            const double gn = sqrt(gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2]);
            if (gn * m.h > GRAD_TINY) {
                const double pn = dL_dn[0] * nv[0] + dL_dn[1] * nv[1] + dL_dn[2] * nv[2];
#pragma unroll
                for (int i = 0; i < 3; ++i) dg[i] = (dL_dn[i] - pn * nv[i]) / gn;
            }
            if (wp) {  // through v_dil = mdot c_1 delta (Eq. evaporDil)
                const double kdil = dilation_coefficient(m);
                const double dL_dv = -W * pi;
                const double delta = mat.zone ? dH * dd * gn : 0.0;
                dm = dL_dv * kdil * delta;
                dphi += dL_dv * md * kdil * (d2H * dd * dd + dH * d2d) * gn;
#pragma unroll
                for (int i = 0; i < 3; ++i) dg[i] += dL_dv * md * kdil * dH * dd * nv[i];
            }
        }
    }
    __syncthreads();
    if (active) {
        for (int s = 0; s < 9; ++s) buf[0][lc][s][t] = gxg[s / 3][s % 3];
        for (int s = 0; s < 3; ++s) buf[0][lc][9 + s][t] = gug[0][s];
        for (int s = 0; s < 6; ++s) buf[1][lc][s][t] = gug[1 + s / 3][s % 3];
        buf[1][lc][6][t] = dphi;
        buf[1][lc][7][t] = dg[0];
        buf[1][lc][8][t] = dg[1];
        buf[1][lc][9][t] = dg[2];
        buf[1][lc][10][t] = dm;
    }
    __syncthreads();
    double tx3[3], tu3[3];
    if (active) {
        for (int k = 0; k < 3; ++k) {
            double s0 = 0, s1 = 0, s2 = 0, u0s = 0, u1s = 0, u2s = 0;
            const int ib = 3 * k;       // gxg[k][*] slots in buf[0]
            const int iu = 9 + 3 * k;   // gug[k][*] slots: 9..17 over buf[0][9..11], buf[1][0..5]
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                const int p0 = r + Q * (b + Q * c), p1 = a + Q * (r + Q * c), p2 = a + Q * (b + Q * r);
                s0 += sDc[r][a] * buf[0][lc][ib + 0][p0];
                s1 += sDc[r][b] * buf[0][lc][ib + 1][p1];
                s2 += sDc[r][c] * buf[0][lc][ib + 2][p2];
                const int j0 = iu + 0, j1 = iu + 1, j2 = iu + 2;
                u0s += sDc[r][a] * (j0 < 12 ? buf[0][lc][j0][p0] : buf[1][lc][j0 - 12][p0]);
                u1s += sDc[r][b] * (j1 < 12 ? buf[0][lc][j1][p1] : buf[1][lc][j1 - 12][p1]);
                u2s += sDc[r][c] * (j2 < 12 ? buf[0][lc][j2][p2] : buf[1][lc][j2 - 12][p2]);
            }
            tx3[k] = gxv[k] + (s0 + s1 + s2);
            tu3[k] = guv[k] + (u0s + u1s + u2s);
        }
        // level-set sensitivities: g_phi[j] = sum_q N_j dL/dphi + grad N_j . dL/dgrad phi, g_mdot[j] = sum_q N_j
        // dL/dmdot with the level-set shape functions N_j of the cell (K per direction), by three sweeps; field f:
        // 0 dL/dphi, 1..3 dL/dgrad phi (x, y, z), 4 dL/dmdot.  Along direction d the 1D factor is the reference
        // derivative DL for field 1 + d, NL otherwise.  x-sweep: [jx][qy][qz].
        if (t < K * Q * Q) {
            const int jx = t % K, qy = (t / K) % Q, qz = (t / K) / Q;
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                double sacc = 0.0;
#pragma unroll
                for (int q = 0; q < Q; ++q)
                    sacc += (f == 1 ? sDL[q][jx] : sNL[q][jx]) * buf[1][lc][6 + f][q + Q * (qy + Q * qz)];
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
        if (t < K * K * Q) {  // y-sweep: [jx][jy][qz]
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
    if (active && t < K * K * K) {  // z-sweep and scatter of level-set node (jx, jy, jz) of the cell
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
        if (gphi) atomicAdd(&gphi[nd], r[0] + m.inv_h * (r[1] + r[2] + r[3]));
        if (gm) atomicAdd(&gm[nd], r[4]);
    }
    if (active)
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            double s = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) s += sS[q][c] * buf[0][lc][f][a + Q * (b + Q * q)];
            buf[1][lc][f][t] = s;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            double s = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) s += sS[q][b] * buf[1][lc][f][a + Q * (q + Q * c)];
            buf[0][lc][f][t] = s;
        }
    __syncthreads();
    if (active)
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            double s = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) s += sS[q][a] * buf[0][lc][f][q + Q * (b + Q * c)];
            if (f < 3) {
                if (gx && !cons) atomicAdd(&gx[f * m.Nu + gidx], s);
            } else if (gu) {
                atomicAdd(&gu[(f - 3) * m.Nu + gidx], s);
            }
        }
}

int launch_adjoint(evap_mesh* h, const double* w, const double* wp, const double* x, double* gx, double* gu,
                   double* gphi, double* gm, cudaStream_t s) {
    const MeshArgs<double>& m = h->m;
    k_adjoint_init<<<blocks_for(3 * m.Nu, 256), 256, 0, s>>>(m.M, m.Nu, m.Nphi, m.faces, w, gx, gu, gphi, gm);  // level set
    EVAP_CHECK_LAUNCH("adjoint_init");
    if (m.P == 2 && m.nsub == 1) {
        constexpr int CB = 7;  // 189 threads: 98 % of the lanes of 6 warps (4 cells: 108 threads, 84 %)
        k_adjoint<2, CB, 2><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 27, 0, s>>>(
            m, h->b, h->phi, h->mdot, h->cell_code, h->table_index, h->table, h->qc, w, wp, x, gx, gu, gphi, gm);
    } else if (m.P == 2) {
        constexpr int CB = 6;  // the subdivided level set's larger test-sweep buffers (static shared memory <= 48 KB)
        k_adjoint<2, CB, 3><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 27, 0, s>>>(
            m, h->b, h->phi, h->mdot, h->cell_code, h->table_index, h->table, h->qc, w, wp, x, gx, gu, gphi, gm);
    } else if (m.nsub == 1) {
        constexpr int CB = 2;
        k_adjoint<3, CB, 2><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 64, 0, s>>>(
            m, h->b, h->phi, h->mdot, h->cell_code, h->table_index, h->table, h->qc, w, wp, x, gx, gu, gphi, gm);
    } else {
        constexpr int CB = 2;
        k_adjoint<3, CB, 3><<<(unsigned)((m.ncell + CB - 1) / CB), CB * 64, 0, s>>>(
            m, h->b, h->phi, h->mdot, h->cell_code, h->table_index, h->table, h->qc, w, wp, x, gx, gu, gphi, gm);
    }
    EVAP_CHECK_LAUNCH("adjoint");
    return EVAP_OK;
}

}  // namespace evap
