// FP32 momentum apply (the inner operator of the mixed-precision solve), line-oriented sum factorization.
//
// Same operator as k_momentum (velocity block of Eq. weakNavierStokes linearized about u0, App. D, corrected stress
// of Eq. modified_viscous_stress, divergence row of Eq. continuity), evaluated in FP32 with the material law from the
// FP32 copy of the FP64 interface table.  The FP32 pipe is 60x faster than FP64 on GB300, so here the limit is the
// load/store unit, not arithmetic; the kernel is laid out to move few operands through shared memory:
//   * (P+1)^2 threads per cell, each owning one line of points; the 1D matrices are kernel parameters indexed at
//     compile time (constant-bank operands, no loads);
//   * the cell index is the fastest thread index (a warp holds the same line of 32 consecutive cells) and shared
//     memory is laid out [slot][cell], so every shared access of a warp touches consecutive words (no bank
//     conflicts), the gather and the scatter of a warp walk along x, and the cell codes load coalesced;
//   * values and gradients by the sweep tree: z-line S and D (registers) -> y-line S, D on S-output and S on
//     D-output -> x-line S, D, S, S: every sweep reads and writes whole lines (no collocation derivative, whose
//     cross-line reads would cost Q loads per point and direction);
//   * the u0 terms come from the quadrature-point cache of set_fields (k_qp_coeffs), rounded to FP32 (W rho u0 and
//     newton W rho grad u0, 12 floats per point) in a layout [block][k][point][cell] that a warp reads as one
//     128-byte line: interpolating u0 on the fly would double the sweep work, the shared-memory traffic and the registers;
//   * the testing runs the tree backwards (x-line S^T/D^T in registers, then y-lines, then z-lines and the atomic
//     scatter); four block barriers per batch of cells.
#include "evap_internal.cuh"

namespace evap {

// Mesh-size factors of the reference-derivative formulation (the 1D tables are compile-time, for the unit cell):
// gradients are computed with D_ref = h D, so the kernel carries the powers of h instead.
struct Scale32 {
    float h2, h3;  // W = w_q h^3 (weights); the divergence row W (tr G - v) = w_q (h^2 tr G_ref - h^3 v)
    float c2h;     // viscous flux tested with D: 2 W mu (sym G - ...) / h = w_q mu (2 h) (sym G_ref - ...) / h^2 * h^2
    float hcm;     // mass term: W rho c_m = w_q rho (h^3 c_m)
};


// blocks per SM for Q2 (a register cap): measured at 64^3 (100 applies, ms) 3 blocks (72 registers) 0.145, 2 (90)
// 0.171, 4 (56, spills) 0.222
#ifndef EVAP_M32_MINB2
#define EVAP_M32_MINB2 3
#endif

template <int P, int CB, int MINB, bool DET>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1), MINB)
    k_momentum32(MeshArgs<float> m, Scale32 hs, const int8_t* __restrict__ code,
                 const int32_t* __restrict__ tindex, const float* __restrict__ table, const float* __restrict__ qc32,
                 const float* __restrict__ x, float* __restrict__ y, float* __restrict__ yp, int colour) {
    static_assert(CB == 32, "the qc32 layout is for 32-cell blocks");
    constexpr int Q = P + 1, NQ = Q * Q * Q, L = Q * Q;
    constexpr int OFF_Z = 3 * NQ, OFF_Y = 6 * NQ, OFF_PD = 9 * NQ, OFF_QD = OFF_PD + 2 * L;
    constexpr int CS = OFF_QD + 4 * Q;  // slots per cell
    const CtBasis<P>& B = kCtBasis<P>;  // S, D (reference), N1, w: immediates after unrolling
    __shared__ float sm[CS * CB];      // slot s of cell lc at sm[s * CB + lc]
    const int tid = threadIdx.x;
    const int lc = tid % CB, l = tid / CB;
    const int n = m.n, M = m.M;
    // A block holds CB consecutive cells of one x-row: (cx, cy, cz) = (CB * xb + lc, row % n, row / n).  In a colour
    // pass (DET, colour = pb + 2 py + 4 pz) the blocks with xb = pb mod 2 of the rows with cy = py, cz = pz mod 2:
    // two such blocks share no node, and inside a block the even cells scatter before the odd ones.  The atomic
    // variant (DET false) is compiled apart: it ignores colour and adds each result as soon as it is formed.
    const int nxc = (n + CB - 1) / CB;
    int cx, cy, cz;
    int64_t cell;
    bool active;
    if constexpr (!DET) {
        const int row = (int)(blockIdx.x / (unsigned)nxc);
        cx = ((int)blockIdx.x - row * nxc) * CB + lc;
        cy = row % n;
        cz = row / n;
        cell = cx + (int64_t)n * row;
        active = cx < n;
    } else {
        const int pb = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
        const int hy = (n - py + 1) >> 1, hxb = (nxc - pb + 1) >> 1;
        const int rowc = (int)(blockIdx.x / (unsigned)hxb);
        const int xb = 2 * ((int)blockIdx.x - rowc * hxb) + pb;
        cx = xb * CB + lc;
        cy = 2 * (rowc % hy) + py;
        cz = 2 * (rowc / hy) + pz;
        cell = cx + (int64_t)n * (cy + (int64_t)n * cz);
        active = cx < n;
    }
    float* cs = sm + lc;
    auto S_ = [cs](int slot) -> float& { return cs[slot * CB]; };
    auto at = [](int z, int yy, int xx) { return xx + Q * (yy + Q * z); };
    // Nodes of this thread's z-line (gx, gy, P cz + k) and whether each is a free (unconstrained) DoF.
    const int64_t MM = (int64_t)M * M;
    int64_t zbase;
    bool keep[Q];
    {
        const int i = l % Q, j = l / Q;
        const int gx = P * cx + i, gy = P * cy + j, gz0 = P * cz;
        const unsigned fc = m.faces;
        const bool cxy = ((fc & 1u) && gx == 0) || ((fc & 2u) && gx == M - 1) || ((fc & 4u) && gy == 0) ||
                         ((fc & 8u) && gy == M - 1);
#pragma unroll
        for (int k = 0; k < Q; ++k)
            keep[k] = !(cxy || ((fc & 16u) && gz0 + k == 0) || ((fc & 32u) && gz0 + k == M - 1));
        zbase = gx + (int64_t)M * gy + MM * gz0;
    }
    // ---------------------------------------------------------------- z-lines: gather, S and D along z
    {
        const int i = l % Q, j = l / Q;
        if (active) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                float v[Q];
                const float* src = x + f * m.Nu + zbase;
#pragma unroll
                for (int k = 0; k < Q; ++k) v[k] = keep[k] ? src[k * MM] : 0.f;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    float a = 0.f, d = 0.f;
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        a += (float)B.S[q][k] * v[k];
                        d += (float)B.D[q][k] * v[k];
                    }
                    S_(f * NQ + at(q, j, i)) = a;
                    S_(OFF_Z + f * NQ + at(q, j, i)) = d;
                }
            }
        }
    }
    __syncthreads();
    // ---------------------------------------------------------------- y-lines: S, D on A; S on Az
    {
        const int i = l % Q, qz = l / Q;
        if (active) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                float a[Q], az[Q];
#pragma unroll
                for (int jj = 0; jj < Q; ++jj) {
                    a[jj] = S_(f * NQ + at(qz, jj, i));
                    az[jj] = S_(OFF_Z + f * NQ + at(qz, jj, i));
                }
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    float bs = 0.f, bd = 0.f, bz = 0.f;
#pragma unroll
                    for (int jj = 0; jj < Q; ++jj) {
                        bs += (float)B.S[q][jj] * a[jj];
                        bd += (float)B.D[q][jj] * a[jj];
                        bz += (float)B.S[q][jj] * az[jj];
                    }
                    S_(f * NQ + at(qz, q, i)) = bs;
                    S_(OFF_Y + f * NQ + at(qz, q, i)) = bd;
                    S_(OFF_Z + f * NQ + at(qz, q, i)) = bz;
                }
            }
        }
    }
    __syncthreads();
    // ---------------------------------------------------------------- x-lines: points, fluxes, x-line testing
    {
        const int qy = l % Q, qz = l / Q;
        if (active) {
            float bs[3][Q], by[3][Q], bz[3][Q];
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int ii = 0; ii < Q; ++ii) {
                    bs[f][ii] = S_(f * NQ + at(qz, qy, ii));
                    by[f][ii] = S_(OFF_Y + f * NQ + at(qz, qy, ii));
                    bz[f][ii] = S_(OFF_Z + f * NQ + at(qz, qy, ii));
                }
            const int8_t cc = code[cell];
            const float* tb = cc == CELL_TABLE ? table + (int64_t)tindex[cell] * TAB_K * NQ : nullptr;
            // the cache's block of 32 x-consecutive cells holding this cell, and its place in it
            const int64_t cblk = DET ? (int64_t)(cy + n * cz) * nxc + cx / CB : (int64_t)blockIdx.x;
            const float* cq = qc32 + cblk * QC32_K * NQ * 32 + (DET ? cx % CB : lc);
            const float wyz = B.wf[qy] * B.wf[qz];
            float Pv[3][Q], Py[3][Q], Pz[3][Q], Pd[2];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int ii = 0; ii < Q; ++ii) Pv[c][ii] = Py[c][ii] = Pz[c][ii] = 0.f;
            Pd[0] = Pd[1] = 0.f;
#pragma unroll
            for (int qx = 0; qx < Q; ++qx) {
                float X[3], G[3][3];
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    float v = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
                    for (int ii = 0; ii < Q; ++ii) {
                        v += (float)B.S[qx][ii] * bs[f][ii];
                        gx += (float)B.D[qx][ii] * bs[f][ii];
                        gy += (float)B.S[qx][ii] * by[f][ii];
                        gz += (float)B.S[qx][ii] * bz[f][ii];
                    }
                    X[f] = v; G[f][0] = gx; G[f][1] = gy; G[f][2] = gz;
                }
                float rho, mu, nz[3], vd;
                const int qi = at(qz, qy, qx);
                if (tb) {
                    rho = tb[qi]; mu = tb[NQ + qi]; nz[0] = tb[2 * NQ + qi]; nz[1] = tb[3 * NQ + qi];
                    nz[2] = tb[4 * NQ + qi]; vd = tb[5 * NQ + qi];
                } else {
                    const bool liq = cc == CELL_LIQUID;
                    rho = liq ? m.rho_H1 : m.rho_H0;
                    mu = liq ? m.mu_H1 : m.mu_H0;
                    nz[0] = nz[1] = nz[2] = 0.f;
                    vd = 0.f;
                }
                const float Wr = B.wf[qx] * wyz;  // reference weight w_q
                const float wr = Wr * rho * hs.hcm;  // W rho c_m
                const float wm = Wr * mu * hs.c2h;   // 2 W mu / h^2
                const float tr = G[0][0] + G[1][1] + G[2][2];
                float cf[QC32_K];
#pragma unroll
                for (int k = 0; k < QC32_K; ++k) cf[k] = cq[(k * NQ + qi) * 32];
                float F[3], T[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    F[c] = wr * X[c] + cf[0] * G[c][0] + cf[1] * G[c][1] + cf[2] * G[c][2] +
                           cf[3 + 3 * c] * X[0] + cf[4 + 3 * c] * X[1] + cf[5 + 3 * c] * X[2];
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int b = 0; b < 3; ++b) T[c][b] = wm * (0.5f * (G[c][b] + G[b][c]) - tr * nz[c] * nz[b]);
                const float rdiv = Wr * (hs.h2 * tr - hs.h3 * vd);
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int ii = 0; ii < Q; ++ii) {
                        Pv[c][ii] += (float)B.S[qx][ii] * F[c] + (float)B.D[qx][ii] * T[c][0];
                        Py[c][ii] += (float)B.S[qx][ii] * T[c][1];
                        Pz[c][ii] += (float)B.S[qx][ii] * T[c][2];
                    }
                Pd[0] += (float)B.N1[qx][0] * rdiv;
                Pd[1] += (float)B.N1[qx][1] * rdiv;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int ii = 0; ii < Q; ++ii) {
                    S_(c * NQ + at(qz, qy, ii)) = Pv[c][ii];
                    S_(OFF_Y + c * NQ + at(qz, qy, ii)) = Py[c][ii];
                    S_(OFF_Z + c * NQ + at(qz, qy, ii)) = Pz[c][ii];
                }
            S_(OFF_PD + 0 * L + qy + Q * qz) = Pd[0];
            S_(OFF_PD + 1 * L + qy + Q * qz) = Pd[1];
        }
    }
    __syncthreads();
    // ---------------------------------------------------------------- y-lines backwards
    {
        const int i = l % Q, qz = l / Q;
        if (active) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float pv[Q], py[Q], pz[Q];
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    pv[q] = S_(c * NQ + at(qz, q, i));
                    py[q] = S_(OFF_Y + c * NQ + at(qz, q, i));
                    pz[q] = S_(OFF_Z + c * NQ + at(qz, q, i));
                }
#pragma unroll
                for (int jj = 0; jj < Q; ++jj) {
                    float r = 0.f, rz = 0.f;
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        r += (float)B.S[q][jj] * pv[q] + (float)B.D[q][jj] * py[q];
                        rz += (float)B.S[q][jj] * pz[q];
                    }
                    S_(c * NQ + at(qz, jj, i)) = r;
                    S_(OFF_Z + c * NQ + at(qz, jj, i)) = rz;
                }
            }
            if (yp && l < 2 * Q) {  // divergence row: y-sweep [jx][jy][qz]
                const int jx = l % 2, qq = l / 2;
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float v = S_(OFF_PD + jx * L + q + Q * qq);
                    s0 += (float)B.N1[q][0] * v;
                    s1 += (float)B.N1[q][1] * v;
                }
                S_(OFF_QD + jx + 2 * (0 + 2 * qq)) = s0;
                S_(OFF_QD + jx + 2 * (1 + 2 * qq)) = s1;
            }
        }
    }
    __syncthreads();
    // ---------------------------------------------------------------- z-lines backwards and scatter
    if constexpr (!DET) {  // atomic adds as soon as each result is formed
        const int i = l % Q, j = l / Q;
        if (active) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float r[Q], rz[Q];
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    r[q] = S_(c * NQ + at(q, j, i));
                    rz[q] = S_(OFF_Z + c * NQ + at(q, j, i));
                }
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    float o = 0.f;
#pragma unroll
                    for (int q = 0; q < Q; ++q) o += (float)B.S[q][k] * r[q] + (float)B.D[q][k] * rz[q];
                    if (keep[k]) atomicAdd(&y[c * m.Nu + zbase + k * MM], o);
                }
            }
            if (yp && l < 4) {  // divergence row: z-sweep, Q1 node (jx, jy, jz)
                const int jx = l % 2, jy = l / 2;
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float v = S_(OFF_QD + jx + 2 * (jy + 2 * q));
                    s0 += (float)B.N1[q][0] * v;
                    s1 += (float)B.N1[q][1] * v;
                }
                const int64_t m1 = n + 1;
                atomicAdd(&yp[(cx + jx) + m1 * ((cy + jy) + m1 * (cz + 0))], s0);
                atomicAdd(&yp[(cx + jx) + m1 * ((cy + jy) + m1 * (cz + 1))], s1);
            }
        }
    } else {  // colour pass: the results kept, then written cell by cell
        const int i = l % Q, j = l / Q;
        float o[3][Q], s0 = 0.f, s1 = 0.f;
        const bool div = yp && l < 4;  // divergence row: z-sweep, Q1 node (jx, jy, jz)
        const int jx = l % 2, jy = l / 2;
        if (active) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float r[Q], rz[Q];
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    r[q] = S_(c * NQ + at(q, j, i));
                    rz[q] = S_(OFF_Z + c * NQ + at(q, j, i));
                }
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    float v = 0.f;
#pragma unroll
                    for (int q = 0; q < Q; ++q) v += (float)B.S[q][k] * r[q] + (float)B.D[q][k] * rz[q];
                    o[c][k] = v;
                }
            }
            if (div) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float v = S_(OFF_QD + jx + 2 * (jy + 2 * q));
                    s0 += (float)B.N1[q][0] * v;
                    s1 += (float)B.N1[q][1] * v;
                }
            }
        }
        // plain read-modify-writes: the even cells of the block first, then (after a block barrier) the odd ones,
        // so that the two cells of a shared x-face never write at once
        for (int par = 0; par < 2; ++par) {
            if (par == 1) __syncthreads();
            if (active && (lc & 1) == par) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int k = 0; k < Q; ++k)
                        if (keep[k]) y[c * m.Nu + zbase + k * MM] += o[c][k];
                if (div) {
                    const int64_t m1 = n + 1;
                    yp[(cx + jx) + m1 * ((cy + jy) + m1 * (cz + 0))] += s0;
                    yp[(cx + jx) + m1 * ((cy + jy) + m1 * (cz + 1))] += s1;
                }
            }
        }
    }
}

template <int P>
static int launch32(const evap_mesh* h, const MeshArgs<float>& m, const Scale32& hs, const float* x, float* y,
                    float* yp, cudaStream_t s) {
    constexpr int L = (P + 1) * (P + 1);
    constexpr int CB = 32;                // one warp per line: 288 / 512 threads
    constexpr int MINB = P == 2 ? EVAP_M32_MINB2 : 1;  // 35 KB / 80 KB of shared memory per block
    if (!h->deterministic) {
        const unsigned grid = (unsigned)(((m.n + CB - 1) / CB) * (int64_t)m.n * m.n);
        k_momentum32<P, CB, MINB, false><<<grid, CB * L, 0, s>>>(m, hs, h->cell_code, h->table_index, h->table32, h->qc32, x,
                                                           y, yp, -1);
        EVAP_CHECK_LAUNCH("momentum32");
        return EVAP_OK;
    }
    const int64_t nxc = (m.n + CB - 1) / CB;
    for (int colour = 0; colour < 8; ++colour) {  // block parity along x and row parities, one launch each
        const int pb = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
        const int64_t hxb = (nxc - pb + 1) / 2, hy = (m.n - py + 1) / 2, hz = (m.n - pz + 1) / 2;
        const int64_t grid = hxb * hy * hz;
        if (grid == 0) continue;
        k_momentum32<P, CB, MINB, true><<<(unsigned)grid, CB * L, 0, s>>>(m, hs, h->cell_code, h->table_index, h->table32,
                                                                     h->qc32, x, y, yp, colour);
        EVAP_CHECK_LAUNCH("momentum32");
    }
    return EVAP_OK;
}

int launch_momentum32(evap_mesh* h, const float* x, float* y, float* yp, cudaStream_t s) {
    const MeshArgs<float> m = mesh_args<float>(h);
    const double hh = h->m.h;
    Scale32 hs;
    hs.h2 = (float)(hh * hh);
    hs.h3 = (float)(hh * hh * hh);
    hs.c2h = (float)(2.0 * hh);
    hs.hcm = (float)(hh * hh * hh * h->m.c_mass);
    return m.P == 2 ? launch32<2>(h, m, hs, x, y, yp, s) : launch32<3>(h, m, hs, x, y, yp, s);
}

}  // namespace evap
