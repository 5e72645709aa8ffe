// The Schur approximation S~ = B diag(A)^(-1) B^T of the velocity-pressure preconditioner, assembled.
//
// B is the divergence row of the momentum apply: B_c[j][v] = sum_q W N1_j d_c N_v over the velocity Gauss rule, with
// the velocity DoFs on Dirichlet faces left out (the apply reads x as 0 there and B^T p vanishes there).  On the
// uniform Cartesian mesh every factor is a tensor product of 1D integrals, B_c[j][v] = prod_d F^c_d[j_d][v_d] with
// F^c_d = g1 (the 1D integral of N1_J N_V', dimensionless) in the direction d = c and a1 (the 1D integral of
// N1_J N_V, h) in the other two; these are exact with the velocity Gauss rule.  So
//   S~[i][j] = sum_c sum_{v free} prod_d (F^c_d[i_d][v_d] F^c_d[j_d][v_d]) / D_c[v],
// D_c[v] the Jacobi diagonal of A (in FP32, as the matrix-free Schur operator uses it).  A pressure node couples with
// the nodes within two cells (a 5^3 = 125-point stencil); S~ is symmetric, so the 63 offsets o >= 0 (in the
// lexicographic order of (oz, oy, ox)) are stored, as FP32 [63][N_p]: offset o of node i is entry |l(o) - 62| of node
// i (l(o) >= 62) or of node i + o (l(o) < 62), with l(o) = 25 (oz + 2) + 5 (oy + 2) + (ox + 2); entry 0 is the diagonal.
// One thread per stored entry sums its (at most 5^3) velocity nodes in a fixed order: no atomics.
//
// With the stencil, the Schur CG of every preconditioner application is one cooperative launch in FP32
// (k_cg_fused32) instead of, per iteration, a matrix-free gradient and divergence over the whole velocity mesh.
#include <algorithm>
#include <cstring>

#include "fused_krylov.cuh"
#include "physics.cuh"

namespace evap {

struct SchurTables {
    float a[2][MAXQ];  // a[a][b] = h sum_q w_q N1_a(t_q) l_b(t_q)
    float g[2][MAXQ];  // g[a][b] =   sum_q w_q N1_a(t_q) l_b'(t_q)
};

// 1D assembled factor of pressure node I (0..n) and velocity node V (0..P n): the cells e in {I - 1, I} that hold both
__device__ __forceinline__ float factor1(const float (&t)[2][MAXQ], int P, int n, int I, int V) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int e = I - 1 + k;
        const int b = V - P * e;
        if (e >= 0 && e < n && b >= 0 && b <= P) s += t[1 - k][b];  // node I is corner 1 of cell I - 1, corner 0 of I
    }
    return s;
}

__global__ void __launch_bounds__(128) k_schur_assemble(int n, int P, int M, unsigned faces, int64_t Nu, int64_t Np,
                                                        SchurTables tab, const float* __restrict__ diag,
                                                        float* __restrict__ S) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= 63 * Np) return;
    const int e = (int)(idx / Np);
    const int64_t node = idx - (int64_t)e * Np;
    const int lin = 62 + e;
    const int o[3] = {lin % 5 - 2, (lin / 5) % 5 - 2, lin / 25 - 2};
    const int m1 = n + 1;
    const int I[3] = {(int)(node % m1), (int)((node / m1) % m1), (int)(node / ((int64_t)m1 * m1))};
    float wa[3][2 * MAXQ - 1], wg[3][2 * MAXQ - 1];
    int lo[3], cnt[3];
    for (int d = 0; d < 3; ++d) {
        const int J = I[d] + o[d];
        if (J < 0 || J > n) {
            S[idx] = 0.f;
            return;
        }
        lo[d] = std::max(P * std::max(I[d], J) - P, 0);
        const int hi = std::min(P * std::min(I[d], J) + P, P * n);
        cnt[d] = std::max(hi - lo[d] + 1, 0);
        for (int k = 0; k < cnt[d]; ++k) {
            const int V = lo[d] + k;
            wa[d][k] = factor1(tab.a, P, n, I[d], V) * factor1(tab.a, P, n, J, V);
            wg[d][k] = factor1(tab.g, P, n, I[d], V) * factor1(tab.g, P, n, J, V);
        }
    }
    float acc = 0.f;
    for (int kz = 0; kz < cnt[2]; ++kz)
        for (int ky = 0; ky < cnt[1]; ++ky)
            for (int kx = 0; kx < cnt[0]; ++kx) {
                const int vx = lo[0] + kx, vy = lo[1] + ky, vz = lo[2] + kz;
                if (constrained_node(vx, vy, vz, M, faces)) continue;
                const int64_t v = vx + (int64_t)M * (vy + (int64_t)M * vz);
                acc += wg[0][kx] * wa[1][ky] * wa[2][kz] / diag[v] + wa[0][kx] * wg[1][ky] * wa[2][kz] / diag[Nu + v] +
                       wa[0][kx] * wa[1][ky] * wg[2][kz] / diag[2 * Nu + v];
            }
    S[idx] = acc;
}

// Row `node` of S~ x and its diagonal, from the stored half stencil (FP32).  Nodes at least two layers inside the
// lattice take an unrolled path with compile-time offsets and no bounds tests (83 % of the nodes at 64^3); the others
// test each neighbour.  Entries are indexed with 32 bits (63 N_p < 2^32, checked on the host).
struct SchurStencil {
    static constexpr int SMEM = 0;
    int n;
    int64_t Np;
    const float* S;
    __device__ __forceinline__ void load(float*) const {}
    template <class X>
    __device__ __forceinline__ float row(int64_t node, const X* x, const float*) const {
        const unsigned m1 = (unsigned)n + 1u, m2 = m1 * m1, nd = (unsigned)node, np = (unsigned)Np;
        const unsigned t = nd / m1, i = nd - t * m1, k = t / m1, j = t - k * m1;
        float acc = 0.f;
        if (i >= 2u && j >= 2u && k >= 2u && i + 2u <= (unsigned)n && j + 2u <= (unsigned)n && k + 2u <= (unsigned)n) {
#pragma unroll
            for (int dz = -2; dz <= 2; ++dz)
#pragma unroll
                for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
                    for (int dx = -2; dx <= 2; ++dx) {
                        const int lin = 25 * (dz + 2) + 5 * (dy + 2) + (dx + 2);
                        const unsigned nb = nd + (unsigned)dx + (unsigned)dy * m1 + (unsigned)dz * m2;
                        const float c = lin >= 62 ? S[(unsigned)(lin - 62) * np + nd] : S[(unsigned)(62 - lin) * np + nb];
                        acc = fmaf(c, (float)x[nb], acc);
                    }
            return acc;
        }
#pragma unroll
        for (int dz = -2; dz <= 2; ++dz) {
            if ((int)k + dz < 0 || (int)k + dz > n) continue;
#pragma unroll
            for (int dy = -2; dy <= 2; ++dy) {
                if ((int)j + dy < 0 || (int)j + dy > n) continue;
#pragma unroll
                for (int dx = -2; dx <= 2; ++dx) {
                    if ((int)i + dx < 0 || (int)i + dx > n) continue;
                    const int lin = 25 * (dz + 2) + 5 * (dy + 2) + (dx + 2);
                    const unsigned nb = nd + (unsigned)dx + (unsigned)dy * m1 + (unsigned)dz * m2;
                    const float c = lin >= 62 ? S[(unsigned)(lin - 62) * np + nd] : S[(unsigned)(62 - lin) * np + nb];
                    acc = fmaf(c, (float)x[nb], acc);
                }
            }
        }
        return acc;
    }
    __device__ __forceinline__ float diag(int64_t node, const float*) const { return S[node]; }
};

// y = S~ x in FP32 arithmetic (x, y FP64), one thread per pressure node.
__global__ void k_schur_apply(SchurStencil op, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (node < op.Np) y[node] = (double)op.row(node, x, nullptr);
}

// Assembles S~ for the mesh's current Jacobi diagonal of A (launch_diagonal), once per diagonal.
int schur_assemble(evap_mesh* h, cudaStream_t s) {
    int rc = launch_diagonal(h, s);
    if (rc) return rc;
    if (h->schur_S && h->schur_stamp == h->diag_stamp) return EVAP_OK;
    const MeshArgs<double>& m = h->m;
    if (63 * m.Np >= (int64_t)1 << 32) {
        set_error("Schur stencil: its 63 N_p entries must be indexable with 32 bits");
        return EVAP_EINVAL;
    }
    if (!h->schur_S) EVAP_CUDA(cudaMalloc(&h->schur_S, 63 * m.Np * sizeof(float)));
    SchurTables tab;
    std::memset(&tab, 0, sizeof(tab));
    const Basis<double>& b = h->b;
    for (int a = 0; a < 2; ++a)
        for (int v = 0; v <= m.P; ++v) {
            double sa = 0.0, sg = 0.0;
            for (int q = 0; q < b.Q; ++q) {
                sa += b.w[q] * b.N1[q][a] * b.S[q][v];
                sg += b.w[q] * b.N1[q][a] * b.D[q][v];
            }
            tab.a[a][v] = (float)(m.h * sa);
            tab.g[a][v] = (float)sg;
        }
    const int64_t total = 63 * m.Np;
    k_schur_assemble<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(m.n, m.P, m.M, m.faces, m.Nu, m.Np, tab,
                                                                     h->diag32, h->schur_S);
    EVAP_CHECK_LAUNCH("schur_assemble");
    h->schur_stamp = h->diag_stamp;
    return EVAP_OK;
}

int launch_schur_apply(evap_mesh* h, const double* x, double* y, cudaStream_t s) {
    int rc = schur_assemble(h, s);
    if (rc) return rc;
    const SchurStencil op{h->m.n, h->m.Np, h->schur_S};
    k_schur_apply<<<(unsigned)((h->m.Np + 255) / 256), 256, 0, s>>>(op, x, y);
    EVAP_CHECK_LAUNCH("schur_apply");
    return EVAP_OK;
}

// z ~ S~^(-1) r: the FP32 single-launch CG (k_cg_fused32) on the assembled stencil with its diagonal as the Jacobi
// preconditioner, from z = 0, at most max_iter iterations or |r| <= rtol |r0|.
int schur_solve(evap_mesh* h, const double* r, double* z, double rtol, int max_iter, int* iters, cudaStream_t s) {
    int rc = schur_assemble(h, s);
    if (rc) return rc;
    int64_t N = h->m.Np;
    FusedSpace f;
    if ((rc = fused_space(h, 3, f))) return rc;  // 3 pair vectors = 6 float vectors of N_phi >= N_p entries
    int G = 0;
    if ((rc = fused_grid(k_cg_fused32<SchurStencil>, 0, FK_MAX_BLOCKS, G))) return rc;
    EVAP_CUDA(cudaMemsetAsync(f.gb, 0, sizeof(GridBarrier), s));
    SchurStencil op{h->m.n, N, h->schur_S};
    const int64_t Nl = ls_args<double>(h).Nphi;  // the vectors' stride: fused_space sizes them for N_phi
    float* base = reinterpret_cast<float*>(f.vec);
    float *xs = base, *r32 = base + Nl, *u = base + 2 * Nl, *p = base + 3 * Nl, *sv = base + 4 * Nl, *w = base + 5 * Nl;
    float* dinv = f.dinv;
    float* part = reinterpret_cast<float*>(f.part);
    GridBarrier* gb = f.gb;
    double* out = f.out;
    double atol = 0.0;
    double* zz = z;
    void* args[] = {&op, &N, &r, &zz, &xs, &dinv, &r32, &u, &p, &sv, &w, &rtol, &atol, &max_iter, &part, &gb, &out};
    EVAP_CUDA(cudaLaunchCooperativeKernel((const void*)k_cg_fused32<SchurStencil>, dim3(G), dim3(FK_THREADS), args, 0,
                                          s));
    EVAP_CHECK_LAUNCH("schur_cg");
    double res[3];
    if ((rc = fused_result(h, f, s, res))) return rc;
    if (iters) *iters += (int)res[0];
    return EVAP_OK;
}

}  // namespace evap

extern "C" int evap_apply_schur(evap_handle h, const double* x, double* y, void* stream) {
    if (!h || !x || !y) {
        evap::set_error("evap_apply_schur: null argument");
        return EVAP_EINVAL;
    }
    if (!h->has_fields) {
        evap::set_error("evap_apply_schur: call evap_set_fields first");
        return EVAP_ENOFIELDS;
    }
    EVAP_CUDA(cudaSetDevice(h->device));
    return evap::launch_schur_apply(h, x, y, (cudaStream_t)stream);
}
