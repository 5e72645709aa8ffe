// Level-set sub-solver on the Q1 level-set space (steps 1 to 3 of Algorithm 2), FP64:
//   advection          (M + theta dt C) phi^(k+1) = (M - (1 - theta) dt C) phi^n, C from u_Gamma(phi^(k))   Eqs. transport, weakFormLevelSet
//                      (a fixed point over the transport velocity; GMRES with the diagonal preconditioner)
//   projected normal   (M + eta_n h^2 K) n_c = (N_i, nbar_c),        nbar = grad phi / |grad phi|   Eq. normal_vector_regularized
//   curvature          (M + eta_k h^2 K) kappa = -(N_i, div n_h)                                    Eq. curvature_regularized
//   reinitialization   (M / dtau + eps K_n) psi^(k+1) = M psi^k / dtau + (grad N_i . n, (1 - psi_k^2)/2)   Eq. reinitialization
// with homogeneous Neumann conditions, each system solved by conjugate gradients with the diagonal (Jacobi)
// preconditioner to |r| <= max(1e-12 |r_0|, 1e-20) (the solver table of the paper).
//
// M + c K has constant coefficients on the uniform Cartesian mesh: M = Mx (x) My (x) Mz, K = Kx My Mz + Mx Ky Mz +
// Mx My Kz with the 1D Q1 mass (h/6, 2h/3 or h/3 at an end, h/6) and stiffness (-1/h, 2/h or 1/h, -1/h) rows, which the
// 2-point Gauss rule integrates exactly.  Its apply is therefore a 27-point stencil, evaluated per node by separable
// sums (x, then y, then z: 93 FMA per node) instead of per-cell quadrature.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>

#include "dfloat.cuh"
#include "fused_krylov.cuh"
#include "physics.cuh"

namespace evap {

// 1D rows of node i in [0, n]: mass m[d] and stiffness k[d] for the neighbours d = -1, 0, +1 (cell edge h).
__device__ __forceinline__ void q1_rows(int i, int n, double h, double ih, double m[3], double k[3]) {
    const bool lo = i > 0, hi = i < n;
    m[0] = lo ? h / 6.0 : 0.0;
    m[2] = hi ? h / 6.0 : 0.0;
    m[1] = (lo ? h / 3.0 : 0.0) + (hi ? h / 3.0 : 0.0);
    k[0] = lo ? -ih : 0.0;
    k[2] = hi ? -ih : 0.0;
    k[1] = (lo ? ih : 0.0) + (hi ? ih : 0.0);
}

// y = (M + c K) x for ncomp component fields of N_phi entries each (component-major), one thread per node.
__global__ void __launch_bounds__(256) k_helmholtz(int n, double h, double c, int ncomp, const double* __restrict__ x,
                                                   double* __restrict__ y) {
    const int m1 = n + 1;
    const int64_t Np = (int64_t)m1 * m1 * m1;
    const double ih = 1.0 / h;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < Np * ncomp; t += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)(t / Np);
        const int64_t node = t - comp * Np;
        const int i = (int)(node % m1), j = (int)((node / m1) % m1), kz = (int)(node / ((int64_t)m1 * m1));
        double mx[3], kx[3], my[3], ky[3], mz[3], kzr[3];
        q1_rows(i, n, h, ih, mx, kx);
        q1_rows(j, n, h, ih, my, ky);
        q1_rows(kz, n, h, ih, mz, kzr);
        const double* xc = x + comp * Np;
        double acc = 0.0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            if ((dz < 0 && kz == 0) || (dz > 0 && kz == n)) continue;
            double smm = 0.0, skm = 0.0, smk = 0.0;  // sums over y of (m_y x-mass), (m_y x-stiff), (k_y x-mass)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                if ((dy < 0 && j == 0) || (dy > 0 && j == n)) continue;
                const double* row = xc + (i + (int64_t)m1 * ((j + dy) + (int64_t)m1 * (kz + dz)));
                double sm = 0.0, sk = 0.0;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if ((dx < 0 && i == 0) || (dx > 0 && i == n)) continue;
                    const double v = row[dx];
                    sm += mx[dx + 1] * v;
                    sk += kx[dx + 1] * v;
                }
                smm += my[dy + 1] * sm;
                skm += my[dy + 1] * sk;
                smk += ky[dy + 1] * sm;
            }
            acc += mz[dz + 1] * (smm + c * (skm + smk)) + c * kzr[dz + 1] * smm;
        }
        y[t] = acc;
    }
}

// The operators of the CG solves in double-float arithmetic (dfloat.cuh): GB300's FP64 pipe bounds the FP64 stencil
// (93 FMA per node: ~40 us at 64^3), the FP32 pipe runs the same sums on hi + lo pairs several times faster.  The
// CG keeps its direction p as pairs beside the FP64 copy, so the operators read their neighbours without converting.
// The node stencil of sum_e A_e from symmetric element matrices stored as pairs, entry (a <= b) of cell e at
// E[(b (b + 1) / 2 + a) ncell + e] (k_reinit_elem): per node, the rows of the (up to 8) cells around it summed by
// offset in double-float; offsets without a cell get 0.  One thread per node, so no atomics and a fixed sum order.
__global__ void __launch_bounds__(256) k_stencil_from_elem(int n, int64_t ncell, int64_t N, const float2* __restrict__ E,
                                                           float2* __restrict__ C) {
    const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (node >= N) return;
    const unsigned m1 = (unsigned)n + 1u, nd = (unsigned)node;
    const unsigned t = nd / m1;
    const int i = (int)(nd - t * m1), k = (int)(t / m1), j = (int)(t - (unsigned)k * m1);
    dfl acc[27];
#pragma unroll
    for (int s = 0; s < 27; ++s) acc[s] = dfl{0.f, 0.f};
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
        const int ox = cc & 1, oy = (cc >> 1) & 1, oz = cc >> 2;  // the node's corner in the cell
        const int cx = i - ox, cy = j - oy, cz = k - oz;
        if (cx < 0 || cy < 0 || cz < 0 || cx >= n || cy >= n || cz >= n) continue;
        const int64_t cell = cx + (int64_t)n * (cy + (int64_t)n * cz);
        const int li = ox + 2 * oy + 4 * oz;
#pragma unroll
        for (int lj = 0; lj < 8; ++lj) {
            const int a = li < lj ? li : lj, b = li < lj ? lj : li;
            const int sx = (lj & 1) - ox, sy = ((lj >> 1) & 1) - oy, sz = (lj >> 2) - oz;
            const int s = 9 * (sz + 1) + 3 * (sy + 1) + (sx + 1);
            acc[s] = df_add(acc[s], ld_df(E + (int64_t)(b * (b + 1) / 2 + a) * ncell + cell));
        }
    }
#pragma unroll
    for (int s = 0; s < 27; ++s) C[s * N + node] = make_float2(acc[s].hi, acc[s].lo);
}



// Q1 cell data at the 2^3 Gauss points: shape values N[q][j] and reference derivative signs.
struct Q1Cell {
    int64_t node[8];
};

__device__ __forceinline__ void q1_cell_nodes(int64_t cell, int n, Q1Cell& c, int& cx, int& cy, int& cz) {
    const int64_t m1 = n + 1;
    cx = (int)(cell % n);
    cy = (int)((cell / n) % n);
    cz = (int)(cell / ((int64_t)n * n));
#pragma unroll
    for (int j = 0; j < 8; ++j)
        c.node[j] = (cx + (j & 1)) + m1 * ((cy + ((j >> 1) & 1)) + m1 * (cz + (j >> 2)));
}

// Value and physical gradient weights of node j at Gauss point q of the 2-point rule (t = g2t).
__device__ __forceinline__ void q1_weights(const double* g2t, int q, double inv_h, double N[8], double G[8][3]) {
    const double tx = g2t[q & 1], ty = g2t[(q >> 1) & 1], tz = g2t[q >> 2];
    const double Nx[2] = {1.0 - tx, tx}, Ny[2] = {1.0 - ty, ty}, Nz[2] = {1.0 - tz, tz};
    const double Dd[2] = {-inv_h, inv_h};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int a = j & 1, b = (j >> 1) & 1, c = j >> 2;
        N[j] = Nx[a] * Ny[b] * Nz[c];
        G[j][0] = Dd[a] * Ny[b] * Nz[c];
        G[j][1] = Nx[a] * Dd[b] * Nz[c];
        G[j][2] = Nx[a] * Ny[b] * Dd[c];
    }
}

// b[c * stride + i] += sum_q W N_i nbar_c, nbar the unit normal of phi at the point (zero where
// |grad phi| h <= GRAD_TINY).
__global__ void __launch_bounds__(128) k_normal_rhs(MeshArgs<double> m, Basis<double> bas, const double* __restrict__ phi,
                                                    double* __restrict__ b, int64_t stride) {
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= m.ncell) return;
    Q1Cell c;
    int cx, cy, cz;
    q1_cell_nodes(cell, m.n, c, cx, cy, cz);
    double pv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) pv[j] = phi[c.node[j]];
    double out[3][8] = {};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double N[8], G[8][3];
        q1_weights(bas.g2t, q, m.inv_h, N, G);
        const double W = bas.g2w[q & 1] * bas.g2w[(q >> 1) & 1] * bas.g2w[q >> 2] * m.vol_w;
        double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int d = 0; d < 3; ++d) g[d] += G[j][d] * pv[j];
        const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        if (!(gn * m.h > GRAD_TINY)) continue;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double wn = W * g[d] / gn;
#pragma unroll
            for (int j = 0; j < 8; ++j) out[d][j] += N[j] * wn;
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int j = 0; j < 8; ++j) atomicAdd(&b[d * stride + c.node[j]], out[d][j]);
}

// b[i] += -sum_q W N_i div n_h for the Q1 vector field nf [3][N_phi].
__global__ void __launch_bounds__(128) k_curvature_rhs(MeshArgs<double> m, Basis<double> bas,
                                                       const double* __restrict__ nf, double* __restrict__ b) {
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= m.ncell) return;
    Q1Cell c;
    int cx, cy, cz;
    q1_cell_nodes(cell, m.n, c, cx, cy, cz);
    double nv[3][8];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int j = 0; j < 8; ++j) nv[d][j] = nf[d * m.Nphi + c.node[j]];
    double out[8] = {};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double N[8], G[8][3];
        q1_weights(bas.g2t, q, m.inv_h, N, G);
        const double W = bas.g2w[q & 1] * bas.g2w[(q >> 1) & 1] * bas.g2w[q >> 2] * m.vol_w;
        double div = 0.0;
#pragma unroll
        for (int j = 0; j < 8; ++j) div += G[j][0] * nv[0][j] + G[j][1] * nv[1][j] + G[j][2] * nv[2][j];
#pragma unroll
        for (int j = 0; j < 8; ++j) out[j] -= N[j] * W * div;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) atomicAdd(&b[c.node[j]], out[j]);
}

// ------------------------------------------------------------------------------- norms of level-set changes
// |a - b|^2 into a device scalar (the advection fixed point's and the reinitialization's change): block sums, then
// the last block to arrive (memory fence + atomic ticket; no block waits on another) adds the partials.
constexpr int CG_THREADS = 256;
constexpr int CG_BLOCKS = 304;

__device__ __forceinline__ double cg_block_sum(double v) {
    __shared__ double sh[CG_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < CG_THREADS / 32; ++i) r += sh[i];
    return r;
}

// Two block partials (valid in thread 0) to part[2][CG_BLOCKS]; returns true in the last block to arrive, whose
// threads then see the totals in tot[0..1].
__device__ __forceinline__ bool cg_finish2(double a, double b, double* part, unsigned* ticket, double tot[2]) {
    __shared__ bool last;
    __shared__ double sums[2];
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a;
        part[CG_BLOCKS + blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double va = 0.0, vb = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        va += __ldcg(&part[i]);
        vb += __ldcg(&part[CG_BLOCKS + i]);
    }
    va = cg_block_sum(va);
    vb = cg_block_sum(vb);
    if (threadIdx.x == 0) {
        sums[0] = va;
        sums[1] = vb;
        *ticket = 0u;
    }
    __syncthreads();
    tot[0] = sums[0];
    tot[1] = sums[1];
    return true;
}

// *out = |a - b|^2
__global__ void __launch_bounds__(CG_THREADS) k_diff_norm(const double* __restrict__ a, const double* __restrict__ b,
                                                          int64_t N, double* part, unsigned* ticket, double* out) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = a[i] - b[i];
        s += d * d;
    }
    double tot[2];
    if (cg_finish2(cg_block_sum(s), 0.0, part, ticket, tot) && threadIdx.x == 0) *out = tot[0];
}

// Workspace: r, z, p, q [N_phi] + partials + scalars + ticket (allocated once per mesh).
static int geo_workspace(evap_mesh* h) {
    if (h->geo_ws) return EVAP_OK;
    const int64_t Np = h->m.Nphi;
    const size_t vec = ((size_t)Np * sizeof(double) + 255) & ~(size_t)255;
    const size_t bytes = 10 * vec + (2 * CG_BLOCKS + 8) * sizeof(double) + 256;
    EVAP_CUDA(cudaMalloc(&h->geo_ws, bytes));
    EVAP_CUDA(cudaMemset(h->geo_ws, 0, bytes));
    if (!h->geo_host) EVAP_CUDA(cudaMallocHost(&h->geo_host, 8 * sizeof(double)));
    return EVAP_OK;
}

struct CgSpace {
    double *r, *z, *p, *q, *b, *d, *t0, *t1, *t2, *part, *S;
    unsigned* ticket;
};

static CgSpace cg_space(evap_mesh* h) {
    const int64_t Np = h->m.Nphi;
    const size_t vec = ((size_t)Np * sizeof(double) + 255) & ~(size_t)255;
    char* base = (char*)h->geo_ws;
    CgSpace w;
    w.r = (double*)(base + 0 * vec);
    w.z = (double*)(base + 1 * vec);
    w.p = (double*)(base + 2 * vec);
    w.q = (double*)(base + 3 * vec);
    w.b = (double*)(base + 4 * vec);
    w.d = (double*)(base + 5 * vec);
    w.t0 = (double*)(base + 6 * vec);
    w.t1 = (double*)(base + 7 * vec);
    w.t2 = (double*)(base + 8 * vec);
    w.part = (double*)(base + 10 * vec);
    w.S = w.part + 2 * CG_BLOCKS;
    w.ticket = (unsigned*)(w.S + 8);
    return w;
}

// Workspace of the single-launch solvers (FusedSpace, fused_krylov.cuh), grown on demand.
static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

int fused_space(evap_mesh* h, int nvec, FusedSpace& f) {
    if (!h->geo_host) EVAP_CUDA(cudaMallocHost(&h->geo_host, 8 * sizeof(double)));  // the result words' mirror
    const int64_t N = ls_args<double>(h).Nphi;
    const size_t vbytes = al256((size_t)nvec * N * sizeof(float2)), dbytes = al256((size_t)N * sizeof(float));
    const size_t pbytes = al256((size_t)(GM_MAX + 2) * FK_MAX_BLOCKS * sizeof(float2));
    const size_t tail = al256(sizeof(GridBarrier) + 4 * sizeof(double)) + HelmholtzStencil::SMEM * sizeof(float2);
    const size_t need = vbytes + dbytes + pbytes + tail;
    if (h->geo_kry_bytes < need) {
        if (h->geo_kry) cudaFree(h->geo_kry);
        h->geo_kry = nullptr;
        h->geo_kry_bytes = 0;
        EVAP_CUDA(cudaMalloc(&h->geo_kry, need));
        h->geo_kry_bytes = need;
    }
    char* base = (char*)h->geo_kry;
    const size_t vcap = h->geo_kry_bytes - dbytes - pbytes - tail;  // the vectors keep whatever room they had
    f.vec = (float2*)base;
    f.dinv = (float*)(base + vcap);
    f.part = (float2*)(base + vcap + dbytes);
    f.gb = (GridBarrier*)(base + vcap + dbytes + pbytes);
    f.out = (double*)(f.gb + 1);
    f.table = (float2*)(base + vcap + dbytes + pbytes + al256(sizeof(GridBarrier) + 4 * sizeof(double)));
    return EVAP_OK;
}

// Reads the solver's result words and the barrier's error word after the launch (one synchronization).
int fused_result(evap_mesh* h, const FusedSpace& f, cudaStream_t s, double res[3]) {
    double* hs = h->geo_host;
    EVAP_CUDA(cudaMemcpyAsync(hs, f.out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    EVAP_CUDA(cudaMemcpyAsync(hs + 4, f.gb, sizeof(GridBarrier), cudaMemcpyDeviceToHost, s));
    EVAP_CUDA(cudaStreamSynchronize(s));
    GridBarrier hb;
    std::memcpy(&hb, hs + 4, sizeof(GridBarrier));
    if (hb.err) {
        set_error("single-launch solver: a block gave up waiting at the grid barrier");
        return EVAP_ETIMEOUT;
    }
    res[0] = hs[0];
    res[1] = hs[1];
    res[2] = hs[2];
    return EVAP_OK;
}

// The single-launch CG (k_cg_fused) on a level-set system: one cooperative launch and one host read per solve,
// stopping at |r| <= max(rtol |r0|, atol) or after max_iter iterations.
template <class Op>
static int cg_solve_fused(evap_mesh* h, Op op, const double* b, double* x, double rtol, double atol, int max_iter,
                          int* iters, double* relres, cudaStream_t s) {
    int64_t N = ls_args<double>(h).Nphi;
    if (N >= (int64_t)1 << 32) {
        set_error("single-launch CG: the level-set stencils index nodes with 32 bits");
        return EVAP_EINVAL;
    }
    FusedSpace f;
    int rc = fused_space(h, 6, f), G = 0;
    if (rc) return rc;
    const size_t smem = Op::SMEM * sizeof(float2);
    if ((rc = fused_grid(k_cg_fused<Op>, smem, FK_MAX_BLOCKS, G))) return rc;
    EVAP_CUDA(cudaMemsetAsync(f.gb, 0, sizeof(GridBarrier), s));
    double* xx = x;
    float2 *xd = f.vec, *r = f.vec + N, *u = f.vec + 2 * N, *p = f.vec + 3 * N, *sv = f.vec + 4 * N, *w = f.vec + 5 * N;
    float* dinv = f.dinv;
    float2* part = f.part;
    GridBarrier* gb = f.gb;
    double* out = f.out;
    void* args[] = {&op, &N, &b, &xx, &xd, &dinv, &r, &u, &p, &sv, &w, &rtol, &atol, &max_iter, &part, &gb, &out};
    EVAP_CUDA(cudaLaunchCooperativeKernel((const void*)k_cg_fused<Op>, dim3(G), dim3(FK_THREADS), args, smem, s));
    EVAP_CHECK_LAUNCH("cg_fused");
    double res[3];
    if ((rc = fused_result(h, f, s, res))) return rc;
    if (iters) *iters += (int)res[0];
    const double rel = res[2] > 0.0 ? res[1] / res[2] : 0.0;
    if (relres && rel > *relres) *relres = rel;
    return res[1] <= std::max(rtol * res[2], atol) ? EVAP_OK : EVAP_ENOTCONV;
}

// The single-launch GMRES(m) (k_gmres_fused) with the right Jacobi preconditioner, started from x.
template <class Op>
static int gmres_solve_fused(evap_mesh* h, Op op, int m, const double* b, double* x, double rtol, double atol,
                             int max_iter, double reorth, int* iters, double* relres, cudaStream_t s) {
    int64_t N = ls_args<double>(h).Nphi;
    if (N >= (int64_t)1 << 32 || m < 1 || m > GM_MAX) {
        set_error("single-launch GMRES: restart must be in [1, 30] and node indices fit 32 bits");
        return EVAP_EINVAL;
    }
    FusedSpace f;
    int rc = fused_space(h, m + 3, f), G = 0;
    if (rc) return rc;
    const size_t smem = Op::SMEM * sizeof(float2);
    if ((rc = fused_grid(k_gmres_fused<Op>, smem, FK_MAX_BLOCKS, G))) return rc;
    EVAP_CUDA(cudaMemsetAsync(f.gb, 0, sizeof(GridBarrier), s));
    double* xx = x;
    float2 *xd = f.vec, *z = f.vec + N, *V = f.vec + 2 * N;
    float* dinv = f.dinv;
    float2* part = f.part;
    GridBarrier* gb = f.gb;
    double* out = f.out;
    void* args[] = {&op, &N, &m, &b, &xx, &xd, &dinv, &z, &V, &rtol, &atol, &max_iter, &reorth, &part, &gb, &out};
    EVAP_CUDA(cudaLaunchCooperativeKernel((const void*)k_gmres_fused<Op>, dim3(G), dim3(FK_THREADS), args, smem, s));
    EVAP_CHECK_LAUNCH("gmres_fused");
    double res[3];
    if ((rc = fused_result(h, f, s, res))) return rc;
    if (iters) *iters += (int)res[0];
    if (relres) *relres = res[2] > 0.0 ? res[1] / res[2] : 0.0;
    return res[1] <= std::max(rtol * res[2], atol) ? EVAP_OK : EVAP_ENOTCONV;
}

static int helmholtz_apply(evap_mesh* h, double c, int ncomp, const double* x, double* y, cudaStream_t s) {
    const MeshArgs<double> lm = ls_args<double>(h);  // the level-set mesh
    const int64_t total = lm.Nphi * ncomp;
    k_helmholtz<<<blocks_for(total, 256, 152 * 16), 256, 0, s>>>(lm.n, lm.h, c, ncomp, x, y);
    EVAP_CHECK_LAUNCH("helmholtz");
    return EVAP_OK;
}

// The Helmholtz stencil of the level-set mesh with its coefficient table uploaded to the workspace (the copy is
// ordered before the solve on the stream; the host table is copied out before cudaMemcpyAsync returns).
static int helmholtz_stencil(evap_mesh* h, const MeshArgs<double>& lm, double c, HelmholtzStencil& op, cudaStream_t s) {
    FusedSpace f;
    int rc = fused_space(h, 6, f);
    if (rc) return rc;
    float2 tab[HelmholtzStencil::SMEM];
    helmholtz_table(lm.h, c, tab);
    EVAP_CUDA(cudaMemcpyAsync(f.table, tab, sizeof(tab), cudaMemcpyHostToDevice, s));
    op.n = lm.n;
    op.table = f.table;
    return EVAP_OK;
}

int geo_helmholtz(evap_mesh* h, double c, int ncomp, const double* x, double* y, cudaStream_t s) {
    return helmholtz_apply(h, c, ncomp, x, y, s);
}

int geo_projected_normal(evap_mesh* h, double* n, int* iters, double* relres, cudaStream_t s) {
    const MeshArgs<double> lm = ls_args<double>(h);  // the level-set mesh
    int rc = geo_workspace(h);
    if (rc) return rc;
    CgSpace w = cg_space(h);
    const int64_t Np = lm.Nphi;
    const int64_t stride = w.t1 - w.t0;  // right-hand sides of the three components in t0, t1, t2
    const double c = h->prm.eta_n * lm.h * lm.h;
    EVAP_CUDA(cudaMemsetAsync(w.t0, 0, 3 * stride * sizeof(double), s));
    k_normal_rhs<<<blocks_for(lm.ncell, 128, 1LL << 40), 128, 0, s>>>(lm, h->b, h->phi, w.t0, stride);
    EVAP_CHECK_LAUNCH("normal_rhs");
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    int status = EVAP_OK;
    HelmholtzStencil op;
    if ((rc = helmholtz_stencil(h, lm, c, op, s))) return rc;
    for (int d = 0; d < 3; ++d) {
        rc = cg_solve_fused(h, op, w.t0 + d * stride, n + d * Np, 1e-12, 1e-20, 1000, iters, relres, s);
        if (rc == EVAP_ENOTCONV) status = rc;
        else if (rc) return rc;
    }
    return status;
}

int geo_curvature(evap_mesh* h, const double* nf, double* kappa, int* iters, double* relres, cudaStream_t s) {
    const MeshArgs<double> lm = ls_args<double>(h);  // the level-set mesh
    int rc = geo_workspace(h);
    if (rc) return rc;
    CgSpace w = cg_space(h);
    const int64_t Np = lm.Nphi;
    const double c = h->prm.eta_kappa * lm.h * lm.h;
    EVAP_CUDA(cudaMemsetAsync(w.b, 0, Np * sizeof(double), s));
    k_curvature_rhs<<<blocks_for(lm.ncell, 128, 1LL << 40), 128, 0, s>>>(lm, h->b, nf, w.b);
    EVAP_CHECK_LAUNCH("curvature_rhs");
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    HelmholtzStencil op;
    if ((rc = helmholtz_stencil(h, lm, c, op, s))) return rc;
    return cg_solve_fused(h, op, w.b, kappa, 1e-12, 1e-20, 1000, iters, relres, s);
}

// Element matrices of the reinitialization operator with the frozen normal, A_e[i][j] = sum_q W (N_i N_j / dtau +
// eps (grad N_i . n)(grad N_j . n)): the normal does not change over a pseudo-time step, so the 36 distinct entries
// of each symmetric 8x8 matrix are formed once (in FP64, stored as pairs) and assembled into the 27-point node
// stencil the CG iterations apply (k_stencil_from_elem).  Layout [36][ncell] (consecutive cells adjacent), entry k of
// (i <= j) at k = j (j + 1) / 2 + i.
__global__ void __launch_bounds__(128) k_reinit_elem(MeshArgs<double> m, Basis<double> bas, const double* __restrict__ phi,
                                                     const double* __restrict__ nf, float2* __restrict__ Edf) {
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= m.ncell) return;
    Q1Cell c;
    int cx, cy, cz;
    q1_cell_nodes(cell, m.n, c, cx, cy, cz);
    double pv[8], nloc[3][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        pv[j] = phi[c.node[j]];
#pragma unroll
        for (int e = 0; e < 3; ++e) nloc[e][j] = nf ? nf[e * m.Nphi + c.node[j]] : 0.0;
    }
    double a[36] = {};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double N[8], G[8][3], nv[3], gn[8];
        q1_weights(bas.g2t, q, m.inv_h, N, G);
        const double W = bas.g2w[q & 1] * bas.g2w[(q >> 1) & 1] * bas.g2w[q >> 2] * m.vol_w;
        ls_frozen_normal<double>(nf ? nloc : nullptr, pv, N, G, m.h, nv);
#pragma unroll
        for (int j = 0; j < 8; ++j) gn[j] = G[j][0] * nv[0] + G[j][1] * nv[1] + G[j][2] * nv[2];
        const double wm = W / m.dtau, wd = W * m.eps;
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int i = 0; i <= j; ++i) a[j * (j + 1) / 2 + i] += wm * N[i] * N[j] + wd * gn[i] * gn[j];
    }
#pragma unroll
    for (int k = 0; k < 36; ++k) {
        const float hi = (float)a[k];
        Edf[k * m.ncell + cell] = make_float2(hi, (float)(a[k] - (double)hi));
    }
}

// Grows the element-matrix buffer of the mesh to `need` 8-byte words.
static int geo_elem_reserve(evap_mesh* h, int64_t need) {
    if (h->geo_elem_len >= need) return EVAP_OK;
    if (h->geo_elem) cudaFree(h->geo_elem);
    h->geo_elem = nullptr;
    h->geo_elem_len = 0;
    EVAP_CUDA(cudaMalloc(&h->geo_elem, need * sizeof(double)));
    h->geo_elem_len = need;
    return EVAP_OK;
}

// `steps` pseudo-time steps of the reinitialization with the frozen normal of the level-set operators.
int geo_reinitialize(evap_mesh* h, double* psi, int steps, int* iters, double* last_change, cudaStream_t s) {
    const MeshArgs<double> lm = ls_args<double>(h);  // the level-set mesh
    int rc = geo_workspace(h);
    if (rc) return rc;
    CgSpace w = cg_space(h);
    const int64_t Np = lm.Nphi;
    if ((rc = geo_elem_reserve(h, 36 * lm.ncell + 27 * Np))) return rc;  // 36 pairs per cell, then 27 per node
    float2* Edf = reinterpret_cast<float2*>(h->geo_elem);
    float2* Cn = Edf + 36 * lm.ncell;
    const unsigned gc = (unsigned)blocks_for(lm.ncell, 128, 1LL << 40);
    k_reinit_elem<<<gc, 128, 0, s>>>(lm, h->b, h->phi, h->ls_normal, Edf);
    EVAP_CHECK_LAUNCH("reinit_elem");
    k_stencil_from_elem<<<(unsigned)blocks_for(Np, 256, 1LL << 40), 256, 0, s>>>(lm.n, lm.ncell, Np, Edf, Cn);
    EVAP_CHECK_LAUNCH("reinit_stencil");
    if (iters) *iters = 0;
    double rel = 0.0;
    int status = EVAP_OK;
    const NodeStencil op{lm.n, Np, Cn};  // q = sum_e A_e p_e, assembled per node
    for (int k = 0; k < steps; ++k) {
        rc = launch_levelset<double>(h, EVAP_REINIT_RHS, psi, w.b, s);
        if (rc) return rc;
        rc = cg_solve_fused(h, op, w.b, w.t0, 1e-12, 1e-20, 1000, iters, &rel, s);
        if (rc == EVAP_ENOTCONV) status = rc;
        else if (rc) return rc;
        if (k == steps - 1 && last_change) {
            k_diff_norm<<<CG_BLOCKS, CG_THREADS, 0, s>>>(w.t0, psi, Np, w.part, w.ticket, w.S + 5);
            EVAP_CHECK_LAUNCH("reinit_change");
        }
        EVAP_CUDA(cudaMemcpyAsync(psi, w.t0, Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    if (last_change) {
        *last_change = 0.0;
        if (steps > 0) {
            EVAP_CUDA(cudaMemcpyAsync(h->geo_host, w.S + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
            EVAP_CUDA(cudaStreamSynchronize(s));
            *last_change = std::sqrt(h->geo_host[0]);
        }
    }
    return status;
}

// ------------------------------------------------------------------------------ level-set advection (step 1)
// Element matrices of the Crank-Nicolson advection operator (EVAP_ADVECT) with the mesh's nodal transport velocity
// interpolated at the point, A_e[i][j] = sum_q W N_i (N_j + theta dt u_Gamma . grad N_j): u_Gamma is fixed within a
// fixed-point pass, so the matrices are formed once per pass and assembled into the node stencil that every GMRES
// iteration of the pass applies (k_stencil_from_elem_full).  Layout [64][ncell], entry i * 8 + j.
__global__ void __launch_bounds__(128) k_advect_elem(MeshArgs<double> m, const double* __restrict__ ug,
                                                     double* __restrict__ E) {
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= m.ncell) return;
    Q1Cell c;
    int cx, cy, cz;
    q1_cell_nodes(cell, m.n, c, cx, cy, cz);
    double uv[3][8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 3; ++e) uv[e][j] = ug[e * m.Nphi + c.node[j]];
    // shape values and reference derivatives at the points are compile-time constants once the loops unroll, so the
    // mass part folds into constants and the advective part costs 24 + 24 + 64 FMA per point
    double a[64] = {};
    const double tw = m.theta * m.dt * m.inv_h;  // physical gradient = reference gradient / h
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const double tq[3] = {g2_point(q & 1), g2_point((q >> 1) & 1), g2_point(q >> 2)};
        double N[8], R[8][3];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int b[3] = {j & 1, (j >> 1) & 1, j >> 2};
            double v[3], dv[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                v[e] = b[e] ? tq[e] : 1.0 - tq[e];
                dv[e] = b[e] ? 1.0 : -1.0;
            }
            N[j] = v[0] * v[1] * v[2];
            R[j][0] = dv[0] * v[1] * v[2];
            R[j][1] = v[0] * dv[1] * v[2];
            R[j][2] = v[0] * v[1] * dv[2];
        }
        double U[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int e = 0; e < 3; ++e) U[e] += N[j] * uv[e][j];
        double sj[8];  // theta dt u . grad N_j at the point
#pragma unroll
        for (int j = 0; j < 8; ++j) sj[j] = tw * (U[0] * R[j][0] + U[1] * R[j][1] + U[2] * R[j][2]);
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[i * 8 + j] += 0.125 * N[i] * (N[j] + sj[j]);  // 2-point weights 1/2^3
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) E[(i * 8 + j) * m.ncell + cell] = m.vol_w * a[i * 8 + j];
    }
}

// The node stencil of sum_e A_e from general element matrices in FP64, entry (i, j) of cell e at E[(8 i + j) ncell + e]
// (k_advect_elem): per node, the rows of the (up to 8) cells around it summed by offset in FP64, then stored as pairs
// C[s N + node]; offsets without a cell get 0.  One thread per node: no atomics, a fixed sum order.
__global__ void __launch_bounds__(128) k_stencil_from_elem_full(int n, int64_t ncell, int64_t N,
                                                                const double* __restrict__ E, float2* __restrict__ C) {
    const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (node >= N) return;
    const unsigned m1 = (unsigned)n + 1u, nd = (unsigned)node;
    const unsigned t = nd / m1;
    const int i = (int)(nd - t * m1), k = (int)(t / m1), j = (int)(t - (unsigned)k * m1);
    double acc[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) acc[q] = 0.0;
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
        const int ox = cc & 1, oy = (cc >> 1) & 1, oz = cc >> 2;  // the node's corner in the cell
        const int cx = i - ox, cy = j - oy, cz = k - oz;
        if (cx < 0 || cy < 0 || cz < 0 || cx >= n || cy >= n || cz >= n) continue;
        const int64_t cell = cx + (int64_t)n * (cy + (int64_t)n * cz);
        const int li = ox + 2 * oy + 4 * oz;
#pragma unroll
        for (int lj = 0; lj < 8; ++lj) {
            const int sx = (lj & 1) - ox, sy = ((lj >> 1) & 1) - oy, sz = (lj >> 2) - oz;
            acc[9 * (sz + 1) + 3 * (sy + 1) + (sx + 1)] += E[(int64_t)(8 * li + lj) * ncell + cell];
        }
    }
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        const float hi = (float)acc[q];
        C[q * N + node] = make_float2(hi, (float)(acc[q] - (double)hi));
    }
}

// b = M phi^n / theta - (1 - theta) / theta A phi^n  (= (M - (1 - theta) dt C) phi^n / theta with A = M + theta dt C)
__global__ void k_advect_rhs(const double* __restrict__ Mphi, const double* __restrict__ Aphi, double theta,
                             double* __restrict__ b, int64_t N) {
    const double a = 1.0 / theta, c = (1.0 - theta) / theta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a * Mphi[i] - c * Aphi[i];
}

// out = phi clamped to [-1, 1] (the range of the level sets the transport velocity is evaluated on)
__global__ void k_clamp_unit(const double* __restrict__ phi, double* __restrict__ out, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = phi[i];
        out[i] = v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v);
    }
}

// Step 1 of Algorithm 2: phi^(0) = phi^n (the mesh's level set); per pass k the transport velocity of the clamped
// iterate phi^(k) (u_Gamma of the mesh's variant, Eqs. transport_vel_*), then phi^(k+1) from the Crank-Nicolson
// system (M + theta dt C) phi^(k+1) = (M - (1 - theta) dt C) phi^n of Eq. (weakFormLevelSet), solved by GMRES with
// the diagonal preconditioner, started from phi^(k), to |r| <= max(1e-12 |b|, 1e-20) (the paper's solver settings,
// the relative one taken against the residual of a zero start).  Stops after max_iters passes or once
// |phi^(k+1) - phi^(k)|_2 <= tol.
constexpr int ADVECT_RESTART = 30;
constexpr double ADVECT_REORTH = 1e-2;  // second Gram-Schmidt pass where the first one cancelled 99 % of |w|^2
int geo_advect_levelset(evap_mesh* h, double* phi, int max_iters, double tol, int* fp_iters, int* lin_iters,
                        double* last_change, cudaStream_t s) {
    const MeshArgs<double> lm = ls_args<double>(h);  // the level-set mesh
    int rc = geo_workspace(h);
    if (rc) return rc;
    CgSpace w = cg_space(h);
    const int64_t Np = lm.Nphi;
    const int G = blocks_for(Np, 256, 152 * 8);
    const unsigned gc = (unsigned)blocks_for(lm.ncell, 128, 1LL << 40);
    if ((rc = geo_elem_reserve(h, 64 * lm.ncell + 27 * Np))) return rc;  // FP64 element matrices, node stencil
    float2* Cn = reinterpret_cast<float2*>(h->geo_elem + 64 * lm.ncell);
    if (Np >= (int64_t)1 << 32) {
        set_error("level-set advection: the node stencil indexes nodes with 32 bits");
        return EVAP_EINVAL;
    }
    EVAP_CUDA(cudaMemcpyAsync(phi, h->phi, Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    int k = 0, lin = 0, status = EVAP_OK;
    double change = 0.0;
    while (k < max_iters) {
        const double* cur = h->phi;
        if (k > 0) {
            k_clamp_unit<<<G, 256, 0, s>>>(phi, w.t0, Np);
            EVAP_CHECK_LAUNCH("advect_clamp");
            cur = w.t0;
        }
        if ((rc = launch_transport_velocity(h, s, cur))) return rc;
        if ((rc = helmholtz_apply(h, 0.0, 1, h->phi, w.t1, s))) return rc;
        if ((rc = launch_levelset<double>(h, EVAP_ADVECT, h->phi, w.t2, s))) return rc;
        k_advect_rhs<<<G, 256, 0, s>>>(w.t1, w.t2, lm.theta, w.b, Np);
        EVAP_CHECK_LAUNCH("advect_rhs");
        k_advect_elem<<<gc, 128, 0, s>>>(lm, h->ugamma, h->geo_elem);
        EVAP_CHECK_LAUNCH("advect_elem");
        k_stencil_from_elem_full<<<(unsigned)blocks_for(Np, 128, 1LL << 40), 128, 0, s>>>(lm.n, lm.ncell, Np,
                                                                                         h->geo_elem, Cn);
        EVAP_CHECK_LAUNCH("advect_stencil");
        EVAP_CUDA(cudaMemcpyAsync(w.r, phi, Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
        double rel = 0.0;
        rc = gmres_solve_fused(h, NodeStencil{lm.n, Np, Cn}, ADVECT_RESTART, w.b, phi, 1e-12, 1e-20, 1000,
                               ADVECT_REORTH, &lin, &rel, s);
        if (rc == EVAP_ENOTCONV) status = rc;
        else if (rc) return rc;
        ++k;
        k_diff_norm<<<CG_BLOCKS, CG_THREADS, 0, s>>>(phi, w.r, Np, w.part, w.ticket, w.S + 5);
        EVAP_CHECK_LAUNCH("advect_change");
        EVAP_CUDA(cudaMemcpyAsync(h->geo_host, w.S + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
        EVAP_CUDA(cudaStreamSynchronize(s));
        change = std::sqrt(h->geo_host[0]);
        if (change <= tol) break;
    }
    EVAP_CUDA(cudaStreamSynchronize(s));
    if (fp_iters) *fp_iters = k;
    if (lin_iters) *lin_iters = lin;
    if (last_change) *last_change = change;
    return status;
}

}  // namespace evap
