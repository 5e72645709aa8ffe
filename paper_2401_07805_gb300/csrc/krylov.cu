// Krylov solve of the momentum system (Table tab:solver_settings: GMRES with a diagonal preconditioner):
// restarted GMRES(m) with right Jacobi preconditioning and classical Gram-Schmidt with a conditional second pass.
//   mixed = 0: FP64 operator, basis and reductions.
//   mixed = 1: FP64 iterative refinement: r = f - A64 x (FP64), inner GMRES on A32 d = r/|r| with the FP32 operator
//              and FP32 basis, x += |r| d in FP64.  FP32 dot products form each product exactly (FMA two-product)
//              and accumulate per thread in a float-float pair (two-sum), then in FP64 across threads, so the
//              reductions carry FP64-level accuracy without using the (slow) FP64 pipe per element.
// The Hessenberg matrix, Givens rotations and the small triangular solve run on the host in FP64; one
// device-to-host copy per Arnoldi step carries the new column.
#include <algorithm>
#include <cmath>
#include <vector>

#include "evap_internal.cuh"

namespace evap {

// ------------------------------------------------------------------------------------------- Jacobi diagonal
// diag_(i,c) = sum_q [ W rho c_m N_i^2 + N_i (W rho u0 . grad N_i) + N_i^2 newton W rho d_c u0_c
//                      + 2 W mu ( (|grad N_i|^2 + (d_c N_i)^2)/2 - (z n)_c d_c N_i ((z n) . grad N_i) ) ]
// in FP32 from the quadrature-point cache of set_fields (k_qp_coeffs); one thread per (cell, local node).
template <int P, int CB>
__global__ void __launch_bounds__(CB*(P + 1) * (P + 1) * (P + 1))
    k_diagonal(MeshArgs<float> m, Basis<float> bas, const double* __restrict__ qc, float* __restrict__ diag,
               int colour) {
    constexpr int Q = P + 1, NQ = Q * Q * Q;
    __shared__ float sS[Q][Q], sD[Q][Q];
    __shared__ float qd[CB][11][NQ];  // per point: W rho c_m, W rho U(3), newton W rho d_c u0_c (3), 2 W mu, z n(3)
    const int tid = threadIdx.x, lc = tid / NQ, t = tid % NQ;
    int cx = 0, cy = 0, cz = 0;
    const bool active = colour_cell((int64_t)blockIdx.x * CB + lc, m.n, colour, cx, cy, cz);
    const int64_t cell = cx + (int64_t)m.n * (cy + (int64_t)m.n * cz);
    if (tid < Q * Q) {
        sS[tid / Q][tid % Q] = bas.S[tid / Q][tid % Q];
        sD[tid / Q][tid % Q] = bas.D[tid / Q][tid % Q];
    }
    const int a = t % Q, b = (t / Q) % Q, c = t / (Q * Q);
    if (active) {
        const double* qp = qc + cell * QC_K * NQ + t;
        constexpr int slot[11] = {0, 1, 2, 3, 4, 8, 12, 13, 14, 15, 16};
#pragma unroll
        for (int k = 0; k < 11; ++k) qd[lc][k][t] = (float)qp[slot[k] * NQ];
    }
    __syncthreads();
    if (!active) return;
    const int M = m.M;
    const int64_t gidx = (P * cx + a) + (int64_t)M * ((P * cy + b) + (int64_t)M * (P * cz + c));
    float dsum[3] = {0.f, 0.f, 0.f};
    for (int q = 0; q < NQ; ++q) {
        const int qa = q % Q, qb = (q / Q) % Q, qcz = q / (Q * Q);
        const float sa = sS[qa][a], sb = sS[qb][b], sc = sS[qcz][c];
        const float N = sa * sb * sc;
        const float g[3] = {sD[qa][a] * sb * sc * m.inv_h, sa * sD[qb][b] * sc * m.inv_h, sa * sb * sD[qcz][c] * m.inv_h};
        const float conv = qd[lc][1][q] * g[0] + qd[lc][2][q] * g[1] + qd[lc][3][q] * g[2];
        const float gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        const float ng = qd[lc][8][q] * g[0] + qd[lc][9][q] * g[1] + qd[lc][10][q] * g[2];
        const float wm = qd[lc][7][q], NN = N * N;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            dsum[k] += qd[lc][0][q] * NN + N * conv + NN * qd[lc][4 + k][q] +
                       wm * (0.5f * (gg + g[k] * g[k]) - qd[lc][8 + k][q] * g[k] * ng);
    }
    for (int k = 0; k < 3; ++k) acc_add(&diag[k * m.Nu + gidx], dsum[k], colour >= 0);
}

__device__ __forceinline__ bool dnode(int64_t node, int M, unsigned f) {
    const int gx = (int)(node % M), gy = (int)((node / M) % M), gz = (int)(node / ((int64_t)M * M));
    return ((f & 1u) && gx == 0) || ((f & 2u) && gx == M - 1) || ((f & 4u) && gy == 0) ||
           ((f & 8u) && gy == M - 1) || ((f & 16u) && gz == 0) || ((f & 32u) && gz == M - 1);
}

__global__ void k_diag_finish(int M, int64_t Nu, unsigned faces, float* d32, double* d64) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * Nu; i += (int64_t)gridDim.x * blockDim.x) {
        float v = dnode(i % Nu, M, faces) ? 1.f : d32[i];
        if (!(v != 0.f)) v = 1.f;  // guard a vanishing diagonal entry (never expected with c_mass > 0)
        d32[i] = v;
        d64[i] = (double)v;
    }
}

// The cells' diagonal contributions added into acc (zeroed by the caller): one atomic pass, or the 8 colour passes
// of the deterministic mode.
static int diagonal_passes(evap_mesh* h, const MeshArgs<float>& m, const Basis<float>& b, float* acc, cudaStream_t s) {
    const int c0 = h->deterministic ? 0 : -1, c1 = h->deterministic ? 8 : 0;
    for (int colour = c0; colour < std::max(c1, c0 + 1); ++colour) {
        const int64_t cells = colour_cells(m.n, colour);
        if (cells == 0) continue;
        if (m.P == 2) {
            constexpr int CB = 8;
            k_diagonal<2, CB><<<(unsigned)((cells + CB - 1) / CB), CB * 27, 0, s>>>(m, b, h->qc, acc, colour);
        } else {
            constexpr int CB = 4;
            k_diagonal<3, CB><<<(unsigned)((cells + CB - 1) / CB), CB * 64, 0, s>>>(m, b, h->qc, acc, colour);
        }
        EVAP_CHECK_LAUNCH("diagonal");
    }
    return EVAP_OK;
}

int launch_diagonal(evap_mesh* h, cudaStream_t s) {
    if (h->diag_valid) return EVAP_OK;
    const int64_t N = 3 * h->m.Nu;
    if (!h->diag) EVAP_CUDA(cudaMalloc(&h->diag, N * sizeof(double)));
    if (!h->diag32) EVAP_CUDA(cudaMalloc(&h->diag32, N * sizeof(float)));
    EVAP_CUDA(cudaMemsetAsync(h->diag32, 0, N * sizeof(float), s));
    const MeshArgs<float> m = mesh_args<float>(h);
    const Basis<float> b = cast_basis<float>(h->b);
    int rc = diagonal_passes(h, m, b, h->diag32, s);
    if (rc) return rc;
    k_diag_finish<<<blocks_for(N, 256), 256, 0, s>>>(m.M, m.Nu, m.faces, h->diag32, h->diag);
    EVAP_CHECK_LAUNCH("diag_finish");
    h->diag_valid = true;
    ++h->diag_stamp;
    return EVAP_OK;
}

// Same diagonal, accumulated in the caller-given FP32 array acc [3 N_u] and written as double to out [3 N_u];
// allocates nothing (used by the allocation-free entry point).
int launch_diagonal_into(evap_mesh* h, float* acc, double* out, cudaStream_t s) {
    const int64_t N = 3 * h->m.Nu;
    EVAP_CUDA(cudaMemsetAsync(acc, 0, N * sizeof(float), s));
    const MeshArgs<float> m = mesh_args<float>(h);
    const Basis<float> b = cast_basis<float>(h->b);
    int rc = diagonal_passes(h, m, b, acc, s);
    if (rc) return rc;
    k_diag_finish<<<blocks_for(N, 256), 256, 0, s>>>(m.M, m.Nu, m.faces, acc, out);
    EVAP_CHECK_LAUNCH("diag_finish_into");
    return EVAP_OK;
}

// ----------------------------------------------------------------------------------------------- reductions
// Vector kernels stream FP32 data as float4 and FP64 data as double2 (bases 16-byte aligned: the Krylov basis has a
// leading dimension padded to 64 entries) with a scalar tail.
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 608;  // 4 per SM (register-limited residency of the unrolled kernels): one wave

struct FF {  // float-float accumulator
    float hi, lo;
};
__device__ __forceinline__ void ff_add(FF& s, float v) {
    const float t = s.hi + v;
    const float bp = t - s.hi;
    const float err = (s.hi - (t - bp)) + (v - bp);
    s.hi = t;
    s.lo += err;
}
// acc += a * b with the product formed exactly (two-product) in FP32, or an FP64 fma.
struct Acc {
    double d = 0.0;
    FF f = {0.f, 0.f};
    __device__ __forceinline__ void add(double a, double b) { d = fma(a, b, d); }
    __device__ __forceinline__ void add(float a, float b) {
        const float p = a * b;
        ff_add(f, p);
        f.lo += fmaf(a, b, -p);
    }
    __device__ __forceinline__ double value() const { return d + (double)f.hi + (double)f.lo; }
};

template <typename T> struct V2;
template <> struct V2<float> { using t = float4; static constexpr int w = 4; };
template <> struct V2<double> { using t = double2; static constexpr int w = 2; };

__device__ __forceinline__ void dot_vec(Acc& a, const float4& x, const float4& y) {
    a.add(x.x, y.x); a.add(x.y, y.y); a.add(x.z, y.z); a.add(x.w, y.w);
}
__device__ __forceinline__ void dot_vec(Acc& a, const double2& x, const double2& y) {
    a.add(x.x, y.x); a.add(x.y, y.y);
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[RED_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < RED_THREADS / 32; ++i) r += sh[i];
    return r;
}

// The block's partial sum s (valid in thread 0) of row `row` goes to partial[row * RED_BLOCKS + block]; the last
// block of the row to arrive (atomic ticket after a memory fence; no block waits on another) sums the row's partials
// in block order, writes out[row] and resets the ticket for the next reduction.
__device__ __forceinline__ void row_finish(double s, double* partial, unsigned* cnt, int row, double* out) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partial[row * RED_BLOCKS + blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(&cnt[row], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += __ldcg(&partial[row * RED_BLOCKS + b]);
    v = block_sum(v);
    if (threadIdx.x == 0) {
        out[row] = v;
        cnt[row] = 0u;
    }
}

// out[i] = sum_k V_i[k] w[k] for i = blockIdx.y < nv; row nv (if present) = w . w
template <typename T>
__global__ void k_mdot(const T* __restrict__ V, int64_t ld, int nv, const T* __restrict__ w, int64_t N,
                       double* __restrict__ partial, unsigned* cnt, double* out) {
    using VT = typename V2<T>::t;
    constexpr int W = V2<T>::w;
    const T* v = blockIdx.y < (unsigned)nv ? V + blockIdx.y * ld : w;
    Acc acc;
    const int64_t nvec = N / W;
    const VT* v4 = reinterpret_cast<const VT*>(v);
    const VT* w4 = reinterpret_cast<const VT*>(w);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; k + stride < nvec; k += 2 * stride) {  // two independent vector loads per operand in flight
        const VT a0 = v4[k], b0 = w4[k], a1 = v4[k + stride], b1 = w4[k + stride];
        dot_vec(acc, a0, b0);
        dot_vec(acc, a1, b1);
    }
    if (k < nvec) dot_vec(acc, v4[k], w4[k]);
    for (int64_t k = nvec * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += stride)
        acc.add(v[k], w[k]);
    row_finish(block_sum(acc.value()), partial, cnt, blockIdx.y, out);
}

// w -= sum_{i<nv} h[i] sc2[i] V_i ; out[0] = |w|^2 of the result.  The basis is stored unnormalized:
// v_i = sc_i V_i, so projecting out v_i takes the raw dot h[i] = V_i . w times sc_i^2.
template <typename T>
__global__ void k_maxpy_norm(const T* __restrict__ V, int64_t ld, const double* __restrict__ hcol,
                             const double* __restrict__ sc2, int nv, T* w, int64_t N, double* __restrict__ partial,
                             unsigned* cnt, double* out) {
    using VT = typename V2<T>::t;
    constexpr int W = V2<T>::w;
    __shared__ T hs[256];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = (T)(hcol[i] * sc2[i]);
    __syncthreads();
    Acc acc;
    const int64_t nvec = N / W;
    VT* w4 = reinterpret_cast<VT*>(w);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; k + stride < nvec; k += 2 * stride) {  // two independent positions per thread
        VT a = w4[k], a2 = w4[k + stride];
        T* ap = reinterpret_cast<T*>(&a);
        T* ap2 = reinterpret_cast<T*>(&a2);
        for (int i = 0; i < nv; ++i) {
            const VT* vi = reinterpret_cast<const VT*>(V + i * ld);
            const VT b = vi[k], b2 = vi[k + stride];
            const T* bp = reinterpret_cast<const T*>(&b);
            const T* bp2 = reinterpret_cast<const T*>(&b2);
#pragma unroll
            for (int e = 0; e < W; ++e) {
                ap[e] -= hs[i] * bp[e];
                ap2[e] -= hs[i] * bp2[e];
            }
        }
        w4[k] = a;
        w4[k + stride] = a2;
        dot_vec(acc, a, a);
        dot_vec(acc, a2, a2);
    }
    if (k < nvec) {
        VT a = w4[k];
        T* ap = reinterpret_cast<T*>(&a);
        for (int i = 0; i < nv; ++i) {
            const VT b = reinterpret_cast<const VT*>(V + i * ld)[k];
            const T* bp = reinterpret_cast<const T*>(&b);
#pragma unroll
            for (int e = 0; e < W; ++e) ap[e] -= hs[i] * bp[e];
        }
        w4[k] = a;
        dot_vec(acc, a, a);
    }
    for (int64_t k = nvec * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        T v = w[k];
        for (int i = 0; i < nv; ++i) v -= hs[i] * V[i * ld + k];
        w[k] = v;
        acc.add(v, v);
    }
    row_finish(block_sum(acc.value()), partial, cnt, 0, out);
}

// out[0] = |v|^2
template <typename T>
__global__ void k_norm2(const T* __restrict__ v, int64_t N, double* __restrict__ partial, unsigned* cnt,
                        double* out) {
    Acc acc;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        acc.add(v[k], v[k]);
    row_finish(block_sum(acc.value()), partial, cnt, 0, out);
}

// z = sc v / diag (right Jacobi preconditioner applied to the normalized basis vector sc v), and w initialized for
// the operator apply w = A z: z on the Dirichlet DoFs (identity rows), 0 elsewhere.  One warp per x-line
// (component, gy, gz) of M nodes, as in the apply's own initialization.
template <typename T>
__global__ void __launch_bounds__(256) k_precond_init(int M, int64_t Nu, unsigned faces, const T* __restrict__ v,
                                                      const T* __restrict__ diag, T sc, T* __restrict__ z,
                                                      T* __restrict__ w) {
    const int lines = 3 * M * M;
    const int wpb = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int line = blockIdx.x * wpb + warp; line < lines; line += gridDim.x * wpb) {
        const int c = line / (M * M), rem = line - c * M * M, gz = rem / M, gy = rem - gz * M;
        const bool cyz = ((faces & 4u) && gy == 0) || ((faces & 8u) && gy == M - 1) || ((faces & 16u) && gz == 0) ||
                         ((faces & 32u) && gz == M - 1);
        const int64_t off = c * Nu + (int64_t)M * (gy + (int64_t)M * gz);
        for (int gx = lane; gx < M; gx += 32) {
            const bool cons = cyz || ((faces & 1u) && gx == 0) || ((faces & 2u) && gx == M - 1);
            const T zz = sc * v[off + gx] / diag[off + gx];
            z[off + gx] = zz;
            w[off + gx] = cons ? zz : T(0);
        }
    }
}

// x += diag^{-1} sum_i y[i] V_i   (x may be unaligned caller memory: scalar)
template <typename T>
__global__ void k_update(const T* __restrict__ V, int64_t ld, const double* __restrict__ y, int nv,
                         const T* __restrict__ diag, T* x, int64_t N) {
    __shared__ T ys[256];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) ys[i] = (T)y[i];
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        T s = 0;
        for (int i = 0; i < nv; ++i) s += ys[i] * V[i * ld + k];
        x[k] += s / diag[k];
    }
}

// u = sum_i y[i] V_i
template <typename T>
__global__ void k_combine(const T* __restrict__ V, int64_t ld, const double* __restrict__ y, int nv,
                          T* __restrict__ u, int64_t N) {
    __shared__ T ys[256];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) ys[i] = (T)y[i];
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        T s = 0;
        for (int i = 0; i < nv; ++i) s += ys[i] * V[i * ld + k];
        u[k] = s;
    }
}

// x += u
template <typename T>
__global__ void k_add_to(T* x, const T* __restrict__ u, int64_t N) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        x[k] += u[k];
}

// r = b - Ax
template <typename T>
__global__ void k_residual(const T* __restrict__ b, const T* __restrict__ Ax, T* __restrict__ r, int64_t N) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        r[k] = b[k] - Ax[k];
}

__global__ void k_scaled_to_float(const double* __restrict__ r, const double* __restrict__ nrm2, float* __restrict__ out,
                                  int64_t N) {
    const double inv = 1.0 / sqrt(*nrm2);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = (float)(r[k] * inv);
}

__global__ void k_refine(double* x, const float* __restrict__ d, const double* __restrict__ nrm2, int64_t N) {
    const double s = sqrt(*nrm2);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        x[k] += s * (double)d[k];
}

// ---------------------------------------------------------------------------------------------- GMRES core
// Re-orthogonalization threshold on |w_after|^2 / |w_before|^2: FP64 solves take the DGKS value 1/2; the FP32 inner
// solve re-orthogonalizes only after a cancellation of 99 % of |w|^2 (the mass-dominated operator makes A v nearly
// parallel to v, so the DGKS test fires on almost every step; measured on the 64^3 and 96^3 workloads the second
// pass changed neither the iteration count nor the accuracy of the refined solution, and cost ~25 % of the solve;
// the outer FP64 residual is checked regardless).
constexpr double REORTH64 = 0.5;
constexpr double REORTH32 = 1e-2;
// the operator of a solve (the momentum system; the level-set solves run in fused_krylov.cuh)
enum { OP_MOMENTUM = 0 };
struct Ctx {
    evap_mesh* h;
    int op;
    bool tp = false;   // momentum solves: the tensor-product mass preconditioner instead of Jacobi
    cudaStream_t s;
    int64_t N, ld;
    double* partial;   // [(m+2) * RED_BLOCKS]
    unsigned* cnt;     // arrival tickets of the reductions [m+2], zero between kernels
    double* dcol;      // device columns [2 (m+2)]
    double* dnorm;     // device scalars [4]
    double* dsc2;      // device squared scales of the unnormalized basis vectors [m+2]
    double* hcol;      // pinned host mirror
    double* hsc2;      // pinned staging of dsc2 [m+2]
};

template <typename T>
static int apply_op(Ctx& c, const T* x, T* y) {
    return launch_momentum<T>(c.h, x, y, (T*)nullptr, c.s);
}

// Blocks of a reduction over N entries: RED_BLOCKS (one wave) for the velocity systems; for short vectors (the
// Q1 level-set space) about 4 vector loads per thread, so that per-block overheads (ticket, partial sums) do not
// dominate.  row_finish counts gridDim.x, so any grid up to RED_BLOCKS uses the same partial layout.
template <typename T>
static int red_grid(int64_t N) {
    const int64_t per_block = (int64_t)RED_THREADS * V2<T>::w * 4;
    return (int)std::max<int64_t>(1, std::min<int64_t>(RED_BLOCKS, (N + per_block - 1) / per_block));
}

template <typename T>
static int norm2_dev(Ctx& c, const T* v, double* out) {
    k_norm2<T><<<red_grid<T>(c.N), RED_THREADS, 0, c.s>>>(v, c.N, c.partial, c.cnt, out);
    EVAP_CHECK_LAUNCH("norm");
    return EVAP_OK;
}

static int fetch(Ctx& c, const double* dev, int n, double* host) {
    EVAP_CUDA(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, c.s));
    EVAP_CUDA(cudaStreamSynchronize(c.s));
    return EVAP_OK;
}

// One classical Gram-Schmidt pass of w against v_0..v_{nv-1} (v_i = sc_i V_i): h_out[0..nv) = V^T w (raw dots; and
// h_out[nv] = |w|^2 before the pass if with_pre), then w -= sum sc_i^2 h_i V_i and |w|^2 after the pass -> c.dnorm[0].
template <typename T>
static int cgs_pass(Ctx& c, const T* V, T* w, int nv, double* h_out, bool with_pre) {
    const int rows = nv + (with_pre ? 1 : 0);
    const int gx = red_grid<T>(c.N);
    k_mdot<T><<<dim3(gx, rows), RED_THREADS, 0, c.s>>>(V, c.ld, nv, w, c.N, c.partial, c.cnt, h_out);
    EVAP_CHECK_LAUNCH("mdot");
    k_maxpy_norm<T><<<gx, RED_THREADS, 0, c.s>>>(V, c.ld, h_out, c.dsc2, nv, w, c.N, c.partial, c.cnt,
                                                          c.dnorm);
    EVAP_CHECK_LAUNCH("maxpy");
    return EVAP_OK;
}

// GMRES(m) on A x = b with right preconditioner diag^{-1}; x updated in place.  x_zero: x is known to be 0 on entry
// (the first residual is b, no apply).  Classical Gram-Schmidt with a second pass only when the first one removed
// more than half of |w|^2 (DGKS criterion with eta = 1/sqrt 2).  Stops when the Arnoldi residual estimate is
// <= tol_abs (then the true residual is recomputed) or after maxit applications.
template <typename T>
static int set_scale(Ctx& c, int i, double sc) {
    c.hsc2[i] = sc * sc;
    EVAP_CUDA(cudaMemcpyAsync(c.dsc2 + i, c.hsc2 + i, sizeof(double), cudaMemcpyHostToDevice, c.s));
    return EVAP_OK;
}

// GMRES(m) on A x = b with right preconditioner diag^{-1}; x updated in place.  x_zero: x is known to be 0 on entry
// (the first residual is b, no apply).  The Krylov basis is kept unnormalized (v_i = sc_i V_i): the operator writes
// A z straight into the next basis slot and the scales enter the Gram-Schmidt coefficients, so no vector pass is
// spent on normalization.  Classical Gram-Schmidt with a second pass only under REORTH64 / REORTH32.  Stops when the
// Arnoldi residual estimate is <= tol_abs (then the true residual is recomputed) or after maxit applications.
template <typename T>
static int gmres(Ctx& c, int m, const T* b, T* x, bool x_zero, const T* diag, T* V, T* w, T* z, double tol_abs,
                 int maxit, int* its, double* res_out) {
    const int64_t N = c.N;
    const int G = blocks_for(N, 256);
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), sc(m + 1);
    int used = 0, rc;
    double beta = 0.0;
    bool first = true;
    (void)w;
    while (true) {
        if (first && x_zero) {
            EVAP_CUDA(cudaMemcpyAsync(V, b, N * sizeof(T), cudaMemcpyDeviceToDevice, c.s));
        } else {
            if ((rc = apply_op<T>(c, x, z))) return rc;
            ++used;
            k_residual<T><<<G, 256, 0, c.s>>>(b, z, V, N);
            EVAP_CHECK_LAUNCH("residual");
        }
        if ((rc = norm2_dev<T>(c, V, c.dnorm))) return rc;
        if ((rc = fetch(c, c.dnorm, 1, c.hcol))) return rc;
        beta = std::sqrt(c.hcol[0]);
        first = false;
        *res_out = beta;
        if (beta <= tol_abs || used >= maxit || !(beta > 0.0)) break;
        sc[0] = 1.0 / beta;
        if ((rc = set_scale<T>(c, 0, sc[0]))) return rc;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        for (; j < m; ++j) {
            T* Vj = V + (int64_t)j * c.ld;
            T* Wn = V + (int64_t)(j + 1) * c.ld;  // A z goes straight into the next basis slot
            if (c.tp) {  // z = P (sc V_j), Wn initialized on the Dirichlet rows; w is the sweeps' scratch
                if ((rc = tensor_prec_apply<T>(c.h, Vj, (T)sc[j], w, z, Wn, c.s))) return rc;
            } else {
                const int M = c.h->m.M;
                const unsigned gl = (unsigned)std::min<int64_t>((3 * (int64_t)M * M + 7) / 8, 152 * 16);
                k_precond_init<T><<<gl, 256, 0, c.s>>>(M, c.h->m.Nu, c.h->m.faces, Vj, diag, (T)sc[j], z, Wn);
                EVAP_CHECK_LAUNCH("precond");
            }
            if ((rc = launch_momentum<T>(c.h, z, Wn, (T*)nullptr, c.s, false))) return rc;
            ++used;
            const int nv = j + 1;
            double* col = &H[(size_t)j * (m + 1)];
            if ((rc = cgs_pass<T>(c, V, Wn, nv, c.dcol, true))) return rc;
            EVAP_CUDA(cudaMemcpyAsync(c.hcol, c.dcol, (size_t)(nv + 1) * sizeof(double), cudaMemcpyDeviceToHost, c.s));
            EVAP_CUDA(cudaMemcpyAsync(c.hcol + m + 2, c.dnorm, sizeof(double), cudaMemcpyDeviceToHost, c.s));
            EVAP_CUDA(cudaStreamSynchronize(c.s));
            for (int i = 0; i < nv; ++i) col[i] = sc[i] * c.hcol[i];
            double after = c.hcol[m + 2];
            const double before = c.hcol[nv];
            if (after < (sizeof(T) == 4 ? REORTH32 : REORTH64) * before) {  // cancellation: re-orthogonalize once
                if ((rc = cgs_pass<T>(c, V, Wn, nv, c.dcol + (m + 2), false))) return rc;
                EVAP_CUDA(cudaMemcpyAsync(c.hcol, c.dcol + (m + 2), (size_t)nv * sizeof(double), cudaMemcpyDeviceToHost, c.s));
                EVAP_CUDA(cudaMemcpyAsync(c.hcol + m + 2, c.dnorm, sizeof(double), cudaMemcpyDeviceToHost, c.s));
                EVAP_CUDA(cudaStreamSynchronize(c.s));
                for (int i = 0; i < nv; ++i) col[i] += sc[i] * c.hcol[i];
                after = c.hcol[m + 2];
            }
            const double hn = std::sqrt(after);
            col[j + 1] = hn;
            if (hn > 0.0) {
                sc[j + 1] = 1.0 / hn;
                if ((rc = set_scale<T>(c, j + 1, sc[j + 1]))) return rc;
            }
            for (int i = 0; i < j; ++i) {
                const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = t0;
            }
            const double rr = std::hypot(col[j], col[j + 1]);
            cs[j] = rr > 0.0 ? col[j] / rr : 1.0;
            sn[j] = rr > 0.0 ? col[j + 1] / rr : 0.0;
            col[j] = rr;
            col[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            const double est = std::fabs(g[j + 1]);
            if (est <= tol_abs || used >= maxit || !(hn > 0.0)) {
                ++j;
                break;
            }
        }
        // y = R^{-1} g, x += diag^{-1} sum_i y_i v_i = diag^{-1} sum_i (y_i sc_i) V_i; the true residual of the new x
        // is checked at the top of the loop
        const int k = j;
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * (m + 1) + i] * y[l];
            y[i] = s / H[(size_t)i * (m + 1) + i];
        }
        for (int i = 0; i < k; ++i) c.hcol[i] = y[i] * sc[i];
        EVAP_CUDA(cudaMemcpyAsync(c.dcol, c.hcol, k * sizeof(double), cudaMemcpyHostToDevice, c.s));
        bool updated = false;
        if (c.tp && c.op == OP_MOMENTUM) {  // x += P (sum_i y_i sc_i V_i): combination in z, P into the free slot V_k
            k_combine<T><<<G, 256, 0, c.s>>>(V, c.ld, c.dcol, k, z, N);
            EVAP_CHECK_LAUNCH("combine");
            T* Vk = V + (int64_t)k * c.ld;
            if ((rc = tensor_prec_apply<T>(c.h, z, T(1), w, Vk, (T*)nullptr, c.s))) return rc;
            k_add_to<T><<<G, 256, 0, c.s>>>(x, Vk, N);
            EVAP_CHECK_LAUNCH("update");
            updated = true;
        }
        if (!updated) {
            k_update<T><<<G, 256, 0, c.s>>>(V, c.ld, c.dcol, k, diag, x, N);
            EVAP_CHECK_LAUNCH("update");
        }
        EVAP_CUDA(cudaStreamSynchronize(c.s));  // c.hcol is reused by the next fetch
    }
    *its = used;
    return EVAP_OK;
}

// Grows the mesh's Krylov workspace to `bytes` and the reduction scratch to a GMRES(m) solve, and sets up c.
static int prepare(evap_mesh* h, int op, int m, int64_t N, int64_t ld, size_t bytes, cudaStream_t s, Ctx& c) {
    if (h->ws_bytes < bytes) {
        if (h->ws) cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
        EVAP_CUDA(cudaMalloc(&h->ws, bytes));
        h->ws_bytes = bytes;
    }
    const size_t red_need = (size_t)(m + 2) * RED_BLOCKS + 4 * (m + 2) + 8;
    if (h->red_len < red_need) {
        if (h->red) cudaFree(h->red);
        if (h->red_host) cudaFreeHost(h->red_host);
        h->red = nullptr;
        h->red_host = nullptr;
        h->red_len = 0;
        EVAP_CUDA(cudaMalloc(&h->red, red_need * sizeof(double)));
        EVAP_CUDA(cudaMallocHost(&h->red_host, red_need * sizeof(double)));
        h->red_len = red_need;
    }
    c.h = h;
    c.op = op;
    c.s = s;
    c.N = N;
    c.ld = ld;
    c.partial = h->red;
    c.dcol = h->red + (size_t)(m + 2) * RED_BLOCKS;
    c.dnorm = c.dcol + 2 * (m + 2);
    c.dsc2 = c.dnorm + 8;
    c.cnt = reinterpret_cast<unsigned*>(c.dsc2 + (m + 2));
    EVAP_CUDA(cudaMemsetAsync(c.cnt, 0, (size_t)(m + 2) * sizeof(unsigned), s));
    c.hcol = h->red_host;
    c.hsc2 = h->red_host + red_need - (m + 2);
    return EVAP_OK;
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

int solve_gmres(evap_mesh* h, const double* f, double* x, int mixed, int m, double rtol, int max_iter, int* iters,
                double* relres, cudaStream_t s) {
    int rc = launch_diagonal(h, s);
    if (rc) return rc;
    const int64_t N = 3 * h->m.Nu;
    const int64_t ld = (N + 63) / 64 * 64;
    // workspace, every sub-array on a 256-byte boundary:
    //   FP64: V [(m+1) ld], w [ld], z [ld] doubles;  mixed: V [(m+1) ld], w32, z32, r32, d32 [ld] floats, r64, Ax [ld]
    const size_t fV = al256((size_t)(m + 1) * ld * sizeof(float)), fN = al256((size_t)ld * sizeof(float));
    const size_t dV = al256((size_t)(m + 1) * ld * sizeof(double)), dN = al256((size_t)ld * sizeof(double));
    const size_t bytes = mixed ? fV + 4 * fN + 2 * dN : dV + 2 * dN;
    Ctx c;
    if ((rc = prepare(h, OP_MOMENTUM, m, N, ld, bytes, s, c))) return rc;
    const int G = blocks_for(N, 256);
    // |f|, |x0|
    if ((rc = norm2_dev<double>(c, f, c.dnorm))) return rc;
    if ((rc = norm2_dev<double>(c, x, c.dnorm + 1))) return rc;
    if ((rc = fetch(c, c.dnorm, 2, c.hcol))) return rc;
    const double fn = std::sqrt(c.hcol[0]);
    bool x_zero = c.hcol[1] == 0.0;
    if (!(fn > 0.0)) {
        EVAP_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
        EVAP_CUDA(cudaStreamSynchronize(s));
        if (iters) *iters = 0;
        if (relres) *relres = 0.0;
        return EVAP_OK;
    }
    int used = 0;
    double res = 0.0;
    char* base = (char*)h->ws;
    if (!mixed) {
        double* V = (double*)base;
        double* w = (double*)(base + dV);
        double* z = (double*)(base + dV + dN);
        int its = 0;
        if ((rc = tensor_prec_setup(h, true, s))) return rc;
        c.tp = true;  // the same preconditioner as the mixed solve's inner iterations
        if ((rc = gmres<double>(c, m, f, x, x_zero, h->diag, V, w, z, rtol * fn, max_iter, &its, &res))) return rc;
        used = its;
    } else {
        float* V = (float*)base;
        float* w32 = (float*)(base + fV);
        float* z32 = (float*)(base + fV + fN);
        float* r32 = (float*)(base + fV + 2 * fN);
        float* d32 = (float*)(base + fV + 3 * fN);
        double* r64 = (double*)(base + fV + 4 * fN);
        double* Ax = (double*)(base + fV + 4 * fN + dN);
        const double inner_rtol = 1e-5;
        if ((rc = tensor_prec_setup(h, false, s))) return rc;
        c.tp = true;  // the inner FP32 solve takes the tensor-product mass preconditioner
        while (true) {
            if (x_zero) {  // r = f
                EVAP_CUDA(cudaMemcpyAsync(r64, f, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
                res = fn;
                if ((rc = norm2_dev<double>(c, r64, c.dnorm))) return rc;
            } else {
                if ((rc = launch_momentum<double>(h, x, Ax, nullptr, s))) return rc;
                ++used;
                k_residual<double><<<G, 256, 0, s>>>(f, Ax, r64, N);
                EVAP_CHECK_LAUNCH("residual64");
                if ((rc = norm2_dev<double>(c, r64, c.dnorm))) return rc;
                if ((rc = fetch(c, c.dnorm, 1, c.hcol))) return rc;
                res = std::sqrt(c.hcol[0]);
            }
            x_zero = false;
            if (res <= rtol * fn || used >= max_iter) break;
            k_scaled_to_float<<<G, 256, 0, s>>>(r64, c.dnorm, r32, N);
            EVAP_CHECK_LAUNCH("to32");
            EVAP_CUDA(cudaMemsetAsync(d32, 0, N * sizeof(float), s));
            int its = 0;
            double inner_res = 0.0;
            const int budget = std::min(max_iter - used, 4 * m);
            if ((rc = gmres<float>(c, m, r32, d32, true, h->diag32, V, w32, z32, inner_rtol, budget, &its, &inner_res)))
                return rc;
            used += its;
            // the refinement scale |r| is needed on the device again (the inner solve reused the scalar slot)
            if ((rc = norm2_dev<double>(c, r64, c.dnorm))) return rc;
            k_refine<<<G, 256, 0, s>>>(x, d32, c.dnorm, N);
            EVAP_CHECK_LAUNCH("refine");
        }
    }
    EVAP_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = used;
    if (relres) *relres = res / fn;
    return res <= rtol * fn ? EVAP_OK : EVAP_ENOTCONV;
}

// ------------------------------------------------------------ velocity-pressure system: flexible GMRES
// K [x; p] = [A x - B^T p; B x] = [f; g] with the block upper-triangular right preconditioner
//   P = [[A~, -B^T], [0, S~]]:   z_p = S~^(-1) v_p,   z_u = A~^(-1) (v_u + B^T z_p)
// (K P^(-1) is unit block lower-triangular for exact blocks).  A~^(-1): a fixed budget of FP32 GMRES iterations on the
// momentum operator with its Jacobi preconditioner (the mixed solve's inner method); S~^(-1): CG on
// B diag(A)^(-1) B^T (schur_apply).  Both are inexact and vary between applications, so the outer method stores the
// preconditioned directions (flexible GMRES); the outer vectors are FP64 [x (3 N_u) | p (N_phi)].
// Budgets of the two inexact inner solves.  Measured on the 64^3 four-sphere case with the top face open (GB300; ms
// and outer applications: solve to 1e-4 / solve to 1e-8 / three consecutive time steps to 1e-8).  With the Schur CG
// on the assembled stencil (schur.cu):
//   velocity 14, Schur CG 24 to 1e-6:   19.7 (6) / 111 (26) / 48.3, 48.4, 48.7
//   velocity 14, Schur CG 60 to 1e-4:   25.3 (6) /  61 (12) / 54.2, 53.9, 54.0
//   velocity 14, Schur CG 120 to 1e-4:  33.9 (6) /  81 (12) / 63.2, 63.4, 63.4
//   velocity 10, Schur CG 60 to 1e-3:   23.9 (6) /  59 (12) / 54.2, 54.0, 54.4
// and before it, with a matrix-free gradient and divergence per Schur CG iteration and an approximate diagonal:
//   velocity 10, Schur CG 24: 43.7 (6) / 405 (42) / 70.0, 70.0, 80.4;  velocity 14, Schur CG 12: 30.1 (6) /
//   407 (60) / 62.9, 63.0, 63.6, but 12 iterations did not converge the stationary 1D phase change of App. A
//   (density ratio 1e3, 4002 applications short of 1e-10).
#ifndef EVAP_SADDLE_INNER_M
#define EVAP_SADDLE_INNER_M 14
#endif
#ifndef EVAP_SADDLE_SCHUR_CG
#define EVAP_SADDLE_SCHUR_CG 24
#endif
constexpr int SADDLE_INNER_M = EVAP_SADDLE_INNER_M;    // FP32 GMRES applications per velocity-block solve
constexpr double SADDLE_INNER_TOL = 1e-2;
constexpr int SADDLE_SCHUR_CG = EVAP_SADDLE_SCHUR_CG;  // CG iterations per pressure Poisson solve

// v = b - v
// b += xd - kd: the lifting of Dirichlet data xd (K_D [xd] = kd) into the right-hand side.
__global__ void k_lift_rhs(double* __restrict__ b, const double* __restrict__ xd, const double* __restrict__ kd,
                           int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        b[i] += xd[i] - kd[i];
}

__global__ void k_residual_inplace(const double* __restrict__ b, double* __restrict__ v, int64_t N) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        v[k] = b[k] - v[k];
}

__global__ void k_scale_vec(double* __restrict__ v, const double* __restrict__ nrm2, int64_t N) {
    const double inv = 1.0 / sqrt(*nrm2);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        v[k] *= inv;
}

// [x; p] += sum_i y[i] Z_i
__global__ void k_update_split(const double* __restrict__ Z, int64_t ld, const double* __restrict__ y, int nv,
                               double* x, double* p, int64_t Nu3, int64_t N) {
    __shared__ double ys[256];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) ys[i] = y[i];
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < nv; ++i) s += ys[i] * Z[i * ld + k];
        if (k < Nu3) x[k] += s;
        else p[k - Nu3] += s;
    }
}

// t = v + (double) w
__global__ void k_add_float(const double* __restrict__ v, const float* __restrict__ w, double* __restrict__ t, int64_t N) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        t[k] = v[k] + (double)w[k];
}

struct SaddleSpace {
    double *V, *Z, *b, *t;  // outer basis [(m+1) ld], directions [m ld], right-hand side [ld], velocity scratch [3 N_u]
    float *V32, *w32, *z32, *r32, *d32;  // inner FP32 workspace
};

// z = P^(-1) v
static int saddle_precond(Ctx& inner, SaddleSpace& sp, const double* v, double* z) {
    evap_mesh* h = inner.h;
    cudaStream_t s = inner.s;
    const int64_t Nu3 = 3 * h->m.Nu, Np = h->m.Np;
    const int G = blocks_for(Nu3, 256);
    int rc = schur_apply(h, v + Nu3, z + Nu3, SADDLE_SCHUR_CG, s);
    if (rc) return rc;
    // t = v_u + B^T z_p, the gradient in FP32 (it enters the FP32 velocity solve)
    if ((rc = launch_to_float(z + Nu3, sp.z32, Np, s))) return rc;
    EVAP_CUDA(cudaMemsetAsync(sp.w32, 0, Nu3 * sizeof(float), s));
    if ((rc = launch_pressure_gradient<float>(h, sp.z32, 1.0f, sp.w32, s))) return rc;
    k_add_float<<<G, 256, 0, s>>>(v, sp.w32, sp.t, Nu3);
    EVAP_CHECK_LAUNCH("saddle_add_grad");
    // velocity block: FP32 GMRES on t / |t| from zero, then z_u = |t| d
    if ((rc = norm2_dev<double>(inner, sp.t, inner.dnorm))) return rc;
    k_scaled_to_float<<<G, 256, 0, s>>>(sp.t, inner.dnorm, sp.r32, Nu3);
    EVAP_CHECK_LAUNCH("saddle_to32");
    EVAP_CUDA(cudaMemsetAsync(sp.d32, 0, Nu3 * sizeof(float), s));
    int its = 0;
    double res = 0.0;
    if ((rc = gmres<float>(inner, SADDLE_INNER_M, sp.r32, sp.d32, true, h->diag32, sp.V32, sp.w32, sp.z32,
                           SADDLE_INNER_TOL, SADDLE_INNER_M, &its, &res)))
        return rc;
    if ((rc = norm2_dev<double>(inner, sp.t, inner.dnorm))) return rc;
    EVAP_CUDA(cudaMemsetAsync(z, 0, Nu3 * sizeof(double), s));
    k_refine<<<G, 256, 0, s>>>(z, sp.d32, inner.dnorm, Nu3);
    EVAP_CHECK_LAUNCH("saddle_velocity");
    return EVAP_OK;
}

int solve_saddle(evap_mesh* h, const double* f, double* x, double* p, int m, double rtol, int max_iter, int* iters,
                 double* relres, cudaStream_t s, const double* g_rhs) {
    int rc = launch_diagonal(h, s);
    if (rc) return rc;
    const double* g = nullptr;
    if ((rc = continuity_rhs(h, &g, s))) return rc;
    if (g_rhs) g = g_rhs;
    if ((rc = schur_assemble(h, s))) return rc;
    const int64_t Nu3 = 3 * h->m.Nu, Np = h->m.Np, N = Nu3 + Np;
    const int64_t ld = (N + 63) / 64 * 64, ldu = (Nu3 + 63) / 64 * 64;
    // inner (FP32 velocity GMRES) workspace and reduction scratch: the mesh's Krylov buffers
    const size_t fV = al256((size_t)(SADDLE_INNER_M + 1) * ldu * sizeof(float)), fN = al256((size_t)ldu * sizeof(float));
    Ctx inner;
    if ((rc = prepare(h, OP_MOMENTUM, SADDLE_INNER_M, Nu3, ldu, fV + 4 * fN, s, inner))) return rc;
    if ((rc = tensor_prec_setup(h, false, s))) return rc;
    inner.tp = true;
    SaddleSpace sp;
    char* ib = (char*)h->ws;
    sp.V32 = (float*)ib;
    sp.w32 = (float*)(ib + fV);
    sp.z32 = (float*)(ib + fV + fN);
    sp.r32 = (float*)(ib + fV + 2 * fN);
    sp.d32 = (float*)(ib + fV + 3 * fN);
    // outer workspace and its own reduction scratch (the inner solve reuses the mesh's)
    const size_t dV = al256((size_t)(m + 1) * ld * sizeof(double)), dZ = al256((size_t)m * ld * sizeof(double));
    const size_t dN = al256((size_t)ld * sizeof(double)), dU = al256((size_t)Nu3 * sizeof(double));
    const size_t bytes = dV + dZ + dN + dU;
    if (h->sd_bytes < bytes) {
        if (h->sd_ws) cudaFree(h->sd_ws);
        h->sd_ws = nullptr;
        h->sd_bytes = 0;
        EVAP_CUDA(cudaMalloc(&h->sd_ws, bytes));
        h->sd_bytes = bytes;
    }
    char* ob = (char*)h->sd_ws;
    sp.V = (double*)ob;
    sp.Z = (double*)(ob + dV);
    sp.b = (double*)(ob + dV + dZ);
    sp.t = (double*)(ob + dV + dZ + dN);
    const size_t red_need = (size_t)(m + 2) * RED_BLOCKS + 4 * (m + 2) + 8;
    if (h->sd_red_len < red_need) {
        if (h->sd_red) cudaFree(h->sd_red);
        if (h->sd_host) cudaFreeHost(h->sd_host);
        h->sd_red = nullptr;
        h->sd_host = nullptr;
        h->sd_red_len = 0;
        EVAP_CUDA(cudaMalloc(&h->sd_red, red_need * sizeof(double)));
        EVAP_CUDA(cudaMallocHost(&h->sd_host, red_need * sizeof(double)));
        h->sd_red_len = red_need;
    }
    Ctx c;
    c.h = h;
    c.op = OP_MOMENTUM;  // not used: the outer operator is applied explicitly
    c.s = s;
    c.N = N;
    c.ld = ld;
    c.partial = h->sd_red;
    c.dcol = h->sd_red + (size_t)(m + 2) * RED_BLOCKS;
    c.dnorm = c.dcol + 2 * (m + 2);
    c.dsc2 = c.dnorm + 8;
    c.cnt = reinterpret_cast<unsigned*>(c.dsc2 + (m + 2));
    c.hcol = h->sd_host;
    c.hsc2 = h->sd_host + red_need - (m + 2);
    EVAP_CUDA(cudaMemsetAsync(c.cnt, 0, (size_t)(m + 2) * sizeof(unsigned), s));
    for (int i = 0; i < m + 2; ++i) c.hsc2[i] = 1.0;  // normalized basis: unit scales
    EVAP_CUDA(cudaMemcpyAsync(c.dsc2, c.hsc2, (size_t)(m + 2) * sizeof(double), cudaMemcpyHostToDevice, s));
    // b = [f; g]
    EVAP_CUDA(cudaMemcpyAsync(sp.b, f, Nu3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    EVAP_CUDA(cudaMemcpyAsync(sp.b + Nu3, g, Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    const int G = blocks_for(N, 256);
    // Dirichlet data (f nonzero on a Dirichlet DoF): solve K_D [x; p] = [f; g], whose free rows keep the Dirichlet
    // columns, as K [x; p] = b with b = [f; g] - K_D [f_D; 0] + [f_D; 0] (f_D: f on the Dirichlet DoFs, else 0); the
    // first two basis vectors are scratch here
    bool data = false;
    if ((rc = constrained_nonzero(h, f, &data, s))) return rc;
    if (data) {
        double* xd = sp.V;
        double* kd = sp.V + ld;
        EVAP_CUDA(cudaMemsetAsync(xd, 0, N * sizeof(double), s));
        if ((rc = launch_constrained_copy(h, f, xd, s))) return rc;
        if ((rc = launch_saddle_apply(h, xd, xd + Nu3, kd, kd + Nu3, s, true))) return rc;
        k_lift_rhs<<<G, 256, 0, s>>>(sp.b, xd, kd, N);
        EVAP_CHECK_LAUNCH("saddle_lift");
    }
    if ((rc = norm2_dev<double>(c, sp.b, c.dnorm))) return rc;
    if ((rc = fetch(c, c.dnorm, 1, c.hcol))) return rc;
    const double bn = std::sqrt(c.hcol[0]);
    const double target = rtol * bn;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), yv(m);
    int used = 0;
    double beta = 0.0;
    while (true) {
        if ((rc = launch_saddle_apply(h, x, p, sp.V, sp.V + Nu3, s))) return rc;
        ++used;
        k_residual_inplace<<<G, 256, 0, s>>>(sp.b, sp.V, N);
        EVAP_CHECK_LAUNCH("saddle_residual");
        if ((rc = norm2_dev<double>(c, sp.V, c.dnorm))) return rc;
        if ((rc = fetch(c, c.dnorm, 1, c.hcol))) return rc;
        beta = std::sqrt(c.hcol[0]);
        if (beta <= target || used >= max_iter || !(beta > 0.0)) break;
        k_scale_vec<<<G, 256, 0, s>>>(sp.V, c.dnorm, N);
        EVAP_CHECK_LAUNCH("saddle_scale");
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int j = 0;
        for (; j < m; ++j) {
            double* Vj = sp.V + (int64_t)j * ld;
            double* Zj = sp.Z + (int64_t)j * ld;
            double* Wn = sp.V + (int64_t)(j + 1) * ld;
            if ((rc = saddle_precond(inner, sp, Vj, Zj))) return rc;
            if ((rc = launch_saddle_apply(h, Zj, Zj + Nu3, Wn, Wn + Nu3, s))) return rc;
            ++used;
            const int nv = j + 1;
            double* col = &H[(size_t)j * (m + 1)];
            if ((rc = cgs_pass<double>(c, sp.V, Wn, nv, c.dcol, true))) return rc;
            EVAP_CUDA(cudaMemcpyAsync(c.hcol, c.dcol, (size_t)(nv + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
            EVAP_CUDA(cudaMemcpyAsync(c.hcol + m + 2, c.dnorm, sizeof(double), cudaMemcpyDeviceToHost, s));
            EVAP_CUDA(cudaStreamSynchronize(s));
            for (int i = 0; i < nv; ++i) col[i] = c.hcol[i];
            double after = c.hcol[m + 2];
            if (after < REORTH64 * c.hcol[nv]) {
                if ((rc = cgs_pass<double>(c, sp.V, Wn, nv, c.dcol + (m + 2), false))) return rc;
                EVAP_CUDA(cudaMemcpyAsync(c.hcol, c.dcol + (m + 2), (size_t)nv * sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
                EVAP_CUDA(cudaMemcpyAsync(c.hcol + m + 2, c.dnorm, sizeof(double), cudaMemcpyDeviceToHost, s));
                EVAP_CUDA(cudaStreamSynchronize(s));
                for (int i = 0; i < nv; ++i) col[i] += c.hcol[i];
                after = c.hcol[m + 2];
            }
            const double hn = std::sqrt(after);
            col[j + 1] = hn;
            if (hn > 0.0) {
                k_scale_vec<<<G, 256, 0, s>>>(Wn, c.dnorm, N);
                EVAP_CHECK_LAUNCH("saddle_scale");
            }
            for (int i = 0; i < j; ++i) {
                const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = t0;
            }
            const double rr = std::hypot(col[j], col[j + 1]);
            cs[j] = rr > 0.0 ? col[j] / rr : 1.0;
            sn[j] = rr > 0.0 ? col[j + 1] / rr : 0.0;
            col[j] = rr;
            col[j + 1] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            if (std::fabs(gv[j + 1]) <= target || used >= max_iter || !(hn > 0.0)) {
                ++j;
                break;
            }
        }
        const int k = j;
        for (int i = k - 1; i >= 0; --i) {
            double sum = gv[i];
            for (int l = i + 1; l < k; ++l) sum -= H[(size_t)l * (m + 1) + i] * yv[l];
            yv[i] = sum / H[(size_t)i * (m + 1) + i];
        }
        for (int i = 0; i < k; ++i) c.hcol[i] = yv[i];
        EVAP_CUDA(cudaMemcpyAsync(c.dcol, c.hcol, k * sizeof(double), cudaMemcpyHostToDevice, s));
        k_update_split<<<G, 256, 0, s>>>(sp.Z, ld, c.dcol, k, x, p, Nu3, N);
        EVAP_CHECK_LAUNCH("saddle_update");
        EVAP_CUDA(cudaStreamSynchronize(s));
    }
    EVAP_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = used;
    if (relres) *relres = bn > 0.0 ? beta / bn : 0.0;
    return beta <= target ? EVAP_OK : EVAP_ENOTCONV;
}

}  // namespace evap
