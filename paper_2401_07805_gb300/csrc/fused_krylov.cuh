// Single-launch Krylov solvers of the level-set sub-solver (Algorithm 2): the Jacobi-preconditioned CG of the
// projected normal, the curvature and the reinitialization, and the diagonally preconditioned GMRES of the
// Crank-Nicolson advection (the paper's solver settings: CG for the symmetric, GMRES for the non-symmetric systems).
//
// On a 64^3 level-set mesh a vector is 275k entries (2.2 MB, resident in L2), so one iteration of a kernel-per-step
// solver is a handful of launches of a few microseconds each plus, for GMRES, a host round trip per Arnoldi step.  Here
// the whole solve is one cooperative launch: each block owns a fixed share of the nodes for all iterations, the grid
// meets at a barrier wherever a step reads other blocks' entries (the operator reads neighbours; a scalar product
// needs every block's partial), and the vectors are double-float pairs (dfloat.cuh) so that the iteration runs on the
// FP32 pipe; FP64 only converts the inputs and the result and forms the scalars.
//
// Scalar products are summed from per-block partials by every block in the same order, so all blocks take the same
// scalars and the same stopping decision and a solve is bitwise reproducible.  The barrier's wait is bounded: a block
// that polls longer than FK_SPIN_LIMIT times sets the error word and every block returns at its next barrier (the host
// reports EVAP_ETIMEOUT); the cooperative launch makes all blocks co-resident, so the limit is only a guard.
#pragma once

#include "dfloat.cuh"

namespace evap {

constexpr int FK_THREADS = 512;
constexpr int FK_WARPS = FK_THREADS / 32;
constexpr unsigned FK_SPIN_LIMIT = 1u << 24;  // polls of one L2 round trip each: ~0.5 s
constexpr int GM_MAX = 30;                    // largest GMRES restart length
constexpr int FK_MAX_BLOCKS = 304;            // largest grid (2 blocks per SM of a 152-SM GPU): sizes the partials

struct GridBarrier {
    unsigned long long count;  // arrivals since the launch (zeroed by the host before it)
    int err;                   // set by a block that gave up waiting
    int pad;
};

__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier on a monotonic arrival counter: block b's k-th barrier waits until the counter reaches
// k * gridDim.x.  The release add publishes the block's writes (ordered before it by the block barrier), the acquire
// load makes the other blocks' writes visible to the whole block (ordered after it by the second block barrier).
// Returns false, in every thread of the block, once any block has given up.
__device__ __forceinline__ bool grid_barrier(GridBarrier* gb, unsigned long long& target) {
    __shared__ int ok;
    target += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add(&gb->count, 1ull);
        int good = 1;
        unsigned polls = 0;
        while (ld_acquire(&gb->count) < target) {
            ++polls;
            if (polls > FK_SPIN_LIMIT || ((polls & 1023u) == 0u && *(volatile int*)&gb->err)) {
                atomicExch(&gb->err, 1);
                good = 0;
                break;
            }
        }
        if (good && *(volatile int*)&gb->err) good = 0;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ dfl warp_sum_df(dfl v) {
    v = df_norm(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const dfl u{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, u);
    }
    return v;  // valid in lane 0
}

__device__ __forceinline__ void st_df(float2* p, dfl a) { *p = make_float2(a.hi, a.lo); }

// K block sums at once (sh: K * FK_WARPS + K pairs), the results in every thread: each warp reduces its values by a
// shuffle tree, then warp k reduces the FK_WARPS warp sums of value k the same way (a fixed order, so the result does
// not depend on timing, and no serial loop over the warps).
template <int K>
__device__ __forceinline__ void block_sum_df(dfl (&v)[K], float2* sh) {
    static_assert(K <= FK_WARPS, "one warp per value");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum_df(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) st_df(sh + k * FK_WARPS + wid, v[k]);
    __syncthreads();
    if (wid < K) {
        dfl t = lane < FK_WARPS ? ld_df(sh + wid * FK_WARPS + lane) : dfl{0.f, 0.f};
        t = warp_sum_df(t);
        if (lane == 0) st_df(sh + K * FK_WARPS + wid, t);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = ld_df(sh + K * FK_WARPS + k);
}

// K grid sums of the partial arrays part[k * gridDim.x + b] (sh: K pairs), the results in every thread: warp k sums
// array k (lane-strided, then a shuffle tree), the same order in every block.
template <int K>
__device__ __forceinline__ void grid_sum_df(const float2* part, float2* sh, dfl (&v)[K]) {
    static_assert(K <= FK_WARPS, "one warp per value");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < K) {
        dfl t{0.f, 0.f};
        for (int i = lane; i < (int)gridDim.x; i += 32) {
            const float2 u = __ldcg(part + wid * gridDim.x + i);
            t = df_add(t, dfl{u.x, u.y});
        }
        t = warp_sum_df(t);
        if (lane == 0) st_df(sh + wid, t);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = ld_df(sh + k);
}

// ------------------------------------------------------------------------------------------- 27-point stencils
// The operators as 27-point stencils on the Q1 node lattice (n + 1 nodes per direction), x as pairs: row `node` is
// sum_s C_s(node) x(node + o_s) over the offsets o_s = (dx, dy, dz) in {-1, 0, 1}^3, s = 9 (dz + 1) + 3 (dy + 1) +
// (dx + 1), one double-float FMA per neighbour.  Offsets that leave the lattice are skipped.  Node indices fit 32
// bits (checked on the host).
template <class Coef>
__device__ __forceinline__ dfl stencil27(int n, int64_t node, const float2* x, Coef coef) {
    const unsigned m1 = (unsigned)n + 1u, nd = (unsigned)node;
    const unsigned t = nd / m1, i = nd - t * m1, k = t / m1, j = t - k * m1;
    dfl acc{0.f, 0.f};
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        if ((dz < 0 && k == 0u) || (dz > 0 && k == (unsigned)n)) continue;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            if ((dy < 0 && j == 0u) || (dy > 0 && j == (unsigned)n)) continue;
            const float2* xr = x + (nd + (unsigned)(dy * (int)m1 + dz * (int)(m1 * m1)));
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                if ((dx < 0 && i == 0u) || (dx > 0 && i == (unsigned)n)) continue;
                df_fma(acc, coef(i, j, k, 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1)), ld_df(xr + dx));
            }
        }
    }
    return df_norm(acc);
}

// (M + c K) for one field: constant coefficients per boundary class.  A node's class in one direction is 0 (first
// node), 1 (interior) or 2 (last node); table[27 class + s] holds C_s of class 9 cz + 3 cy + cx as pairs
// (helmholtz_table), staged in shared memory by load().
struct HelmholtzStencil {
    static constexpr int SMEM = 27 * 27;  // pairs
    int n;
    const float2* table;
    __device__ __forceinline__ void load(float2* sm) const {
        for (int t = threadIdx.x; t < SMEM; t += blockDim.x) sm[t] = table[t];
    }
    __device__ __forceinline__ dfl row(int64_t node, const float2* x, const float2* sm) const {
        return stencil27(n, node, x, [&](unsigned i, unsigned j, unsigned k, int s) {
            const unsigned cx = i == 0u ? 0u : (i == (unsigned)n ? 2u : 1u);
            const unsigned cy = j == 0u ? 0u : (j == (unsigned)n ? 2u : 1u);
            const unsigned cz = k == 0u ? 0u : (k == (unsigned)n ? 2u : 1u);
            return ld_df(sm + 27u * (9u * cz + 3u * cy + cx) + (unsigned)s);
        });
    }
    // the diagonal entry (offset 13 = (0, 0, 0)) to FP32, for the Jacobi scaling
    __device__ __forceinline__ float diag(int64_t node, const float2* sm) const {
        const unsigned m1 = (unsigned)n + 1u, nd = (unsigned)node;
        const unsigned t = nd / m1, i = nd - t * m1, k = t / m1, j = t - k * m1;
        const unsigned cx = i == 0u ? 0u : (i == (unsigned)n ? 2u : 1u);
        const unsigned cy = j == 0u ? 0u : (j == (unsigned)n ? 2u : 1u);
        const unsigned cz = k == 0u ? 0u : (k == (unsigned)n ? 2u : 1u);
        return sm[27u * (9u * cz + 3u * cy + cx) + 13u].x;
    }
};

// Host: the 27 x 27 coefficient table of (M + c K) on a lattice of spacing h, formed in FP64 from the 1D rows
// h/6, 2h/3, h/6 (mass) and -1/h, 2/h, -1/h (stiffness), with h/3 and 1/h as the centre entry of an end node.
inline void helmholtz_table(double h, double c, float2* out) {
    double M[3][3], K[3][3];  // [class][offset + 1]
    const double mi[3] = {h / 6.0, 2.0 * h / 3.0, h / 6.0}, ki[3] = {-1.0 / h, 2.0 / h, -1.0 / h};
    for (int o = 0; o < 3; ++o) {
        M[1][o] = mi[o];
        K[1][o] = ki[o];
    }
    M[0][0] = 0.0;     M[0][1] = h / 3.0; M[0][2] = h / 6.0;
    K[0][0] = 0.0;     K[0][1] = 1.0 / h; K[0][2] = -1.0 / h;
    M[2][0] = h / 6.0; M[2][1] = h / 3.0; M[2][2] = 0.0;
    K[2][0] = -1.0 / h; K[2][1] = 1.0 / h; K[2][2] = 0.0;
    for (int cz = 0; cz < 3; ++cz)
        for (int cy = 0; cy < 3; ++cy)
            for (int cx = 0; cx < 3; ++cx)
                for (int dz = 0; dz < 3; ++dz)
                    for (int dy = 0; dy < 3; ++dy)
                        for (int dx = 0; dx < 3; ++dx) {
                            const double mx = M[cx][dx], my = M[cy][dy], mz = M[cz][dz];
                            const double v = mx * my * mz + c * (K[cx][dx] * my * mz + mx * K[cy][dy] * mz +
                                                                 mx * my * K[cz][dz]);
                            const dfl d = df_from_double(v);
                            out[27 * (9 * cz + 3 * cy + cx) + 9 * dz + 3 * dy + dx] = make_float2(d.hi, d.lo);
                        }
}

// An operator assembled per node: C[s N + node] = C_s(node) as pairs (coalesced per offset).
struct NodeStencil {
    static constexpr int SMEM = 0;
    int n;
    int64_t N;
    const float2* C;
    __device__ __forceinline__ void load(float2*) const {}
    __device__ __forceinline__ dfl row(int64_t node, const float2* x, const float2*) const {
        const float2* c = C + node;
        const int64_t NN = N;
        return stencil27(n, node, x, [&](unsigned, unsigned, unsigned, int s) { return ld_df(c + s * NN); });
    }
    __device__ __forceinline__ float diag(int64_t node, const float2*) const { return C[13 * N + node].x; }
};

// ------------------------------------------------------------------------------------ conjugate gradients
// A x = b from x = 0, CG preconditioned by the operator's diagonal D (op.diag, in FP32), in the Chronopoulos-Gear
// arrangement (Chronopoulos and Gear, J. Comput. Appl. Math. 25, 1989): the two scalar products of an iteration, (r, u) and (A u, u), are formed in the same pass as
// the operator, with s = A p carried by its own recurrence, so an iteration needs two grid barriers (after the
// operator and its products; after the vector updates) instead of three.  With u = D^-1 r, w = A u:
//   gamma = (r, u), delta = (w, u), beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
//   (beta = 0, alpha = gamma / delta at the start), p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s.
// It stops once |r| <= max(rtol |r0|, atol) or after max_iter updates.  Vectors of N entries: xd, r, u, p, sv, w as
// pairs (u is read by op.row across blocks), dinv the FP32 inverse diagonal (any positive diagonal is a valid
// preconditioner; FP32 changes only the iteration count).  part holds 3 gridDim.x pairs.  out[0] = updates,
// out[1] = |r|, out[2] = |r0| (block 0).
template <class Op>
__global__ void __launch_bounds__(FK_THREADS) k_cg_fused(Op op, int64_t N, const double* __restrict__ b, double* x,
                                                         float2* xd,
                                                         float* dinv, float2* r, float2* u, float2* p, float2* sv,
                                                         float2* w, double rtol, double atol, int max_iter,
                                                         float2* part, GridBarrier* gb, double* out) {
    extern __shared__ float2 op_sm[];  // Op::SMEM pairs staged by op.load
    __shared__ float2 sh[3 * FK_WARPS + 3];
    __shared__ double s_res, s_r0;
    __shared__ dfl s_alpha, s_beta;
    __shared__ int s_go;
    unsigned long long bar = 0;
    const int64_t i0 = blockIdx.x * (int64_t)FK_THREADS + threadIdx.x, stride = (int64_t)gridDim.x * FK_THREADS;
    op.load(op_sm);
    __syncthreads();
    const dfl zero{0.f, 0.f};
    for (int64_t i = i0; i < N; i += stride) {
        const dfl ri = df_from_double(b[i]);
        const float di = 1.0f / op.diag(i, op_sm);
        st_df(xd + i, zero);
        st_df(r + i, ri);
        st_df(u + i, df_norm(dfl{ri.hi * di, __fmaf_rn(ri.hi, di, -ri.hi * di) + ri.lo * di}));
        st_df(p + i, zero);
        st_df(sv + i, zero);
        dinv[i] = di;
    }
    if (!grid_barrier(gb, bar)) return;
    double gamma_old = 0.0, alpha_old = 1.0, target = 0.0;  // thread 0's copies (the same in every block)
    int it = 0;
    for (;;) {
        dfl acc[3] = {zero, zero, zero};  // (r, u), (w, u), (r, r)
        for (int64_t i = i0; i < N; i += stride) {
            const dfl wi = op.row(i, u, op_sm), ui = ld_df(u + i), ri = ld_df(r + i);
            st_df(w + i, wi);
            df_fma(acc[0], ri, ui);
            df_fma(acc[1], wi, ui);
            df_fma(acc[2], ri, ri);
        }
        block_sum_df<3>(acc, sh);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < 3; ++k) st_df(part + k * gridDim.x + blockIdx.x, acc[k]);
        if (!grid_barrier(gb, bar)) return;
        grid_sum_df<3>(part, sh, acc);
        if (threadIdx.x == 0) {
            const double gam = df_to_double(acc[0]), del = df_to_double(acc[1]);
            const double res = sqrt(fmax(df_to_double(acc[2]), 0.0));
            if (it == 0) {
                s_r0 = res;
                target = fmax(rtol * res, atol);
            }
            s_res = res;
            s_go = res > target && it < max_iter;
            const double beta = it == 0 ? 0.0 : (gamma_old != 0.0 ? gam / gamma_old : 0.0);
            const double den = it == 0 ? del : del - beta * gam / alpha_old;
            const double alpha = den != 0.0 ? gam / den : 0.0;
            s_alpha = df_from_double(alpha);
            s_beta = df_from_double(beta);
            gamma_old = gam;
            alpha_old = alpha;
        }
        __syncthreads();
        if (!s_go) break;
        ++it;
        const dfl alpha = s_alpha, nalpha = df_neg(s_alpha), beta = s_beta;
        for (int64_t i = i0; i < N; i += stride) {
            const dfl ui = ld_df(u + i), wi = ld_df(w + i);
            dfl pi = ui, si = wi, xi = ld_df(xd + i), ri = ld_df(r + i);
            df_fma(pi, beta, ld_df(p + i));
            df_fma(si, beta, ld_df(sv + i));
            pi = df_norm(pi);
            si = df_norm(si);
            df_fma(xi, alpha, pi);
            df_fma(ri, nalpha, si);
            ri = df_norm(ri);
            const float di = dinv[i];
            const dfl un = df_norm(dfl{ri.hi * di, __fmaf_rn(ri.hi, di, -ri.hi * di) + ri.lo * di});
            st_df(p + i, pi);
            st_df(sv + i, si);
            st_df(xd + i, df_norm(xi));
            st_df(r + i, ri);
            st_df(u + i, un);
        }
        if (!grid_barrier(gb, bar)) return;
    }
    for (int64_t i = i0; i < N; i += stride) x[i] = df_to_double(ld_df(xd + i));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[0] = (double)it;
        out[1] = s_res;
        out[2] = s_r0;
    }
}

// ------------------------------------------------------------------------------------------------- GMRES
// GMRES(m) for A x = b with the right Jacobi preconditioner D^-1 (D = op.diag in FP32; A D^-1 y = b, x = D^-1 y),
// started from x, with classical Gram-Schmidt: the norm of the orthogonalized vector by the Pythagorean form |w|^2 -
// sum h_k^2 (its subtraction then shares the pass that normalizes it: two grid barriers per Arnoldi step), unless
// that cancels more than `reorth` of |w|^2, when the subtraction and its norm are explicit and a second pass follows
// (|w_after|^2 < reorth |w_before|^2).  The Hessenberg matrix, its Givens rotations and the least-squares solve are
// kept by thread 0 of every block (the same FP64 arithmetic on the same sums, so the same values everywhere).  It
// stops when the true residual |b - A x| (formed at the start of each cycle) is <= max(rtol |b|, atol), or once
// max_iter operator applications are spent; within a cycle the rotated residual estimate ends the cycle.
// Vectors of N entries as pairs: xd (the iterate, read across blocks by the residual's operator), z = D^-1 v_j (read
// across blocks by the Arnoldi operator), the basis V[(m + 1) N]; dinv the FP32 inverse diagonal.  part holds
// (GM_MAX + 2) gridDim.x pairs.  out[0] = applications, out[1] = the last true |r|, out[2] = |b| (block 0).
template <class Op>
__global__ void __launch_bounds__(FK_THREADS) k_gmres_fused(Op op, int64_t N, int m, const double* __restrict__ b,
                                                            double* x, float2* xd,
                                                            float* dinv, float2* z, float2* V, double rtol, double atol,
                                                            int max_iter, double reorth, float2* part, GridBarrier* gb,
                                                            double* out) {
    extern __shared__ float2 op_sm[];
    __shared__ float2 sh[(GM_MAX + 2) * FK_WARPS];
    __shared__ dfl s_h[GM_MAX + 2];
    __shared__ double H[(GM_MAX + 1) * GM_MAX], cs[GM_MAX], sn[GM_MAX], g[GM_MAX + 1];
    __shared__ dfl s_y[GM_MAX], s_scale;
    __shared__ double s_res, s_bn;
    __shared__ int s_go, s_more, s_norm, s_pass2, s_fast;
    unsigned long long bar = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t i0 = blockIdx.x * (int64_t)FK_THREADS + threadIdx.x, stride = (int64_t)gridDim.x * FK_THREADS;
    const dfl zero{0.f, 0.f};
    op.load(op_sm);
    __syncthreads();
    // per-warp sums of K values (sh[k FK_WARPS + warp]) written as block partials part[k G + b]: warp q reduces values
    // q, q + FK_WARPS, ... by a shuffle tree
    auto partials = [&](int K) {
        __syncthreads();
        for (int k = wid; k < K; k += FK_WARPS) {
            dfl t = lane < FK_WARPS ? ld_df(sh + k * FK_WARPS + lane) : zero;
            t = warp_sum_df(t);
            if (lane == 0) st_df(part + k * gridDim.x + blockIdx.x, t);
        }
    };
    // grid sums of K partial arrays into s_h (warp q sums arrays q, q + FK_WARPS, ...), fixed order
    auto grid_sums = [&](int K) {
        for (int k = wid; k < K; k += FK_WARPS) {
            dfl v = zero;
            for (int i = lane; i < (int)gridDim.x; i += 32) {
                const float2 t = __ldcg(part + k * gridDim.x + i);
                v = df_add(v, dfl{t.x, t.y});
            }
            v = warp_sum_df(v);
            if (lane == 0) s_h[k] = v;
        }
        __syncthreads();
    };
    // dot products of the vector W (own entries) with V_0..V_{K-1} (and with itself at index K when self): per-warp
    // sums to sh, then block partials
    auto dots = [&](const float2* W, int K, bool self) {
        for (int k = 0; k < K + (self ? 1 : 0); ++k) {
            const float2* Vk = k < K ? V + (int64_t)k * N : W;
            dfl acc = zero;
            for (int64_t i = i0; i < N; i += stride) df_fma(acc, ld_df(W + i), ld_df(Vk + i));
            acc = warp_sum_df(acc);
            if (lane == 0) st_df(sh + k * FK_WARPS + wid, acc);
        }
        partials(K + (self ? 1 : 0));
    };
    // init: dinv, xd = x, |b|^2
    {
        dfl bb = zero;
        for (int64_t i = i0; i < N; i += stride) {
            dinv[i] = 1.0f / op.diag(i, op_sm);
            st_df(xd + i, df_from_double(x[i]));
            const dfl bi = df_from_double(b[i]);
            df_fma(bb, bi, bi);
        }
        bb = warp_sum_df(bb);
        if (lane == 0) st_df(sh + wid, bb);
        partials(1);
    }
    if (!grid_barrier(gb, bar)) return;
    grid_sums(1);
    if (threadIdx.x == 0) s_bn = sqrt(fmax(df_to_double(s_h[0]), 0.0));
    __syncthreads();
    const double target = fmax(rtol * s_bn, atol);
    int used = 0;
    for (;;) {
        // true residual r = b - A x into V_0
        {
            dfl rr = zero;
            for (int64_t i = i0; i < N; i += stride) {
                const dfl ri = df_sub(df_from_double(b[i]), op.row(i, xd, op_sm));
                st_df(V + i, ri);
                df_fma(rr, ri, ri);
            }
            rr = warp_sum_df(rr);
            if (lane == 0) st_df(sh + wid, rr);
            partials(1);
        }
        ++used;
        if (!grid_barrier(gb, bar)) return;
        grid_sums(1);
        if (threadIdx.x == 0) {
            const double beta = sqrt(fmax(df_to_double(s_h[0]), 0.0));
            s_res = beta;
            s_go = beta > target && used < max_iter && beta > 0.0;
            if (s_go) {
                for (int k = 0; k <= m; ++k) g[k] = 0.0;
                g[0] = beta;
                s_scale = df_from_double(1.0 / beta);
            }
        }
        __syncthreads();
        if (!s_go) break;
        // v_0 = r / beta, z = D^-1 v_0
        for (int64_t i = i0; i < N; i += stride) {
            const dfl vi = df_mul(ld_df(V + i), s_scale);
            st_df(V + i, vi);
            const float di = dinv[i];
            st_df(z + i, df_norm(dfl{vi.hi * di, __fmaf_rn(vi.hi, di, -vi.hi * di) + vi.lo * di}));
        }
        if (!grid_barrier(gb, bar)) return;
        int j = 0;
        for (; j < m; ++j) {
            float2* W = V + (int64_t)(j + 1) * N;
            for (int64_t i = i0; i < N; i += stride) st_df(W + i, op.row(i, z, op_sm));
            ++used;
            dots(W, j + 1, true);  // h_k = (w, v_k), k <= j, and |w|^2 at index j + 1
            if (!grid_barrier(gb, bar)) return;
            grid_sums(j + 2);
            double hk[GM_MAX + 1];  // thread 0: the column before the rotations
            const double before = df_to_double(s_h[j + 1]);
            // |w - sum_k h_k v_k|^2 = |w|^2 - sum_k h_k^2 for orthonormal v_k (the Pythagorean form of classical
            // Gram-Schmidt): taken unless it cancels more than `reorth` of |w|^2, when the subtraction is done
            // explicitly, its norm summed, and a second pass follows as before
            if (threadIdx.x == 0) {
                dfl a = s_h[j + 1];
                for (int k = 0; k <= j; ++k) df_fma(a, df_neg(s_h[k]), s_h[k]);
                const double after = df_to_double(df_norm(a));
                s_fast = after > 0.0 && after >= reorth * before;
                if (s_fast) {
                    for (int k = 0; k <= j; ++k) hk[k] = df_to_double(s_h[k]);
                    hk[j + 1] = sqrt(after);
                }
            }
            __syncthreads();
            for (int pass = 0; pass < 2 && !s_fast; ++pass) {
                // w -= sum_k h_k v_k, |w|^2
                dfl aft = zero;
                for (int64_t i = i0; i < N; i += stride) {
                    dfl wi = ld_df(W + i);
                    for (int k = 0; k <= j; ++k) df_fma(wi, df_neg(s_h[k]), ld_df(V + (int64_t)k * N + i));
                    wi = df_norm(wi);
                    st_df(W + i, wi);
                    df_fma(aft, wi, wi);
                }
                if (threadIdx.x == 0)
                    for (int k = 0; k <= j; ++k) hk[k] = (pass == 0 ? 0.0 : hk[k]) + df_to_double(s_h[k]);
                aft = warp_sum_df(aft);
                if (lane == 0) st_df(sh + wid, aft);
                partials(1);
                if (!grid_barrier(gb, bar)) return;
                grid_sums(1);
                if (threadIdx.x == 0) {
                    const double after = df_to_double(s_h[0]);
                    s_pass2 = pass == 0 && after < reorth * before;
                    hk[j + 1] = sqrt(fmax(after, 0.0));
                }
                __syncthreads();
                if (!s_pass2) break;
                dots(W, j + 1, false);  // second pass: the projections left in w
                if (!grid_barrier(gb, bar)) return;
                grid_sums(j + 1);
            }
            if (threadIdx.x == 0) {
                double* col = H + j * (GM_MAX + 1);
                for (int k = 0; k <= j + 1; ++k) col[k] = hk[k];
                for (int k = 0; k < j; ++k) {
                    const double t0 = cs[k] * col[k] + sn[k] * col[k + 1];
                    col[k + 1] = -sn[k] * col[k] + cs[k] * col[k + 1];
                    col[k] = t0;
                }
                const double hn = hk[j + 1];
                const double rr = hypot(col[j], col[j + 1]);
                cs[j] = rr > 0.0 ? col[j] / rr : 1.0;
                sn[j] = rr > 0.0 ? col[j + 1] / rr : 0.0;
                col[j] = rr;
                col[j + 1] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                const double est = fabs(g[j + 1]);
                s_norm = hn > 0.0;
                s_more = !(est <= target || used >= max_iter || !(hn > 0.0)) && j + 1 < m;
                if (hn > 0.0) s_scale = df_from_double(1.0 / hn);
            }
            __syncthreads();
            if (s_norm && s_more) {  // v_{j+1} = w / |w|, z = D^-1 v_{j+1}: the next operator reads z
                for (int64_t i = i0; i < N; i += stride) {
                    dfl wi = ld_df(W + i);
                    if (s_fast) {  // the subtraction of the Pythagorean path, in the same pass
                        for (int k = 0; k <= j; ++k) df_fma(wi, df_neg(s_h[k]), ld_df(V + (int64_t)k * N + i));
                        wi = df_norm(wi);
                    }
                    const dfl vi = df_mul(wi, s_scale);
                    st_df(W + i, vi);
                    const float di = dinv[i];
                    st_df(z + i, df_norm(dfl{vi.hi * di, __fmaf_rn(vi.hi, di, -vi.hi * di) + vi.lo * di}));
                }
                if (!grid_barrier(gb, bar)) return;
            }
            if (!s_more) {
                ++j;
                break;
            }
        }
        // y = R^-1 g (thread 0), x += D^-1 sum_k y_k v_k; the next cycle's residual reads xd across blocks
        if (threadIdx.x == 0) {
            double y[GM_MAX];
            for (int i = j - 1; i >= 0; --i) {
                double t = g[i];
                for (int k = i + 1; k < j; ++k) t -= H[k * (GM_MAX + 1) + i] * y[k];
                const double d = H[i * (GM_MAX + 1) + i];
                y[i] = d != 0.0 ? t / d : 0.0;
            }
            for (int i = 0; i < j; ++i) s_y[i] = df_from_double(y[i]);
        }
        __syncthreads();
        for (int64_t i = i0; i < N; i += stride) {
            dfl acc = zero;
            for (int k = 0; k < j; ++k) df_fma(acc, s_y[k], ld_df(V + (int64_t)k * N + i));
            acc = df_norm(acc);
            const float di = dinv[i];
            dfl xi = ld_df(xd + i);
            xi = df_add(xi, df_norm(dfl{acc.hi * di, __fmaf_rn(acc.hi, di, -acc.hi * di) + acc.lo * di}));
            st_df(xd + i, xi);
        }
        if (!grid_barrier(gb, bar)) return;
    }
    for (int64_t i = i0; i < N; i += stride) x[i] = df_to_double(ld_df(xd + i));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[0] = (double)used;
        out[1] = s_res;
        out[2] = s_bn;
    }
}

// ------------------------------------------------------------------------------------- FP32 conjugate gradients
// The same Chronopoulos-Gear CG in FP32 for operators whose solve only has to be approximate (the Schur solve inside
// the velocity-pressure preconditioner): vectors and coefficients in FP32, the scalar products summed in FP32 in a
// fixed order (warp shuffle trees, then the blocks' partials), the scalars formed in FP64 by thread 0.  Op::row
// returns float.  b and x are FP64 (converted once in and out).  Same out[] convention as k_cg_fused.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;  // valid in lane 0
}

template <class Op>
__global__ void __launch_bounds__(FK_THREADS) k_cg_fused32(Op op, int64_t N, const double* __restrict__ b, double* x,
                                                           float* xs, float* dinv, float* r, float* u, float* p,
                                                           float* sv, float* w, double rtol, double atol, int max_iter,
                                                           float* part, GridBarrier* gb, double* out) {
    extern __shared__ float op_sm32[];
    __shared__ float sh[3 * FK_WARPS];
    __shared__ double s_res, s_r0;
    __shared__ float s_alpha, s_beta;
    __shared__ int s_go;
    unsigned long long bar = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t i0 = blockIdx.x * (int64_t)FK_THREADS + threadIdx.x, stride = (int64_t)gridDim.x * FK_THREADS;
    op.load(op_sm32);
    __syncthreads();
    for (int64_t i = i0; i < N; i += stride) {
        const float ri = (float)b[i], di = 1.0f / op.diag(i, op_sm32);
        xs[i] = 0.f;
        r[i] = ri;
        u[i] = ri * di;
        p[i] = 0.f;
        sv[i] = 0.f;
        dinv[i] = di;
    }
    if (!grid_barrier(gb, bar)) return;
    double gamma_old = 0.0, alpha_old = 1.0, target = 0.0;  // thread 0's copies (the same in every block)
    int it = 0;
    for (;;) {
        float acc[3] = {0.f, 0.f, 0.f};  // (r, u), (w, u), (r, r)
        for (int64_t i = i0; i < N; i += stride) {
            const float wi = op.row(i, u, op_sm32), ui = u[i], ri = r[i];
            w[i] = wi;
            acc[0] = fmaf(ri, ui, acc[0]);
            acc[1] = fmaf(wi, ui, acc[1]);
            acc[2] = fmaf(ri, ri, acc[2]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[k] = warp_sum_f(acc[k]);
        __syncthreads();
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 3; ++k) sh[k * FK_WARPS + wid] = acc[k];
        __syncthreads();
        if (wid < 3) {
            float t = lane < FK_WARPS ? sh[wid * FK_WARPS + lane] : 0.f;
            t = warp_sum_f(t);
            if (lane == 0) part[wid * gridDim.x + blockIdx.x] = t;
        }
        if (!grid_barrier(gb, bar)) return;
        if (wid < 3) {
            float t = 0.f;
            for (int q = lane; q < (int)gridDim.x; q += 32) t += __ldcg(part + wid * gridDim.x + q);
            t = warp_sum_f(t);
            if (lane == 0) sh[wid] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double gam = sh[0], del = sh[1], res = sqrt(fmax((double)sh[2], 0.0));
            if (it == 0) {
                s_r0 = res;
                target = fmax(rtol * res, atol);
            }
            s_res = res;
            s_go = res > target && it < max_iter;
            const double beta = it == 0 ? 0.0 : (gamma_old != 0.0 ? gam / gamma_old : 0.0);
            const double den = it == 0 ? del : del - beta * gam / alpha_old;
            const double alpha = den != 0.0 ? gam / den : 0.0;
            s_alpha = (float)alpha;
            s_beta = (float)beta;
            gamma_old = gam;
            alpha_old = alpha;
        }
        __syncthreads();
        if (!s_go) break;
        ++it;
        const float alpha = s_alpha, beta = s_beta;
        for (int64_t i = i0; i < N; i += stride) {
            const float pi = fmaf(beta, p[i], u[i]), si = fmaf(beta, sv[i], w[i]);
            const float ri = fmaf(-alpha, si, r[i]);
            p[i] = pi;
            sv[i] = si;
            xs[i] = fmaf(alpha, pi, xs[i]);
            r[i] = ri;
            u[i] = ri * dinv[i];
        }
        if (!grid_barrier(gb, bar)) return;
    }
    for (int64_t i = i0; i < N; i += stride) x[i] = (double)xs[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[0] = (double)it;
        out[1] = s_res;
        out[2] = s_r0;
    }
}

// ------------------------------------------------------------------------------------------ host-side workspace
// Workspace of the single-launch solvers, kept with the mesh (geometry.cu): nvec pair vectors of N_phi entries (or,
// read as floats, 2 nvec float vectors), an FP32 vector, (GM_MAX + 2) CG_BLOCKS partial pairs, the barrier, 4 result
// words and the Helmholtz coefficient table.
struct FusedSpace {
    float2* vec;  // vector k at vec + k N
    float* dinv;
    float2* part;
    GridBarrier* gb;
    double* out;
    float2* table;
};
int fused_space(evap_mesh* h, int nvec, FusedSpace& f);
// the launch's result words (iterations, |r|, |r0|) and its barrier's error word, after one synchronization
int fused_result(evap_mesh* h, const FusedSpace& f, cudaStream_t s, double res[3]);

// Grid of a single-launch solver: as many blocks as can be co-resident, at most 2 per SM and `cap` in all.
template <class K>
inline int fused_grid(K kernel, size_t smem, int cap, int& G) {
    int dev = 0, sms = 0, per_sm = 0;
    EVAP_CUDA(cudaGetDevice(&dev));
    EVAP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    EVAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, FK_THREADS, smem));
    G = per_sm < 2 ? per_sm * sms : 2 * sms;
    if (G > cap) G = cap;
    if (G < 1) {
        set_error("single-launch solver: no block of " + std::to_string(FK_THREADS) + " threads fits on an SM");
        return EVAP_ECUDA;
    }
    return EVAP_OK;
}

}  // namespace evap
