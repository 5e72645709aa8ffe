// Tensor-product mass preconditioner of the FP32 inner solve of the momentum system.
//
// The velocity block is dominated by its inertia term rho c_m M (at dt = 1e-4 the viscous and convective parts are
// below 1 % of it), and on the uniform mesh the Q_p mass matrix is a Kronecker product M = Mx (x) My (x) Mz of the 1D
// Q_p mass matrices.  The preconditioner is
//     P = Sigma (Mx (x) My (x) Mz)^(-1) Sigma,   Sigma = diag( sqrt( diag(M) / diag(A) ) )
// on the free (unconstrained) velocity DoFs and the identity on the Dirichlet ones: the Jacobi diagonal of A sets
// the local density and viscous scale, the Kronecker inverse removes the mass matrix's own conditioning.  Within a
// phase P A ~ I; the density jump across the interface leaves a bounded cluster of outliers.  (Measured with the
// assembled operator of the four-sphere workload: GMRES(16) to 1e-10 needed 47 / 63 / 71 iterations with Jacobi
// and 9 / 18 / 19 with P on 12^3 / 20^3 / 28^3 cells.)
//
// The free DoFs of a face-constrained box form a tensor product of per-axis ranges, so M^(-1) on them is three
// sweeps of banded 1D solves (bandwidth p): one block per tile of 32 lines, staged through shared memory so that
// global loads and stores stay coalesced for every axis (eight warps keep the loads in flight); each lane of the
// first warp solves one line with the LU factors of its axis (factorized once on the host in FP64, no pivoting: the
// 1D mass matrix is symmetric positive definite).
#include <cmath>
#include <vector>

#include "physics.cuh"

namespace evap {

constexpr int TP_LANES = 32;     // lines per tile (one solving warp)
constexpr int TP_THREADS = 256;  // threads of a block: all load and store the tile, the first warp solves

// Factor layout per axis (floats, Mf = hi - lo + 1 free nodes): rows k = 0..P-1 hold L[i][i-1-k], rows P..2P-1 hold
// U[i][i+1+(k-P)], row 2P holds 1 / U[i][i].
template <typename T, int P>
__device__ __forceinline__ void tp_solve_line(const T* __restrict__ fac, int Mf, T* __restrict__ col, int stride) {
    // The last P values of each recurrence stay in registers (win[0] the nearest), so a step waits on FMAs only; the
    // factor rows are zero where a neighbour falls outside the line, so no step needs a branch.
    T win[P];
#pragma unroll
    for (int k = 0; k < P; ++k) win[k] = T(0);
    // forward: L y = d (unit lower)
#pragma unroll 4
    for (int i = 0; i < Mf; ++i) {
        T v = col[i * stride];
#pragma unroll
        for (int k = 0; k < P; ++k) v -= fac[k * Mf + i] * win[k];
        col[i * stride] = v;
#pragma unroll
        for (int k = P - 1; k > 0; --k) win[k] = win[k - 1];
        win[0] = v;
    }
    // backward: U x = y
#pragma unroll
    for (int k = 0; k < P; ++k) win[k] = T(0);
#pragma unroll 4
    for (int i = Mf - 1; i >= 0; --i) {
        T v = col[i * stride];
#pragma unroll
        for (int k = 0; k < P; ++k) v -= fac[(P + k) * Mf + i] * win[k];
        v *= fac[2 * P * Mf + i];
        col[i * stride] = v;
#pragma unroll
        for (int k = P - 1; k > 0; --k) win[k] = win[k - 1];
        win[0] = v;
    }
}

// One sweep along AXIS for all three components (v enters scaled by sc).  MODE 0: t = M_axis^(-1) (Sigma sc v);
// MODE 1: t = M_axis^(-1) t; MODE 2: z = Sigma M_axis^(-1) t on the free DoFs, z = sc v on the Dirichlet ones, and
// w = (Dirichlet ? z : 0) (the initialization of the operator apply that follows).  One block per tile of TP_LANES
// lines; lines whose transverse position is constrained are all-Dirichlet and are solved only as a copy in MODE 2.
template <typename T, int P, int AXIS, int MODE>
__global__ void __launch_bounds__(TP_THREADS) k_tp_sweep(int M, int64_t Nu, unsigned faces, const T* __restrict__ fac_all,
                                                     int lo, int hi, const T* __restrict__ sigma,
                                                     const T* __restrict__ v, T sc, T* __restrict__ t,
                                                     T* __restrict__ z, T* __restrict__ w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* smem = reinterpret_cast<T*>(smem_raw);
    const int Mf = hi - lo + 1;
    T* fac = smem;                     // (2P + 1) Mf
    T* tile = smem + (2 * P + 1) * Mf;  // [M][TP_LANES + 1]
    const int tid = threadIdx.x;
    for (int i = tid; i < (2 * P + 1) * Mf; i += TP_THREADS) fac[i] = fac_all[i];
    // tile -> (component, first line); line l of the tile has transverse coordinates (ta, tb) and base address
    const int64_t M2 = (int64_t)M * M;
    int comp;
    int64_t first;  // first line index within the component
    int nlines;     // lines in this tile
    if (AXIS == 1) {  // y-lines: 32 consecutive x at fixed (z, component)
        const int tiles_x = (M + TP_LANES - 1) / TP_LANES;
        const int64_t b = blockIdx.x;
        comp = (int)(b / ((int64_t)tiles_x * M));
        const int64_t r = b - (int64_t)comp * tiles_x * M;
        const int zz = (int)(r / tiles_x), tx = (int)(r % tiles_x);
        first = (int64_t)zz * M + tx * TP_LANES;  // line id x + M z
        nlines = min(TP_LANES, M - tx * TP_LANES);
    } else {  // x-lines (id y + M z) or z-lines (id x + M y): 32 consecutive ids per component
        const int tiles = (int)((M2 + TP_LANES - 1) / TP_LANES);
        comp = blockIdx.x / tiles;
        first = (int64_t)(blockIdx.x % tiles) * TP_LANES;
        nlines = (int)min((int64_t)TP_LANES, M2 - first);
    }
    const int64_t cbase = (int64_t)comp * Nu;
    // per-lane line: base address, element stride, transverse constraint
    auto line_base = [&](int l, bool& cons) -> int64_t {
        const int64_t id = first + l;
        int ta, tb;  // transverse node coordinates
        int64_t base;
        if (AXIS == 0) {  // id = y + M z
            ta = (int)(id % M); tb = (int)(id / M);
            base = id * M;
            cons = constrained_node(1, ta, tb, M, faces & ~3u);
        } else if (AXIS == 1) {  // id = x + M z
            ta = (int)(id % M); tb = (int)(id / M);
            base = ta + M2 * tb;
            cons = constrained_node(ta, 1, tb, M, faces & ~12u);
        } else {  // id = x + M y
            ta = (int)(id % M); tb = (int)(id / M);
            base = id;
            cons = constrained_node(ta, tb, 1, M, faces & ~48u);
        }
        return cbase + base;
    };
    const int64_t es = AXIS == 0 ? 1 : (AXIS == 1 ? M : M2);  // element stride along the line
    // per-line base address and constraint flag, once per tile (the element loops below divide nothing)
    __shared__ int64_t s_base[TP_LANES];
    __shared__ int s_cons[TP_LANES];
    if (tid < nlines) {
        bool cons;
        s_base[tid] = line_base(tid, cons);
        s_cons[tid] = cons ? 1 : 0;
    }
    __syncthreads();
    // element loops: x-lines are contiguous, so each line is read by consecutive threads; for y- and z-lines a warp
    // reads one element of 32 neighbouring lines (contiguous in memory) and the eight warps take every eighth element
    constexpr int ROWS = TP_THREADS / TP_LANES;
    const int lane = tid % TP_LANES, row = tid / TP_LANES;
    auto load = [&](int64_t a) -> T { return MODE == 0 ? sc * v[a] * sigma[a] : t[a]; };
    if (AXIS == 0) {
        for (int l = 0; l < nlines; ++l) {
            if (s_cons[l]) continue;
            const int64_t b = s_base[l] + lo;
            for (int e = tid; e < Mf; e += TP_THREADS) tile[e * (TP_LANES + 1) + l] = load(b + e);
        }
    } else if (lane < nlines && !s_cons[lane]) {
        const int64_t b = s_base[lane] + (int64_t)lo * es;
        for (int e = row; e < Mf; e += ROWS) tile[e * (TP_LANES + 1) + lane] = load(b + (int64_t)e * es);
    }
    __syncthreads();
    if (tid < nlines && !s_cons[tid]) tp_solve_line<T, P>(fac, Mf, tile + tid, TP_LANES + 1);
    __syncthreads();
    if (MODE < 2) {
        if (AXIS == 0) {
            for (int l = 0; l < nlines; ++l) {
                if (s_cons[l]) continue;
                const int64_t b = s_base[l] + lo;
                for (int e = tid; e < Mf; e += TP_THREADS) t[b + e] = tile[e * (TP_LANES + 1) + l];
            }
        } else if (lane < nlines && !s_cons[lane]) {
            const int64_t b = s_base[lane] + (int64_t)lo * es;
            for (int e = row; e < Mf; e += ROWS) t[b + (int64_t)e * es] = tile[e * (TP_LANES + 1) + lane];
        }
    } else {  // every node of the tile's lines: free -> Sigma t, Dirichlet -> sc v; w = Dirichlet ? z : 0
        auto put = [&](int l, int e, int64_t a) {
            const bool dir = s_cons[l] || e < lo || e > hi;
            const T zz = dir ? sc * v[a] : sigma[a] * tile[(e - lo) * (TP_LANES + 1) + l];
            z[a] = zz;
            if (w) w[a] = dir ? zz : T(0);
        };
        if (AXIS == 0) {
            for (int l = 0; l < nlines; ++l) {
                const int64_t b = s_base[l];
                for (int e = tid; e < M; e += TP_THREADS) put(l, e, b + e);
            }
        } else if (lane < nlines) {
            const int64_t b = s_base[lane];
            for (int e = row; e < M; e += ROWS) put(lane, e, b + (int64_t)e * es);
        }
    }
}

// Sigma = sqrt(diag(M) / diag(A)) on the free DoFs (1 on the Dirichlet ones); md: the 1D mass diagonal [M].
template <typename T>
__global__ void k_tp_sigma(int M, int64_t Nu, unsigned faces, const double* __restrict__ md,
                           const T* __restrict__ diag, T* __restrict__ sigma) {
    const int64_t N = 3 * Nu;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = i % Nu;
        const int x = (int)(node % M), y = (int)((node / M) % M), zc = (int)(node / ((int64_t)M * M));
        sigma[i] = constrained_node(x, y, zc, M, faces) ? T(1) : (T)sqrt(md[x] * md[y] * md[zc] / (double)diag[i]);
    }
}

// Host: the 1D Q_p mass matrix (consistent, (p+1)-point Gauss) of n cells of width h, its diagonal, and the banded
// LU factors of its restriction to [lo, hi].
static void mass_1d(const Basis<double>& b, int n, double h, std::vector<double>& Mg) {
    const int P = b.P, M = P * n + 1;
    Mg.assign((size_t)M * M, 0.0);
    for (int c = 0; c < n; ++c)
        for (int a = 0; a <= P; ++a)
            for (int bb = 0; bb <= P; ++bb) {
                double s = 0.0;
                for (int q = 0; q <= P; ++q) s += b.w[q] * b.S[q][a] * b.S[q][bb];
                Mg[(size_t)(P * c + a) * M + (P * c + bb)] += h * s;
            }
}

static void factor_band(const std::vector<double>& Mg, int M, int P, int lo, int hi, std::vector<double>& out) {
    const int Mf = hi - lo + 1;
    std::vector<double> A((size_t)Mf * Mf);
    for (int i = 0; i < Mf; ++i)
        for (int j = 0; j < Mf; ++j) A[(size_t)i * Mf + j] = Mg[(size_t)(lo + i) * M + (lo + j)];
    for (int j = 0; j < Mf; ++j)
        for (int i = j + 1; i <= std::min(j + P, Mf - 1); ++i) {
            const double l = A[(size_t)i * Mf + j] / A[(size_t)j * Mf + j];
            A[(size_t)i * Mf + j] = l;
            for (int c = j + 1; c <= std::min(j + P, Mf - 1); ++c) A[(size_t)i * Mf + c] -= l * A[(size_t)j * Mf + c];
        }
    out.assign((size_t)(2 * P + 1) * Mf, 0.0);
    for (int i = 0; i < Mf; ++i) {
        for (int k = 0; k < P; ++k) {
            if (i - 1 - k >= 0) out[(size_t)k * Mf + i] = A[(size_t)i * Mf + (i - 1 - k)];
            if (i + 1 + k < Mf) out[(size_t)(P + k) * Mf + i] = A[(size_t)i * Mf + (i + 1 + k)];
        }
        out[(size_t)2 * P * Mf + i] = 1.0 / A[(size_t)i * Mf + i];
    }
}

// Factors of the three axes (FP64 and FP32 copies, then the 1D mass diagonal in FP64): they depend on the mesh
// and its Dirichlet faces only, so they are built and uploaded once per mesh (a synchronous copy).  Sigma follows
// the Jacobi diagonal: the FP32 scale after every new diagonal, the FP64 one only when an FP64 solve asks for it;
// both are enqueued on the stream without a host synchronization.
int tensor_prec_setup(evap_mesh* h, bool fp64, cudaStream_t s) {
    const MeshArgs<double>& m = h->m;
    const int P = m.P, M = m.M;
    const int64_t N = 3 * m.Nu;
    if (!h->tp_fac) {
        std::vector<double> Mg;
        mass_1d(h->b, m.n, m.h, Mg);
        std::vector<double> all;
        for (int a = 0; a < 3; ++a) {
            const int lo = (m.faces & (1u << (2 * a))) ? 1 : 0;
            const int hi = (m.faces & (1u << (2 * a + 1))) ? M - 2 : M - 1;
            h->tp_lo[a] = lo;
            h->tp_hi[a] = hi;
            h->tp_off[a] = (int64_t)all.size();
            std::vector<double> f;
            factor_band(Mg, M, P, lo, hi, f);
            all.insert(all.end(), f.begin(), f.end());
        }
        const size_t nf = all.size();
        for (int i = 0; i < M; ++i) all.push_back(Mg[(size_t)i * M + i]);
        // device layout (bytes): factors FP64 [nf], mass diagonal FP64 [M], factors FP32 [nf]
        const size_t bytes = (nf + M) * sizeof(double) + nf * sizeof(float);
        EVAP_CUDA(cudaMalloc(&h->tp_fac, bytes));
        std::vector<float> f32(all.begin(), all.begin() + nf);
        double* fac64 = (double*)h->tp_fac;
        EVAP_CUDA(cudaMemcpy(fac64, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice));
        EVAP_CUDA(cudaMemcpy(fac64 + nf + M, f32.data(), nf * sizeof(float), cudaMemcpyHostToDevice));
        h->tp_nf = (int64_t)nf;
    }
    const double* md = (const double*)h->tp_fac + h->tp_nf;
    if (!h->tp_valid) {
        if (!h->tp_sigma) EVAP_CUDA(cudaMalloc(&h->tp_sigma, N * sizeof(float)));
        k_tp_sigma<float><<<blocks_for(N, 256), 256, 0, s>>>(M, m.Nu, m.faces, md, h->diag32, h->tp_sigma);
        EVAP_CHECK_LAUNCH("tp_sigma");
        h->tp_valid = true;
        h->tp64_valid = false;
    }
    if (fp64 && !h->tp64_valid) {
        if (!h->tp_sigma64) EVAP_CUDA(cudaMalloc(&h->tp_sigma64, N * sizeof(double)));
        k_tp_sigma<double><<<blocks_for(N, 256), 256, 0, s>>>(M, m.Nu, m.faces, md, h->diag, h->tp_sigma64);
        EVAP_CHECK_LAUNCH("tp_sigma");
        h->tp64_valid = true;
    }
    return EVAP_OK;
}

template <typename T, int P, int AXIS, int MODE>
static int tp_launch(evap_mesh* h, const T* v, T sc, T* t, T* z, T* w, cudaStream_t s) {
    const MeshArgs<double>& m = h->m;
    const int M = m.M;
    const int lo = h->tp_lo[AXIS], hi = h->tp_hi[AXIS], Mf = hi - lo + 1;
    const size_t smem = ((size_t)(2 * P + 1) * Mf + (size_t)M * (TP_LANES + 1)) * sizeof(T);
    if (smem > 48 * 1024)
        EVAP_CUDA(cudaFuncSetAttribute(k_tp_sweep<T, P, AXIS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    const double* fac64 = (const double*)h->tp_fac;
    const T* fac = sizeof(T) == 8 ? (const T*)fac64 : (const T*)(const void*)((const float*)(fac64 + h->tp_nf + M));
    const T* sigma = sizeof(T) == 8 ? (const T*)h->tp_sigma64 : (const T*)h->tp_sigma;
    const int64_t M2 = (int64_t)M * M;
    const int64_t blocks = AXIS == 1 ? 3 * (int64_t)((M + TP_LANES - 1) / TP_LANES) * M
                                     : 3 * ((M2 + TP_LANES - 1) / TP_LANES);
    k_tp_sweep<T, P, AXIS, MODE><<<(unsigned)blocks, TP_THREADS, smem, s>>>(M, m.Nu, m.faces, fac + h->tp_off[AXIS],
                                                                         lo, hi, sigma, v, sc, t, z, w);
    EVAP_CHECK_LAUNCH("tp_sweep");
    return EVAP_OK;
}

// z = P (sc v) (and w = Dirichlet ? z : 0 when w is given); t: scratch [3 N_u]; z must not alias v or t.
template <typename T>
int tensor_prec_apply(evap_mesh* h, const T* v, T sc, T* t, T* z, T* w, cudaStream_t s) {
    int rc;
    if (h->m.P == 2) {
        if ((rc = tp_launch<T, 2, 0, 0>(h, v, sc, t, z, w, s))) return rc;
        if ((rc = tp_launch<T, 2, 1, 1>(h, v, sc, t, z, w, s))) return rc;
        return tp_launch<T, 2, 2, 2>(h, v, sc, t, z, w, s);
    }
    if ((rc = tp_launch<T, 3, 0, 0>(h, v, sc, t, z, w, s))) return rc;
    if ((rc = tp_launch<T, 3, 1, 1>(h, v, sc, t, z, w, s))) return rc;
    return tp_launch<T, 3, 2, 2>(h, v, sc, t, z, w, s);
}
template int tensor_prec_apply<float>(evap_mesh*, const float*, float, float*, float*, float*, cudaStream_t);
template int tensor_prec_apply<double>(evap_mesh*, const double*, double, double*, double*, double*, cudaStream_t);

}  // namespace evap
