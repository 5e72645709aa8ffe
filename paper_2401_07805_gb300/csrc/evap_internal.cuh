// Internal declarations of the GB300 evaporation-operator library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/evap.h"
#include "basis_ct.cuh"

namespace evap {

constexpr int MAXQ = 4;  // up to degree 3 velocity: 4 Gauss points per direction

// 1D tables of the tensor-product bases (Sec. 2.5): Lagrange polynomials l_a on the Gauss-Lobatto support points of
// degree P evaluated at the Q = P + 1 Gauss-Legendre points t_q of [0, 1].
template <typename T>
struct Basis {
    int P, Q;
    T S[MAXQ][MAXQ];   // S[q][a]  = l_a(t_q)
    T D[MAXQ][MAXQ];   // D[q][a]  = l_a'(t_q)
    T Dc[MAXQ][MAXQ];  // Dc[q][r] = L_r'(t_q), L_r the Lagrange polynomials through the Gauss points (collocation)
    T w[MAXQ];         // Gauss weights on [0, 1]
    T t[MAXQ];         // Gauss points on [0, 1]
    T N1[MAXQ][2];     // Q1 shape values (1 - t_q, t_q) (pressure space)
    T g2t[2], g2w[2];  // 2-point Gauss rule of the Q1 operators
    // level-set space on one velocity cell (Q1 on the n_sub sub-intervals per direction, Sec. 2.5): the n_sub + 1
    // piecewise-linear hats at the Gauss points, NL[q][a], and their reference derivatives DL[q][a] (d/dt; divide by
    // h for physical units); a Gauss point on a sub-interval boundary takes the upper sub-interval's slopes
    T NL[MAXQ][3], DL[MAXQ][3];
};

// Scalars every kernel needs (passed by value).
template <typename T>
struct MeshArgs {
    int n, P, M;
    int64_t Nu, Nphi, ncell;
    int nsub, nl;  // level-set mesh: the velocity mesh subdivided nsub times per direction, nl = nsub n cells per axis
    int64_t Np;    // Q1 pressure nodes (n + 1)^3; Nphi = (nl + 1)^3 level-set nodes
    T h, inv_h, vol_w;  // cell size, 1/h, h^3
    T rho_l, rho_g, mu_l, mu_g, c_mass;
    T rho_H1, rho_H0, mu_H1, mu_H0;  // Eqs. (rhoEff), (muEff) evaluated at H = 1 and H = 0
    T eps, dt, theta, dtau;
    int newton, stress, corr_zone, variant;
    unsigned faces;
};

enum CellCode : int8_t { CELL_GAS = 0, CELL_LIQUID = 1, CELL_TABLE = 2 };
constexpr int TAB_K = 6;  // table entries per quadrature point: rho, mu, z n_x, z n_y, z n_z, v_dil
constexpr int QC_K = 19;  // cached momentum coefficients per quadrature point (see k_qp_coeffs)
constexpr int QC32_K = 12;  // of which the u0 terms, in FP32 for the FP32 apply (slots 1..12)

template <typename T>
struct Coeffs {            // quadrature-point coefficients of the momentum operator
    const int8_t* cell_code;
    const int32_t* table_index;
    const T* table;        // [ntable][TAB_K][nq]
    const T* u0;           // [3 N_u]
};

// Deterministic accumulation (evap_set_deterministic): the cells are taken in 8 passes, one per parity class
// colour = px + 2 py + 4 pz (cx = px, cy = py, cz = pz mod 2).  Two cells of one class differ by at least 2 in some
// coordinate, so they share no node of any of the meshes' spaces (velocity, pressure, level set): within a pass every
// entry is written by at most one cell, with a plain load and store, and every entry sums its cells in class order.
// colour < 0: all cells at once, accumulated by atomic adds (the default).
__host__ __device__ inline int64_t colour_cells(int n, int colour) {
    if (colour < 0) return (int64_t)n * n * n;
    const int64_t hx = (n - (colour & 1) + 1) / 2, hy = (n - ((colour >> 1) & 1) + 1) / 2, hz = (n - (colour >> 2) + 1) / 2;
    return hx * hy * hz;
}
// Cell (cx, cy, cz) of launch index idx in the pass `colour`, lexicographic within the class; false past its end.
__device__ __forceinline__ bool colour_cell(int64_t idx, int n, int colour, int& cx, int& cy, int& cz) {
    if (colour < 0) {
        if (idx >= (int64_t)n * n * n) return false;
        cx = (int)(idx % n);
        cy = (int)((idx / n) % n);
        cz = (int)(idx / ((int64_t)n * n));
        return true;
    }
    const int px = colour & 1, py = (colour >> 1) & 1, pz = colour >> 2;
    const int hx = (n - px + 1) >> 1, hy = (n - py + 1) >> 1, hz = (n - pz + 1) >> 1;
    if (idx >= (int64_t)hx * hy * hz) return false;
    cx = 2 * (int)(idx % hx) + px;
    cy = 2 * (int)((idx / hx) % hy) + py;
    cz = 2 * (int)(idx / ((int64_t)hx * hy)) + pz;
    return true;
}
// y += v: a plain read-modify-write inside a colour pass, else an atomic add
template <typename T>
__device__ __forceinline__ void acc_add(T* y, T v, bool plain) {
    if (plain)
        *y += v;
    else
        atomicAdd(y, v);
}

void host_basis(int P, Basis<double>& b, int nsub = 1);
template <typename T>
Basis<T> cast_basis(const Basis<double>& b);

}  // namespace evap

struct evap_mesh {
    evap::MeshArgs<double> m;
    evap::Basis<double> b;
    evap_params prm;
    int device = 0;
    bool has_fields = false;
    // fields (library-owned copies)
    double* phi = nullptr;
    double* u = nullptr;
    double* mdot = nullptr;
    float* u32 = nullptr;
    float* phi32 = nullptr;
    // quadrature-point coefficient table of the interface cells
    int8_t* cell_code = nullptr;
    int32_t* table_index = nullptr;
    int32_t* table_count = nullptr;  // device counter
    int64_t table_cap = 0;           // cells the table can hold
    double* table = nullptr;
    float* table32 = nullptr;
    float2* adj_table = nullptr;  // [table_cap][ADJ_K][nq] pairs for the adjoint
    // quadrature-point coefficients of the FP64 momentum operator, all cells [ncell][QC_K][nq]
    double* qc = nullptr;
    // the same coefficients as double-float pairs (hi, lo) [ncell][QC_K][nq] for the double-float FP64 apply
    float* qcdf = nullptr;
    int64_t qcdf_len = 0;  // floats
    // FP32 copy of the u0 coefficients (slots 1..12 of qc) in the 32-cell block layout of the FP32 apply
    float* qc32 = nullptr;
    int64_t qc32_len = 0;
    int64_t qc_len = 0;
    // transport velocity
    double* ugamma = nullptr;
    float* ugamma32 = nullptr;
    float* ugammadf = nullptr;  // double-float pairs (hi, lo) [3][N_phi] of u_Gamma for the double-float advection
    int32_t* cpp_flags = nullptr;
    unsigned long long* flag_count = nullptr;
    int32_t* band_list = nullptr;   // Q1 nodes that run the closest-point iteration
    int32_t* band_count = nullptr;  // [0] band nodes, [1] work counter of the closest-point pass
    double* band_y = nullptr;       // closest point (cell units) of band entry b at [3 b]
    unsigned long long* cpp_evals = nullptr;  // point evaluations of the last closest-point pass
    // frozen normal of the reinitialization operators: nodal Q1 field [3][N_phi] (FP64 and FP32) or none
    double* ls_normal = nullptr;
    float* ls_normal32 = nullptr;
    double* ls_normal_store = nullptr;  // owned storage behind ls_normal
    float* ls_normal32_store = nullptr;
    // geometry sub-solver workspace (first use) and its pinned scalars
    void* geo_ws = nullptr;
    double* geo_host = nullptr;
    double* geo_elem = nullptr;  // element matrices: reinitialization [36][ncell] or advection [64][ncell]
    int64_t geo_elem_len = 0;
    void* geo_kry = nullptr;     // single-launch Krylov solvers: pair vectors, inverse diagonal, partials, barrier
    size_t geo_kry_bytes = 0;
    // Jacobi diagonal and Krylov workspace (allocated by the first solve)
    double* diag = nullptr;
    float* diag32 = nullptr;
    bool diag_valid = false;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    double* red = nullptr;   // device reduction scratch
    double* red_host = nullptr;  // pinned host mirror
    size_t red_len = 0;
    // velocity-pressure system: continuity right-hand side of the current fields, the flexible GMRES workspace
    // (device) and its reduction scratch with a pinned host mirror
    double* cont_rhs = nullptr;
    bool cont_valid = false;
    void* sd_ws = nullptr;
    size_t sd_bytes = 0;
    double* sd_red = nullptr;
    double* sd_host = nullptr;
    size_t sd_red_len = 0;
    // input checks (evap_set_checks): device counter of non-finite entries
    bool checks = false;
    // deterministic accumulation (evap_set_deterministic): 8 colour passes instead of atomic adds
    bool deterministic = false;
    // assembled Schur approximation of the velocity-pressure preconditioner (schur.cu): [63][N_p] FP32, valid while
    // schur_stamp equals diag_stamp (incremented whenever the Jacobi diagonal of A is rebuilt)
    float* schur_S = nullptr;
    unsigned long long schur_stamp = 0, diag_stamp = 0;
    unsigned long long* nonfinite = nullptr;
    // time step workspace: inertia load [3 N_u], advected level set [N_phi], projected normal [3 N_phi]
    double* step_ws = nullptr;
    // tensor-product mass preconditioner of the momentum solves: banded LU factors of the three axes (FP64 [nf],
    // the 1D mass diagonal FP64 [M], FP32 copy of the factors [nf]), Sigma [3 N_u] in FP32 and FP64; valid with the
    // Jacobi diagonal it was built from
    void* tp_fac = nullptr;
    int64_t tp_nf = 0;
    float* tp_sigma = nullptr;
    double* tp_sigma64 = nullptr;
    int tp_lo[3] = {0, 0, 0}, tp_hi[3] = {0, 0, 0};
    int64_t tp_off[3] = {0, 0, 0};
    bool tp_valid = false;    // FP32 Sigma of the current diagonal
    bool tp64_valid = false;  // FP64 Sigma of the current diagonal
};

// Adjoint table, per quadrature point of a table cell (double-float pairs, the FP64 values of k_fill_table): the
// factors of the adjoint's chain rule that depend only on phi and mdot (Eqs. heaviside, rhoEff, muEff,
// normal_vector, delta, evaporDil): see adjoint.cu.
enum AdjSlot : int {
    ADJ_CRHO = 0,  // (drho/dH) H'(d) d'(phi) in the zone, else 0
    ADJ_CMU,       // (dmu/dH) H'(d) d'(phi) in the zone, else 0
    ADJ_N,         // 3 slots: the unit normal (0 where |grad phi| h <= GRAD_TINY)
    ADJ_ZG = ADJ_N + 3,  // correction gate z (1 or 0)
    ADJ_IGN,       // 1 / |grad phi| (0 where the normal is 0)
    ADJ_KD1,       // c_1 delta (the v_dil factor of mdot)
    ADJ_KD2,       // mdot c_1 (H''(d) d'(phi)^2 + H'(d) d''(phi)) |grad phi|
    ADJ_KD3,       // mdot c_1 H'(d) d'(phi)
    ADJ_IRHO,      // 1 / rho
    ADJ_RHO,       // rho
    ADJ_ZONE,      // 1 in the zone |phi| < tanh(3/2), else 0
    ADJ_K
};

#include <functional>  // host-side declarations below

namespace evap {

void set_error(const std::string& msg);
int cuda_fail(const char* what, cudaError_t e);
void count_launch();
#define EVAP_CHECK_LAUNCH(what)                                         \
    do {                                                                \
        ::evap::count_launch();                                         \
        cudaError_t _e = cudaGetLastError();                            \
        if (_e != cudaSuccess) return ::evap::cuda_fail(what, _e);      \
    } while (0)
#define EVAP_CUDA(call)                                                 \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::evap::cuda_fail(#call, _e);     \
    } while (0)

template <typename T>
MeshArgs<T> mesh_args(const evap_mesh* h);
// The same arguments for kernels that work on the level-set mesh alone (Q1 level-set operators, geometry): n, h, inv_h,
// vol_w and ncell of the subdivided mesh (identical to mesh_args for n_sub = 1).
template <typename T>
MeshArgs<T> ls_args(const evap_mesh* h);

// kernels launchers (each returns an evap_status)
int launch_setup_coefficients(evap_mesh* h, cudaStream_t s);
int launch_qp_coeffs(evap_mesh* h, cudaStream_t s);
int launch_momentum32(evap_mesh* h, const float* x, float* y, float* yp, cudaStream_t s);
// the FP64-accurate apply in double-float arithmetic (momentum_df.cu), after the init kernel; m carries the faces
int launch_momentum_df(evap_mesh* h, const MeshArgs<double>& m, const double* x, double* y, double* yp,
                       const double* p, cudaStream_t s);
// u_Gamma of the mesh's level set, or of `phi` (a clamped Q1 field) when given, into h->ugamma / h->ugamma32.
// The FP32 and double-float copies of h->ugamma (after every change of it).
int refresh_ugamma_copies(evap_mesh* h, cudaStream_t s);
int launch_transport_velocity(evap_mesh* h, cudaStream_t s, const double* phi = nullptr);
// the points of the last transport-velocity pass, y [3 N_phi] physical coordinates (evap_get_closest_points)
int launch_closest_points(evap_mesh* h, double* y, cudaStream_t s);
// y = A x (+ divergence row into yp if not null).  init = false: y already holds x on the Dirichlet DoFs and 0
// elsewhere (and yp is null), e.g. written by the solver's fused preconditioner kernel.
template <typename T>
// y = A x (+ the pressure term -B^T p when p is given, FP64 only), y_p = B x - g when yp is given.
// all_columns (FP64 only, with init): the Dirichlet entries of x are read as they are, so the free rows are those of
// the unconstrained operator (the lifting of Dirichlet data); the constrained rows are still y = x.
int launch_momentum(evap_mesh* h, const T* x, T* y, T* yp, cudaStream_t s, bool init = true, const T* p = nullptr,
                    bool all_columns = false);
// dst = src on the Dirichlet DoFs of the mesh's faces (other entries untouched); [3 N_u] vectors
int launch_constrained_copy(evap_mesh* h, const double* src, double* dst, cudaStream_t s);
// *any (host) = whether src has a nonzero entry on a Dirichlet DoF (synchronizes the stream)
int constrained_nonzero(evap_mesh* h, const double* src, bool* any, cudaStream_t s);
template <typename T>
int launch_levelset(evap_mesh* h, int mode, const T* x, T* y, cudaStream_t s);
int launch_adjoint(evap_mesh* h, const double* w, const double* wp, const double* x, double* gx, double* gu,
                   double* gphi, double* gm, cudaStream_t s);
int launch_diagonal(evap_mesh* h, cudaStream_t s);
int geo_helmholtz(evap_mesh* h, double c, int ncomp, const double* x, double* y, cudaStream_t s);
int geo_projected_normal(evap_mesh* h, double* n, int* iters, double* relres, cudaStream_t s);
int geo_curvature(evap_mesh* h, const double* nf, double* kappa, int* iters, double* relres, cudaStream_t s);
int geo_reinitialize(evap_mesh* h, double* psi, int steps, int* iters, double* last_change, cudaStream_t s);
int geo_advect_levelset(evap_mesh* h, double* phi, int max_iters, double tol, int* fp_iters, int* lin_iters,
                        double* last_change, cudaStream_t s);
// Jacobi diagonal (in the geometry workspace, valid until the next geometry call) for CG on the pressure Schur
// velocity-pressure coupling (saddle.cu)
template <typename T>
int launch_pressure_gradient(evap_mesh* h, const T* p, T scale, T* y, cudaStream_t s);
int continuity_rhs(evap_mesh* h, const double** g, cudaStream_t s);
// [y; y_p] = K [x; p]; lifted: the system K_D of non-homogeneous Dirichlet data, whose free rows keep the columns of
// the Dirichlet DoFs (y = A_full x - B^T p on free rows, x on constrained rows; y_p = B_full x)
int launch_saddle_apply(evap_mesh* h, const double* x, const double* p, double* y, double* yp, cudaStream_t s,
                        bool lifted = false);
// f = sum_q W rho N_i (c_m u + g) (FP64; Dirichlet rows 0)
int launch_mass_load(evap_mesh* h, const double* u, const double g[3], double* f, cudaStream_t s);
// copy the fields and compute the flow operators' coefficients (evap_set_fields without the transport velocity)
int set_fields_flow(evap_mesh* h, const double* phi, const double* u, const double* mdot, cudaStream_t s);
// one coupled time step (step.cu; see evap_time_step)
int time_step(evap_mesh* h, double* phi, double* u, double* p, const double* mdot, const double* u_prev,
              const double g[3], double alpha, int picard_iters, double picard_atol, int fp_iters, int reinit_steps,
              double ns_rtol, int* ns_iters, double* ns_relres, double* picard_res, cudaStream_t s);
// y_p += B D^(-1) x (the divergence row without its source; Dirichlet entries of x read as 0; D = diag, or the
// identity when diag is null)
template <typename T>
int launch_divergence(evap_mesh* h, const T* x, const T* diag, T* yp, cudaStream_t s);
// z = S~^(-1) r by at most cg_iters CG iterations on S~ = B diag(A)^(-1) B^T (applied in FP32) with the Jacobi
// The assembled Schur approximation S~ = B diag(A)^-1 B^T (schur.cu): assembly for the current diagonal of A, y = S~ x,
// and z ~ S~^-1 r by the FP32 single-launch CG (at most max_iter iterations or |r| <= rtol |r0|).
int schur_assemble(evap_mesh* h, cudaStream_t s);
int launch_schur_apply(evap_mesh* h, const double* x, double* y, cudaStream_t s);
int schur_solve(evap_mesh* h, const double* r, double* z, double rtol, int max_iter, int* iters, cudaStream_t s);
// z ~ S~^-1 r for the velocity-pressure preconditioner (saddle.cu): schur_solve with the preconditioner's tolerance
int schur_apply(evap_mesh* h, const double* r, double* z, int cg_iters, cudaStream_t st);
int launch_surface_tension(evap_mesh* h, const double* nf, const double* kappa, double alpha, double* out,
                           cudaStream_t s);
int launch_diagonal_into(evap_mesh* h, float* acc, double* out, cudaStream_t s);
// tensor-product mass preconditioner of the momentum solves (precond.cu): setup after the Jacobi diagonal, apply
// z = P (sc v) with scratch t (and w = Dirichlet ? z : 0 when w is given)
int tensor_prec_setup(evap_mesh* h, bool fp64, cudaStream_t s);
template <typename T>
int tensor_prec_apply(evap_mesh* h, const T* v, T sc, T* t, T* z, T* w, cudaStream_t s);
int solve_gmres(evap_mesh* h, const double* f, double* x, int mixed, int restart, double rtol, int max_iter,
                int* iters, double* relres, cudaStream_t s);
// Flexible GMRES on the velocity-pressure system K [x; p] = [f; g] (see evap_solve_saddle); g is the continuity
// right-hand side of the fields unless g_rhs is given.
int solve_saddle(evap_mesh* h, const double* f, double* x, double* p, int restart, double rtol, int max_iter,
                 int* iters, double* relres, cudaStream_t s, const double* g_rhs = nullptr);

// small vector kernels used by several files
template <typename T>
int launch_fill(T* p, int64_t n, T v, cudaStream_t s);
int launch_to_float(const double* a, float* b, int64_t n, cudaStream_t s);
int launch_to_double(const float* a, double* b, int64_t n, cudaStream_t s);

inline int blocks_for(int64_t n, int threads, int64_t cap = 152 * 64) {
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace evap
