// C ABI entry points: argument validation, library-owned state, dispatch to the kernel launchers.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <atomic>
#include <initializer_list>
#include <new>

#include "evap_internal.cuh"

namespace evap {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(const char* what, cudaError_t e) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? EVAP_ENOMEM : EVAP_ECUDA;
}

// 2-point Gauss-Legendre rule on [0, 1] (Q1 level-set operators).
static void gauss_rule2(double* t, double* w) {
    constexpr double r = 0.5773502691896257645091488;  // 1 / sqrt 3
    t[0] = 0.5 * (1.0 - r);
    t[1] = 0.5 * (1.0 + r);
    w[0] = w[1] = 0.5;
}

template <int P>
static void copy_ct_basis(Basis<double>& b) {
    constexpr CtBasis<P> c = make_ct_basis<P>();
    for (int q = 0; q <= P; ++q) {
        b.t[q] = c.t[q];
        b.w[q] = c.w[q];
        b.N1[q][0] = c.N1[q][0];
        b.N1[q][1] = c.N1[q][1];
        for (int k = 0; k <= P; ++k) {
            b.S[q][k] = c.S[q][k];
            b.D[q][k] = c.D[q][k];
            b.Dc[q][k] = c.Dc[q][k];
        }
    }
}

// The mesh's basis: the compile-time tables of basis_ct.cuh (also used as immediates by the FP32 apply).
void host_basis(int P, Basis<double>& b, int nsub) {
    std::memset(&b, 0, sizeof(b));
    b.P = P;
    b.Q = P + 1;
    if (P == 2)
        copy_ct_basis<2>(b);
    else
        copy_ct_basis<3>(b);
    gauss_rule2(b.g2t, b.g2w);
    for (int q = 0; q < b.Q; ++q) {  // level-set hats of the n_sub times subdivided interval
        const double s = nsub * b.t[q];
        const int k = std::min(std::max((int)std::floor(s), 0), nsub - 1);
        const double xi = s - k;
        b.NL[q][k] = 1.0 - xi;
        b.NL[q][k + 1] = xi;
        b.DL[q][k] = -(double)nsub;
        b.DL[q][k + 1] = (double)nsub;
    }
}

template <typename T>
Basis<T> cast_basis(const Basis<double>& b) {
    Basis<T> o;
    std::memset(&o, 0, sizeof(o));
    o.P = b.P;
    o.Q = b.Q;
    for (int i = 0; i < MAXQ; ++i) {
        for (int j = 0; j < MAXQ; ++j) {
            o.S[i][j] = (T)b.S[i][j];
            o.D[i][j] = (T)b.D[i][j];
            o.Dc[i][j] = (T)b.Dc[i][j];
        }
        o.w[i] = (T)b.w[i];
        o.t[i] = (T)b.t[i];
        o.N1[i][0] = (T)b.N1[i][0];
        o.N1[i][1] = (T)b.N1[i][1];
        for (int j = 0; j < 3; ++j) {
            o.NL[i][j] = (T)b.NL[i][j];
            o.DL[i][j] = (T)b.DL[i][j];
        }
    }
    for (int i = 0; i < 2; ++i) {
        o.g2t[i] = (T)b.g2t[i];
        o.g2w[i] = (T)b.g2w[i];
    }
    return o;
}
template Basis<double> cast_basis<double>(const Basis<double>&);
template Basis<float> cast_basis<float>(const Basis<double>&);

template <typename T>
MeshArgs<T> mesh_args(const evap_mesh* h) {
    const MeshArgs<double>& m = h->m;
    MeshArgs<T> o;
    o.n = m.n; o.P = m.P; o.M = m.M;
    o.Nu = m.Nu; o.Nphi = m.Nphi; o.ncell = m.ncell;
    o.h = (T)m.h; o.inv_h = (T)m.inv_h; o.vol_w = (T)m.vol_w;
    o.rho_l = (T)m.rho_l; o.rho_g = (T)m.rho_g; o.mu_l = (T)m.mu_l; o.mu_g = (T)m.mu_g; o.c_mass = (T)m.c_mass;
    o.rho_H1 = (T)m.rho_H1; o.rho_H0 = (T)m.rho_H0; o.mu_H1 = (T)m.mu_H1; o.mu_H0 = (T)m.mu_H0;
    o.eps = (T)m.eps; o.dt = (T)m.dt; o.theta = (T)m.theta; o.dtau = (T)m.dtau;
    o.newton = m.newton; o.stress = m.stress; o.corr_zone = m.corr_zone; o.variant = m.variant;
    o.faces = m.faces;
    o.nsub = m.nsub; o.nl = m.nl; o.Np = m.Np;
    return o;
}
template MeshArgs<double> mesh_args<double>(const evap_mesh*);
template MeshArgs<float> mesh_args<float>(const evap_mesh*);

template <typename T>
MeshArgs<T> ls_args(const evap_mesh* h) {
    MeshArgs<T> o = mesh_args<T>(h);
    const double hl = h->m.h / h->m.nsub;
    o.n = h->m.nl;
    o.ncell = (int64_t)o.n * o.n * o.n;
    o.h = (T)hl;
    o.inv_h = (T)(1.0 / hl);
    o.vol_w = (T)(hl * hl * hl);
    return o;
}
template MeshArgs<double> ls_args<double>(const evap_mesh*);
template MeshArgs<float> ls_args<float>(const evap_mesh*);

}  // namespace evap

using namespace evap;

static int fail(int code, const char* msg) {
    set_error(msg);
    return code;
}

// Input checks: the number of NaN / Inf entries of the listed arrays (one device counter, one synchronization).
template <typename T>
__global__ void k_count_nonfinite(const T* __restrict__ a, int64_t n, unsigned long long* cnt) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += isfinite(a[i]) ? 0ull : 1ull;
    if (c) atomicAdd(cnt, c);
}

struct InArr {
    const void* p;
    int64_t n;
    bool f32;
};

static int check_inputs(evap_mesh* h, const char* who, cudaStream_t s, std::initializer_list<InArr> arrs) {
    if (!h->checks) return EVAP_OK;
    if (!h->nonfinite) EVAP_CUDA(cudaMalloc(&h->nonfinite, sizeof(unsigned long long)));
    EVAP_CUDA(cudaMemsetAsync(h->nonfinite, 0, sizeof(unsigned long long), s));
    for (const InArr& a : arrs) {
        if (!a.p || a.n <= 0) continue;
        const int grid = blocks_for(a.n, 256, 152 * 8);
        if (a.f32)
            k_count_nonfinite<float><<<grid, 256, 0, s>>>((const float*)a.p, a.n, h->nonfinite);
        else
            k_count_nonfinite<double><<<grid, 256, 0, s>>>((const double*)a.p, a.n, h->nonfinite);
        EVAP_CHECK_LAUNCH("count_nonfinite");
    }
    unsigned long long c = 0;
    EVAP_CUDA(cudaMemcpyAsync(&c, h->nonfinite, sizeof(c), cudaMemcpyDeviceToHost, s));
    EVAP_CUDA(cudaStreamSynchronize(s));
    if (c) {
        set_error(std::string(who) + ": " + std::to_string(c) + " non-finite input entries");
        return EVAP_ENONFINITE;
    }
    return EVAP_OK;
}

static void free_all(evap_mesh* h) {
    void* ptrs[] = {h->phi, h->u, h->mdot, h->u32, h->phi32, h->cell_code, h->table_index, h->table_count,
                    h->table, h->table32, h->adj_table, h->qc, h->qcdf, h->qc32, h->ugamma, h->ugamma32, h->ugammadf, h->cpp_flags, h->flag_count, h->band_list,
                    h->band_count, h->band_y, h->cpp_evals, h->ls_normal_store, h->ls_normal32_store, h->geo_ws, h->geo_elem, h->geo_kry, h->schur_S, h->diag,
                    h->diag32, h->ws, h->red, h->cont_rhs, h->sd_ws, h->sd_red, h->nonfinite, h->step_ws,
                    h->tp_fac, h->tp_sigma, h->tp_sigma64};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->red_host) cudaFreeHost(h->red_host);
    if (h->geo_host) cudaFreeHost(h->geo_host);
    if (h->sd_host) cudaFreeHost(h->sd_host);
}

extern "C" {

const char* evap_status_string(int status) {
    switch (status) {
        case EVAP_OK: return "EVAP_OK";
        case EVAP_EINVAL: return "EVAP_EINVAL";
        case EVAP_ECUDA: return "EVAP_ECUDA";
        case EVAP_ENOTCONV: return "EVAP_ENOTCONV";
        case EVAP_ENOFIELDS: return "EVAP_ENOFIELDS";
        case EVAP_ENOMEM: return "EVAP_ENOMEM";
        case EVAP_ENONFINITE: return "EVAP_ENONFINITE";
        case EVAP_ETIMEOUT: return "EVAP_ETIMEOUT";
        default: return "EVAP_UNKNOWN";
    }
}

const char* evap_last_error(void) { return g_last_error.c_str(); }

int64_t evap_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

int evap_create_mesh(int n_cells, int degree_u, double L, const evap_params* prm, evap_handle* out) {
    if (!out || !prm) return fail(EVAP_EINVAL, "evap_create_mesh: null argument");
    if (n_cells < 1 || n_cells > 1024) return fail(EVAP_EINVAL, "evap_create_mesh: n_cells must be in [1, 1024]");
    if (degree_u != 2 && degree_u != 3) return fail(EVAP_EINVAL, "evap_create_mesh: degree_u must be 2 or 3");
    if (!(L > 0.0)) return fail(EVAP_EINVAL, "evap_create_mesh: L must be positive");
    if (!(prm->rho_l > 0.0) || !(prm->rho_g > 0.0) || !(prm->eps > 0.0) || !(prm->dtau > 0.0) ||
        !(prm->mu_l >= 0.0) || !(prm->mu_g >= 0.0))
        return fail(EVAP_EINVAL, "evap_create_mesh: rho_l, rho_g, eps, dtau must be > 0 and mu >= 0");
    if (prm->variant < 1 || prm->variant > 3) return fail(EVAP_EINVAL, "evap_create_mesh: variant must be 1, 2 or 3");
    if (prm->cpp_kmax < 0 || !(prm->cpp_tol > 0.0))
        return fail(EVAP_EINVAL, "evap_create_mesh: cpp_tol must be > 0 and cpp_kmax >= 0");
    if (!(prm->eta_n >= 0.0) || !(prm->eta_kappa >= 0.0))
        return fail(EVAP_EINVAL, "evap_create_mesh: eta_n and eta_kappa must be >= 0");
    const int nsub = prm->n_sub == 0 ? 1 : prm->n_sub;
    if (nsub != 1 && nsub != 2) return fail(EVAP_EINVAL, "evap_create_mesh: n_sub must be 1 or 2");
    evap_mesh* h = new (std::nothrow) evap_mesh();
    if (!h) return fail(EVAP_ENOMEM, "evap_create_mesh: host allocation failed");
    cudaGetDevice(&h->device);
    h->prm = *prm;
    MeshArgs<double>& m = h->m;
    m.n = n_cells;
    m.P = degree_u;
    m.M = degree_u * n_cells + 1;
    m.Nu = (int64_t)m.M * m.M * m.M;
    m.nsub = nsub;
    m.nl = nsub * n_cells;
    m.Nphi = (int64_t)(m.nl + 1) * (m.nl + 1) * (m.nl + 1);
    m.Np = (int64_t)(n_cells + 1) * (n_cells + 1) * (n_cells + 1);
    m.ncell = (int64_t)n_cells * n_cells * n_cells;
    m.h = L / n_cells;
    m.inv_h = 1.0 / m.h;
    m.vol_w = m.h * m.h * m.h;
    m.rho_l = prm->rho_l; m.rho_g = prm->rho_g; m.mu_l = prm->mu_l; m.mu_g = prm->mu_g;
    m.rho_H1 = 1.0 / (1.0 / prm->rho_l + (1.0 - 1.0) / prm->rho_g);
    m.rho_H0 = 1.0 / (0.0 / prm->rho_l + (1.0 - 0.0) / prm->rho_g);
    m.mu_H1 = 1.0 * prm->mu_l + (1.0 - 1.0) * prm->mu_g;
    m.mu_H0 = 0.0 * prm->mu_l + (1.0 - 0.0) * prm->mu_g;
    m.c_mass = prm->c_mass; m.eps = prm->eps; m.dt = prm->dt; m.theta = prm->theta; m.dtau = prm->dtau;
    m.newton = prm->newton ? 1 : 0;
    m.stress = prm->stress ? 1 : 0;
    m.corr_zone = prm->corr_zone ? 1 : 0;
    m.variant = prm->variant;
    m.faces = prm->dirichlet_faces & 0x3Fu;
    host_basis(degree_u, h->b, nsub);
    const int64_t Nu = m.Nu, Np = m.Nphi;
    cudaError_t e = cudaSuccess;
    auto al = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    al((void**)&h->phi, Np * sizeof(double));
    al((void**)&h->u, 3 * Nu * sizeof(double));
    al((void**)&h->mdot, Np * sizeof(double));
    al((void**)&h->u32, 3 * Nu * sizeof(float));
    al((void**)&h->phi32, Np * sizeof(float));
    al((void**)&h->cell_code, m.ncell * sizeof(int8_t));
    al((void**)&h->table_index, m.ncell * sizeof(int32_t));
    al((void**)&h->table_count, sizeof(int32_t));
    al((void**)&h->ugamma, 3 * Np * sizeof(double));
    al((void**)&h->ugamma32, 3 * Np * sizeof(float));
    al((void**)&h->ugammadf, 3 * Np * 2 * sizeof(float));
    al((void**)&h->cpp_flags, Np * sizeof(int32_t));
    al((void**)&h->flag_count, sizeof(unsigned long long));
    al((void**)&h->band_list, Np * sizeof(int32_t));
    al((void**)&h->band_count, 2 * sizeof(int32_t));
    al((void**)&h->band_y, 3 * Np * sizeof(double));
    al((void**)&h->cpp_evals, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        int rc = cuda_fail("evap_create_mesh: cudaMalloc", e);
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return EVAP_OK;
}

int evap_destroy(evap_handle h) {
    if (!h) return EVAP_OK;
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return EVAP_OK;
}

int evap_sizes(evap_handle h, int64_t* n_u, int64_t* n_phi) {
    if (!h) return fail(EVAP_EINVAL, "evap_sizes: null handle");
    if (n_u) *n_u = h->m.Nu;
    if (n_phi) *n_phi = h->m.Nphi;
    return EVAP_OK;
}

int evap_pressure_size(evap_handle h, int64_t* n_p) {
    if (!h) return fail(EVAP_EINVAL, "evap_pressure_size: null handle");
    if (n_p) *n_p = h->m.Np;
    return EVAP_OK;
}

int evap_set_checks(evap_handle h, int on) {
    if (!h) return fail(EVAP_EINVAL, "evap_set_checks: null handle");
    h->checks = on != 0;
    return EVAP_OK;
}

int evap_set_deterministic(evap_handle h, int on) {
    if (!h) return fail(EVAP_EINVAL, "evap_set_deterministic: null handle");
    h->deterministic = on != 0;
    h->diag_valid = false;  // the Jacobi diagonal is rebuilt the chosen way
    return EVAP_OK;
}

}  // extern "C"

namespace evap {
// The fields and every coefficient of the flow operators (no transport velocity).
int set_fields_flow(evap_mesh* h, const double* phi, const double* u, const double* mdot, cudaStream_t s) {
    const int64_t Nu = h->m.Nu, Np = h->m.Nphi;
    if (phi != h->phi) EVAP_CUDA(cudaMemcpyAsync(h->phi, phi, Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (u != h->u) EVAP_CUDA(cudaMemcpyAsync(h->u, u, 3 * Nu * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (mdot != h->mdot) EVAP_CUDA(cudaMemcpyAsync(h->mdot, mdot, Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    int rc = launch_setup_coefficients(h, s);  // clamps phi, FP32 copies, coefficient table
    if (rc) return rc;
    rc = launch_qp_coeffs(h, s);  // quadrature-point coefficients of the momentum operator
    if (rc) return rc;
    h->has_fields = true;
    h->diag_valid = false;
    h->tp_valid = false;
    h->cont_valid = false;
    return EVAP_OK;
}
}  // namespace evap

extern "C" {

int evap_set_fields(evap_handle h, const double* phi, const double* u, const double* mdot, void* stream) {
    if (!h || !phi || !u || !mdot) return fail(EVAP_EINVAL, "evap_set_fields: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t Nu = h->m.Nu, Np = h->m.Nphi;
    int rc0 = check_inputs(h, "evap_set_fields", s, {{phi, Np, false}, {u, 3 * Nu, false}, {mdot, Np, false}});
    if (rc0) return rc0;
    int rc = set_fields_flow(h, phi, u, mdot, s);
    if (rc) return rc;
    return launch_transport_velocity(h, s);
}

int evap_set_transport_velocity(evap_handle h, const double* u_gamma, void* stream) {
    if (!h || !u_gamma) return fail(EVAP_EINVAL, "evap_set_transport_velocity: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t Np = h->m.Nphi;
    int rc0 = check_inputs(h, "evap_set_transport_velocity", s, {{u_gamma, 3 * Np, false}});
    if (rc0) return rc0;
    EVAP_CUDA(cudaMemcpyAsync(h->ugamma, u_gamma, 3 * Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    int rc = refresh_ugamma_copies(h, s);
    if (rc) return rc;
    EVAP_CUDA(cudaMemsetAsync(h->cpp_flags, 0, Np * sizeof(int32_t), s));
    EVAP_CUDA(cudaMemsetAsync(h->flag_count, 0, sizeof(unsigned long long), s));
    return EVAP_OK;
}

int evap_get_transport_velocity(evap_handle h, double* u_gamma, int32_t* flags, int64_t* n_flagged, void* stream) {
    if (!h) return fail(EVAP_EINVAL, "evap_get_transport_velocity: null handle");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_get_transport_velocity: fields not set");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t Np = h->m.Nphi;
    if (u_gamma)
        EVAP_CUDA(cudaMemcpyAsync(u_gamma, h->ugamma, 3 * Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (flags) EVAP_CUDA(cudaMemcpyAsync(flags, h->cpp_flags, Np * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (n_flagged) {
        unsigned long long c = 0;
        EVAP_CUDA(cudaMemcpyAsync(&c, h->flag_count, sizeof(c), cudaMemcpyDeviceToHost, s));
        EVAP_CUDA(cudaStreamSynchronize(s));
        *n_flagged = (int64_t)c;
    }
    return EVAP_OK;
}

int evap_get_closest_points(evap_handle h, double* y, void* stream) {
    if (!h || !y) return fail(EVAP_EINVAL, "evap_get_closest_points: null argument");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_get_closest_points: fields not set");
    return launch_closest_points(h, y, (cudaStream_t)stream);
}

int evap_update_transport_velocity(evap_handle h, void* stream) {
    if (!h) return fail(EVAP_EINVAL, "evap_update_transport_velocity: null handle");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_update_transport_velocity: fields not set");
    return launch_transport_velocity(h, (cudaStream_t)stream);
}

int evap_transport_stats(evap_handle h, int64_t* band_nodes, int64_t* evaluations, int64_t* flagged, void* stream) {
    if (!h) return fail(EVAP_EINVAL, "evap_transport_stats: null handle");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_transport_stats: fields not set");
    cudaStream_t s = (cudaStream_t)stream;
    int32_t cnt[2] = {0, 0};
    unsigned long long ev = 0, fl = 0;
    EVAP_CUDA(cudaMemcpyAsync(cnt, h->band_count, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    EVAP_CUDA(cudaMemcpyAsync(&ev, h->cpp_evals, sizeof(ev), cudaMemcpyDeviceToHost, s));
    EVAP_CUDA(cudaMemcpyAsync(&fl, h->flag_count, sizeof(fl), cudaMemcpyDeviceToHost, s));
    EVAP_CUDA(cudaStreamSynchronize(s));
    const bool projected = h->m.variant != 1;
    if (band_nodes) *band_nodes = projected ? cnt[0] : 0;
    if (evaluations) *evaluations = projected ? (int64_t)ev : 0;
    if (flagged) *flagged = (int64_t)fl;
    return EVAP_OK;
}

int evap_projected_normal(evap_handle h, double* n, int* iters, double* relres, void* stream) {
    if (!h || !n) return fail(EVAP_EINVAL, "evap_projected_normal: null argument");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_projected_normal: fields not set");
    return geo_projected_normal(h, n, iters, relres, (cudaStream_t)stream);
}

int evap_curvature(evap_handle h, const double* n, double* kappa, int* iters, double* relres, void* stream) {
    if (!h || !n || !kappa) return fail(EVAP_EINVAL, "evap_curvature: null argument");
    if ((const void*)n == (const void*)kappa) return fail(EVAP_EINVAL, "evap_curvature: n and kappa must not alias");
    int rc0 = check_inputs(h, "evap_curvature", (cudaStream_t)stream, {{n, 3 * h->m.Nphi, false}});
    if (rc0) return rc0;
    return geo_curvature(h, n, kappa, iters, relres, (cudaStream_t)stream);
}

int evap_set_levelset_normal(evap_handle h, const double* n, void* stream) {
    if (!h) return fail(EVAP_EINVAL, "evap_set_levelset_normal: null handle");
    cudaStream_t s = (cudaStream_t)stream;
    if (!n) {
        h->ls_normal = nullptr;
        h->ls_normal32 = nullptr;
        return EVAP_OK;
    }
    const int64_t Np = h->m.Nphi;
    int rc0 = check_inputs(h, "evap_set_levelset_normal", s, {{n, 3 * Np, false}});
    if (rc0) return rc0;
    if (!h->ls_normal_store) EVAP_CUDA(cudaMalloc(&h->ls_normal_store, 3 * Np * sizeof(double)));
    if (!h->ls_normal32_store) EVAP_CUDA(cudaMalloc(&h->ls_normal32_store, 3 * Np * sizeof(float)));
    EVAP_CUDA(cudaMemcpyAsync(h->ls_normal_store, n, 3 * Np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    int rc = launch_to_float(h->ls_normal_store, h->ls_normal32_store, 3 * Np, s);
    if (rc) return rc;
    h->ls_normal = h->ls_normal_store;
    h->ls_normal32 = h->ls_normal32_store;
    return EVAP_OK;
}

int evap_reinitialize(evap_handle h, double* psi, int steps, int* iters, double* last_change, void* stream) {
    if (!h || !psi) return fail(EVAP_EINVAL, "evap_reinitialize: null argument");
    if (steps < 0) return fail(EVAP_EINVAL, "evap_reinitialize: steps must be >= 0");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_reinitialize: call evap_set_fields first");
    int rc0 = check_inputs(h, "evap_reinitialize", (cudaStream_t)stream, {{psi, h->m.Nphi, false}});
    if (rc0) return rc0;
    return geo_reinitialize(h, psi, steps, iters, last_change, (cudaStream_t)stream);
}

int evap_advect_levelset(evap_handle h, double* phi, int max_iters, double tol, int* fp_iters, int* lin_iters,
                         double* last_change, void* stream) {
    if (!h || !phi) return fail(EVAP_EINVAL, "evap_advect_levelset: null argument");
    if (max_iters < 0 || !(tol >= 0.0)) return fail(EVAP_EINVAL, "evap_advect_levelset: max_iters and tol must be >= 0");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_advect_levelset: call evap_set_fields first");
    return geo_advect_levelset(h, phi, max_iters, tol, fp_iters, lin_iters, last_change, (cudaStream_t)stream);
}

int evap_apply_saddle(evap_handle h, const double* x, const double* p, double* y, double* y_p, void* stream) {
    if (!h || !x || !p || !y || !y_p) return fail(EVAP_EINVAL, "evap_apply_saddle: null argument");
    if (x == y) return fail(EVAP_EINVAL, "evap_apply_saddle: x and y must not alias");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_apply_saddle: call evap_set_fields first");
    int rc0 = check_inputs(h, "evap_apply_saddle", (cudaStream_t)stream,
                           {{x, 3 * h->m.Nu, false}, {p, h->m.Np, false}});
    if (rc0) return rc0;
    return launch_saddle_apply(h, x, p, y, y_p, (cudaStream_t)stream);
}

int evap_solve_saddle(evap_handle h, const double* f, double* x, double* p, int restart, double rtol, int max_iter,
                      int* iters, double* relres, void* stream) {
    if (!h || !f || !x || !p) return fail(EVAP_EINVAL, "evap_solve_saddle: null argument");
    if (restart < 1 || restart > 255 || !(rtol > 0.0) || max_iter < 1)
        return fail(EVAP_EINVAL, "evap_solve_saddle: need 1 <= restart <= 255, rtol > 0, max_iter >= 1");
    if ((h->m.faces & 0x3Fu) == 0x3Fu)
        return fail(EVAP_EINVAL, "evap_solve_saddle: every face is Dirichlet (the pressure level is undetermined)");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_solve_saddle: call evap_set_fields first");
    int rc0 = check_inputs(h, "evap_solve_saddle", (cudaStream_t)stream,
                           {{f, 3 * h->m.Nu, false}, {x, 3 * h->m.Nu, false}, {p, h->m.Np, false}});
    if (rc0) return rc0;
    return solve_saddle(h, f, x, p, restart, rtol, max_iter, iters, relres, (cudaStream_t)stream);
}

int evap_time_step(evap_handle h, double* phi, double* u, double* p, const double* mdot, const double* u_prev,
                   const double* gravity, double alpha, int picard_iters, double picard_atol, int fp_iters,
                   int reinit_steps, double ns_rtol, int* ns_iters, double* ns_relres, double* picard_res,
                   void* stream) {
    if (!h || !phi || !u || !p || !mdot) return fail(EVAP_EINVAL, "evap_time_step: null argument");
    if (!(h->m.dt > 0.0)) return fail(EVAP_EINVAL, "evap_time_step: dt must be > 0");
    if ((h->m.faces & 0x3Fu) == 0x3Fu)
        return fail(EVAP_EINVAL, "evap_time_step: every face is Dirichlet (the pressure level is undetermined)");
    if (alpha != 0.0 && !(h->m.rho_l != h->m.rho_g))
        return fail(EVAP_EINVAL, "evap_time_step: surface tension needs rho_l != rho_g (c_rho)");
    if (picard_iters < 1 || !(picard_atol >= 0.0) || fp_iters < 1 || reinit_steps < 0 || !(ns_rtol > 0.0))
        return fail(EVAP_EINVAL, "evap_time_step: need picard_iters >= 1, picard_atol >= 0, fp_iters >= 1, "
                                 "reinit_steps >= 0, ns_rtol > 0");
    cudaStream_t s = (cudaStream_t)stream;
    int rc0 = check_inputs(h, "evap_time_step", s, {{p, h->m.Np, false}, {u_prev, 3 * h->m.Nu, false}});
    if (rc0) return rc0;
    double g[3] = {0.0, 0.0, 0.0};
    if (gravity) {
        g[0] = gravity[0];
        g[1] = gravity[1];
        g[2] = gravity[2];
    }
    return time_step(h, phi, u, p, mdot, u_prev, g, alpha, picard_iters, picard_atol, fp_iters, reinit_steps, ns_rtol,
                     ns_iters, ns_relres, picard_res, s);
}

int evap_surface_tension(evap_handle h, const double* n, const double* kappa, double alpha, double* f, void* stream) {
    if (!h || !n || !kappa || !f) return fail(EVAP_EINVAL, "evap_surface_tension: null argument");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_surface_tension: call evap_set_fields first");
    if (!(h->m.rho_l != h->m.rho_g)) return fail(EVAP_EINVAL, "evap_surface_tension: c_rho needs rho_l != rho_g");
    int rc0 = check_inputs(h, "evap_surface_tension", (cudaStream_t)stream,
                           {{n, 3 * h->m.Nphi, false}, {kappa, h->m.Nphi, false}});
    if (rc0) return rc0;
    return launch_surface_tension(h, n, kappa, alpha, f, (cudaStream_t)stream);
}

int evap_apply_momentum(evap_handle h, int prec, const void* x, void* y, void* y_p, void* stream) {
    if (!h || !x || !y) return fail(EVAP_EINVAL, "evap_apply_momentum: null argument");
    if (prec != 64 && prec != 32) return fail(EVAP_EINVAL, "evap_apply_momentum: prec must be 64 or 32");
    if (x == y) return fail(EVAP_EINVAL, "evap_apply_momentum: x and y must not alias");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_apply_momentum: call evap_set_fields first");
    cudaStream_t s = (cudaStream_t)stream;
    int rc0 = check_inputs(h, "evap_apply_momentum", s, {{x, 3 * h->m.Nu, prec == 32}});
    if (rc0) return rc0;
    if (prec == 64) return launch_momentum<double>(h, (const double*)x, (double*)y, (double*)y_p, s);
    return launch_momentum<float>(h, (const float*)x, (float*)y, (float*)y_p, s);
}

int evap_apply_levelset(evap_handle h, int mode, int prec, const void* x, void* y, void* stream) {
    if (!h || !x || !y) return fail(EVAP_EINVAL, "evap_apply_levelset: null argument");
    if (mode < EVAP_ADVECT || mode > EVAP_REINIT_RHS) return fail(EVAP_EINVAL, "evap_apply_levelset: bad mode");
    if (prec != 64 && prec != 32) return fail(EVAP_EINVAL, "evap_apply_levelset: prec must be 64 or 32");
    if (x == y) return fail(EVAP_EINVAL, "evap_apply_levelset: x and y must not alias");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_apply_levelset: call evap_set_fields first");
    cudaStream_t s = (cudaStream_t)stream;
    int rc0 = check_inputs(h, "evap_apply_levelset", s, {{x, h->m.Nphi, prec == 32}});
    if (rc0) return rc0;
    if (prec == 64) return launch_levelset<double>(h, mode, (const double*)x, (double*)y, s);
    return launch_levelset<float>(h, mode, (const float*)x, (float*)y, s);
}

int evap_apply_adjoint(evap_handle h, const double* w, const double* w_p, const double* x, double* g_x,
                       double* g_u0, double* g_phi, double* g_mdot, void* stream) {
    if (!h || !w || !x) return fail(EVAP_EINVAL, "evap_apply_adjoint: null argument");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_apply_adjoint: call evap_set_fields first");
    int rc0 = check_inputs(h, "evap_apply_adjoint", (cudaStream_t)stream,
                           {{w, 3 * h->m.Nu, false}, {w_p, h->m.Np, false}, {x, 3 * h->m.Nu, false}});
    if (rc0) return rc0;
    return launch_adjoint(h, w, w_p, x, g_x, g_u0, g_phi, g_mdot, (cudaStream_t)stream);
}

int evap_jacobi_diagonal(evap_handle h, double* diag, void* stream) {
    if (!h || !diag) return fail(EVAP_EINVAL, "evap_jacobi_diagonal: null argument");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_jacobi_diagonal: call evap_set_fields first");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_diagonal(h, s);
    if (rc) return rc;
    EVAP_CUDA(cudaMemcpyAsync(diag, h->diag, 3 * h->m.Nu * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return EVAP_OK;
}

int evap_solve(evap_handle h, const double* f, double* x, int mixed, int restart, double rtol, int max_iter,
               int* iters_out, double* relres_out, void* stream) {
    if (!h || !f || !x) return fail(EVAP_EINVAL, "evap_solve: null argument");
    if (f == x) return fail(EVAP_EINVAL, "evap_solve: f and x must not alias");
    if (restart < 1 || restart > 200) return fail(EVAP_EINVAL, "evap_solve: restart must be in [1, 200]");
    if (!(rtol > 0.0) || max_iter < 1) return fail(EVAP_EINVAL, "evap_solve: rtol > 0 and max_iter >= 1 required");
    if (!h->has_fields) return fail(EVAP_ENOFIELDS, "evap_solve: call evap_set_fields first");
    int rc0 = check_inputs(h, "evap_solve", (cudaStream_t)stream, {{f, 3 * h->m.Nu, false}, {x, 3 * h->m.Nu, false}});
    if (rc0) return rc0;
    return solve_gmres(h, f, x, mixed ? 1 : 0, restart, rtol, max_iter, iters_out, relres_out, (cudaStream_t)stream);
}

}  // extern "C"
