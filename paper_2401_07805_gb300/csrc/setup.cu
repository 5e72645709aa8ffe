// evap_set_fields work: field preparation, FP64 quadrature-point coefficient table of the interface cells, and
// the level-set transport velocity with closest-point projection (App. C).
#include <cmath>

#include "dfloat.cuh"
#include "physics.cuh"

namespace evap {

template <typename T>
__global__ void k_fill(T* p, int64_t n, T v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

template <typename T>
int launch_fill(T* p, int64_t n, T v, cudaStream_t s) {
    k_fill<T><<<blocks_for(n, 256), 256, 0, s>>>(p, n, v);
    EVAP_CHECK_LAUNCH("fill");
    return EVAP_OK;
}
template int launch_fill<double>(double*, int64_t, double, cudaStream_t);
template int launch_fill<float>(float*, int64_t, float, cudaStream_t);

int launch_to_float(const double* a, float* b, int64_t n, cudaStream_t s) {
    k_to_float<<<blocks_for(n, 256), 256, 0, s>>>(a, b, n);
    EVAP_CHECK_LAUNCH("to_float");
    return EVAP_OK;
}

__global__ void k_to_double(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

// b = (float)a and c = (hi, lo) of a
__global__ void k_to_float_df(const double* __restrict__ a, float* __restrict__ b, float2* __restrict__ c, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = a[i];
        const float hi = (float)v;
        b[i] = hi;
        c[i] = make_float2(hi, (float)(v - (double)hi));
    }
}

int refresh_ugamma_copies(evap_mesh* h, cudaStream_t s) {
    const int64_t n = 3 * h->m.Nphi;
    k_to_float_df<<<blocks_for(n, 256), 256, 0, s>>>(h->ugamma, h->ugamma32, (float2*)h->ugammadf, n);
    EVAP_CHECK_LAUNCH("ugamma_copies");
    return EVAP_OK;
}

int launch_to_double(const float* a, double* b, int64_t n, cudaStream_t s) {
    k_to_double<<<blocks_for(n, 256), 256, 0, s>>>(a, b, n);
    EVAP_CHECK_LAUNCH("to_double");
    return EVAP_OK;
}

// phi clamped to [-1, 1]; FP32 copies of phi and u.
__global__ void k_prepare(double* phi, float* phi32, const double* __restrict__ u, float* __restrict__ u32,
                          int64_t Np, int64_t Nu3) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Np; i += stride) {
        double v = phi[i];
        v = v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v);
        phi[i] = v;
        phi32[i] = (float)v;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nu3; i += stride) u32[i] = (float)u[i];
}

// Cell classification: all quadrature points liquid (H = 1), all gas (H = 0), or a table cell (interface zone,
// mixed phases, or correction applied everywhere).  Table cells get a slot by an atomic counter.
__global__ void k_classify(MeshArgs<double> m, Basis<double> b, const double* __restrict__ phi, int8_t* code,
                           int32_t* tindex, int32_t* counter) {
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= m.ncell) return;
    const int n = m.n;
    const int cx = (int)(cell % n), cy = (int)((cell / n) % n), cz = (int)(cell / ((int64_t)n * n));
    bool all_liq = true, all_gas = true;
    for (int qz = 0; qz < b.Q; ++qz)
        for (int qy = 0; qy < b.Q; ++qy)
            for (int qx = 0; qx < b.Q; ++qx) {
                double v, g[3];
                ls_at(phi, m, cx, cy, cz, b.t[qx], b.t[qy], b.t[qz], v, g);
                all_liq = all_liq && (v >= PHI_BAND);
                all_gas = all_gas && (v <= -PHI_BAND);
            }
    const bool everywhere = m.stress != 0 && m.corr_zone != 0;
    int8_t c = (!everywhere && all_liq) ? CELL_LIQUID : ((!everywhere && all_gas) ? CELL_GAS : CELL_TABLE);
    code[cell] = c;
    tindex[cell] = c == CELL_TABLE ? atomicAdd(counter, 1) : -1;
}

// Table entries at one quadrature point of a table cell: rho, mu, z n (z = correction gate), v_dil (Eq. evaporDil
// with the sign of App. A, dilation_coefficient).
__global__ void k_fill_table(MeshArgs<double> m, Basis<double> b, const double* __restrict__ phi,
                             const double* __restrict__ mdot, const int8_t* __restrict__ code,
                             const int32_t* __restrict__ tindex, double* table, float* table32, float2* adj) {
    const int nq = b.Q * b.Q * b.Q;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t cell = gid / nq;
    if (cell >= m.ncell || code[cell] != CELL_TABLE) return;
    const int q = (int)(gid % nq);
    const int qx = q % b.Q, qy = (q / b.Q) % b.Q, qz = q / (b.Q * b.Q);
    const int n = m.n;
    const int cx = (int)(cell % n), cy = (int)((cell / n) % n), cz = (int)(cell / ((int64_t)n * n));
    double ph, g[3], md, gm[3];
    ls_at(phi, m, cx, cy, cz, b.t[qx], b.t[qy], b.t[qz], ph, g);
    ls_at(mdot, m, cx, cy, cz, b.t[qx], b.t[qy], b.t[qz], md, gm);
    const Material mat = material(ph, g[0], g[1], g[2], m);
    const double z = correction_on(m, mat.zone) ? 1.0 : 0.0;
    const double vals[TAB_K] = {mat.rho, mat.mu, z * mat.n[0], z * mat.n[1], z * mat.n[2],
                                md * dilation_coefficient(m) * mat.delta};
    const int64_t base = (int64_t)tindex[cell] * TAB_K * nq + q;
#pragma unroll
    for (int k = 0; k < TAB_K; ++k) {
        table[base + (int64_t)k * nq] = vals[k];
        table32[base + (int64_t)k * nq] = (float)vals[k];
    }
    // adjoint factors: H'(d) d'(phi) and its phi-derivative (H''(d) d'(phi)^2 + H'(d) d''(phi)) in the zone
    double dHdd = 0.0, d2 = 0.0;
    if (mat.zone) {
        const double d = m.eps * log((1.0 + ph) / (1.0 - ph));
        double sn, cs;
        sincos(PI * d / (3.0 * m.eps), &sn, &cs);
        const double dH = (1.0 + cs) / (6.0 * m.eps), d2H = -PI * sn / (18.0 * m.eps * m.eps);
        const double om = 1.0 - ph * ph;
        const double dd = 2.0 * m.eps / om, d2d = 4.0 * m.eps * ph / (om * om);
        dHdd = dH * dd;
        d2 = d2H * dd * dd + dH * d2d;
    }
    const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const double kdil = dilation_coefficient(m);
    double av[ADJ_K];
    av[ADJ_CRHO] = -mat.rho * mat.rho * (1.0 / m.rho_l - 1.0 / m.rho_g) * dHdd;
    av[ADJ_CMU] = (m.mu_l - m.mu_g) * dHdd;
    av[ADJ_N + 0] = mat.n[0];
    av[ADJ_N + 1] = mat.n[1];
    av[ADJ_N + 2] = mat.n[2];
    av[ADJ_ZG] = z;
    av[ADJ_IGN] = gn * m.h > GRAD_TINY ? 1.0 / gn : 0.0;
    av[ADJ_KD1] = kdil * mat.delta;
    av[ADJ_KD2] = md * kdil * d2 * gn;
    av[ADJ_KD3] = md * kdil * dHdd;
    av[ADJ_IRHO] = 1.0 / mat.rho;
    av[ADJ_RHO] = mat.rho;
    av[ADJ_ZONE] = mat.zone ? 1.0 : 0.0;
    const int64_t abase = (int64_t)tindex[cell] * ADJ_K * nq + q;
#pragma unroll
    for (int k = 0; k < ADJ_K; ++k) {
        const dfl v = df_from_double(av[k]);
        adj[abase + (int64_t)k * nq] = make_float2(v.hi, v.lo);
    }
}

int launch_setup_coefficients(evap_mesh* h, cudaStream_t s) {
    const MeshArgs<double>& m = h->m;
    k_prepare<<<blocks_for(3 * m.Nu, 256), 256, 0, s>>>(h->phi, h->phi32, h->u, h->u32, m.Nphi, 3 * m.Nu);
    EVAP_CHECK_LAUNCH("prepare");
    EVAP_CUDA(cudaMemsetAsync(h->table_count, 0, sizeof(int32_t), s));
    k_classify<<<blocks_for(m.ncell, 128, 1LL << 40), 128, 0, s>>>(m, h->b, h->phi, h->cell_code, h->table_index,
                                                                   h->table_count);
    EVAP_CHECK_LAUNCH("classify");
    int32_t count = 0;
    EVAP_CUDA(cudaMemcpyAsync(&count, h->table_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    EVAP_CUDA(cudaStreamSynchronize(s));
    const int nq = h->b.Q * h->b.Q * h->b.Q;
    if (count > h->table_cap) {
        if (h->table) cudaFree(h->table);
        if (h->table32) cudaFree(h->table32);
        if (h->adj_table) cudaFree(h->adj_table);
        h->table = nullptr;
        h->table32 = nullptr;
        h->adj_table = nullptr;
        h->table_cap = 0;
        const int64_t cap = count + count / 8 + 16;
        EVAP_CUDA(cudaMalloc(&h->table, cap * TAB_K * nq * sizeof(double)));
        EVAP_CUDA(cudaMalloc(&h->table32, cap * TAB_K * nq * sizeof(float)));
        EVAP_CUDA(cudaMalloc(&h->adj_table, cap * ADJ_K * nq * sizeof(float2)));
        h->table_cap = cap;
    }
    if (count > 0) {
        const int64_t total = m.ncell * nq;
        k_fill_table<<<blocks_for(total, 256, 1LL << 40), 256, 0, s>>>(m, h->b, h->phi, h->mdot, h->cell_code,
                                                                       h->table_index, h->table, h->table32,
                                                                       h->adj_table);
        EVAP_CHECK_LAUNCH("fill_table");
    }
    return EVAP_OK;
}

// ------------------------------------------------------------------------------------------ transport velocity
// Point evaluation in cell units s = y / h of the level-set mesh (m: the level-set view of the mesh, ls_args):
// cell = clamp(floor(s), 0, n - 1), trilinear phi; the Q_p velocity from the velocity cell located the same way at
// s / n_sub (nu cells per axis).
struct PointEval {
    const double* phi;
    const double* u;
    MeshArgs<double> m;
    int nu;           // velocity cells per axis
    double inv_sub;   // 1 / n_sub
    double gl[MAXQ];  // Gauss-Lobatto support points of the velocity element

    __device__ void locate(const double s[3], int k[3], double xi[3]) const {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int c = (int)floor(s[a]);
            c = c < 0 ? 0 : (c > m.n - 1 ? m.n - 1 : c);
            k[a] = c;
            xi[a] = s[a] - c;
        }
    }
    __device__ void phi_grad(const double s[3], double& val, double g[3]) const {
        int k[3];
        double xi[3];
        locate(s, k, xi);
        q1_at(phi, m.n, k[0], k[1], k[2], xi[0], xi[1], xi[2], m.inv_h, val, g);
    }
    __device__ void velocity(const double s_ls[3], double out[3]) const {
        int k[3];
        double xi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double s = s_ls[a] * inv_sub;
            int c = (int)floor(s);
            c = c < 0 ? 0 : (c > nu - 1 ? nu - 1 : c);
            k[a] = c;
            xi[a] = s - c;
        }
        const int P = m.P, Q = P + 1;
        double l[3][MAXQ];
        for (int d = 0; d < 3; ++d)
            for (int a = 0; a < Q; ++a) {
                double v = 1.0;
                for (int j = 0; j < Q; ++j)
                    if (j != a) v *= (xi[d] - gl[j]) / (gl[a] - gl[j]);
                l[d][a] = v;
            }
        out[0] = out[1] = out[2] = 0.0;
        for (int c = 0; c < Q; ++c)
            for (int b = 0; b < Q; ++b)
                for (int a = 0; a < Q; ++a) {
                    const int64_t node = (int64_t)(P * k[0] + a) +
                                         (int64_t)m.M * ((int64_t)(P * k[1] + b) + (int64_t)m.M * (P * k[2] + c));
                    const double wgt = l[0][a] * l[1][b] * l[2][c];
                    out[0] += wgt * u[node];
                    out[1] += wgt * u[m.Nu + node];
                    out[2] += wgt * u[2 * m.Nu + node];
                }
    }
};

constexpr double PHI_CLAMP = 1.0 - 0x1p-40;
constexpr int CPP_NORMAL_STEPS = 20;  // projection of the node
constexpr int CPP_TRIAL_STEPS = 6;    // projection of a trial point of the tangential step
constexpr int CPP_BACKTRACK = 6;
constexpr double CPP_STALL = 1e-12;   // an accepted step shortening |y - x| by less than this fraction ends it

__device__ __forceinline__ double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ double dist3(const double a[3], const double b[3]) {
    const double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
    return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

// Closest point of x on d(phi_h) = d_t with the backtracked tangential step (App. C), written as a state machine
// in which every trip of the loop makes exactly one point evaluation of phi_h and grad phi_h: the projection of the
// node (phase 0, at most CPP_NORMAL_STEPS normal steps), the tangential direction at y (phase 1), the projection of a
// trial point y - omega t (phase 2, at most CPP_TRIAL_STEPS normal steps, omega = 1, 1/2, ..., 1/2^(CPP_BACKTRACK-1)).
// Lanes of a warp run their own nodes but share the expensive part of every trip (the FP64 evaluation), and a lane
// whose node is done takes the next band entry, so warps stay full.  The sequence of evaluations and updates of a
// node is: project x (normal steps y <- y - (d(y) - d*) / |grad d(y)| n(y) until |d(y) - d*| <= tol h); then
// repeat up to kmax times: tangential part t of y - x at y; for omega = 1, 1/2, ...: project y - omega t; accept
// the first trial point that reached the isocontour and is strictly closer to x; stop when none is, when the accepted
// step is <= tol or shortens |y - x| by <= CPP_STALL of it.  Not converged: the first projection failed or kmax
// outer iterations ran without a stop.
struct CppLane {
    int b = -1;  // band entry, -1 none
    int phase = 0, steps = 0, k = 0, bt = 0, trips = 0;
    double x[3], y[3], yn[3], tp[3];
    double dist = 0.0, dist_prev = 0.0, omega = 1.0;
};

// phi_h and grad phi_h (physical units) at s (cell units) by successive linear interpolation along x, y, z
// (the trilinear Q1 interpolant of Sec. 2.5; fewer FP64 operations than the weighted sum over the 8 nodes).
__device__ __forceinline__ void q1_lerp(const PointEval& e, const double s[3], double& val, double g[3]) {
    int k[3];
    double t[3];
    e.locate(s, k, t);
    const int64_t m1 = e.m.n + 1;
    const double* f = e.phi + k[0] + m1 * (k[1] + m1 * k[2]);
    double ex[2][2], dx[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const double v0 = f[m1 * (b + m1 * c)], v1 = f[1 + m1 * (b + m1 * c)];
            dx[c][b] = v1 - v0;
            ex[c][b] = fma(t[0], dx[c][b], v0);
        }
    double exy[2], dxy[2], dyx[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        dyx[c] = ex[c][1] - ex[c][0];
        exy[c] = fma(t[1], dyx[c], ex[c][0]);
        dxy[c] = fma(t[1], dx[c][1] - dx[c][0], dx[c][0]);
    }
    const double dz = exy[1] - exy[0];
    val = fma(t[2], dz, exy[0]);
    g[0] = fma(t[2], dxy[1] - dxy[0], dxy[0]) * e.m.inv_h;
    g[1] = fma(t[2], dyx[1] - dyx[0], dyx[0]) * e.m.inv_h;
    g[2] = dz * e.m.inv_h;
}

// Transport velocity at Q1 node `node` from the point y (cell units) whose velocity is extended:
// u_Gamma = u(y) + mdot/rho_* n(x), n(x) the point-located normal at the node.
__device__ void transport_finish(const PointEval& e, const double* __restrict__ mdot, int64_t node, const double y[3],
                                 double rho_t, double* __restrict__ ug) {
    const MeshArgs<double>& m = e.m;
    const int m1 = m.n + 1;
    const double sx[3] = {(double)(node % m1), (double)((node / m1) % m1), (double)(node / ((int64_t)m1 * m1))};
    double ph, g[3];
    e.phi_grad(sx, ph, g);
    const double nrm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    double nx[3] = {0.0, 0.0, 0.0};
    if (nrm * m.h > GRAD_TINY) { nx[0] = g[0] / nrm; nx[1] = g[1] / nrm; nx[2] = g[2] / nrm; }
    double out[3];
    e.velocity(y, out);
    const double c = mdot[node] / rho_t;
    ug[node] = out[0] + c * nx[0];
    ug[m.Nphi + node] = out[1] + c * nx[1];
    ug[2 * m.Nphi + node] = out[2] + c * nx[2];
}

__device__ __forceinline__ bool in_projection_band(int variant, double phx) {
    return variant == 2 ? (-PHI_GAS_BAND < phx) && (phx < PHI_BAND) : (-PHI_BAND < phx) && (phx < PHI_GAS_BAND);
}

// Pass 1, one thread per Q1 node: variant 1 (Eq. transport_vel_local_continuous) and the nodes of variants 2/3
// outside the projection band (y = x) are finished here; band nodes are appended to a list for pass 2, so that
// the iterating nodes fill whole warps.
__global__ void k_transport_direct(PointEval e, const double* __restrict__ mdot, double* __restrict__ ug,
                                   int32_t* __restrict__ flags, int32_t* __restrict__ band, int32_t* band_count) {
    const MeshArgs<double>& m = e.m;
    const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (node >= m.Nphi) return;
    const double phx = e.phi[node];
    flags[node] = 0;
    if (m.variant == 1) {
        const int m1 = m.n + 1;
        const int i = (int)(node % m1), j = (int)((node / m1) % m1), k = (int)(node / ((int64_t)m1 * m1));
        const double sx[3] = {(double)i, (double)j, (double)k};
        double ph, g[3];
        e.phi_grad(sx, ph, g);
        const double nrm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        double nx[3] = {0.0, 0.0, 0.0};
        if (nrm * m.h > GRAD_TINY) { nx[0] = g[0] / nrm; nx[1] = g[1] / nrm; nx[2] = g[2] / nrm; }
        const Material mat = material(phx, 0.0, 0.0, 0.0, m);
        double uv[3];
        if (m.nsub == 1 || m.nsub == m.P) {  // the node is a velocity node
            const int st = m.nsub == 1 ? m.P : 1;
            const int64_t vn = (int64_t)(st * i) + (int64_t)m.M * ((int64_t)(st * j) + (int64_t)m.M * (st * k));
            uv[0] = e.u[vn];
            uv[1] = e.u[m.Nu + vn];
            uv[2] = e.u[2 * m.Nu + vn];
        } else {
            e.velocity(sx, uv);
        }
        const double c = mdot[node] / mat.rho;
        ug[node] = uv[0] + c * nx[0];
        ug[m.Nphi + node] = uv[1] + c * nx[1];
        ug[2 * m.Nphi + node] = uv[2] + c * nx[2];
        return;
    }
    if (in_projection_band(m.variant, phx)) {
        band[atomicAdd(band_count, 1)] = (int32_t)node;
        return;
    }
    const int m1 = m.n + 1;
    const double y[3] = {(double)(node % m1), (double)((node / m1) % m1), (double)(node / ((int64_t)m1 * m1))};
    transport_finish(e, mdot, node, y, m.variant == 2 ? m.rho_l : m.rho_g, ug);
}

// Pass 2, persistent: closest points of the band nodes on the liquid (variant 2) or gas (variant 3) end of the zone,
// y of band entry b to band_y[3 b], the convergence flag to flags[node].  band_count[1] hands out the entries.
__global__ void __launch_bounds__(32) k_transport_band(PointEval e, double tol, int kmax, const int32_t* __restrict__ band,
                                                       int32_t* band_count, double* __restrict__ band_y,
                                                       int32_t* __restrict__ flags, unsigned long long* flag_count,
                                                       unsigned long long* evals) {
    const MeshArgs<double>& m = e.m;
    const int count = band_count[0];
    const int m1 = m.n + 1;
    const double d_t = m.variant == 2 ? 3.0 * m.eps : -3.0 * m.eps;
    const double eps = m.eps, h = m.h, nn = (double)m.n;
    CppLane L;
    auto take = [&]() {
        L.b = atomicAdd(&band_count[1], 1);
        if (L.b >= count) {
            L.b = -1;
            return;
        }
        const int64_t node = band[L.b];
        L.x[0] = (double)(node % m1);
        L.x[1] = (double)((node / m1) % m1);
        L.x[2] = (double)(node / ((int64_t)m1 * m1));
        L.y[0] = L.x[0]; L.y[1] = L.x[1]; L.y[2] = L.x[2];
        L.phase = 0;
        L.steps = 0;
        L.trips = 0;
    };
    auto finish = [&](bool converged) {
        band_y[3 * (int64_t)L.b + 0] = L.y[0];
        band_y[3 * (int64_t)L.b + 1] = L.y[1];
        band_y[3 * (int64_t)L.b + 2] = L.y[2];
        flags[band[L.b]] = converged ? 0 : 1;
        if (!converged) atomicAdd(flag_count, 1ULL);
        atomicAdd(evals, (unsigned long long)L.trips);
        take();
    };
    take();
    const double c_step = 1.0 / (2.0 * eps * h);  // step (cell units) = r / (|grad d| h), |grad d| = 2 eps |g| / (1 - ph^2)
    while (__any_sync(0xffffffffu, L.b >= 0)) {
        if (L.b < 0) continue;
        ++L.trips;
        // the trip's point evaluation and the quantities every phase needs (computed by all lanes alike)
        const bool trial = L.phase == 2;
        double p[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) p[a] = trial ? L.yn[a] : L.y[a];
        double ph, g[3];
        q1_lerp(e, p, ph, g);
        ph = clampd(ph, -PHI_CLAMP, PHI_CLAMP);
        const double r = eps * log((1.0 + ph) / (1.0 - ph)) - d_t;
        const double nrm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        const double nv[3] = {g[0] * inv, g[1] * inv, g[2] * inv};
        const bool on = fabs(r) <= tol * h;
        const int max_steps = trial ? CPP_TRIAL_STEPS : CPP_NORMAL_STEPS;
        const bool can_step = !on && L.steps < max_steps && nrm > 0.0;
        if (L.phase != 1 && can_step) {  // normal step of the point being projected
            const double step = r * (1.0 - ph * ph) * inv * c_step;
#pragma unroll
            for (int a = 0; a < 3; ++a) p[a] = clampd(p[a] - step * nv[a], 0.0, nn);
            ++L.steps;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (trial) L.yn[a] = p[a];
                else L.y[a] = p[a];
            }
            continue;
        }
        if (L.phase == 0) {  // projection of the node ended
            if (on) {
                L.dist = dist3(L.y, L.x);
                L.k = 0;
                if (kmax <= 0) finish(false);
                else L.phase = 1;
            } else {
                finish(false);
            }
        } else if (L.phase == 1) {  // tangential part of y - x at y, first trial point
            L.tp[0] = L.tp[1] = L.tp[2] = 0.0;
            if (nrm > 0.0) {
                const bool alt = fabs(nv[0]) > 0.9;  // v = e_y instead of e_x
                const double vn = alt ? nv[1] : nv[0];
                double t0[3] = {(alt ? 0.0 : 1.0) - vn * nv[0], (alt ? 1.0 : 0.0) - vn * nv[1], -vn * nv[2]};
                const double t0n = sqrt(t0[0] * t0[0] + t0[1] * t0[1] + t0[2] * t0[2]);
                if (t0n > 0.0) {
                    const double it = 1.0 / t0n;
                    t0[0] *= it; t0[1] *= it; t0[2] *= it;
                }
                const double t1[3] = {nv[1] * t0[2] - nv[2] * t0[1], nv[2] * t0[0] - nv[0] * t0[2],
                                      nv[0] * t0[1] - nv[1] * t0[0]};
                const double dl[3] = {L.y[0] - L.x[0], L.y[1] - L.x[1], L.y[2] - L.x[2]};
                const double a0 = dl[0] * t0[0] + dl[1] * t0[1] + dl[2] * t0[2];
                const double a1 = dl[0] * t1[0] + dl[1] * t1[1] + dl[2] * t1[2];
#pragma unroll
                for (int a = 0; a < 3; ++a) L.tp[a] = a0 * t0[a] + a1 * t1[a];
            }
            L.omega = 1.0;
            L.bt = 0;
            L.dist_prev = L.dist;
#pragma unroll
            for (int a = 0; a < 3; ++a) L.yn[a] = clampd(L.y[a] - L.omega * L.tp[a], 0.0, nn);
            L.steps = 0;
            L.phase = 2;
        } else {  // projection of the trial point ended: on the isocontour (on) or failed
            const double dn = dist3(L.yn, L.x);
            if (on && dn < L.dist) {  // accepted
                L.dist = dn;
                const double step = dist3(L.yn, L.y);
                const double gain = L.dist_prev - L.dist;
                L.y[0] = L.yn[0]; L.y[1] = L.yn[1]; L.y[2] = L.yn[2];
                if (step <= tol || gain <= CPP_STALL * L.dist) finish(true);
                else if (++L.k == kmax) finish(false);
                else L.phase = 1;
            } else if (++L.bt == CPP_BACKTRACK) {  // no shorter point on the isocontour
                finish(true);
            } else {
                L.omega *= 0.5;
#pragma unroll
                for (int a = 0; a < 3; ++a) L.yn[a] = clampd(L.y[a] - L.omega * L.tp[a], 0.0, nn);
                L.steps = 0;
            }
        }
    }
}

// Pass 3, one thread per band entry: u_Gamma at the band nodes from their closest points.
__global__ void k_transport_band_finish(PointEval e, const double* __restrict__ mdot, const int32_t* __restrict__ band,
                                        const int32_t* __restrict__ band_count, const double* __restrict__ band_y,
                                        double* __restrict__ ug) {
    const int count = band_count[0];
    const double rho_t = e.m.variant == 2 ? e.m.rho_l : e.m.rho_g;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x) {
        const double y[3] = {band_y[3 * (int64_t)b], band_y[3 * (int64_t)b + 1], band_y[3 * (int64_t)b + 2]};
        transport_finish(e, mdot, band[b], y, rho_t, ug);
    }
}

// Points whose velocity the last pass took, y [3][N_phi] (physical coordinates, component-major): the node itself,
// then (second kernel) the closest point of every band node.
__global__ void k_node_points(int n, int64_t Np, double h, double* __restrict__ y) {
    const int m1 = n + 1;
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < Np;
         node += (int64_t)gridDim.x * blockDim.x) {
        y[node] = h * (double)(node % m1);
        y[Np + node] = h * (double)((node / m1) % m1);
        y[2 * Np + node] = h * (double)(node / ((int64_t)m1 * m1));
    }
}

__global__ void k_band_points(const int32_t* __restrict__ band, const int32_t* __restrict__ band_count,
                              const double* __restrict__ band_y, double h, int64_t Np, double* __restrict__ y) {
    const int count = band_count[0];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x) {
        const int64_t node = band[b];
#pragma unroll
        for (int a = 0; a < 3; ++a) y[a * Np + node] = h * band_y[3 * (int64_t)b + a];
    }
}

int launch_closest_points(evap_mesh* h, double* y, cudaStream_t s) {
    const MeshArgs<double> m = ls_args<double>(h);
    k_node_points<<<blocks_for(m.Nphi, 256), 256, 0, s>>>(m.n, m.Nphi, m.h, y);
    EVAP_CHECK_LAUNCH("node_points");
    if (m.variant != 1) {
        k_band_points<<<blocks_for(m.Nphi, 256), 256, 0, s>>>(h->band_list, h->band_count, h->band_y, m.h, m.Nphi, y);
        EVAP_CHECK_LAUNCH("band_points");
    }
    return EVAP_OK;
}

int launch_transport_velocity(evap_mesh* h, cudaStream_t s, const double* phi) {
    PointEval e;
    e.phi = phi ? phi : h->phi;
    e.u = h->u;
    e.m = ls_args<double>(h);
    e.nu = h->m.n;
    e.inv_sub = 1.0 / h->m.nsub;
    const int P = h->m.P;
    if (P == 2) {
        e.gl[0] = 0.0; e.gl[1] = 0.5; e.gl[2] = 1.0; e.gl[3] = 0.0;
    } else {
        const double r = 0.5 / std::sqrt(5.0);
        e.gl[0] = 0.0; e.gl[1] = 0.5 - r; e.gl[2] = 0.5 + r; e.gl[3] = 1.0;
    }
    EVAP_CUDA(cudaMemsetAsync(h->flag_count, 0, sizeof(unsigned long long), s));
    EVAP_CUDA(cudaMemsetAsync(h->band_count, 0, 2 * sizeof(int32_t), s));
    EVAP_CUDA(cudaMemsetAsync(h->cpp_evals, 0, sizeof(unsigned long long), s));
    k_transport_direct<<<blocks_for(h->m.Nphi, 128, 1LL << 40), 128, 0, s>>>(e, h->mdot, h->ugamma, h->cpp_flags,
                                                                            h->band_list, h->band_count);
    EVAP_CHECK_LAUNCH("transport_direct");
    if (h->m.variant != 1) {
        // Persistent pass sized to about 2 band nodes per lane (lanes that finish early take the remaining entries,
        // so warps stay full until the tail), at most 8 warps per SM: the FP64 pipe, not occupancy, bounds it.
        // Measured on the 64^3 four-sphere band (49 k nodes): 2 nodes per lane 3.9 ms, 4 nodes 5.0 ms, 1 node 4.3 ms;
        // on the 128^3 deformed sphere (181 k nodes, capped at 8 warps per SM) 9.6 ms, and 10.6 ms at 16 warps.
        int32_t count = 0;
        EVAP_CUDA(cudaMemcpyAsync(&count, h->band_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        EVAP_CUDA(cudaStreamSynchronize(s));
        const int grid = (int)std::min<int64_t>(std::max<int64_t>(((int64_t)count + 63) / 64, 1), 152 * 8);
        k_transport_band<<<grid, 32, 0, s>>>(e, h->prm.cpp_tol, h->prm.cpp_kmax, h->band_list, h->band_count,
                                             h->band_y, h->cpp_flags, h->flag_count, h->cpp_evals);
        EVAP_CHECK_LAUNCH("transport_band");
        k_transport_band_finish<<<blocks_for(h->m.Nphi, 128, 152 * 16), 128, 0, s>>>(e, h->mdot, h->band_list,
                                                                                      h->band_count, h->band_y,
                                                                                      h->ugamma);
        EVAP_CHECK_LAUNCH("transport_band_finish");
    }
    return refresh_ugamma_copies(h, s);
}

}  // namespace evap
