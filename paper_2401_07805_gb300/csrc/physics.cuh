// Material law of the diffuse-interface model at one point, FP64 (device).
#pragma once

#include "evap_internal.cuh"

namespace evap {

// Whether node (gx, gy, gz) of an M^3 grid lies on a face selected by the bit mask f (bit 2 axis: face 0, bit
// 2 axis + 1: face M - 1).
__device__ __forceinline__ bool constrained_node(int gx, int gy, int gz, int M, unsigned f) {
    return ((f & 1u) && gx == 0) || ((f & 2u) && gx == M - 1) || ((f & 4u) && gy == 0) ||
           ((f & 8u) && gy == M - 1) || ((f & 16u) && gz == 0) || ((f & 32u) && gz == M - 1);
}

// Points of the 2-point Gauss rule on [0, 1], (1 -+ 1/sqrt 3) / 2 (the literal of the host basis).
__host__ __device__ constexpr double g2_point(int i) {
    return i ? 0.5 * (1.0 + 0.5773502691896257645091488) : 0.5 * (1.0 - 0.5773502691896257645091488);
}

// phi at d = 3 eps: tanh(3/2), the edge of the interface zone 0 < H < 1 (Eqs. initial_phi, heaviside).
constexpr double PHI_BAND = 0x1.cf6f9786df577p-1;      // tanh(3/2), correctly rounded
constexpr double PHI_GAS_BAND = 0x1.fd77d111a0b00p-1;  // tanh(3), correctly rounded (d = 6 eps)
constexpr double PI = 3.14159265358979323846;
// The normal grad phi/|grad phi| (Eq. normal_vector) is taken as 0 where |grad phi| h <= GRAD_TINY: phi varies by
// less than 1e-4 across the cell (more than ~9 eps from the interface), where the direction is ill-conditioned
// (rounding noise where phi has saturated to +-1).
constexpr double GRAD_TINY = 1e-4;

struct Material {
    double H, rho, mu, n[3], delta;
    bool zone;
};

// Eq. (heaviside) with d from Eq. (distance), Eq. (rhoEff), Eq. (muEff), Eq. (normal_vector), Eq. (delta).
// Outside the zone (|phi| >= tanh(3/2)) H is 0 or 1 and the logarithm is not evaluated.
__device__ __forceinline__ Material material(double phi, double gx, double gy, double gz, const MeshArgs<double>& m) {
    Material r;
    r.zone = fabs(phi) < PHI_BAND;
    double dH = 0.0, dd = 0.0;
    if (r.zone) {
        const double d = m.eps * log((1.0 + phi) / (1.0 - phi));
        double sn, cs;
        sincos(PI * d / (3.0 * m.eps), &sn, &cs);
        r.H = 0.5 + d / (6.0 * m.eps) + sn / (2.0 * PI);
        dH = (1.0 + cs) / (6.0 * m.eps);
        dd = 2.0 * m.eps / (1.0 - phi * phi);
    } else {
        r.H = phi >= PHI_BAND ? 1.0 : 0.0;
    }
    r.rho = 1.0 / (r.H / m.rho_l + (1.0 - r.H) / m.rho_g);
    r.mu = r.H * m.mu_l + (1.0 - r.H) * m.mu_g;
    const double gn = sqrt(gx * gx + gy * gy + gz * gz);
    if (gn * m.h > GRAD_TINY) {
        r.n[0] = gx / gn; r.n[1] = gy / gn; r.n[2] = gz / gn;
    } else {
        r.n[0] = r.n[1] = r.n[2] = 0.0;
    }
    r.delta = r.zone ? dH * dd * gn : 0.0;
    return r;
}

// Frozen normal of the reinitialization operators at a Q1 quadrature point (Eq. reinitialization): with a nodal
// field nf (nf[c][j] at the cell's 8 nodes) the normalized interpolant n_h / |n_h| (zero where |n_h| <= 1e-4), else the
// unit normal grad phi / |grad phi| (zero where |grad phi| h <= GRAD_TINY).  N[j], G[j][d]: Q1 values and
// physical gradients at the point; pv[j]: phi at the nodes.
constexpr double NODAL_NORMAL_TINY = 1e-4;
template <typename T>
__device__ __forceinline__ void ls_frozen_normal(const T (*nf)[8], const T pv[8], const T N[8], const T (*G)[3], T h,
                                                 T nv[3]) {
    T g[3] = {T(0), T(0), T(0)};
    if (nf) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int d = 0; d < 3; ++d) g[d] += N[j] * nf[d][j];
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int d = 0; d < 3; ++d) g[d] += G[j][d] * pv[j];
    }
    const T gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const bool ok = nf ? gn > T(NODAL_NORMAL_TINY) : gn * h > T(GRAD_TINY);
    nv[0] = nv[1] = nv[2] = T(0);
    if (ok) {
        const T ig = T(1) / gn;
        nv[0] = g[0] * ig;
        nv[1] = g[1] * ig;
        nv[2] = g[2] * ig;
    }
}

// c_1 = 1/rho_g - 1/rho_l, the factor of mdot delta in the dilation rate v = div u (Eq. evaporDil).  Sign: the
// printed Eq. (evaporDil) has the bracket reversed with respect to the paper's 1D solution (App. A,
// Eq. stefan_diffuse_velocity: div u = mdot (1/rho_g - 1/rho_l) delta) and to the c_1 of the variant-1 derivation;
// the latter is taken, so evaporation (mdot > 0, rho_g < rho_l) expands the volume.
__device__ __forceinline__ double dilation_coefficient(const MeshArgs<double>& m) {
    return 1.0 / m.rho_g - 1.0 / m.rho_l;
}

// Q1 field value and physical gradient at reference point (t[qx], t[qy], t[qz]) of cell (cx, cy, cz).
__device__ __forceinline__ void q1_at(const double* __restrict__ f, int n, int cx, int cy, int cz, double x, double y,
                                      double z, double inv_h, double& val, double g[3]) {
    const int m1 = n + 1;
    val = 0.0;
    g[0] = g[1] = g[2] = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const double v = f[(cx + a) + (int64_t)m1 * ((cy + b) + (int64_t)m1 * (cz + c))];
                const double wx = a ? x : 1.0 - x, wy = b ? y : 1.0 - y, wz = c ? z : 1.0 - z;
                const double dx = a ? 1.0 : -1.0, dy = b ? 1.0 : -1.0, dz = c ? 1.0 : -1.0;
                val += wx * wy * wz * v;
                g[0] += dx * wy * wz * v;
                g[1] += wx * dy * wz * v;
                g[2] += wx * wy * dz * v;
            }
    g[0] *= inv_h;
    g[1] *= inv_h;
    g[2] *= inv_h;
}

// Level-set field (value and physical gradient) at the reference point (x, y, z) of velocity cell (cx, cy, cz): the
// Q1 interpolant of the level-set cell containing it, the velocity cell subdivided nsub times per direction (Sec.
// 2.5; sub-cell floor(nsub t) clamped, so a point on a sub-cell face takes the upper sub-cell).
__device__ __forceinline__ void ls_at(const double* __restrict__ f, const MeshArgs<double>& m, int cx, int cy, int cz,
                                      double x, double y, double z, double& val, double g[3]) {
    const int k = m.nsub;
    if (k == 1) {
        q1_at(f, m.n, cx, cy, cz, x, y, z, m.inv_h, val, g);
        return;
    }
    const double s[3] = {x * k, y * k, z * k};
    int sub[3];
    double loc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int c = (int)floor(s[a]);
        c = c < 0 ? 0 : (c > k - 1 ? k - 1 : c);
        sub[a] = c;
        loc[a] = s[a] - c;
    }
    q1_at(f, m.nl, k * cx + sub[0], k * cy + sub[1], k * cz + sub[2], loc[0], loc[1], loc[2], m.inv_h * k, val, g);
}

// Whether the corrected-strain term is active at a point (Sec. 2.4.2; zone gate or everywhere).
__device__ __forceinline__ bool correction_on(const MeshArgs<double>& m, bool zone) {
    return m.stress != 0 && (m.corr_zone != 0 || zone);
}

}  // namespace evap
