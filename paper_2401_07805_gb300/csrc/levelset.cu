// Matrix-free Q1 level-set operators with the 2^3 Gauss rule (Sec. 2.5), one thread per cell:
//   EVAP_ADVECT      y_i = sum_q W [ N_i x + theta dt N_i (u_Gamma . grad x) ]            Eq. (weakFormLevelSet), CN
//   EVAP_REINIT      y_i = sum_q W [ N_i x / dtau + eps (grad N_i . n)(grad x . n) ]      Eq. (reinitialization)
//   EVAP_REINIT_RHS  y_i = sum_q W [ N_i x / dtau + (grad N_i . n) (1 - x^2) / 2 ]        explicit compressive flux
// with n the frozen normal at the quadrature point: grad phi / |grad phi| of the level set (Eq. normal_vector), or,
// when a nodal normal field is set (e.g. the projected normal of Eq. normal_vector_regularized), its normalized
// interpolant (ls_frozen_normal).  The FP64 advection runs in double-float arithmetic (the FP64 pipe bounds the FP64
// version), sum-factorized (k_levelset_advect_sf; k_levelset_advect_df evaluates the same sums directly); the
// reinitialization operators stay in FP64.
#include <type_traits>

#include "dfloat.cuh"
#include "physics.cuh"

namespace evap {

template <typename T, int MODE, bool DET>
__global__ void __launch_bounds__(128) k_levelset(MeshArgs<T> m, Basis<T> bas, const T* __restrict__ phi,
                                                  const T* __restrict__ nf, const T* __restrict__ ug,
                                                  const T* __restrict__ x, T* __restrict__ y, int colour) {
    int cx, cy, cz;
    if constexpr (DET) {
        if (!colour_cell(blockIdx.x * (int64_t)blockDim.x + threadIdx.x, m.n, colour, cx, cy, cz)) return;
    } else {  // written out: the shared helper's form of this test cost the atomic variant 100 registers
        const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (cell >= m.ncell) return;
        cx = (int)(cell % m.n), cy = (int)((cell / m.n) % m.n), cz = (int)(cell / ((int64_t)m.n * m.n));
    }
    const int n = m.n;
    const int64_t m1 = n + 1;
    int64_t node[8];
    T xv[8], pv[8], uv[3][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        node[j] = (cx + (j & 1)) + m1 * ((cy + ((j >> 1) & 1)) + m1 * (cz + (j >> 2)));
        xv[j] = x[node[j]];
        if (MODE == EVAP_ADVECT) {
#pragma unroll
            for (int k = 0; k < 3; ++k) uv[k][j] = ug[k * m.Nphi + node[j]];
        } else if (nf) {
#pragma unroll
            for (int k = 0; k < 3; ++k) uv[k][j] = nf[k * m.Nphi + node[j]];
            pv[j] = T(0);
        } else {
            pv[j] = phi[node[j]];
        }
    }
    T out[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) out[j] = 0;
    const T ih = m.inv_h;
    const T W = T(0.125) * m.vol_w;  // 2-point Gauss weights 1/2 in each direction
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        // shape values and reference derivatives at the point: compile-time constants once the loops are unrolled
        const int qx = q & 1, qy = (q >> 1) & 1, qz = q >> 2;
        const T tx = T(g2_point(qx)), ty = T(g2_point(qy)), tz = T(g2_point(qz));
        const T Nx[2] = {T(1) - tx, tx}, Ny[2] = {T(1) - ty, ty}, Nz[2] = {T(1) - tz, tz};
        const T Dd[2] = {T(-1), T(1)};
        T N[8], dR[8][3];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int ja = j & 1, jb = (j >> 1) & 1, jc = j >> 2;
            N[j] = Nx[ja] * Ny[jb] * Nz[jc];
            dR[j][0] = Dd[ja] * Ny[jb] * Nz[jc];
            dR[j][1] = Nx[ja] * Dd[jb] * Nz[jc];
            dR[j][2] = Nx[ja] * Ny[jb] * Dd[jc];
        }
        T X = 0, GX[3] = {0, 0, 0};  // value and reference gradient (physical gradient = GX / h)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            X += N[j] * xv[j];
#pragma unroll
            for (int d = 0; d < 3; ++d) GX[d] += dR[j][d] * xv[j];
        }
        T Fv, Gf[3] = {0, 0, 0};  // Gf: flux tested with the reference gradients (physical flux / h)
        if (MODE == EVAP_ADVECT) {
            T U[3] = {0, 0, 0};
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) U[k] += N[j] * uv[k][j];
            Fv = W * (X + m.theta * m.dt * ih * (U[0] * GX[0] + U[1] * GX[1] + U[2] * GX[2]));
        } else {
            T nv[3];
            ls_frozen_normal<T>(nf ? uv : nullptr, pv, N, dR, T(1), nv);  // |grad_ref phi| = |grad phi| h
            Fv = W * X / m.dtau;
            const T s = (MODE == EVAP_REINIT) ? W * m.eps * ih * ih * (GX[0] * nv[0] + GX[1] * nv[1] + GX[2] * nv[2])
                                              : W * T(0.5) * ih * (T(1) - X * X);
#pragma unroll
            for (int d = 0; d < 3; ++d) Gf[d] = s * nv[d];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) out[j] += N[j] * Fv + dR[j][0] * Gf[0] + dR[j][1] * Gf[1] + dR[j][2] * Gf[2];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) acc_add(&y[node[j]], out[j], DET);
}

// EVAP_ADVECT for the FP64 applies in double-float arithmetic (dfloat.cuh): the same sums with x converted per node,
// u_Gamma read from its double-float copy, every product and sum on hi + lo FP32 pairs, the scatter in FP64.  The
// shape values at the Gauss points are compile-time doubles split into pairs.
template <bool DET>
__global__ void __launch_bounds__(128) k_levelset_advect_df(MeshArgs<double> m, dfl W, dfl thdt_ih,
                                                            const float2* __restrict__ ug, const double* __restrict__ x,
                                                            double* __restrict__ y, int colour) {
    int cx, cy, cz;
    if constexpr (DET) {
        if (!colour_cell(blockIdx.x * (int64_t)blockDim.x + threadIdx.x, m.n, colour, cx, cy, cz)) return;
    } else {  // written out: the shared helper's form of this test cost the atomic variant 100 registers
        const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (cell >= m.ncell) return;
        cx = (int)(cell % m.n), cy = (int)((cell / m.n) % m.n), cz = (int)(cell / ((int64_t)m.n * m.n));
    }
    const int n = m.n;
    const int64_t m1 = n + 1;
    int64_t node[8];
    dfl xv[8], uv[3][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        node[j] = (cx + (j & 1)) + m1 * ((cy + ((j >> 1) & 1)) + m1 * (cz + (j >> 2)));
        xv[j] = df_from_double(x[node[j]]);
#pragma unroll
        for (int k = 0; k < 3; ++k) uv[k][j] = ld_df(ug + k * m.Nphi + node[j]);
    }
    dfl out[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) out[j] = dfl{0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int qx = q & 1, qy = (q >> 1) & 1, qz = q >> 2;
        const double tx = g2_point(qx), ty = g2_point(qy), tz = g2_point(qz);
        const double Nx[2] = {1.0 - tx, tx}, Ny[2] = {1.0 - ty, ty}, Nz[2] = {1.0 - tz, tz};
        dfl N[8], dR[8][3];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int ja = j & 1, jb = (j >> 1) & 1, jc = j >> 2;
            const double sx = ja ? 1.0 : -1.0, sy = jb ? 1.0 : -1.0, sz = jc ? 1.0 : -1.0;
            N[j] = df_from_double(Nx[ja] * Ny[jb] * Nz[jc]);
            dR[j][0] = df_from_double(sx * Ny[jb] * Nz[jc]);
            dR[j][1] = df_from_double(Nx[ja] * sy * Nz[jc]);
            dR[j][2] = df_from_double(Nx[ja] * Ny[jb] * sz);
        }
        dfl X = df_prod(N[0], xv[0]), GX[3], U[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            GX[d] = df_prod(dR[0][d], xv[0]);
            U[d] = df_prod(N[0], uv[d][0]);
        }
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            df_fma(X, N[j], xv[j]);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                df_fma(GX[d], dR[j][d], xv[j]);
                df_fma(U[d], N[j], uv[d][j]);
            }
        }
        dfl ug_gx = df_prod(df_norm(U[0]), df_norm(GX[0]));
        df_fma(ug_gx, df_norm(U[1]), df_norm(GX[1]));
        df_fma(ug_gx, df_norm(U[2]), df_norm(GX[2]));
        dfl v = df_norm(X);
        df_fma(v, thdt_ih, df_norm(ug_gx));
        const dfl Fv = df_mul(W, df_norm(v));
#pragma unroll
        for (int j = 0; j < 8; ++j) df_fma(out[j], N[j], Fv);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) acc_add(&y[node[j]], df_to_double(df_norm(out[j])), DET);
}

// The same operator by sum factorization: the trilinear interpolation of x and u_Gamma to the 2^3 Gauss points and
// the testing with the shape functions as three 1D sweeps of the 2 x 2 matrix N[q][j] (N_0 = 1 - t, N_1 = t at the
// Gauss points t), the reference gradient of x as differences along its own direction interpolated along the other
// two: 132 two-term double-float dot products per cell in place of the direct sums' 8 x 7 eight-term ones.
constexpr float dfc_hi(double v) { return (float)v; }
constexpr float dfc_lo(double v) { return (float)(v - (double)(float)v); }
__device__ __forceinline__ dfl dot2(dfl c0, dfl v0, dfl c1, dfl v1) {
    dfl s = df_prod(c0, v0);
    df_fma(s, c1, v1);
    return df_norm(s);
}
template <bool DET>
__global__ void __launch_bounds__(128) k_levelset_advect_sf(MeshArgs<double> m, dfl W, dfl thdt_ih,
                                                            const float2* __restrict__ ug, const double* __restrict__ x,
                                                            double* __restrict__ y, int colour) {
    int cx, cy, cz;
    if constexpr (DET) {
        if (!colour_cell(blockIdx.x * (int64_t)blockDim.x + threadIdx.x, m.n, colour, cx, cy, cz)) return;
    } else {
        const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (cell >= m.ncell) return;
        cx = (int)(cell % m.n), cy = (int)((cell / m.n) % m.n), cz = (int)(cell / ((int64_t)m.n * m.n));
    }
    constexpr double t0 = g2_point(0), t1 = g2_point(1);
    // N[q][j]: shape function j (0: 1 - t, 1: t) at Gauss point q
    const dfl N[2][2] = {{{dfc_hi(1.0 - t0), dfc_lo(1.0 - t0)}, {dfc_hi(t0), dfc_lo(t0)}},
                         {{dfc_hi(1.0 - t1), dfc_lo(1.0 - t1)}, {dfc_hi(t1), dfc_lo(t1)}}};
    const int n = m.n;
    const int64_t m1 = n + 1;
    int64_t node[8];  // j = ja + 2 jb + 4 jc
#pragma unroll
    for (int j = 0; j < 8; ++j) node[j] = (cx + (j & 1)) + m1 * ((cy + ((j >> 1) & 1)) + m1 * (cz + (j >> 2)));
    // values of a nodal field at the points q = qx + 2 qy + 4 qz
    auto interp = [&](const dfl* f, dfl* out) {
        dfl fx[8], fxy[8];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 2; ++q) fx[q + 2 * r] = dot2(N[q][0], f[2 * r], N[q][1], f[2 * r + 1]);
#pragma unroll
        for (int jc = 0; jc < 2; ++jc)
#pragma unroll
            for (int qy = 0; qy < 2; ++qy)
#pragma unroll
                for (int qx = 0; qx < 2; ++qx)
                    fxy[qx + 2 * (qy + 2 * jc)] = dot2(N[qy][0], fx[qx + 2 * (0 + 2 * jc)], N[qy][1], fx[qx + 2 * (1 + 2 * jc)]);
#pragma unroll
        for (int qz = 0; qz < 2; ++qz)
#pragma unroll
            for (int r = 0; r < 4; ++r) out[r + 4 * qz] = dot2(N[qz][0], fxy[r], N[qz][1], fxy[r + 4]);
    };
    dfl X[8], GXx[4], GXy[4], GXz[4];  // GXx[qy + 2 qz], GXy[qx + 2 qz], GXz[qx + 2 qy] (reference gradient)
    {
        dfl f[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] = df_from_double(x[node[j]]);
        dfl fx[8], dx[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int q = 0; q < 2; ++q) fx[q + 2 * r] = dot2(N[q][0], f[2 * r], N[q][1], f[2 * r + 1]);
            dx[r] = df_sub(f[2 * r + 1], f[2 * r]);  // r = jb + 2 jc
        }
        dfl fxy[8], dxb[4], dy[4];
#pragma unroll
        for (int jc = 0; jc < 2; ++jc) {
#pragma unroll
            for (int qy = 0; qy < 2; ++qy) {
#pragma unroll
                for (int qx = 0; qx < 2; ++qx)
                    fxy[qx + 2 * (qy + 2 * jc)] = dot2(N[qy][0], fx[qx + 2 * (0 + 2 * jc)], N[qy][1], fx[qx + 2 * (1 + 2 * jc)]);
                dxb[qy + 2 * jc] = dot2(N[qy][0], dx[0 + 2 * jc], N[qy][1], dx[1 + 2 * jc]);
            }
#pragma unroll
            for (int qx = 0; qx < 2; ++qx) dy[qx + 2 * jc] = df_sub(fx[qx + 2 * (1 + 2 * jc)], fx[qx + 2 * (0 + 2 * jc)]);
        }
#pragma unroll
        for (int qz = 0; qz < 2; ++qz) {
#pragma unroll
            for (int r = 0; r < 4; ++r) X[r + 4 * qz] = dot2(N[qz][0], fxy[r], N[qz][1], fxy[r + 4]);
#pragma unroll
            for (int qy = 0; qy < 2; ++qy) GXx[qy + 2 * qz] = dot2(N[qz][0], dxb[qy], N[qz][1], dxb[qy + 2]);
#pragma unroll
            for (int qx = 0; qx < 2; ++qx) GXy[qx + 2 * qz] = dot2(N[qz][0], dy[qx], N[qz][1], dy[qx + 2]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) GXz[r] = df_sub(fxy[r + 4], fxy[r]);
    }
    dfl Fv[8];
    {
        dfl U[3][8];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            dfl f[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) f[j] = ld_df(ug + d * m.Nphi + node[j]);
            interp(f, U[d]);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int qx = q & 1, qy = (q >> 1) & 1, qz = q >> 2;
            dfl ug_gx = df_prod(U[0][q], GXx[qy + 2 * qz]);
            df_fma(ug_gx, U[1][q], GXy[qx + 2 * qz]);
            df_fma(ug_gx, U[2][q], GXz[qx + 2 * qy]);
            dfl v = X[q];
            df_fma(v, thdt_ih, df_norm(ug_gx));
            Fv[q] = df_mul(W, df_norm(v));
        }
    }
    // test: out_j = sum_q N_j(q) Fv_q by the transposed sweeps z, y, x
    dfl T1[8], T2[8];
#pragma unroll
    for (int jc = 0; jc < 2; ++jc)
#pragma unroll
        for (int r = 0; r < 4; ++r) T1[r + 4 * jc] = dot2(N[0][jc], Fv[r], N[1][jc], Fv[r + 4]);  // r = qx + 2 qy
#pragma unroll
    for (int jc = 0; jc < 2; ++jc)
#pragma unroll
        for (int jb = 0; jb < 2; ++jb)
#pragma unroll
            for (int qx = 0; qx < 2; ++qx)
                T2[qx + 2 * (jb + 2 * jc)] = dot2(N[0][jb], T1[qx + 2 * (0 + 2 * jc)], N[1][jb], T1[qx + 2 * (1 + 2 * jc)]);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int ja = 0; ja < 2; ++ja) {
            const dfl o = dot2(N[0][ja], T2[2 * r], N[1][ja], T2[2 * r + 1]);
            acc_add(&y[node[ja + 2 * r]], df_to_double(o), DET);
        }
}

// Level-set advection kernel: 1 the sum-factorized k_levelset_advect_sf, 0 the direct sums of k_levelset_advect_df.
// Measured at 64^3 (275 k DoFs, 100 back-to-back applies): 45.2 against 57.8 us per apply.
#ifndef EVAP_LS_SF
#define EVAP_LS_SF 1
#endif

template <typename T>
int launch_levelset(evap_mesh* h, int mode, const T* x, T* y, cudaStream_t s) {
    const MeshArgs<T> m = ls_args<T>(h);  // Q1 on the level-set mesh
    const Basis<T> b = cast_basis<T>(h->b);
    const bool dbl = sizeof(T) == 8;
    const T* phi = dbl ? (const T*)h->phi : (const T*)h->phi32;
    const T* ug = dbl ? (const T*)h->ugamma : (const T*)h->ugamma32;
    const T* nf = dbl ? (const T*)h->ls_normal : (const T*)h->ls_normal32;
    int rc = launch_fill<T>(y, m.Nphi, T(0), s);
    if (rc) return rc;
    const int threads = 128;
    // colour passes (deterministic) or one atomic pass, each variant compiled apart
    auto go = [&](auto det) -> int {
        constexpr bool DET = decltype(det)::value;
        for (int colour = DET ? 0 : -1; colour < (DET ? 8 : 0); ++colour) {
            const int64_t cells = colour_cells(m.n, colour);
            if (cells == 0) continue;
            const unsigned grid = (unsigned)((cells + threads - 1) / threads);
            bool done = false;
            if constexpr (sizeof(T) == 8) {
                if (mode == EVAP_ADVECT) {  // FP64-accurate advection in double-float arithmetic
                    const dfl W = df_from_double(0.125 * (double)m.vol_w);  // 2-point Gauss weights 1/2 per direction
                    const dfl thdt_ih = df_from_double((double)m.theta * (double)m.dt * (double)m.inv_h);
                    (EVAP_LS_SF ? k_levelset_advect_sf<DET> : k_levelset_advect_df<DET>)<<<grid, threads, 0, s>>>(
                        m, W, thdt_ih, (const float2*)h->ugammadf,
                                                                       (const double*)x, (double*)y, colour);
                    done = true;
                }
            }
            if (done) {
            } else if (mode == EVAP_ADVECT) {
                k_levelset<T, EVAP_ADVECT, DET><<<grid, threads, 0, s>>>(m, b, phi, nullptr, ug, x, y, colour);
            } else if (mode == EVAP_REINIT) {
                k_levelset<T, EVAP_REINIT, DET><<<grid, threads, 0, s>>>(m, b, phi, nf, ug, x, y, colour);
            } else {
                k_levelset<T, EVAP_REINIT_RHS, DET><<<grid, threads, 0, s>>>(m, b, phi, nf, ug, x, y, colour);
            }
            EVAP_CHECK_LAUNCH("levelset");
        }
        return EVAP_OK;
    };
    return h->deterministic ? go(std::true_type{}) : go(std::false_type{});
}
template int launch_levelset<double>(evap_mesh*, int, const double*, double*, cudaStream_t);
template int launch_levelset<float>(evap_mesh*, int, const float*, float*, cudaStream_t);

}  // namespace evap
