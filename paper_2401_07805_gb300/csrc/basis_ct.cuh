// Compile-time 1D tables of the tensor-product Q_P velocity element (P = 2, 3) on [0, 1] (Sec. 2.5):
//   support points: Gauss-Lobatto points of degree P (P = 2: 0, 1/2, 1; P = 3: 0, 1/2 -+ 1/(2 sqrt 5), 1),
//   quadrature: the (P+1)-point Gauss-Legendre rule,
//   S[q][a] = l_a(t_q), D[q][a] = l_a'(t_q) (reference derivative), Dc[q][r] = L_r'(t_q) with L_r the Lagrange
//   polynomials through the Gauss points (collocation derivative), N1[q] = (1 - t_q, t_q).
// The irrational points and weights are decimal literals of the closed forms (correctly rounded by the compiler).
// Being constexpr, the tables enter kernels as instruction immediates (no constant-bank loads) and let the compiler
// drop the structural zeros (e.g. l_1'(1/2) = 0 for P = 2).  The host basis of a mesh is copied from the same tables.
#pragma once

namespace evap {

template <int P>
struct CtBasis {
    static constexpr int Q = P + 1;
    double t[Q] = {}, w[Q] = {}, gl[Q] = {};
    double S[Q][Q] = {}, D[Q][Q] = {}, Dc[Q][Q] = {}, N1[Q][2] = {};
    float wf[Q] = {};  // w rounded to FP32
};

// l_a(x) and l_a'(x) of the Lagrange basis through nodes[0..m) (product formula)
constexpr double ct_lagrange(const double* nodes, int m, int a, double x) {
    double v = 1.0;
    for (int k = 0; k < m; ++k)
        if (k != a) v *= (x - nodes[k]) / (nodes[a] - nodes[k]);
    return v;
}
constexpr double ct_lagrange_d(const double* nodes, int m, int a, double x) {
    double d = 0.0;
    for (int k = 0; k < m; ++k) {
        if (k == a) continue;
        double term = 1.0 / (nodes[a] - nodes[k]);
        for (int j = 0; j < m; ++j)
            if (j != a && j != k) term *= (x - nodes[j]) / (nodes[a] - nodes[j]);
        d += term;
    }
    return d;
}

template <int P>
constexpr CtBasis<P> make_ct_basis() {
    static_assert(P == 2 || P == 3, "degree 2 or 3");
    CtBasis<P> b{};
    constexpr int Q = P + 1;
    double x[Q] = {}, W[Q] = {};  // Gauss-Legendre on [-1, 1]
    if constexpr (P == 2) {
        constexpr double r = 0.7745966692414833770358531;  // sqrt(3/5)
        x[0] = -r; x[1] = 0.0; x[2] = r;
        W[0] = W[2] = 5.0 / 9.0;
        W[1] = 8.0 / 9.0;
        b.gl[0] = 0.0; b.gl[1] = 0.5; b.gl[2] = 1.0;
    } else {
        constexpr double a = 0.3399810435848562648026658;   // sqrt(3/7 - 2/7 sqrt(6/5))
        constexpr double c = 0.8611363115940525752239465;   // sqrt(3/7 + 2/7 sqrt(6/5))
        constexpr double wa = 0.6521451548625461426269360;  // (18 + sqrt 30) / 36
        constexpr double wc = 0.3478548451374538573730639;  // (18 - sqrt 30) / 36
        constexpr double r = 0.2236067977499789696409174;   // 1 / (2 sqrt 5)
        x[0] = -c; x[1] = -a; x[2] = a; x[3] = c;
        W[0] = wc; W[1] = wa; W[2] = wa; W[3] = wc;
        b.gl[0] = 0.0; b.gl[1] = 0.5 - r; b.gl[2] = 0.5 + r; b.gl[3] = 1.0;
    }
    for (int q = 0; q < Q; ++q) {
        b.t[q] = 0.5 * (x[q] + 1.0);
        b.w[q] = 0.5 * W[q];
        b.wf[q] = (float)b.w[q];
    }
    for (int q = 0; q < Q; ++q) {
        for (int k = 0; k < Q; ++k) {
            b.S[q][k] = ct_lagrange(b.gl, Q, k, b.t[q]);
            b.D[q][k] = ct_lagrange_d(b.gl, Q, k, b.t[q]);
            b.Dc[q][k] = ct_lagrange_d(b.t, Q, k, b.t[q]);
        }
        b.N1[q][0] = 1.0 - b.t[q];
        b.N1[q][1] = b.t[q];
    }
    return b;
}

// Device copy of the tables (a constant global with a known initializer: loads at indices that are constant after
// unrolling fold into immediates).
template <int P>
__device__ constexpr CtBasis<P> kCtBasis = make_ct_basis<P>();

}  // namespace evap
