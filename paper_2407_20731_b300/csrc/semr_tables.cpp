// Host-side basis tables of the CUDA path: GLL nodes and weights and the
// discretely orthonormal Legendre analysis/synthesis matrices.
//
// The nodes are the roots of (1 - x^2) P_N'(x), which is proportional to
// P_{N-1}(x) - P_{N+1}(x); Newton's method on q = P_{N+1} - P_{N-1} uses
// q' = (2N + 1) P_N (a standard Legendre identity), in long double, from
// Chebyshev-Lobatto starting points.  Weights w_j = 2 / (N (N+1) P_N(x_j)^2).
// Basis phi_k = P_k / sqrt(gamma_k) with gamma_k = 2 / (2k + 1) for k < N and
// gamma_N = 2 / N, the GLL-quadrature norm of P_N, so that Phi^T W Phi = I and
// the analysis matrix A = Phi^T W inverts Phi.  (These are the standard SEM
// constructions behind the JPEG-like spectral truncation of arXiv 2407.20731,
// Sec. IV-B.)
#include "semr_internal.h"

#include <cmath>

namespace semr {

namespace {

long double legendre_ld(int k, long double x) {
    if (k == 0) return 1.0L;
    long double a = 1.0L, b = x;
    for (int n = 2; n <= k; ++n) {
        long double c = ((2 * n - 1) * x * b - (n - 1) * a) / n;
        a = b;
        b = c;
    }
    return b;
}

}  // namespace

int gll_nodes_weights(int lx, double* x, double* w) {
    if (lx < 2 || lx > kLxMaxTables || !x || !w) return SEMR_EINVAL;
    const int N = lx - 1;
    long double xs[kLxMaxTables];
    const long double pi = 3.141592653589793238462643383279502884L;
    xs[0] = -1.0L;
    xs[N] = 1.0L;
    for (int j = 1; j < N; ++j) {
        long double v = -std::cos(pi * j / N);
        for (int it = 0; it < 200; ++it) {
            long double q = legendre_ld(N + 1, v) - legendre_ld(N - 1, v);
            long double dq = (2 * N + 1) * legendre_ld(N, v);
            long double step = q / dq;
            v -= step;
            if (std::fabs(step) < 1e-19L) break;
        }
        xs[j] = v;
    }
    // exact mirror symmetry x_{N-j} = -x_j (the folded transforms rely on it)
    for (int j = 0; j < lx / 2; ++j) {
        long double h = (xs[N - j] - xs[j]) / 2;
        xs[j] = -h;
        xs[N - j] = h;
    }
    if (lx & 1) xs[N / 2] = 0.0L;
    for (int j = 0; j < lx; ++j) {
        long double p = legendre_ld(N, xs[j]);
        x[j] = (double)xs[j];
        w[j] = (double)(2.0L / ((long double)N * (N + 1) * p * p));
    }
    // the weights are mirror-symmetric too
    for (int j = 0; j < lx / 2; ++j) w[N - j] = w[j];
    return SEMR_OK;
}

int basis_tables(int lx, double* A, double* Phi, double* w_out) {
    double x[kLxMaxTables], w[kLxMaxTables];
    int rc = gll_nodes_weights(lx, x, w);
    if (rc) return rc;
    const int N = lx - 1;
    for (int k = 0; k < lx; ++k) {
        long double gamma = (k < N) ? 2.0L / (2 * k + 1) : 2.0L / N;
        long double s = 1.0L / std::sqrt(gamma);
        for (int i = 0; i < lx; ++i) {
            long double v = legendre_ld(k, (long double)x[i]) * s;
            // exact parity phi_k(-x) = (-1)^k phi_k(x) on the mirrored nodes
            if (i > N - i) {
                long double m = legendre_ld(k, (long double)x[N - i]) * s;
                v = (k & 1) ? -m : m;
            }
            Phi[i * lx + k] = (double)v;
            A[k * lx + i] = (double)(v * (long double)w[i]);
        }
    }
    if (w_out)
        for (int i = 0; i < lx; ++i) w_out[i] = w[i];
    return SEMR_OK;
}

}  // namespace semr
