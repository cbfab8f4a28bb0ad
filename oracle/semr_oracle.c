/*
 * semr_oracle.c -- plain FP64 CPU oracle for the in-situ reduction of
 * spectral-element (SEM) field snapshots.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the package's
 * smoke() check and the CPU-baseline leg of the benchmark load this file's
 * library.  It shares no code, header, table or constant with the CUDA path:
 * it builds its own Gauss-Lobatto-Legendre (GLL) rule and Legendre basis and
 * writes its own payload.  It is deliberately slow and obvious: every step is
 * a plain loop in the order the method states it, summed in increasing index
 * order, in IEEE double precision (compile without -ffast-math and with
 * -ffp-contract=off so that no fused multiply-add changes a rounding).
 *
 * What it computes (arXiv 2407.20731, Sec. IV-B, "Turbulence with data
 * compression"): the physics-based lossy compression of SEM fields that the
 * paper runs in situ on the GPU.  The paper describes the method only in
 * words: it is JPEG-like (a transform to a spectral basis followed by
 * truncation), it keeps only the most energetic part of each element's data
 * (after Otero et al.), and the amount kept is set by a maximal allowed
 * error.  The paper prints no formula for it, so the steps below are the
 * standard SEM constructions, with the unstated choices resolved as follows:
 *
 *   1. GLL rule (the SEM text the paper cites in Sec. IV-A, Deville, Fischer
 *      & Mund 2002): nodes are -1, +1 and the roots of P_N', N = lx-1;
 *      weights w_j = 2 / (N (N+1) P_N(x_j)^2).
 *   2. Basis: discretely orthonormal Legendre polynomials
 *      phi_k = P_k / sqrt(gamma_k), gamma_k = 2/(2k+1) for k < N and
 *      gamma_N = 2/N (the GLL-quadrature norm of P_N), so that with
 *      Phi[i][k] = phi_k(x_i) and W = diag(w), Phi^T W Phi = I, and the
 *      forward matrix A = Phi^T W is the exact inverse of Phi.
 *   3. Forward transform a = (A x A x A) u, contracted along i, then j, then k.
 *   4. Energy S_e = sum_m a_m^2 (equal to the GLL-weighted energy of the
 *      element block by Parseval; the Jacobian cancels in the test below).
 *   5. Truncation: keep mode m iff a_m^2 >= tau * S_e (ties keep).
 *   6. Quantisation with a power-of-two step q_e = 2^{s_e},
 *      s_e = floor(log2 sqrt(t)), t = tau * S_e, taken exactly from the
 *      binary exponent of t: t = mu * 2^ex, mu in [1/2, 1), s_e =
 *      floor((ex - 1) / 2).  Codes c_m = rint(a_m / q_e), ties to even.
 *   7. Payload: header, per-field mask/step/count sections, then all codes.
 *   8. Reconstruction u~ = (Phi x Phi x Phi) a~ with a~_m = c_m q_e for kept
 *      modes and 0 otherwise.
 *   9. Error norms: e2_e = J_e sum w_i w_j w_k (u - u~)^2, E_e = J_e sum
 *      w_i w_j w_k u^2, Linf_e = max |u - u~|; per field L2_abs = sqrt(sum e2),
 *      L2_rel = sqrt(sum e2 / sum E), Linf_abs, Linf_rel = Linf_abs / max|u|.
 *  10. Fragile list: the decisions that rounding could flip (see
 *      oracle_reduce below).
 *
 * Variant (truncation = 1, cumulative energy): the maximal allowed error read
 * as a budget on the discarded energy, the sort-based form behind the paper's
 * "two sorting kernels" (Sec. IV-B): sort the element's mode energies a_m^2
 * ascending, drop the longest prefix whose running sum (in that order) stays
 * <= tau S_e, and keep every mode whose energy is at least the first energy
 * not dropped (equal energies are kept together).  Step and codes as above.
 *
 * Special cases: tau = 0 is lossless mode (keep every mode, store the raw
 * FP64 coefficients).  An element whose threshold t = tau * S_e is below the
 * smallest normal double (this includes S_e = 0) keeps nothing and stores the
 * step sentinel INT16_MIN.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_LX_MIN 2
#define ORACLE_LX_MAX 16

/* Status codes (mirrors the meaning, not the code, of the library's). */
#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOSPACE 2

/* Payload flag bits. */
#define ORACLE_FLAG_LOSSLESS 1u
#define ORACLE_FLAG_CODE32 2u
#define ORACLE_FLAG_CUMULATIVE 8u

/* Legendre polynomial P_k(x) by the three-term (Bonnet) recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
double oracle_legendre(int k, double x)
{
    if (k == 0) return 1.0;
    double pm1 = 1.0, p = x;
    for (int n = 1; n < k; ++n) {
        double pp1 = ((2.0 * n + 1.0) * x * p - n * pm1) / (n + 1.0);
        pm1 = p;
        p = pp1;
    }
    return p;
}

/* GLL nodes x[0..lx-1] (ascending) and weights w[0..lx-1]. */
int oracle_gll(int lx, double *x, double *w)
{
    if (lx < ORACLE_LX_MIN || lx > ORACLE_LX_MAX || !x || !w) return ORACLE_EINVAL;
    const int N = lx - 1;
    const double pi = 3.14159265358979323846;
    x[0] = -1.0;
    x[N] = 1.0;
    for (int j = 1; j < N; ++j) {
        /* Newton iteration on P_N'(x) = 0 from the Chebyshev-Lobatto guess. */
        double xj = -cos(pi * j / N);
        for (int it = 0; it < 100; ++it) {
            double pN = oracle_legendre(N, xj);
            double pNm1 = oracle_legendre(N - 1, xj);
            double one_m_x2 = 1.0 - xj * xj;
            /* (1-x^2) P_N' = N (P_{N-1} - x P_N) */
            double d1 = N * (pNm1 - xj * pN) / one_m_x2;
            /* (1-x^2) P_N'' = 2 x P_N' - N (N+1) P_N */
            double d2 = (2.0 * xj * d1 - N * (N + 1.0) * pN) / one_m_x2;
            double dx = d1 / d2;
            xj -= dx;
            if (fabs(dx) < 1e-15) break;
        }
        x[j] = xj;
    }
    /* Symmetrise: x_{N-j} = -x_j exactly, and the middle node of an odd rule is 0. */
    for (int j = 0; j < lx / 2; ++j) {
        double s = 0.5 * (x[N - j] - x[j]);
        x[j] = -s;
        x[N - j] = s;
    }
    if (lx % 2 == 1) x[N / 2] = 0.0;
    for (int j = 0; j < lx; ++j) {
        double pN = oracle_legendre(N, x[j]);
        w[j] = 2.0 / (N * (N + 1.0) * pN * pN);
    }
    return ORACLE_OK;
}

/* Basis tables: phi[i*lx + k] = phi_k(x_i) (inverse / synthesis matrix Phi)
 * and amat[k*lx + i] = phi_k(x_i) * w_i (forward / analysis matrix A = Phi^T W). */
int oracle_tables(int lx, double *phi, double *amat)
{
    double x[ORACLE_LX_MAX], w[ORACLE_LX_MAX];
    int rc = oracle_gll(lx, x, w);
    if (rc) return rc;
    const int N = lx - 1;
    for (int k = 0; k < lx; ++k) {
        double gamma = (k < N) ? 2.0 / (2.0 * k + 1.0) : 2.0 / N;
        double scale = 1.0 / sqrt(gamma);
        for (int i = 0; i < lx; ++i) {
            double v = oracle_legendre(k, x[i]) * scale;
            if (phi) phi[i * lx + k] = v;
            if (amat) amat[k * lx + i] = v * w[i];
        }
    }
    return ORACLE_OK;
}

/* Forward transform of one element block u[k][j][i] (i fastest) to modal
 * coefficients a[r][q][p] (p fastest, m = p + lx (q + lx r)). */
void oracle_forward(int lx, const double *amat, const double *u, double *a)
{
    const int n = lx * lx * lx;
    double *t1 = (double *)malloc(sizeof(double) * n);
    double *t2 = (double *)malloc(sizeof(double) * n);
    /* along i: t1[k][j][p] = sum_i A[p][i] u[k][j][i] */
    for (int k = 0; k < lx; ++k)
        for (int j = 0; j < lx; ++j)
            for (int p = 0; p < lx; ++p) {
                double s = 0.0;
                for (int i = 0; i < lx; ++i) s += amat[p * lx + i] * u[(k * lx + j) * lx + i];
                t1[(k * lx + j) * lx + p] = s;
            }
    /* along j: t2[k][q][p] = sum_j A[q][j] t1[k][j][p] */
    for (int k = 0; k < lx; ++k)
        for (int q = 0; q < lx; ++q)
            for (int p = 0; p < lx; ++p) {
                double s = 0.0;
                for (int j = 0; j < lx; ++j) s += amat[q * lx + j] * t1[(k * lx + j) * lx + p];
                t2[(k * lx + q) * lx + p] = s;
            }
    /* along k: a[r][q][p] = sum_k A[r][k] t2[k][q][p] */
    for (int r = 0; r < lx; ++r)
        for (int q = 0; q < lx; ++q)
            for (int p = 0; p < lx; ++p) {
                double s = 0.0;
                for (int k = 0; k < lx; ++k) s += amat[r * lx + k] * t2[(k * lx + q) * lx + p];
                a[(r * lx + q) * lx + p] = s;
            }
    free(t1);
    free(t2);
}

/* Inverse (synthesis) transform u[k][j][i] = sum_{r,q,p} Phi[k][r] Phi[j][q]
 * Phi[i][p] a[r][q][p], contracted along p (i), then q (j), then r (k). */
void oracle_inverse(int lx, const double *phi, const double *a, double *u)
{
    const int n = lx * lx * lx;
    double *t1 = (double *)malloc(sizeof(double) * n);
    double *t2 = (double *)malloc(sizeof(double) * n);
    /* along p: t1[r][q][i] = sum_p Phi[i][p] a[r][q][p] */
    for (int r = 0; r < lx; ++r)
        for (int q = 0; q < lx; ++q)
            for (int i = 0; i < lx; ++i) {
                double s = 0.0;
                for (int p = 0; p < lx; ++p) s += phi[i * lx + p] * a[(r * lx + q) * lx + p];
                t1[(r * lx + q) * lx + i] = s;
            }
    /* along q: t2[r][j][i] = sum_q Phi[j][q] t1[r][q][i] */
    for (int r = 0; r < lx; ++r)
        for (int j = 0; j < lx; ++j)
            for (int i = 0; i < lx; ++i) {
                double s = 0.0;
                for (int q = 0; q < lx; ++q) s += phi[j * lx + q] * t1[(r * lx + q) * lx + i];
                t2[(r * lx + j) * lx + i] = s;
            }
    /* along r: u[k][j][i] = sum_r Phi[k][r] t2[r][j][i] */
    for (int k = 0; k < lx; ++k)
        for (int j = 0; j < lx; ++j)
            for (int i = 0; i < lx; ++i) {
                double s = 0.0;
                for (int r = 0; r < lx; ++r) s += phi[k * lx + r] * t2[(r * lx + j) * lx + i];
                u[(k * lx + j) * lx + i] = s;
            }
    free(t1);
    free(t2);
}

/* ---------------------------------------------------------------- payload */

static int64_t pad16(int64_t b) { return (b + 15) & ~(int64_t)15; }

/* Byte layout of the payload (all little-endian):
 *   header: "SEMR", u16 version(=1), u16 lx, u16 n_fields, u16 flags,
 *           u32 header_bytes, u64 n_elem, f64 tau, u64 code_base,
 *           u64 code_total, u64 code_count[n_fields]; padded to 16 bytes
 *   for each field f: mask  [n_elem][ceil(lx^3/8)] bytes (bit m of element e
 *                           is bit (m & 7) of byte e*mb + (m >> 3)), pad 16
 *                     step  int16 [n_elem], pad 16
 *                     count uint16[n_elem], pad 16
 *   codes: code_total entries of 2 (int16), 4 (int32) or 8 (f64, lossless)
 *          bytes, in (field, element, mode) ascending order, at code_base.
 */
int64_t oracle_header_bytes(int n_fields) { return pad16(48 + 8 * (int64_t)n_fields); }

int64_t oracle_field_fixed_bytes(int lx, int64_t n_elem)
{
    int64_t mb = (lx * lx * lx + 7) / 8;
    return pad16(n_elem * mb) + 2 * pad16(2 * n_elem);
}

static void put_u16(uint8_t *p, uint16_t v) { memcpy(p, &v, 2); }
static void put_u32(uint8_t *p, uint32_t v) { memcpy(p, &v, 4); }
static void put_u64(uint8_t *p, uint64_t v) { memcpy(p, &v, 8); }
static void put_f64(uint8_t *p, double v) { memcpy(p, &v, 8); }

/* Step exponent s = floor((ex - 1) / 2) for t = mu * 2^ex, mu in [1/2, 1). */
static int oracle_step_exponent(double t, double *mu_out)
{
    int ex = 0;
    double mu = frexp(t, &ex);
    if (mu_out) *mu_out = mu;
    int num = ex - 1;
    return (num >= 0) ? num / 2 : -((-num + 1) / 2);
}

/* Sort helper: indices by energy ascending, ties by index (per-thread key array). */
static _Thread_local const double *g_sort_e;
static int cmp_energy(const void *x, const void *y)
{
    int i = *(const int *)x, j = *(const int *)y;
    if (g_sort_e[i] < g_sort_e[j]) return -1;
    if (g_sort_e[i] > g_sort_e[j]) return 1;
    return (i > j) - (i < j);
}

/* Cumulative-energy boundary: energies e[0..n-1], budget t.  Returns the
 * smallest kept energy T (keep m iff e[m] >= T), or +inf when everything
 * fits the budget; *c_drop / *c_next get the running sums just before and
 * after the boundary, *e_last the largest dropped energy (-1 when none is
 * dropped), all for the fragile list. */
static double cumulative_boundary(int n, const double *e, double t, double *c_drop, double *c_next, double *e_last)
{
    int *idx = (int *)malloc(sizeof(int) * n);
    for (int m = 0; m < n; ++m) idx[m] = m;
    g_sort_e = e;
    qsort(idx, (size_t)n, sizeof(int), cmp_energy);
    double c = 0.0;
    int k = 0;
    while (k < n && c + e[idx[k]] <= t) {
        c += e[idx[k]];
        ++k;
    }
    *c_drop = c;
    *c_next = (k < n) ? c + e[idx[k]] : c;
    *e_last = (k > 0) ? e[idx[k - 1]] : -1.0;
    double T = (k < n) ? e[idx[k]] : INFINITY;
    free(idx);
    return T;
}

/*
 * oracle_reduce: the whole reduction of one snapshot.
 *
 *   fields      [n_fields][n_elem][lx^3] FP64, element blocks u[k][j][i]
 *   jac         [n_elem] element Jacobians (mass scale), > 0
 *   tau         threshold, tau >= 0 (tau == 0 is lossless mode)
 *   payload     output bytes (capacity cap); *payload_bytes gets the size
 *   elem_report [n_fields][n_elem][3] = (e2_e, E_e, Linf_e), or NULL
 *   field_report[n_fields][8] = (L2_abs, L2_rel, Linf_abs, Linf_rel,
 *               sum e2, sum E, max|u|, kept) or NULL
 *   recon       [n_fields][n_elem][lx^3] reconstruction, or NULL
 *   coeffs      [n_fields][n_elem][lx^3] modal coefficients a, or NULL
 *   fragile     [fragile_cap][4] = (field, element, mode or -1, kind):
 *               kind 1: |a_m^2 - t| <= 1e-9 t            (threshold decision)
 *               kind 2: kept and |frac(|a_m|/q) - 1/2| <= 1e-9 |a_m|/q
 *                                                        (rounding decision)
 *               kind 3: mode -1, mu within 1e-9 of 1/2 or 1 (step exponent)
 *               kind 4: mode -1, cumulative variant: the running sum at the
 *                       boundary (last dropped or first kept) within 1e-9 t,
 *                       or the last dropped and first kept energies within
 *                       1e-9 t of each other
 *   n_threads   OpenMP threads for the per-element loop (<= 0: default)
 *   truncation  0: per-coefficient threshold, 1: cumulative energy
 *
 * Returns ORACLE_OK, ORACLE_EINVAL or ORACLE_ENOSPACE (payload capacity; the
 * required size is still stored in *payload_bytes).  Fragile entries beyond
 * fragile_cap are counted in *n_fragile but not stored.
 */
int oracle_reduce(int lx, int64_t n_elem, int n_fields, const double *fields, const double *jac,
                  double tau, uint8_t *payload, int64_t cap, int64_t *payload_bytes,
                  double *elem_report, double *field_report, double *recon, double *coeffs,
                  int64_t *fragile, int64_t fragile_cap, int64_t *n_fragile, int n_threads, int truncation)
{
    if (lx < ORACLE_LX_MIN || lx > ORACLE_LX_MAX || n_elem < 0 || n_fields < 1 || n_fields > 64)
        return ORACLE_EINVAL;
    if (!(tau >= 0.0) || isinf(tau) || !payload_bytes || !n_fragile) return ORACLE_EINVAL;
    if (n_elem > 0 && (!fields || !jac)) return ORACLE_EINVAL;
    if (truncation != 0 && truncation != 1) return ORACLE_EINVAL;

    const int n = lx * lx * lx;
    const int mb = (n + 7) / 8;
    const int lossless = (tau == 0.0);
    const int code32 = !lossless && !(tau * 32767.0 * 32767.0 > 4.0);
    const int width = lossless ? 8 : (code32 ? 4 : 2);

    double phi[ORACLE_LX_MAX * ORACLE_LX_MAX], amat[ORACLE_LX_MAX * ORACLE_LX_MAX];
    double x[ORACLE_LX_MAX], w[ORACLE_LX_MAX];
    oracle_tables(lx, phi, amat);
    oracle_gll(lx, x, w);

    const int64_t nfe = (int64_t)n_fields * n_elem;
    /* Per element-field results of the parallel pass. */
    uint8_t *keep = (uint8_t *)calloc((size_t)(nfe * n + 1), 1);
    double *acoef = (double *)malloc(sizeof(double) * (size_t)(nfe * n + 1));
    int16_t *step = (int16_t *)malloc(sizeof(int16_t) * (size_t)(nfe + 1));
    uint16_t *count = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)(nfe + 1));
    double *rep = (double *)malloc(sizeof(double) * (size_t)(3 * nfe + 1));
    double *umaxe = (double *)malloc(sizeof(double) * (size_t)(nfe + 1));
    if (!keep || !acoef || !step || !count || !rep || !umaxe) {
        free(keep); free(acoef); free(step); free(count); free(rep); free(umaxe);
        return ORACLE_EINVAL;
    }

#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nt)
#endif
    for (int64_t fe = 0; fe < nfe; ++fe) {
        const int64_t e = fe % n_elem;
        const double *u = fields + fe * n;
        double *a = acoef + fe * n;
        uint8_t *kp = keep + fe * n;
        double *at = (double *)malloc(sizeof(double) * n);
        double *ut = (double *)malloc(sizeof(double) * n);

        oracle_forward(lx, amat, u, a);
        double S = 0.0;
        for (int m = 0; m < n; ++m) S += a[m] * a[m];

        int s = INT16_MIN;
        int cnt = 0;
        if (lossless) {
            for (int m = 0; m < n; ++m) { kp[m] = 1; at[m] = a[m]; }
            cnt = n;
        } else {
            double t = tau * S;
            if (t >= DBL_MIN) {
                s = oracle_step_exponent(t, NULL);
                double T = t, cd, cn, el;
                if (truncation == 1) {
                    double *en = (double *)malloc(sizeof(double) * n);
                    for (int m = 0; m < n; ++m) en[m] = a[m] * a[m];
                    T = cumulative_boundary(n, en, t, &cd, &cn, &el);
                    free(en);
                }
                for (int m = 0; m < n; ++m) {
                    if (a[m] * a[m] >= T) {
                        kp[m] = 1;
                        double c = nearbyint(ldexp(a[m], -s));
                        at[m] = ldexp(c, s);
                        ++cnt;
                    } else {
                        at[m] = 0.0;
                    }
                }
            } else {
                for (int m = 0; m < n; ++m) at[m] = 0.0;
            }
        }
        step[fe] = (int16_t)s;
        count[fe] = (uint16_t)cnt;

        oracle_inverse(lx, phi, at, ut);
        double e2 = 0.0, en = 0.0, linf = 0.0, umax = 0.0;
        for (int k = 0; k < lx; ++k)
            for (int j = 0; j < lx; ++j)
                for (int i = 0; i < lx; ++i) {
                    int idx = (k * lx + j) * lx + i;
                    double wq = w[i] * w[j] * w[k];
                    double d = u[idx] - ut[idx];
                    e2 += wq * (d * d);
                    en += wq * (u[idx] * u[idx]);
                    if (fabs(d) > linf) linf = fabs(d);
                    if (fabs(u[idx]) > umax) umax = fabs(u[idx]);
                }
        rep[3 * fe + 0] = jac[e] * e2;
        rep[3 * fe + 1] = jac[e] * en;
        rep[3 * fe + 2] = linf;
        umaxe[fe] = umax;
        if (recon) memcpy(recon + fe * n, ut, sizeof(double) * n);
        free(at);
        free(ut);
    }

    /* Payload size and field sums (serial, element order ascending). */
    const int64_t hdr = oracle_header_bytes(n_fields);
    const int64_t fixed = oracle_field_fixed_bytes(lx, n_elem);
    const int64_t code_base = hdr + n_fields * fixed;
    int64_t total_codes = 0;
    for (int64_t fe = 0; fe < nfe; ++fe) total_codes += count[fe];
    const int64_t bytes = code_base + total_codes * width;
    *payload_bytes = bytes;

    for (int f = 0; f < n_fields; ++f) {
        double se2 = 0.0, sen = 0.0, linf = 0.0, umax = 0.0;
        int64_t kept = 0;
        for (int64_t e = 0; e < n_elem; ++e) {
            int64_t fe = (int64_t)f * n_elem + e;
            se2 += rep[3 * fe + 0];
            sen += rep[3 * fe + 1];
            if (rep[3 * fe + 2] > linf) linf = rep[3 * fe + 2];
            if (umaxe[fe] > umax) umax = umaxe[fe];
            kept += count[fe];
        }
        if (field_report) {
            double *fr = field_report + 8 * f;
            fr[0] = sqrt(se2);
            fr[1] = (sen > 0.0) ? sqrt(se2 / sen) : 0.0;
            fr[2] = linf;
            fr[3] = (umax > 0.0) ? linf / umax : 0.0;
            fr[4] = se2;
            fr[5] = sen;
            fr[6] = umax;
            fr[7] = (double)kept;
        }
    }
    if (elem_report) memcpy(elem_report, rep, sizeof(double) * 3 * nfe);
    if (coeffs) memcpy(coeffs, acoef, sizeof(double) * n * nfe);

    /* Fragile list. */
    int64_t nfr = 0;
    if (!lossless) {
        for (int64_t fe = 0; fe < nfe; ++fe) {
            const double *a = acoef + fe * n;
            double S = 0.0;
            for (int m = 0; m < n; ++m) S += a[m] * a[m];
            double t = tau * S;
            if (!(t >= DBL_MIN)) continue;
            double mu = 0.0;
            int s = oracle_step_exponent(t, &mu);
            double q = ldexp(1.0, s);
            int64_t f = fe / n_elem, e = fe % n_elem;
            if (fabs(mu - 0.5) <= 1e-9 || fabs(mu - 1.0) <= 1e-9) {
                if (fragile && nfr < fragile_cap) {
                    fragile[4 * nfr + 0] = f; fragile[4 * nfr + 1] = e;
                    fragile[4 * nfr + 2] = -1; fragile[4 * nfr + 3] = 3;
                }
                ++nfr;
            }
            if (truncation == 1) {
                double *en = (double *)malloc(sizeof(double) * n);
                for (int m = 0; m < n; ++m) en[m] = a[m] * a[m];
                double cd, cn, el;
                const double T = cumulative_boundary(n, en, t, &cd, &cn, &el);
                free(en);
                /* a running sum at the boundary within rounding of the budget, or the
                 * last dropped and the first kept energy within rounding of each other
                 * (then the order of the two, and with it the kept set, is fragile) */
                if (fabs(cd - t) <= 1e-9 * t || fabs(cn - t) <= 1e-9 * t ||
                    (el >= 0.0 && isfinite(T) && T - el <= 1e-9 * t)) {
                    if (fragile && nfr < fragile_cap) {
                        fragile[4 * nfr + 0] = f; fragile[4 * nfr + 1] = e;
                        fragile[4 * nfr + 2] = -1; fragile[4 * nfr + 3] = 4;
                    }
                    ++nfr;
                }
            }
            for (int m = 0; m < n; ++m) {
                double a2 = a[m] * a[m];
                int kind = 0;
                if (truncation == 0 && fabs(a2 - t) <= 1e-9 * t) kind = 1;
                else if (keep[fe * n + m]) {
                    double y = fabs(a[m]) / q;
                    double fr = y - floor(y);
                    if (fabs(fr - 0.5) <= 1e-9 * y) kind = 2;
                }
                if (kind) {
                    if (fragile && nfr < fragile_cap) {
                        fragile[4 * nfr + 0] = f; fragile[4 * nfr + 1] = e;
                        fragile[4 * nfr + 2] = m; fragile[4 * nfr + 3] = kind;
                    }
                    ++nfr;
                }
            }
        }
    }
    *n_fragile = nfr;

    int rc = ORACLE_OK;
    if (!payload || cap < bytes) {
        rc = ORACLE_ENOSPACE;
    } else {
        memset(payload, 0, (size_t)bytes);
        memcpy(payload, "SEMR", 4);
        put_u16(payload + 4, 1);
        put_u16(payload + 6, (uint16_t)lx);
        put_u16(payload + 8, (uint16_t)n_fields);
        put_u16(payload + 10, (uint16_t)((lossless ? ORACLE_FLAG_LOSSLESS : 0u) |
                                         (code32 ? ORACLE_FLAG_CODE32 : 0u) |
                                         (truncation == 1 && !lossless ? ORACLE_FLAG_CUMULATIVE : 0u)));
        put_u32(payload + 12, (uint32_t)hdr);
        put_u64(payload + 16, (uint64_t)n_elem);
        put_f64(payload + 24, tau);
        put_u64(payload + 32, (uint64_t)code_base);
        put_u64(payload + 40, (uint64_t)total_codes);
        int64_t pos = code_base;
        for (int f = 0; f < n_fields; ++f) {
            uint8_t *sec = payload + hdr + f * fixed;
            uint8_t *msk = sec;
            uint8_t *stp = sec + pad16(n_elem * mb);
            uint8_t *cnt = stp + pad16(2 * n_elem);
            int64_t kept = 0;
            for (int64_t e = 0; e < n_elem; ++e) {
                int64_t fe = (int64_t)f * n_elem + e;
                const double *a = acoef + fe * n;
                int s = step[fe];
                for (int m = 0; m < n; ++m) {
                    if (!keep[fe * n + m]) continue;
                    msk[e * mb + (m >> 3)] |= (uint8_t)(1u << (m & 7));
                    if (lossless) {
                        put_f64(payload + pos, a[m]);
                    } else {
                        double c = nearbyint(ldexp(a[m], -s));
                        if (code32) put_u32(payload + pos, (uint32_t)(int32_t)c);
                        else put_u16(payload + pos, (uint16_t)(int16_t)c);
                    }
                    pos += width;
                }
                put_u16(stp + 2 * e, (uint16_t)step[fe]);
                put_u16(cnt + 2 * e, count[fe]);
                kept += count[fe];
            }
            put_u64(payload + 48 + 8 * f, (uint64_t)kept);
        }
    }

    free(keep); free(acoef); free(step); free(count); free(rep); free(umaxe);
    return rc;
}

/*
 * oracle_decode: rebuild the fields from a payload, with the same loops as
 * oracle_reduce's reconstruction.  recon gets [n_fields][n_elem][lx^3].
 * Returns ORACLE_EINVAL on a malformed payload, ORACLE_ENOSPACE if
 * recon_cap (in doubles) is too small.
 */
int oracle_decode(const uint8_t *payload, int64_t bytes, double *recon, int64_t recon_cap)
{
    if (!payload || bytes < 48 || memcmp(payload, "SEMR", 4) != 0) return ORACLE_EINVAL;
    uint16_t version, lx, nf, flags;
    uint32_t hdr;
    uint64_t ne, code_base, code_total;
    memcpy(&version, payload + 4, 2);
    memcpy(&lx, payload + 6, 2);
    memcpy(&nf, payload + 8, 2);
    memcpy(&flags, payload + 10, 2);
    memcpy(&hdr, payload + 12, 4);
    memcpy(&ne, payload + 16, 8);
    memcpy(&code_base, payload + 32, 8);
    memcpy(&code_total, payload + 40, 8);
    if (version != 1 || lx < ORACLE_LX_MIN || lx > ORACLE_LX_MAX || nf < 1) return ORACLE_EINVAL;
    const int n = lx * lx * lx, mb = (n + 7) / 8;
    const int lossless = (flags & ORACLE_FLAG_LOSSLESS) != 0;
    const int width = lossless ? 8 : ((flags & ORACLE_FLAG_CODE32) ? 4 : 2);
    const int64_t n_elem = (int64_t)ne;
    const int64_t fixed = oracle_field_fixed_bytes(lx, n_elem);
    if ((int64_t)hdr != oracle_header_bytes(nf) || (int64_t)code_base != hdr + nf * fixed) return ORACLE_EINVAL;
    if ((int64_t)(code_base + code_total * width) > bytes) return ORACLE_EINVAL;
    if (recon_cap < (int64_t)nf * n_elem * n) return ORACLE_ENOSPACE;

    double phi[ORACLE_LX_MAX * ORACLE_LX_MAX];
    oracle_tables(lx, phi, NULL);
    double *at = (double *)malloc(sizeof(double) * n);
    int64_t pos = (int64_t)code_base;
    for (int f = 0; f < nf; ++f) {
        const uint8_t *sec = payload + hdr + f * fixed;
        const uint8_t *msk = sec;
        const uint8_t *stp = sec + pad16(n_elem * mb);
        const uint8_t *cnt = stp + pad16(2 * n_elem);
        for (int64_t e = 0; e < n_elem; ++e) {
            int16_t s;
            uint16_t c_n;
            memcpy(&s, stp + 2 * e, 2);
            memcpy(&c_n, cnt + 2 * e, 2);
            int seen = 0;
            for (int m = 0; m < n; ++m) {
                if (msk[e * mb + (m >> 3)] & (1u << (m & 7))) {
                    if (pos + width > bytes) { free(at); return ORACLE_EINVAL; }
                    if (lossless) {
                        double v;
                        memcpy(&v, payload + pos, 8);
                        at[m] = v;
                    } else if (width == 4) {
                        int32_t c;
                        memcpy(&c, payload + pos, 4);
                        at[m] = ldexp((double)c, s);
                    } else {
                        int16_t c;
                        memcpy(&c, payload + pos, 2);
                        at[m] = ldexp((double)c, s);
                    }
                    pos += width;
                    ++seen;
                } else {
                    at[m] = 0.0;
                }
            }
            if (seen != c_n) { free(at); return ORACLE_EINVAL; }
            oracle_inverse(lx, phi, at, recon + ((int64_t)f * n_elem + e) * n);
        }
    }
    free(at);
    return ORACLE_OK;
}

/* Threads the OpenMP runtime would use by default (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
