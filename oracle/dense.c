/*
 * FP64 CPU oracle: plain dense IMQ products.  TEST INFRASTRUCTURE ONLY --
 * called from tests/, __graft_entry__.smoke() and bench.py's CPU baseline,
 * never from the product library.
 *
 * Definitions (arXiv 2205.04194, Section 2):
 *   Eq. (4)-(5): A_ij = phi(|x_i - x_j|) = 1/sqrt(t^2 + |x_i - x_j|^2),
 *   with the shape parameter t written c here; b = A u sums j = 1..N in index
 *   order, the diagonal included (A_ii = 1/c).
 *   Eq. (2): the interpolant P(x) = sum_j coef_j phi(|x - x_j|) at off-node x.
 *   dA/dc = -c / (r^2 + c^2)^{3/2} (derivative of Eq. (5) in its parameter).
 *
 * Compiled with -O2 -ffp-contract=off and no fast-math, so every expression is
 * evaluated in IEEE binary64 exactly as written.  Rows are split across
 * OpenMP threads; each row's sum is sequential in j, so the result does not
 * depend on the thread count.
 */
#include <math.h>
#include <stdint.h>

/* b[r*n + i] = sum_j A_ij u[r*n + j] for r < nrhs. pts is [n][2] row-major. */
void oracle_dense_matvec(const double *pts, int64_t n, double c,
                         const double *u, double *b, int nrhs)
{
    const double c2 = c * c;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        const double xi = pts[2 * i], yi = pts[2 * i + 1];
        for (int r = 0; r < nrhs; ++r) {
            const double *ur = u + (int64_t)r * n;
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                const double dx = xi - pts[2 * j];
                const double dy = yi - pts[2 * j + 1];
                const double a = 1.0 / sqrt(dx * dx + dy * dy + c2);
                s += a * ur[j];
            }
            b[(int64_t)r * n + i] = s;
        }
    }
}

/* Same as above for the listed rows only: b[k] = (A u)_{rows[k]}. */
void oracle_dense_rows(const double *pts, int64_t n, double c, const double *u,
                       const int64_t *rows, int64_t nrows, double *b)
{
    const double c2 = c * c;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t k = 0; k < nrows; ++k) {
        const int64_t i = rows[k];
        const double xi = pts[2 * i], yi = pts[2 * i + 1];
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double dx = xi - pts[2 * j];
            const double dy = yi - pts[2 * j + 1];
            const double a = 1.0 / sqrt(dx * dx + dy * dy + c2);
            s += a * u[j];
        }
        b[k] = s;
    }
}

/* Off-node evaluation: out[k] = sum_j coef_j phi(|t_k - x_j|)  (Eq. (2)).
 * With deriv != 0 the kernel is dphi/dc = -c (r^2+c^2)^{-3/2}. */
void oracle_evaluate(const double *src, int64_t n, const double *tgt, int64_t m,
                     double c, const double *coef, double *out, int deriv)
{
    const double c2 = c * c;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < m; ++k) {
        const double xt = tgt[2 * k], yt = tgt[2 * k + 1];
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double dx = xt - src[2 * j];
            const double dy = yt - src[2 * j + 1];
            const double q = dx * dx + dy * dy + c2;
            if (deriv) {
                s += coef[j] * (-c / (q * sqrt(q)));
            } else {
                s += coef[j] / sqrt(q);
            }
        }
        out[k] = s;
    }
}

/* Transposed evaluation: out[j] = sum_k r_k phi(|t_k - x_j|)  (E^T r). */
void oracle_evaluate_transpose(const double *src, int64_t n, const double *tgt, int64_t m,
                               double c, const double *r, double *out)
{
    const double c2 = c * c;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < n; ++j) {
        const double xs = src[2 * j], ys = src[2 * j + 1];
        double s = 0.0;
        for (int64_t k = 0; k < m; ++k) {
            const double dx = tgt[2 * k] - xs;
            const double dy = tgt[2 * k + 1] - ys;
            s += r[k] / sqrt(dx * dx + dy * dy + c2);
        }
        out[j] = s;
    }
}

/* Dense matrix assembly (small N only): A[i*n + j]. deriv selects dA/dc. */
void oracle_assemble(const double *pts, int64_t n, double c, double *A, int deriv)
{
    const double c2 = c * c;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            const double dx = pts[2 * i] - pts[2 * j];
            const double dy = pts[2 * i + 1] - pts[2 * j + 1];
            const double q = dx * dx + dy * dy + c2;
            A[i * n + j] = deriv ? (-c / (q * sqrt(q))) : (1.0 / sqrt(q));
        }
    }
}

int oracle_num_threads(void)
{
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            t = omp_get_num_threads();
#endif
        }
    }
    return t;
}
