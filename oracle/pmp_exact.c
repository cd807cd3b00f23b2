/*
 * CPU oracle for the exact pan matrix profile -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no source with the CUDA path.
 *
 * Definitions followed (Sec. 2, "Background and Problem"):
 *   Z_{i,m} = (T_{i,m} - mu_{i,m}) / sigma_{i,m}, population sigma; windows
 *   with sigma = 0 (constant windows) are ignored;
 *   d_m(i,j) = || Z_{i,m} - Z_{j,m} ||_2;
 *   a pair is valid when |i - j| >= excl;
 *   P_m[i] = min over valid j of d_m(i,j), I_m[i] = the lowest such j.
 *
 * Tier i  (oracle_pmp_direct / oracle_pmp_cells): the definition written out,
 *   two-pass FP64 moments and a direct FP64 sum of squared differences.
 * Tier ii (oracle_pmp_diag): the same minimum computed with the closed form
 *   d^2 = 2m(1 - rho), m*rho = (T_i.T_j - m mu_i mu_j)/(sigma_i sigma_j)
 *   (Sec. 2), where T_i.T_j runs along each diagonal by the sliding update
 *   QT(i+1,j+1) = QT(i,j) - t_i t_j + t_{i+m} t_{j+m}, recomputed directly
 *   every 1024 steps.  It is checked against tier i on small inputs.
 *
 * Profile rows are laid out [L][n] (row m - m_min, column i); columns
 * i > n - m, constant windows and cells without a valid neighbour hold
 * P = +inf and I = -1.
 *
 * A constant window is one whose maximum equals its minimum (exact test).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -2

static void set_threads(int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int32_t oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Two-pass FP64 mean and population standard deviation of every length-m
 * window; is_const[i] = 1 when the window's maximum equals its minimum. */
int32_t oracle_moments(const double *x, int64_t n, int32_t m, double *mu, double *sigma,
                       uint8_t *is_const) {
    if (!x || m < 1 || n < m) return ORACLE_EINVAL;
    int64_t nw = n - m + 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nw; ++i) {
        double s = 0.0, lo = x[i], hi = x[i];
        for (int32_t r = 0; r < m; ++r) {
            double v = x[i + r];
            s += v;
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        double mean = s / m, q = 0.0;
        for (int32_t r = 0; r < m; ++r) {
            double dv = x[i + r] - mean;
            q += dv * dv;
        }
        mu[i] = mean;
        sigma[i] = sqrt(q / m);
        is_const[i] = (uint8_t)(lo == hi);
    }
    return ORACLE_OK;
}

/* Direct FP64 z-normalised distance of one pair (Sec. 2). Returns +inf when
 * either window is constant. */
double oracle_dist(const double *x, int64_t n, int32_t m, int64_t i, int64_t j) {
    if (m < 1 || i < 0 || j < 0 || i + m > n || j + m > n) return NAN;
    double si = 0, sj = 0, li = x[i], hi = x[i], lj = x[j], hj = x[j];
    for (int32_t r = 0; r < m; ++r) {
        si += x[i + r];
        sj += x[j + r];
        if (x[i + r] < li) li = x[i + r];
        if (x[i + r] > hi) hi = x[i + r];
        if (x[j + r] < lj) lj = x[j + r];
        if (x[j + r] > hj) hj = x[j + r];
    }
    if (li == hi || lj == hj) return INFINITY;
    double mi = si / m, mj = sj / m, qi = 0, qj = 0;
    for (int32_t r = 0; r < m; ++r) {
        qi += (x[i + r] - mi) * (x[i + r] - mi);
        qj += (x[j + r] - mj) * (x[j + r] - mj);
    }
    double ii = 1.0 / sqrt(qi / m), ij = 1.0 / sqrt(qj / m), acc = 0.0;
    for (int32_t r = 0; r < m; ++r) {
        double dz = (x[i + r] - mi) * ii - (x[j + r] - mj) * ij;
        acc += dz * dz;
    }
    return sqrt(acc);
}

/* z-normalised windows of one length, row-major [nw][m]. */
static double *znorm_matrix(const double *x, int64_t n, int32_t m, uint8_t *is_const) {
    int64_t nw = n - m + 1;
    double *mu = (double *)malloc(sizeof(double) * nw);
    double *sg = (double *)malloc(sizeof(double) * nw);
    double *z = (double *)malloc(sizeof(double) * nw * m);
    if (!mu || !sg || !z) {
        free(mu); free(sg); free(z);
        return NULL;
    }
    oracle_moments(x, n, m, mu, sg, is_const);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nw; ++i) {
        double inv = is_const[i] ? 0.0 : 1.0 / sg[i];
        for (int32_t r = 0; r < m; ++r) z[i * m + r] = (x[i + r] - mu[i]) * inv;
    }
    free(mu);
    free(sg);
    return z;
}

static void fill_empty(double *P, int64_t *I, int64_t count) {
    for (int64_t t = 0; t < count; ++t) {
        P[t] = INFINITY;
        I[t] = -1;
    }
}

/* Tier i: every valid pair at every length, direct FP64 distances. */
int32_t oracle_pmp_direct(const double *x, int64_t n, int32_t m_min, int32_t m_max, int32_t excl,
                          double *P, int64_t *I, int32_t nthreads) {
    if (!x || !P || !I || m_min < 2 || m_max < m_min || excl < 1) return ORACLE_EINVAL;
    set_threads(nthreads);
    int32_t L = m_max - m_min + 1;
    fill_empty(P, I, (int64_t)L * n);
    for (int32_t m = m_min; m <= m_max; ++m) {
        if (n < m) continue;
        int64_t nw = n - m + 1;
        uint8_t *cst = (uint8_t *)malloc(nw);
        if (!cst) return ORACLE_ENOMEM;
        double *z = znorm_matrix(x, n, m, cst);
        if (!z) {
            free(cst);
            return ORACLE_ENOMEM;
        }
        double *Prow = P + (int64_t)(m - m_min) * n;
        int64_t *Irow = I + (int64_t)(m - m_min) * n;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < nw; ++i) {
            if (cst[i]) continue;
            double best = INFINITY;
            int64_t arg = -1;
            const double *zi = z + i * m;
            for (int64_t j = 0; j < nw; ++j) {
                if (cst[j] || llabs(i - j) < excl) continue;
                const double *zj = z + j * m;
                double acc = 0.0;
                for (int32_t r = 0; r < m; ++r) {
                    double dz = zi[r] - zj[r];
                    acc += dz * dz;
                }
                /* ascending j and strict '<' keep the lowest index on ties */
                if (acc < best) {
                    best = acc;
                    arg = j;
                }
            }
            Prow[i] = sqrt(best);
            Irow[i] = arg;
        }
        free(z);
        free(cst);
    }
    return ORACLE_OK;
}

/* Tier i restricted to chosen cells of one length: for each listed start i,
 * the exact (P_m[i], I_m[i]) over every valid j.  Used to check sampled cells
 * of series too long for the full oracle.  O(count * n * m). */
int32_t oracle_pmp_cells(const double *x, int64_t n, int32_t m, int32_t excl, const int64_t *rows,
                         int64_t count, double *P, int64_t *I, int32_t nthreads) {
    if (!x || !rows || !P || !I || m < 2 || n < m || excl < 1) return ORACLE_EINVAL;
    set_threads(nthreads);
    int64_t nw = n - m + 1;
    double *mu = (double *)malloc(sizeof(double) * nw);
    double *sg = (double *)malloc(sizeof(double) * nw);
    uint8_t *cst = (uint8_t *)malloc(nw);
    if (!mu || !sg || !cst) {
        free(mu); free(sg); free(cst);
        return ORACLE_ENOMEM;
    }
    oracle_moments(x, n, m, mu, sg, cst);
    for (int64_t t = 0; t < count; ++t) {
        int64_t i = rows[t];
        P[t] = INFINITY;
        I[t] = -1;
        if (i < 0 || i >= nw || cst[i]) continue;
        double best = INFINITY;
        int64_t arg = -1;
        double ii = 1.0 / sg[i];
#pragma omp parallel
        {
            double lbest = INFINITY;
            int64_t larg = -1;
#pragma omp for schedule(static)
            for (int64_t j = 0; j < nw; ++j) {
                if (cst[j] || llabs(i - j) < excl) continue;
                double ij = 1.0 / sg[j], acc = 0.0;
                for (int32_t r = 0; r < m; ++r) {
                    double dz = (x[i + r] - mu[i]) * ii - (x[j + r] - mu[j]) * ij;
                    acc += dz * dz;
                }
                if (acc < lbest || (acc == lbest && j < larg)) {
                    lbest = acc;
                    larg = j;
                }
            }
#pragma omp critical
            {
                if (larg >= 0 && (lbest < best || (lbest == best && larg < arg))) {
                    best = lbest;
                    arg = larg;
                }
            }
        }
        P[t] = sqrt(best);
        I[t] = arg;
    }
    free(mu);
    free(sg);
    free(cst);
    return ORACLE_OK;
}

/* Tier ii: closed-form distances from per-diagonal sliding dot products. */
int32_t oracle_pmp_diag(const double *x, int64_t n, int32_t m_min, int32_t m_max, int32_t excl,
                        double *P, int64_t *I, int32_t nthreads) {
    if (!x || !P || !I || m_min < 2 || m_max < m_min || excl < 1) return ORACLE_EINVAL;
    set_threads(nthreads);
    int32_t L = m_max - m_min + 1;
    fill_empty(P, I, (int64_t)L * n);
    for (int32_t m = m_min; m <= m_max; ++m) {
        if (n < m) continue;
        int64_t nw = n - m + 1;
        double *mu = (double *)malloc(sizeof(double) * nw);
        double *sg = (double *)malloc(sizeof(double) * nw);
        uint8_t *cst = (uint8_t *)malloc(nw);
        if (!mu || !sg || !cst) {
            free(mu); free(sg); free(cst);
            return ORACLE_ENOMEM;
        }
        oracle_moments(x, n, m, mu, sg, cst);
        double *Prow = P + (int64_t)(m - m_min) * n;
        int64_t *Irow = I + (int64_t)(m - m_min) * n;
        int nth = oracle_max_threads();
        /* per-thread private rows, merged in a fixed order afterwards */
        double *Pt = (double *)malloc(sizeof(double) * nw * nth);
        int64_t *It = (int64_t *)malloc(sizeof(int64_t) * nw * nth);
        if (!Pt || !It) {
            free(mu); free(sg); free(cst); free(Pt); free(It);
            return ORACLE_ENOMEM;
        }
        fill_empty(Pt, It, nw * nth);
#pragma omp parallel
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            double *Pp = Pt + (int64_t)tid * nw;
            int64_t *Ip = It + (int64_t)tid * nw;
#pragma omp for schedule(dynamic, 8)
            for (int64_t diag = excl; diag < nw; ++diag) {
                double qt = 0.0;
                for (int64_t i = 0; i + diag < nw; ++i) {
                    int64_t j = i + diag;
                    if ((i & 1023) == 0) {
                        qt = 0.0;
                        for (int32_t r = 0; r < m; ++r) qt += x[i + r] * x[j + r];
                    } else {
                        qt += x[i + m - 1] * x[j + m - 1] - x[i - 1] * x[j - 1];
                    }
                    if (cst[i] || cst[j]) continue;
                    double rho = (qt - m * mu[i] * mu[j]) / (m * sg[i] * sg[j]);
                    double d2 = 2.0 * m * (1.0 - rho);
                    if (d2 < 0.0) d2 = 0.0;
                    if (d2 < Pp[i] || (d2 == Pp[i] && j < Ip[i])) {
                        Pp[i] = d2;
                        Ip[i] = j;
                    }
                    if (d2 < Pp[j] || (d2 == Pp[j] && i < Ip[j])) {
                        Pp[j] = d2;
                        Ip[j] = i;
                    }
                }
            }
        }
        for (int64_t i = 0; i < nw; ++i) {
            double best = INFINITY;
            int64_t arg = -1;
            for (int t = 0; t < nth; ++t) {
                double v = Pt[(int64_t)t * nw + i];
                int64_t a = It[(int64_t)t * nw + i];
                if (a >= 0 && (v < best || (v == best && a < arg))) {
                    best = v;
                    arg = a;
                }
            }
            Prow[i] = arg >= 0 ? sqrt(best) : INFINITY;
            Irow[i] = arg;
        }
        free(Pt); free(It); free(mu); free(sg); free(cst);
    }
    return ORACLE_OK;
}
