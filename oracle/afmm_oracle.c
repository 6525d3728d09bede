/*
 * AFMM oracle: a plain, slow, obviously correct CPU statement of what the
 * AFMM method of Singh, Chakraborty and Mallick (arXiv 1308.2400) computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file.  Only the test suite, the smoke check of the package
 * entry module and the CPU-baseline leg of the benchmark use it.  It shares
 * no code, header, table or constant with the CUDA library.
 *
 * What it computes (Sec. 2, Case-A and Case-B listings; Sec. 2.1 Point 1):
 *   Z = X * Y for two dense n x n row-major matrices, Z starting at zero,
 *   every term formed by adding the real "Base" value to Z[i][j] "Rep-factor"
 *   times instead of multiplying, and zero Base values skipped.
 *
 * Readings of the printed listings (each also stated where it is used):
 *   - The upper limit of the inner sum is the Rep-factor just read
 *     (Y[k][j] in Case A, X[i][k] in Case B).  The listing prints floor(mu),
 *     but Sec. 2.1 Point 1 says each Base is summed Y[K,J] times and the
 *     addition count of Sec. 2.2 needs exactly that.
 *   - Case B tests Base = Y[k][j] inside the J loop; a zero Base skips that
 *     single j.  Leaving the whole J loop (the literal "beginning of the K
 *     loop") would not give X*Y, contradicting Sec. 2.1.
 *   - "Z <- Z + sum Base" adds Base into Z[i][j] once per unit of the
 *     Rep-factor (Rep-factor additions into Z).
 *   - A Rep-factor is a non-negative integer (Sec. 2 type lines; Sec. 2.1
 *     "rep-factor ... integer").  A negative one is rejected (return -1).
 *   - Loops run 0-based; the paper's are 1-based.
 *
 * Addition count: every "Z <- Z + Base" is one addition, so the returned
 * count equals sum over (i, k, j) with Base != 0 of the Rep-factor.
 * Its expectation is mu' * d1 * d2 * n^3 (Sec. 2.2).
 *
 * Row ranges: each entry point computes rows [i0, i1) of Z and stores row i
 * at Z + (i - i0) * n, so a large product can be checked on sampled rows.
 * Rows are independent (Sec. 2.1: the I-th row is final once its K loop is
 * exhausted); they run in parallel across OpenMP threads, each row serially
 * in k, j order, so the result does not depend on the thread count.
 *
 * Arithmetic: FP64 with round-to-nearest-even when Base is real; int64 when
 * both factors are integers (exact).
 */
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Case A (Sec. 2, Case-A): X real, Y integer Rep-factors.  The *_cols
 * forms compute the columns [j0, j1) of the rows [i0, i1) of Z (Z holds
 * j1 - j0 values per row), with every element formed exactly as in the
 * full row; the plain forms are the window [0, n). */
int afmm_oracle_caseA_f64_cols(int64_t n, int64_t i0, int64_t i1, int64_t j0,
                               int64_t j1, const double* X, const int64_t* Y,
                          double* Z, uint64_t* adds_out)
{
    int64_t bad = 0;
    uint64_t adds = 0;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : adds, bad)
    for (i = i0; i < i1; ++i) {
        double* z = Z + (i - i0) * (j1 - j0);
        for (int64_t j = j0; j < j1; ++j) z[j - j0] = 0.0;          /* Z starts at zero */
        for (int64_t k = 0; k < n; ++k) {
            const double base = X[i * n + k];                  /* Base <- X[I,K] */
            if (base == 0.0) continue;                         /* zero Base: next K */
            for (int64_t j = j0; j < j1; ++j) {
                const int64_t rep = Y[k * n + j];              /* Rep-factor <- Y[K,J] */
                if (rep < 0) { bad += 1; continue; }
                for (int64_t p = 0; p < rep; ++p) z[j - j0] += base; /* Rep additions */
                adds += (uint64_t)rep;
            }
        }
    }
    if (adds_out) *adds_out = adds;
    return bad ? -1 : 0;
}

int afmm_oracle_caseA_f64(int64_t n, int64_t i0, int64_t i1,
                          const double* X, const int64_t* Y,
                          double* Z, uint64_t* adds_out)
{
    return afmm_oracle_caseA_f64_cols(n, i0, i1, 0, n, X, Y, Z, adds_out);
}

/* Case B (Sec. 2, Case-B): X integer Rep-factors, Y real. */
int afmm_oracle_caseB_f64_cols(int64_t n, int64_t i0, int64_t i1, int64_t j0,
                               int64_t j1, const int64_t* X, const double* Y,
                          double* Z, uint64_t* adds_out)
{
    int64_t bad = 0;
    uint64_t adds = 0;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : adds, bad)
    for (i = i0; i < i1; ++i) {
        double* z = Z + (i - i0) * (j1 - j0);
        for (int64_t j = j0; j < j1; ++j) z[j - j0] = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            const int64_t rep = X[i * n + k];                  /* Rep-factor <- X[I,K] */
            if (rep < 0) { bad += 1; continue; }
            for (int64_t j = j0; j < j1; ++j) {
                const double base = Y[k * n + j];              /* Base <- Y[K,J] */
                if (base == 0.0) continue;                     /* zero Base: next J */
                for (int64_t p = 0; p < rep; ++p) z[j - j0] += base;
                adds += (uint64_t)rep;
            }
        }
    }
    if (adds_out) *adds_out = adds;
    return bad ? -1 : 0;
}

int afmm_oracle_caseB_f64(int64_t n, int64_t i0, int64_t i1,
                          const int64_t* X, const double* Y,
                          double* Z, uint64_t* adds_out)
{
    return afmm_oracle_caseB_f64_cols(n, i0, i1, 0, n, X, Y, Z, adds_out);
}

/* Case A with an integer-valued Base (both factors integer): exact int64. */
int afmm_oracle_caseA_i64_cols(int64_t n, int64_t i0, int64_t i1, int64_t j0,
                               int64_t j1, const int64_t* X, const int64_t* Y,
                          int64_t* Z, uint64_t* adds_out)
{
    int64_t bad = 0;
    uint64_t adds = 0;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : adds, bad)
    for (i = i0; i < i1; ++i) {
        int64_t* z = Z + (i - i0) * (j1 - j0);
        for (int64_t j = j0; j < j1; ++j) z[j - j0] = 0;
        for (int64_t k = 0; k < n; ++k) {
            const int64_t base = X[i * n + k];
            if (base == 0) continue;
            for (int64_t j = j0; j < j1; ++j) {
                const int64_t rep = Y[k * n + j];
                if (rep < 0) { bad += 1; continue; }
                for (int64_t p = 0; p < rep; ++p) z[j - j0] += base;
                adds += (uint64_t)rep;
            }
        }
    }
    if (adds_out) *adds_out = adds;
    return bad ? -1 : 0;
}

int afmm_oracle_caseA_i64(int64_t n, int64_t i0, int64_t i1,
                          const int64_t* X, const int64_t* Y,
                          int64_t* Z, uint64_t* adds_out)
{
    return afmm_oracle_caseA_i64_cols(n, i0, i1, 0, n, X, Y, Z, adds_out);
}

/* Case B with an integer-valued Base (both factors integer): exact int64. */
int afmm_oracle_caseB_i64_cols(int64_t n, int64_t i0, int64_t i1, int64_t j0,
                               int64_t j1, const int64_t* X, const int64_t* Y,
                          int64_t* Z, uint64_t* adds_out)
{
    int64_t bad = 0;
    uint64_t adds = 0;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : adds, bad)
    for (i = i0; i < i1; ++i) {
        int64_t* z = Z + (i - i0) * (j1 - j0);
        for (int64_t j = j0; j < j1; ++j) z[j - j0] = 0;
        for (int64_t k = 0; k < n; ++k) {
            const int64_t rep = X[i * n + k];
            if (rep < 0) { bad += 1; continue; }
            for (int64_t j = j0; j < j1; ++j) {
                const int64_t base = Y[k * n + j];
                if (base == 0) continue;
                for (int64_t p = 0; p < rep; ++p) z[j - j0] += base;
                adds += (uint64_t)rep;
            }
        }
    }
    if (adds_out) *adds_out = adds;
    return bad ? -1 : 0;
}

int afmm_oracle_caseB_i64(int64_t n, int64_t i0, int64_t i1,
                          const int64_t* X, const int64_t* Y,
                          int64_t* Z, uint64_t* adds_out)
{
    return afmm_oracle_caseB_i64_cols(n, i0, i1, 0, n, X, Y, Z, adds_out);
}

/*
 * The classical loops the paper times beside AFMM (Sec. 2.3.1, Table 1:
 * "ijk" and "ikj"), multiply-add in FP64.  They serve as a second
 * statement of Z = X * Y for the oracle's own checks and as the classical
 * CPU baseline.  Rows [i0, i1) as above.
 */
void afmm_classical_ijk_f64(int64_t n, int64_t i0, int64_t i1,
                            const double* X, const double* Y, double* Z)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = i0; i < i1; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int64_t k = 0; k < n; ++k) s += X[i * n + k] * Y[k * n + j];
            Z[(i - i0) * n + j] = s;
        }
}

void afmm_classical_ikj_f64(int64_t n, int64_t i0, int64_t i1,
                            const double* X, const double* Y, double* Z)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = i0; i < i1; ++i) {
        double* z = Z + (i - i0) * n;
        for (int64_t j = 0; j < n; ++j) z[j] = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            const double x = X[i * n + k];
            for (int64_t j = 0; j < n; ++j) z[j] += x * Y[k * n + j];
        }
    }
}

/* Number of OpenMP threads a parallel region of this library uses. */
int afmm_oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void afmm_oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
