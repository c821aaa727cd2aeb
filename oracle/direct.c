/*
 * Plain FP64 direct-sum oracle for the DDA interaction matrix (test
 * infrastructure only: the product path never links or calls this file).
 *
 * The linear system of the Discrete Dipole Approximation (OpenDDA, Eq. 1,
 * written in Gaussian units with lattice spacing d = 1):
 *
 *     sum_l A_jl P_l = E_inc,j,          A_jj = alpha_j^{-1},
 *     A_jl = exp(ikr)/r^3 [ k^2 (r r - r^2 I) + (ikr - 1)/r^2 (3 r r - r^2 I) ],
 *
 * r = r_j - r_l, r = |r|, "r r" the dyadic product of Eq. 2.  The paper's SI
 * form carries a prefactor k^2/eps0 and 1/(4 pi); multiplying it out gives
 * exactly this expression divided by 4 pi eps0, so the two systems share
 * their solution up to the unit of P.
 *
 * Everything here is the definition written out: every pair (j, l) is
 * summed on the fly, nothing is stored, no FFT, no blocking.  Complex
 * vectors are interleaved (re, im) doubles; vectors are laid out [3][n]
 * (component-major), matching the compressed polarisation vectors of Sec. 4.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Six independent components (xx, xy, xz, yy, yz, zz) of A_jl for r != 0
 * (Eq. 1 with Eq. 2; the tensor is symmetric, Sec. 3). */
static void interaction_tensor(double k, double rx, double ry, double rz, double complex t[6]) {
    const double r2 = rx * rx + ry * ry + rz * rz;
    const double r = sqrt(r2);
    const double complex e = cexp(I * k * r) / (r2 * r);
    const double complex f = (I * k * r - 1.0) / r2;
    const double rr[6] = {rx * rx, rx * ry, rx * rz, ry * ry, ry * rz, rz * rz};
    const int diag[6] = {1, 0, 0, 1, 0, 1};
    for (int m = 0; m < 6; ++m) {
        const double d = diag[m] ? r2 : 0.0;
        t[m] = e * (k * k * (rr[m] - d) + f * (3.0 * rr[m] - d));
    }
}

/* Exposed for the tests: the six components at one displacement. */
void oracle_interaction_tensor(double k, double rx, double ry, double rz, double* out12) {
    double complex t[6];
    interaction_tensor(k, rx, ry, rz, t);
    for (int m = 0; m < 6; ++m) {
        out12[2 * m] = creal(t[m]);
        out12[2 * m + 1] = cimag(t[m]);
    }
}

/* (row, col) -> index into the six stored components */
static const int comp_of[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

/*
 * y = A p for n dipoles at integer coordinates coords[n][3] (x, y, z).
 * ainv[n][3] (complex, interleaved) is alpha^{-1} of dipole j acting on
 * component c (the composition may differ per axis, Sec. 2).
 * p, y: [3][n] complex interleaved.  Rows are independent, so they are
 * shared among nthreads OpenMP threads (a reported baseline only).
 */
void oracle_direct_matvec(int64_t n, const int32_t* coords, const double* ainv, double k,
                          const double* p, double* y, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t j = 0; j < n; ++j) {
        double complex acc[3];
        for (int c = 0; c < 3; ++c) {
            const double complex a = ainv[(j * 3 + c) * 2] + I * ainv[(j * 3 + c) * 2 + 1];
            const double complex pj = p[(c * n + j) * 2] + I * p[(c * n + j) * 2 + 1];
            acc[c] = a * pj;
        }
        for (int64_t l = 0; l < n; ++l) {
            if (l == j) continue;
            double complex t[6];
            interaction_tensor(k, (double)(coords[3 * j] - coords[3 * l]),
                               (double)(coords[3 * j + 1] - coords[3 * l + 1]),
                               (double)(coords[3 * j + 2] - coords[3 * l + 2]), t);
            double complex pl[3];
            for (int c = 0; c < 3; ++c) pl[c] = p[(c * n + l) * 2] + I * p[(c * n + l) * 2 + 1];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc[a] += t[comp_of[a][b]] * pl[b];
        }
        for (int c = 0; c < 3; ++c) {
            y[(c * n + j) * 2] = creal(acc[c]);
            y[(c * n + j) * 2 + 1] = cimag(acc[c]);
        }
    }
}

/*
 * Selected rows of y = A p: out[c][q] = (A p)_{c, rows[q]} for q < nrows,
 * out laid out [3][nrows].  The same sum as oracle_direct_matvec, for
 * checking a few outputs of a large lattice one by one.
 */
void oracle_direct_matvec_rows(int64_t n, const int32_t* coords, const double* ainv, double k,
                               const double* p, const int64_t* rows, int64_t nrows, double* out,
                               int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int64_t q = 0; q < nrows; ++q) {
        const int64_t j = rows[q];
        double ar[3] = {0, 0, 0}, ai[3] = {0, 0, 0};
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : ar[:3], ai[:3])
#endif
        for (int64_t l = 0; l < n; ++l) {
            double complex pl[3];
            for (int c = 0; c < 3; ++c) pl[c] = p[(c * n + l) * 2] + I * p[(c * n + l) * 2 + 1];
            if (l == j) {
                for (int c = 0; c < 3; ++c) {
                    const double complex a = ainv[(j * 3 + c) * 2] + I * ainv[(j * 3 + c) * 2 + 1];
                    const double complex v = a * pl[c];
                    ar[c] += creal(v);
                    ai[c] += cimag(v);
                }
                continue;
            }
            double complex t[6];
            interaction_tensor(k, (double)(coords[3 * j] - coords[3 * l]),
                               (double)(coords[3 * j + 1] - coords[3 * l + 1]),
                               (double)(coords[3 * j + 2] - coords[3 * l + 2]), t);
            for (int a = 0; a < 3; ++a) {
                double complex s = 0.0;
                for (int b = 0; b < 3; ++b) s += t[comp_of[a][b]] * pl[b];
                ar[a] += creal(s);
                ai[a] += cimag(s);
            }
        }
        for (int c = 0; c < 3; ++c) {
            out[(c * nrows + q) * 2] = ar[c];
            out[(c * nrows + q) * 2 + 1] = ai[c];
        }
    }
}

/*
 * Dense A (3n x 3n, row-major, complex interleaved), unknown ordering
 * [3][n] to match the vectors: row index a*n + j, column index b*n + l.
 */
void oracle_dense_matrix(int64_t n, const int32_t* coords, const double* ainv, double k, double* A) {
    const int64_t N3 = 3 * n;
    for (int64_t i = 0; i < N3 * N3 * 2; ++i) A[i] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        for (int c = 0; c < 3; ++c) {
            const int64_t row = c * n + j;
            A[(row * N3 + row) * 2] = ainv[(j * 3 + c) * 2];
            A[(row * N3 + row) * 2 + 1] = ainv[(j * 3 + c) * 2 + 1];
        }
        for (int64_t l = 0; l < n; ++l) {
            if (l == j) continue;
            double complex t[6];
            interaction_tensor(k, (double)(coords[3 * j] - coords[3 * l]),
                               (double)(coords[3 * j + 1] - coords[3 * l + 1]),
                               (double)(coords[3 * j + 2] - coords[3 * l + 2]), t);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const int64_t row = a * n + j, col = b * n + l;
                    A[(row * N3 + col) * 2] = creal(t[comp_of[a][b]]);
                    A[(row * N3 + col) * 2 + 1] = cimag(t[comp_of[a][b]]);
                }
        }
    }
}

/*
 * Scattering cross section as the exact double sum over dipole pairs of the
 * power radiated by the dipole array (Draine 1988, cited in Sec. 1):
 *
 *   C_sca = 4 pi k [ (2/3) k^3 sum_j |P_j|^2 + sum_{j != l} P_j^H Im(G_jl) P_l ],
 *
 * where G_jl = -A_jl is the field at r_j of a unit dipole at r_l; the
 * j = l term is the limit Im G(0) = (2/3) k^3 I.  |E_0| = 1.
 */
double oracle_csca_double_sum(int64_t n, const int32_t* coords, double k, const double* P, int nthreads) {
    double total = 0.0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
#endif
    for (int64_t j = 0; j < n; ++j) {
        double complex pj[3];
        double self = 0.0;
        for (int c = 0; c < 3; ++c) {
            pj[c] = P[(c * n + j) * 2] + I * P[(c * n + j) * 2 + 1];
            self += creal(pj[c] * conj(pj[c]));
        }
        double sum = (2.0 / 3.0) * k * k * k * self;
        for (int64_t l = 0; l < n; ++l) {
            if (l == j) continue;
            double complex t[6];
            interaction_tensor(k, (double)(coords[3 * j] - coords[3 * l]),
                               (double)(coords[3 * j + 1] - coords[3 * l + 1]),
                               (double)(coords[3 * j + 2] - coords[3 * l + 2]), t);
            double complex pl[3];
            for (int c = 0; c < 3; ++c) pl[c] = P[(c * n + l) * 2] + I * P[(c * n + l) * 2 + 1];
            double complex s = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) s += conj(pj[a]) * (-cimag(t[comp_of[a][b]])) * pl[b];
            sum += creal(s);
        }
        total += sum;
    }
    return 4.0 * M_PI * k * total;
}
