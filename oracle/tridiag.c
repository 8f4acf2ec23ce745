/*
 * Oracle (test infrastructure only): dense Hermitian eigen-kernels in plain C, FP64.
 *
 * Nothing in the CUDA library links, includes or calls this file; only the test suite,
 * the benchmark's CPU-baseline leg and the smoke check load it (through oracle/direct.py).
 *
 *  - oracle_tridiag_qr: eigenvalues (and optionally eigenvectors) of a real symmetric
 *    tridiagonal matrix by the implicit symmetric QR step with Wilkinson shift and
 *    bulge chasing (Golub & Van Loan, Matrix Computations, sec. 8.3).  This is the
 *    tridiagonal stage of the direct dense solver that defines "the lowest nev
 *    eigenpairs of the pencil" (Section 1 and 2 of the paper: the direct solvers
 *    BXINV/MRRR that ChFSI is compared with).
 *  - oracle_jacobi_hermitian: cyclic Jacobi for a complex Hermitian matrix (an
 *    independent algorithm, used to cross-check the tridiagonal route on small n).
 *
 * Built with -ffp-contract=off so that results do not depend on FMA contraction.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

static double sign1(double x) { return x < 0.0 ? -1.0 : 1.0; }

/* d[0..n-1] diagonal, e[0..n-2] off-diagonal (T[i+1,i] = e[i]); both overwritten.
 * If z != NULL it is an n x n column-major real matrix (leading dimension ldz) whose
 * columns are multiplied by the accumulated rotations: pass the identity to get the
 * eigenvectors of T.  Eigenvalues are left unsorted in d.  Returns 0, or -1 when the
 * iteration limit (30 QR steps per eigenvalue on average) is exceeded. */
int oracle_tridiag_qr(int n, double *d, double *e, double *z, int ldz)
{
    if (n <= 1) return 0;
    long steps = 0, limit = 30L * n;
    int q = n - 1;
    while (q > 0) {
        /* deflate from the bottom */
        if (fabs(e[q - 1]) <= DBL_EPSILON * (fabs(d[q - 1]) + fabs(d[q]))) {
            e[q - 1] = 0.0;
            --q;
            continue;
        }
        /* start p of the unreduced block [p, q] */
        int p = q - 1;
        while (p > 0 && fabs(e[p - 1]) > DBL_EPSILON * (fabs(d[p - 1]) + fabs(d[p]))) --p;
        if (p > 0) e[p - 1] = 0.0;
        if (++steps > limit) return -1;

        /* Wilkinson shift from the trailing 2 x 2 block [[d[q-1], e[q-1]], [e[q-1], d[q]]] */
        double delta = 0.5 * (d[q - 1] - d[q]);
        double b = e[q - 1];
        double mu = d[q] - b * b / (delta + sign1(delta) * hypot(delta, b));

        /* implicit QR step: first rotation from the shifted first column, then chase */
        double x = d[p] - mu, y = e[p];
        for (int k = p; k < q; ++k) {
            double r = hypot(x, y);
            double c = 1.0, s = 0.0;
            if (r != 0.0) { c = x / r; s = y / r; }
            if (k > p) e[k - 1] = r;
            double ak = d[k], ak1 = d[k + 1], bk = e[k];
            d[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
            d[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
            e[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
            if (k + 1 < q) {
                x = e[k];
                y = s * e[k + 1];     /* bulge at (k+2, k) */
                e[k + 1] = c * e[k + 1];
            }
            if (z) {
                double *zk = z + (long)k * ldz, *zk1 = z + (long)(k + 1) * ldz;
                for (int i = 0; i < n; ++i) {
                    double u = zk[i], v = zk1[i];
                    zk[i] = c * u + s * v;
                    zk1[i] = -s * u + c * v;
                }
            }
        }
    }
    return 0;
}

/* a: n x n complex Hermitian, column-major, interleaved (re, im); overwritten (diagonalised).
 * v: n x n complex column-major output, the unitary whose columns are eigenvectors.
 * w: n eigenvalues (unsorted, w[i] belongs to column i of v).
 * Sweeps until the off-diagonal Frobenius norm is <= tol * ||A||_F.
 * Returns the number of sweeps, or -1 when max_sweeps did not suffice. */
int oracle_jacobi_hermitian(int n, double *a_ri, double *v_ri, double *w, double tol, int max_sweeps)
{
    double complex *a = (double complex *)a_ri, *v = (double complex *)v_ri;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) v[i + (long)j * n] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (long t = 0; t < (long)n * n; ++t) fro += creal(a[t] * conj(a[t]));
    fro = sqrt(fro);
    int sweep;
    for (sweep = 0; sweep <= max_sweeps; ++sweep) {
        double off = 0.0;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                if (i != j) off += creal(a[i + (long)j * n] * conj(a[i + (long)j * n]));
        if (sqrt(off) <= tol * fro) break;
        if (sweep == max_sweeps) return -1;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double complex apq = a[p + (long)q * n];
                double r = cabs(apq);
                if (r == 0.0) continue;
                double complex ph = apq / r;                   /* e^{i phi} */
                double app = creal(a[p + (long)p * n]), aqq = creal(a[q + (long)q * n]);
                double tau = (aqq - app) / (2.0 * r);
                double t = sign1(tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* U on (p, q): column p = (c, -s e^{-i phi}), column q = (s, c e^{-i phi}) */
                double complex upp = c, uqp = -s * conj(ph), upq = s, uqq = c * conj(ph);
                for (int i = 0; i < n; ++i) {          /* A <- A U, V <- V U */
                    double complex x = a[i + (long)p * n], y = a[i + (long)q * n];
                    a[i + (long)p * n] = x * upp + y * uqp;
                    a[i + (long)q * n] = x * upq + y * uqq;
                    x = v[i + (long)p * n]; y = v[i + (long)q * n];
                    v[i + (long)p * n] = x * upp + y * uqp;
                    v[i + (long)q * n] = x * upq + y * uqq;
                }
                for (int j = 0; j < n; ++j) {          /* A <- U^H A */
                    double complex x = a[p + (long)j * n], y = a[q + (long)j * n];
                    a[p + (long)j * n] = conj(upp) * x + conj(uqp) * y;
                    a[q + (long)j * n] = conj(upq) * x + conj(uqq) * y;
                }
                a[p + (long)q * n] = 0.0;
                a[q + (long)p * n] = 0.0;
                a[p + (long)p * n] = creal(a[p + (long)p * n]);
                a[q + (long)q * n] = creal(a[q + (long)q * n]);
            }
        }
    }
    for (int i = 0; i < n; ++i) w[i] = creal(a[i + (long)i * n]);
    return sweep;
}
