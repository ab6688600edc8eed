/*
 * mr3_oracle.c -- TEST INFRASTRUCTURE ONLY (never part of the product path).
 *
 * A plain, serial, obviously-correct FP64 CPU reference for the real symmetric
 * tridiagonal eigenproblem  T z = lambda z,  T = tridiag(e, d, e).  It computes
 * the eigen-decomposition by means independent of MRRR:
 *
 *   - Gershgorin interval            (App. B, Alg. "Gershgorin"; |beta_1| used, see below)
 *   - Sturm count on T               (App. B, Alg. "NegCount" on T and its remarks)
 *   - Bisection                      (Sec. 3.2.2, Alg. "Bisection")
 *   - inverse iteration with modified Gram-Schmidt inside absolute-gap chains
 *                                    (Sec. 2.3.1, "Bisection and inverse iteration")
 *   - cyclic Jacobi on a small dense symmetric matrix (textbook brute force, n <= 64)
 *
 * Readings of the paper taken here, where the printed algorithms are ambiguous or garbled:
 *   - Gershgorin: the first row's radius is |beta_1|; the printed algorithm writes
 *     beta_1 without the absolute value, which would be wrong for beta_1 < 0.
 *   - Bisection stop test: iterate while the width exceeds
 *     max(rtol * max(|lo|,|hi|), atol) (the printed test joins the two clauses with "or").
 *   - NegCount counts eigenvalues strictly below sigma; SignBit(-0) = 1 (App. B remarks).
 *   - A zero off-diagonal decouples the recurrence: the pivot restarts at alpha_i - sigma.
 *
 * Only tests/, the smoke check and the bench's CPU-baseline leg may load this file.
 * It shares no code with the CUDA library.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EPS (DBL_EPSILON * 0.5) /* unit roundoff 2^-53 */
#define ORC_SAFMIN DBL_MIN          /* underflow threshold omega */

/* ---------------------------------------------------------------- Gershgorin */
/* App. B, Alg. "Gershgorin": interval [gl, gu] containing every eigenvalue of T,
 * widened by (2n + 10) * bnorm * eps. */
void orc_gershgorin(int n, const double *d, const double *e, double *gl, double *gu)
{
    if (n <= 0) { *gl = 0.0; *gu = 0.0; return; }
    double lo, hi;
    if (n == 1) {
        lo = d[0];
        hi = d[0];
    } else {
        lo = d[0] - fabs(e[0]);
        hi = d[0] + fabs(e[0]);
        for (int i = 1; i < n - 1; i++) {
            double r = fabs(e[i - 1]) + fabs(e[i]);
            if (d[i] - r < lo) lo = d[i] - r;
            if (d[i] + r > hi) hi = d[i] + r;
        }
        double r = fabs(e[n - 2]);
        if (d[n - 1] - r < lo) lo = d[n - 1] - r;
        if (d[n - 1] + r > hi) hi = d[n - 1] + r;
    }
    double bnorm = fmax(fabs(lo), fabs(hi));
    *gl = lo - (2.0 * n + 10.0) * bnorm * ORC_EPS;
    *gu = hi + (2.0 * n + 10.0) * bnorm * ORC_EPS;
}

/* ---------------------------------------------------------------- NegCount(T) */
/* App. B, Alg. "NegCount" on T: number of eigenvalues of T strictly below sigma,
 * by the pivots of the LDL^T factorization of T - sigma I (Sylvester's law of
 * inertia, Sec. 3.2.2).  SignBit(-0) = 1, SignBit(+0) = 0. */
int orc_negcount(int n, const double *d, const double *e, double sigma)
{
    int count = 0;
    double piv = d[0] - sigma;
    count += signbit(piv) ? 1 : 0;
    for (int i = 1; i < n; i++) {
        double b = e[i - 1];
        if (b == 0.0)
            piv = d[i] - sigma;
        else
            piv = (d[i] - sigma) - (b * b) / piv;
        count += signbit(piv) ? 1 : 0;
    }
    return count;
}

/* Number of eigenvalues of T that are <= x, as n - NegCount(-T, -x): the
 * eigenvalues of -T below -x are the eigenvalues of T above x. */
int orc_count_le(int n, const double *d, const double *e, double x)
{
    int count = 0;
    double piv = -d[0] + x;
    count += signbit(piv) ? 1 : 0;
    for (int i = 1; i < n; i++) {
        double b = e[i - 1];
        if (b == 0.0)
            piv = -d[i] + x;
        else
            piv = (-d[i] + x) - (b * b) / piv;
        count += signbit(piv) ? 1 : 0;
    }
    return n - count;
}

/* ---------------------------------------------------------------- Bisection */
/* Sec. 3.2.2, Alg. "Bisection": shrink [lo, hi] with NegCount(T, lo) < k <=
 * NegCount(T, hi) until width <= max(rtol * max(|lo|,|hi|), atol).  The loop also
 * stops when the midpoint is no longer strictly inside the interval (no
 * representable point left) or after maxit halvings.  Returns the halvings done. */
int orc_bisect(int n, const double *d, const double *e, int k, double rtol, double atol,
               double *lo, double *hi, int maxit)
{
    double wl = *lo, wu = *hi;
    int it = 0;
    while (it < maxit) {
        double width = wu - wl;
        double tol = fmax(rtol * fmax(fabs(wl), fabs(wu)), atol);
        if (!(width > tol)) break;
        double w = wl + 0.5 * width;
        if (!(w > wl && w < wu)) break;
        if (orc_negcount(n, d, e, w) < k)
            wl = w;
        else
            wu = w;
        it++;
    }
    *lo = wl;
    *hi = wu;
    return it;
}

/* Eigenvalues il..iu (1-based, ascending) of T to full accuracy: bisection from the
 * Gershgorin interval with rtol = 2 eps and atol = 4 omega.  w[j] is the interval
 * midpoint, wlo/whi (may be NULL) the final interval. */
void orc_eigvals(int n, const double *d, const double *e, int il, int iu,
                 double *w, double *wlo, double *whi)
{
    double gl, gu;
    orc_gershgorin(n, d, e, &gl, &gu);
    for (int k = il; k <= iu; k++) {
        double lo = gl, hi = gu;
        orc_bisect(n, d, e, k, 2.0 * ORC_EPS, 4.0 * ORC_SAFMIN, &lo, &hi, 4096);
        w[k - il] = lo + 0.5 * (hi - lo);
        if (wlo) wlo[k - il] = lo;
        if (whi) whi[k - il] = hi;
    }
}

/* ---------------------------------------------------------------- SplitMix64 */
/* Counter-based SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): output for counter i
 * of stream seed.  Used only for the inverse-iteration start vectors. */
static uint64_t orc_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double orc_uniform_pm1(uint64_t seed, uint64_t i)
{
    return 2.0 * ((double)(orc_splitmix64(seed, i) >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

/* ---------------------------------------------------------------- inverse iteration */
/* Tridiagonal Gaussian elimination with partial pivoting of A = T - lambda I
 * (textbook).  U has a diagonal u0 and two superdiagonals u1, u2; mult[i] and
 * swap[i] record the elimination of row i+1.  Pivots smaller in magnitude than tiny
 * (eps ||T||_1) are replaced by +-tiny, keeping their sign, so the solve amplifies the
 * eigenvector direction instead of overflowing (e.g. a denormal pivot when lambda is an
 * eigenvalue next to zero). */
static void orc_tri_lu(int n, const double *d, const double *e, double lambda, double tiny,
                       double *u0, double *u1, double *u2, double *mult, int *swp)
{
    double r0 = d[0] - lambda;
    double r1 = n > 1 ? e[0] : 0.0;
    double r2 = 0.0;
    for (int i = 0; i < n - 1; i++) {
        double s0 = e[i];
        double s1 = d[i + 1] - lambda;
        double s2 = (i + 1 < n - 1) ? e[i + 1] : 0.0;
        if (fabs(s0) > fabs(r0)) {
            double t;
            t = r0; r0 = s0; s0 = t;
            t = r1; r1 = s1; s1 = t;
            t = r2; r2 = s2; s2 = t;
            swp[i] = 1;
        } else {
            swp[i] = 0;
        }
        if (fabs(r0) < tiny) r0 = (r0 < 0.0) ? -tiny : tiny;
        double m = s0 / r0;
        mult[i] = m;
        u0[i] = r0;
        u1[i] = r1;
        u2[i] = r2;
        r0 = s1 - m * r1;
        r1 = s2 - m * r2;
        r2 = 0.0;
    }
    if (fabs(r0) < tiny) r0 = (r0 < 0.0) ? -tiny : tiny;
    u0[n - 1] = r0;
    u1[n - 1] = 0.0;
    u2[n - 1] = 0.0;
}

static void orc_tri_solve(int n, const double *u0, const double *u1, const double *u2,
                          const double *mult, const int *swp, double *y)
{
    for (int i = 0; i < n - 1; i++) {
        if (swp[i]) { double t = y[i]; y[i] = y[i + 1]; y[i + 1] = t; }
        y[i + 1] -= mult[i] * y[i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = y[i];
        if (i + 1 < n) s -= u1[i] * y[i + 1];
        if (i + 2 < n) s -= u2[i] * y[i + 2];
        y[i] = s / u0[i];
    }
}

static double orc_nrm2(int n, const double *x)
{
    double scale = 0.0, ssq = 1.0;
    for (int i = 0; i < n; i++) {
        if (x[i] != 0.0) {
            double a = fabs(x[i]);
            if (scale < a) { ssq = 1.0 + ssq * (scale / a) * (scale / a); scale = a; }
            else ssq += (a / scale) * (a / scale);
        }
    }
    return scale * sqrt(ssq);
}

/* Output sign convention: the entry of largest magnitude is positive (ties go to
 * the lowest index). */
static void orc_fix_sign(int n, double *z)
{
    int imax = 0;
    double amax = -1.0;
    for (int i = 0; i < n; i++)
        if (fabs(z[i]) > amax) { amax = fabs(z[i]); imax = i; }
    if (z[imax] < 0.0)
        for (int i = 0; i < n; i++) z[i] = -z[i];
}

/* Sec. 2.3.1: inverse iteration for the m eigenvectors of the ascending
 * eigenvalue approximations w[0..m-1].  Consecutive eigenvalues whose gap is below
 * chain_tol * ||T||_1 form a chain; inside a chain each new vector is
 * re-orthogonalised (modified Gram-Schmidt) against the earlier chain vectors after
 * every solve.  Equal approximations inside a chain are separated by 10 eps |lambda|.
 * Each vector takes at most maxit solves; once the growth ||y|| of a solve with a
 * unit right-hand side exceeds 1 / (10 sqrt(n) eps ||T||_1) one more solve is done.
 * Z is column-major with leading dimension ldz.  work needs 5n doubles, iwork n ints.
 * Returns the number of vectors that never reached the growth threshold. */
int orc_inverse_iteration(int n, const double *d, const double *e, int m, const double *w,
                          double *Z, int ldz, uint64_t seed, double chain_tol, int maxit,
                          double *work, int *iwork)
{
    double *u0 = work, *u1 = work + n, *u2 = work + 2 * n, *mult = work + 3 * n;
    double *y = work + 4 * n;
    int *swp = iwork;
    int nfail = 0;
    double anorm = 0.0; /* ||T||_1 */
    for (int i = 0; i < n; i++) {
        double s = fabs(d[i]);
        if (i > 0) s += fabs(e[i - 1]);
        if (i < n - 1) s += fabs(e[i]);
        if (s > anorm) anorm = s;
    }
    if (anorm == 0.0) anorm = 1.0;
    double tiny = ORC_EPS * anorm;
    double growth_tol = 1.0 / (10.0 * sqrt((double)n) * ORC_EPS * anorm);
    int chain_start = 0;
    double lam_prev = 0.0;
    for (int j = 0; j < m; j++) {
        double lam = w[j];
        if (j > 0 && (w[j] - w[j - 1]) < chain_tol * anorm) {
            double pert = 10.0 * ORC_EPS * fabs(lam);
            if (lam < lam_prev + pert) lam = lam_prev + pert;
        } else {
            chain_start = j;
        }
        lam_prev = lam;
        double *z = Z + (size_t)j * ldz;
        if (n == 1) { z[0] = 1.0; continue; }
        orc_tri_lu(n, d, e, lam, tiny, u0, u1, u2, mult, swp);
        for (int i = 0; i < n; i++) y[i] = orc_uniform_pm1(seed, (uint64_t)j * (uint64_t)n + i);
        double nrm = orc_nrm2(n, y);
        for (int i = 0; i < n; i++) y[i] /= nrm;
        int converged = 0, extra_done = 0;
        for (int it = 0; it < maxit; it++) {
            orc_tri_solve(n, u0, u1, u2, mult, swp, y);
            double growth = orc_nrm2(n, y);
            /* modified Gram-Schmidt against earlier vectors of this chain */
            for (int p = chain_start; p < j; p++) {
                const double *zp = Z + (size_t)p * ldz;
                double dot = 0.0;
                for (int i = 0; i < n; i++) dot += zp[i] * y[i];
                for (int i = 0; i < n; i++) y[i] -= dot * zp[i];
            }
            nrm = orc_nrm2(n, y);
            if (!(nrm > 0.0) || !isfinite(nrm)) break;
            for (int i = 0; i < n; i++) y[i] /= nrm;
            if (converged) { extra_done = 1; break; }
            if (growth >= growth_tol) converged = 1;
        }
        if (!converged) nfail++;
        (void)extra_done;
        for (int i = 0; i < n; i++) z[i] = y[i];
        orc_fix_sign(n, z);
    }
    return nfail;
}

/* ---------------------------------------------------------------- cyclic Jacobi */
/* Textbook cyclic-by-row Jacobi for a dense symmetric n x n matrix A (row-major,
 * overwritten).  Rotation for pivot (p,q): theta = (a_qq - a_pp) / (2 a_pq),
 * t = sign(theta) / (|theta| + sqrt(1 + theta^2)), c = 1/sqrt(1+t^2), s = t c.
 * Sweeps until the off-diagonal Frobenius norm is below eps * ||A||_F / n or 100
 * sweeps.  On return w holds the ascending eigenvalues and V (row-major n x n) the
 * eigenvectors as columns, with the sign convention of orc_fix_sign.
 * Returns the number of sweeps. */
int orc_jacobi(int n, double *A, double *w, double *V)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int i = 0; i < n * n; i++) fro += A[i] * A[i];
    fro = sqrt(fro);
    int sweep;
    for (sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                if (i != j) off += A[i * n + j] * A[i * n + j];
        off = sqrt(off);
        if (off <= ORC_EPS * fro / (n > 0 ? n : 1) || off == 0.0) break;
        for (int p = 0; p < n - 1; p++) {
            for (int q = p + 1; q < n; q++) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double app = A[p * n + p], aqq = A[q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                /* A <- J^T A J with J the rotation in the (p,q) plane */
                for (int k = 0; k < n; k++) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < n; i++) w[i] = A[i * n + i];
    /* selection sort of the eigenvalues with their vectors (n is small) */
    for (int i = 0; i < n - 1; i++) {
        int kmin = i;
        for (int k = i + 1; k < n; k++)
            if (w[k] < w[kmin]) kmin = k;
        if (kmin != i) {
            double t = w[i]; w[i] = w[kmin]; w[kmin] = t;
            for (int r = 0; r < n; r++) {
                t = V[r * n + i]; V[r * n + i] = V[r * n + kmin]; V[r * n + kmin] = t;
            }
        }
    }
    /* sign convention on each column */
    for (int j = 0; j < n; j++) {
        int imax = 0;
        double amax = -1.0;
        for (int i = 0; i < n; i++)
            if (fabs(V[i * n + j]) > amax) { amax = fabs(V[i * n + j]); imax = i; }
        if (V[imax * n + j] < 0.0)
            for (int i = 0; i < n; i++) V[i * n + j] = -V[i * n + j];
    }
    return sweep;
}
