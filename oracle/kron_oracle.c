/*
 * kron_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the
 * mu-mode product, the Tucker operator and what they drive.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the CUDA library links, includes or
 * calls this file; it shares no code, header, table or helper with it.  Only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * Conventions (Appendix A, definition of vec): every tensor is stored
 * column-major, the first index running fastest; indices are 0-based here
 * (the paper is 1-based).  A matrix L of size n x m is stored column-major
 * with leading dimension ldL >= n, element (i, j) at L[i + ldL * j].
 *
 * Every function returns 0 on success and a negative number on bad input.
 * Parallelism: OpenMP over independent output fibres only; each output value
 * is still a single ascending-index FP64 sum, so results do not depend on the
 * thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 16

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int64_t prod_range(const int64_t *m, int lo, int hi)
{
    int64_t p = 1;
    for (int k = lo; k < hi; ++k) p *= m[k];
    return p;
}

/*
 * mu-mode product, Definition "mu-mode product" and Eq. (mmp):
 *     S^{(mu)} = op(L) T^{(mu)},
 * i.e. every mu-fibre of T is multiplied by op(L).  T has sizes m[0..d-1];
 * S has the same sizes except n in position mu (0-based).  op(L) = L
 * (n x m_mu, ld ldL) when transL == 0, and L^T where L is m_mu x n (ld ldL)
 * when transL != 0.
 *
 * Element form: S(p, i, q) = sum_j op(L)(i, j) T(p, j, q), with
 * p the linear index over modes before mu (P = prod_{k<mu} m_k) and q over
 * modes after mu (Q = prod_{k>mu} m_k); the index map is the vec map of
 * Appendix A, so T(p, j, q) sits at p + P*j + P*m_mu*q.
 */
int oracle_mump(int d, const int64_t *m, int mu, int64_t n, const double *T,
                const double *L, int64_t ldL, int transL, double *S)
{
    if (d < 1 || d > ORC_MAXD || mu < 0 || mu >= d || n < 0) return -1;
    const int64_t P = prod_range(m, 0, mu);
    const int64_t Q = prod_range(m, mu + 1, d);
    const int64_t mm = m[mu];
    if (!transL && ldL < (n > 1 ? n : 1)) return -2;
    if (transL && ldL < (mm > 1 ? mm : 1)) return -2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t q = 0; q < Q; ++q) {
        for (int64_t i = 0; i < n; ++i) {
            double *s = S + P * i + P * n * q;
            for (int64_t p = 0; p < P; ++p) s[p] = 0.0;
            for (int64_t j = 0; j < mm; ++j) {
                const double l = transL ? L[j + ldL * i] : L[i + ldL * j];
                const double *t = T + P * j + P * mm * q;
                for (int64_t p = 0; p < P; ++p) s[p] += l * t[p];
            }
        }
    }
    return 0;
}

/*
 * Tucker operator, Definition "Tucker operator" and Eq. (tuckerop):
 *     S = T x_1 op(L_1) x_2 op(L_2) ... x_d op(L_d),
 * evaluated as d consecutive mu-mode products in the order 1, 2, ..., d
 * (the order the definition writes; equivalent to summing Eq. (nestedmumode)
 * from the innermost index outwards).  n[mu] is the number of rows of
 * op(L_mu).  The two scratch tensors are allocated here (malloc).
 */
int oracle_tucker(int d, const int64_t *m, const int64_t *n, const double *T,
                  const double *const *L, const int64_t *ldL, int transL,
                  double *S)
{
    if (d < 1 || d > ORC_MAXD) return -1;
    int64_t cur[ORC_MAXD];
    int64_t maxel = 1;
    for (int k = 0; k < d; ++k) cur[k] = m[k];
    for (int mu = 0; mu < d; ++mu) {
        cur[mu] = n[mu];
        int64_t e = prod_range(cur, 0, d);
        if (e > maxel) maxel = e;
    }
    for (int k = 0; k < d; ++k) cur[k] = m[k];
    double *buf[2];
    buf[0] = (double *)malloc(sizeof(double) * (size_t)(maxel > 0 ? maxel : 1));
    buf[1] = (double *)malloc(sizeof(double) * (size_t)(maxel > 0 ? maxel : 1));
    if (!buf[0] || !buf[1]) { free(buf[0]); free(buf[1]); return -3; }
    const double *src = T;
    int rc = 0;
    for (int mu = 0; mu < d && rc == 0; ++mu) {
        double *dst = (mu == d - 1) ? S : buf[mu & 1];
        rc = oracle_mump(d, cur, mu, n[mu], src, L[mu], ldL[mu], transL, dst);
        cur[mu] = n[mu];
        src = dst;
    }
    free(buf[0]);
    free(buf[1]);
    return rc;
}

/*
 * Brute-force element-wise formula, Eq. (nestedmumode):
 *     s_{i_1..i_d} = sum_{j_d} ... sum_{j_1} t_{j_1..j_d} prod_mu l^mu_{i_mu j_mu}.
 * Cost prod(n) * prod(m) * d: tiny inputs only.  transL as in oracle_mump.
 */
int oracle_tucker_nested(int d, const int64_t *m, const int64_t *n,
                         const double *T, const double *const *L,
                         const int64_t *ldL, int transL, double *S)
{
    if (d < 1 || d > ORC_MAXD) return -1;
    const int64_t NO = prod_range(n, 0, d), NI = prod_range(m, 0, d);
    for (int64_t io = 0; io < NO; ++io) {
        int64_t iv[ORC_MAXD];
        int64_t r = io;
        for (int k = 0; k < d; ++k) { iv[k] = r % n[k]; r /= n[k]; }
        double s = 0.0;
        for (int64_t ji = 0; ji < NI; ++ji) {
            int64_t jv[ORC_MAXD];
            int64_t rr = ji;
            for (int k = 0; k < d; ++k) { jv[k] = rr % m[k]; rr /= m[k]; }
            double pr = T[ji];
            for (int k = 0; k < d; ++k)
                pr *= transL ? L[k][jv[k] + ldL[k] * iv[k]]
                             : L[k][iv[k] + ldL[k] * jv[k]];
            s += pr;
        }
        S[io] = s;
    }
    return 0;
}

/*
 * Kronecker product, Appendix A: for A (ra x ca) and B (rb x cb), both dense
 * column-major, C = A (x) B is (ra rb) x (ca cb) with
 *     C(ia*rb + ib, ja*cb + jb) = a_{ia ja} b_{ib jb}.
 */
int oracle_kron(int64_t ra, int64_t ca, const double *A, int64_t rb,
                int64_t cb, const double *B, double *C)
{
    const int64_t rc = ra * rb;
    for (int64_t ja = 0; ja < ca; ++ja)
        for (int64_t jb = 0; jb < cb; ++jb)
            for (int64_t ia = 0; ia < ra; ++ia)
                for (int64_t ib = 0; ib < rb; ++ib)
                    C[(ia * rb + ib) + rc * (ja * cb + jb)] =
                        A[ia + ra * ja] * B[ib + rb * jb];
    return 0;
}

/* y = A x, A dense r x c column-major: a plain matrix-vector product. */
int oracle_matvec(int64_t r, int64_t c, const double *A, const double *x,
                  double *y)
{
    for (int64_t i = 0; i < r; ++i) y[i] = 0.0;
    for (int64_t j = 0; j < c; ++j)
        for (int64_t i = 0; i < r; ++i) y[i] += A[i + r * j] * x[j];
    return 0;
}

/*
 * Adjoint of the Tucker operator.  Forward: X_1 = T, X_{mu+1} = X_mu x_mu L_mu,
 * S = X_{d+1}.  With the cotangent dS of S:
 *   - the transpose of (L_d (x) ... (x) L_1) is L_d^T (x) ... (x) L_1^T
 *     (Appendix A, property 5, with Lemma "krontomu"), so the pulled-back
 *     cotangents are G_{d+1} = dS, G_mu = G_{mu+1} x_mu L_mu^T, and dT = G_1;
 *   - from Eq. (mmp), Z^{(mu)} = L_mu X_mu^{(mu)} for Z = X_{mu+1}, hence
 *     dL_mu = G_{mu+1}^{(mu)} (X_mu^{(mu)})^T, a sum over every index but mu.
 * All X_mu are stored (no recomputation).  L_mu is n_mu x m_mu with ld ldL.
 * dT (size prod m) and dL[mu] (n_mu x m_mu, ld n_mu) may be NULL to skip.
 */
int oracle_tucker_adjoint(int d, const int64_t *m, const int64_t *n,
                          const double *T, const double *const *L,
                          const int64_t *ldL, const double *dS, double *dT,
                          double *const *dL)
{
    if (d < 1 || d > ORC_MAXD) return -1;
    double *X[ORC_MAXD + 1];
    int64_t dims[ORC_MAXD + 1][ORC_MAXD];
    for (int k = 0; k < d; ++k) dims[0][k] = m[k];
    X[0] = (double *)T;
    for (int mu = 0; mu < d; ++mu) {
        for (int k = 0; k < d; ++k) dims[mu + 1][k] = dims[mu][k];
        dims[mu + 1][mu] = n[mu];
        X[mu + 1] = (double *)malloc(sizeof(double) *
                                     (size_t)prod_range(dims[mu + 1], 0, d));
        oracle_mump(d, dims[mu], mu, n[mu], X[mu], L[mu], ldL[mu], 0, X[mu + 1]);
    }
    /* G holds the cotangent of X_{mu+1}; start from dS. */
    double *G = (double *)malloc(sizeof(double) * (size_t)prod_range(n, 0, d));
    memcpy(G, dS, sizeof(double) * (size_t)prod_range(n, 0, d));
    for (int mu = d - 1; mu >= 0; --mu) {
        const int64_t P = prod_range(dims[mu], 0, mu);
        const int64_t Q = prod_range(dims[mu], mu + 1, d);
        const int64_t nm = n[mu], mm = m[mu];
        if (dL && dL[mu]) {
            double *g = dL[mu];
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t j = 0; j < mm; ++j)
                for (int64_t i = 0; i < nm; ++i) {
                    double s = 0.0;
                    for (int64_t q = 0; q < Q; ++q)
                        for (int64_t p = 0; p < P; ++p)
                            s += G[p + P * i + P * nm * q] *
                                 X[mu][p + P * j + P * mm * q];
                    g[i + nm * j] = s;
                }
        }
        /* G_mu = G_{mu+1} x_mu L_mu^T: dims of G_mu are dims[mu]. */
        double *Gn = (double *)malloc(sizeof(double) *
                                      (size_t)prod_range(dims[mu], 0, d));
        int64_t gd[ORC_MAXD];
        for (int k = 0; k < d; ++k) gd[k] = dims[mu + 1][k];
        oracle_mump(d, gd, mu, mm, G, L[mu], ldL[mu], 1, Gn);
        free(G);
        G = Gn;
    }
    if (dT) memcpy(dT, G, sizeof(double) * (size_t)prod_range(m, 0, d));
    free(G);
    for (int mu = 1; mu <= d; ++mu) free(X[mu]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Matrix exponentials (Section "Action of the matrix exponential").         */
/* Both are long double and neither uses the GPU's Pade method.              */
/* ------------------------------------------------------------------------ */

/*
 * exp(t A) for the tridiagonal Toeplitz A = tridiag(a, b, c) of size n
 * (a on the sub-diagonal, b on the diagonal, c on the super-diagonal),
 * a c > 0.  Textbook closed form: with r = sqrt(a / c) and
 * D = diag(r^1, ..., r^n), D^{-1} A D is symmetric tridiagonal with
 * off-diagonal g = sign(a) sqrt(a c), whose eigenpairs are
 *     lambda_k = b + 2 g cos(k pi / (n + 1)),
 *     v_k(j)   = sqrt(2 / (n + 1)) sin(j k pi / (n + 1)),   j, k = 1..n,
 * so exp(t A)(i, j) = r^{i-j} sum_k v_k(i) exp(t lambda_k) v_k(j).
 * Output E dense n x n column-major (ld n), rounded to double.
 */
int oracle_expm_tridiag_toeplitz(int64_t n, double a, double b, double c,
                                 double t, double *E)
{
    if (n < 1 || !(a * c > 0)) return -1;
    const long double pi = 3.141592653589793238462643383279502884L;
    const long double np1 = (long double)(n + 1);
    const long double g = (a > 0 ? 1.0L : -1.0L) * sqrtl((long double)a * (long double)c);
    const long double lr = 0.5L * logl((long double)a / (long double)c);
    long double *ex = (long double *)malloc(sizeof(long double) * (size_t)n);
    long double *V = (long double *)malloc(sizeof(long double) * (size_t)(n * n));
    if (!ex || !V) { free(ex); free(V); return -3; }
    const long double sc = sqrtl(2.0L / np1);
    for (int64_t k = 1; k <= n; ++k) {
        const long double lam = (long double)b + 2.0L * g * cosl((long double)k * pi / np1);
        ex[k - 1] = expl((long double)t * lam);
        for (int64_t j = 1; j <= n; ++j)
            V[(j - 1) + n * (k - 1)] = sc * sinl((long double)((j * k) % (2 * (n + 1))) * pi / np1);
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
            long double s = 0.0L;
            for (int64_t k = 0; k < n; ++k) s += V[i + n * k] * ex[k] * V[j + n * k];
            E[i + n * j] = (double)(expl(lr * (long double)(i - j)) * s);
        }
    free(ex);
    free(V);
    return 0;
}

/*
 * exp(t A) for a small dense A (n x n, ld n) by the Taylor series with
 * scaling and squaring, all in long double: choose s with
 * ||t A||_1 / 2^s <= 1/2, sum the series of B = t A / 2^s until a term is
 * below 1e-30 of the partial sum (1-norm), then square s times.
 */
int oracle_expm_taylor(int64_t n, const double *A, double t, double *E)
{
    if (n < 1) return -1;
    const size_t nn = (size_t)(n * n);
    long double *B = (long double *)malloc(sizeof(long double) * nn);
    long double *S = (long double *)malloc(sizeof(long double) * nn);
    long double *Tm = (long double *)malloc(sizeof(long double) * nn);
    long double *W = (long double *)malloc(sizeof(long double) * nn);
    if (!B || !S || !Tm || !W) { free(B); free(S); free(Tm); free(W); return -3; }
    long double nrm = 0.0L;
    for (int64_t j = 0; j < n; ++j) {
        long double cs = 0.0L;
        for (int64_t i = 0; i < n; ++i) cs += fabsl((long double)t * A[i + n * j]);
        if (cs > nrm) nrm = cs;
    }
    int s = 0;
    while (nrm > 0.5L) { nrm *= 0.5L; ++s; }
    const long double scale = ldexpl(1.0L, -s);
    for (size_t e = 0; e < nn; ++e) B[e] = (long double)t * A[e] * scale;
    for (size_t e = 0; e < nn; ++e) { S[e] = 0.0L; Tm[e] = 0.0L; }
    for (int64_t i = 0; i < n; ++i) { S[i + n * i] = 1.0L; Tm[i + n * i] = 1.0L; }
    for (int k = 1; k < 200; ++k) {
        /* Tm <- Tm * B / k */
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) {
                long double acc = 0.0L;
                for (int64_t l = 0; l < n; ++l) acc += Tm[i + n * l] * B[l + n * j];
                W[i + n * j] = acc / (long double)k;
            }
        long double tn = 0.0L, sn = 0.0L;
        for (size_t e = 0; e < nn; ++e) {
            Tm[e] = W[e];
            S[e] += W[e];
            tn += fabsl(W[e]);
            sn += fabsl(S[e]);
        }
        if (tn <= 1e-30L * sn) break;
    }
    for (int r = 0; r < s; ++r) {
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) {
                long double acc = 0.0L;
                for (int64_t l = 0; l < n; ++l) acc += S[i + n * l] * S[l + n * j];
                W[i + n * j] = acc;
            }
        memcpy(S, W, sizeof(long double) * nn);
    }
    for (size_t e = 0; e < nn; ++e) E[e] = (double)S[e];
    free(B); free(S); free(Tm); free(W);
    return 0;
}

/*
 * Stepping with the exponential of a Kronecker sum, Eqs. (expmat) and
 * (exptucker): one step maps U to U x_1 E_1 x_2 ... x_d E_d with
 * E_mu = exp(tau A_mu) given (n_mu x n_mu, ld n_mu).  Applies nsteps such
 * steps to U (sizes n[0..d-1]) in place, each step a plain Tucker operator.
 */
int oracle_expkronsum_steps(int d, const int64_t *n, const double *const *E,
                            int nsteps, double *U)
{
    if (d < 1 || d > ORC_MAXD || nsteps < 0) return -1;
    int64_t ld[ORC_MAXD];
    for (int k = 0; k < d; ++k) ld[k] = n[k];
    const int64_t N = prod_range(n, 0, d);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    if (!tmp) return -3;
    for (int s = 0; s < nsteps; ++s) {
        int rc = oracle_tucker(d, n, n, U, E, ld, 0, tmp);
        if (rc) { free(tmp); return rc; }
        memcpy(U, tmp, sizeof(double) * (size_t)N);
    }
    free(tmp);
    return 0;
}

/*
 * Action of a Kronecker sum, Eq. (actkron):
 *     (L_d (+) ... (+) L_1) vec(V) = vec( sum_mu V x_mu L_mu ),
 * with square L_mu (n_mu x n_mu, ld ldL[mu]).  Each term is a plain
 * mu-mode product; the terms are summed in the order mu = 1..d.
 */
int oracle_kronsumv(int d, const int64_t *n, const double *V,
                    const double *const *L, const int64_t *ldL, double *S)
{
    if (d < 1 || d > ORC_MAXD) return -1;
    const int64_t N = prod_range(n, 0, d);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    if (!tmp) return -3;
    for (int64_t e = 0; e < N; ++e) S[e] = 0.0;
    for (int mu = 0; mu < d; ++mu) {
        oracle_mump(d, n, mu, n[mu], V, L[mu], ldL[mu], 0, tmp);
        for (int64_t e = 0; e < N; ++e) S[e] += tmp[e];
    }
    free(tmp);
    return 0;
}
