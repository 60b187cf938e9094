/*
 * CPU oracle for blocked LU with partial pivoting (arXiv 1804.07017).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously-correct
 * statement of what the GPU library computes.  It is used by tests/, by
 * __graft_entry__.smoke() and by the cpu_baseline leg of bench.py, and by
 * nothing else.  It shares no code, header, table or helper with the CUDA
 * library under paper_1804_07017_gb300/.
 *
 * Precision: FP64 throughout (the paper's experiments are all in double
 * precision real arithmetic, Sec. 6.1).  Compile with -ffp-contract=off so
 * that every a - l*u is a rounded multiply followed by a rounded subtract on
 * every host architecture.
 *
 * Storage: column-major, element (i, j) of an m x n matrix at A[i + j*lda].
 * Pivots: LAPACK getrf convention, ipiv[j] = 1-based row swapped with row j+1
 * at step j (sequential interchanges).
 *
 * What each routine follows:
 *   oracle_getrf   -- LU_unb of algorithm LU_blk (RL1, Sec. 3): the unblocked
 *                     right-looking elimination with partial pivoting.  The
 *                     blocked algorithm (RL1-RL3) and the look-ahead variant
 *                     (Sec. 4, Listing 5) re-order exactly these operations,
 *                     so in exact arithmetic they produce these factors.
 *   oracle_laswp   -- the row permutation ("laswp") of the netlib getrf
 *                     decomposition used as MTB-LU (Sec. 3.4).
 *   oracle_trsm_lower_unit -- RL2, A12 := trilu(A11)^{-1} A12.
 *   oracle_gemm_update     -- RL3, A22 := A22 - A21 A12.
 *   oracle_getrs   -- forward/backward substitution with the factors (the
 *                     solve step; not in the paper, it is the getrs that pairs
 *                     with getrf).
 *   oracle_residual_inf / oracle_norm_inf -- the normwise backward error of a
 *                     solve, eta = ||b - A x|| / (||A|| ||x|| + ||b||) (inf-norms),
 *                     with compensated (Neumaier) sums so the residual is
 *                     accurate to ~1 ulp of its terms.
 *   oracle_potrf   -- Cholesky A = L L^T of a symmetric positive definite
 *                     matrix by the unblocked right-looking algorithm, the
 *                     factorization the paper names as fitting the same
 *                     blocked/look-ahead skeleton (Sec. 1, Sec. 7); lower
 *                     triangle only.
 *   oracle_chol_error -- ||A0 - L L^T|| / (n ||A0||) (inf-norms, compensated).
 *   oracle_geqr2   -- QR factorization A = Q R by Householder reflectors, the
 *                     unblocked form of the geqrf the paper's QR experiments
 *                     reorganise with look-ahead (Sec. 6): reflector j maps the
 *                     updated column j onto beta e_j, beta = -sign(a_jj) ||x||,
 *                     and is applied to the columns to its right.
 *   oracle_round_bf16 / oracle_round_fp16 / oracle_quant_e4m3 -- IEEE-style
 *                     round-to-nearest-even onto the narrow formats used for
 *                     the mixed-precision trailing update operands.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, ld) ((int64_t)(i) + (int64_t)(j) * (int64_t)(ld))

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Unblocked right-looking LU with partial pivoting of an m x n matrix
 * (RL1, LU_unb).  For j = 0 .. min(m,n)-1:
 *   p  = smallest i >= j maximising |A(i,j)|   (first maximum wins; NaN
 *        candidates are never chosen, and p = j when all of them are NaN)
 *   ipiv[j] = p + 1
 *   if A(p,j) == 0: record info = j+1 (first only), skip scaling and update
 *   swap whole rows j and p (all n columns)
 *   A(i,j) := A(i,j) / A(j,j)            for i > j      (a true division)
 *   A(i,c) := A(i,c) - A(i,j) * A(j,c)   for i > j, c > j
 * gap[j] (if non-NULL) = (|first| - |second|) / |first| over the candidates
 * of column j (1 when there is a single candidate, 0 when the column is zero).
 * Only the column loop of the rank-1 update is split across threads; every
 * element still sees the same operation sequence, so results do not depend on
 * the thread count.
 * Returns info: 0, or the 1-based index of the first exactly-zero pivot.
 * oracle_getrf_steps stops after the first `steps` elimination steps (all of
 * them when steps < 0): the leading part of the same computation, used to
 * time a bounded sample of a large factorization.
 */
int oracle_getrf_steps(int64_t m, int64_t n, double *A, int64_t lda, int32_t *ipiv,
                       double *gap, int nthreads, int64_t steps)
{
    int info = 0;
    int64_t kmax = m < n ? m : n;
    if (steps >= 0 && steps < kmax) kmax = steps;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = omp_get_max_threads();
#else
    (void)nthreads;
#endif
    for (int64_t j = 0; j < kmax; ++j) {
        /* NaN is unordered, so it maximises nothing: it is skipped, and a
         * column whose every candidate is NaN keeps its diagonal position. */
        int64_t p = -1;
        double best = 0.0;
        for (int64_t i = j; i < m; ++i) {
            double v = fabs(A[IDX(i, j, lda)]);
            if (isnan(v)) continue;
            if (p < 0 || v > best) { best = v; p = i; }
        }
        if (p < 0) p = j;
        if (gap) {
            double second = -1.0;
            for (int64_t i = j; i < m; ++i) {
                if (i == p) continue;
                double v = fabs(A[IDX(i, j, lda)]);
                if (v > second) second = v;
            }
            if (best == 0.0) gap[j] = 0.0;
            else if (second < 0.0) gap[j] = 1.0;
            else gap[j] = (best - second) / best;
        }
        ipiv[j] = (int32_t)(p + 1);
        if (A[IDX(p, j, lda)] == 0.0) {
            if (info == 0) info = (int)(j + 1);
            continue;
        }
        if (p != j) {
            for (int64_t c = 0; c < n; ++c) {
                double t = A[IDX(j, c, lda)];
                A[IDX(j, c, lda)] = A[IDX(p, c, lda)];
                A[IDX(p, c, lda)] = t;
            }
        }
        double piv = A[IDX(j, j, lda)];
        for (int64_t i = j + 1; i < m; ++i)
            A[IDX(i, j, lda)] = A[IDX(i, j, lda)] / piv;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static) if ((n - j) * (m - j) > 65536)
#endif
        for (int64_t c = j + 1; c < n; ++c) {
            double u = A[IDX(j, c, lda)];
            double *col = A + IDX(0, c, lda);
            const double *l = A + IDX(0, j, lda);
            for (int64_t i = j + 1; i < m; ++i) {
                double prod = l[i] * u;
                col[i] = col[i] - prod;
            }
        }
    }
    return info;
}

int oracle_getrf(int64_t m, int64_t n, double *A, int64_t lda, int32_t *ipiv,
                 double *gap, int nthreads)
{
    return oracle_getrf_steps(m, n, A, lda, ipiv, gap, nthreads, -1);
}

/*
 * Apply the sequential row interchanges ipiv[k1], ..., ipiv[k2-1] (1-based row
 * numbers) to columns 0 .. ncols-1 of A: for k = k1 .. k2-1 swap rows k and
 * ipiv[k]-1.
 */
void oracle_laswp(int64_t ncols, double *A, int64_t lda, int64_t k1, int64_t k2,
                  const int32_t *ipiv)
{
    for (int64_t k = k1; k < k2; ++k) {
        int64_t p = (int64_t)ipiv[k] - 1;
        if (p == k) continue;
        for (int64_t c = 0; c < ncols; ++c) {
            double t = A[IDX(k, c, lda)];
            A[IDX(k, c, lda)] = A[IDX(p, c, lda)];
            A[IDX(p, c, lda)] = t;
        }
    }
}

/* B := L^{-1} B with L the unit lower triangle of the m x m matrix at L (RL2). */
void oracle_trsm_lower_unit(int64_t m, int64_t n, const double *L, int64_t ldl,
                            double *B, int64_t ldb)
{
    for (int64_t c = 0; c < n; ++c) {
        double *b = B + IDX(0, c, ldb);
        for (int64_t j = 0; j < m; ++j) {
            double bj = b[j];
            for (int64_t i = j + 1; i < m; ++i) {
                double prod = L[IDX(i, j, ldl)] * bj;
                b[i] = b[i] - prod;
            }
        }
    }
}

/* B := U^{-1} B with U the upper triangle (with its diagonal) of the m x m matrix at U. */
void oracle_trsm_upper(int64_t m, int64_t n, const double *U, int64_t ldu,
                       double *B, int64_t ldb)
{
    for (int64_t c = 0; c < n; ++c) {
        double *b = B + IDX(0, c, ldb);
        for (int64_t j = m - 1; j >= 0; --j) {
            b[j] = b[j] / U[IDX(j, j, ldu)];
            double bj = b[j];
            for (int64_t i = 0; i < j; ++i) {
                double prod = U[IDX(i, j, ldu)] * bj;
                b[i] = b[i] - prod;
            }
        }
    }
}

/* C := C - A B, A m x k, B k x n, C m x n (RL3); plain triple loop, k innermost-last. */
void oracle_gemm_update(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                        const double *B, int64_t ldb, double *C, int64_t ldc)
{
    for (int64_t c = 0; c < n; ++c)
        for (int64_t p = 0; p < k; ++p) {
            double b = B[IDX(p, c, ldb)];
            for (int64_t i = 0; i < m; ++i) {
                double prod = A[IDX(i, p, lda)] * b;
                C[IDX(i, c, ldc)] = C[IDX(i, c, ldc)] - prod;
            }
        }
}

/*
 * Solve A X = B given the getrf factors of A (LU, ipiv): apply the
 * interchanges to B, then B := L^{-1} B (unit lower), then B := U^{-1} B.
 */
void oracle_getrs(int64_t n, int64_t nrhs, const double *LU, int64_t lda,
                  const int32_t *ipiv, double *B, int64_t ldb)
{
    oracle_laswp(nrhs, B, ldb, 0, n, ipiv);
    oracle_trsm_lower_unit(n, nrhs, LU, lda, B, ldb);
    oracle_trsm_upper(n, nrhs, LU, lda, B, ldb);
}

/* Neumaier compensated accumulation of one term. */
static inline void neumaier_add(double *s, double *c, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
    else *c += (v - t) + *s;
    *s = t;
}

/* ||A||_inf of an m x n matrix: max over rows of the sum of |a_ij|. */
double oracle_norm_inf(int64_t m, int64_t n, const double *A, int64_t lda)
{
    double best = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0, c = 0.0;
        for (int64_t j = 0; j < n; ++j) neumaier_add(&s, &c, fabs(A[IDX(i, j, lda)]));
        double r = s + c;
        if (r > best || isnan(r)) best = r;
    }
    return best;
}

/*
 * R := B - A X for an n x n A and n x nrhs X, B (compensated row sums).
 * Returns max over columns c of
 *   ||R(:,c)||_inf / (||A||_inf ||X(:,c)||_inf + ||B(:,c)||_inf),
 * the normwise backward error of each solve.  R may be NULL.
 */
double oracle_backward_error(int64_t n, int64_t nrhs, const double *A, int64_t lda,
                             const double *X, int64_t ldx, const double *B, int64_t ldb,
                             double *R, int64_t ldr)
{
    double anorm = oracle_norm_inf(n, n, A, lda);
    double worst = 0.0;
    for (int64_t c = 0; c < nrhs; ++c) {
        double rmax = 0.0, xmax = 0.0, bmax = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double s = B[IDX(i, c, ldb)], comp = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                /* exact product split is not needed: the product is rounded once,
                 * the compensated sum then keeps the total accurate. */
                neumaier_add(&s, &comp, -(A[IDX(i, j, lda)] * X[IDX(j, c, ldx)]));
            }
            double r = s + comp;
            if (R) R[IDX(i, c, ldr)] = r;
            if (fabs(r) > rmax || isnan(r)) rmax = fabs(r);
            if (fabs(X[IDX(i, c, ldx)]) > xmax) xmax = fabs(X[IDX(i, c, ldx)]);
            if (fabs(B[IDX(i, c, ldb)]) > bmax) bmax = fabs(B[IDX(i, c, ldb)]);
        }
        double denom = anorm * xmax + bmax;
        double eta = denom > 0.0 ? rmax / denom : (rmax > 0.0 ? INFINITY : 0.0);
        if (eta > worst || isnan(eta)) worst = eta;
    }
    return worst;
}

/*
 * Factorization backward error ||P A - L U||_inf / (n ||A||_inf) of the getrf
 * output LU/ipiv against the original square matrix A0 (n x n).  The product
 * L U is formed with compensated sums.
 */
double oracle_factor_error(int64_t n, const double *A0, int64_t lda0, const double *LU,
                           int64_t lda, const int32_t *ipiv)
{
    /* PA: apply interchanges to a copy of A0 row indices. */
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = (int64_t)ipiv[k] - 1;
        int64_t t = perm[k]; perm[k] = perm[p]; perm[p] = t;
    }
    double worst = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s_row = 0.0, c_row = 0.0;
        for (int64_t c = 0; c < n; ++c) {
            /* (L U)(i,c) = sum_{p <= min(i,c)} L(i,p) U(p,c), L(i,i) = 1 */
            double s = 0.0, comp = 0.0;
            int64_t pmax = i < c ? i : c;
            for (int64_t p = 0; p <= pmax; ++p) {
                double l = (p == i) ? 1.0 : LU[IDX(i, p, lda)];
                neumaier_add(&s, &comp, l * LU[IDX(p, c, lda)]);
            }
            neumaier_add(&s, &comp, -A0[IDX(perm[i], c, lda0)]);
            neumaier_add(&s_row, &c_row, fabs(s + comp));
        }
        double r = s_row + c_row;
        if (r > worst || isnan(r)) worst = r;
    }
    free(perm);
    double anorm = oracle_norm_inf(n, n, A0, lda0);
    if (n == 0) return 0.0;
    return anorm > 0.0 ? worst / ((double)n * anorm) : (worst > 0.0 ? INFINITY : 0.0);
}

/* ---------------------------------------------------------------------------
 * Narrow-format rounding (round to nearest, ties to even), stated from the
 * formats' definitions:
 *   bf16: 1 sign, 8 exponent (bias 127), 7 fraction bits; inf/nan kept.
 *   fp16: 1 sign, 5 exponent (bias 15), 10 fraction bits; subnormals down to
 *         2^-24; values whose rounded magnitude exceeds 65504 become inf.
 *   e4m3 (the "fn" variant): 1 sign, 4 exponent (bias 7), 3 fraction bits,
 *         no infinities, max finite 448, subnormals down to 2^-9; here values
 *         beyond 448 saturate to +-448 (the quantiser always scales first so
 *         this only guards rounding at the top binade).
 * All three are computed with frexp/ldexp and an explicit ties-to-even rule on
 * the scaled significand, independent of any hardware conversion.
 * ------------------------------------------------------------------------- */

/* Round x to a binary format with `mant` fraction bits, minimum normal
 * exponent emin (value 2^emin), without overflow handling. */
static double round_to_format(double x, int mant, int emin)
{
    if (x == 0.0 || isnan(x) || isinf(x)) return x;
    int e;
    double f = frexp(fabs(x), &e); /* |x| = f * 2^e, f in [0.5, 1) */
    int exp_unbiased = e - 1;      /* |x| = (2f) * 2^(e-1), 2f in [1,2) */
    if (exp_unbiased < emin) exp_unbiased = emin; /* subnormal spacing */
    /* quantum = 2^(exp_unbiased - mant) */
    double scaled = ldexp(fabs(x), mant - exp_unbiased); /* exact */
    double fl = floor(scaled);
    double rem = scaled - fl;
    double q;
    if (rem > 0.5) q = fl + 1.0;
    else if (rem < 0.5) q = fl;
    else q = (fmod(fl, 2.0) == 0.0) ? fl : fl + 1.0;
    double r = ldexp(q, exp_unbiased - mant);
    return x < 0 ? -r : r;
}

void oracle_round_bf16(int64_t count, const double *in, double *out)
{
    /* bf16 max finite = (2 - 2^-7) * 2^127; beyond the halfway point -> inf */
    const double maxf = ldexp(2.0 - ldexp(1.0, -7), 127);
    for (int64_t i = 0; i < count; ++i) {
        double r = round_to_format(in[i], 7, -126);
        if (fabs(r) > maxf && !isinf(r) && !isnan(r)) r = r > 0 ? INFINITY : -INFINITY;
        out[i] = r;
    }
}

void oracle_round_fp16(int64_t count, const double *in, double *out)
{
    for (int64_t i = 0; i < count; ++i) {
        double r = round_to_format(in[i], 10, -14);
        if (fabs(r) > 65504.0 && !isinf(r) && !isnan(r)) r = r > 0 ? INFINITY : -INFINITY;
        out[i] = r;
    }
}

void oracle_round_e4m3(int64_t count, const double *in, double *out)
{
    for (int64_t i = 0; i < count; ++i) {
        double r = round_to_format(in[i], 3, -6);
        if (fabs(r) > 448.0 && !isnan(r)) r = r > 0 ? 448.0 : -448.0;
        out[i] = r;
    }
}

/* Round x (already an FP32-representable or any double) to FP32 by the same
 * ties-to-even rule (24-bit significand, subnormals to 2^-149). */
void oracle_round_fp32(int64_t count, const double *in, double *out)
{
    const double maxf = ldexp(2.0 - ldexp(1.0, -23), 127);
    for (int64_t i = 0; i < count; ++i) {
        double r = round_to_format(in[i], 23, -126);
        if (fabs(r) > maxf && !isinf(r) && !isnan(r)) r = r > 0 ? INFINITY : -INFINITY;
        out[i] = r;
    }
}

/*
 * Power-of-two block scaling onto e4m3 for the FP8 trailing update.  Each
 * block (one row of the L21 operand, or one column of the U12 operand) gets
 * the scale 2^e with e the smallest integer such that amax / 2^e <= 448, the
 * largest finite e4m3 value: with amax = f 2^x, f in [0.5, 1), and
 * 448 = 0.875 2^9, e = x - 9 + (f > 0.875).  A block of zeros gets e = 0.
 * The stored value is e4m3(v / 2^e) (ties to even, saturating), so
 * q * 2^e is the dequantised operand.  The exponent is an exact integer
 * decision taken from the block's maximum, identical in any precision that
 * represents amax exactly.
 *   X: nblk blocks of len values; block b starts at X + b*bstride, its
 *      elements are estride apart.  Q: same layout.  scale[b] = 2^e.
 */
void oracle_quant_e4m3_blocks(int64_t nblk, int64_t len, const double *X, int64_t bstride,
                              int64_t estride, double *Q, double *scale)
{
    for (int64_t b = 0; b < nblk; ++b) {
        double amax = 0.0;
        for (int64_t i = 0; i < len; ++i) {
            double v = fabs(X[b * bstride + i * estride]);
            if (v > amax) amax = v;
        }
        int e = 0;
        if (amax > 0.0) {
            int x;
            double f = frexp(amax, &x);
            e = x - 9 + (f > 0.875 ? 1 : 0);
        }
        double sc = ldexp(1.0, e);
        scale[b] = sc;
        for (int64_t i = 0; i < len; ++i) {
            double v = X[b * bstride + i * estride] / sc;
            double r = round_to_format(v, 3, -6);
            if (fabs(r) > 448.0 && !isnan(r)) r = r > 0 ? 448.0 : -448.0;
            Q[b * bstride + i * estride] = r;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Cholesky factorization A = L L^T (lower), unblocked and right-looking: at
 * step j the diagonal entry of the updated matrix must be positive; its square
 * root is l_jj, the column below is divided by l_jj, and the trailing lower
 * triangle loses the outer product of that column with itself.  Only the lower
 * triangle (i >= j) is read or written.  Returns 0, or j+1 when the updated
 * diagonal entry at step j is not positive (or NaN): the leading (j+1) x (j+1)
 * minor is not positive definite; the matrix is then left as it was at that step.
 * ------------------------------------------------------------------------- */
int oracle_potrf(int64_t n, double *A, int64_t lda)
{
    for (int64_t j = 0; j < n; ++j) {
        const double d = A[IDX(j, j, lda)];
        if (!(d > 0.0)) return (int)(j + 1);
        const double ljj = sqrt(d);
        A[IDX(j, j, lda)] = ljj;
        for (int64_t i = j + 1; i < n; ++i) A[IDX(i, j, lda)] = A[IDX(i, j, lda)] / ljj;
        for (int64_t c = j + 1; c < n; ++c) {
            const double lcj = A[IDX(c, j, lda)];
            for (int64_t i = c; i < n; ++i) A[IDX(i, c, lda)] = A[IDX(i, c, lda)] - A[IDX(i, j, lda)] * lcj;
        }
    }
    return 0;
}

/* ||A0 - L L^T||_inf / (n ||A0||_inf) for an n x n symmetric A0 (both
 * triangles read) and the lower triangle of L; products summed compensated. */
double oracle_chol_error(int64_t n, const double *A0, int64_t lda0, const double *L, int64_t ldl)
{
    if (n == 0) return 0.0;
    double worst = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s_row = 0.0, c_row = 0.0;
        for (int64_t c = 0; c < n; ++c) {
            /* (L L^T)(i,c) = sum_{p <= min(i,c)} L(i,p) L(c,p) */
            double s = 0.0, comp = 0.0;
            const int64_t pmax = i < c ? i : c;
            for (int64_t p = 0; p <= pmax; ++p) neumaier_add(&s, &comp, L[IDX(i, p, ldl)] * L[IDX(c, p, ldl)]);
            neumaier_add(&s, &comp, -A0[IDX(i, c, lda0)]);
            neumaier_add(&s_row, &c_row, fabs(s + comp));
        }
        const double r = s_row + c_row;
        if (r > worst || isnan(r)) worst = r;
    }
    const double anorm = oracle_norm_inf(n, n, A0, lda0);
    return anorm > 0.0 ? worst / ((double)n * anorm) : (worst > 0.0 ? INFINITY : 0.0);
}

/* ---------------------------------------------------------------------------
 * Householder QR of an m x n matrix, unblocked.  Step j (j < min(m, n)) takes
 * x = A(j:m, j), alpha = x_0 and sigma = ||x(1:)||_2.  If sigma == 0 the
 * reflector is the identity (tau_j = 0).  Otherwise beta = -sign(alpha)
 * sqrt(alpha^2 + sigma^2), tau_j = (beta - alpha) / beta and
 * v = [1; x(1:) / (alpha - beta)], so that (I - tau_j v v^T) x = beta e_0;
 * A(j, j) := beta, A(j+1:m, j) := v(1:), and every column c > j becomes
 * A(j:m, c) - tau_j v (v^T A(j:m, c)).  R is the upper triangle of the result.
 * (No rescaling of norms near the underflow threshold.)
 * ------------------------------------------------------------------------- */
void oracle_geqr2(int64_t m, int64_t n, double *A, int64_t lda, double *tau)
{
    const int64_t k = m < n ? m : n;
    for (int64_t j = 0; j < k; ++j) {
        double ss = 0.0;
        for (int64_t i = j + 1; i < m; ++i) ss += A[IDX(i, j, lda)] * A[IDX(i, j, lda)];
        const double alpha = A[IDX(j, j, lda)];
        if (ss == 0.0) {
            tau[j] = 0.0;
            continue;
        }
        const double norm = sqrt(alpha * alpha + ss);
        const double beta = alpha >= 0.0 ? -norm : norm;
        tau[j] = (beta - alpha) / beta;
        const double scale = 1.0 / (alpha - beta);
        for (int64_t i = j + 1; i < m; ++i) A[IDX(i, j, lda)] = A[IDX(i, j, lda)] * scale;
        A[IDX(j, j, lda)] = beta;
        for (int64_t c = j + 1; c < n; ++c) {
            double w = A[IDX(j, c, lda)];
            for (int64_t i = j + 1; i < m; ++i) w += A[IDX(i, j, lda)] * A[IDX(i, c, lda)];
            const double tw = tau[j] * w;
            A[IDX(j, c, lda)] = A[IDX(j, c, lda)] - tw;
            for (int64_t i = j + 1; i < m; ++i) A[IDX(i, c, lda)] = A[IDX(i, c, lda)] - A[IDX(i, j, lda)] * tw;
        }
    }
}
