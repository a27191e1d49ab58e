/*
 * CPU ORACLE -- test infrastructure only.  Nothing in the product library
 * links, loads or calls this file; only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark do.
 *
 * Plain FP64 simplicial "up-looking" sparse LDL^T with D diagonal and no
 * pivoting (static pivoting), as the paper uses for the K2r and K1 systems
 * (Section 3.1, paragraph "Sparse LDL^T factorization", and Section 4.3).
 *
 *   A = L D L^T,  L unit lower triangular, D diagonal.
 *
 * Row k of L is the solution of  L(0:k,0:k) D(0:k) l_k = A(0:k, k):
 * a sparse triangular solve whose nonzero pattern is the set of
 * elimination-tree ancestors of the nonzeros of A(0:k, k) below k
 * (the "row subtree").  d_k = A(k,k) - sum_i l_ki^2 d_i.
 * This is the textbook up-looking algorithm as T. A. Davis states it in
 * "Algorithm 849: A concise sparse Cholesky factorization package" (ACM
 * Trans. Math. Software 31(4), 2005): the symbolic pass (elimination tree
 * and column counts) and the numeric pass (one row subtree per row, then
 * the forward / diagonal / backward solves) follow that published
 * algorithm's steps and its variable naming.
 *
 * Zero-pivot policy (Section 3.1, cases (i) and (ii)): if |d_k| <= eps,
 *   policy 0 (perturb): d_k := sign_k * eps, counted as perturbed, where
 *                       sign_k is +1 for a primal index, -1 for a dual
 *                       index (the block of the matrix before reordering);
 *   policy 1 (stop):    the pivot is counted as a zero eigenvalue and
 *                       the caller is told to stop (case (i)); d_k is
 *                       still set to sign_k * eps so that the remaining
 *                       pivots stay finite and the reported inertia is
 *                       that of the whole matrix with those pivots zero.
 * Inertia = signs of D (Sylvester's law of inertia).
 *
 * Input matrices are given as the upper triangle (row <= column) in CSC
 * form, already symmetrically permuted by the caller; each column's row
 * indices need not be sorted.
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>

/* Elimination tree and column counts of L (strictly below the diagonal). */
void oracle_ldl_symbolic(int64_t N, const int64_t* Ap, const int64_t* Ai,
                         int64_t* parent, int64_t* Lnz, int64_t* flag)
{
    for (int64_t k = 0; k < N; k++) {
        parent[k] = -1;
        flag[k] = k;
        Lnz[k] = 0;
        for (int64_t p = Ap[k]; p < Ap[k + 1]; p++) {
            int64_t i = Ai[p];
            if (i >= k) continue;
            /* walk from i towards the root until a node already seen in row k */
            while (flag[i] != k) {
                if (parent[i] == -1) parent[i] = k;
                Lnz[i]++;          /* L(k, i) is a nonzero */
                flag[i] = k;
                i = parent[i];
            }
        }
    }
}

/*
 * Numeric factorisation.  Lp (N+1) holds the column starts computed from
 * Lnz; on return Li/Lx hold the strictly-lower entries of L by column, D
 * the pivots.  sign[k] in {+1,-1} is the block sign of (permuted) index k.
 * Returns 0, or -1 if a pivot is NaN/Inf.
 * counts[0..3] = (n_pos, n_neg, n_zero, n_perturbed).
 */
int oracle_ldl_numeric(int64_t N, const int64_t* Ap, const int64_t* Ai, const double* Ax,
                       const int64_t* Lp, const int64_t* parent, const int* sign,
                       double eps, int policy,
                       int64_t* Lnz, int64_t* Li, double* Lx, double* D,
                       double* Y, int64_t* pattern, int64_t* flag, int64_t* counts)
{
    int bad = 0;
    counts[0] = counts[1] = counts[2] = counts[3] = 0;
    for (int64_t k = 0; k < N; k++) {
        Y[k] = 0.0;
        int64_t top = N;
        flag[k] = k;
        Lnz[k] = 0;
        for (int64_t p = Ap[k]; p < Ap[k + 1]; p++) {
            int64_t i = Ai[p];
            if (i > k) continue;
            Y[i] += Ax[p];
            int64_t len = 0;
            while (flag[i] != k) {       /* collect the path up the etree */
                pattern[len++] = i;
                flag[i] = k;
                i = parent[i];
            }
            while (len > 0) pattern[--top] = pattern[--len];
        }
        double dk = Y[k];
        Y[k] = 0.0;
        for (; top < N; top++) {         /* sparse triangular solve for row k */
            int64_t i = pattern[top];
            double yi = Y[i];
            Y[i] = 0.0;
            int64_t pend = Lp[i] + Lnz[i];
            for (int64_t p = Lp[i]; p < pend; p++) Y[Li[p]] -= Lx[p] * yi;
            double lki = yi / D[i];
            dk -= lki * yi;
            Li[pend] = k;
            Lx[pend] = lki;
            Lnz[i]++;
        }
        if (!isfinite(dk)) bad = 1;
        if (fabs(dk) <= eps) {
            dk = (sign[k] < 0 ? -eps : eps);
            D[k] = dk;
            if (policy == 0) counts[3]++;
            else { counts[2]++; continue; }
        }
        D[k] = dk;
        if (dk > 0) counts[0]++;
        else if (dk < 0) counts[1]++;
        else counts[2]++;
    }
    return bad ? -1 : 0;
}

/* x := (L D L^T)^{-1} x, in place (permuted numbering). */
void oracle_ldl_solve(int64_t N, const int64_t* Lp, const int64_t* Lnz, const int64_t* Li,
                      const double* Lx, const double* D, double* x)
{
    for (int64_t j = 0; j < N; j++) {            /* L y = b */
        double xj = x[j];
        for (int64_t p = Lp[j]; p < Lp[j] + Lnz[j]; p++) x[Li[p]] -= Lx[p] * xj;
    }
    for (int64_t j = 0; j < N; j++) x[j] /= D[j];  /* D z = y */
    for (int64_t j = N - 1; j >= 0; j--) {       /* L^T x = z */
        double s = x[j];
        for (int64_t p = Lp[j]; p < Lp[j] + Lnz[j]; p++) s -= Lx[p] * x[Li[p]];
        x[j] = s;
    }
}
