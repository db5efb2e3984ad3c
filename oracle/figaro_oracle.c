/*
 * Figaro two-table oracle: plain, slow, obviously-correct FP64 CPU code.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * What it computes ("Figaro on GPUs: Two Tables", arXiv 2503.23385):
 *   J      = the natural (inner) join of A (m1 x n1, key kA) and B (m2 x n2,
 *            key kB): one row [A_i, B_j] per pair with kA_i == kB_j.  With a
 *            single key this is the Cartesian product of Section 1 ("Theory").
 *   R      = the upper-triangular factor of QR(J) with a non-negative diagonal
 *            (Section 1: R is the Cholesky factor of J^T J).
 *   sigma  = the singular values of J, equal to those of R (Section 3, SVD via
 *            QR then SVD of R).
 *
 * Three independent routes:
 *   O1  materialise J block by block and run textbook Householder QR
 *       (the algorithm the paper's baseline uses, Section 2), then one-sided
 *       Jacobi on R.
 *   O2  build the reduced matrix from the QR head / QR tail operators of
 *       Section 1 (the H and T definitions and Claim 1, applied per key group
 *       and once more to the head rows), then the same Householder QR.
 *   O3  J^T J from per-group sums, with no QR at all.
 *
 * Parity pins (all in tests/test_oracle_*.py): LAPACK QR / SVD on small
 * matrices, brute-force joins built in Python, Claim 1 on tiny Cartesian
 * products, R^T R = J^T J, prod(diag R) = |det J| for square J,
 * sum sigma^2 = ||J||_F^2, and closed forms.
 *
 * oracle_set_mutation() plants known mistakes so tests can show that the
 * pins catch them; it is 0 (off) for every real use.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int g_mutation = 0;
void oracle_set_mutation(int m) { g_mutation = m; }
int oracle_get_mutation(void) { return g_mutation; }

/* ------------------------------------------------------------------------ */
/* Key grouping: stable sort of row indices by key (bottom-up merge sort).   */
/* Within a key, rows keep their input order.                                */
/* ------------------------------------------------------------------------ */

static int key_before(int32_t ka, int32_t kb, int32_t ia, int32_t ib) {
  if (g_mutation == 6) { /* planted: ties broken by descending index */
    if (ka != kb) return ka < kb;
    return ia > ib;
  }
  return ka < kb || (ka == kb && ia < ib);
}

/* perm[i] = input row of the i-th row in key order; sorted_key[i] its key. */
void oracle_stable_sort(const int32_t* key, int64_t m, int32_t* perm, int32_t* sorted_key) {
  if (m <= 0) return;
  int32_t* a = perm;
  int32_t* b = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  for (int64_t i = 0; i < m; ++i) a[i] = (int32_t)i;
  for (int64_t w = 1; w < m; w *= 2) {
    for (int64_t lo = 0; lo < m; lo += 2 * w) {
      int64_t mid = lo + w < m ? lo + w : m;
      int64_t hi = lo + 2 * w < m ? lo + 2 * w : m;
      int64_t p = lo, q = mid, o = lo;
      while (p < mid && q < hi) {
        if (key_before(key[a[q]], key[a[p]], a[q], a[p]))
          b[o++] = a[q++];
        else
          b[o++] = a[p++];
      }
      while (p < mid) b[o++] = a[p++];
      while (q < hi) b[o++] = a[q++];
    }
    int32_t* t = a;
    a = b;
    b = t;
  }
  if (a != perm) {
    memcpy(perm, a, sizeof(int32_t) * (size_t)m);
    free(a);
  } else {
    free(b);
  }
  for (int64_t i = 0; i < m; ++i) sorted_key[i] = key[perm[i]];
}

/* Run-length encoding of sorted keys: uniq[u], offset[u] (offset[U] = m).  */
int64_t oracle_runs(const int32_t* sorted_key, int64_t m, int32_t* uniq, int32_t* offset) {
  int64_t U = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (i == 0 || sorted_key[i] != sorted_key[i - 1]) {
      uniq[U] = sorted_key[i];
      offset[U] = (int32_t)i;
      ++U;
    }
  }
  offset[U] = (int32_t)m;
  return U;
}

/* Keys present in both tables, ascending (inner natural join).  For each
 * matched key g: its run in A (offA[g], m1[g]) and in B (offB[g], m2[g]).   */
int64_t oracle_match(const int32_t* uA, const int32_t* oA, int64_t UA, const int32_t* uB, const int32_t* oB,
                     int64_t UB, int32_t* gkey, int32_t* goffA, int32_t* gm1, int32_t* goffB, int32_t* gm2) {
  int64_t p = 0, q = 0, G = 0;
  while (p < UA && q < UB) {
    if (uA[p] < uB[q]) {
      ++p;
    } else if (uB[q] < uA[p]) {
      ++q;
    } else {
      gkey[G] = uA[p];
      goffA[G] = oA[p];
      gm1[G] = oA[p + 1] - oA[p];
      goffB[G] = oB[q];
      gm2[G] = oB[q + 1] - oB[q];
      ++G;
      ++p;
      ++q;
    }
  }
  return G;
}

/* ------------------------------------------------------------------------ */
/* Householder QR (textbook; the algorithm named as the paper's baseline).   */
/* S is column-major with `rows` rows and n columns, leading dimension ld.   */
/* On return its top n x n upper triangle holds R (unnormalised signs).      */
/* ------------------------------------------------------------------------ */
static void householder_inplace(double* S, int64_t rows, int n, int64_t ld) {
  double* v = (double*)malloc(sizeof(double) * (size_t)rows);
  int kmax = (int64_t)n < rows ? n : (int)rows;
  for (int k = 0; k < kmax; ++k) {
    double* col = S + (int64_t)k * ld;
    double norm2 = 0.0;
    for (int64_t i = k; i < rows; ++i) norm2 += col[i] * col[i];
    double norm = sqrt(norm2);
    if (norm == 0.0) continue;
    double alpha = col[k] >= 0.0 ? -norm : norm; /* H x = alpha e_k */
    for (int64_t i = k; i < rows; ++i) v[i] = col[i];
    v[k] -= alpha;
    double vtv = 0.0;
    for (int64_t i = k; i < rows; ++i) vtv += v[i] * v[i];
    if (vtv == 0.0) continue;
    for (int j = k; j < n; ++j) {
      double* cj = S + (int64_t)j * ld;
      double d = 0.0;
      for (int64_t i = k; i < rows; ++i) d += v[i] * cj[i];
      double tau = 2.0 * d / vtv;
      if (g_mutation == 5) tau = -tau; /* planted: wrong reflector sign */
      for (int64_t i = k; i < rows; ++i) cj[i] -= tau * v[i];
    }
  }
  free(v);
}

/* Streaming QR: R (n x n, row-major) <- upper factor of [R; X], X row-major
 * (rows x n, leading dimension ldx).  Starting from R = 0 gives QR(X).     */
void oracle_qr_update(double* R, int n, const double* X, int64_t rows, int64_t ldx) {
  int64_t tot = n + rows;
  double* S = (double*)calloc((size_t)(tot * n), sizeof(double));
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) S[(int64_t)j * tot + i] = R[(int64_t)i * n + j];
    for (int64_t r = 0; r < rows; ++r) S[(int64_t)j * tot + n + r] = X[r * ldx + j];
  }
  householder_inplace(S, tot, n, tot);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) R[(int64_t)i * n + j] = j >= i ? S[(int64_t)j * tot + i] : 0.0;
  free(S);
}

/* Rows of R scaled by -1 where the diagonal is negative (R unique for full
 * column rank once diag >= 0).                                              */
void oracle_sign_normalise(double* R, int n) {
  for (int i = 0; i < n; ++i) {
    if (R[(int64_t)i * n + i] < 0.0)
      for (int j = 0; j < n; ++j) R[(int64_t)i * n + j] = -R[(int64_t)i * n + j];
  }
}

/* ------------------------------------------------------------------------ */
/* One-sided (Hestenes) Jacobi SVD of an n x n matrix (row-major input).     */
/* Cyclic sweeps over column pairs, each rotation chosen from the 2 x 2 Gram */
/* matrix of the pair so that the two columns become orthogonal.             */
/* sigma: the column norms at convergence, descending.  Returns sweeps used,  */
/* or -1 if max_sweeps was reached before convergence.  A column whose       */
/* squared norm is at most (n 2^-53)^2 ||R||_F^2 is rounding noise of a      */
/* rank-deficient R (a zero singular value) and is left out of rotations:    */
/* the relative orthogonality test can never be met by such columns.         */
/* ------------------------------------------------------------------------ */
int oracle_jacobi_sigma(const double* Rin, int n, double* sigma, int max_sweeps) {
  double* U = (double*)malloc(sizeof(double) * (size_t)n * n); /* column-major */
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) U[(int64_t)j * n + i] = Rin[(int64_t)i * n + j];
  const double tol = (double)n * 1.1102230246251565e-16; /* n * 2^-53 */
  double fro2 = 0.0;
  for (int64_t e = 0; e < (int64_t)n * n; ++e) fro2 += U[e] * U[e];
  const double negligible = tol * tol * fro2;
  int sweeps = 0, converged = 0;
  while (sweeps < max_sweeps) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double* up = U + (int64_t)p * n;
        double* uq = U + (int64_t)q * n;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = 0; i < n; ++i) {
          a += up[i] * up[i];
          b += uq[i] * uq[i];
          g += up[i] * uq[i];
        }
        if (a <= negligible || b <= negligible || g == 0.0) continue;
        double rel = fabs(g) / sqrt(a * b);
        if (rel > off) off = rel;
        if (rel <= tol) continue;
        double zeta = (b - a) / (2.0 * g);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        if (g_mutation == 7) s = -s; /* planted: rotation in the wrong sense */
        for (int i = 0; i < n; ++i) {
          double x = up[i], y = uq[i];
          up[i] = c * x - s * y;
          uq[i] = s * x + c * y;
        }
      }
    }
    ++sweeps;
    if (off <= tol) {
      converged = 1;
      break;
    }
  }
  for (int j = 0; j < n; ++j) {
    double s2 = 0.0;
    for (int i = 0; i < n; ++i) s2 += U[(int64_t)j * n + i] * U[(int64_t)j * n + i];
    sigma[j] = sqrt(s2);
  }
  /* insertion sort, descending */
  for (int i = 1; i < n; ++i) {
    double v = sigma[i];
    int j = i - 1;
    while (j >= 0 && sigma[j] < v) {
      sigma[j + 1] = sigma[j];
      --j;
    }
    sigma[j + 1] = v;
  }
  free(U);
  return converged ? sweeps : -1;
}

/* ------------------------------------------------------------------------ */
/* Singular values and right singular vectors of a square R (Section 1's    */
/* applications: the SVD of J, e.g. for its principal components; Section 3:*/
/* J = Q R, so J and R share sigma and V).  The same cyclic one-sided       */
/* Jacobi as oracle_jacobi_sigma, with every rotation also applied to the    */
/* columns of V (V starts as I, so R V = U keeps orthogonal columns and      */
/* sigma_j = ||U_j||).  Output: sigma descending, V row-major (column j the  */
/* unit right singular vector of sigma_j), each column's largest-magnitude   */
/* component made positive.  Returns the sweeps, or -1 without convergence.  */
/* ------------------------------------------------------------------------ */
int oracle_jacobi_svd(const double* Rin, int n, double* sigma, double* Vout, int max_sweeps) {
  double* U = (double*)malloc(sizeof(double) * (size_t)n * n); /* column-major */
  double* V = (double*)malloc(sizeof(double) * (size_t)n * n); /* column-major */
  int* order = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  double* norm = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      U[(int64_t)j * n + i] = Rin[(int64_t)i * n + j];
      V[(int64_t)j * n + i] = i == j ? 1.0 : 0.0;
    }
  const double tol = (double)n * 1.1102230246251565e-16; /* n * 2^-53 */
  double fro2 = 0.0;
  for (int64_t e = 0; e < (int64_t)n * n; ++e) fro2 += U[e] * U[e];
  const double negligible = tol * tol * fro2;
  int sweeps = 0, converged = n <= 1;
  while (!converged && sweeps < max_sweeps) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double* up = U + (int64_t)p * n;
        double* uq = U + (int64_t)q * n;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = 0; i < n; ++i) {
          a += up[i] * up[i];
          b += uq[i] * uq[i];
          g += up[i] * uq[i];
        }
        if (a <= negligible || b <= negligible || g == 0.0) continue;
        double rel = fabs(g) / sqrt(a * b);
        if (rel > off) off = rel;
        if (rel <= tol) continue;
        double zeta = (b - a) / (2.0 * g);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        for (int i = 0; i < n; ++i) {
          double x = up[i], y = uq[i];
          up[i] = c * x - s * y;
          uq[i] = s * x + c * y;
        }
        if (g_mutation != 8) { /* planted (8): V not rotated */
          double* vp = V + (int64_t)p * n;
          double* vq = V + (int64_t)q * n;
          for (int i = 0; i < n; ++i) {
            double x = vp[i], y = vq[i];
            vp[i] = c * x - s * y;
            vq[i] = s * x + c * y;
          }
        }
      }
    }
    ++sweeps;
    if (off <= tol) converged = 1;
  }
  for (int j = 0; j < n; ++j) {
    double s2 = 0.0;
    for (int i = 0; i < n; ++i) s2 += U[(int64_t)j * n + i] * U[(int64_t)j * n + i];
    norm[j] = sqrt(s2);
    order[j] = j;
  }
  /* insertion sort of the column indices by descending norm (stable) */
  for (int i = 1; i < n; ++i) {
    int v = order[i];
    int j = i - 1;
    while (j >= 0 && norm[order[j]] < norm[v]) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = v;
  }
  for (int j = 0; j < n; ++j) {
    const double* vc = V + (int64_t)order[j] * n;
    sigma[j] = norm[order[j]];
    int big = 0;
    for (int i = 1; i < n; ++i)
      if (fabs(vc[i]) > fabs(vc[big])) big = i;
    const double sg = vc[big] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < n; ++i) Vout[(int64_t)i * n + j] = sg * vc[i];
  }
  free(U);
  free(V);
  free(order);
  free(norm);
  return converged ? sweeps : -1;
}

/* ------------------------------------------------------------------------ */
/* Grouping of both tables (helper used by O1, O2, O3).                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t *permA, *permB, *skA, *skB, *uA, *oA, *uB, *oB;
  int32_t *gkey, *goffA, *gm1, *goffB, *gm2;
  int64_t UA, UB, G;
} groups_t;

static void groups_build(groups_t* g, const int32_t* kA, int64_t m1, const int32_t* kB, int64_t m2) {
  size_t a = (size_t)(m1 > 0 ? m1 : 1), b = (size_t)(m2 > 0 ? m2 : 1);
  g->permA = (int32_t*)malloc(4 * a);
  g->skA = (int32_t*)malloc(4 * a);
  g->uA = (int32_t*)malloc(4 * a);
  g->oA = (int32_t*)malloc(4 * (a + 1));
  g->permB = (int32_t*)malloc(4 * b);
  g->skB = (int32_t*)malloc(4 * b);
  g->uB = (int32_t*)malloc(4 * b);
  g->oB = (int32_t*)malloc(4 * (b + 1));
  size_t gm = a < b ? a : b;
  g->gkey = (int32_t*)malloc(4 * gm);
  g->goffA = (int32_t*)malloc(4 * gm);
  g->gm1 = (int32_t*)malloc(4 * gm);
  g->goffB = (int32_t*)malloc(4 * gm);
  g->gm2 = (int32_t*)malloc(4 * gm);
  oracle_stable_sort(kA, m1, g->permA, g->skA);
  oracle_stable_sort(kB, m2, g->permB, g->skB);
  g->UA = oracle_runs(g->skA, m1, g->uA, g->oA);
  g->UB = oracle_runs(g->skB, m2, g->uB, g->oB);
  g->G = oracle_match(g->uA, g->oA, g->UA, g->uB, g->oB, g->UB, g->gkey, g->goffA, g->gm1, g->goffB, g->gm2);
}

static void groups_free(groups_t* g) {
  free(g->permA); free(g->skA); free(g->uA); free(g->oA);
  free(g->permB); free(g->skB); free(g->uB); free(g->oB);
  free(g->gkey); free(g->goffA); free(g->gm1); free(g->goffB); free(g->gm2);
}

/* Number of rows of J = sum over matched keys of m1g * m2g. */
int64_t oracle_join_rows(const int32_t* kA, int64_t m1, const int32_t* kB, int64_t m2) {
  groups_t g;
  groups_build(&g, kA, m1, kB, m2);
  int64_t rows = 0;
  for (int64_t t = 0; t < g.G; ++t) rows += (int64_t)g.gm1[t] * g.gm2[t];
  groups_free(&g);
  return rows;
}

/* Materialise rows [first, first+count) of J (keys ascending, then A's row
 * order within the key, then B's) into X (count x (n1+n2), row-major).      */
int64_t oracle_join_materialize(const double* A, int64_t m1, int n1, int64_t lda, const int32_t* kA, const double* B,
                                int64_t m2, int n2, int64_t ldb, const int32_t* kB, int64_t first, int64_t count,
                                double* X) {
  groups_t g;
  groups_build(&g, kA, m1, kB, m2);
  int n = n1 + n2;
  int64_t r = 0, w = 0;
  for (int64_t t = 0; t < g.G && w < count; ++t) {
    for (int32_t i = 0; i < g.gm1[t] && w < count; ++i) {
      const double* a = A + (int64_t)g.permA[g.goffA[t] + i] * lda;
      for (int32_t j = 0; j < g.gm2[t] && w < count; ++j, ++r) {
        if (r < first) continue;
        const double* b = B + (int64_t)g.permB[g.goffB[t] + j] * ldb;
        double* x = X + w * n;
        for (int c = 0; c < n1; ++c) x[c] = a[c];
        for (int c = 0; c < n2; ++c) x[n1 + c] = b[c];
        ++w;
      }
    }
  }
  groups_free(&g);
  return w;
}

/* O1: R of QR(J), J materialised in blocks of at most block_rows rows.     */
void oracle_join_r_materialized(const double* A, int64_t m1, int n1, int64_t lda, const int32_t* kA,
                                const double* B, int64_t m2, int n2, int64_t ldb, const int32_t* kB,
                                int64_t block_rows, double* R) {
  int n = n1 + n2;
  if (block_rows <= 0) block_rows = 65536;
  groups_t g;
  groups_build(&g, kA, m1, kB, m2);
  memset(R, 0, sizeof(double) * (size_t)n * n);
  double* X = (double*)malloc(sizeof(double) * (size_t)block_rows * n);
  int64_t w = 0;
  for (int64_t t = 0; t < g.G; ++t) {
    for (int32_t i = 0; i < g.gm1[t]; ++i) {
      const double* a = A + (int64_t)g.permA[g.goffA[t] + i] * lda;
      for (int32_t j = 0; j < g.gm2[t]; ++j) {
        const double* b = B + (int64_t)g.permB[g.goffB[t] + j] * ldb;
        double* x = X + w * n;
        for (int c = 0; c < n1; ++c) x[c] = a[c];
        for (int c = 0; c < n2; ++c) x[n1 + c] = b[c];
        if (++w == block_rows) {
          oracle_qr_update(R, n, X, w, n);
          w = 0;
        }
      }
    }
  }
  if (w > 0) oracle_qr_update(R, n, X, w, n);
  oracle_sign_normalise(R, n);
  free(X);
  groups_free(&g);
}

/* ------------------------------------------------------------------------ */
/* QR head and QR tail operators (Section 1, the definitions of H and T).    */
/* X: m rows (given through a row-pointer table so a key group can be read   */
/* in place), n columns.  head: 1 x n.  tail: (m-1) x n, row-major.          */
/*   H(X)   = (1/sqrt(m)) * sum_{k=1..m} X_k                                 */
/*   T(X)_i = (1/sqrt(i+1)) * ( sqrt(i) X_{i+1} - (1/sqrt(i)) sum_{k<=i} X_k )*/
/* Written in this direct form on purpose: no running means, no reuse.      */
/* ------------------------------------------------------------------------ */
void oracle_qr_head(const double* const* rows, int64_t m, int n, double* head) {
  for (int c = 0; c < n; ++c) {
    double s = 0.0;
    for (int64_t k = 0; k < m; ++k) s += rows[k][c];
    head[c] = s / sqrt((double)m);
  }
}

void oracle_qr_tail(const double* const* rows, int64_t m, int n, double* tail) {
  /* pref[c] = sum_{k=1..i} X_{k,c} (1-based), kept as a running sum over i. */
  double* pref = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  for (int64_t i = 1; i < m; ++i) { /* paper's i = 1..m-1; rows[i] is X_{i+1} */
    for (int c = 0; c < n; ++c) pref[c] += rows[i - 1][c];
    double si = sqrt((double)i);
    double sgn = g_mutation == 2 ? 1.0 : -1.0; /* planted: wrong sign */
    for (int c = 0; c < n; ++c) {
      double p = g_mutation == 3 ? pref[c] - rows[i - 1][c] : pref[c]; /* planted: prefix one row short */
      tail[(i - 1) * n + c] = (si * rows[i][c] + sgn * p / si) / sqrt((double)(i + 1));
    }
  }
  free(pref);
}

/* O2 reduced matrix.  Per matched key group g (ascending key) with m1g rows
 * of A and m2g rows of B (stable order), Claim 1 applied to A_g x B_g and
 * once more to its m1g head rows [sqrt(m2g) A_i, H(B_g)] gives the rows
 *   head: [ sqrt(m2g) H(A_g), sqrt(m1g) H(B_g) ]            1 row
 *   TA  : [ sqrt(m2g) T(A_g), 0 ]                           m1g-1 rows
 *   TB  : [ 0, sqrt(m1g) T(B_g) ]                           m2g-1 rows
 * whose Gram matrix equals that of the group's m1g*m2g join rows.
 * Outputs (row-major, group order): Hd (G x n), TA (sum(m1g-1) x n1),
 * TB (sum(m2g-1) x n2).  Returns G; *nta, *ntb receive the tail counts.     */
int64_t oracle_reduce(const double* A, int64_t m1, int n1, int64_t lda, const int32_t* kA, const double* B,
                      int64_t m2, int n2, int64_t ldb, const int32_t* kB, double* Hd, double* TA, double* TB,
                      int64_t* nta, int64_t* ntb) {
  groups_t g;
  groups_build(&g, kA, m1, kB, m2);
  int n = n1 + n2;
  int64_t ta = 0, tb = 0;
  for (int64_t t = 0; t < g.G; ++t) {
    int64_t a_m = g.gm1[t], b_m = g.gm2[t];
    const double** ra = (const double**)malloc(sizeof(double*) * (size_t)a_m);
    const double** rb = (const double**)malloc(sizeof(double*) * (size_t)b_m);
    for (int64_t i = 0; i < a_m; ++i) ra[i] = A + (int64_t)g.permA[g.goffA[t] + i] * lda;
    for (int64_t j = 0; j < b_m; ++j) rb[j] = B + (int64_t)g.permB[g.goffB[t] + j] * ldb;
    double wa = sqrt((double)b_m); /* weight on A's head and tails: sqrt(m2g) */
    double wb = sqrt((double)a_m); /* weight on B's head and tails: sqrt(m1g) */
    if (g_mutation == 1) wa = 1.0;  /* planted: weight dropped */
    if (g_mutation == 4) {          /* planted: weights swapped */
      double s = wa;
      wa = wb;
      wb = s;
    }
    double* h = Hd + t * n;
    oracle_qr_head(ra, a_m, n1, h);
    oracle_qr_head(rb, b_m, n2, h + n1);
    for (int c = 0; c < n1; ++c) h[c] *= wa;
    for (int c = 0; c < n2; ++c) h[n1 + c] *= wb;
    if (a_m > 1) {
      oracle_qr_tail(ra, a_m, n1, TA + ta * n1);
      for (int64_t k = 0; k < (a_m - 1) * n1; ++k) TA[ta * n1 + k] *= wa;
      ta += a_m - 1;
    }
    if (b_m > 1) {
      oracle_qr_tail(rb, b_m, n2, TB + tb * n2);
      for (int64_t k = 0; k < (b_m - 1) * n2; ++k) TB[tb * n2 + k] *= wb;
      tb += b_m - 1;
    }
    free(ra);
    free(rb);
  }
  *nta = ta;
  *ntb = tb;
  int64_t G = g.G;
  groups_free(&g);
  return G;
}

/* Sizes of the O2 outputs, so callers can allocate: returns G. */
int64_t oracle_reduce_sizes(const int32_t* kA, int64_t m1, const int32_t* kB, int64_t m2, int64_t* nta,
                            int64_t* ntb) {
  groups_t g;
  groups_build(&g, kA, m1, kB, m2);
  int64_t ta = 0, tb = 0;
  for (int64_t t = 0; t < g.G; ++t) {
    ta += g.gm1[t] - 1;
    tb += g.gm2[t] - 1;
  }
  *nta = ta;
  *ntb = tb;
  int64_t G = g.G;
  groups_free(&g);
  return G;
}

/* O2: R of QR(J) through the reduced matrix: rows [Hd; (TA,0); (0,TB)]
 * streamed through the Householder update in blocks.                        */
void oracle_join_r_reduced(const double* A, int64_t m1, int n1, int64_t lda, const int32_t* kA, const double* B,
                           int64_t m2, int n2, int64_t ldb, const int32_t* kB, int64_t block_rows, double* R) {
  int n = n1 + n2;
  if (block_rows <= 0) block_rows = 65536;
  int64_t nta, ntb;
  int64_t G = oracle_reduce_sizes(kA, m1, kB, m2, &nta, &ntb);
  double* Hd = (double*)malloc(sizeof(double) * (size_t)((G > 0 ? G : 1) * n));
  double* TA = (double*)malloc(sizeof(double) * (size_t)((nta > 0 ? nta : 1) * n1));
  double* TB = (double*)malloc(sizeof(double) * (size_t)((ntb > 0 ? ntb : 1) * n2));
  oracle_reduce(A, m1, n1, lda, kA, B, m2, n2, ldb, kB, Hd, TA, TB, &nta, &ntb);
  memset(R, 0, sizeof(double) * (size_t)n * n);
  double* X = (double*)malloc(sizeof(double) * (size_t)block_rows * n);
  int64_t w = 0;
  int64_t total = G + nta + ntb;
  for (int64_t r = 0; r < total; ++r) {
    double* x = X + w * n;
    memset(x, 0, sizeof(double) * (size_t)n);
    if (r < G) {
      memcpy(x, Hd + r * n, sizeof(double) * (size_t)n);
    } else if (r < G + nta) {
      memcpy(x, TA + (r - G) * n1, sizeof(double) * (size_t)n1);
    } else {
      memcpy(x + n1, TB + (r - G - nta) * n2, sizeof(double) * (size_t)n2);
    }
    if (++w == block_rows) {
      oracle_qr_update(R, n, X, w, n);
      w = 0;
    }
  }
  if (w > 0) oracle_qr_update(R, n, X, w, n);
  oracle_sign_normalise(R, n);
  free(X);
  free(Hd);
  free(TA);
  free(TB);
}

/* O3: J^T J without QR.  With s_A(g), s_B(g) the column sums of a group,
 *   J^T J = [[ sum_g m2g A_g^T A_g , sum_g s_A(g) s_B(g)^T ],
 *            [ .                   , sum_g m1g B_g^T B_g   ]].             */
void oracle_join_gram(const double* A, int64_t m1, int n1, int64_t lda, const int32_t* kA, const double* B,
                      int64_t m2, int n2, int64_t ldb, const int32_t* kB, double* JtJ) {
  int n = n1 + n2;
  groups_t g;
  groups_build(&g, kA, m1, kB, m2);
  memset(JtJ, 0, sizeof(double) * (size_t)n * n);
  double* sa = (double*)malloc(sizeof(double) * (size_t)(n1 > 0 ? n1 : 1));
  double* sb = (double*)malloc(sizeof(double) * (size_t)(n2 > 0 ? n2 : 1));
  for (int64_t t = 0; t < g.G; ++t) {
    double w2 = (double)g.gm2[t], w1 = (double)g.gm1[t];
    memset(sa, 0, sizeof(double) * (size_t)n1);
    memset(sb, 0, sizeof(double) * (size_t)n2);
    for (int32_t i = 0; i < g.gm1[t]; ++i) {
      const double* a = A + (int64_t)g.permA[g.goffA[t] + i] * lda;
      for (int p = 0; p < n1; ++p) {
        sa[p] += a[p];
        for (int q = 0; q < n1; ++q) JtJ[(int64_t)p * n + q] += w2 * a[p] * a[q];
      }
    }
    for (int32_t j = 0; j < g.gm2[t]; ++j) {
      const double* b = B + (int64_t)g.permB[g.goffB[t] + j] * ldb;
      for (int p = 0; p < n2; ++p) {
        sb[p] += b[p];
        for (int q = 0; q < n2; ++q) JtJ[(int64_t)(n1 + p) * n + n1 + q] += w1 * b[p] * b[q];
      }
    }
    for (int p = 0; p < n1; ++p)
      for (int q = 0; q < n2; ++q) {
        JtJ[(int64_t)p * n + n1 + q] += sa[p] * sb[q];
        JtJ[(int64_t)(n1 + q) * n + p] += sa[p] * sb[q];
      }
  }
  free(sa);
  free(sb);
  groups_free(&g);
}
