/*
 * dfacto_oracle.c -- plain FP64 CPU restatement of DFacTo (Choi & Vishwanathan,
 * "DFacTo: Distributed Factorization of Tensors", NIPS 2014).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA library is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * load it; the library never calls it and shares no code, header or table with it.
 *
 * Everything here is deliberately slow and literal:
 *   - the flattened CSR copies are built by sorting (o,f,in) tuples with qsort;
 *   - the MTTKRP is its plain definition, a straight per-nonzero sum over the COO
 *     tensor (Lemma 2 shows DFacTo reaches exactly this value, Sec. 3);
 *   - ALS (Algorithm 2 / Algorithm 4), GD (Algorithm 3 / Algorithm 5) and the fit
 *     are taken step by step in the paper's order, in FP64 throughout.
 *
 * Conventions (0-based, as in the index matrix S of Appendix D):
 *   tensor X is I x J x K; nonzero t has coordinates idx[0*nnz+t] (i),
 *   idx[1*nnz+t] (j), idx[2*nnz+t] (k) and value val[t] (fp32, widened exactly).
 *   Factor matrices are row-major: F[m][row*R + r].
 *   For mode n (0,1,2): o = axis n, in = axis (n+1)%3, f = axis (n+2)%3, so that
 *   mode 0 is X^1 (C kr B) computed through (X^2)^T with rows (i,k) and entries j,
 *   mode 1 is X^2 (A kr C) through (X^3)^T with rows (j,i) and entries k,
 *   mode 2 is X^3 (B kr A) through (X^1)^T with rows (k,j) and entries i
 *   (Eq. x1 and Algorithm 4).
 *
 * Status codes match the library's: 0 ok, 1 invalid argument, 2 index out of
 * range, 3 duplicate coordinate, 4 out of memory, 6 singular system (the
 * pseudo-inverse was used), 7 line search failed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ERANGE 2
#define ORC_EDUP 3
#define ORC_ENOMEM 4
#define ORC_ESINGULAR 6
#define ORC_ELSFAIL 7

static int ax_o(int mode) { return mode; }
static int ax_in(int mode) { return (mode + 1) % 3; }
static int ax_f(int mode) { return (mode + 2) % 3; }

int orc_axes(int mode, int32_t* o, int32_t* in, int32_t* f) {
  if (mode < 0 || mode > 2) return ORC_EINVAL;
  *o = ax_o(mode);
  *in = ax_in(mode);
  *f = ax_f(mode);
  return ORC_OK;
}

/* Observed entries must lie inside the I x J x K box (notation of Sec. 2). */
int orc_check_coo(int64_t nnz, const int32_t* idx, const int32_t* dims) {
  for (int m = 0; m < 3; ++m)
    if (dims[m] <= 0) return ORC_EINVAL;
  if (nnz < 0) return ORC_EINVAL;
  for (int m = 0; m < 3; ++m)
    for (int64_t t = 0; t < nnz; ++t) {
      int32_t v = idx[(int64_t)m * nnz + t];
      if (v < 0 || v >= dims[m]) return ORC_ERANGE;
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Flattened CSR copies (Sec. 3, Lemma 3 and Lemma 4).                        */
/* ------------------------------------------------------------------------- */

typedef struct {
  int32_t o, f, in;
  int64_t t; /* position in the COO input */
} orc_tuple;

static int cmp_tuple(const void* a, const void* b) {
  const orc_tuple* x = (const orc_tuple*)a;
  const orc_tuple* y = (const orc_tuple*)b;
  if (x->o != y->o) return x->o < y->o ? -1 : 1;
  if (x->f != y->f) return x->f < y->f ? -1 : 1;
  if (x->in != y->in) return x->in < y->in ? -1 : 1;
  return 0;
}

/*
 * Build the CSR of (X^{n+1})^T with its all-zero rows removed, plus the fixed
 * sparsity pattern of the intermediate matrix M^r (Sec. 3):
 *   - the rows of (X^2)^T are indexed k + (i-1)K (proof of Lemma 4), i.e. ordered
 *     i-major then k, so for mode n the rows are the distinct (o,f) pairs in
 *     lexicographic order ("fibers");
 *   - each row holds the entries in ascending column order (the CSR example of
 *     Sec. 3), the column being the index `in`;
 *   - M^r is dim_o x dim_f with one nonzero per fiber (Lemma 4); its row array
 *     fiber_ptr has dim_o+1 entries, empty rows included, its column array is
 *     fiber_idx (= f) and its value array is filled by the first SpMV.
 * Outputs (caller-allocated, nnz entries is always enough for the fiber arrays):
 *   fiber_ptr[dim_o+1], fiber_idx[nfib], nz_ptr[nfib+1], nz_idx[nnz], nz_val[nnz].
 * Returns ORC_EDUP if two nonzeros share a coordinate.
 */
int orc_build_csr(int mode, int64_t nnz, const int32_t* idx, const float* val,
                  const int32_t* dims, int64_t* fiber_ptr, int32_t* fiber_idx,
                  int64_t* nz_ptr, int32_t* nz_idx, float* nz_val, int64_t* nfib_out) {
  if (mode < 0 || mode > 2) return ORC_EINVAL;
  int st = orc_check_coo(nnz, idx, dims);
  if (st != ORC_OK) return st;
  const int o = ax_o(mode), in = ax_in(mode), f = ax_f(mode);
  const int64_t dim_o = dims[o];
  orc_tuple* tup = (orc_tuple*)malloc(sizeof(orc_tuple) * (size_t)(nnz > 0 ? nnz : 1));
  if (!tup) return ORC_ENOMEM;
  for (int64_t t = 0; t < nnz; ++t) {
    tup[t].o = idx[(int64_t)o * nnz + t];
    tup[t].f = idx[(int64_t)f * nnz + t];
    tup[t].in = idx[(int64_t)in * nnz + t];
    tup[t].t = t;
  }
  qsort(tup, (size_t)nnz, sizeof(orc_tuple), cmp_tuple);
  for (int64_t p = 1; p < nnz; ++p)
    if (cmp_tuple(&tup[p - 1], &tup[p]) == 0) {
      free(tup);
      return ORC_EDUP;
    }
  int64_t nfib = 0;
  for (int64_t p = 0; p < nnz; ++p) {
    int new_fiber = (p == 0) || tup[p].o != tup[p - 1].o || tup[p].f != tup[p - 1].f;
    if (new_fiber) {
      nz_ptr[nfib] = p;
      fiber_idx[nfib] = tup[p].f;
      ++nfib;
    }
    nz_idx[p] = tup[p].in;
    nz_val[p] = val[tup[p].t];
  }
  nz_ptr[nfib] = nnz;
  /* row(M^r): fiber_ptr[r] = number of fibers whose row is < r. */
  int64_t fib = 0;
  for (int64_t r = 0; r <= dim_o; ++r) {
    while (fib < nfib && tup[nz_ptr[fib]].o < r) ++fib;
    fiber_ptr[r] = fib;
  }
  *nfib_out = nfib;
  free(tup);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* MTTKRP: N = X^n (F_f kr F_in), by definition.                              */
/* ------------------------------------------------------------------------- */

/*
 * Column c of X^n pairs the indices (in, f); the Khatri-Rao product (Appendix A,
 * Eq. khatraodef) of F_f and F_in has entry F_f[f,r] * F_in[in,r] in that row.
 * Hence N[o,r] = sum over observed (i,j,k) of x_ijk * F_in[in,r] * F_f[f,r].
 * F[0], F[1], F[2] are A, B, C.  out is dims[mode] x R.
 */
void orc_mttkrp(int mode, int64_t nnz, const int32_t* idx, const float* val,
                const int32_t* dims, int R, const double* A, const double* B,
                const double* C, double* out) {
  const double* F[3] = {A, B, C};
  const int o = ax_o(mode), in = ax_in(mode), f = ax_f(mode);
  const int64_t len = (int64_t)dims[o] * R;
  memset(out, 0, sizeof(double) * (size_t)len);
#ifdef _OPENMP
  /* Multi-core timing build only: each thread sums its share of the nonzeros
     into its own heap copy of out; the copies are added at the end. */
  {
    const int nth = omp_get_max_threads();
    double* priv = nth > 1 ? (double*)calloc((size_t)nth * (size_t)len, sizeof(double)) : NULL;
    if (priv) {
#pragma omp parallel
      {
        double* my = priv + (size_t)omp_get_thread_num() * (size_t)len;
#pragma omp for
        for (int64_t t = 0; t < nnz; ++t) {
          const int64_t io = idx[(int64_t)o * nnz + t];
          const int64_t ii = idx[(int64_t)in * nnz + t];
          const int64_t iff = idx[(int64_t)f * nnz + t];
          const double x = (double)val[t];
          for (int r = 0; r < R; ++r) my[io * R + r] += x * F[in][ii * R + r] * F[f][iff * R + r];
        }
      }
#pragma omp parallel for
      for (int64_t e = 0; e < len; ++e)
        for (int th = 0; th < nth; ++th) out[e] += priv[(size_t)th * (size_t)len + e];
      free(priv);
      return;
    }
  }
#endif
  for (int64_t t = 0; t < nnz; ++t) {
    const int64_t io = idx[(int64_t)o * nnz + t];
    const int64_t ii = idx[(int64_t)in * nnz + t];
    const int64_t iff = idx[(int64_t)f * nnz + t];
    const double x = (double)val[t];
    for (int r = 0; r < R; ++r)
      out[io * R + r] += x * F[in][ii * R + r] * F[f][iff * R + r];
  }
}

/*
 * The same sum restricted to the output rows listed in rows[0..nrows) (distinct,
 * any order); out is nrows x R in the order of rows.  Used to check sampled rows
 * of very large problems.
 */
int orc_mttkrp_rows(int mode, int64_t nnz, const int32_t* idx, const float* val,
                    const int32_t* dims, int R, const double* A, const double* B,
                    const double* C, int64_t nrows, const int64_t* rows, double* out) {
  const double* F[3] = {A, B, C};
  const int o = ax_o(mode), in = ax_in(mode), f = ax_f(mode);
  int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)dims[o]);
  if (!slot) return ORC_ENOMEM;
  for (int64_t r = 0; r < dims[o]; ++r) slot[r] = -1;
  for (int64_t s = 0; s < nrows; ++s) {
    if (rows[s] < 0 || rows[s] >= dims[o]) {
      free(slot);
      return ORC_ERANGE;
    }
    slot[rows[s]] = s;
  }
  memset(out, 0, sizeof(double) * (size_t)nrows * (size_t)R);
  for (int64_t t = 0; t < nnz; ++t) {
    const int64_t s = slot[idx[(int64_t)o * nnz + t]];
    if (s < 0) continue;
    const int64_t ii = idx[(int64_t)in * nnz + t];
    const int64_t iff = idx[(int64_t)f * nnz + t];
    const double x = (double)val[t];
    for (int r = 0; r < R; ++r) out[s * R + r] += x * F[in][ii * R + r] * F[f][iff * R + r];
  }
  free(slot);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Small dense linear algebra (R x R, FP64).                                  */
/* ------------------------------------------------------------------------- */

/* G = F^T F for an n x R row-major F (the Grams in Eq. kr-product). */
void orc_gram(int64_t n, int R, const double* F, double* G) {
  const int64_t RR = (int64_t)R * R;
  memset(G, 0, sizeof(double) * (size_t)RR);
#pragma omp parallel for reduction(+ : G[0:RR])
  for (int64_t i = 0; i < n; ++i)
    for (int r = 0; r < R; ++r)
      for (int s = 0; s < R; ++s) G[r * R + s] += F[i * R + r] * F[i * R + s];
}

/*
 * Lower Cholesky factor in place (textbook column-by-column form).  Returns 0 if
 * the matrix is numerically positive definite: every pivot must exceed
 * R * eps times its original diagonal entry, otherwise the factorization is
 * declared failed (a pivot at rounding level means a singular matrix).
 */
static int chol_lower(int R, double* L) {
  for (int j = 0; j < R; ++j) {
    const double diag = L[j * R + j];
    double d = diag;
    for (int k = 0; k < j; ++k) d -= L[j * R + k] * L[j * R + k];
    if (!(diag > 0.0) || !(d > (double)R * 2.220446049250313e-16 * diag)) return -1;
    d = sqrt(d);
    L[j * R + j] = d;
    for (int i = j + 1; i < R; ++i) {
      double s = L[i * R + j];
      for (int k = 0; k < j; ++k) s -= L[i * R + k] * L[j * R + k];
      L[i * R + j] = s / d;
    }
  }
  for (int i = 0; i < R; ++i)
    for (int j = i + 1; j < R; ++j) L[i * R + j] = 0.0;
  return 0;
}

/*
 * Symmetric eigen-decomposition by the cyclic Jacobi method (Golub & Van Loan,
 * Matrix Computations, Sec. 8.5): A (R x R, overwritten) -> eigenvalues w and
 * eigenvectors in the columns of V.
 */
int orc_sym_eig_jacobi(int R, double* A, double* V, double* w) {
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < R; ++j) V[i * R + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < R; ++i)
      for (int j = 0; j < R; ++j) {
        tot += A[i * R + j] * A[i * R + j];
        if (i != j) off += A[i * R + j] * A[i * R + j];
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < R - 1; ++p)
      for (int q = p + 1; q < R; ++q) {
        double apq = A[p * R + q];
        if (apq == 0.0) continue;
        double app = A[p * R + p], aqq = A[q * R + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < R; ++k) { /* A <- A J (columns p, q) */
          double akp = A[k * R + p], akq = A[k * R + q];
          A[k * R + p] = c * akp - s * akq;
          A[k * R + q] = s * akp + c * akq;
        }
        for (int k = 0; k < R; ++k) { /* A <- J^T A (rows p, q) */
          double apk = A[p * R + k], aqk = A[q * R + k];
          A[p * R + k] = c * apk - s * aqk;
          A[q * R + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < R; ++k) { /* V <- V J */
          double vkp = V[k * R + p], vkq = V[k * R + q];
          V[k * R + p] = c * vkp - s * vkq;
          V[k * R + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < R; ++i) w[i] = A[i * R + i];
  return ORC_OK;
}

/*
 * Moore-Penrose pseudo-inverse of a symmetric R x R matrix through its Jacobi
 * eigen-decomposition; eigenvalues with |w| <= R * eps * max|w| count as zero
 * (the pseudo-inverse of Eq. kr-pseudo for a singular Hadamard of Grams).
 */
int orc_pinv_sym(int R, const double* S, double* P) {
  double* A = (double*)malloc(sizeof(double) * (size_t)R * R);
  double* V = (double*)malloc(sizeof(double) * (size_t)R * R);
  double* w = (double*)malloc(sizeof(double) * (size_t)R);
  if (!A || !V || !w) {
    free(A); free(V); free(w);
    return ORC_ENOMEM;
  }
  memcpy(A, S, sizeof(double) * (size_t)R * R);
  orc_sym_eig_jacobi(R, A, V, w);
  double wmax = 0.0;
  for (int i = 0; i < R; ++i) wmax = fmax(wmax, fabs(w[i]));
  const double cut = (double)R * 2.220446049250313e-16 * wmax;
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < R; ++j) {
      double s = 0.0;
      for (int k = 0; k < R; ++k)
        if (fabs(w[k]) > cut) s += V[i * R + k] * V[j * R + k] / w[k];
      P[i * R + j] = s;
    }
  free(A); free(V); free(w);
  return ORC_OK;
}

/*
 * Solve X Gamma = N for X (n x R), Gamma symmetric: Cholesky with forward and
 * backward substitution per row, or, if Gamma is not positive definite, X = N
 * pinv(Gamma).  Returns ORC_OK or ORC_ESINGULAR (pseudo-inverse used).
 */
int orc_solve_normal(int64_t n, int R, const double* Gamma, const double* Nmat, double* X) {
  double* L = (double*)malloc(sizeof(double) * (size_t)R * R);
  if (!L) return ORC_ENOMEM;
  memcpy(L, Gamma, sizeof(double) * (size_t)R * R);
  if (chol_lower(R, L) == 0) {
#pragma omp parallel for
    for (int64_t i = 0; i < n; ++i) {
      /* x Gamma = b  <=>  Gamma x^T = b^T  <=>  L L^T x^T = b^T */
      double y[R];
      for (int r = 0; r < R; ++r) {
        double s = Nmat[i * R + r];
        for (int k = 0; k < r; ++k) s -= L[r * R + k] * y[k];
        y[r] = s / L[r * R + r];
      }
      for (int r = R - 1; r >= 0; --r) {
        double s = y[r];
        for (int k = r + 1; k < R; ++k) s -= L[k * R + r] * X[i * R + k];
        X[i * R + r] = s / L[r * R + r];
      }
    }
    free(L);
    return ORC_OK;
  }
  free(L);
  double* P = (double*)malloc(sizeof(double) * (size_t)R * R);
  if (!P) return ORC_ENOMEM;
  int st = orc_pinv_sym(R, Gamma, P);
  if (st != ORC_OK) { free(P); return st; }
#pragma omp parallel for
  for (int64_t i = 0; i < n; ++i)
    for (int r = 0; r < R; ++r) {
      double s = 0.0;
      for (int k = 0; k < R; ++k) s += Nmat[i * R + k] * P[k * R + r];
      X[i * R + r] = s;
    }
  free(P);
  return ORC_ESINGULAR;
}

/* ------------------------------------------------------------------------- */
/* CP-ALS (Algorithm 2, with the MTTKRP of Algorithm 4).                      */
/* ------------------------------------------------------------------------- */

/*
 * One factor update of ALS for `mode`:
 *   N = X^n (F_f kr F_in)                           (Algorithm 4)
 *   Gamma = F_f^T F_f * F_in^T F_in + lambda_reg I  (Eq. als-astep-sol-rw and the
 *                                                    regularized Eq.
 *                                                    tensorapprx-ref-sol)
 *   F_n = N Gamma^{-1}, then normalise its columns  (Algorithm 2)
 * lambda[r] receives the 2-norm of column r before normalisation; a zero column
 * is left as it is with lambda[r] = 0.
 */
int orc_als_mode_update(int mode, int64_t nnz, const int32_t* idx, const float* val,
                        const int32_t* dims, int R, double lambda_reg, double* A,
                        double* B, double* C, double* lambda) {
  double* F[3] = {A, B, C};
  const int o = ax_o(mode), in = ax_in(mode), f = ax_f(mode);
  const int64_t n = dims[o];
  double* Nm = (double*)malloc(sizeof(double) * (size_t)n * R);
  double* Gf = (double*)malloc(sizeof(double) * (size_t)R * R);
  double* Gi = (double*)malloc(sizeof(double) * (size_t)R * R);
  if (!Nm || !Gf || !Gi) {
    free(Nm); free(Gf); free(Gi);
    return ORC_ENOMEM;
  }
  orc_mttkrp(mode, nnz, idx, val, dims, R, A, B, C, Nm);
  orc_gram(dims[f], R, F[f], Gf);
  orc_gram(dims[in], R, F[in], Gi);
  for (int r = 0; r < R; ++r)
    for (int s = 0; s < R; ++s) Gf[r * R + s] *= Gi[r * R + s];
  for (int r = 0; r < R; ++r) Gf[r * R + r] += lambda_reg;
  int st = orc_solve_normal(n, R, Gf, Nm, F[o]);
#pragma omp parallel for
  for (int r = 0; r < R; ++r) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += F[o][i * R + r] * F[o][i * R + r];
    s = sqrt(s);
    lambda[r] = s;
    if (s > 0.0)
      for (int64_t i = 0; i < n; ++i) F[o][i * R + r] /= s;
  }
  free(Nm); free(Gf); free(Gi);
  return st;
}

/* ||X||^2 = sum of squared observed values. */
double orc_norm2(int64_t nnz, const float* val) {
  double s = 0.0;
  for (int64_t t = 0; t < nnz; ++t) s += (double)val[t] * (double)val[t];
  return s;
}

/*
 * <X, [[lambda; A, B, C]]> = sum over observed (i,j,k) of
 * x_ijk * sum_r lambda_r a_ir b_jr c_kr  (Eq. parafac); lambda may be NULL (all 1).
 */
double orc_inner(int64_t nnz, const int32_t* idx, const float* val, int R,
                 const double* lambda, const double* A, const double* B, const double* C) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s)
  for (int64_t t = 0; t < nnz; ++t) {
    const int64_t i = idx[t], j = idx[nnz + t], k = idx[2 * nnz + t];
    double m = 0.0;
    for (int r = 0; r < R; ++r)
      m += (lambda ? lambda[r] : 1.0) * A[i * R + r] * B[j * R + r] * C[k * R + r];
    s += (double)val[t] * m;
  }
  return s;
}

/*
 * ||[[lambda; A, B, C]]||^2 = lambda^T (A^T A * B^T B * C^T C) lambda: the squared
 * norm of a Kruskal tensor, from Eq. kr-product applied twice.
 */
double orc_model_norm2(const int32_t* dims, int R, const double* lambda, const double* A,
                       const double* B, const double* C) {
  double* G[3];
  const double* F[3] = {A, B, C};
  for (int m = 0; m < 3; ++m) {
    G[m] = (double*)malloc(sizeof(double) * (size_t)R * R);
    orc_gram(dims[m], R, F[m], G[m]);
  }
  double s = 0.0;
  for (int r = 0; r < R; ++r)
    for (int q = 0; q < R; ++q) {
      double lr = lambda ? lambda[r] : 1.0, lq = lambda ? lambda[q] : 1.0;
      s += lr * lq * G[0][r * R + q] * G[1][r * R + q] * G[2][r * R + q];
    }
  for (int m = 0; m < 3; ++m) free(G[m]);
  return s;
}

/*
 * Fit of the model of Eq. parafac: 1 - ||X - Xhat|| / ||X||, with
 * ||X - Xhat||^2 = ||X||^2 - 2 <X, Xhat> + ||Xhat||^2 (clamped at 0).
 * The paper never defines a fit; this is the usual CP fit.
 */
double orc_fit(int64_t nnz, const int32_t* idx, const float* val, const int32_t* dims,
               int R, const double* lambda, const double* A, const double* B,
               const double* C) {
  const double nx2 = orc_norm2(nnz, val);
  const double ip = orc_inner(nnz, idx, val, R, lambda, A, B, C);
  const double nm2 = orc_model_norm2(dims, R, lambda, A, B, C);
  double res2 = nx2 - 2.0 * ip + nm2;
  if (res2 < 0.0) res2 = 0.0;
  if (nx2 <= 0.0) return 0.0;
  return 1.0 - sqrt(res2) / sqrt(nx2);
}

/*
 * One ALS sweep: A, then B, then C, each with the latest other factors
 * (Algorithm 2 / Algorithm 4), then the fit of [[lambda; A, B, C]] with lambda
 * from the last (mode-3) normalisation.  Returns the first non-OK status of the
 * three updates (ESINGULAR is informational), the fit in *fit_out (nullable).
 */
int orc_als_sweep(int64_t nnz, const int32_t* idx, const float* val, const int32_t* dims,
                  int R, double lambda_reg, double* A, double* B, double* C,
                  double* lambda, double* fit_out) {
  int worst = ORC_OK;
  for (int mode = 0; mode < 3; ++mode) {
    int st = orc_als_mode_update(mode, nnz, idx, val, dims, R, lambda_reg, A, B, C, lambda);
    if (st == ORC_ENOMEM) return st;
    if (st != ORC_OK && worst == ORC_OK) worst = st;
  }
  if (fit_out) *fit_out = orc_fit(nnz, idx, val, dims, R, lambda, A, B, C);
  return worst;
}

/* ------------------------------------------------------------------------- */
/* CP-GD (Algorithm 3 / Algorithm 5).                                         */
/* ------------------------------------------------------------------------- */

static double frob2(int64_t n, int R, const double* F) {
  double s = 0.0;
  for (int64_t t = 0; t < n * R; ++t) s += F[t] * F[t];
  return s;
}

/*
 * GD objective (Eq. gd-obj-fn, regularized form Eq. gd-obj-fn-reg):
 *   f = 1/2 ||X - [[A,B,C]]||^2 + 1/2 lambda_reg (||A||^2 + ||B||^2 + ||C||^2)
 * with the squared residual expanded as ||X||^2 - 2<X,[[A,B,C]]> + ||[[A,B,C]]||^2
 * (no CP weights: the GD model has none).
 */
double orc_loss(int64_t nnz, const int32_t* idx, const float* val, const int32_t* dims,
                int R, double lambda_reg, const double* A, const double* B, const double* C) {
  const double nx2 = orc_norm2(nnz, val);
  const double ip = orc_inner(nnz, idx, val, R, NULL, A, B, C);
  const double nm2 = orc_model_norm2(dims, R, NULL, A, B, C);
  double f = 0.5 * (nx2 - 2.0 * ip + nm2);
  if (lambda_reg != 0.0)
    f += 0.5 * lambda_reg *
         (frob2(dims[0], R, A) + frob2(dims[1], R, B) + frob2(dims[2], R, C));
  return f;
}

/*
 * Gradients at the current point (Eq. gd-A and its regularized form):
 *   dF_n = -X^n (F_f kr F_in) + F_n (F_f^T F_f * F_in^T F_in + lambda_reg I).
 * Algorithm 5 prints "+N"; Eq. gd-A and Algorithm 3 give -N, which is the
 * derivative of the objective, so -N is used.  All three gradients are taken at
 * the same (A,B,C), as in Algorithm 3/5 where no factor changes before the step.
 */
int orc_gd_gradient(int64_t nnz, const int32_t* idx, const float* val, const int32_t* dims,
                    int R, double lambda_reg, const double* A, const double* B,
                    const double* C, double* GA, double* GB, double* GC) {
  const double* F[3] = {A, B, C};
  double* Gout[3] = {GA, GB, GC};
  double* Gm[3];
  for (int m = 0; m < 3; ++m) {
    Gm[m] = (double*)malloc(sizeof(double) * (size_t)R * R);
    if (!Gm[m]) return ORC_ENOMEM;
    orc_gram(dims[m], R, F[m], Gm[m]);
  }
  double* Gam = (double*)malloc(sizeof(double) * (size_t)R * R);
  for (int mode = 0; mode < 3; ++mode) {
    const int o = ax_o(mode), in = ax_in(mode), f = ax_f(mode);
    const int64_t n = dims[o];
    orc_mttkrp(mode, nnz, idx, val, dims, R, A, B, C, Gout[mode]);
    for (int r = 0; r < R; ++r)
      for (int s = 0; s < R; ++s)
        Gam[r * R + s] = Gm[f][r * R + s] * Gm[in][r * R + s] + (r == s ? lambda_reg : 0.0);
    for (int64_t i = 0; i < n; ++i)
      for (int r = 0; r < R; ++r) {
        double s = 0.0;
        for (int k = 0; k < R; ++k) s += F[o][i * R + k] * Gam[k * R + r];
        Gout[mode][i * R + r] = -Gout[mode][i * R + r] + s;
      }
  }
  for (int m = 0; m < 3; ++m) free(Gm[m]);
  free(Gam);
  return ORC_OK;
}

/*
 * One GD step (Algorithm 5 with the sign of Eq. gd-A):
 *   1. gradients at the current point; g2 = ||grad f||^2 (Eq. grad-f);
 *   2. step size by backtracking (the paper only says a backtracking line search
 *      was used): alpha0 = min(2 * alpha_prev, 1) (1 if alpha_prev <= 0); accept
 *      the first alpha with f(theta - alpha grad) <= f(theta) - 1e-4 alpha g2,
 *      halving up to 100 trials; each trial evaluates f from scratch;
 *   3. A <- A - alpha dA, B <- B - alpha dB, C <- C - alpha dC.
 * On failure the factors are left unchanged and ORC_ELSFAIL is returned.
 * *alpha_io carries alpha_prev in and the accepted alpha out; *loss_out gets the
 * objective at the returned point.
 */
int orc_gd_step(int64_t nnz, const int32_t* idx, const float* val, const int32_t* dims,
                int R, double lambda_reg, double* A, double* B, double* C,
                double* alpha_io, double* loss_out, double* g2_out) {
  double* F[3] = {A, B, C};
  double* G[3];
  double* T[3];
  for (int m = 0; m < 3; ++m) {
    G[m] = (double*)malloc(sizeof(double) * (size_t)dims[m] * R);
    T[m] = (double*)malloc(sizeof(double) * (size_t)dims[m] * R);
    if (!G[m] || !T[m]) return ORC_ENOMEM;
  }
  orc_gd_gradient(nnz, idx, val, dims, R, lambda_reg, A, B, C, G[0], G[1], G[2]);
  double g2 = 0.0;
  for (int m = 0; m < 3; ++m) g2 += frob2(dims[m], R, G[m]);
  const double f0 = orc_loss(nnz, idx, val, dims, R, lambda_reg, A, B, C);
  double alpha = (*alpha_io > 0.0) ? fmin(2.0 * (*alpha_io), 1.0) : 1.0;
  int accepted = 0;
  double fa = f0;
  for (int trial = 0; trial < 100; ++trial) {
    for (int m = 0; m < 3; ++m)
      for (int64_t t = 0; t < (int64_t)dims[m] * R; ++t) T[m][t] = F[m][t] - alpha * G[m][t];
    fa = orc_loss(nnz, idx, val, dims, R, lambda_reg, T[0], T[1], T[2]);
    if (fa <= f0 - 1e-4 * alpha * g2) {
      accepted = 1;
      break;
    }
    alpha *= 0.5;
  }
  if (g2_out) *g2_out = g2;
  int st = ORC_OK;
  if (accepted) {
    for (int m = 0; m < 3; ++m) memcpy(F[m], T[m], sizeof(double) * (size_t)dims[m] * R);
    *alpha_io = alpha;
    if (loss_out) *loss_out = fa;
  } else {
    st = ORC_ELSFAIL;
    if (loss_out) *loss_out = f0;
  }
  for (int m = 0; m < 3; ++m) {
    free(G[m]);
    free(T[m]);
  }
  return st;
}

/*
 * The GD objective along the search ray, phi(alpha) = f(A - alpha GA,
 * B - alpha GB, C - alpha GC) with f of Eq. gd-obj-fn (regularized form
 * Eq. gd-obj-fn-reg), is a polynomial of degree 6 in alpha.  Its coefficients
 * coef[0..6] are taken term by term from the definition:
 *   1/2 ||X||^2;
 *   -<X, [[.]]>: each observed entry contributes x * sum_r of the product of
 *     three linear polynomials (F_n[i_n, r] - alpha G_n[i_n, r]), n = A, B, C;
 *   +1/2 ||[[.]]||^2 = 1/2 sum_rs prod_n M_n(alpha)[r, s] with the Gram
 *     M_n(alpha) = (F_n - alpha G_n)^T (F_n - alpha G_n) (Eq. kr-product),
 *     a quadratic in alpha entry by entry;
 *   +1/2 lambda_reg sum_n ||F_n - alpha G_n||^2.
 * Used by the exact line search, an option beside the backtracking rule.
 */
int orc_gd_ray_poly(int64_t nnz, const int32_t* idx, const float* val, const int32_t* dims,
                    int R, double lambda_reg, const double* A, const double* B,
                    const double* C, const double* GA, const double* GB, const double* GC,
                    double* coef) {
  const double* F[3] = {A, B, C};
  const double* G[3] = {GA, GB, GC};
  for (int k = 0; k < 7; ++k) coef[k] = 0.0;
  coef[0] = 0.5 * orc_norm2(nnz, val);
  /* data term */
  for (int64_t t = 0; t < nnz; ++t) {
    const double x = (double)val[t];
    for (int r = 0; r < R; ++r) {
      double p[4] = {1.0, 0.0, 0.0, 0.0};
      for (int n = 0; n < 3; ++n) {
        const int64_t row = idx[(int64_t)n * nnz + t];
        const double u0 = F[n][row * R + r], u1 = -G[n][row * R + r];
        double q[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < 3; ++k) {
          q[k] += p[k] * u0;
          q[k + 1] += p[k] * u1;
        }
        for (int k = 0; k < 4; ++k) p[k] = q[k];
      }
      for (int k = 0; k < 4; ++k) coef[k] -= x * p[k];
    }
  }
  /* model term: Grams of F_n - alpha G_n as quadratics */
  double* M[3];
  for (int n = 0; n < 3; ++n) {
    M[n] = (double*)calloc((size_t)3 * R * R, sizeof(double));
    if (!M[n]) return ORC_ENOMEM;
    for (int64_t i = 0; i < dims[n]; ++i)
      for (int r = 0; r < R; ++r)
        for (int s = 0; s < R; ++s) {
          const double fr = F[n][i * R + r], fs = F[n][i * R + s];
          const double gr = G[n][i * R + r], gs = G[n][i * R + s];
          M[n][r * R + s] += fr * fs;
          M[n][R * R + r * R + s] -= fr * gs + gr * fs;
          M[n][2 * R * R + r * R + s] += gr * gs;
        }
  }
  for (int e = 0; e < R * R; ++e) {
    double p[7] = {1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int deg = 0;
    for (int n = 0; n < 3; ++n) {
      double q[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int i = 0; i <= deg; ++i)
        for (int j = 0; j < 3; ++j) q[i + j] += p[i] * M[n][j * R * R + e];
      deg += 2;
      for (int i = 0; i <= deg; ++i) p[i] = q[i];
    }
    for (int k = 0; k < 7; ++k) coef[k] += 0.5 * p[k];
  }
  for (int n = 0; n < 3; ++n) free(M[n]);
  /* ridge */
  if (lambda_reg != 0.0)
    for (int n = 0; n < 3; ++n)
      for (int64_t t = 0; t < (int64_t)dims[n] * R; ++t) {
        coef[0] += 0.5 * lambda_reg * F[n][t] * F[n][t];
        coef[1] -= lambda_reg * F[n][t] * G[n][t];
        coef[2] += 0.5 * lambda_reg * G[n][t] * G[n][t];
      }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Joint matrix completion and tensor factorization (Appendix F).            */
/* ------------------------------------------------------------------------- */

/*
 * The model shares the user factor A (rows i) and the item factor B (rows j)
 * between a ratings matrix Y (observed entries (i, j) in Omega^Y, yidx[0][t] =
 * i, yidx[1][t] = j, value yval[t]) and the user x item x word tensor X:
 *   f = 1/2 sum_{(i,j) in Omega^Y} (y_ij - a_i . b_j)^2
 *       + mu 1/2 ||X - [[A, B, C]]||^2 + lambda 1/2 (||A||^2 + ||B||^2 + ||C||^2)
 * (Eq. joint-obj-fn; the tensor term runs over every cell, as in Eq. gd-obj-fn).
 */
double orc_joint_loss(int64_t nnzY, const int32_t* yidx, const float* yval, int64_t nnz,
                      const int32_t* idx, const float* val, const int32_t* dims, int R, double mu,
                      double lambda, const double* A, const double* B, const double* C) {
  double fy = 0.0;
  for (int64_t t = 0; t < nnzY; ++t) {
    const int64_t i = yidx[t], j = yidx[nnzY + t];
    double p = 0.0;
    for (int r = 0; r < R; ++r) p += A[i * R + r] * B[j * R + r];
    const double e = (double)yval[t] - p;
    fy += 0.5 * e * e;
  }
  const double ft = orc_loss(nnz, idx, val, dims, R, 0.0, A, B, C);
  return fy + mu * ft +
         0.5 * lambda * (frob2(dims[0], R, A) + frob2(dims[1], R, B) + frob2(dims[2], R, C));
}

/*
 * Row system of one factor row (Eq. grad-joint-A and the ALS solution below
 * it).  For the user factor (side 0) and row i:
 *   rhs = sum_{j in Omega_i} y_ij b_j + mu N_A[i]          (y_i,: B + mu x^1_i,: (C kr B))
 *   H   = sum_{j in Omega_i} b_j^T b_j + mu (C^T C * B^T B) + lambda I
 * where Omega_i are the observed items of user i (the printed sum over Omega^Y
 * is read as the one over the row, the derivative of Eq. joint-prob-A).  The
 * item factor (side 1) swaps the roles of A and B (Omega_j, N_B, A^T A * C^T C);
 * the word factor (side 2) has no ratings: rhs = mu N_C[k], H = mu (B^T B *
 * A^T A) + lambda I.  N is the mode's MTTKRP, Gam its Gram-Hadamard product.
 */
static void joint_row_system(int side, int64_t row, int64_t nnzY, const int32_t* yidx,
                             const float* yval, int R, double mu, double lambda,
                             const double* other, const double* N, const double* Gam,
                             double* rhs, double* H) {
  for (int r = 0; r < R; ++r) {
    rhs[r] = mu * N[row * R + r];
    for (int s = 0; s < R; ++s) H[r * R + s] = mu * Gam[r * R + s] + (r == s ? lambda : 0.0);
  }
  if (side == 2) return;
  for (int64_t t = 0; t < nnzY; ++t) {
    if (yidx[(int64_t)side * nnzY + t] != row) continue;
    const int64_t o = yidx[(int64_t)(1 - side) * nnzY + t];
    const double y = (double)yval[t];
    for (int r = 0; r < R; ++r) {
      rhs[r] += y * other[o * R + r];
      for (int s = 0; s < R; ++s) H[r * R + s] += other[o * R + r] * other[o * R + s];
    }
  }
}

/* Gram-Hadamard product of the two factors that are not `side` (mode n = side). */
static int joint_gamma(int side, const int32_t* dims, int R, const double* const* F, double* Gam) {
  double* Gf = (double*)malloc(sizeof(double) * (size_t)R * R);
  double* Gi = (double*)malloc(sizeof(double) * (size_t)R * R);
  if (!Gf || !Gi) { free(Gf); free(Gi); return ORC_ENOMEM; }
  orc_gram(dims[ax_f(side)], R, F[ax_f(side)], Gf);
  orc_gram(dims[ax_in(side)], R, F[ax_in(side)], Gi);
  for (int e = 0; e < R * R; ++e) Gam[e] = Gf[e] * Gi[e];
  free(Gf);
  free(Gi);
  return ORC_OK;
}

/*
 * Gradients at the current point, every row by Eq. grad-joint-A:
 *   grad_i = -rhs_i + a_i H_i  (side 0), the same for B (side 1) and C (side 2).
 */
int orc_joint_gradient(int64_t nnzY, const int32_t* yidx, const float* yval, int64_t nnz,
                       const int32_t* idx, const float* val, const int32_t* dims, int R, double mu,
                       double lambda, const double* A, const double* B, const double* C,
                       double* GA, double* GB, double* GC) {
  const double* F[3] = {A, B, C};
  double* Gout[3] = {GA, GB, GC};
  double* N = NULL;
  double* Gam = (double*)malloc(sizeof(double) * (size_t)R * R);
  double* H = (double*)malloc(sizeof(double) * (size_t)R * R);
  double* rhs = (double*)malloc(sizeof(double) * (size_t)R);
  if (!Gam || !H || !rhs) return ORC_ENOMEM;
  for (int side = 0; side < 3; ++side) {
    N = (double*)malloc(sizeof(double) * (size_t)dims[side] * R);
    if (!N) return ORC_ENOMEM;
    orc_mttkrp(side, nnz, idx, val, dims, R, A, B, C, N);
    joint_gamma(side, dims, R, F, Gam);
    const double* other = side == 0 ? B : A;
    for (int64_t row = 0; row < dims[side]; ++row) {
      joint_row_system(side, row, nnzY, yidx, yval, R, mu, lambda, other, N, Gam, rhs, H);
      for (int s = 0; s < R; ++s) {
        double v = -rhs[s];
        for (int r = 0; r < R; ++r) v += F[side][row * R + r] * H[r * R + s];
        Gout[side][row * R + s] = v;
      }
    }
    free(N);
  }
  free(Gam);
  free(H);
  free(rhs);
  return ORC_OK;
}

/*
 * One ALS sweep of the joint model: A row by row (a_i = rhs_i H_i^-1, the
 * closed form of Appendix F), then B with the new A, then C with the new A and
 * B.  H_i is symmetric positive definite when lambda > 0; the solve is the
 * oracle's Cholesky solve (pseudo-inverse when it fails, status ORC_ESINGULAR).
 */
int orc_joint_als_sweep(int64_t nnzY, const int32_t* yidx, const float* yval, int64_t nnz,
                        const int32_t* idx, const float* val, const int32_t* dims, int R,
                        double mu, double lambda, double* A, double* B, double* C) {
  double* F[3] = {A, B, C};
  double* Gam = (double*)malloc(sizeof(double) * (size_t)R * R);
  double* H = (double*)malloc(sizeof(double) * (size_t)R * R);
  double* rhs = (double*)malloc(sizeof(double) * (size_t)R);
  if (!Gam || !H || !rhs) return ORC_ENOMEM;
  int status = ORC_OK;
  for (int side = 0; side < 3; ++side) {
    double* N = (double*)malloc(sizeof(double) * (size_t)dims[side] * R);
    if (!N) return ORC_ENOMEM;
    orc_mttkrp(side, nnz, idx, val, dims, R, A, B, C, N);
    joint_gamma(side, dims, R, (const double* const*)F, Gam);
    const double* other = side == 0 ? B : A;
    for (int64_t row = 0; row < dims[side]; ++row) {
      joint_row_system(side, row, nnzY, yidx, yval, R, mu, lambda, other, N, Gam, rhs, H);
      const int st = orc_solve_normal(1, R, H, rhs, F[side] + row * R);
      if (st == ORC_ESINGULAR) status = ORC_ESINGULAR;
      else if (st != ORC_OK) return st;
    }
    free(N);
  }
  free(Gam);
  free(H);
  free(rhs);
  return status;
}

/*
 * One GD step of the joint model: the three gradients at the current point,
 * then the backtracking rule of orc_gd_step on f of Eq. joint-obj-fn (the
 * paper used backtracking for the joint model), then the update.
 */
int orc_joint_gd_step(int64_t nnzY, const int32_t* yidx, const float* yval, int64_t nnz,
                      const int32_t* idx, const float* val, const int32_t* dims, int R, double mu,
                      double lambda, double* A, double* B, double* C, double* alpha_io,
                      double* loss_out, double* g2_out) {
  double* F[3] = {A, B, C};
  double* G[3];
  double* T[3];
  for (int m = 0; m < 3; ++m) {
    G[m] = (double*)malloc(sizeof(double) * (size_t)dims[m] * R);
    T[m] = (double*)malloc(sizeof(double) * (size_t)dims[m] * R);
    if (!G[m] || !T[m]) return ORC_ENOMEM;
  }
  int st = orc_joint_gradient(nnzY, yidx, yval, nnz, idx, val, dims, R, mu, lambda, A, B, C, G[0],
                              G[1], G[2]);
  if (st != ORC_OK) return st;
  double g2 = 0.0;
  for (int m = 0; m < 3; ++m) g2 += frob2(dims[m], R, G[m]);
  const double f0 = orc_joint_loss(nnzY, yidx, yval, nnz, idx, val, dims, R, mu, lambda, A, B, C);
  double alpha = (*alpha_io > 0.0) ? fmin(2.0 * (*alpha_io), 1.0) : 1.0;
  int accepted = 0;
  double fa = f0;
  for (int trial = 0; trial < 100; ++trial) {
    for (int m = 0; m < 3; ++m)
      for (int64_t t = 0; t < (int64_t)dims[m] * R; ++t) T[m][t] = F[m][t] - alpha * G[m][t];
    fa = orc_joint_loss(nnzY, yidx, yval, nnz, idx, val, dims, R, mu, lambda, T[0], T[1], T[2]);
    if (fa <= f0 - 1e-4 * alpha * g2) {
      accepted = 1;
      break;
    }
    alpha *= 0.5;
  }
  if (g2_out) *g2_out = g2;
  st = ORC_OK;
  if (accepted) {
    for (int m = 0; m < 3; ++m) memcpy(F[m], T[m], sizeof(double) * (size_t)dims[m] * R);
    *alpha_io = alpha;
    if (loss_out) *loss_out = fa;
  } else {
    st = ORC_ELSFAIL;
    if (loss_out) *loss_out = f0;
  }
  for (int m = 0; m < 3; ++m) {
    free(G[m]);
    free(T[m]);
  }
  return st;
}
