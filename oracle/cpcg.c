/*
 * Plain C solvers of the oracle (test infrastructure and the timed CPU
 * baseline only; nothing on the GPU path calls them).
 *
 * oracle_pcg: Algorithm 1 (§3.3), Jacobi-preconditioned CG on a CSR matrix,
 *   in the same order and with the same readings as oracle/pcg.py: stop when
 *   r^T P^-1 r <= rtol^2 b^T P^-1 b, delta_old <- delta_new every iteration,
 *   the true residual recomputed when i > 0 and i % period == 0. The
 *   products and sums run over `threads` OpenMP threads (one thread is the
 *   paper's one-core baseline, §5.2).
 *
 * oracle_ichol: incomplete Cholesky with a drop tolerance (the CPU solver the
 *   paper compares with in Table 2 of §5.2, droptol 1e-3), row by row: row i
 *   of L is l_ik = (a_ik - sum_{m<k} l_im l_km) / l_kk for k < i in increasing
 *   order, fill-in included, and an entry is dropped when
 *   |l_ik| < droptol * ||A(k:n, k)||_1; l_ii = sqrt(a_ii - sum_k l_ik^2). A
 *   non-positive pivot is a breakdown (return 1).
 *
 * oracle_pcg_ic: CG preconditioned by (L L^T)^-1 (two triangular solves per
 *   iteration), with Algorithm 1's stopping rule on r^T P^-1 r (P the Jacobi
 *   diagonal) so that its iteration counts compare with oracle_pcg's.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void spmv(int n, const long long* rp, const int* ci, const double* v, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (long long k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
    y[i] = s;
  }
}

/* sum_i a_i b_i w_i (w NULL: 1) */
static double wdot(int n, const double* a, const double* b, const double* w) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int i = 0; i < n; ++i) s += a[i] * b[i] * (w ? w[i] : 1.0);
  return s;
}

static void set_threads(int threads) {
#ifdef _OPENMP
  omp_set_num_threads(threads > 0 ? threads : 1);
#else
  (void)threads;
#endif
}

int oracle_threads_available(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

/* x (in: x0, out: solution); out[0] iterations, out[1] delta_final, out[2] delta_b */
int oracle_pcg(int n, const long long* rp, const int* ci, const double* v, const double* b, double* x,
               const double* pinv, double rtol, int max_iter, int period, int threads, double* out) {
  set_threads(threads);
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  if (!r || !d || !q || !s) {
    free(r); free(d); free(q); free(s);
    return 2;
  }
  spmv(n, rp, ci, v, x, q);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    r[i] = b[i] - q[i];
    d[i] = pinv[i] * r[i];
  }
  double delta_new = wdot(n, r, d, NULL);
  const double delta_b = wdot(n, b, b, pinv);
  const double threshold = rtol * rtol * delta_b;
  int it = 0;
  while (it < max_iter && delta_new > threshold) {
    spmv(n, rp, ci, v, d, q);
    const double alpha = delta_new / wdot(n, d, q, NULL);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) x[i] += alpha * d[i];
    if (it > 0 && it % period == 0) {
      spmv(n, rp, ci, v, x, q);
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
    } else {
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) r[i] -= alpha * q[i];
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) s[i] = pinv[i] * r[i];
    const double delta_old = delta_new;
    delta_new = wdot(n, r, s, NULL);
    const double beta = delta_new / delta_old;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) d[i] = s[i] + beta * d[i];
    ++it;
  }
  out[0] = (double)it;
  out[1] = delta_new;
  out[2] = delta_b;
  free(r); free(d); free(q); free(s);
  return 0;
}

/* ------------------------------------------------------------------ IC(tau) */

typedef struct {
  int n;
  long long nnz, cap;
  long long* rp;   /* rows of L, strictly lower part, columns increasing */
  int* ci;
  int* row;        /* the row of each stored entry */
  double* v;
  double* diag;
  long long* next; /* column lists: entries of column k in row order */
  long long* head;
  long long* tail;
} ICFactor;

static void heap_push(int* h, int* hn, int x) {
  int i = (*hn)++;
  h[i] = x;
  while (i > 0) {
    const int p = (i - 1) / 2;
    if (h[p] <= h[i]) break;
    const int t = h[p];
    h[p] = h[i];
    h[i] = t;
    i = p;
  }
}

static int heap_pop(int* h, int* hn) {
  const int top = h[0];
  h[0] = h[--(*hn)];
  int i = 0;
  for (;;) {
    const int l = 2 * i + 1, r = l + 1;
    int m = i;
    if (l < *hn && h[l] < h[m]) m = l;
    if (r < *hn && h[r] < h[m]) m = r;
    if (m == i) break;
    const int t = h[m];
    h[m] = h[i];
    h[i] = t;
    i = m;
  }
  return top;
}

void oracle_ichol_free(void* f) {
  ICFactor* F = (ICFactor*)f;
  if (!F) return;
  free(F->rp); free(F->ci); free(F->row); free(F->v); free(F->diag); free(F->next); free(F->head); free(F->tail);
  free(F);
}

/* A: full symmetric CSR (both triangles). Returns 0 and *out on success,
   1 on a breakdown (non-positive pivot), 2 when out of memory. */
int oracle_ichol(int n, const long long* rp, const int* ci, const double* v, double droptol, void** out,
                 long long* nnz_out) {
  *out = NULL;
  double* colnorm = (double*)calloc((size_t)n, sizeof(double));
  double* w = (double*)calloc((size_t)n, sizeof(double));
  char* mark = (char*)calloc((size_t)n, 1);
  int* heap = (int*)malloc(sizeof(int) * (size_t)n);
  ICFactor* F = (ICFactor*)calloc(1, sizeof(ICFactor));
  if (!colnorm || !w || !mark || !heap || !F) goto oom;
  F->n = n;
  F->cap = 16 * (long long)n + 16;
  F->rp = (long long*)malloc(sizeof(long long) * ((size_t)n + 1));
  F->ci = (int*)malloc(sizeof(int) * (size_t)F->cap);
  F->row = (int*)malloc(sizeof(int) * (size_t)F->cap);
  F->v = (double*)malloc(sizeof(double) * (size_t)F->cap);
  F->next = (long long*)malloc(sizeof(long long) * (size_t)F->cap);
  F->diag = (double*)malloc(sizeof(double) * (size_t)n);
  F->head = (long long*)malloc(sizeof(long long) * (size_t)n);
  F->tail = (long long*)malloc(sizeof(long long) * (size_t)n);
  if (!F->rp || !F->ci || !F->row || !F->v || !F->next || !F->diag || !F->head || !F->tail) goto oom;
  for (int k = 0; k < n; ++k) F->head[k] = F->tail[k] = -1;
  /* ||A(k:n, k)||_1 = sum over rows i >= k of |a_ik| = sum over row k's entries with column >= k (symmetry) */
  for (int k = 0; k < n; ++k)
    for (long long e = rp[k]; e < rp[k + 1]; ++e)
      if (ci[e] >= k) colnorm[k] += fabs(v[e]);
  F->rp[0] = 0;
  for (int i = 0; i < n; ++i) {
    int hn = 0;
    double wii = 0.0;
    for (long long e = rp[i]; e < rp[i + 1]; ++e) {
      const int k = ci[e];
      if (k < i) {
        if (!mark[k]) {
          mark[k] = 1;
          heap_push(heap, &hn, k);
        }
        w[k] += v[e];
      } else if (k == i) {
        wii += v[e];
      }
    }
    while (hn > 0) {
      const int k = heap_pop(heap, &hn);
      mark[k] = 0;
      const double lik = w[k] / F->diag[k];
      w[k] = 0.0;
      if (fabs(lik) < droptol * colnorm[k]) continue;  /* dropped */
      /* the rows j of column k computed so far (k < j < i): w_j -= l_ik l_jk */
      for (long long e = F->head[k]; e >= 0; e = F->next[e]) {
        const int j = F->row[e];
        if (!mark[j]) {
          mark[j] = 1;
          heap_push(heap, &hn, j);
        }
        w[j] -= lik * F->v[e];
      }
      /* store l_ik: row i of L, and the tail of column k's list */
      if (F->nnz == F->cap) {
        const long long cap = 2 * F->cap;
        int* ci2 = (int*)realloc(F->ci, sizeof(int) * (size_t)cap);
        if (ci2) F->ci = ci2;
        int* r2 = (int*)realloc(F->row, sizeof(int) * (size_t)cap);
        if (r2) F->row = r2;
        double* v2 = (double*)realloc(F->v, sizeof(double) * (size_t)cap);
        if (v2) F->v = v2;
        long long* n2 = (long long*)realloc(F->next, sizeof(long long) * (size_t)cap);
        if (n2) F->next = n2;
        if (!ci2 || !r2 || !v2 || !n2) goto oom;
        F->cap = cap;
      }
      const long long pos = F->nnz++;
      F->ci[pos] = k;
      F->row[pos] = i;
      F->v[pos] = lik;
      F->next[pos] = -1;
      if (F->tail[k] < 0) F->head[k] = pos;
      else F->next[F->tail[k]] = pos;
      F->tail[k] = pos;
      wii -= lik * lik;
    }
    if (!(wii > 0.0)) {
      free(colnorm); free(w); free(mark); free(heap);
      oracle_ichol_free(F);
      return 1;
    }
    F->diag[i] = sqrt(wii);
    F->rp[i + 1] = F->nnz;
  }
  free(colnorm); free(w); free(mark); free(heap);
  *out = F;
  *nnz_out = F->nnz;
  return 0;
oom:
  free(colnorm); free(w); free(mark); free(heap);
  oracle_ichol_free(F);
  return 2;
}

/* L's entries: rp (n+1), ci, v (strictly lower part) and diag (n). */
void oracle_ichol_export(const void* f, long long* rp, int* ci, double* v, double* diag) {
  const ICFactor* F = (const ICFactor*)f;
  memcpy(rp, F->rp, sizeof(long long) * ((size_t)F->n + 1));
  memcpy(ci, F->ci, sizeof(int) * (size_t)F->nnz);
  memcpy(v, F->v, sizeof(double) * (size_t)F->nnz);
  memcpy(diag, F->diag, sizeof(double) * (size_t)F->n);
}

/* z = (L L^T)^-1 r: forward L y = r by rows, backward L^T z = y by rows taken
   from the last (each row's entries scatter into the earlier unknowns). */
static void ic_apply(const ICFactor* F, const double* r, double* z) {
  const int n = F->n;
  for (int i = 0; i < n; ++i) {
    double s = r[i];
    for (long long e = F->rp[i]; e < F->rp[i + 1]; ++e) s -= F->v[e] * z[F->ci[e]];
    z[i] = s / F->diag[i];
  }
  for (int i = n - 1; i >= 0; --i) {
    z[i] /= F->diag[i];
    const double zi = z[i];
    for (long long e = F->rp[i]; e < F->rp[i + 1]; ++e) z[F->ci[e]] -= F->v[e] * zi;
  }
}

/* CG preconditioned by (L L^T)^-1, one thread. out as oracle_pcg. */
int oracle_pcg_ic(int n, const long long* rp, const int* ci, const double* v, const double* b, double* x,
                  const double* pinv, const void* f, double rtol, int max_iter, double* out) {
  set_threads(1);
  const ICFactor* F = (const ICFactor*)f;
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  if (!r || !d || !q || !z) {
    free(r); free(d); free(q); free(z);
    return 2;
  }
  spmv(n, rp, ci, v, x, q);
  for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
  ic_apply(F, r, z);
  memcpy(d, z, sizeof(double) * (size_t)n);
  double rz = wdot(n, r, z, NULL);
  const double delta_b = wdot(n, b, b, pinv);
  const double threshold = rtol * rtol * delta_b;
  double rpr = wdot(n, r, r, pinv);
  int it = 0;
  while (it < max_iter && rpr > threshold) {
    spmv(n, rp, ci, v, d, q);
    const double alpha = rz / wdot(n, d, q, NULL);
    for (int i = 0; i < n; ++i) {
      x[i] += alpha * d[i];
      r[i] -= alpha * q[i];
    }
    ic_apply(F, r, z);
    const double rz_new = wdot(n, r, z, NULL);
    const double beta = rz_new / rz;
    rz = rz_new;
    for (int i = 0; i < n; ++i) d[i] = z[i] + beta * d[i];
    rpr = wdot(n, r, r, pinv);
    ++it;
  }
  out[0] = (double)it;
  out[1] = rpr;
  out[2] = delta_b;
  free(r); free(d); free(q); free(z);
  return 0;
}
