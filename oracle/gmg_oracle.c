/*
 * CPU oracle of the multigrid solve (Alg. 1 "Multigrid solver" and Alg. 2
 * "Multigrid Iteration (V-cycle)"), plain FP64 C.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference the CUDA library is checked against; only the tests, the smoke
 * check and the bench's CPU-baseline leg may load it.  It shares no code with
 * the CUDA library.
 *
 * What it computes, in the paper's order:
 *   setup  (Alg. 1): A_1 = A; A_{l+1} = P_l^T A_l P_l for every given P_l;
 *                    a dense Cholesky factor of the coarsest A_lambda.
 *   MGI    (Alg. 2): pre-relaxation, residual, restriction P_l^T r, recursive
 *                    call with zero initial guess, prolongation and
 *                    correction, post-relaxation; direct solve on the
 *                    coarsest level.
 *   solve  (Alg. 1): repeat x <- MGI(x, b, 1) until ||A x - b|| <= eps ||b||.
 *
 * Readings of the paper that this file fixes:
 *   - the post-relaxation starts from y + P_l u, where y is the pre-relaxed
 *     iterate (the paper prints x + P_l u in Alg. 2);
 *   - relaxation is multicolour Gauss-Seidel: each level's colouring is the
 *     one with fewer colours of two greedy first-fit colourings (increasing
 *     row index; smallest-last order), each improved by iterated-greedy
 *     passes, unless the caller gives one; pre-relaxation visits colours in
 *     ascending order, post-relaxation in descending order (a symmetric cycle),
 *     or ascending when `post_forward` is set;
 *   - the Galerkin product adds its terms (P_iJ P_jK) A_ij in a fixed order,
 *     each with one rounding (C99 fma), and is mirrored to exact symmetry: for
 *     J > K the entry (J, K) takes the value computed for (K, J);
 *   - the convergence test uses the Euclidean 2-norm and runs after every
 *     cycle (repeat-until); b = 0 returns x = 0 after 0 cycles;
 *   - the coarsest level is solved with a dense Cholesky factorisation.
 *
 * Compile with -ffp-contract=off so results do not depend on the host's FMA
 * contraction rules.
 *
 * The default build is single-threaded.  Built with -fopenmp, the loops over
 * independent rows (the rows of one colour in a Gauss-Seidel sweep, the rows
 * of a residual, product or prolongation, the coarse rows of the Galerkin
 * product, the rows below a Cholesky pivot) run on all host cores with the
 * same arithmetic per row, so those results are bit-identical to the
 * single-threaded build; only the dot products and norms of the outer
 * iteration sum in a thread-dependent order.  The threaded build serves only
 * as the timed all-cores CPU baseline; the parity tests use the default one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXLEV 32

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_NOT_SPD = 2, OR_ERR_EMPTY_COL = 3, OR_ERR_CHOL = 4, OR_ERR_NOT_CONV = 5 };

typedef struct {
  int64_t n, nnz;
  int64_t *rowptr;
  int32_t *col;
  double *val;
  int32_t *color;   /* greedy colour of each row */
  int ncolor;
  int64_t *cstart;  /* rows of colour c are crows[cstart[c] .. cstart[c+1]) */
  int32_t *crows;
  /* prolongation P_l to the next level (absent on the coarsest) */
  int64_t nc;
  int32_t *pidx;    /* 3 per row */
  double *pw;       /* 3 per row, 0 = unused slot */
  double *x, *b, *r;
} olevel;

typedef struct {
  int nlev;
  olevel lev[OR_MAXLEV];
  double *chol;     /* dense lower factor of the coarsest operator, row-major */
  int nu_pre, nu_post, post_forward;
} octx;

static void *xmalloc(size_t n) { return malloc(n ? n : 1); }

/* Rows of each colour, ascending: rows of colour c are crows[cstart[c] ..
 * cstart[c+1]). */
static void color_classes(olevel *L) {
  int64_t n = L->n;
  int ncolor = L->ncolor;
  L->cstart = (int64_t *)calloc((size_t)ncolor + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) L->cstart[L->color[i] + 1]++;
  for (int c = 0; c < ncolor; ++c) L->cstart[c + 1] += L->cstart[c];
  int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)ncolor);
  memcpy(fill, L->cstart, sizeof(int64_t) * (size_t)ncolor);
  L->crows = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) L->crows[fill[L->color[i]]++] = (int32_t)i;
  free(fill);
}

/* First fit along `order`: each row in turn takes the smallest colour that no
 * neighbour coloured before it in this pass has.  Returns the colour count. */
static int first_fit(const olevel *L, const int32_t *order, int32_t *color) {
  int64_t n = L->n;
  int64_t *seen = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t c = 0; c <= n; ++c) seen[c] = -1;
  for (int64_t i = 0; i < n; ++i) color[i] = -1;
  int ncolor = 0;
  for (int64_t step = 0; step < n; ++step) {
    int32_t i = order[step];
    for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) {
      int32_t j = L->col[k];
      if (j != i && color[j] >= 0) seen[color[j]] = step;
    }
    int32_t c = 0;
    while (seen[c] == step) ++c;
    color[i] = c;
    if (c + 1 > ncolor) ncolor = c + 1;
  }
  free(seen);
  return ncolor;
}

/* Iterated greedy (Culberson): visit the colour classes from the highest
 * colour to colour 0, rows in increasing index inside a class, and colour
 * them again by first fit.  The count never grows. */
static int recolour(const olevel *L, int ncolor, int32_t *color) {
  int64_t n = L->n;
  int32_t *order = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)n);
  int64_t pos = 0;
  for (int c = ncolor - 1; c >= 0; --c)
    for (int64_t i = 0; i < n; ++i)
      if (color[i] == c) order[pos++] = (int32_t)i;
  int nc = first_fit(L, order, color);
  free(order);
  return nc;
}

/* Smallest-last order (Matula-Beck): repeatedly take out a row with the
 * fewest neighbours still present and list the rows in reverse order of
 * removal.  Rows with the same count form a stack: the initial stacks hold
 * the rows with the smallest index on top, a row whose count drops is put on
 * top of its new stack (neighbours handled in pattern order), and the row
 * taken out is the top of the lowest non-empty stack. */
static void smallest_last_order(const olevel *L, int32_t *order) {
  int64_t n = L->n;
  int32_t *cnt = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)n);
  int32_t *up = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)n);   /* toward the top */
  int32_t *down = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)n); /* toward the bottom */
  char *out = (char *)calloc((size_t)n, 1);
  int maxc = 0;
  for (int64_t i = 0; i < n; ++i) {
    int c = 0;
    for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k)
      if (L->col[k] != i) ++c;
    cnt[i] = c;
    if (c > maxc) maxc = c;
  }
  int32_t *top = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(maxc + 1));
  for (int c = 0; c <= maxc; ++c) top[c] = -1;
#define OR_PUT(v, c) do { down[v] = top[c]; up[v] = -1; if (top[c] >= 0) up[top[c]] = (v); top[c] = (v); } while (0)
#define OR_TAKE(v, c) do { if (up[v] >= 0) down[up[v]] = down[v]; else top[c] = down[v]; \
                           if (down[v] >= 0) up[down[v]] = up[v]; } while (0)
  for (int64_t i = n - 1; i >= 0; --i) OR_PUT((int32_t)i, cnt[i]);
  int low = 0;
  for (int64_t left = n; left > 0; --left) {
    if (low > 0) --low; /* one removal lowers the minimum count by at most one */
    while (top[low] < 0) ++low;
    int32_t v = top[low];
    OR_TAKE(v, low);
    out[v] = 1;
    order[left - 1] = v;
    for (int64_t k = L->rowptr[v]; k < L->rowptr[v + 1]; ++k) {
      int32_t u = L->col[k];
      if (u == v || out[u]) continue;
      OR_TAKE(u, cnt[u]);
      cnt[u] -= 1;
      OR_PUT(u, cnt[u]);
    }
  }
#undef OR_PUT
#undef OR_TAKE
  free(cnt); free(up); free(down); free(out); free(top);
}

#define OR_RECOLOUR_PASSES 8

/* The colouring of a level: first fit in increasing row index and first fit
 * in smallest-last order, each followed by OR_RECOLOUR_PASSES iterated-greedy
 * passes; the one with fewer colours is kept (the first on a tie). */
static void greedy_color(olevel *L) {
  int64_t n = L->n;
  int32_t *order = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)n);
  int32_t *ca = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)n);
  int32_t *cb = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
  int na = first_fit(L, order, ca);
  for (int p = 0; p < OR_RECOLOUR_PASSES; ++p) na = recolour(L, na, ca);
  smallest_last_order(L, order);
  int nb = first_fit(L, order, cb);
  for (int p = 0; p < OR_RECOLOUR_PASSES; ++p) nb = recolour(L, nb, cb);
  if (nb < na) { L->color = cb; L->ncolor = nb; free(ca); }
  else { L->color = ca; L->ncolor = na; free(cb); }
  free(order);
  color_classes(L);
}

/* A given colouring: every colour in [0, n), no two adjacent rows alike
 * (otherwise OR_ERR_ARG). */
static int given_color(olevel *L, const int32_t *color) {
  int64_t n = L->n;
  int ncolor = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (color[i] < 0 || color[i] >= n) return OR_ERR_ARG;
    if (color[i] + 1 > ncolor) ncolor = color[i] + 1;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k)
      if (L->col[k] != i && color[L->col[k]] == color[i]) return OR_ERR_ARG;
  L->color = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)n);
  memcpy(L->color, color, sizeof(int32_t) * (size_t)n);
  L->ncolor = ncolor;
  color_classes(L);
  return OR_OK;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Galerkin coarse operator A_c = P^T A P (Alg. 1, build level matrix).
 * Entry (J, K) = sum_i sum_j (P_iJ P_jK) A_ij, accumulated for each coarse row J
 * over the fine rows i of column J of P (ascending), the entries j of row i of
 * A (ascending) and the slots of row j of P, each term added with a fused
 * multiply-add (one rounding), then mirrored to exact symmetry. */
static int galerkin(const olevel *F, olevel *C) {
  int64_t nf = F->n, nc = F->nc;
  /* columns of P: fine rows i with P_iJ != 0, ascending i */
  int64_t *tp = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  for (int64_t i = 0; i < nf; ++i)
    for (int s = 0; s < 3; ++s)
      if (F->pw[3 * i + s] != 0.0) tp[F->pidx[3 * i + s] + 1]++;
  for (int64_t J = 0; J < nc; ++J) {
    if (tp[J + 1] == 0) { free(tp); return OR_ERR_EMPTY_COL; }
    tp[J + 1] += tp[J];
  }
  int32_t *ti = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)tp[nc]);
  double *tw = (double *)xmalloc(sizeof(double) * (size_t)tp[nc]);
  int64_t *fill = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)nc);
  memcpy(fill, tp, sizeof(int64_t) * (size_t)nc);
  for (int64_t i = 0; i < nf; ++i)
    for (int s = 0; s < 3; ++s)
      if (F->pw[3 * i + s] != 0.0) {
        int64_t q = fill[F->pidx[3 * i + s]]++;
        ti[q] = (int32_t)i;
        tw[q] = F->pw[3 * i + s];
      }
  free(fill);

  /* every coarse row J on its own (private accumulator per thread), kept in
     a buffer of its own, then concatenated in row order */
  int32_t **rcol = (int32_t **)xmalloc(sizeof(int32_t *) * (size_t)nc);
  double **rval = (double **)xmalloc(sizeof(double *) * (size_t)nc);
  int64_t *rlen = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)nc);
#pragma omp parallel
  {
    double *acc = (double *)xmalloc(sizeof(double) * (size_t)nc);
    int64_t *mark = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)nc);
    for (int64_t K = 0; K < nc; ++K) mark[K] = -1;
    int32_t *touched = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)nc);
#pragma omp for schedule(dynamic, 64)
    for (int64_t J = 0; J < nc; ++J) {
      int64_t nt = 0;
      for (int64_t q = tp[J]; q < tp[J + 1]; ++q) {
        int32_t i = ti[q];
        double wiJ = tw[q];
        for (int64_t k = F->rowptr[i]; k < F->rowptr[i + 1]; ++k) {
          int32_t j = F->col[k];
          double a = F->val[k];
          for (int s = 0; s < 3; ++s) {
            double wjK = F->pw[3 * j + s];
            if (wjK == 0.0) continue;
            int32_t K = F->pidx[3 * j + s];
            if (mark[K] != J) { mark[K] = J; acc[K] = 0.0; touched[nt++] = K; }
            acc[K] = fma(wiJ * wjK, a, acc[K]);
          }
        }
      }
      qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
      rcol[J] = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)nt);
      rval[J] = (double *)xmalloc(sizeof(double) * (size_t)nt);
      rlen[J] = nt;
      for (int64_t q = 0; q < nt; ++q) { rcol[J][q] = touched[q]; rval[J][q] = acc[touched[q]]; }
    }
    free(acc); free(mark); free(touched);
  }
  int64_t *crp = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)(nc + 1));
  crp[0] = 0;
  for (int64_t J = 0; J < nc; ++J) crp[J + 1] = crp[J] + rlen[J];
  int64_t nnz = crp[nc];
  int32_t *ccol = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)nnz);
  double *cval = (double *)xmalloc(sizeof(double) * (size_t)nnz);
  for (int64_t J = 0; J < nc; ++J) {
    memcpy(ccol + crp[J], rcol[J], sizeof(int32_t) * (size_t)rlen[J]);
    memcpy(cval + crp[J], rval[J], sizeof(double) * (size_t)rlen[J]);
    free(rcol[J]); free(rval[J]);
  }
  free(rcol); free(rval); free(rlen);
  /* mirror: the lower entry takes the upper entry's value */
  for (int64_t J = 0; J < nc; ++J)
    for (int64_t k = crp[J]; k < crp[J + 1]; ++k) {
      int32_t K = ccol[k];
      if (K >= J) continue;
      int64_t lo = crp[K], hi = crp[K + 1] - 1;
      while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (ccol[mid] < J) lo = mid + 1;
        else if (ccol[mid] > J) hi = mid - 1;
        else { cval[k] = cval[mid]; break; }
      }
    }
  free(tp); free(ti); free(tw);
  C->n = nc;
  C->nnz = nnz;
  C->rowptr = crp;
  C->col = ccol;
  C->val = cval;
  return OR_OK;
}

static double diag_of(const olevel *L, int64_t i) {
  for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k)
    if (L->col[k] == i) return L->val[k];
  return 0.0;
}

/* Dense Cholesky A = L L^T, column by column: L_jj = sqrt(A_jj - sum_{k<j}
 * L_jk^2), then L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj for i > j (each
 * sum over k ascending). */
static int dense_cholesky(const olevel *C, double *Lf) {
  int64_t n = C->n;
  memset(Lf, 0, sizeof(double) * (size_t)(n * n));
  double *Ad = (double *)calloc((size_t)(n * n), sizeof(double));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = C->rowptr[i]; k < C->rowptr[i + 1]; ++k) Ad[i * n + C->col[k]] = C->val[k];
  for (int64_t j = 0; j < n; ++j) {
    double d = Ad[j * n + j];
    for (int64_t k = 0; k < j; ++k) d -= Lf[j * n + k] * Lf[j * n + k];
    if (!(d > 0.0)) { free(Ad); return OR_ERR_CHOL; }
    const double ljj = sqrt(d);
    Lf[j * n + j] = ljj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; ++i) {
      double s = Ad[i * n + j];
      for (int64_t k = 0; k < j; ++k) s -= Lf[i * n + k] * Lf[j * n + k];
      Lf[i * n + j] = s / ljj;
    }
  }
  free(Ad);
  return OR_OK;
}

/* ---------------------------------------------------------------- public */

void or_destroy(octx *c) {
  if (!c) return;
  for (int l = 0; l < c->nlev; ++l) {
    olevel *L = &c->lev[l];
    free(L->rowptr); free(L->col); free(L->val); free(L->color); free(L->cstart); free(L->crows);
    free(L->pidx); free(L->pw); free(L->x); free(L->b); free(L->r);
  }
  free(c->chol);
  free(c);
}

/* Setup of Alg. 1: copies A and the prolongations, forms every Galerkin level,
 * colours every level (the given colouring of a level when `coloring` holds one
 * for it, else greedy first fit) and factors the coarsest one. */
int or_create(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val, int nP,
              const int64_t *ncoarse, const int32_t *const *pidx, const double *const *pw,
              int nu_pre, int nu_post, int post_forward, const int32_t *const *coloring, octx **out) {
  *out = NULL;
  if (nP < 0 || nP + 1 > OR_MAXLEV || n <= 0) return OR_ERR_ARG;
  octx *c = (octx *)calloc(1, sizeof(octx));
  c->nlev = nP + 1;
  c->nu_pre = nu_pre;
  c->nu_post = nu_post;
  c->post_forward = post_forward;
  olevel *L0 = &c->lev[0];
  L0->n = n;
  L0->nnz = rowptr[n];
  L0->rowptr = (int64_t *)xmalloc(sizeof(int64_t) * (size_t)(n + 1));
  L0->col = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)L0->nnz);
  L0->val = (double *)xmalloc(sizeof(double) * (size_t)L0->nnz);
  memcpy(L0->rowptr, rowptr, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(L0->col, col, sizeof(int32_t) * (size_t)L0->nnz);
  memcpy(L0->val, val, sizeof(double) * (size_t)L0->nnz);
  for (int l = 0; l < c->nlev; ++l) {
    olevel *F = &c->lev[l];
    for (int64_t i = 0; i < F->n; ++i)
      if (!(diag_of(F, i) > 0.0)) { or_destroy(c); return OR_ERR_NOT_SPD; }
    F->x = (double *)calloc((size_t)F->n, sizeof(double));
    F->b = (double *)calloc((size_t)F->n, sizeof(double));
    F->r = (double *)calloc((size_t)F->n, sizeof(double));
    if (coloring && coloring[l]) {
      if (given_color(F, coloring[l])) { or_destroy(c); return OR_ERR_ARG; }
    } else {
      greedy_color(F);
    }
    if (l == nP) break;
    F->nc = ncoarse[l];
    F->pidx = (int32_t *)xmalloc(sizeof(int32_t) * (size_t)(3 * F->n));
    F->pw = (double *)xmalloc(sizeof(double) * (size_t)(3 * F->n));
    memcpy(F->pidx, pidx[l], sizeof(int32_t) * (size_t)(3 * F->n));
    memcpy(F->pw, pw[l], sizeof(double) * (size_t)(3 * F->n));
    for (int64_t q = 0; q < 3 * F->n; ++q)
      if (F->pidx[q] < 0 || F->pidx[q] >= F->nc) { or_destroy(c); return OR_ERR_ARG; }
    int st = galerkin(F, &c->lev[l + 1]);
    if (st) { or_destroy(c); return st; }
  }
  olevel *C = &c->lev[c->nlev - 1];
  c->chol = (double *)xmalloc(sizeof(double) * (size_t)(C->n * C->n));
  int st = dense_cholesky(C, c->chol);
  if (st) { or_destroy(c); return st; }
  *out = c;
  return OR_OK;
}

int or_nlev(const octx *c) { return c->nlev; }

void or_level_dims(const octx *c, int l, int64_t *n, int64_t *nnz, int *ncolor) {
  *n = c->lev[l].n;
  *nnz = c->lev[l].nnz;
  *ncolor = c->lev[l].ncolor;
}

void or_level_export(const octx *c, int l, int64_t *rowptr, int32_t *col, double *val, int32_t *color) {
  const olevel *L = &c->lev[l];
  if (rowptr) memcpy(rowptr, L->rowptr, sizeof(int64_t) * (size_t)(L->n + 1));
  if (col) memcpy(col, L->col, sizeof(int32_t) * (size_t)L->nnz);
  if (val) memcpy(val, L->val, sizeof(double) * (size_t)L->nnz);
  if (color) memcpy(color, L->color, sizeof(int32_t) * (size_t)L->n);
}

void or_chol_export(const octx *c, double *Lf) {
  int64_t n = c->lev[c->nlev - 1].n;
  memcpy(Lf, c->chol, sizeof(double) * (size_t)(n * n));
}

/* Relax (Alg. 2): `nsweep` multicolour Gauss-Seidel sweeps on level l.  For a
 * row i of the current colour: x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii with
 * the current values of x; rows of one colour are never adjacent. */
void or_smooth(const octx *c, int l, double *x, const double *b, int nsweep, int descending) {
  const olevel *L = &c->lev[l];
  for (int s = 0; s < nsweep; ++s)
    for (int q = 0; q < L->ncolor; ++q) {
      int cc = descending ? L->ncolor - 1 - q : q;
#pragma omp parallel for schedule(static)
      for (int64_t p = L->cstart[cc]; p < L->cstart[cc + 1]; ++p) {
        int32_t i = L->crows[p];
        double sum = b[i], d = 0.0;
        for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) {
          int32_t j = L->col[k];
          if (j == i) d = L->val[k];
          else sum -= L->val[k] * x[j];
        }
        x[i] = sum / d;
      }
    }
}

/* r = b - A_l x */
void or_residual(const octx *c, int l, const double *x, const double *b, double *r) {
  const olevel *L = &c->lev[l];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < L->n; ++i) {
    double s = b[i];
    for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) s -= L->val[k] * x[L->col[k]];
    r[i] = s;
  }
}

/* y = A_l x */
void or_apply(const octx *c, int l, const double *x, double *y) {
  const olevel *L = &c->lev[l];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < L->n; ++i) {
    double s = 0.0;
    for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) s += L->val[k] * x[L->col[k]];
    y[i] = s;
  }
}

/* bc = P_l^T r */
void or_restrict(const octx *c, int l, const double *r, double *bc) {
  const olevel *L = &c->lev[l];
  memset(bc, 0, sizeof(double) * (size_t)L->nc);
  for (int64_t i = 0; i < L->n; ++i)
    for (int s = 0; s < 3; ++s)
      if (L->pw[3 * i + s] != 0.0) bc[L->pidx[3 * i + s]] += L->pw[3 * i + s] * r[i];
}

/* x += P_l u */
void or_prolong_add(const octx *c, int l, const double *u, double *x) {
  const olevel *L = &c->lev[l];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < L->n; ++i)
    for (int s = 0; s < 3; ++s)
      if (L->pw[3 * i + s] != 0.0) x[i] += L->pw[3 * i + s] * u[L->pidx[3 * i + s]];
}

/* Direct solve on the coarsest level (Alg. 2): L y = b, then L^T x = y. */
void or_coarse_solve(const octx *c, const double *b, double *x) {
  int64_t n = c->lev[c->nlev - 1].n;
  const double *Lf = c->chol;
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int64_t k = 0; k < i; ++k) s -= Lf[i * n + k] * x[k];
    x[i] = s / Lf[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int64_t k = i + 1; k < n; ++k) s -= Lf[k * n + i] * x[k];
    x[i] = s / Lf[i * n + i];
  }
}

/* MGI(x, b, l) of Alg. 2; x is updated in place. */
void or_mgi(const octx *c, int l, double *x, const double *b) {
  if (l == c->nlev - 1) { or_coarse_solve(c, b, x); return; }
  const olevel *L = &c->lev[l];
  const olevel *C = &c->lev[l + 1];
  or_smooth(c, l, x, b, c->nu_pre, 0);                 /* y = Relax(A_l, x, b) */
  or_residual(c, l, x, b, L->r);                       /* b - A_l y            */
  or_restrict(c, l, L->r, C->b);                       /* P_l^T (b - A_l y)    */
  memset(C->x, 0, sizeof(double) * (size_t)C->n);
  or_mgi(c, l + 1, C->x, C->b);                        /* u = MGI(0, ., l+1)   */
  or_prolong_add(c, l, C->x, x);                       /* y + P_l u            */
  or_smooth(c, l, x, b, c->nu_post, !c->post_forward); /* Relax(A_l, ., b)     */
}

static double norm2(const double *v, int64_t n) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < n; ++i) s += v[i] * v[i];
  return sqrt(s);
}
static double dotp(const double *a, const double *b, int64_t n) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Alg. 1 iteration.  mode 0: x <- MGI(x, b, 1) until ||b - A x|| <= tol ||b||.
 * mode 1: conjugate gradients preconditioned by one cycle MGI(0, r, 1) per
 * iteration (Polak-Ribiere beta), stopping on the recursively updated
 * residual and confirmed on the true one.  hist[k] = relative residual after k
 * iterations (hist[0] for the initial guess); returns OR_ERR_NOT_CONV when
 * max_iter is reached first. */
int or_solve(const octx *c, int mode, const double *b, double *x, double tol, int max_iter, double *hist,
             int *iters) {
  const olevel *L = &c->lev[0];
  int64_t n = L->n;
  double nb = norm2(b, n);
  *iters = 0;
  if (nb == 0.0) {
    memset(x, 0, sizeof(double) * (size_t)n);
    if (hist) hist[0] = 0.0;
    return OR_OK;
  }
  double *r = (double *)xmalloc(sizeof(double) * (size_t)n);
  or_residual(c, 0, x, b, r);
  double rel = norm2(r, n) / nb;
  if (hist) hist[0] = rel;
  int k = 0, st = OR_ERR_NOT_CONV;
  if (mode == 0) {
    while (k < max_iter) {
      or_mgi(c, 0, x, b);
      ++k;
      or_residual(c, 0, x, b, r);
      rel = norm2(r, n) / nb;
      if (hist) hist[k] = rel;
      if (rel <= tol) { st = OR_OK; break; }
    }
  } else {
    double *z = (double *)calloc((size_t)n, sizeof(double));
    double *p = (double *)xmalloc(sizeof(double) * (size_t)n);
    double *q = (double *)xmalloc(sizeof(double) * (size_t)n);
    double *rold = (double *)xmalloc(sizeof(double) * (size_t)n);
    int restart = 1;
    double rz = 0.0;
    while (k < max_iter) {
      if (restart) {
        or_residual(c, 0, x, b, r);
        memset(z, 0, sizeof(double) * (size_t)n);
        or_mgi(c, 0, z, r);
        memcpy(p, z, sizeof(double) * (size_t)n);
        rz = dotp(r, z, n);
        restart = 0;
      }
      or_apply(c, 0, p, q); /* q = A p */
      double alpha = rz / dotp(p, q, n);
      memcpy(rold, r, sizeof(double) * (size_t)n);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
      ++k;
      rel = norm2(r, n) / nb;
      if (rel <= tol) {
        double *tr = (double *)xmalloc(sizeof(double) * (size_t)n);
        or_residual(c, 0, x, b, tr);
        double trel = norm2(tr, n) / nb;
        free(tr);
        if (hist) hist[k] = trel;
        if (trel <= tol) { st = OR_OK; break; }
        restart = 1;
        continue;
      }
      if (hist) hist[k] = rel;
      memset(z, 0, sizeof(double) * (size_t)n);
      or_mgi(c, 0, z, r);
      double num = 0.0;
#pragma omp parallel for reduction(+ : num) schedule(static)
      for (int64_t i = 0; i < n; ++i) num += z[i] * (r[i] - rold[i]);
      double beta = num / rz;
      rz = dotp(r, z, n);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    free(z); free(p); free(q); free(rold);
  }
  free(r);
  *iters = k;
  return st;
}
