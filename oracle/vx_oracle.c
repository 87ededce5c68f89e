/*
 * vx_oracle.c -- CPU oracle for CSF-amortized interval subdivision.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this library; the product path never calls it, and it shares
 * no code, header, table or helper with the CUDA library.
 *
 * A plain, slow, single-threaded statement of the method of G. Moroz, "Sparse Tensors and
 * Subdivision Methods for Finding the Zero Set of Polynomial Equations" (arXiv 2406.09857):
 *
 *   csf_build()      the Compressed Sparse Fiber tree of a set of grid indices (Sec. 2.1):
 *                    depth-j nodes are the distinct length-j prefixes, children ascending.
 *   horner_group()   Algorithm 1 (Horner scheme on an interval, sparse exponents).
 *   eval_rec()       Algorithm 2 (EvaluationCSF): at each depth-j node the polynomial is
 *                    partially evaluated in x_j on the node's interval and the result is
 *                    handed to the node's children.
 *   orc_enclose()    Algorithm 3 (breadth-first subdivision) with the exclusion criterion
 *                    C0 of Sec. 3.2: a box is dropped iff 0 is outside the interval value
 *                    of some polynomial of the system.
 *   orc_dense_powerform()  the mode-by-mode midpoint-radius enclosure on a tensor grid
 *                    (Property 1's contractions, one variable at a time), the reference for
 *                    the dense tensor-core level.
 *   orc_taylor_boxes(), orc_enclose_taylor()  C0 on the Taylor form of order m (Def. 3).
 *   orc_eval_csf_gen(), orc_enclose_gen()  systems of equations and inequalities (F = 0,
 *                    F <= 0, F >= 0, F < 0, F > 0) with interval coefficients (Sec. 4).
 *   orc_c1_boxes(), orc_enclose_c1()  the inclusion criterion C1 for one equation (Sec. 3.2:
 *                    vertex signs, or the Taylor form at the two vertices extremal for its
 *                    linear part) and Algorithm 3 with both criteria.
 *
 * Readings of the paper taken here (where it is silent or ambiguous):
 *   - Rounding (Sec. 3.2 only gives [a,b]+[c,d]=[a+c,b+d]): every lower endpoint is
 *     rounded down and every upper endpoint rounded up, in IEEE binary64.  The product
 *     of two intervals is [min, max] of the four endpoint products, each rounded in its
 *     own direction; min/max are the selects (b<a)?b:a and (b>a)?b:a.
 *   - Algorithm 1 with an exponent gap g multiplies by the interval g times (repeated
 *     multiplication, not an interval power), and the result is multiplied by the interval
 *     e_0 more times when the lowest exponent e_0 is positive (the printed loop stops at
 *     a_0 and leaves that factor out).
 *   - Variable x_1 is at the root of the CSF, x_k at the leaves; F(I, x_2, ...) is formed
 *     by running Algorithm 1 in x_1 once per distinct monomial in the remaining variables.
 *   - The grid: box t on axis i at level l is [lo_i + t w_i, lo_i + (t+1) w_i] with
 *     w_i = (hi_i - lo_i) / 2^l; the left end is rounded down and the right end up (both
 *     exact on dyadic domains, which are the only ones orc_domain_exact() accepts).
 *   - Algorithm 3 without an inclusion test stops by depth: levels 0..depth are tested
 *     and the survivors of level `depth` are returned.  With C1 it stops when no box is
 *     left or after level `depth` (boxes that touch the zero set only where F has no sign
 *     change, e.g. at a vertex, are never certified); "size < threshold" is a first level
 *     c1_level from which C1 is applied.
 *   - An inequality drops a box when the enclosure proves it false on the whole box (F <= 0:
 *     lo > 0; F < 0: lo >= 0; F >= 0: hi < 0; F > 0: hi <= 0); an interval coefficient
 *     [c_lo, c_hi] enters Horner as that interval (a coefficient such as sqrt(3) is given as
 *     the two binary64 numbers around it).
 *   - The Taylor C1 picks V_max by the sign of each first-derivative interval's midpoint
 *     (lo >= -hi counts as >= 0) and tests only the orientation the paper states (lower
 *     bound at V_max > 0, upper bound at V_min < 0).
 *
 * The rounding mode is set to FE_DOWNWARD at the entry of each exported function and
 * restored on exit; an upward-rounded result is formed as -RD(-x), which is the same
 * double as RU(x).  Build with -O2 -frounding-math -ffp-contract=off (no FMA contraction).
 */
#include <complex.h>
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>


#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_KMAX 8

/* ------------------------------------------------------------------------------------ */
/* Interval arithmetic, outward rounding (Sec. 3.2, "Exclusion Criterion").              */
/* Every function below runs with the rounding mode FE_DOWNWARD.                         */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  double lo, hi;
} ivl;

static double rd_mul(double a, double b) { return a * b; }
static double ru_mul(double a, double b) { return -((-a) * b); }
static double rd_add(double a, double b) { return a + b; }
static double ru_add(double a, double b) { return -((-a) - b); }
static double sel_min(double a, double b) { return (b < a) ? b : a; }
static double sel_max(double a, double b) { return (b > a) ? b : a; }

static ivl i_mul(ivl x, ivl y) {
  ivl r;
  r.lo = sel_min(sel_min(rd_mul(x.lo, y.lo), rd_mul(x.lo, y.hi)),
                 sel_min(rd_mul(x.hi, y.lo), rd_mul(x.hi, y.hi)));
  r.hi = sel_max(sel_max(ru_mul(x.lo, y.lo), ru_mul(x.lo, y.hi)),
                 sel_max(ru_mul(x.hi, y.lo), ru_mul(x.hi, y.hi)));
  return r;
}

static ivl i_add(ivl x, ivl y) {
  ivl r;
  r.lo = rd_add(x.lo, y.lo);
  r.hi = ru_add(x.hi, y.hi);
  return r;
}

/* ------------------------------------------------------------------------------------ */
/* Partial evaluation plan.                                                              */
/*                                                                                       */
/* Stage s (0-based) evaluates variable x_{s+1}.  Its input is a list of terms in the    */
/* variables x_{s+1}..x_k; the terms are grouped by their exponents in x_{s+2}..x_k (the */
/* "suffix"), and each group is one run of Algorithm 1 in x_{s+1}.  The output has one   */
/* term per distinct suffix.  The plan only fixes which input term goes where; it does   */
/* no arithmetic.                                                                         */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  int nin, nout, nsuf; /* input terms, output terms, variables left after the stage */
  int *grp;            /* [nout+1] group boundaries into ord[] */
  int *ord;            /* [nin] input term index; exponents ascending within a group */
  int *ex;             /* [nin] exponent of the evaluated variable, aligned with ord[] */
  int *oexp;           /* [nout*nsuf] suffix exponents of each output term */
} stage;

typedef struct {
  int k;
  int nterms;
  stage st[ORC_KMAX];
} plan;

static const int *g_sort_exps; /* comparator context (the oracle is single-threaded) */
static int g_sort_nv;

static int cmp_suffix_then_first(const void *pa, const void *pb) {
  int a = *(const int *)pa, b = *(const int *)pb;
  const int *ea = g_sort_exps + (size_t)a * g_sort_nv, *eb = g_sort_exps + (size_t)b * g_sort_nv;
  for (int v = 1; v < g_sort_nv; ++v)
    if (ea[v] != eb[v]) return ea[v] < eb[v] ? -1 : 1;
  if (ea[0] != eb[0]) return ea[0] < eb[0] ? -1 : 1;
  return 0;
}

static void plan_free(plan *P) {
  for (int s = 0; s < ORC_KMAX; ++s) {
    free(P->st[s].grp);
    free(P->st[s].ord);
    free(P->st[s].ex);
    free(P->st[s].oexp);
  }
  memset(P, 0, sizeof(*P));
}

/* exps: [nterms][k].  Fails on negative exponents or repeated monomials. */
static int plan_build(plan *P, int k, int nterms, const int32_t *exps) {
  memset(P, 0, sizeof(*P));
  P->k = k;
  P->nterms = nterms;
  if (nterms == 0) return ORC_OK;
  int nv = k, nin = nterms;
  int *cur = (int *)malloc(sizeof(int) * (size_t)nin * nv); /* current term exponents */
  if (!cur) return ORC_ENOMEM;
  for (size_t i = 0; i < (size_t)nin * nv; ++i) {
    if (exps[i] < 0) {
      free(cur);
      return ORC_EINVAL;
    }
    cur[i] = exps[i];
  }
  for (int s = 0; s < k; ++s) {
    stage *S = &P->st[s];
    S->nin = nin;
    S->nsuf = nv - 1;
    S->ord = (int *)malloc(sizeof(int) * nin);
    S->ex = (int *)malloc(sizeof(int) * nin);
    S->grp = (int *)malloc(sizeof(int) * (nin + 1));
    S->oexp = (int *)malloc(sizeof(int) * (size_t)nin * (nv > 1 ? nv - 1 : 1));
    if (!S->ord || !S->ex || !S->grp || !S->oexp) {
      free(cur);
      plan_free(P);
      return ORC_ENOMEM;
    }
    for (int i = 0; i < nin; ++i) S->ord[i] = i;
    g_sort_exps = cur;
    g_sort_nv = nv;
    qsort(S->ord, nin, sizeof(int), cmp_suffix_then_first);
    int nout = 0;
    for (int i = 0; i < nin; ++i) {
      const int *e = cur + (size_t)S->ord[i] * nv;
      S->ex[i] = e[0];
      int newgrp = (i == 0);
      if (!newgrp) {
        const int *p = cur + (size_t)S->ord[i - 1] * nv;
        for (int v = 1; v < nv; ++v)
          if (p[v] != e[v]) newgrp = 1;
        if (!newgrp && p[0] == e[0]) { /* same monomial twice */
          free(cur);
          plan_free(P);
          return ORC_EINVAL;
        }
      }
      if (newgrp) {
        S->grp[nout] = i;
        for (int v = 1; v < nv; ++v) S->oexp[(size_t)nout * (nv - 1) + (v - 1)] = e[v];
        ++nout;
      }
    }
    S->grp[nout] = nin;
    S->nout = nout;
    /* the next stage's input terms are this stage's output terms */
    int *nxt = (int *)malloc(sizeof(int) * (size_t)nout * (nv > 1 ? nv - 1 : 1));
    if (!nxt) {
      free(cur);
      plan_free(P);
      return ORC_ENOMEM;
    }
    memcpy(nxt, S->oexp, sizeof(int) * (size_t)nout * (nv - 1));
    free(cur);
    cur = nxt;
    nin = nout;
    nv -= 1;
  }
  free(cur);
  return ORC_OK;
}

/* Algorithm 1 on one group: coefficients in[ord[b..e-1]] with ascending exponents ex[]. */
static ivl horner_group(const stage *S, int g, const ivl *in, ivl X, int64_t *work) {
  int b = S->grp[g], e = S->grp[g + 1];
  ivl J = in[S->ord[e - 1]];
  for (int t = e - 2; t >= b; --t) {
    for (int gap = S->ex[t + 1] - S->ex[t]; gap > 0; --gap) {
      J = i_mul(J, X);
      ++*work;
    }
    J = i_add(J, in[S->ord[t]]);
  }
  for (int gap = S->ex[b]; gap > 0; --gap) {
    J = i_mul(J, X);
    ++*work;
  }
  return J;
}

/* F(X, x_{s+2}, ...): one Algorithm-1 run per output term. */
static void run_stage(const stage *S, const ivl *in, ivl X, ivl *out, int64_t *work) {
  for (int g = 0; g < S->nout; ++g) out[g] = horner_group(S, g, in, X, work);
}

/* ------------------------------------------------------------------------------------ */
/* Box intervals: the grid of Sec. 3.2 scaled to a general domain, or explicit lists.     */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  const double *dom; /* [2k] lo, hi per axis (grid mode) */
  int level;
  const int64_t *xoff; /* [k+1] offsets into xlo/xhi (list mode) */
  const double *xlo, *xhi;
} boxsrc;

static ivl box_ivl(const boxsrc *B, int axis, int32_t t) {
  ivl r;
  if (B->xlo) {
    r.lo = B->xlo[B->xoff[axis] + t];
    r.hi = B->xhi[B->xoff[axis] + t];
    return r;
  }
  double lo = B->dom[2 * axis], hi = B->dom[2 * axis + 1];
  double s = ldexp(1.0, -B->level);
  double wd = rd_mul(rd_add(hi, -lo), s);
  double wu = ru_mul(ru_add(hi, -lo), s);
  r.lo = rd_add(lo, rd_mul((double)t, wd));
  r.hi = ru_add(lo, ru_mul((double)t + 1.0, wu));
  return r;
}

/* ------------------------------------------------------------------------------------ */
/* CSF of a set of grid indices (Sec. 2.1).                                               */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  int k;
  int64_t N[ORC_KMAX];    /* N_j, nodes at depth j+1 */
  int32_t *lab[ORC_KMAX]; /* labels at depth j+1 */
  int64_t *ptr[ORC_KMAX]; /* [N_j+1] children range at depth j+2 (j < k-1) */
} csf;

static void csf_free(csf *T) {
  for (int j = 0; j < ORC_KMAX; ++j) {
    free(T->lab[j]);
    free(T->ptr[j]);
  }
  memset(T, 0, sizeof(*T));
}

/* tuples: [n][k], must be strictly increasing in lexicographic order */
static int csf_build(csf *T, int k, const int32_t *tup, int64_t n) {
  memset(T, 0, sizeof(*T));
  T->k = k;
  for (int64_t i = 0; i < n; ++i) {
    for (int c = 0; c < k; ++c)
      if (tup[i * k + c] < 0) return ORC_EINVAL;
    if (i > 0) {
      int c = 0;
      while (c < k && tup[i * k + c] == tup[(i - 1) * k + c]) ++c;
      if (c == k || tup[i * k + c] < tup[(i - 1) * k + c]) return ORC_EINVAL;
    }
  }
  for (int j = 0; j < k; ++j) {
    T->lab[j] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    T->ptr[j] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!T->lab[j] || !T->ptr[j]) {
      csf_free(T);
      return ORC_ENOMEM;
    }
  }
  /* a depth-(j+1) node starts at tuple i when i is first or the first j+1 coordinates differ */
  for (int64_t i = 0; i < n; ++i) {
    int first_diff = 0;
    if (i > 0)
      while (first_diff < k && tup[i * k + first_diff] == tup[(i - 1) * k + first_diff]) ++first_diff;
    for (int j = first_diff; j < k; ++j) {
      if (j + 1 < k) T->ptr[j][T->N[j]] = T->N[j + 1];
      T->lab[j][T->N[j]] = tup[i * k + j];
      T->N[j]++;
    }
  }
  for (int j = 0; j + 1 < k; ++j) T->ptr[j][T->N[j]] = T->N[j + 1];
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 2 (EvaluationCSF).                                                          */
/* ------------------------------------------------------------------------------------ */

static void eval_rec(const plan *P, const csf *T, const boxsrc *B, int j, const ivl *in,
                     int64_t nb, int64_t ne, ivl *const *buf, ivl *leaf, int64_t *work) {
  for (int64_t n = nb; n < ne; ++n) {
    ivl X = box_ivl(B, j, T->lab[j][n]);
    run_stage(&P->st[j], in, X, buf[j], work);
    if (j == P->k - 1)
      leaf[n] = buf[j][0];
    else
      eval_rec(P, T, B, j + 1, buf[j], T->ptr[j][n], T->ptr[j][n + 1], buf, leaf, work);
  }
}

/* Evaluates one polynomial on every leaf of T. */
static int eval_poly_csf(const plan *P, const double *clo, const double *chi, const csf *T,
                         const boxsrc *B, ivl *leaf, int64_t *work) {
  int64_t n = T->N[P->k - 1];
  if (P->nterms == 0) {
    for (int64_t i = 0; i < n; ++i) leaf[i].lo = leaf[i].hi = 0.0;
    return ORC_OK;
  }
  ivl *in = (ivl *)malloc(sizeof(ivl) * P->nterms);
  ivl *buf[ORC_KMAX] = {0};
  int rc = ORC_OK;
  if (!in) return ORC_ENOMEM;
  for (int i = 0; i < P->nterms; ++i) {
    in[i].lo = clo[i];
    in[i].hi = chi[i];
  }
  for (int j = 0; j < P->k; ++j) {
    buf[j] = (ivl *)malloc(sizeof(ivl) * (size_t)P->st[j].nout);
    if (!buf[j]) rc = ORC_ENOMEM;
  }
  if (rc == ORC_OK) eval_rec(P, T, B, 0, in, 0, T->N[0], buf, leaf, work);
  for (int j = 0; j < P->k; ++j) free(buf[j]);
  free(in);
  return rc;
}

/* Nested Horner on a single box: stage after stage, no CSF. */
/* The centre of box t on an axis as a point interval (exact on the grids accepted here). */
static ivl centre_ivl(const boxsrc *B, int axis, int32_t t) {
  ivl r;
  double lo = B->dom[2 * axis], hi = B->dom[2 * axis + 1];
  double s = ldexp(1.0, -B->level);
  double wd = rd_mul(rd_add(hi, -lo), s);
  double wu = ru_mul(ru_add(hi, -lo), s);
  r.lo = rd_add(lo, rd_mul((double)t + 0.5, wd));
  r.hi = ru_add(lo, ru_mul((double)t + 0.5, wu));
  return r;
}

/* Nested Horner of one polynomial with interval coefficients [clo, chi] on box `tup`, or on
 * its centre when `point` is set. */
static ivl eval_poly_box_ivl(const plan *P, const double *clo, const double *chi,
                             const boxsrc *B, const int32_t *tup, int point, int64_t *work,
                             int *rc) {
  ivl z = {0.0, 0.0};
  if (P->nterms == 0) return z;
  ivl *cur = (ivl *)malloc(sizeof(ivl) * P->nterms);
  ivl *nxt = (ivl *)malloc(sizeof(ivl) * P->nterms);
  if (!cur || !nxt) {
    free(cur);
    free(nxt);
    *rc = ORC_ENOMEM;
    return z;
  }
  for (int i = 0; i < P->nterms; ++i) {
    cur[i].lo = clo[i];
    cur[i].hi = chi[i];
  }
  for (int j = 0; j < P->k; ++j) {
    run_stage(&P->st[j], cur, point ? centre_ivl(B, j, tup[j]) : box_ivl(B, j, tup[j]), nxt,
              work);
    ivl *t = cur;
    cur = nxt;
    nxt = t;
  }
  z = cur[0];
  free(cur);
  free(nxt);
  return z;
}

static ivl eval_poly_box(const plan *P, const double *coefs, const boxsrc *B, const int32_t *tup,
                         int64_t *work, int *rc) {
  ivl z = {0.0, 0.0};
  if (P->nterms == 0) return z;
  ivl *cur = (ivl *)malloc(sizeof(ivl) * P->nterms);
  ivl *nxt = (ivl *)malloc(sizeof(ivl) * P->nterms);
  if (!cur || !nxt) {
    free(cur);
    free(nxt);
    *rc = ORC_ENOMEM;
    return z;
  }
  for (int i = 0; i < P->nterms; ++i) cur[i].lo = cur[i].hi = coefs[i];
  for (int j = 0; j < P->k; ++j) {
    run_stage(&P->st[j], cur, box_ivl(B, j, tup[j]), nxt, work);
    ivl *t = cur;
    cur = nxt;
    nxt = t;
  }
  z = cur[0];
  free(cur);
  free(nxt);
  return z;
}

/* ------------------------------------------------------------------------------------ */
/* Exported interface (ctypes).                                                          */
/*                                                                                       */
/* A polynomial system is npoly polynomials in k variables: polynomial f owns terms      */
/* term_off[f] .. term_off[f+1]-1 of exps ([total][k] int32) and coefs (double).         */
/* ------------------------------------------------------------------------------------ */

static int check_system(int k, int npoly, const int64_t *term_off) {
  if (k < 1 || k > ORC_KMAX || npoly < 1) return ORC_EINVAL;
  for (int f = 0; f < npoly; ++f)
    if (term_off[f + 1] < term_off[f]) return ORC_EINVAL;
  return ORC_OK;
}

static int build_plans(plan *plans, int k, int npoly, const int64_t *term_off, const int32_t *exps,
                       const double *coefs) {
  for (int f = 0; f < npoly; ++f) {
    int64_t nt = term_off[f + 1] - term_off[f];
    for (int64_t i = term_off[f]; i < term_off[f + 1]; ++i)
      if (!isfinite(coefs[i])) return ORC_EINVAL;
    int rc = plan_build(&plans[f], k, (int)nt, exps + term_off[f] * k);
    if (rc != ORC_OK) {
      for (int g = 0; g < f; ++g) plan_free(&plans[g]);
      return rc;
    }
  }
  return ORC_OK;
}

static void free_plans(plan *plans, int npoly) {
  for (int f = 0; f < npoly; ++f) plan_free(&plans[f]);
}

/* 1 if every grid point lo + t (hi-lo)/2^level, 0 <= t <= 2^level, of every axis is a double. */
int orc_domain_exact(int k, const double *domain, int level) {
  int old = fegetround();
  int ok = 1;
  fesetround(FE_DOWNWARD);
  if (level < 0 || level > 30) ok = 0;
  for (int i = 0; ok && i < k; ++i) {
    double lo = domain[2 * i], hi = domain[2 * i + 1];
    if (!isfinite(lo) || !isfinite(hi) || !(lo < hi)) {
      ok = 0;
      break;
    }
    boxsrc B = {domain, level, 0, 0, 0};
    for (int64_t t = 0; ok && t < ((int64_t)1 << level); ++t) {
      ivl x = box_ivl(&B, i, (int32_t)t);
      /* exact iff rounding down and up agree on both ends */
      double s = ldexp(1.0, -level);
      double l_up = ru_add(lo, ru_mul((double)t, ru_mul(ru_add(hi, -lo), s)));
      double h_dn = rd_add(lo, rd_mul((double)t + 1.0, rd_mul(rd_add(hi, -lo), s)));
      if (l_up != x.lo || h_dn != x.hi) ok = 0;
    }
  }
  fesetround(old);
  return ok;
}

/* C0 for one polynomial of a system of equations and inequalities (Sec. 3.2, Sec. 4): the
 * box is dropped iff the enclosure [lo, hi] of F on it proves the relation false at every
 * point of it.  An enclosure with a NaN end proves nothing (every comparison is false). */
#define ORC_EQ 0 /* F = 0 */
#define ORC_LE 1 /* F <= 0 */
#define ORC_GE 2 /* F >= 0 */
#define ORC_LT 3 /* F < 0 */
#define ORC_GT 4 /* F > 0 */
static int c0_drops(ivl v, int rel) {
  switch (rel) {
    case ORC_LE: return v.lo > 0.0;
    case ORC_GE: return v.hi < 0.0;
    case ORC_LT: return v.lo >= 0.0;
    case ORC_GT: return v.hi <= 0.0;
    default: return v.lo > 0.0 || v.hi < 0.0;
  }
}

/* checks interval coefficients (chi may be NULL: point coefficients) and relations */
static int check_ivl_rel(int npoly, const int64_t *term_off, const double *clo, const double *chi,
                         const int32_t *rel) {
  for (int f = 0; f < npoly; ++f) {
    if (rel && (rel[f] < ORC_EQ || rel[f] > ORC_GT)) return ORC_EINVAL;
    for (int64_t i = term_off[f]; chi && i < term_off[f + 1]; ++i)
      if (!isfinite(chi[i]) || !(clo[i] <= chi[i])) return ORC_EINVAL;
  }
  return ORC_OK;
}

static int eval_csf_common(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                           const double *coefs, const double *coefs_hi, const int32_t *rel,
                           const boxsrc *B, const int32_t *tuples, int64_t n, double *lo,
                           double *hi, uint8_t *keep, int64_t *work) {
  plan plans[16];
  csf T;
  int rc = check_system(k, npoly, term_off);
  if (rc != ORC_OK) return rc;
  if (npoly > 16) return ORC_EINVAL;
  rc = check_ivl_rel(npoly, term_off, coefs, coefs_hi, rel);
  if (rc != ORC_OK) return rc;
  rc = build_plans(plans, k, npoly, term_off, exps, coefs);
  if (rc != ORC_OK) return rc;
  rc = csf_build(&T, k, tuples, n);
  if (rc != ORC_OK) {
    free_plans(plans, npoly);
    return rc;
  }
  ivl *leaf = (ivl *)malloc(sizeof(ivl) * (size_t)(n > 0 ? n : 1));
  int64_t w = 0;
  if (!leaf) rc = ORC_ENOMEM;
  if (keep)
    for (int64_t i = 0; i < n; ++i) keep[i] = 1;
  for (int f = 0; rc == ORC_OK && f < npoly; ++f) {
    rc = eval_poly_csf(&plans[f], coefs + term_off[f], (coefs_hi ? coefs_hi : coefs) + term_off[f],
                       &T, B, leaf, &w);
    for (int64_t i = 0; rc == ORC_OK && i < n; ++i) {
      if (lo) lo[(int64_t)f * n + i] = leaf[i].lo;
      if (hi) hi[(int64_t)f * n + i] = leaf[i].hi;
      /* C0: the box is dropped iff the enclosure of some polynomial proves its relation
       * false on the box (for an equation: 0 is provably outside [lo, hi]) */
      if (keep && c0_drops(leaf[i], rel ? rel[f] : ORC_EQ)) keep[i] = 0;
    }
  }
  if (work) *work = w;
  free(leaf);
  csf_free(&T);
  free_plans(plans, npoly);
  return rc;
}

/* Algorithm 2 on the boxes `tuples` (lex-sorted, unique) of the level-`level` grid. */
int orc_eval_csf(int k, int npoly, const int64_t *term_off, const int32_t *exps, const double *coefs,
                 const double *domain, int level, const int32_t *tuples, int64_t n, double *lo,
                 double *hi, uint8_t *keep, int64_t *work) {
  int old = fegetround();
  fesetround(FE_DOWNWARD);
  boxsrc B = {domain, level, 0, 0, 0};
  int rc = eval_csf_common(k, npoly, term_off, exps, coefs, 0, 0, &B, tuples, n, lo, hi, keep,
                           work);
  fesetround(old);
  return rc;
}

/* orc_eval_csf for a system of equations and inequalities with interval coefficients:
 * polynomial f has coefficients [coefs[t], coefs_hi[t]] (coefs_hi NULL: points) and the
 * relation rel[f] (ORC_EQ .. ORC_GT; rel NULL: all equations). */
int orc_eval_csf_gen(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                     const double *coefs, const double *coefs_hi, const int32_t *rel,
                     const double *domain, int level, const int32_t *tuples, int64_t n,
                     double *lo, double *hi, uint8_t *keep, int64_t *work) {
  int old = fegetround();
  fesetround(FE_DOWNWARD);
  boxsrc B = {domain, level, 0, 0, 0};
  int rc = eval_csf_common(k, npoly, term_off, exps, coefs, coefs_hi, rel, &B, tuples, n, lo, hi,
                           keep, work);
  fesetround(old);
  return rc;
}

/* Algorithm 2 on explicit per-axis interval lists: axis i owns xlo/xhi[xoff[i] .. xoff[i+1]). */
int orc_eval_grid(int k, int npoly, const int64_t *term_off, const int32_t *exps, const double *coefs,
                  const int64_t *xoff, const double *xlo, const double *xhi, const int32_t *tuples,
                  int64_t n, double *lo, double *hi, uint8_t *keep, int64_t *work) {
  int old = fegetround();
  fesetround(FE_DOWNWARD);
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < k; ++c)
      if (tuples[i * k + c] >= xoff[c + 1] - xoff[c]) {
        fesetround(old);
        return ORC_EINVAL;
      }
  boxsrc B = {0, 0, xoff, xlo, xhi};
  int rc = eval_csf_common(k, npoly, term_off, exps, coefs, 0, 0, &B, tuples, n, lo, hi, keep,
                           work);
  fesetround(old);
  return rc;
}

/* Nested Horner of each polynomial on each box independently (no CSF, no sharing). */
int orc_eval_boxes(int k, int npoly, const int64_t *term_off, const int32_t *exps, const double *coefs,
                   const double *domain, int level, const int32_t *tuples, int64_t n, double *lo,
                   double *hi, uint8_t *keep, int64_t *work) {
  plan plans[16];
  int old = fegetround();
  int rc = check_system(k, npoly, term_off);
  if (rc != ORC_OK) return rc;
  if (npoly > 16) return ORC_EINVAL;
  fesetround(FE_DOWNWARD);
  rc = build_plans(plans, k, npoly, term_off, exps, coefs);
  if (rc != ORC_OK) {
    fesetround(old);
    return rc;
  }
  boxsrc B = {domain, level, 0, 0, 0};
  int64_t w = 0;
  for (int64_t i = 0; rc == ORC_OK && i < n; ++i) {
    int kp = 1;
    for (int f = 0; f < npoly; ++f) {
      ivl v = eval_poly_box(&plans[f], coefs + term_off[f], &B, tuples + i * k, &w, &rc);
      if (lo) lo[(int64_t)f * n + i] = v.lo;
      if (hi) hi[(int64_t)f * n + i] = v.hi;
      if (v.lo > 0.0 || v.hi < 0.0) kp = 0;
    }
    if (keep) keep[i] = (uint8_t)kp;
  }
  if (work) *work = w;
  free_plans(plans, npoly);
  fesetround(old);
  return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Mode-wise midpoint-radius power form on a tensor grid (the enclosure of the dense      */
/* tensor-core level, written out plainly).  Property 1 (Sec. 1) contracts the dense      */
/* coefficient tensor one variable at a time; on a box with centre c and half-width r per */
/* axis, contracting variable j maps midpoint-radius coefficients <m_a, q_a> to           */
/*   mid = sum_a m_a c^a,   rad = sum_a |m_a| ((|c|+r)^a - |c|^a) + q_a (|c|+r)^a,        */
/* which holds every value of sum_a y_a x^a for x in the box and |y_a - m_a| <= q_a.      */
/* Evaluated in binary64 with rounding to nearest, no safety margins: the reference the   */
/* device's (margined) enclosure must contain.  k = 3.                                    */
/* ------------------------------------------------------------------------------------ */
int orc_dense_powerform(const int32_t *exps, const double *coefs, int64_t nterms,
                        const double *domain, int level, const int32_t *tuples, int64_t n,
                        double *mid, double *rad) {
  int D[3] = {0, 0, 0};
  if (level < 0 || level > 30 || nterms < 1) return ORC_EINVAL;
  for (int64_t t = 0; t < nterms; ++t)
    for (int i = 0; i < 3; ++i) {
      if (exps[t * 3 + i] < 0) return ORC_EINVAL;
      if (exps[t * 3 + i] > D[i]) D[i] = exps[t * 3 + i];
    }
  const int64_t n1 = D[0] + 1, n2 = D[1] + 1, n3 = D[2] + 1;
  double *C = calloc((size_t)(n1 * n2 * n3), sizeof(double));
  double *m1 = malloc(sizeof(double) * (size_t)(n2 * n3)), *q1 = malloc(sizeof(double) * (size_t)(n2 * n3));
  double *m2 = malloc(sizeof(double) * (size_t)n3), *q2 = malloc(sizeof(double) * (size_t)n3);
  if (!C || !m1 || !q1 || !m2 || !q2) {
    free(C); free(m1); free(q1); free(m2); free(q2);
    return ORC_ENOMEM;
  }
  int old = fegetround();
  fesetround(FE_TONEAREST);
  for (int64_t t = 0; t < nterms; ++t)
    C[(exps[t * 3] * n2 + exps[t * 3 + 1]) * n3 + exps[t * 3 + 2]] += coefs[t];
  const double side = (double)((int64_t)1 << level);
  for (int64_t b = 0; b < n; ++b) {
    double c[3], r[3];
    for (int i = 0; i < 3; ++i) {
      const double w = (domain[2 * i + 1] - domain[2 * i]) / side;
      const double l = domain[2 * i] + (double)tuples[b * 3 + i] * w;
      c[i] = l + 0.5 * w;
      r[i] = 0.5 * w;
    }
    /* mode 1: variable x1 */
    for (int64_t j = 0; j < n2 * n3; ++j) {
      double m = 0.0, q = 0.0, p = 1.0, pa = 1.0, pu = 1.0;
      for (int64_t a = 0; a < n1; ++a) {
        const double y = C[a * n2 * n3 + j];
        m += y * p;
        q += fabs(y) * (pu - pa);
        p *= c[0];
        pa *= fabs(c[0]);
        pu *= fabs(c[0]) + r[0];
      }
      m1[j] = m;
      q1[j] = q;
    }
    /* mode 2: variable x2 */
    for (int64_t a3 = 0; a3 < n3; ++a3) {
      double m = 0.0, q = 0.0, p = 1.0, pa = 1.0, pu = 1.0;
      for (int64_t a2 = 0; a2 < n2; ++a2) {
        const double y = m1[a2 * n3 + a3], e = q1[a2 * n3 + a3];
        m += y * p;
        q += fabs(y) * (pu - pa) + e * pu;
        p *= c[1];
        pa *= fabs(c[1]);
        pu *= fabs(c[1]) + r[1];
      }
      m2[a3] = m;
      q2[a3] = q;
    }
    /* mode 3: variable x3 */
    double m = 0.0, q = 0.0, p = 1.0, pa = 1.0, pu = 1.0;
    for (int64_t a3 = 0; a3 < n3; ++a3) {
      m += m2[a3] * p;
      q += fabs(m2[a3]) * (pu - pa) + q2[a3] * pu;
      p *= c[2];
      pa *= fabs(c[2]);
      pu *= fabs(c[2]) + r[2];
    }
    mid[b] = m;
    rad[b] = q;
  }
  fesetround(old);
  free(C); free(m1); free(q1); free(m2); free(q2);
  return ORC_OK;
}

/* CSF arrays of a lex-sorted tuple set: N[k]; labels concatenated by depth; ptr for depths
 * 1..k-1 concatenated (N_j + 1 entries each).  Pass labels == NULL to get only N. */
int orc_csf(int k, const int32_t *tuples, int64_t n, int64_t *N, int32_t *labels, int64_t *ptr) {
  csf T;
  if (k < 1 || k > ORC_KMAX) return ORC_EINVAL;
  int rc = csf_build(&T, k, tuples, n);
  if (rc != ORC_OK) return rc;
  int64_t lo = 0, po = 0;
  for (int j = 0; j < k; ++j) {
    N[j] = T.N[j];
    if (labels) memcpy(labels + lo, T.lab[j], sizeof(int32_t) * (size_t)T.N[j]);
    if (ptr && j + 1 < k) memcpy(ptr + po, T.ptr[j], sizeof(int64_t) * (size_t)(T.N[j] + 1));
    lo += T.N[j];
    if (j + 1 < k) po += T.N[j] + 1;
  }
  csf_free(&T);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 3: breadth-first subdivision with the C0 test at every level.               */
/* ------------------------------------------------------------------------------------ */

typedef struct orc_result {
  int k, depth;
  int64_t n;
  int32_t *tuples;  /* survivors of the last level, lex order */
  int64_t *tested;  /* [depth+1] |S_l| */
  int64_t *kept;    /* [depth+1] */
  int64_t *nodes;   /* [(depth+1)*k] N_j(S_l) */
  int64_t *work;    /* [depth+1] interval multiply-adds */
  /* with an inclusion criterion C1: the boxes it certified, ordered by level, then lex */
  int64_t n_inc;
  int32_t *inc_levels; /* [n_inc] */
  int32_t *inc_tuples; /* [n_inc][k] indices at the box's own level */
  int64_t *included;   /* [depth+1] boxes certified at level l */
} orc_result;

static int g_cmp_k;
static int cmp_tuple(const void *pa, const void *pb) {
  const int32_t *a = (const int32_t *)pa, *b = (const int32_t *)pb;
  for (int c = 0; c < g_cmp_k; ++c)
    if (a[c] != b[c]) return a[c] < b[c] ? -1 : 1;
  return 0;
}

void orc_result_free(orc_result *R) {
  if (!R) return;
  free(R->tuples);
  free(R->tested);
  free(R->kept);
  free(R->nodes);
  free(R->work);
  free(R->inc_levels);
  free(R->inc_tuples);
  free(R->included);
  free(R);
}

/* Algorithm 3 with S initialised to the boxes start[n0][k] (lex-sorted, unique) of level
 * start_level: levels start_level..depth are tested.  orc_enclose is the case S = {domain}. */
int orc_enclose_from(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                     const double *coefs, const double *domain, int start_level,
                     const int32_t *start, int64_t n0, int depth, orc_result **out);

/* ------------------------------------------------------------------------------------ */
/* Taylor form of order m (Def. 3).  With c the centre of B and x - c in [-r, r] per axis:  */
/*   T_m(F, B) = sum_{|a| < m} G_a(c) (x - c)^a + sum_{|a| = m} []G_a(B) (x - c)^a,         */
/* G_a = (d^a F / dx^a) / a! = sum_e f_e prod_i binom(e_i, a_i) x^(e - a), the multi-index */
/* a running over |a| <= m in lexicographic order of (a_1, ..., a_k).  Each G_a has       */
/* interval coefficients [RD(f_e C), RU(f_e C)], C = prod binom(e_i, a_i); G_a(c) is its   */
/* nested Horner value on the point interval [c, c]; (x_i - c_i)^(a_i) ranges over [1, 1] */
/* (a_i = 0), [0, r^a_i] (even) or [-r^a_i, r^a_i] (odd); the terms are interval products */
/* summed in the order of the multi-indices, outward rounded.                               */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  int na;                   /* multi-indices */
  int alpha[64][ORC_KMAX];  /* lexicographic */
  plan pl[64];
  int nterms[64];
  double *clo[64], *chi[64];
} taylor_sys;

static int enum_alphas(int k, int m, int alpha[][ORC_KMAX], int cap) {
  int n = 0, a[ORC_KMAX] = {0};
  for (;;) {
    int tot = 0;
    for (int i = 0; i < k; ++i) tot += a[i];
    if (tot <= m) {
      if (n >= cap) return -1;
      for (int i = 0; i < k; ++i) alpha[n][i] = a[i];
      ++n;
    }
    int i = k - 1; /* next tuple in lexicographic order, entries 0..m */
    while (i >= 0 && a[i] == m) a[i--] = 0;
    if (i < 0) break;
    ++a[i];
  }
  return n;
}

static double binom(int n, int r) {
  double b = 1.0;
  for (int i = 1; i <= r; ++i) b = b * (double)(n - r + i) / (double)i; /* exact: integers < 2^53 */
  return b;
}

static void taylor_free(taylor_sys *T) {
  for (int a = 0; a < T->na; ++a) {
    plan_free(&T->pl[a]);
    free(T->clo[a]);
    free(T->chi[a]);
  }
}

/* the derived polynomials G_a of one polynomial (rounding mode FE_DOWNWARD) */
static int taylor_build(taylor_sys *T, int k, int m, int nterms, const int32_t *exps,
                        const double *coefs, const double *coefs_hi) {
  memset(T, 0, sizeof(*T));
  T->na = enum_alphas(k, m, T->alpha, 64);
  if (T->na < 0) return ORC_EINVAL;
  int rc = ORC_OK;
  for (int a = 0; a < T->na && rc == ORC_OK; ++a) {
    const int *al = T->alpha[a];
    int nt = 0;
    for (int t = 0; t < nterms; ++t) {
      int ok = 1;
      for (int i = 0; i < k; ++i) ok = ok && exps[(size_t)t * k + i] >= al[i];
      nt += ok;
    }
    int32_t *de = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt > 0 ? nt : 1) * k);
    T->clo[a] = (double *)malloc(sizeof(double) * (size_t)(nt > 0 ? nt : 1));
    T->chi[a] = (double *)malloc(sizeof(double) * (size_t)(nt > 0 ? nt : 1));
    if (!de || !T->clo[a] || !T->chi[a]) {
      free(de);
      rc = ORC_ENOMEM;
      break;
    }
    int j = 0;
    for (int t = 0; t < nterms; ++t) {
      int ok = 1;
      for (int i = 0; i < k; ++i) ok = ok && exps[(size_t)t * k + i] >= al[i];
      if (!ok) continue;
      double C = 1.0;
      for (int i = 0; i < k; ++i) C *= binom(exps[(size_t)t * k + i], al[i]);
      T->clo[a][j] = rd_mul(coefs[t], C);
      T->chi[a][j] = ru_mul(coefs_hi[t], C);
      for (int i = 0; i < k; ++i) de[(size_t)j * k + i] = exps[(size_t)t * k + i] - al[i];
      ++j;
    }
    T->nterms[a] = nt;
    rc = plan_build(&T->pl[a], k, nt, de);
    free(de);
  }
  if (rc != ORC_OK) taylor_free(T);
  return rc;
}

/* (x - c)^a over [-r, r] for one axis */
static ivl pow_range(double r, int a) {
  ivl z;
  if (a == 0) {
    z.lo = z.hi = 1.0;
    return z;
  }
  double p = r;
  for (int i = 1; i < a; ++i) p = ru_mul(p, r);
  z.hi = p;
  z.lo = (a & 1) ? -p : 0.0;
  return z;
}

static ivl taylor_box(const taylor_sys *T, int k, int m, const boxsrc *B, const int32_t *tup,
                      int64_t *work, int *rc) {
  ivl acc = {0.0, 0.0};
  double r[ORC_KMAX];
  for (int i = 0; i < k; ++i) {
    ivl X = box_ivl(B, i, tup[i]);
    r[i] = ru_mul(ru_add(X.hi, -X.lo), 0.5);
  }
  for (int a = 0; a < T->na; ++a) {
    int tot = 0;
    for (int i = 0; i < k; ++i) tot += T->alpha[a][i];
    ivl V = eval_poly_box_ivl(&T->pl[a], T->clo[a], T->chi[a], B, tup, tot < m, work, rc);
    ivl P = {1.0, 1.0};
    for (int i = 0; i < k; ++i) P = i_mul(P, pow_range(r[i], T->alpha[a][i]));
    acc = i_add(acc, i_mul(V, P));
  }
  return acc;
}

/* ------------------------------------------------------------------------------------ */
/* Inclusion criterion C1 for one equation (Sec. 3.2, "Inclusion Criterion").  True means */
/* F has a zero in the closed box B: two points of B where F has certified opposite signs */
/* (B is connected).                                                                        */
/*  - vertex test: F at each of the 2^k vertices by nested interval Horner on the point   */
/*    interval of the vertex; true iff one vertex has lo > 0 and another hi < 0;            */
/*  - Taylor test (order m >= 2): with g_i = G_{e_i}(c) (the centre values of the first   */
/*    derivatives), V_max = c + s r with s_i = +1 if g_i's midpoint is >= 0 (lo >= -hi),    */
/*    else -1, and V_min = c - s r, the vertices where the linear part of T_m is largest and */
/*    smallest; F(V) lies in sum_a V_a (V - c)^a (the Taylor form at the point V, the       */
/*    factors (s_i r_i)^{a_i} as point intervals multiplied by interval products); true iff */
/*    the lower bound at V_max is > 0 and the upper bound at V_min is < 0.                   */
/* ------------------------------------------------------------------------------------ */
#define ORC_C1_TAYLOR 1
#define ORC_C1_VERTEX 2

/* nested Horner of a polynomial with interval coefficients on explicit intervals X[k] */
static ivl eval_poly_at(const plan *P, const double *clo, const double *chi, const ivl *X,
                        int64_t *work, int *rc) {
  ivl z = {0.0, 0.0};
  if (P->nterms == 0) return z;
  ivl *cur = (ivl *)malloc(sizeof(ivl) * P->nterms);
  ivl *nxt = (ivl *)malloc(sizeof(ivl) * P->nterms);
  if (!cur || !nxt) {
    free(cur);
    free(nxt);
    *rc = ORC_ENOMEM;
    return z;
  }
  for (int i = 0; i < P->nterms; ++i) {
    cur[i].lo = clo[i];
    cur[i].hi = chi[i];
  }
  for (int j = 0; j < P->k; ++j) {
    run_stage(&P->st[j], cur, X[j], nxt, work);
    ivl *t = cur;
    cur = nxt;
    nxt = t;
  }
  z = cur[0];
  free(cur);
  free(nxt);
  return z;
}

static int c1_vertex_box(const plan *P, const double *coefs, int k, const boxsrc *B,
                         const int32_t *tup, int64_t *work, int *rc) {
  int pos = 0, neg = 0;
  for (int v = 0; v < (1 << k) && *rc == ORC_OK; ++v) {
    ivl X[ORC_KMAX];
    for (int i = 0; i < k; ++i) {
      ivl b = box_ivl(B, i, tup[i]);
      double x = ((v >> (k - 1 - i)) & 1) ? b.hi : b.lo;
      X[i].lo = X[i].hi = x;
    }
    ivl y = eval_poly_at(P, coefs, coefs, X, work, rc);
    if (y.lo > 0.0) pos = 1;
    if (y.hi < 0.0) neg = 1;
  }
  return pos && neg;
}

static int taylor_c1_box(const taylor_sys *T, int k, int m, const boxsrc *B, const int32_t *tup,
                         int64_t *work, int *rc) {
  double r[ORC_KMAX];
  ivl V[64];
  for (int i = 0; i < k; ++i) {
    ivl X = box_ivl(B, i, tup[i]);
    r[i] = ru_mul(ru_add(X.hi, -X.lo), 0.5);
  }
  for (int a = 0; a < T->na; ++a) {
    int tot = 0;
    for (int i = 0; i < k; ++i) tot += T->alpha[a][i];
    V[a] = eval_poly_box_ivl(&T->pl[a], T->clo[a], T->chi[a], B, tup, tot < m, work, rc);
  }
  int s[ORC_KMAX];
  for (int i = 0; i < k; ++i) {
    int e = -1;
    for (int a = 0; a < T->na && e < 0; ++a) {
      int ok = 1;
      for (int j = 0; j < k; ++j) ok = ok && T->alpha[a][j] == (j == i ? 1 : 0);
      if (ok) e = a;
    }
    s[i] = (V[e].lo >= -V[e].hi) ? 1 : -1;
  }
  ivl at[2];
  for (int side = 0; side < 2; ++side) { /* 0: V_max, 1: V_min */
    ivl acc = {0.0, 0.0};
    for (int a = 0; a < T->na; ++a) {
      ivl P = {1.0, 1.0};
      for (int i = 0; i < k; ++i) {
        double x = (side == 0 ? s[i] : -s[i]) > 0 ? r[i] : -r[i];
        ivl q = {x, x};
        for (int e = 0; e < T->alpha[a][i]; ++e) P = i_mul(P, q);
      }
      acc = i_add(acc, i_mul(V[a], P));
    }
    at[side] = acc;
  }
  return at[0].lo > 0.0 && at[1].hi < 0.0;
}

/* C1 of one polynomial (npoly must be 1) on boxes tuples[n][k] of a level: inc[i] = 1 when
 * certified.  kind ORC_C1_VERTEX or ORC_C1_TAYLOR (order m >= 2). */
int orc_c1_boxes(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                 const double *coefs, const double *domain, int level, int kind, int m,
                 const int32_t *tuples, int64_t n, uint8_t *inc) {
  int old = fegetround();
  int rc = check_system(k, npoly, term_off);
  if (rc != ORC_OK) return rc;
  if (npoly != 1 || (kind != ORC_C1_VERTEX && kind != ORC_C1_TAYLOR)) return ORC_EINVAL;
  if (kind == ORC_C1_TAYLOR && (m < 2 || m > 8)) return ORC_EINVAL;
  fesetround(FE_DOWNWARD);
  boxsrc B = {domain, level, 0, 0, 0};
  int64_t w = 0;
  if (kind == ORC_C1_VERTEX) {
    plan P;
    rc = build_plans(&P, k, 1, term_off, exps, coefs);
    if (rc == ORC_OK) {
      for (int64_t i = 0; i < n && rc == ORC_OK; ++i)
        inc[i] = (uint8_t)c1_vertex_box(&P, coefs, k, &B, tuples + i * k, &w, &rc);
      free_plans(&P, 1);
    }
  } else {
    taylor_sys T;
    rc = taylor_build(&T, k, m, (int)(term_off[1] - term_off[0]), exps, coefs, coefs);
    if (rc == ORC_OK) {
      for (int64_t i = 0; i < n && rc == ORC_OK; ++i)
        inc[i] = (uint8_t)taylor_c1_box(&T, k, m, &B, tuples + i * k, &w, &rc);
      taylor_free(&T);
    }
  }
  fesetround(old);
  return rc;
}

/* The Taylor form of order m of each polynomial on each box (lo/hi [npoly][n]) and the C0
 * decision (keep = 0 in every polynomial's form). */
int orc_taylor_boxes(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                     const double *coefs, const double *domain, int level, int m,
                     const int32_t *tuples, int64_t n, double *lo, double *hi, uint8_t *keep) {
  int old = fegetround();
  int rc = check_system(k, npoly, term_off);
  if (rc != ORC_OK) return rc;
  if (m < 1 || m > 8) return ORC_EINVAL;
  fesetround(FE_DOWNWARD);
  boxsrc B = {domain, level, 0, 0, 0};
  int64_t w = 0;
  for (int64_t i = 0; i < n && keep; ++i) keep[i] = 1;
  for (int f = 0; f < npoly && rc == ORC_OK; ++f) {
    taylor_sys T;
    rc = taylor_build(&T, k, m, (int)(term_off[f + 1] - term_off[f]), exps + term_off[f] * k,
                      coefs + term_off[f], coefs + term_off[f]);
    if (rc != ORC_OK) break;
    for (int64_t i = 0; i < n && rc == ORC_OK; ++i) {
      ivl v = taylor_box(&T, k, m, &B, tuples + i * k, &w, &rc);
      if (lo) lo[(int64_t)f * n + i] = v.lo;
      if (hi) hi[(int64_t)f * n + i] = v.hi;
      if (keep && (v.lo > 0.0 || v.hi < 0.0)) keep[i] = 0;
    }
    taylor_free(&T);
  }
  fesetround(old);
  return rc;
}

int orc_enclose(int k, int npoly, const int64_t *term_off, const int32_t *exps, const double *coefs,
                const double *domain, int depth, orc_result **out) {
  int32_t root[ORC_KMAX] = {0};
  return orc_enclose_from(k, npoly, term_off, exps, coefs, domain, 0, root, 1, depth, out);
}

static int enclose_core(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                        const double *coefs, const double *coefs_hi, const int32_t *rel,
                        const double *domain, int start_level, const int32_t *start, int64_t n0,
                        int depth, int taylor_m, int c1_kind, int c1_level, orc_result **out);

int orc_enclose_from(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                     const double *coefs, const double *domain, int start_level,
                     const int32_t *start, int64_t n0, int depth, orc_result **out) {
  return enclose_core(k, npoly, term_off, exps, coefs, 0, 0, domain, start_level, start, n0, depth,
                      0, 0, 0, out);
}

/* Algorithm 3 with C0 on the Taylor form of order m (Def. 3) instead of interval Horner. */
int orc_enclose_taylor(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                       const double *coefs, const double *domain, int depth, int m,
                       orc_result **out) {
  int32_t root[ORC_KMAX] = {0};
  if (m < 1 || m > 8) return ORC_EINVAL;
  return enclose_core(k, npoly, term_off, exps, coefs, 0, 0, domain, 0, root, 1, depth, m, 0, 0,
                      out);
}

/* Algorithm 3 with both criteria, for one equation: at every level the boxes C0 excludes are
 * dropped; from level c1_level on (the boxes are then below the size threshold) the boxes C1
 * certifies go to the result (inc_levels, inc_tuples) and are not bisected; the loop ends when
 * no box is left or after level `depth`, whose remaining boxes (neither excluded nor
 * certified) are the result's `tuples`.  C0 is interval Horner (taylor_m = 0) or the Taylor
 * form of order taylor_m; C1 is the vertex test or the Taylor test (which needs taylor_m >= 2
 * and uses the same form). */
int orc_enclose_c1(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                   const double *coefs, const double *domain, int depth, int taylor_m,
                   int c1_kind, int c1_level, orc_result **out) {
  int32_t root[ORC_KMAX] = {0};
  *out = 0;
  if (npoly != 1 || taylor_m < 0 || taylor_m > 8 || c1_level < 0) return ORC_EINVAL;
  if (c1_kind != ORC_C1_VERTEX && c1_kind != ORC_C1_TAYLOR) return ORC_EINVAL;
  if (c1_kind == ORC_C1_TAYLOR && taylor_m < 2) return ORC_EINVAL;
  return enclose_core(k, npoly, term_off, exps, coefs, 0, 0, domain, 0, root, 1, depth, taylor_m,
                      c1_kind, c1_level, out);
}

/* Algorithm 3 for a system of equations and inequalities with interval coefficients (Sec. 4):
 * coefs_hi / rel as for orc_eval_csf_gen; C0 on interval Horner (taylor_m = 0) or on the
 * Taylor form of order taylor_m. */
int orc_enclose_gen(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                    const double *coefs, const double *coefs_hi, const int32_t *rel,
                    const double *domain, int depth, int taylor_m, orc_result **out) {
  int32_t root[ORC_KMAX] = {0};
  *out = 0;
  if (taylor_m < 0 || taylor_m > 8) return ORC_EINVAL;
  return enclose_core(k, npoly, term_off, exps, coefs, coefs_hi, rel, domain, 0, root, 1, depth,
                      taylor_m, 0, 0, out);
}

static int enclose_core(int k, int npoly, const int64_t *term_off, const int32_t *exps,
                        const double *coefs, const double *coefs_hi, const int32_t *rel,
                        const double *domain, int start_level, const int32_t *start, int64_t n0,
                        int depth, int taylor_m, int c1_kind, int c1_level, orc_result **out) {
  int old = fegetround();
  int rc = check_system(k, npoly, term_off);
  *out = 0;
  if (rc != ORC_OK) return rc;
  rc = check_ivl_rel(npoly, term_off, coefs, coefs_hi, rel);
  if (rc != ORC_OK) return rc;
  if (!coefs_hi) coefs_hi = coefs;
  if (depth < 0 || depth > 30 || npoly > 16) return ORC_EINVAL;
  if (start_level < 0 || start_level > depth || n0 < 0) return ORC_EINVAL;
  if (!orc_domain_exact(k, domain, depth)) return ORC_EINVAL;
  fesetround(FE_DOWNWARD);
  orc_result *R = (orc_result *)calloc(1, sizeof(orc_result));
  plan plans[16];
  if (!R) {
    fesetround(old);
    return ORC_ENOMEM;
  }
  R->k = k;
  R->depth = depth;
  R->tested = (int64_t *)calloc(depth + 1, sizeof(int64_t));
  R->kept = (int64_t *)calloc(depth + 1, sizeof(int64_t));
  R->nodes = (int64_t *)calloc((size_t)(depth + 1) * k, sizeof(int64_t));
  R->work = (int64_t *)calloc(depth + 1, sizeof(int64_t));
  R->included = (int64_t *)calloc(depth + 1, sizeof(int64_t));
  int64_t inc_cap = 0;
  rc = build_plans(plans, k, npoly, term_off, exps, coefs);
  if (rc != ORC_OK) {
    orc_result_free(R);
    fesetround(old);
    return rc;
  }
  int64_t n = n0;
  int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n0 > 0 ? n0 : 1) * k);
  if (S) memcpy(S, start, sizeof(int32_t) * (size_t)n0 * k);
  for (int l = start_level; S && rc == ORC_OK && l <= depth; ++l) {
    csf T;
    boxsrc B = {domain, l, 0, 0, 0};
    rc = csf_build(&T, k, S, n);
    if (rc != ORC_OK) break;
    uint8_t *keep = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    ivl *leaf = (ivl *)malloc(sizeof(ivl) * (size_t)(n > 0 ? n : 1));
    if (!keep || !leaf) rc = ORC_ENOMEM;
    for (int64_t i = 0; i < n && keep; ++i) keep[i] = 1;
    for (int f = 0; rc == ORC_OK && f < npoly; ++f) {
      if (taylor_m > 0) {
        taylor_sys TS;
        rc = taylor_build(&TS, k, taylor_m, (int)(term_off[f + 1] - term_off[f]),
                          exps + term_off[f] * k, coefs + term_off[f], coefs_hi + term_off[f]);
        for (int64_t i = 0; rc == ORC_OK && i < n; ++i) {
          ivl v = taylor_box(&TS, k, taylor_m, &B, S + i * k, &R->work[l], &rc);
          if (c0_drops(v, rel ? rel[f] : ORC_EQ)) keep[i] = 0;
        }
        if (rc == ORC_OK || TS.na > 0) taylor_free(&TS);
        continue;
      }
      rc = eval_poly_csf(&plans[f], coefs + term_off[f], coefs_hi + term_off[f], &T, &B, leaf,
                         &R->work[l]);
      for (int64_t i = 0; rc == ORC_OK && i < n; ++i)
        if (c0_drops(leaf[i], rel ? rel[f] : ORC_EQ)) keep[i] = 0;
    }
    R->tested[l] = n;
    for (int j = 0; j < k; ++j) R->nodes[(size_t)l * k + j] = T.N[j];
    csf_free(&T);
    free(leaf);
    if (rc != ORC_OK) {
      free(keep);
      break;
    }
    /* S <- boxes of S not satisfying C0 */
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
      if (keep[i]) {
        memmove(S + m * k, S + i * k, sizeof(int32_t) * k);
        ++m;
      }
    free(keep);
    R->kept[l] = m;
    n = m;
    if (c1_kind && l >= c1_level && n > 0) {
      /* R <- R + the boxes of S satisfying C1; S <- the others */
      uint8_t *inc = (uint8_t *)malloc((size_t)n);
      taylor_sys TC;
      int built = 0;
      if (!inc) rc = ORC_ENOMEM;
      if (rc == ORC_OK && c1_kind == ORC_C1_TAYLOR) {
        rc = taylor_build(&TC, k, taylor_m, (int)(term_off[1] - term_off[0]), exps, coefs, coefs);
        built = rc == ORC_OK;
      }
      for (int64_t i = 0; rc == ORC_OK && i < n; ++i)
        inc[i] = (uint8_t)(c1_kind == ORC_C1_TAYLOR
                               ? taylor_c1_box(&TC, k, taylor_m, &B, S + i * k, &R->work[l], &rc)
                               : c1_vertex_box(&plans[0], coefs, k, &B, S + i * k, &R->work[l],
                                               &rc));
      if (built) taylor_free(&TC);
      int64_t q = 0;
      for (int64_t i = 0; rc == ORC_OK && i < n; ++i) {
        if (!inc[i]) {
          memmove(S + q * k, S + i * k, sizeof(int32_t) * k);
          ++q;
          continue;
        }
        if (R->n_inc == inc_cap) {
          inc_cap = inc_cap ? 2 * inc_cap : 1024;
          int32_t *a = (int32_t *)realloc(R->inc_levels, sizeof(int32_t) * (size_t)inc_cap);
          if (a) R->inc_levels = a;
          int32_t *b = (int32_t *)realloc(R->inc_tuples, sizeof(int32_t) * (size_t)inc_cap * k);
          if (b) R->inc_tuples = b;
          if (!a || !b) {
            rc = ORC_ENOMEM;
            break;
          }
        }
        R->inc_levels[R->n_inc] = l;
        memcpy(R->inc_tuples + R->n_inc * k, S + i * k, sizeof(int32_t) * k);
        ++R->n_inc;
        ++R->included[l];
      }
      free(inc);
      if (rc != ORC_OK) break;
      n = q;
      if (n == 0) break;
    }
    if (l == depth) break;
    /* S <- the 2^k boxes bisected from each box of S, sorted */
    int64_t nc = n << k;
    int32_t *C = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1) * k);
    if (!C) {
      rc = ORC_ENOMEM;
      break;
    }
    for (int64_t i = 0; i < n; ++i)
      for (int b = 0; b < (1 << k); ++b)
        for (int c = 0; c < k; ++c) C[((i << k) + b) * k + c] = 2 * S[i * k + c] + ((b >> (k - 1 - c)) & 1);
    g_cmp_k = k;
    qsort(C, (size_t)nc, sizeof(int32_t) * k, cmp_tuple);
    free(S);
    S = C;
    n = nc;
  }
  free_plans(plans, npoly);
  fesetround(old);
  if (rc != ORC_OK) {
    free(S);
    orc_result_free(R);
    return rc;
  }
  R->n = n;
  R->tuples = S;
  *out = R;
  return ORC_OK;
}

int64_t orc_result_count(const orc_result *R) { return R->n; }

void orc_result_copy(const orc_result *R, int32_t *tuples, int64_t *tested, int64_t *kept,
                     int64_t *nodes, int64_t *work) {
  if (tuples) memcpy(tuples, R->tuples, sizeof(int32_t) * (size_t)R->n * R->k);
  if (tested) memcpy(tested, R->tested, sizeof(int64_t) * (R->depth + 1));
  if (kept) memcpy(kept, R->kept, sizeof(int64_t) * (R->depth + 1));
  if (nodes) memcpy(nodes, R->nodes, sizeof(int64_t) * (size_t)(R->depth + 1) * R->k);
  if (work) memcpy(work, R->work, sizeof(int64_t) * (R->depth + 1));
}

int64_t orc_result_inc_count(const orc_result *R) { return R->n_inc; }

void orc_result_inc_copy(const orc_result *R, int32_t *levels, int32_t *tuples,
                         int64_t *included) {
  if (levels && R->n_inc) memcpy(levels, R->inc_levels, sizeof(int32_t) * (size_t)R->n_inc);
  if (tuples && R->n_inc)
    memcpy(tuples, R->inc_tuples, sizeof(int32_t) * (size_t)R->n_inc * R->k);
  if (included) memcpy(included, R->included, sizeof(int64_t) * (R->depth + 1));
}

/* Every box of the level-`level` grid tested independently with nested Horner; keep is in
 * lexicographic order of the box indices ((2^level)^k entries). */
int orc_brute_force(int k, int npoly, const int64_t *term_off, const int32_t *exps, const double *coefs,
                    const double *domain, int level, uint8_t *keep) {
  int64_t side = (int64_t)1 << level, total = 1;
  for (int c = 0; c < k; ++c) total *= side;
  int32_t tup[ORC_KMAX];
  for (int64_t i = 0; i < total; ++i) {
    int64_t r = i;
    for (int c = k - 1; c >= 0; --c) {
      tup[c] = (int32_t)(r % side);
      r /= side;
    }
    int rc = orc_eval_boxes(k, npoly, term_off, exps, coefs, domain, level, tup, 1, 0, 0, keep + i, 0);
    if (rc != ORC_OK) return rc;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 2 over complex points (round to nearest), for the DFT application of        */
/* Sec. 3.1: the same plan and CSF traversal with complex values in place of intervals.  */
/* ------------------------------------------------------------------------------------ */

static double complex horner_group_c(const stage *S, int g, const double complex *in, double complex x) {
  int b = S->grp[g], e = S->grp[g + 1];
  double complex J = in[S->ord[e - 1]];
  for (int t = e - 2; t >= b; --t) {
    for (int gap = S->ex[t + 1] - S->ex[t]; gap > 0; --gap) J = J * x;
    J = J + in[S->ord[t]];
  }
  for (int gap = S->ex[b]; gap > 0; --gap) J = J * x;
  return J;
}

static void eval_rec_c(const plan *P, const csf *T, const int64_t *xoff, const double *xre,
                       const double *xim, int j, const double complex *in, int64_t nb, int64_t ne,
                       double complex *const *buf, double complex *leaf) {
  for (int64_t n = nb; n < ne; ++n) {
    int32_t t = T->lab[j][n];
    double complex x = xre[xoff[j] + t] + I * xim[xoff[j] + t];
    const stage *S = &P->st[j];
    for (int g = 0; g < S->nout; ++g) buf[j][g] = horner_group_c(S, g, in, x);
    if (j == P->k - 1)
      leaf[n] = buf[j][0];
    else
      eval_rec_c(P, T, xoff, xre, xim, j + 1, buf[j], T->ptr[j][n], T->ptr[j][n + 1], buf, leaf);
  }
}

int orc_eval_grid_complex(int k, int64_t nterms, const int32_t *exps, const double *cre,
                          const double *cim, const int64_t *xoff, const double *xre,
                          const double *xim, const int32_t *tuples, int64_t n, double *vre,
                          double *vim) {
  int old = fegetround();
  plan P;
  csf T;
  if (k < 1 || k > ORC_KMAX || nterms < 1) return ORC_EINVAL;
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < k; ++c)
      if (tuples[i * k + c] >= xoff[c + 1] - xoff[c]) return ORC_EINVAL;
  fesetround(FE_TONEAREST);
  int rc = plan_build(&P, k, (int)nterms, exps);
  if (rc != ORC_OK) {
    fesetround(old);
    return rc;
  }
  rc = csf_build(&T, k, tuples, n);
  if (rc != ORC_OK) {
    plan_free(&P);
    fesetround(old);
    return rc;
  }
  double complex *in = (double complex *)malloc(sizeof(double complex) * (size_t)nterms);
  double complex *leaf = (double complex *)malloc(sizeof(double complex) * (size_t)(n > 0 ? n : 1));
  double complex *buf[ORC_KMAX] = {0};
  if (!in || !leaf) rc = ORC_ENOMEM;
  for (int j = 0; rc == ORC_OK && j < k; ++j) {
    buf[j] = (double complex *)malloc(sizeof(double complex) * (size_t)P.st[j].nout);
    if (!buf[j]) rc = ORC_ENOMEM;
  }
  if (rc == ORC_OK) {
    for (int64_t i = 0; i < nterms; ++i) in[i] = cre[i] + I * cim[i];
    eval_rec_c(&P, &T, xoff, xre, xim, 0, in, 0, T.N[0], buf, leaf);
    for (int64_t i = 0; i < n; ++i) {
      vre[i] = creal(leaf[i]);
      vim[i] = cimag(leaf[i]);
    }
  }
  for (int j = 0; j < k; ++j) free(buf[j]);
  free(in);
  free(leaf);
  csf_free(&T);
  plan_free(&P);
  fesetround(old);
  return rc;
}

/* Directed-rounding primitives, exported so that tests can pin them against exact rationals. */
void orc_prim(int op, const double *a, const double *b, int64_t n, double *out) {
  int old = fegetround();
  fesetround(FE_DOWNWARD);
  for (int64_t i = 0; i < n; ++i) {
    switch (op) {
      case 0: out[i] = rd_mul(a[i], b[i]); break;
      case 1: out[i] = ru_mul(a[i], b[i]); break;
      case 2: out[i] = rd_add(a[i], b[i]); break;
      default: out[i] = ru_add(a[i], b[i]); break;
    }
  }
  fesetround(old);
}

/* Interval product (4-product form), exported for the same reason. */
void orc_imul(const double *alo, const double *ahi, const double *blo, const double *bhi, int64_t n,
              double *lo, double *hi) {
  int old = fegetround();
  fesetround(FE_DOWNWARD);
  for (int64_t i = 0; i < n; ++i) {
    ivl x = {alo[i], ahi[i]}, y = {blo[i], bhi[i]};
    ivl r = i_mul(x, y);
    lo[i] = r.lo;
    hi[i] = r.hi;
  }
  fesetround(old);
}
