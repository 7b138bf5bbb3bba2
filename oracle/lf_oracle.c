/*
 * Layered-field oracle: plain, slow, FP64 CPU reference of one explicit
 * time-iteration of the concurrently evolving layered fields (Zayer, Mlakar,
 * Steinberger, Seidel, "Layered Fields for Natural Tessellations on
 * Surfaces", arXiv 1804.09152).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may call this code.  It shares nothing with
 * the CUDA library (no headers, helpers or generated tables) and the library
 * never calls it.
 *
 * Storage.  The paper keeps the field as Phi, an (n_r x n_v) sparse matrix,
 * one row per layer and one column per vertex, in CSC (Sec. 3.2, Eq. 14;
 * Sec. 4).  CSC(Phi) is the same array triple as CSR(Phi^T): here a field is
 * a vertex-major CSR with one row per vertex, layer ids sorted ascending.
 * Layers 0..k-1 belong to the seeds, layer k is the base layer (Sec. 3.1).
 * The Laplacian of the mesh is symmetric, so the paper's L_t = Phi L^T
 * (Algorithm 1, "L_t" line) is the vertex-major product G = L F.
 *
 * Each function cites the passage it follows.  Readings of passages that are
 * silent or ambiguous are marked READING.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_DEGENERATE (-2)
#define ORC_ERR_NOMEM (-3)
#define ORC_ERR_ZERO_SUM (-4)

/* ------------------------------------------------------------------------- */
/* Mesh Laplacian (Sec. 3.2 "Laplacian computation": precomputed once).      */
/* READING: the paper names no discretisation; the cotangent Laplacian is    */
/* used, L_ij = (cot alpha_ij + cot beta_ij) / 2 over the angles opposite    */
/* edge ij (one term on a boundary edge), L_ii = -sum_{j != i} L_ij, no mass */
/* matrix.  Every mesh edge is a structural entry even when its weight is 0. */
/* ------------------------------------------------------------------------- */

typedef struct { int32_t r, c; double w; } triplet;

static int cmp_triplet(const void* pa, const void* pb) {
  const triplet* a = (const triplet*)pa;
  const triplet* b = (const triplet*)pb;
  if (a->r != b->r) return a->r < b->r ? -1 : 1;
  if (a->c != b->c) return a->c < b->c ? -1 : 1;
  return 0;
}

/* cotangent of the angle at corner p of triangle (p, q, s) */
static double corner_cot(const double* p, const double* q, const double* s, int* bad) {
  double u[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
  double v[3] = {s[0] - p[0], s[1] - p[1], s[2] - p[2]};
  double dot = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
  double cx = u[1] * v[2] - u[2] * v[1];
  double cy = u[2] * v[0] - u[0] * v[2];
  double cz = u[0] * v[1] - u[1] * v[0];
  double area2 = sqrt(cx * cx + cy * cy + cz * cz);
  if (!(area2 > 0.0)) { *bad = 1; return 0.0; }
  return dot / area2;
}

/*
 * Builds L as CSR with sorted columns and an explicit diagonal.
 * rowptr: n_v + 1 entries; col/val: capacity n_v + 6 n_f.
 * Returns nnz, or a negative error code.
 */
int64_t orc_cotan_laplacian(int64_t n_v, const double* V, int64_t n_f, const int32_t* F,
                            int64_t* rowptr, int32_t* col, double* val) {
  if (n_v < 1 || n_f < 0) return ORC_ERR_INVALID;
  int64_t nt = 6 * n_f + n_v;
  triplet* t = (triplet*)malloc(sizeof(triplet) * (size_t)(nt > 0 ? nt : 1));
  if (!t) return ORC_ERR_NOMEM;
  int64_t m = 0;
  int bad = 0;
  for (int64_t f = 0; f < n_f; ++f) {
    int32_t v[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
    for (int c = 0; c < 3; ++c) {
      if (v[c] < 0 || v[c] >= n_v) { free(t); return ORC_ERR_INVALID; }
    }
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) { free(t); return ORC_ERR_DEGENERATE; }
    for (int c = 0; c < 3; ++c) {
      /* the angle at corner c is opposite the edge (c+1, c+2) */
      int32_t p = v[c], q = v[(c + 1) % 3], s = v[(c + 2) % 3];
      double ct = corner_cot(V + 3 * p, V + 3 * q, V + 3 * s, &bad);
      t[m++] = (triplet){q, s, 0.5 * ct};
      t[m++] = (triplet){s, q, 0.5 * ct};
    }
  }
  if (bad) { free(t); return ORC_ERR_DEGENERATE; }
  for (int64_t i = 0; i < n_v; ++i) t[m++] = (triplet){(int32_t)i, (int32_t)i, 0.0};
  qsort(t, (size_t)m, sizeof(triplet), cmp_triplet);
  /* merge duplicates, then set the diagonal to minus the off-diagonal sum */
  int64_t nnz = 0;
  for (int64_t i = 0; i <= n_v; ++i) rowptr[i] = 0;
  for (int64_t a = 0; a < m;) {
    int64_t b = a;
    double w = 0.0;
    while (b < m && t[b].r == t[a].r && t[b].c == t[a].c) { w += t[b].w; ++b; }
    col[nnz] = t[a].c;
    val[nnz] = w;
    rowptr[t[a].r + 1] = nnz + 1;
    ++nnz;
    a = b;
  }
  for (int64_t i = 1; i <= n_v; ++i)
    if (rowptr[i] < rowptr[i - 1]) rowptr[i] = rowptr[i - 1];
  for (int64_t i = 0; i < n_v; ++i) {
    double off = 0.0;
    int64_t di = -1;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      if (col[p] == i) di = p; else off += val[p];
    }
    val[di] = -off;
  }
  free(t);
  return nnz;
}

/* ------------------------------------------------------------------------- */
/* Initialisation (Algorithm 1, first line; Sec. 3.2 "Initialization";     */
/* Sec. 3.1 base layer): a seed vertex gets 1 in its own layer and 0 in the  */
/* base layer; every other vertex gets 1 in the base layer (id k).           */
/* ------------------------------------------------------------------------- */
int orc_seed(int64_t n_v, int32_t k, const int32_t* seeds, int64_t* rowptr, int32_t* id, double* val) {
  if (k < 1 || n_v < 1) return ORC_ERR_INVALID;
  int32_t* owner = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_v);
  if (!owner) return ORC_ERR_NOMEM;
  for (int64_t i = 0; i < n_v; ++i) owner[i] = k;
  for (int32_t s = 0; s < k; ++s) {
    if (seeds[s] < 0 || seeds[s] >= n_v || owner[seeds[s]] != k) { free(owner); return ORC_ERR_INVALID; }
    owner[seeds[s]] = s;
  }
  for (int64_t i = 0; i < n_v; ++i) {
    rowptr[i] = i;
    id[i] = owner[i];
    val[i] = 1.0;
  }
  rowptr[n_v] = n_v;
  free(owner);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Coefficients of Algorithm 1 (w_jl, a_jl, e_jk; Eq. 2, Eq. 11-12).         */
/* The energy sums over pairs i < j only, so a layer has no coefficient with */
/* itself: w_jj = a_jj = e_jj = 0.  Experiments use scalars (Sec. 7); two   */
/* classes of pairs are distinguished:                                       */
/*   cell-cell  (two seed layers):          w_cc, a_cc, e_cc                 */
/*   cell-base  (a seed layer and layer k): w_cb, a_cb, e_cb (cell row),     */
/*                                          e_bc (base row)                  */
/* READING (Sec. 3.1 fixes w = 0.2 and a factor 5 between w and a): a = w/5.*/
/* READING (Sec. 3.2, initialisation: the energy models the interaction     */
/*   between cells; the base layer exists so that cells grow freely):        */
/*   w_cb = 0.                                                               */
/* READING (Eq. 12: the left side is a difference of derivatives, hence     */
/*   antisymmetric in (i, j)): e_ji = -e_ij, so e_cc = 0 between two cells   */
/*   and e_bc = -e_cb for the base.                                          */
/* Callers may instead pass dense n_layers x n_layers matrices.              */
/* coefs = {dt, mu, w_cc, w_cb, a_cc, a_cb, e_cc, e_cb, e_bc}.               */
/* ------------------------------------------------------------------------- */
typedef struct { double dt, mu, w_cc, w_cb, a_cc, a_cb, e_cc, e_cb, e_bc; } orc_coefs;

static orc_coefs unpack(const double* c) {
  orc_coefs o = {c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7], c[8]};
  return o;
}

/* symmetric class rule for w and a; base id = n_layers - 1 */
static inline double coef_sym(const double* M, double cc, double cb, int32_t n_layers, int32_t j, int32_t l) {
  if (M) return M[(int64_t)j * n_layers + l];
  if (j == l) return 0.0;
  int32_t base = n_layers - 1;
  return (j == base || l == base) ? cb : cc;
}

/* e_jk: e_cc between cells, e_cb in a cell row against the base, e_bc in the base row */
static inline double coef_e(const double* M, const orc_coefs* c, int32_t n_layers, int32_t j, int32_t k) {
  if (M) return M[(int64_t)j * n_layers + k];
  if (j == k) return 0.0;
  int32_t base = n_layers - 1;
  if (j == base) return c->e_bc;
  if (k == base) return c->e_cb;
  return c->e_cc;
}

/* insertion sort of a short list of layer ids */
static void sort_ids(int32_t* a, int32_t n) {
  for (int32_t x = 1; x < n; ++x) {
    int32_t v = a[x], y = x - 1;
    while (y >= 0 && a[y] > v) { a[y + 1] = a[y]; --y; }
    a[y + 1] = v;
  }
}

/* ------------------------------------------------------------------------- */
/* L_t = Phi L^T (Algorithm 1, "L_t" line; Sec. 4 "Laplacian").  Vertex-    */
/* major: G(i, l) = sum over the stored entries (i, j) of L of L_ij F(j, l). */
/* The pattern is structural: every layer present at some j in row i of L.   */
/* Output rows are sorted by layer id.                                        */
/* ------------------------------------------------------------------------- */

/* per-thread scratch of one row of L_t: accumulators indexed by layer */
typedef struct { double* acc; double* aab; char* mark; int32_t* touched; } lt_scratch;

static int lt_scratch_init(lt_scratch* s, int32_t n_layers) {
  s->acc = (double*)calloc((size_t)n_layers, sizeof(double));
  s->aab = (double*)calloc((size_t)n_layers, sizeof(double));
  s->mark = (char*)calloc((size_t)n_layers, 1);
  s->touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_layers);
  return s->acc && s->aab && s->mark && s->touched;
}

static void lt_scratch_free(lt_scratch* s) {
  free(s->acc); free(s->aab); free(s->mark); free(s->touched);
}

/* Row i of G: the layers touched, sorted, left in s->touched[0..return) with
 * their sums in s->acc and the sums of the magnitudes of the products in
 * s->aab (indexed by layer); s->mark stays set until lt_row_clear. */
static int32_t lt_row(int64_t i, const int64_t* Lrp, const int32_t* Lcol, const double* Lval,
                      const int64_t* Frp, const int32_t* Fid, const double* Fval, lt_scratch* s) {
  int32_t nt = 0;
  for (int64_t q = Lrp[i]; q < Lrp[i + 1]; ++q) {
    int32_t j = Lcol[q];
    double lij = Lval[q];
    for (int64_t p = Frp[j]; p < Frp[j + 1]; ++p) {
      int32_t l = Fid[p];
      if (!s->mark[l]) { s->mark[l] = 1; s->touched[nt++] = l; s->acc[l] = 0.0; s->aab[l] = 0.0; }
      s->acc[l] += lij * Fval[p];
      s->aab[l] += fabs(lij * Fval[p]);
    }
  }
  sort_ids(s->touched, nt);
  return nt;
}

static void lt_row_clear(lt_scratch* s, int32_t nt) {
  for (int32_t x = 0; x < nt; ++x) s->mark[s->touched[x]] = 0;
}

/* Returns nnz(G), or -(needed) - 16 when cap is too small, or a negative
 * error code. */
static int64_t lt_product(int64_t n_v, int32_t n_layers,
                          const int64_t* Lrp, const int32_t* Lcol, const double* Lval,
                          const int64_t* Frp, const int32_t* Fid, const double* Fval,
                          int64_t cap, int64_t* Grp, int32_t* Gid, double* Gval, double* Gabs) {
  lt_scratch s;
  if (!lt_scratch_init(&s, n_layers)) { lt_scratch_free(&s); return ORC_ERR_NOMEM; }
  int64_t o = 0;
  Grp[0] = 0;
  for (int64_t i = 0; i < n_v; ++i) {
    int32_t nt = lt_row(i, Lrp, Lcol, Lval, Frp, Fid, Fval, &s);
    for (int32_t x = 0; x < nt; ++x) {
      if (o < cap) {
        Gid[o] = s.touched[x];
        Gval[o] = s.acc[s.touched[x]];
        if (Gabs) Gabs[o] = s.aab[s.touched[x]];
      }
      ++o;
    }
    lt_row_clear(&s, nt);
    Grp[i + 1] = o;
  }
  lt_scratch_free(&s);
  return o > cap ? -o - 16 : o;
}

int64_t orc_lt(int64_t n_v, int32_t n_layers,
               const int64_t* Lrp, const int32_t* Lcol, const double* Lval,
               const int64_t* Frp, const int32_t* Fid, const double* Fval,
               int64_t cap, int64_t* Grp, int32_t* Gid, double* Gval) {
  return lt_product(n_v, n_layers, Lrp, Lcol, Lval, Frp, Fid, Fval, cap, Grp, Gid, Gval, NULL);
}

/* per-thread scratch of one vertex's update: the interest entries */
typedef struct { int32_t* S; double* SF; double* SG; double* SGa; } upd_scratch;

static int upd_scratch_init(upd_scratch* u, int32_t n_layers) {
  u->S = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_layers);
  u->SF = (double*)malloc(sizeof(double) * (size_t)n_layers);
  u->SG = (double*)malloc(sizeof(double) * (size_t)n_layers);
  u->SGa = (double*)malloc(sizeof(double) * (size_t)n_layers);
  return u->S && u->SF && u->SG && u->SGa;
}

static void upd_scratch_free(upd_scratch* u) {
  free(u->S); free(u->SF); free(u->SG); free(u->SGa);
}

/*
 * Steps (2) and (3) below for one vertex: the sorted rows F(i, .) (nf
 * entries) and G(i, .) (ng entries, with the magnitude sums gab) are merged;
 * the interest entries get the explicit Euler update and the clamp.  Writes
 * the n interest entries (ids ascending, values not yet normalised) to
 * Hid/Hval and returns n; mg3 (nullable) receives the margins described at
 * orc_step.
 */
static int32_t vertex_update(const orc_coefs* cp, int32_t n_layers, const double* Wm, const double* Am,
                             const double* Em, const int32_t* fid, const double* fval, int64_t nf,
                             const int32_t* gid, const double* gval, const double* gab, int64_t ng,
                             upd_scratch* u, int32_t* Hid, double* Hval, double* mg3) {
  const orc_coefs c = *cp;
  int32_t* S = u->S;
  double* SF = u->SF;
  double* SG = u->SG;
  double* SGa = u->SGa;
  /* merge the sorted patterns of F(i, .) and G(i, .) */
  int64_t pf = 0, pg = 0;
  int32_t n = 0;
  double mG = HUGE_VAL, mC = HUGE_VAL;
  while (pf < nf || pg < ng) {
    int32_t lf = pf < nf ? fid[pf] : INT32_MAX;
    int32_t lg = pg < ng ? gid[pg] : INT32_MAX;
    int32_t l = lf < lg ? lf : lg;
    double fv = (lf == l) ? fval[pf] : 0.0;
    double gv = (lg == l) ? gval[pg] : 0.0;
    double ga = (lg == l) ? gab[pg] : 0.0;
    if (lf == l) ++pf;
    if (lg == l) ++pg;
    if (fv == 0.0 && ga > 0.0 && fabs(gv) / ga < mG) mG = fabs(gv) / ga;
    if (fv > 0.0 || (fv == 0.0 && gv > 0.0)) {
      S[n] = l; SF[n] = fv; SG[n] = gv; SGa[n] = ga; ++n;
    }
  }
  for (int32_t jj = 0; jj < n; ++jj) {
    int32_t j = S[jj];
    double d = 0.0, dabs = 0.0;
    for (int32_t kk = 0; kk < n; ++kk) {
      int32_t kx = S[kk];
      double sum = 0.0, sabs = 0.0;
      for (int32_t ll = 0; ll < n; ++ll) {
        int32_t l = S[ll];
        double ca = 0.5 * (coef_sym(Am, c.a_cc, c.a_cb, n_layers, j, l) - coef_sym(Am, c.a_cc, c.a_cb, n_layers, kx, l));
        double tw = (coef_sym(Wm, c.w_cc, c.w_cb, n_layers, j, l) - coef_sym(Wm, c.w_cc, c.w_cb, n_layers, kx, l)) * SF[ll];
        sum += ca * SG[ll] + tw;
        sabs += fabs(ca) * SGa[ll] + fabs(tw);
      }
      double te = coef_e(Em, &c, n_layers, j, kx) * sqrt(SF[jj] * SF[kk]);
      d += -(c.mu / n) * (sum - te);
      dabs += (c.mu / n) * (sabs + fabs(te));
    }
    double v = SF[jj] + d * c.dt;
    double vscale = fabs(SF[jj]) + c.dt * dabs;
    if (vscale > 0.0 && fabs(v) / vscale < mC) mC = fabs(v) / vscale;
    if (v > 1.0) v = 1.0;
    if (v <= 0.0) v = 0.0;
    Hid[jj] = j;
    Hval[jj] = v;
  }
  if (mg3) {
    mg3[0] = mG;
    mg3[1] = mC;
    mg3[2] = (double)n;
  }
  return n;
}

/* Step (4) for one vertex: divide its n entries by their sum.  Returns 0, or
 * ORC_ERR_ZERO_SUM when the sum is not positive. */
static int normalise_row(double* Hval, int64_t n) {
  double s = 0.0;
  for (int64_t p = 0; p < n; ++p) s += Hval[p];
  if (!(s > 0.0)) return ORC_ERR_ZERO_SUM;
  for (int64_t p = 0; p < n; ++p) Hval[p] = Hval[p] / s;
  return ORC_OK;
}

/*
 * One explicit time-iteration (the body of the time loop of Algorithm 1),
 * in the paper's order:
 *   (1) L_t = Phi L^T, here G = L F (lt_product above);
 *   (2) for every vertex i, the interest rows irows = {l : F(i,l) > 0} union
 *       {l : F(i,l) = 0 and G(i,l) > 0} and n_i = |irows| (Sec. 4 "Update",
 *       the interest skeleton);
 *   (3) for j in irows: d = sum_k -(mu/n_i) (sum_jk - e_jk sqrt(F_j F_k)),
 *       sum_jk = sum_l 1/2 (a_jl - a_kl) G_l + (w_jl - w_kl) F_l, all three
 *       indices over irows (Eq. 11-13 as Algorithm 1 evaluates them);
 *       F_j + d dt, then clamp: above 1 -> 1, at or below 0 -> 0;
 *   (4) normalise every vertex (a column of Phi) by the sum of its entries;
 *   (5) drop the zero entries (Sec. 4 "Normalization", compaction).
 * READING (Sec. 4 "Update": the output is an updated copy of Phi-hat): every
 * d uses the pre-step values (Jacobi), not values updated in place.
 * READING: the divisor is n_i = |irows| (Algorithm 1), not the global n of Eq. 11.
 *
 * coefs: see above.  Wm/Am/Em: optional dense coefficient matrices.
 * Output arrays have capacity out_cap.  Returns the output nnz, or
 * -(needed nnz) - 16 when out_cap is too small, or a negative error code.
 * skeleton: if non-NULL receives sum_i n_i.
 * margins: if non-NULL, 3 doubles per vertex describing how far its two
 *   discrete decisions are from flipping under rounding:
 *   [0] min over the entries of G with F(i,l) = 0 of |G_il| / sum_j |L_ij F_jl|
 *       (the irows test),
 *   [1] min over irows of |F_j + d dt| / (|F_j| + dt sum of |terms of d|),
 *       each G_l in those terms counted as sum_j |L_ij F_jl| since G_l is
 *       itself a cancelling sum (the clamp to zero),
 *   [2] n_i.  HUGE_VAL where there is no such entry.
 */
int64_t orc_step(int64_t n_v, int32_t n_layers,
                 const int64_t* Lrp, const int32_t* Lcol, const double* Lval,
                 const int64_t* Frp, const int32_t* Fid, const double* Fval,
                 const double* coefs, const double* Wm, const double* Am, const double* Em,
                 int64_t out_cap, int64_t* Orp, int32_t* Oid, double* Oval,
                 int64_t* skeleton, double* margins) {
  const orc_coefs c = unpack(coefs);
  int64_t ret = 0;
  int64_t* Grp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_v + 1));
  int64_t gcap = 8 * (Frp[n_v] + n_v) + 16;
  int32_t* Gid = NULL;
  double* Gval = NULL;
  double* Gab = NULL;
  int64_t* Hrp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_v + 1));
  int32_t* Hid = NULL;
  double* Hval = NULL;
  upd_scratch u;
  int uok = upd_scratch_init(&u, n_layers);
  if (!Grp || !Hrp || !uok) { ret = ORC_ERR_NOMEM; goto done; }

  /* (1) L_t */
  for (;;) {
    Gid = (int32_t*)malloc(sizeof(int32_t) * (size_t)gcap);
    Gval = (double*)malloc(sizeof(double) * (size_t)gcap);
    Gab = (double*)malloc(sizeof(double) * (size_t)gcap);
    if (!Gid || !Gval || !Gab) { ret = ORC_ERR_NOMEM; goto done; }
    int64_t g = lt_product(n_v, n_layers, Lrp, Lcol, Lval, Frp, Fid, Fval, gcap, Grp, Gid, Gval, Gab);
    if (g >= 0) break;
    free(Gid); free(Gval); free(Gab); Gid = NULL; Gval = NULL; Gab = NULL;
    if (g > -16) { ret = g; goto done; }
    gcap = -(g + 16);
  }

  /* (2)+(3): interest skeleton and the update into the copy Phi-hat (H) */
  int64_t hcap = Grp[n_v] + Frp[n_v] + 1;
  Hid = (int32_t*)malloc(sizeof(int32_t) * (size_t)hcap);
  Hval = (double*)malloc(sizeof(double) * (size_t)hcap);
  if (!Hid || !Hval) { ret = ORC_ERR_NOMEM; goto done; }
  int64_t skel = 0;
  Hrp[0] = 0;
  for (int64_t i = 0; i < n_v; ++i) {
    int32_t n = vertex_update(&c, n_layers, Wm, Am, Em, Fid + Frp[i], Fval + Frp[i], Frp[i + 1] - Frp[i],
                              Gid + Grp[i], Gval + Grp[i], Gab + Grp[i], Grp[i + 1] - Grp[i], &u,
                              Hid + Hrp[i], Hval + Hrp[i], margins ? margins + 3 * i : NULL);
    skel += n;
    Hrp[i + 1] = Hrp[i] + n;
  }
  if (skeleton) *skeleton = skel;

  /* (4) normalise each vertex by the sum of its entries */
  for (int64_t i = 0; i < n_v; ++i) {
    if (normalise_row(Hval + Hrp[i], Hrp[i + 1] - Hrp[i]) != ORC_OK) { ret = ORC_ERR_ZERO_SUM; goto done; }
  }

  /* (5) compaction: keep the nonzero entries */
  {
    int64_t nnz = 0;
    for (int64_t p = 0; p < Hrp[n_v]; ++p) nnz += (Hval[p] != 0.0);
    if (nnz > out_cap) { ret = -nnz - 16; goto done; }
    int64_t o = 0;
    Orp[0] = 0;
    for (int64_t i = 0; i < n_v; ++i) {
      for (int64_t p = Hrp[i]; p < Hrp[i + 1]; ++p) {
        if (Hval[p] != 0.0) { Oid[o] = Hid[p]; Oval[o] = Hval[p]; ++o; }
      }
      Orp[i + 1] = o;
    }
    ret = nnz;
  }

done:
  free(Grp); free(Gid); free(Gval); free(Gab); free(Hrp); free(Hid); free(Hval);
  upd_scratch_free(&u);
  return ret;
}

/*
 * The same time-iteration computed by several OpenMP threads (the timed CPU
 * baseline): each thread takes a contiguous range of vertices and runs
 * steps (1)-(5) for one vertex at a time with the helpers of orc_step, so
 * every vertex gets the same operations in the same order and the result is
 * identical to orc_step's.  Every vertex's work reads only the input, so the
 * threads need no locks; each keeps its output rows in a buffer of its own,
 * and a prefix sum of the per-thread counts places them in the output,
 * where every thread copies its own rows.
 * n_threads <= 0 uses every online core.  Same outputs and return codes as
 * orc_step.
 */
typedef struct {
  int64_t lo, hi;
  int32_t n_layers;
  const int64_t *Lrp, *Frp;
  const int32_t *Lcol, *Fid;
  const double *Lval, *Fval, *Wm, *Am, *Em;
  const orc_coefs* c;
  double* margins;
  int64_t* counts;       /* per vertex: output entries */
  int32_t* oid;          /* this thread's output entries */
  double* oval;
  int64_t n_out, cap, skel;
  int err;
} mt_task;

static void* mt_worker(void* arg) {
  mt_task* t = (mt_task*)arg;
  lt_scratch s;
  upd_scratch u;
  int ok = lt_scratch_init(&s, t->n_layers) & upd_scratch_init(&u, t->n_layers);
  int32_t* gid = (int32_t*)malloc(sizeof(int32_t) * (size_t)t->n_layers);
  double* gval = (double*)malloc(sizeof(double) * (size_t)t->n_layers);
  double* gab = (double*)malloc(sizeof(double) * (size_t)t->n_layers);
  int32_t* hid = (int32_t*)malloc(sizeof(int32_t) * (size_t)t->n_layers);
  double* hval = (double*)malloc(sizeof(double) * (size_t)t->n_layers);
  t->cap = 1024;
  t->oid = (int32_t*)malloc(sizeof(int32_t) * (size_t)t->cap);
  t->oval = (double*)malloc(sizeof(double) * (size_t)t->cap);
  t->n_out = 0;
  t->skel = 0;
  t->err = ORC_OK;
  if (!ok || !gid || !gval || !gab || !hid || !hval || !t->oid || !t->oval) { t->err = ORC_ERR_NOMEM; goto out; }
  for (int64_t i = t->lo; i < t->hi; ++i) {
    int32_t ng = lt_row(i, t->Lrp, t->Lcol, t->Lval, t->Frp, t->Fid, t->Fval, &s);
    for (int32_t x = 0; x < ng; ++x) {
      gid[x] = s.touched[x];
      gval[x] = s.acc[s.touched[x]];
      gab[x] = s.aab[s.touched[x]];
    }
    lt_row_clear(&s, ng);
    int32_t n = vertex_update(t->c, t->n_layers, t->Wm, t->Am, t->Em, t->Fid + t->Frp[i], t->Fval + t->Frp[i],
                              t->Frp[i + 1] - t->Frp[i], gid, gval, gab, ng, &u, hid, hval,
                              t->margins ? t->margins + 3 * i : NULL);
    t->skel += n;
    if (normalise_row(hval, n) != ORC_OK) { t->err = ORC_ERR_ZERO_SUM; goto out; }
    if (t->n_out + n > t->cap) {
      while (t->n_out + n > t->cap) t->cap *= 2;
      int32_t* a = (int32_t*)realloc(t->oid, sizeof(int32_t) * (size_t)t->cap);
      if (a) t->oid = a;
      double* b = (double*)realloc(t->oval, sizeof(double) * (size_t)t->cap);
      if (b) t->oval = b;
      if (!a || !b) { t->err = ORC_ERR_NOMEM; goto out; }
    }
    int64_t kept = 0;
    for (int32_t p = 0; p < n; ++p) {
      if (hval[p] != 0.0) { t->oid[t->n_out + kept] = hid[p]; t->oval[t->n_out + kept] = hval[p]; ++kept; }
    }
    t->n_out += kept;
    t->counts[i] = kept;
  }
out:
  lt_scratch_free(&s);
  upd_scratch_free(&u);
  free(gid); free(gval); free(gab); free(hid); free(hval);
  return NULL;
}

int64_t orc_step_threads(int32_t n_threads, int64_t n_v, int32_t n_layers,
                         const int64_t* Lrp, const int32_t* Lcol, const double* Lval,
                         const int64_t* Frp, const int32_t* Fid, const double* Fval,
                         const double* coefs, const double* Wm, const double* Am, const double* Em,
                         int64_t out_cap, int64_t* Orp, int32_t* Oid, double* Oval,
                         int64_t* skeleton, double* margins) {
  const orc_coefs c = unpack(coefs);
  if (n_threads <= 0) n_threads = omp_get_num_procs();
  if (n_threads > n_v) n_threads = n_v > 0 ? (int32_t)n_v : 1;
  mt_task* tasks = (mt_task*)calloc((size_t)n_threads, sizeof(mt_task));
  int64_t* counts = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_v > 0 ? n_v : 1));
  int64_t* offs = (int64_t*)calloc((size_t)n_threads + 1, sizeof(int64_t));
  if (!tasks || !counts || !offs) { free(tasks); free(counts); free(offs); return ORC_ERR_NOMEM; }
  int64_t ret = 0, nnz = 0, skel = 0;
  int nt_used = 1;
#pragma omp parallel num_threads(n_threads)
  {
    const int k = omp_get_thread_num();
    const int nt = omp_get_num_threads();
    mt_task* t = &tasks[k];
    t->lo = n_v * k / nt;
    t->hi = n_v * (k + 1) / nt;
    t->n_layers = n_layers;
    t->Lrp = Lrp; t->Lcol = Lcol; t->Lval = Lval;
    t->Frp = Frp; t->Fid = Fid; t->Fval = Fval;
    t->Wm = Wm; t->Am = Am; t->Em = Em;
    t->c = &c;
    t->margins = margins;
    t->counts = counts;
    mt_worker(t);
#pragma omp barrier
#pragma omp single
    {
      /* prefix sum of the per-thread counts: each thread's rows in place */
      nt_used = nt;
      for (int x = 0; x < nt; ++x) {
        if (tasks[x].err != ORC_OK && ret == 0) ret = tasks[x].err;
        offs[x + 1] = offs[x] + tasks[x].n_out;
        skel += tasks[x].skel;
      }
      nnz = offs[nt];
      if (ret == 0 && nnz > out_cap) ret = -nnz - 16;
    }
    if (ret == 0) {
      memcpy(Oid + offs[k], t->oid, sizeof(int32_t) * (size_t)t->n_out);
      memcpy(Oval + offs[k], t->oval, sizeof(double) * (size_t)t->n_out);
      int64_t o = offs[k];
      if (k == 0) Orp[0] = 0;
      for (int64_t i = t->lo; i < t->hi; ++i) {
        o += counts[i];
        Orp[i + 1] = o;
      }
    }
  }
  if (ret == 0) {
    if (skeleton) *skeleton = skel;
    ret = nnz;
  }
  for (int32_t x = 0; x < nt_used && x < n_threads; ++x) { free(tasks[x].oid); free(tasks[x].oval); }
  free(tasks); free(counts); free(offs);
  return ret;
}

/*
 * Closed form of the same update for the class coefficients, used only to
 * cross-check the literal triple loop.  With S = C u B (C the cell layers of
 * irows, B = {base} or empty, n = |S|), Algorithm 1's double sum over k and l
 * collapses because sum_jk = 1/2 (A_j - A_k) + (W_j - W_k), where
 * A_j = sum_{l in S} a_jl G_l and W_j = sum_{l in S} w_jl F_l:
 *   d_j = -(mu/n) [ 1/2 (n A_j - sum_S A) + (n W_j - sum_S W) ]
 *         + (mu/n) sqrt(F_j) sum_{k in S} e_jk sqrt(F_k).
 * For a cell j: A_j = a_cc (sG_C - G_j) + [B] a_cb G_b;  for the base:
 * A_b = a_cb sG_C (likewise W with w and F), with sG_C the sum over C.
 * Same phases and outputs as orc_step.
 */
int64_t orc_step_closed(int64_t n_v, int32_t n_layers,
                        const int64_t* Lrp, const int32_t* Lcol, const double* Lval,
                        const int64_t* Frp, const int32_t* Fid, const double* Fval,
                        const double* coefs, int64_t out_cap, int64_t* Orp, int32_t* Oid, double* Oval,
                        int64_t* skeleton) {
  const orc_coefs c = unpack(coefs);
  const int32_t base = n_layers - 1;
  double* acc = (double*)calloc((size_t)n_layers, sizeof(double));
  char* mark = (char*)calloc((size_t)n_layers, 1);
  int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_layers);
  double* SF = (double*)malloc(sizeof(double) * (size_t)n_layers);
  double* SG = (double*)malloc(sizeof(double) * (size_t)n_layers);
  int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_layers);
  double* fval = (double*)calloc((size_t)n_layers, sizeof(double));
  int64_t ret = 0, skel = 0, o = 0;
  int overflow = 0;
  if (!acc || !mark || !touched || !SF || !SG || !S || !fval) { ret = ORC_ERR_NOMEM; goto done2; }
  Orp[0] = 0;
  for (int64_t i = 0; i < n_v; ++i) {
    int32_t nt = 0;
    for (int64_t q = Lrp[i]; q < Lrp[i + 1]; ++q) {
      int32_t j = Lcol[q];
      for (int64_t p = Frp[j]; p < Frp[j + 1]; ++p) {
        int32_t l = Fid[p];
        if (!mark[l]) { mark[l] = 1; touched[nt++] = l; acc[l] = 0.0; }
        acc[l] += Lval[q] * Fval[p];
      }
    }
    for (int64_t p = Frp[i]; p < Frp[i + 1]; ++p) {
      int32_t l = Fid[p];
      fval[l] = Fval[p];
      if (!mark[l]) { mark[l] = 1; touched[nt++] = l; acc[l] = 0.0; }
    }
    sort_ids(touched, nt);
    int32_t n = 0;
    for (int32_t x = 0; x < nt; ++x) {
      int32_t l = touched[x];
      double fv = fval[l], gv = acc[l];
      if (fv > 0.0 || (fv == 0.0 && gv > 0.0)) { S[n] = l; SF[n] = fv; SG[n] = gv; ++n; }
      mark[l] = 0;
      fval[l] = 0.0;
    }
    skel += n;
    /* per-vertex sums over the cell layers of S and the base entry */
    double sG = 0.0, sF = 0.0, r = 0.0, Gb = 0.0, Fb = 0.0;
    int32_t nC = 0, hasb = 0;
    for (int32_t x = 0; x < n; ++x) {
      if (S[x] == base) { hasb = 1; Gb = SG[x]; Fb = SF[x]; }
      else { sG += SG[x]; sF += SF[x]; r += sqrt(SF[x]); ++nC; }
    }
    double sumA = c.a_cc * (nC - 1) * sG + (hasb ? c.a_cb * (nC * Gb + sG) : 0.0);
    double sumW = c.w_cc * (nC - 1) * sF + (hasb ? c.w_cb * (nC * Fb + sF) : 0.0);
    double tot = 0.0;
    for (int32_t x = 0; x < n; ++x) {
      double A, W, R;
      if (S[x] == base) {
        A = c.a_cb * sG; W = c.w_cb * sF; R = c.e_bc * r;
      } else {
        A = c.a_cc * (sG - SG[x]) + (hasb ? c.a_cb * Gb : 0.0);
        W = c.w_cc * (sF - SF[x]) + (hasb ? c.w_cb * Fb : 0.0);
        R = c.e_cc * (r - sqrt(SF[x])) + (hasb ? c.e_cb * sqrt(Fb) : 0.0);
      }
      double d = -(c.mu / n) * (0.5 * (n * A - sumA) + (n * W - sumW)) + (c.mu / n) * sqrt(SF[x]) * R;
      double v = SF[x] + d * c.dt;
      if (v > 1.0) v = 1.0;
      if (v <= 0.0) v = 0.0;
      SF[x] = v;
      tot += v;
    }
    if (!(tot > 0.0)) { ret = ORC_ERR_ZERO_SUM; goto done2; }
    for (int32_t x = 0; x < n; ++x) {
      double v = SF[x] / tot;
      if (v != 0.0) {
        if (o < out_cap) { Oid[o] = S[x]; Oval[o] = v; } else { overflow = 1; }
        ++o;
      }
    }
    Orp[i + 1] = o;
  }
  ret = overflow ? -o - 16 : o;
  if (skeleton) *skeleton = skel;
done2:
  free(acc); free(mark); free(touched); free(SF); free(SG); free(S); free(fval);
  return ret;
}

/* ------------------------------------------------------------------------- */
/* Sharp labels (Sec. 6, Fig. "beetle_mesh": the field of largest influence  */
/* at each vertex).  READING: ties go to the lowest layer id; a vertex whose  */
/* largest entry is the base layer (id n_layers - 1) is labelled -1.          */
/* ------------------------------------------------------------------------- */
int orc_labels(int64_t n_v, int32_t n_layers, const int64_t* Frp, const int32_t* Fid, const double* Fval,
               int32_t* labels, double* maxval) {
  for (int64_t i = 0; i < n_v; ++i) {
    int32_t best = -1;
    double bv = -HUGE_VAL;
    for (int64_t p = Frp[i]; p < Frp[i + 1]; ++p) {
      if (Fval[p] > bv || (Fval[p] == bv && Fid[p] < best)) { bv = Fval[p]; best = Fid[p]; }
    }
    labels[i] = (best == n_layers - 1) ? -1 : best;
    if (maxval) maxval[i] = bv;
  }
  return ORC_OK;
}
