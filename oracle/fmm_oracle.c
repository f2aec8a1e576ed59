/*
 * fmm_oracle.c -- plain, slow, FP64 CPU oracle of the angular-momentum
 * conserving Cartesian FMM (Marcello 2017, arXiv:1706.06989, built on
 * Dehnen 2000).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it (through oracle/__init__.py).  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * Compile with -ffp-contract=off: the centre of mass, R_max and the opening
 * criterion are evaluated here in a fixed order of correctly rounded
 * operations, and the CUDA tree must reproduce them bit for bit.
 *
 * What each stage follows:
 *   Morton keys / octree ........ Sec. 2 (cells hold at most n_crit bodies)
 *   Z, R_max, opening criterion . Sec. 2, opening criterion (Eq. preceding
 *                                  Eq. 1) and the definitions after it
 *   moments ...................... Eqs. (1)-(3), octupole definition after the
 *                                  net torque equation, generalised moments of
 *                                  App. A -- computed from their definition,
 *                                  directly from the bodies of every cell
 *   D tensors .................... the four printed derivatives of G=-1/R
 *                                  (Sec. 2) and the fourth derivative that the
 *                                  torque correction needs (derived)
 *   M2L at P=3 ................... Eqs. (3), (4) evaluated at every body of
 *                                  the two cells (no L2L shift: the plain form)
 *   TC / TCO correction .......... Eq. (7) and Eq. (8) with the coefficient
 *                                  of App. A (1/(n!(P-n)!) = 1/6 at P=3)
 *   general order P .............. App. A: accelerations on A and B, the
 *                                  corrective force F_c and the projected
 *                                  alternative F'_c
 *   near field ................... Sec. 2: remaining nearby bodies summed
 *                                  directly (each pair once, both bodies)
 *   balance metric, errors ....... Sec. 3 (numerical test)
 *
 * Readings of the paper that this file takes (the paper's R = Z_B - Z_A
 * disagrees with the printed Taylor series):
 *   - every derivative tensor is evaluated at r = Z_A - Z_B, the vector from
 *     B's centre to A's centre; Eqs. (3) and (4) are then used as printed;
 *   - the corrective force of Eq. (7) is
 *       F_c,i = (1/6) (M_A O_B,jkl - O_A,jkl M_B) D_ijkl(r),
 *     applied as +F_c/M_A to every body of A and -F_c/M_B to every body of B;
 *   - dipole moments about a centre of mass vanish analytically and are not
 *     fed into the order-3 interaction (Sec. 2 notes that they drop out);
 *   - a pair of bodies (or cells) at zero separation contributes nothing.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "fmm_oracle.h"

#define MAXLEVEL 21

/* ------------------------------------------------------------------------ */
/* state                                                                     */
/* ------------------------------------------------------------------------ */

struct orc {
  int n, n_crit, P;
  double theta;
  double eps2; /* Plummer softening length squared (0: the unsoftened 1/R) */
  /* Morton keys: bounding cube origin and scale */
  double lo[3], scale;
  uint64_t *key; /* sorted keys */
  int *order;    /* sorted position -> caller index */
  double *X[3];  /* sorted positions */
  double *mu;    /* sorted masses */
  /* cells (breadth-first numbering) */
  int ncell, cap;
  int *begin, *count, *level, *parent, *first_child, *nchild;
  double *S[3], *M, *Z[3], *Rmax;
  int nmom;     /* moments of order 0..P, multi-index (a,b,c) */
  double *mom;  /* [ncell][nmom] */
  /* interaction lists */
  int n_m2l, cap_m2l, *m2l; /* pairs (A,B), A<B */
  int n_p2p, cap_p2p, *p2p; /* leaf pairs (A,B), A<B */
  int n_self, cap_self, *self;
};

static void *xmalloc(size_t n) {
  void *p = malloc(n ? n : 1);
  if (!p) abort();
  return p;
}
static void *xcalloc(size_t n, size_t s) {
  void *p = calloc(n ? n : 1, s ? s : 1);
  if (!p) abort();
  return p;
}

/* ------------------------------------------------------------------------ */
/* multi-indices: moments and derivatives of total order n are stored by    */
/* exponent triple (a,b,c), a+b+c = n, in the order a = n..0, b = n-a..0.   */
/* ------------------------------------------------------------------------ */

static int mi_offset(int n) { return n * (n + 1) * (n + 2) / 6; }

static int mi_index(int a, int b, int c) {
  int n = a + b + c;
  /* position of (a,b,c) within order n */
  int pos = 0;
  for (int aa = n; aa > a; --aa) pos += n - aa + 1;
  pos += (n - a) - b;
  (void)c;
  return mi_offset(n) + pos;
}

static int mi_count(int maxorder) { return mi_offset(maxorder + 1); }

/* index tuple (l_1..l_n) over {0,1,2} encoded in base 3, least significant
 * digit = l_1; return the multi-index slot of the symmetric component. */
static int mi_of_tuple(int n, int t) {
  int cnt[3] = {0, 0, 0};
  for (int s = 0; s < n; ++s) {
    cnt[t % 3]++;
    t /= 3;
  }
  return mi_index(cnt[0], cnt[1], cnt[2]);
}

static int ipow3(int n) {
  int p = 1;
  while (n-- > 0) p *= 3;
  return p;
}

static double factorial(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= k;
  return f;
}

/* ------------------------------------------------------------------------ */
/* a1: bounding cube and Morton keys                                         */
/* ------------------------------------------------------------------------ */

static uint64_t spread3(uint64_t q) {
  /* bit b of q goes to bit 3b */
  uint64_t k = 0;
  for (int b = 0; b < MAXLEVEL; ++b) k |= ((q >> b) & 1ull) << (3 * b);
  return k;
}

static uint64_t quantise(double v, double lo, double scale) {
  double t = (v - lo) * scale;
  double f = floor(t);
  const double qmax = (double)((1u << MAXLEVEL) - 1);
  if (f > qmax) f = qmax;
  return (uint64_t)f;
}

int orc_morton(int n, const double *x, const double *y, const double *z,
               uint64_t *keys, double *lo_out, double *scale_out) {
  if (n < 1) return ORC_EINVAL;
  double lo[3] = {x[0], y[0], z[0]}, hi[3] = {x[0], y[0], z[0]};
  for (int i = 0; i < n; ++i) {
    const double p[3] = {x[i], y[i], z[i]};
    for (int d = 0; d < 3; ++d) {
      if (!isfinite(p[d])) return ORC_EINVAL;
      if (p[d] < lo[d]) lo[d] = p[d];
      if (p[d] > hi[d]) hi[d] = p[d];
    }
  }
  double ext = hi[0] - lo[0];
  if (hi[1] - lo[1] > ext) ext = hi[1] - lo[1];
  if (hi[2] - lo[2] > ext) ext = hi[2] - lo[2];
  /* scale = 2^21 / ext; a cube of zero extent maps every body to key 0 */
  double scale = ext > 0.0 ? (double)(1u << MAXLEVEL) / ext : 0.0;
  for (int i = 0; i < n; ++i) {
    uint64_t qx = quantise(x[i], lo[0], scale);
    uint64_t qy = quantise(y[i], lo[1], scale);
    uint64_t qz = quantise(z[i], lo[2], scale);
    keys[i] = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
  }
  for (int d = 0; d < 3; ++d) lo_out[d] = lo[d];
  *scale_out = scale;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a2: sort by (key, caller index)                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t key;
  int idx;
} keyidx;

static int cmp_keyidx(const void *pa, const void *pb) {
  const keyidx *a = (const keyidx *)pa, *b = (const keyidx *)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return (a->idx > b->idx) - (a->idx < b->idx);
}

/* ------------------------------------------------------------------------ */
/* a3: octree, breadth-first                                                 */
/* ------------------------------------------------------------------------ */

static int digit_at(uint64_t key, int level) {
  /* octant digit selecting the child at `level` (1..21) */
  return (int)((key >> (3 * (MAXLEVEL - level))) & 7ull);
}

static int is_leaf(const struct orc *t, int c) { return t->nchild[c] == 0; }

static void grow_cells(struct orc *t, int need) {
  if (need <= t->cap) return;
  int cap = t->cap ? t->cap : 64;
  while (cap < need) cap *= 2;
  int **iv[] = {&t->begin, &t->count, &t->level, &t->parent, &t->first_child, &t->nchild};
  for (int k = 0; k < 6; ++k) {
    int *p = (int *)realloc(*iv[k], sizeof(int) * (size_t)cap);
    if (!p) abort();
    *iv[k] = p;
  }
  t->cap = cap;
}

static void build_tree(struct orc *t) {
  t->ncell = 0;
  grow_cells(t, 1);
  t->begin[0] = 0;
  t->count[0] = t->n;
  t->level[0] = 0;
  t->parent[0] = -1;
  t->first_child[0] = -1;
  t->nchild[0] = 0;
  t->ncell = 1;
  /* FIFO over cells in id order: children are appended level by level, and
   * within a level in the order of their parents and octants, i.e. by key
   * prefix. */
  for (int c = 0; c < t->ncell; ++c) {
    const int b = t->begin[c], cnt = t->count[c], lev = t->level[c];
    /* leaf <=> at most n_crit bodies, or the key resolution is exhausted */
    if (cnt <= t->n_crit || lev == MAXLEVEL) continue;
    int first = t->ncell, nch = 0;
    int s = b;
    while (s < b + cnt) {
      int dgt = digit_at(t->key[s], lev + 1);
      int e = s + 1;
      while (e < b + cnt && digit_at(t->key[e], lev + 1) == dgt) ++e;
      grow_cells(t, t->ncell + 1);
      int k = t->ncell++;
      t->begin[k] = s;
      t->count[k] = e - s;
      t->level[k] = lev + 1;
      t->parent[k] = c;
      t->first_child[k] = -1;
      t->nchild[k] = 0;
      ++nch;
      s = e;
    }
    t->first_child[c] = first;
    t->nchild[c] = nch;
  }
}

/* ------------------------------------------------------------------------ */
/* a4: centre of mass, R_max, moments                                        */
/* ------------------------------------------------------------------------ */

static void upward(struct orc *t) {
  const int nc = t->ncell;
  for (int d = 0; d < 3; ++d) {
    t->S[d] = (double *)xmalloc(sizeof(double) * nc);
    t->Z[d] = (double *)xmalloc(sizeof(double) * nc);
  }
  t->M = (double *)xmalloc(sizeof(double) * nc);
  t->Rmax = (double *)xmalloc(sizeof(double) * nc);
  /* mass and mass-weighted position sum: a leaf sums its bodies in sorted
   * order, any other cell sums its children in octant order; Z = S / M. */
  for (int c = nc - 1; c >= 0; --c) {
    double s[3] = {0.0, 0.0, 0.0}, m = 0.0;
    if (is_leaf(t, c)) {
      for (int i = t->begin[c]; i < t->begin[c] + t->count[c]; ++i) {
        for (int d = 0; d < 3; ++d) s[d] = s[d] + t->mu[i] * t->X[d][i];
        m = m + t->mu[i];
      }
    } else {
      for (int k = t->first_child[c]; k < t->first_child[c] + t->nchild[c]; ++k) {
        for (int d = 0; d < 3; ++d) s[d] = s[d] + t->S[d][k];
        m = m + t->M[k];
      }
    }
    for (int d = 0; d < 3; ++d) {
      t->S[d][c] = s[d];
      t->Z[d][c] = s[d] / m;
    }
    t->M[c] = m;
  }
  /* R_max: the largest distance from a body of the cell to its centre of
   * mass, over every body of the cell (exact, not a bound). */
  for (int c = 0; c < nc; ++c) {
    double best = 0.0;
    for (int i = t->begin[c]; i < t->begin[c] + t->count[c]; ++i) {
      double dx = t->X[0][i] - t->Z[0][c];
      double dy = t->X[1][i] - t->Z[1][c];
      double dz = t->X[2][i] - t->Z[2][c];
      double d2 = (dx * dx + dy * dy) + dz * dz;
      if (d2 > best) best = d2;
    }
    t->Rmax[c] = sqrt(best);
  }
  /* moments M_{l1..ln} = sum mu x_l1 .. x_ln about Z, n = 0..P, from their
   * definition over the bodies of the cell (Eqs. 1-3, App. A). */
  t->nmom = mi_count(t->P);
  t->mom = (double *)xcalloc((size_t)nc * t->nmom, sizeof(double));
  for (int c = 0; c < nc; ++c) {
    double *mc = t->mom + (size_t)c * t->nmom;
    for (int i = t->begin[c]; i < t->begin[c] + t->count[c]; ++i) {
      double x = t->X[0][i] - t->Z[0][c];
      double y = t->X[1][i] - t->Z[1][c];
      double z = t->X[2][i] - t->Z[2][c];
      for (int n = 0; n <= t->P; ++n)
        for (int a = n; a >= 0; --a)
          for (int b = n - a; b >= 0; --b) {
            int cc = n - a - b;
            double v = t->mu[i];
            for (int k = 0; k < a; ++k) v *= x;
            for (int k = 0; k < b; ++k) v *= y;
            for (int k = 0; k < cc; ++k) v *= z;
            mc[mi_index(a, b, cc)] += v;
          }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* a5, a6: dual-tree walk and opening criterion                              */
/* ------------------------------------------------------------------------ */

static void push_pair(int **arr, int *n, int *cap, int a, int b) {
  if (*n == *cap) {
    *cap = *cap ? 2 * *cap : 1024;
    int *p = (int *)realloc(*arr, sizeof(int) * 2 * (size_t)*cap);
    if (!p) abort();
    *arr = p;
  }
  (*arr)[2 * *n] = a < b ? a : b;
  (*arr)[2 * *n + 1] = a < b ? b : a;
  ++*n;
}

/* |Z_A - Z_B| >= (R_A + R_B) / theta, evaluated as
 * theta^2 * |Z_A - Z_B|^2 >= (R_A + R_B)^2 with equality accepted. */
static int well_separated(const struct orc *t, int A, int B) {
  double dx = t->Z[0][A] - t->Z[0][B];
  double dy = t->Z[1][A] - t->Z[1][B];
  double dz = t->Z[2][A] - t->Z[2][B];
  double d2 = (dx * dx + dy * dy) + dz * dz;
  double th2 = t->theta * t->theta;
  double s = t->Rmax[A] + t->Rmax[B];
  return th2 * d2 >= s * s;
}

static void walk(struct orc *t, int A, int B) {
  if (A == B) {
    if (is_leaf(t, A)) {
      if (t->n_self == t->cap_self) {
        t->cap_self = t->cap_self ? 2 * t->cap_self : 1024;
        int *p = (int *)realloc(t->self, sizeof(int) * (size_t)t->cap_self);
        if (!p) abort();
        t->self = p;
      }
      t->self[t->n_self++] = A;
      return;
    }
    const int f = t->first_child[A], k = t->nchild[A];
    for (int i = 0; i < k; ++i) walk(t, f + i, f + i);
    for (int i = 0; i < k; ++i)
      for (int j = i + 1; j < k; ++j) walk(t, f + i, f + j);
    return;
  }
  if (well_separated(t, A, B)) {
    push_pair(&t->m2l, &t->n_m2l, &t->cap_m2l, A, B);
    return;
  }
  const int la = is_leaf(t, A), lb = is_leaf(t, B);
  if (la && lb) {
    push_pair(&t->p2p, &t->n_p2p, &t->cap_p2p, A, B);
    return;
  }
  int split, other;
  if (la) {
    split = B;
    other = A;
  } else if (lb) {
    split = A;
    other = B;
  } else {
    /* larger R_max; ties to the shallower cell, then the smaller id */
    int pickA;
    if (t->Rmax[A] != t->Rmax[B]) pickA = t->Rmax[A] > t->Rmax[B];
    else if (t->level[A] != t->level[B]) pickA = t->level[A] < t->level[B];
    else pickA = A < B;
    split = pickA ? A : B;
    other = pickA ? B : A;
  }
  for (int c = t->first_child[split]; c < t->first_child[split] + t->nchild[split]; ++c)
    walk(t, c, other);
}

/* ------------------------------------------------------------------------ */
/* derivative tensors of G(R) = -1/R                                         */
/* ------------------------------------------------------------------------ */

/* D, D_i, D_ij, D_ijk as printed in Sec. 2, and the fourth derivative
 *   D_ijkl = -105 r_i r_j r_k r_l / R^9
 *            + 15 (d_ij r_k r_l + d_ik r_j r_l + d_il r_j r_k
 *                  + d_jk r_i r_l + d_jl r_i r_k + d_kl r_i r_j) / R^7
 *            - 3 (d_ij d_kl + d_ik d_jl + d_il d_jk) / R^5
 * obtained by differentiating D_ijk once more. */
static double kd(int i, int j) { return i == j ? 1.0 : 0.0; }

typedef struct {
  double D0, D1[3], D2[3][3], D3[3][3][3], D4[3][3][3][3];
} dtens;

static void dtensors(const double r[3], double eps2, dtens *T) {
  double R2 = ((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]) + eps2;
  double R = sqrt(R2);
  double R3 = R2 * R, R5 = R3 * R2, R7 = R5 * R2, R9 = R7 * R2;
  T->D0 = -1.0 / R;
  for (int i = 0; i < 3; ++i) {
    T->D1[i] = r[i] / R3;
    for (int j = 0; j < 3; ++j) {
      T->D2[i][j] = -(3.0 * r[i] * r[j] - kd(i, j) * R2) / R5;
      for (int k = 0; k < 3; ++k) {
        T->D3[i][j][k] = (15.0 * r[i] * r[j] * r[k] -
                          3.0 * (kd(i, j) * r[k] + kd(j, k) * r[i] + kd(k, i) * r[j]) * R2) / R7;
        for (int l = 0; l < 3; ++l) {
          double t4 = -105.0 * r[i] * r[j] * r[k] * r[l] / R9;
          double t2 = 15.0 * (kd(i, j) * r[k] * r[l] + kd(i, k) * r[j] * r[l] + kd(i, l) * r[j] * r[k] +
                              kd(j, k) * r[i] * r[l] + kd(j, l) * r[i] * r[k] + kd(k, l) * r[i] * r[j]) / R7;
          double t0 = -3.0 * (kd(i, j) * kd(k, l) + kd(i, k) * kd(j, l) + kd(i, l) * kd(j, k)) / R5;
          T->D4[i][j][k][l] = t4 + t2 + t0;
        }
      }
    }
  }
}

/* D'_ijkl of Eq. (8): D_ijkl with every term that carries the factor r_i
 * removed (i is the direction of the corrective force). */
static void dprime4(const double r[3], double eps2, double Dp[3][3][3][3]) {
  double R2 = ((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]) + eps2;
  double R = sqrt(R2);
  double R5 = R2 * R2 * R, R7 = R5 * R2;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l)
          Dp[i][j][k][l] =
              15.0 * (kd(i, j) * r[k] * r[l] + kd(i, k) * r[j] * r[l] + kd(i, l) * r[j] * r[k]) / R7 -
              3.0 * (kd(i, j) * kd(k, l) + kd(i, k) * kd(j, l) + kd(i, l) * kd(j, k)) / R5;
}

/* Derivative of any order of G = -1/R for one symmetric component, from the
 * chain rule on G(u), u = r.r:  d^n G / dr_{l1}..dr_{ln} is the sum over
 * every way of grouping the n slots into k pairs and n-2k singles of
 *   c_{n-k} * prod_{pairs} delta * prod_{singles} r,
 * with c_m = 2^m d^m G/du^m = -(-1)^m (2m-1)!! R^-(2m+1). */
static double dcoef(int m, double R) {
  double df = 1.0;
  for (int k = 2 * m - 1; k > 1; k -= 2) df *= k;
  double s = (m % 2 == 0) ? -1.0 : 1.0;
  return s * df / pow(R, 2 * m + 1);
}

static double pairings(const int *l, int n, int used, const double r[3], int npairs, double R) {
  int p = 0;
  while (p < n && (used >> p) & 1) ++p;
  if (p == n) return dcoef(n - npairs, R);
  double acc = r[l[p]] * pairings(l, n, used | (1 << p), r, npairs, R);
  for (int q = p + 1; q < n; ++q) {
    if ((used >> q) & 1) continue;
    if (l[p] != l[q]) continue;
    acc += pairings(l, n, used | (1 << p) | (1 << q), r, npairs + 1, R);
  }
  return acc;
}

static int dtensor_generic_e2(const double *r, double eps2, int n, double *out) {
  /* out[mi_index(a,b,c) - mi_offset(n)] for every (a,b,c) of order n */
  if (n < 0 || n > 12) return ORC_EINVAL;
  double R = sqrt(((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]) + eps2);
  for (int a = n; a >= 0; --a)
    for (int b = n - a; b >= 0; --b) {
      int c = n - a - b, l[16], s = 0;
      for (int k = 0; k < a; ++k) l[s++] = 0;
      for (int k = 0; k < b; ++k) l[s++] = 1;
      for (int k = 0; k < c; ++k) l[s++] = 2;
      out[mi_index(a, b, c) - mi_offset(n)] = pairings(l, n, 0, r, 0, R);
    }
  return ORC_OK;
}

int orc_dtensor_generic(const double *r, double eps, int n, double *out) {
  return dtensor_generic_e2(r, eps * eps, n, out);
}

int orc_dtensor_p3(const double *r, double eps, double *d0, double *d1, double *d2, double *d3, double *d4,
                   double *d4prime) {
  dtens T;
  dtensors(r, eps * eps, &T);
  *d0 = T.D0;
  memcpy(d1, T.D1, sizeof T.D1);
  memcpy(d2, T.D2, sizeof T.D2);
  memcpy(d3, T.D3, sizeof T.D3);
  memcpy(d4, T.D4, sizeof T.D4);
  double Dp[3][3][3][3];
  dprime4(r, eps * eps, Dp);
  memcpy(d4prime, Dp, sizeof Dp);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a7: one accepted pair at P = 3, Eqs. (3), (4), (7), (8)                   */
/* ------------------------------------------------------------------------ */

static void cell_q_o(const struct orc *t, int c, double Q[3][3], double O[3][3][3]) {
  const double *mc = t->mom + (size_t)c * t->nmom;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Q[i][j] = mc[mi_of_tuple(2, i + 3 * j)];
      for (int k = 0; k < 3; ++k) O[i][j][k] = mc[mi_of_tuple(3, i + 3 * j + 9 * k)];
    }
}

/* Adds the accelerations that the interaction of the well-separated cells A
 * and B induces on every body of A and of B (sorted-order arrays acc[3]). */
static void m2l_p3_pair(const struct orc *t, int A, int B, int variant, double *acc[3],
                        const unsigned char *want) {
  double r[3] = {t->Z[0][A] - t->Z[0][B], t->Z[1][A] - t->Z[1][B], t->Z[2][A] - t->Z[2][B]};
  if ((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2] == 0.0) return;
  dtens T;
  dtensors(r, t->eps2, &T);
  const double MA = t->M[A], MB = t->M[B];
  double QA[3][3], OA[3][3][3], QB[3][3], OB[3][3][3];
  cell_q_o(t, A, QA, OA);
  cell_q_o(t, B, QB, OB);

  /* body-independent brackets of Eq. (3) (field of B in A) and Eq. (4)
   * (field of A in B), with the dipole terms dropped */
  double a0[3], b0[3];
  for (int i = 0; i < 3; ++i) {
    double qa = 0.0, qb = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        qb += QB[j][k] * T.D3[i][j][k];
        qa += QA[j][k] * T.D3[i][j][k];
      }
    a0[i] = MB * T.D1[i] + 0.5 * qb;
    b0[i] = -MA * T.D1[i] - 0.5 * qa;
  }
  /* corrective force, Eq. (7) (TC) or Eq. (8) (TCO) */
  double F[3] = {0.0, 0.0, 0.0};
  if (variant != ORC_UC) {
    double Dp[3][3][3][3];
    if (variant == ORC_TCO) dprime4(r, t->eps2, Dp);
    for (int i = 0; i < 3; ++i) {
      double f = 0.0;
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) {
            double w = MA * OB[j][k][l] - OA[j][k][l] * MB;
            double D = variant == ORC_TC ? T.D4[i][j][k][l] : Dp[i][j][k][l];
            f += w * D;
          }
      F[i] = f / 6.0;
    }
  }
  /* Eq. (3) at every body of A, plus F_c / M_A */
  for (int n = t->begin[A]; n < t->begin[A] + t->count[A]; ++n) {
    if (want && !want[n]) continue;
    double x[3] = {t->X[0][n] - t->Z[0][A], t->X[1][n] - t->Z[1][A], t->X[2][n] - t->Z[2][A]};
    for (int i = 0; i < 3; ++i) {
      double lin = 0.0, quad = 0.0;
      for (int j = 0; j < 3; ++j) {
        lin += x[j] * MB * T.D2[i][j];
        for (int k = 0; k < 3; ++k) quad += x[j] * x[k] * MB * T.D3[i][j][k];
      }
      double g = -(a0[i] + lin + 0.5 * quad);
      acc[i][n] += g + F[i] / MA;
    }
  }
  /* Eq. (4) at every body of B, minus F_c / M_B */
  for (int n = t->begin[B]; n < t->begin[B] + t->count[B]; ++n) {
    if (want && !want[n]) continue;
    double y[3] = {t->X[0][n] - t->Z[0][B], t->X[1][n] - t->Z[1][B], t->X[2][n] - t->Z[2][B]};
    for (int i = 0; i < 3; ++i) {
      double lin = 0.0, quad = 0.0;
      for (int j = 0; j < 3; ++j) {
        lin += y[j] * MA * T.D2[i][j];
        for (int k = 0; k < 3; ++k) quad += y[j] * y[k] * MA * T.D3[i][j][k];
      }
      /* g = -[ (-M_A D_i - 1/2 Q_A D_ijk) + y_j M_A D_ij - 1/2 y_j y_k M_A D_ijk ] */
      double g = -(b0[i] + lin - 0.5 * quad);
      acc[i][n] += g - F[i] / MB;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* a7': one accepted pair at general order P (App. A)                        */
/* ------------------------------------------------------------------------ */

/* Derivatives of order 0..P+1 at r, by symmetric component. */
static double *dtab_generic(const double r[3], double eps2, int P) {
  double *tab = (double *)xmalloc(sizeof(double) * mi_count(P + 1));
  for (int n = 0; n <= P + 1; ++n) dtensor_generic_e2(r, eps2, n, tab + mi_offset(n));
  return tab;
}

/* D_{L k Q} for full index tuples L (length m) and Q (length n), k one index */
static double dfull(const double *tab, int m, int tl, int k, int n, int tq) {
  int cnt[3] = {0, 0, 0};
  for (int s = 0; s < m; ++s) {
    cnt[tl % 3]++;
    tl /= 3;
  }
  if (k >= 0) cnt[k]++;
  for (int s = 0; s < n; ++s) {
    cnt[tq % 3]++;
    tq /= 3;
  }
  return tab[mi_index(cnt[0], cnt[1], cnt[2])];
}

static double mom_full(const struct orc *t, int c, int n, int tup) {
  if (n == 0) return t->M[c];
  return t->mom[(size_t)c * t->nmom + mi_of_tuple(n, tup)];
}

static void tuple_product(const double x[3], int m, int tup, double *v) {
  double p = 1.0;
  for (int s = 0; s < m; ++s) {
    p *= x[tup % 3];
    tup /= 3;
  }
  *v = p;
}

static void m2l_generic_pair(const struct orc *t, int A, int B, int variant, double *acc[3],
                             const unsigned char *want) {
  const int P = t->P;
  double r[3] = {t->Z[0][A] - t->Z[0][B], t->Z[1][A] - t->Z[1][B], t->Z[2][A] - t->Z[2][B]};
  double r2 = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
  if (r2 == 0.0) return;
  double *tab = dtab_generic(r, t->eps2, P);
  const int nm = P; /* local orders m = 0..P-1 */
  /* Local coefficients: the acceleration on a body of A at x is
   *   g_k = - sum_{m} 1/m! x_{l1..lm} LA[m][k][L],
   *   LA[m][k][L] = sum_{n <= P-1-m} (-1)^n / n! D_{L k Q} M_B,Q
   * and on a body of B at y
   *   g_k = + sum_{n} 1/n! y_{q1..qn} LB[n][k][Q],
   *   LB[n][k][Q] = sum_{m <= P-1-n} (-1)^n / m! M_A,L D_{L k Q}. */
  double **LA = (double **)xmalloc(sizeof(double *) * nm);
  double **LB = (double **)xmalloc(sizeof(double *) * nm);
  for (int m = 0; m < nm; ++m) {
    int tm = ipow3(m);
    LA[m] = (double *)xcalloc((size_t)3 * tm, sizeof(double));
    LB[m] = (double *)xcalloc((size_t)3 * tm, sizeof(double));
  }
  for (int m = 0; m < nm; ++m)
    for (int n = 0; m + n <= P - 1; ++n) {
      const double sgn = (n % 2 == 0) ? 1.0 : -1.0;
      const int tm = ipow3(m), tn = ipow3(n);
      for (int k = 0; k < 3; ++k)
        for (int tl = 0; tl < tm; ++tl)
          for (int tq = 0; tq < tn; ++tq) {
            double D = dfull(tab, m, tl, k, n, tq);
            /* field of B at A: expansion order m in x, moment order n of B */
            LA[m][k * tm + tl] += sgn / factorial(n) * D * mom_full(t, B, n, tq);
            /* field of A at B: moment order m of A, expansion order n in y */
            LB[n][k * tn + tq] += sgn / factorial(m) * mom_full(t, A, m, tl) * D;
          }
    }
  /* corrective force (App. A): F_c,k = - sum_n (-1)^n / (n! (P-n)!)
   *   M_A,L(P-n) M_B,Q(n) D_{L Q k}; TCO removes its component along r. */
  double F[3] = {0.0, 0.0, 0.0};
  if (variant != ORC_UC) {
    for (int n = 0; n <= P; ++n) {
      const double coef = -((n % 2 == 0) ? 1.0 : -1.0) / (factorial(n) * factorial(P - n));
      const int tl_n = ipow3(P - n), tq_n = ipow3(n);
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int tl = 0; tl < tl_n; ++tl) {
          double ma = mom_full(t, A, P - n, tl);
          if (ma == 0.0) continue;
          for (int tq = 0; tq < tq_n; ++tq)
            s += ma * mom_full(t, B, n, tq) * dfull(tab, P - n, tl, k, n, tq);
        }
        F[k] += coef * s;
      }
    }
    if (variant == ORC_TCO) {
      /* D'_{k L} = D_{k L} - r_k r_j / r^2 D_{j L}: F'_c = F_c - r (r.F_c) / r^2 */
      double rf = (r[0] * F[0] + r[1] * F[1]) + r[2] * F[2];
      for (int k = 0; k < 3; ++k) F[k] -= r[k] * rf / r2;
    }
  }
  for (int nb = t->begin[A]; nb < t->begin[A] + t->count[A]; ++nb) {
    if (want && !want[nb]) continue;
    double x[3] = {t->X[0][nb] - t->Z[0][A], t->X[1][nb] - t->Z[1][A], t->X[2][nb] - t->Z[2][A]};
    for (int k = 0; k < 3; ++k) {
      double g = 0.0;
      for (int m = 0; m < nm; ++m) {
        const int tm = ipow3(m);
        double s = 0.0;
        for (int tl = 0; tl < tm; ++tl) {
          double xp;
          tuple_product(x, m, tl, &xp);
          s += xp * LA[m][k * tm + tl];
        }
        g += s / factorial(m);
      }
      acc[k][nb] += -g + F[k] / t->M[A];
    }
  }
  for (int nb = t->begin[B]; nb < t->begin[B] + t->count[B]; ++nb) {
    if (want && !want[nb]) continue;
    double y[3] = {t->X[0][nb] - t->Z[0][B], t->X[1][nb] - t->Z[1][B], t->X[2][nb] - t->Z[2][B]};
    for (int k = 0; k < 3; ++k) {
      double g = 0.0;
      for (int n = 0; n < nm; ++n) {
        const int tn = ipow3(n);
        double s = 0.0;
        for (int tq = 0; tq < tn; ++tq) {
          double yp;
          tuple_product(y, n, tq, &yp);
          s += yp * LB[n][k * tn + tq];
        }
        g += s / factorial(n);
      }
      acc[k][nb] += g - F[k] / t->M[B];
    }
  }
  for (int m = 0; m < nm; ++m) {
    free(LA[m]);
    free(LB[m]);
  }
  free(LA);
  free(LB);
  free(tab);
}

/* ------------------------------------------------------------------------ */
/* a8: near field, every pair of bodies once, force on both                  */
/* ------------------------------------------------------------------------ */

static void p2p_bodies(const struct orc *t, int i, int j, double *acc[3], const unsigned char *want) {
  if (want && !want[i] && !want[j]) return;
  double d[3] = {t->X[0][j] - t->X[0][i], t->X[1][j] - t->X[1][i], t->X[2][j] - t->X[2][i]};
  double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
  if (d2 == 0.0) return;
  double r2 = d2 + t->eps2; /* Plummer softening: G = -1/sqrt(R^2 + eps^2) */
  double inv3 = 1.0 / (r2 * sqrt(r2));
  for (int k = 0; k < 3; ++k) {
    acc[k][i] += t->mu[j] * d[k] * inv3;
    acc[k][j] -= t->mu[i] * d[k] * inv3;
  }
}

/* ------------------------------------------------------------------------ */
/* public entry points                                                       */
/* ------------------------------------------------------------------------ */

orc_t *orc_create(int n, const double *x, const double *y, const double *z, const double *m,
                  int n_crit, double theta, int P, int *err) {
  *err = ORC_OK;
  if (n < 1 || n_crit < 1 || !(theta > 0.0 && theta <= 1.0) || P < 1 || P > 8) {
    *err = ORC_EINVAL;
    return NULL;
  }
  for (int i = 0; i < n; ++i)
    if (!(m[i] > 0.0) || !isfinite(m[i])) {
      *err = ORC_EINVAL;
      return NULL;
    }
  struct orc *t = (struct orc *)xcalloc(1, sizeof(struct orc));
  t->n = n;
  t->n_crit = n_crit;
  t->theta = theta;
  t->P = P;
  uint64_t *k0 = (uint64_t *)xmalloc(sizeof(uint64_t) * n);
  int rc = orc_morton(n, x, y, z, k0, t->lo, &t->scale);
  if (rc != ORC_OK) {
    free(k0);
    free(t);
    *err = rc;
    return NULL;
  }
  keyidx *ki = (keyidx *)xmalloc(sizeof(keyidx) * n);
  for (int i = 0; i < n; ++i) {
    ki[i].key = k0[i];
    ki[i].idx = i;
  }
  qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
  t->key = (uint64_t *)xmalloc(sizeof(uint64_t) * n);
  t->order = (int *)xmalloc(sizeof(int) * n);
  for (int d = 0; d < 3; ++d) t->X[d] = (double *)xmalloc(sizeof(double) * n);
  t->mu = (double *)xmalloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) {
    int o = ki[i].idx;
    t->key[i] = ki[i].key;
    t->order[i] = o;
    t->X[0][i] = x[o];
    t->X[1][i] = y[o];
    t->X[2][i] = z[o];
    t->mu[i] = m[o];
  }
  free(ki);
  free(k0);
  build_tree(t);
  upward(t);
  walk(t, 0, 0);
  return t;
}

void orc_destroy(orc_t *t) {
  if (!t) return;
  free(t->key);
  free(t->order);
  for (int d = 0; d < 3; ++d) {
    free(t->X[d]);
    free(t->S[d]);
    free(t->Z[d]);
  }
  free(t->mu);
  free(t->begin);
  free(t->count);
  free(t->level);
  free(t->parent);
  free(t->first_child);
  free(t->nchild);
  free(t->M);
  free(t->Rmax);
  free(t->mom);
  free(t->m2l);
  free(t->p2p);
  free(t->self);
  free(t);
}

/* Plummer softening for the evaluation: every derivative tensor and every
 * direct pair then uses G(R) = -1/sqrt(R^2 + eps^2) (the paper's Sec. 4
 * remarks that the correction holds for any G that depends only on the
 * distance).  The tree and the walk do not change.  eps = 0: unsoftened. */
int orc_set_softening(orc_t *t, double eps) {
  if (!(eps >= 0.0) || !isfinite(eps)) return ORC_EINVAL;
  t->eps2 = eps * eps;
  return ORC_OK;
}

int orc_sizes(const orc_t *t, int *out) {
  out[0] = t->n;
  out[1] = t->ncell;
  out[2] = t->n_m2l;
  out[3] = t->n_p2p;
  out[4] = t->n_self;
  out[5] = t->nmom;
  return ORC_OK;
}

int orc_get_keys(const orc_t *t, uint64_t *key, int *order, double *lo, double *scale) {
  memcpy(key, t->key, sizeof(uint64_t) * t->n);
  memcpy(order, t->order, sizeof(int) * t->n);
  memcpy(lo, t->lo, sizeof t->lo);
  *scale = t->scale;
  return ORC_OK;
}

int orc_get_cells(const orc_t *t, int *begin, int *count, int *level, int *parent,
                  int *first_child, int *nchild) {
  size_t b = sizeof(int) * (size_t)t->ncell;
  memcpy(begin, t->begin, b);
  memcpy(count, t->count, b);
  memcpy(level, t->level, b);
  memcpy(parent, t->parent, b);
  memcpy(first_child, t->first_child, b);
  memcpy(nchild, t->nchild, b);
  return ORC_OK;
}

int orc_get_geometry(const orc_t *t, double *M, double *Z, double *Rmax, double *mom) {
  for (int c = 0; c < t->ncell; ++c) {
    M[c] = t->M[c];
    Rmax[c] = t->Rmax[c];
    for (int d = 0; d < 3; ++d) Z[3 * c + d] = t->Z[d][c];
  }
  memcpy(mom, t->mom, sizeof(double) * (size_t)t->ncell * t->nmom);
  return ORC_OK;
}

int orc_get_lists(const orc_t *t, int *m2l, int *p2p, int *self) {
  memcpy(m2l, t->m2l, sizeof(int) * 2 * (size_t)t->n_m2l);
  memcpy(p2p, t->p2p, sizeof(int) * 2 * (size_t)t->n_p2p);
  memcpy(self, t->self, sizeof(int) * (size_t)t->n_self);
  return ORC_OK;
}

/* Replaces the interaction lists with caller-given ones (pairs as (A, B),
 * stored as (min, max)).  Used to evaluate the forces of a pair selection
 * other than the plain criterion's (the learned selector of the GPU path is
 * judged this way).  Every index must name a cell; P2P pairs and self
 * entries must name leaves. */
int orc_set_lists(orc_t *t, const int *m2l, int n_m2l, const int *p2p, int n_p2p, const int *self,
                  int n_self) {
  if (n_m2l < 0 || n_p2p < 0 || n_self < 0) return ORC_EINVAL;
  for (int k = 0; k < 2 * n_m2l; ++k)
    if (m2l[k] < 0 || m2l[k] >= t->ncell) return ORC_EINVAL;
  for (int k = 0; k < 2 * n_p2p; ++k)
    if (p2p[k] < 0 || p2p[k] >= t->ncell || !is_leaf(t, p2p[k])) return ORC_EINVAL;
  for (int k = 0; k < n_self; ++k)
    if (self[k] < 0 || self[k] >= t->ncell || !is_leaf(t, self[k])) return ORC_EINVAL;
  t->n_m2l = t->n_p2p = t->n_self = 0;
  for (int k = 0; k < n_m2l; ++k) push_pair(&t->m2l, &t->n_m2l, &t->cap_m2l, m2l[2 * k], m2l[2 * k + 1]);
  for (int k = 0; k < n_p2p; ++k) push_pair(&t->p2p, &t->n_p2p, &t->cap_p2p, p2p[2 * k], p2p[2 * k + 1]);
  int *ns = (int *)realloc(t->self, sizeof(int) * (size_t)(n_self > 0 ? n_self : 1));
  if (!ns) abort();
  t->self = ns;
  t->cap_self = n_self > 0 ? n_self : 1;
  memcpy(t->self, self, sizeof(int) * (size_t)n_self);
  t->n_self = n_self;
  return ORC_OK;
}

static void unpermute(const orc_t *t, double *acc[3], double *ax, double *ay, double *az) {
  for (int i = 0; i < t->n; ++i) {
    ax[t->order[i]] = acc[0][i];
    ay[t->order[i]] = acc[1][i];
    az[t->order[i]] = acc[2][i];
  }
}

int orc_eval(const orc_t *t, int variant, int generic, int parts, const unsigned char *mask,
             double *ax, double *ay, double *az) {
  if (variant < ORC_UC || variant > ORC_TCO) return ORC_EINVAL;
  if (!generic && t->P != 3) return ORC_EINVAL;
  double *acc[3];
  for (int d = 0; d < 3; ++d) acc[d] = (double *)xcalloc((size_t)t->n, sizeof(double));
  /* optional target mask (caller order): only flagged bodies are evaluated,
   * and pairs of cells without a flagged body are skipped */
  unsigned char *want = NULL, *cellwant = NULL;
  if (mask) {
    want = (unsigned char *)xcalloc((size_t)t->n, 1);
    for (int i = 0; i < t->n; ++i) want[i] = mask[t->order[i]] != 0;
    cellwant = (unsigned char *)xcalloc((size_t)t->ncell, 1);
    for (int c = 0; c < t->ncell; ++c)
      for (int i = t->begin[c]; i < t->begin[c] + t->count[c]; ++i)
        if (want[i]) {
          cellwant[c] = 1;
          break;
        }
  }
  if (parts & ORC_PART_FAR) {
    for (int k = 0; k < t->n_m2l; ++k) {
      const int A = t->m2l[2 * k], B = t->m2l[2 * k + 1];
      if (cellwant && !cellwant[A] && !cellwant[B]) continue;
      if (generic) m2l_generic_pair(t, A, B, variant, acc, want);
      else m2l_p3_pair(t, A, B, variant, acc, want);
    }
  }
  if (parts & ORC_PART_NEAR) {
    for (int k = 0; k < t->n_p2p; ++k) {
      const int A = t->p2p[2 * k], B = t->p2p[2 * k + 1];
      if (cellwant && !cellwant[A] && !cellwant[B]) continue;
      for (int i = t->begin[A]; i < t->begin[A] + t->count[A]; ++i)
        for (int j = t->begin[B]; j < t->begin[B] + t->count[B]; ++j) p2p_bodies(t, i, j, acc, want);
    }
    for (int k = 0; k < t->n_self; ++k) {
      const int A = t->self[k];
      if (cellwant && !cellwant[A]) continue;
      for (int i = t->begin[A]; i < t->begin[A] + t->count[A]; ++i)
        for (int j = i + 1; j < t->begin[A] + t->count[A]; ++j) p2p_bodies(t, i, j, acc, want);
    }
  }
  unpermute(t, acc, ax, ay, az);
  for (int d = 0; d < 3; ++d) free(acc[d]);
  free(want);
  free(cellwant);
  return ORC_OK;
}

int orc_pair_accel(const orc_t *t, int A, int B, int variant, int generic, double *ax, double *ay,
                   double *az) {
  if (A < 0 || B < 0 || A >= t->ncell || B >= t->ncell || A == B) return ORC_EINVAL;
  if (!generic && t->P != 3) return ORC_EINVAL;
  double *acc[3];
  for (int d = 0; d < 3; ++d) acc[d] = (double *)xcalloc((size_t)t->n, sizeof(double));
  if (generic) m2l_generic_pair(t, A, B, variant, acc, NULL);
  else m2l_p3_pair(t, A, B, variant, acc, NULL);
  unpermute(t, acc, ax, ay, az);
  for (int d = 0; d < 3; ++d) free(acc[d]);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* exact direct summation (Sec. 3: the reference of the error metric)       */
/* ------------------------------------------------------------------------ */

/* Neumaier's compensated summation */
static void neumaier_add(double *sum, double *comp, double v) {
  double t = *sum + v;
  if (fabs(*sum) >= fabs(v)) *comp += (*sum - t) + v;
  else *comp += (v - t) + *sum;
  *sum = t;
}

int orc_direct(int n, const double *x, const double *y, const double *z, const double *m, int nt,
               const int *targets, double eps, double *ax, double *ay, double *az) {
  const double eps2 = eps * eps;
  for (int t = 0; t < nt; ++t) {
    const int i = targets[t];
    if (i < 0 || i >= n) return ORC_EINVAL;
    double s[3] = {0, 0, 0}, c[3] = {0, 0, 0};
    for (int j = 0; j < n; ++j) {
      double d[3] = {x[j] - x[i], y[j] - y[i], z[j] - z[i]};
      double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
      if (d2 == 0.0) continue;
      double r2 = d2 + eps2;
      double inv3 = 1.0 / (r2 * sqrt(r2));
      for (int k = 0; k < 3; ++k) neumaier_add(&s[k], &c[k], m[j] * d[k] * inv3);
    }
    ax[t] = s[0] + c[0];
    ay[t] = s[1] + c[1];
    az[t] = s[2] + c[2];
  }
  return ORC_OK;
}

/* Net balance of Sec. 3:
 *   sqrt( sum_d (sum_n mu_n A_nd)^2 / sum_d (sum_n mu_n |A_nd|)^2 )
 * for A = acceleration (force balance) and A = X x acceleration (torque). */
int orc_balance(int n, const double *x, const double *y, const double *z, const double *m,
                const double *ax, const double *ay, const double *az, double *out) {
  double fs[3] = {0, 0, 0}, fc[3] = {0, 0, 0}, fa[3] = {0, 0, 0};
  double ts[3] = {0, 0, 0}, tc[3] = {0, 0, 0}, ta[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i) {
    double a[3] = {ax[i], ay[i], az[i]};
    double tq[3] = {y[i] * az[i] - z[i] * ay[i], z[i] * ax[i] - x[i] * az[i], x[i] * ay[i] - y[i] * ax[i]};
    for (int d = 0; d < 3; ++d) {
      neumaier_add(&fs[d], &fc[d], m[i] * a[d]);
      fa[d] += m[i] * fabs(a[d]);
      neumaier_add(&ts[d], &tc[d], m[i] * tq[d]);
      ta[d] += m[i] * fabs(tq[d]);
    }
  }
  double fn = 0, fd = 0, tn = 0, td = 0;
  for (int d = 0; d < 3; ++d) {
    double f = fs[d] + fc[d], tt = ts[d] + tc[d];
    fn += f * f;
    fd += fa[d] * fa[d];
    tn += tt * tt;
    td += ta[d] * ta[d];
  }
  out[0] = fd > 0 ? sqrt(fn / fd) : 0.0;
  out[1] = td > 0 ? sqrt(tn / td) : 0.0;
  return ORC_OK;
}
