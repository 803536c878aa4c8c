/*
 * clv_freezeout.c -- plain FP64 CPU oracle of the freeze-out hypersurface
 * finder.  TEST INFRASTRUCTURE ONLY, under the same rules as clv_oracle.c:
 * only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it, and it shares no code with the CUDA library.
 *
 * What it computes.  Sec. 4 integrates the Cooper-Frye formula, Eq.
 * (cooper_frye), over surface elements dSigma_mu of the hypersurface of
 * constant freeze-out temperature T_f or energy density eps_f, and the
 * closing paragraph of the appendix on the reduction says the finder runs on
 * the GPU.  The paper cites its finder without describing it, so this file
 * follows one reading with a plain definition (F1-F6).
 *   F1 Hypercubes.  Between two time slices tau0 < tau1 of the grid, the
 *      hypercube (i, j, k) has its 16 corners at the cell centres
 *      (i + a, j + b, k + c), a, b, c in {0, 1}, of both slices: there are
 *      (nx-1)(ny-1)(neta-1) of them.  Corner q carries the bits
 *      (tau, x, y, eta) = (q & 1, q >> 1 & 1, q >> 2 & 1, q >> 3 & 1).
 *   F2 Interpolant.  eps is continued piecewise linearly over the Freudenthal
 *      (Kuhn) triangulation of each hypercube: one 4-simplex per ordering
 *      (s0, s1, s2, s3) of the four axes, with vertices v0 = corner 0 and
 *      v(m+1) = v(m) + unit step along axis s(m).  The surface is the level
 *      set eps = eps_f of that interpolant (constant T_f maps to constant
 *      eps_f through the monotone equation of state).  A corner is inside
 *      (hot) when eps >= eps_f.
 *   F3 Pieces.  Inside one simplex the level set is planar: a tetrahedron
 *      when one vertex is on its own side, a triangular prism (cut into
 *      three tetrahedra) when two are.  Its points lie on the simplex edges
 *      between an inside vertex a and an outside vertex b, at the fraction
 *      t = f_a / (f_a - f_b) from a (f = eps - eps_f).
 *   F4 Elements.  Geometry is taken in coordinate space (tau, x, y, eta_s)
 *      treated as R^4.  A piece of 3-volume A with normal along the simplex
 *      gradient contributes dSigma_mu = -grad_mu(eps) / |grad eps| times the
 *      integral of tau over the piece (sqrt(-g) = tau in Milne coordinates;
 *      1 in Cartesian mode), which is A times tau at the piece's centroid.
 *      The covariant vector points down the gradient, so p^mu dSigma_mu > 0
 *      for particles leaving the hot region.  A hypercube that has corners
 *      on both sides gives one element: the sum over its pieces.
 *   F5 Position.  The element sits at the 3-volume weighted mean of the
 *      piece centroids (the hypercube centre if all pieces are degenerate).
 *   F6 Fields.  u~^x, u~^y, u~^eta and the ten pi~ components are
 *      interpolated at that position with the same piecewise-linear
 *      interpolant (the simplex that holds the point: local coordinates
 *      sorted in decreasing order, ties by axis order), and
 *      u~^tau = sqrt(1 + u~_x^2 + u~_y^2 + u~_eta^2).
 * Element record (22 values): dSigma_tau, dSigma_x, dSigma_y, dSigma_eta,
 * tau, x, y, eta_s, u~^tau, u~^x, u~^y, u~^eta, pi~ (tt tx ty te xx xy xe yy
 * ye ee).  Elements come in increasing hypercube order (i, then j, then k).
 *
 * Pins (tests/test_oracle_freezeout.py): planar level sets against exact
 * integrals, each simplex against the closed form of the coarea formula with
 * the Curry-Schoenberg B-spline, closed level sets summing to zero, affine
 * fields interpolated exactly, and brute-force counts.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifndef PLANT
#define PLANT 0
#endif

#define FO_NREC 22
#define FO_NF 13 /* interpolated fields per slice: u~ (3), pi~ (10) */

typedef struct {
  int nx, ny, neta;
  double dx, dy, deta;
  double tau0, tau1;
  int cartesian;
} orc_fo_grid;

typedef struct {
  double dS[4];   /* sum of the pieces' dSigma_mu */
  double A;       /* sum of the pieces' 3-volumes */
  double Ac[4];   /* sum of 3-volume x centroid */
} fo_acc;

/* 3-volume of the tetrahedron p0..p3 in R^4: |a ^ b ^ c| / 6 with a, b, c
 * the edges from p0, through the four 3x3 minors (the 4-d cross product). */
static double tet_volume(const double p0[4], const double p1[4], const double p2[4], const double p3[4]) {
  double a[4], b[4], c[4];
  for (int m = 0; m < 4; ++m) {
    a[m] = p1[m] - p0[m];
    b[m] = p2[m] - p0[m];
    c[m] = p3[m] - p0[m];
  }
  double n2 = 0.0;
  for (int skip = 0; skip < 4; ++skip) {
    int ix[3], q = 0;
    for (int m = 0; m < 4; ++m)
      if (m != skip) ix[q++] = m;
    double det = a[ix[0]] * (b[ix[1]] * c[ix[2]] - b[ix[2]] * c[ix[1]])
               - a[ix[1]] * (b[ix[0]] * c[ix[2]] - b[ix[2]] * c[ix[0]])
               + a[ix[2]] * (b[ix[0]] * c[ix[1]] - b[ix[1]] * c[ix[0]]);
    n2 += det * det;
  }
  return sqrt(n2) / 6.0;
}

/* adds one tetrahedron of a piece with unit normal nhat (F4, F5) */
static void add_tet(const orc_fo_grid* g, const double* p0, const double* p1, const double* p2,
                    const double* p3, const double nhat[4], double tau_lo, fo_acc* acc) {
  double A = tet_volume(p0, p1, p2, p3);
  double c[4];
  for (int m = 0; m < 4; ++m) c[m] = 0.25 * (p0[m] + p1[m] + p2[m] + p3[m]);
  double w = g->cartesian ? 1.0 : ((PLANT == 11) ? tau_lo : c[0]);
  for (int m = 0; m < 4; ++m) {
    acc->dS[m] += nhat[m] * A * w;
    acc->Ac[m] += A * c[m];
  }
  acc->A += A;
}

/* the piece of the level set inside the simplex with vertices P[0..4]
 * (physical coordinates) and values f[0..4] = eps - eps_f (F3, F4) */
static void simplex_piece(const orc_fo_grid* g, double P[5][4], const double f[5], const double grad[4],
                          fo_acc* acc) {
  int in[5], out[5], nin = 0, nout = 0;
  for (int v = 0; v < 5; ++v) {
    if (f[v] >= 0.0) in[nin++] = v;
    else out[nout++] = v;
  }
  if (nin == 0 || nout == 0) return;
  double gn = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2] + grad[3] * grad[3]);
  double nhat[4];
  for (int m = 0; m < 4; ++m) nhat[m] = ((PLANT == 9) ? 1.0 : -1.0) * grad[m] / gn;
  /* X[a][b]: the level-set point on the edge between inside vertex in[a]
   * and outside vertex out[b] */
  double X[4][4][4];
  for (int a = 0; a < nin; ++a)
    for (int b = 0; b < nout; ++b) {
      double fa = f[in[a]], fb = f[out[b]];
      double t = fa / (fa - fb);
      for (int m = 0; m < 4; ++m) X[a][b][m] = P[in[a]][m] + t * (P[out[b]][m] - P[in[a]][m]);
    }
  double tau_lo = g->tau0;
  if (nin == 1) {
    add_tet(g, X[0][0], X[0][1], X[0][2], X[0][3], nhat, tau_lo, acc);
  } else if (nout == 1) {
    add_tet(g, X[0][0], X[1][0], X[2][0], X[3][0], nhat, tau_lo, acc);
  } else {
    /* prism: the two vertices on one side give its two triangles; point
     * (r, s) with r over the pair and s over the triple */
    double* Q[2][3];
    for (int r = 0; r < 2; ++r)
      for (int s = 0; s < 3; ++s) Q[r][s] = (nin == 2) ? X[r][s] : X[s][r];
    add_tet(g, Q[0][0], Q[0][1], Q[0][2], Q[1][0], nhat, tau_lo, acc);
    if (PLANT != 10) add_tet(g, Q[0][1], Q[0][2], Q[1][0], Q[1][1], nhat, tau_lo, acc);
    add_tet(g, Q[0][2], Q[1][0], Q[1][1], Q[1][2], nhat, tau_lo, acc);
  }
}

static size_t cell(const orc_fo_grid* g, int i, int j, int k) {
  return ((size_t)i * g->ny + j) * g->neta + k;
}

/* value of slice array pair (a0 at tau0, a1 at tau1) at corner q of hypercube (i, j, k) */
static double corner(const orc_fo_grid* g, const double* a0, const double* a1, int i, int j, int k, int q) {
  const double* a = (q & 1) ? a1 : a0;
  return a[cell(g, i + (q >> 1 & 1), j + (q >> 2 & 1), k + (q >> 3 & 1))];
}

/* The 24 orderings of the axes, in lexicographic order. */
static int orderings(int perm[24][4]) {
  int n = 0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c)
        for (int d = 0; d < 4; ++d)
          if (a != b && a != c && a != d && b != c && b != d && c != d) {
            perm[n][0] = a; perm[n][1] = b; perm[n][2] = c; perm[n][3] = d;
            ++n;
          }
  return n;
}

/* The element of hypercube (i, j, k); returns 0 when the level set misses it. */
static int cube_element(const orc_fo_grid* g, const double* e0, const double* e1, const double* f0,
                        const double* f1, double eps_f, int i, int j, int k, double rec[FO_NREC]) {
  double fq[16];
  int nin = 0;
  for (int q = 0; q < 16; ++q) {
    fq[q] = corner(g, e0, e1, i, j, k, q) - eps_f;
    nin += fq[q] >= 0.0;
  }
  if (nin == 0 || nin == 16) return 0;
  const double h[4] = {g->tau1 - g->tau0, g->dx, g->dy, g->deta};
  const double o[4] = {g->tau0, (i - 0.5 * (g->nx - 1)) * g->dx, (j - 0.5 * (g->ny - 1)) * g->dy,
                       (k - 0.5 * (g->neta - 1)) * g->deta};
  int perm[24][4];
  int np = orderings(perm);
  if (PLANT == 12) np = 23;
  fo_acc acc;
  memset(&acc, 0, sizeof(acc));
  for (int s = 0; s < np; ++s) {
    int v[5];
    v[0] = 0;
    for (int m = 0; m < 4; ++m) v[m + 1] = v[m] | (1 << perm[s][m]);
    double P[5][4], f[5], grad[4];
    for (int m = 0; m < 5; ++m) {
      f[m] = fq[v[m]];
      for (int a = 0; a < 4; ++a) P[m][a] = o[a] + h[a] * (double)(v[m] >> a & 1);
    }
    for (int m = 0; m < 4; ++m) grad[perm[s][m]] = (f[m + 1] - f[m]) / h[perm[s][m]];
    simplex_piece(g, P, f, grad, &acc);
  }
  double pos[4];
  for (int a = 0; a < 4; ++a) pos[a] = acc.A > 0.0 ? acc.Ac[a] / acc.A : o[a] + 0.5 * h[a];
  /* F6: the simplex holding pos and its barycentric weights */
  double sl[4];
  int ord[4];
  for (int a = 0; a < 4; ++a) {
    sl[a] = (pos[a] - o[a]) / h[a];
    if (sl[a] < 0.0) sl[a] = 0.0;
    if (sl[a] > 1.0) sl[a] = 1.0;
    ord[a] = a;
  }
  for (int a = 1; a < 4; ++a) /* insertion sort, decreasing, stable */
    for (int b = a; b > 0 && sl[ord[b]] > sl[ord[b - 1]]; --b) {
      int t = ord[b]; ord[b] = ord[b - 1]; ord[b - 1] = t;
    }
  double w[5];
  int vq[5];
  w[0] = 1.0 - sl[ord[0]];
  for (int m = 1; m < 4; ++m) w[m] = sl[ord[m - 1]] - sl[ord[m]];
  w[4] = sl[ord[3]];
  vq[0] = 0;
  for (int m = 0; m < 4; ++m) vq[m + 1] = vq[m] | (1 << ord[m]);
  double F[FO_NF];
  size_t N = (size_t)g->nx * g->ny * g->neta;
  for (int fi = 0; fi < FO_NF; ++fi) {
    double s = 0.0;
    for (int m = 0; m < 5; ++m) s += w[m] * corner(g, f0 + fi * N, f1 + fi * N, i, j, k, vq[m]);
    F[fi] = s;
  }
  for (int a = 0; a < 4; ++a) rec[a] = acc.dS[a];
  for (int a = 0; a < 4; ++a) rec[4 + a] = pos[a];
  rec[8] = sqrt(1.0 + F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
  for (int m = 0; m < 3; ++m) rec[9 + m] = F[m];
  for (int q = 0; q < 10; ++q) rec[12 + q] = F[3 + q];
  return 1;
}

/* All elements between the slices (e0, f0) at tau0 and (e1, f1) at tau1.
 * e*: N = nx*ny*neta values of eps; f*: 13 x N values (u~^x, u~^y, u~^eta,
 * pi~ tt..ee, each a full grid).  Writes at most `capacity` records (22
 * doubles each) to rec and their hypercube indices ((i*(ny-1) + j)*(neta-1)
 * + k) to cube (nullable); returns the number of elements (which may exceed
 * capacity), or -1 for a bad grid. */
int64_t orc_freezeout(const orc_fo_grid* g, const double* e0, const double* e1, const double* f0,
                      const double* f1, double eps_f, double* rec, int64_t* cube, int64_t capacity) {
  if (g->nx < 2 || g->ny < 2 || g->neta < 2 || !(g->tau1 > g->tau0)) return -1;
  int64_t n = 0;
  for (int i = 0; i < g->nx - 1; ++i)
    for (int j = 0; j < g->ny - 1; ++j)
      for (int k = 0; k < g->neta - 1; ++k) {
        double r[FO_NREC];
        if (!cube_element(g, e0, e1, f0, f1, eps_f, i, j, k, r)) continue;
        if (n < capacity) {
          memcpy(rec + n * FO_NREC, r, sizeof(r));
          if (cube) cube[n] = ((int64_t)i * (g->ny - 1) + j) * (g->neta - 1) + k;
        }
        ++n;
      }
  return n;
}

/* Only the contribution of simplex `s` (lexicographic ordering index) of
 * hypercube (i, j, k) to dSigma_mu; for the per-simplex pin. */
void orc_freezeout_simplex(const orc_fo_grid* g, const double* e0, const double* e1, double eps_f, int i,
                           int j, int k, int s, double dS[4]) {
  int perm[24][4];
  orderings(perm);
  const double h[4] = {g->tau1 - g->tau0, g->dx, g->dy, g->deta};
  const double o[4] = {g->tau0, (i - 0.5 * (g->nx - 1)) * g->dx, (j - 0.5 * (g->ny - 1)) * g->dy,
                       (k - 0.5 * (g->neta - 1)) * g->deta};
  int v[5];
  v[0] = 0;
  for (int m = 0; m < 4; ++m) v[m + 1] = v[m] | (1 << perm[s][m]);
  double P[5][4], f[5], grad[4];
  for (int m = 0; m < 5; ++m) {
    f[m] = corner(g, e0, e1, i, j, k, v[m]) - eps_f;
    for (int a = 0; a < 4; ++a) P[m][a] = o[a] + h[a] * (double)(v[m] >> a & 1);
  }
  for (int m = 0; m < 4; ++m) grad[perm[s][m]] = (f[m + 1] - f[m]) / h[perm[s][m]];
  fo_acc acc;
  memset(&acc, 0, sizeof(acc));
  simplex_piece(g, P, f, grad, &acc);
  for (int a = 0; a < 4; ++a) dS[a] = acc.dS[a];
}
