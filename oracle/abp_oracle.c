/*
 * abp_oracle.c -- plain FP64 CPU oracle for the adaptive-biasing-potential
 * (ABP) force call of Dickson et al., "A fast, open source implementation of
 * adaptive biasing potentials ..." (arXiv:1609.09833).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark call this file. The product path (the CUDA
 * library) never links it, and this file includes no header of that library.
 *
 * What it computes, one walker step at MD step t (all in double precision):
 *   a1  the collective variables s_k(x) and their Jacobians ds_k/dx
 *       (centre-of-mass distance, dihedral, coordination number);
 *   a2  on a deposit step (t % stride == 0) the well-tempered height
 *       h = w exp(-V_b(s_t) / dT), dT = (gamma - 1) kT, read from the grid
 *       BEFORE this step's deposit (one exponential per hill, Section
 *       "Timing of the implementation", WTmetaD paragraph);
 *   a3  the deposit of a Gaussian hill h exp(-|xi - s_t|^2 / 2 sigma^2) and
 *       of its derivative along every CV onto the grid points inside a cutoff
 *       box (the value/derivative pair of Eq. (histos) updated as in
 *       Eq. (update), restricted to a neighbourhood of the trajectory as in
 *       Eq. (Cupdate), and scaled by the hill height for WTmetaD);
 *   a4  V_b(s_t) and dV_b/ds_k(s_t) by multilinear interpolation of the
 *       value field and of each derivative field (the "look-up in the
 *       histograms" after Eq. (ghill));
 *   a5  the bias force on every CV atom, F = - sum_k dV_b/ds_k ds_k/dx
 *       (returned to the owner of the atoms, SI "Minimization of
 *       Interprocess Communications").
 *
 * Conventions taken where the paper is silent (the CUDA library follows
 * the same ones, written independently; each is the plain reading of the
 * method where the text leaves a choice open):
 *   - grid nodes: non-periodic axis xi_i = lo + i*D, D = (hi-lo)/(n-1),
 *     i = 0..n-1; periodic axis D = (hi-lo)/n with wrap-around;
 *   - hill centre index i_c = floor(u + 1/2), u = (s - lo)/D (wrapped into
 *     [0, n) on a periodic axis); stencil = integer box i_c-R..i_c+R with
 *     R = ceil(cutoff * sigma / D); nodes outside a non-periodic axis are
 *     dropped; on a periodic axis the node-to-centre distance is the minimum
 *     image in [-L/2, L/2);
 *   - the hill is exp(-|d|^2 / (2 sigma^2)) (the paper's Eq. (ghill) has
 *     alpha^2 = 2 sigma^2);
 *   - the derivative fields hold dV/dxi_k (derivative with respect to the
 *     grid coordinate);
 *   - interpolation: u clamped to [0, n-1] on a non-periodic axis, where a
 *     clamped axis also gets a zero gradient; the lower corner is
 *     min(floor(u), n-2);
 *   - deposit on every step with step % stride == 0 (step 0 included); V and
 *     grad V used for the force are read after this step's deposit; walkers
 *     that share one grid all read their heights before any deposit of the
 *     step and their forces after all of them (Jacobi order), deposits being
 *     applied in walker order.
 *
 * The mABP method with compact hills (SI "Streamlined bias potential
 * updates") is the second method a walker may use (or_hill.method):
 *   a3' at the nearest grid node xi* to s_t, the histograms h and h'_i get
 *       the product hill S_a^p(xi* - xi) of Eq. (compacthill) and its
 *       derivative along xi_i (Eq. (Cupdate)), on every node within a of
 *       xi* per axis, scaled by w (w = 1 and stride 1 is the paper's update
 *       at every timestep);
 *   a4' V_b and dV_b/dxi_i from h and h' at xi* by Eq. (apfm) and
 *       Eq. (btraj-grad) (a look-up, no interpolation), with beta^-1 = kT;
 * with the conventions: xi* = the node floor(u + 1/2), limited to the grid on
 * a non-periodic axis (where the gradient along a limited axis is zero); the
 * stencil half-width is floor(a / D) nodes; the derivative field h'_i holds
 * dh/dxi_i.
 * The RMSD CV (SI "Definition of the RMSD") is offset by 0.01 so that it is
 * never zero: s = (sum_i |x_i - x0_i|^2 / N + 0.01)^(1/2), no fit.
 *
 * The CV range limit (the restraint "which limits the maximum value of the
 * CVs", Applications section; the paper gives no form) is read as a
 * flat-bottomed harmonic wall per CV, U = kwall/2 (s_k - smax_k)^2 for
 * s_k > smax_k: its gradient is added to dV_b/ds_k before the chain rule
 * (dV reports the sum), kwall = 0 turns it off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXCV 3

enum { OR_CV_COM_DIST = 0, OR_CV_DIHEDRAL = 1, OR_CV_COORD = 2, OR_CV_POS_X = 3, OR_CV_RMSD = 4 };
enum { OR_METHOD_WT_GAUSS = 0, OR_METHOD_MABP_COMPACT = 1 };

enum {
  OR_FLAG_DEPOSIT = 1,   /* a hill was deposited on this step */
  OR_FLAG_OOR = 2,       /* a CV lay outside a non-periodic grid range */
  OR_FLAG_SINGULAR = 4,  /* a CV Jacobian was undefined (zero length) */
  OR_FLAG_BADARG = 8
};

/* One collective variable over the walker's own atom block. */
typedef struct {
  int type;             /* OR_CV_* */
  int na, nb;           /* COM: groups A, B; DIHEDRAL: na = 4; COORD: ligand A x pocket B */
  const int *ia, *ib;   /* atom indices into the walker's block */
  const double *ma, *mb;/* masses for COM (NULL = unit masses) */
  double r0;            /* COORD switching radius */
  int nn, mm;           /* COORD exponents of (1 - (r/r0)^n) / (1 - (r/r0)^m) */
  int pbc;              /* minimum image on difference vectors */
  double box[3];        /* orthorhombic box edge lengths */
  const double *ref;    /* RMSD: reference positions x0 of the atoms ia (na x 3) */
} or_cv;

typedef struct {
  int d;                /* number of CVs = grid dimension, 1..3 */
  int n[3];
  int periodic[3];
  double lo[3], hi[3];
} or_grid;

typedef struct {
  double w;             /* initial hill height */
  double sigma[3];      /* Gaussian width per CV */
  double cutoff;        /* half-width of the stencil box, in units of sigma */
  double gamma;         /* bias factor */
  double kT;            /* thermal energy */
  int64_t stride;       /* deposit every `stride` MD steps */
  int method;           /* OR_METHOD_*; the fields below are mABP's */
  double a[3];          /* compact hill half-width per CV */
  int p;                /* compact hill shape exponent, >= 1 */
  double b, c;          /* mABP parameters of Eq. (apfm) */
  double smax[3];       /* CV range limit: wall above smax_k ... */
  double kwall;         /* ... with force constant kwall (0: no wall) */
} or_hill;

typedef struct {
  or_grid g;
  or_hill hill;
  or_cv cv[OR_MAXCV];
  int natoms;
} or_walker;

/* The model dynamics of a closed-loop run (see or_md_move). */
enum { OR_POT_NONE = 0, OR_POT_DOUBLE_WELL = 1, OR_POT_MULLER_BROWN = 2 };
typedef struct {
  double dt;            /* time step (ps) */
  double mu;            /* mobility (nm^2 / (kJ/mol ps)) */
  double kT;            /* thermal energy of the noise (kJ/mol) */
  uint64_t seed;        /* Philox key */
  int pot;              /* OR_POT_* */
  double dw_a, dw_b;    /* double well A (s_0^2 - B^2)^2 */
  double mb_scale;      /* Mueller-Brown: energy scale */
  double mb_map[4];     /* X = map[0] s_0 + map[1], Y = map[2] s_1 + map[3] */
  double mb_A[4], mb_a[4], mb_b[4], mb_c[4], mb_x0[4], mb_y0[4];
  int state_f32;        /* nonzero: positions are stored in binary32 after every
                           move (an engine that keeps FP32 coordinates) */
} or_md;

/* Per-walker error-analysis outputs of one step (or_batch_step): the slopes
 * and absolute scale of the interpolation (or_interp_aux; a CV range wall
 * adds kwall to H[4k] above smax) and each CV's rounding bound in units of
 * the unit roundoff (or_cv_round_bound). */
typedef struct {
  double H[9];
  double A[4];
  double sb[3];
} or_stepaux;

/* What the step deposited (one record per hill). */
typedef struct {
  int64_t step;
  int32_t walker;
  int32_t ic[3];
  double s[3];
  double height;
} or_deposit;

/* ------------------------------------------------------------------ */
/* grid geometry                                                        */
/* ------------------------------------------------------------------ */

static double grid_spacing(const or_grid *g, int k) {
  return g->periodic[k] ? (g->hi[k] - g->lo[k]) / g->n[k]
                        : (g->hi[k] - g->lo[k]) / (g->n[k] - 1);
}

long or_grid_nodes(const or_grid *g) {
  long n = 1;
  for (int k = 0; k < g->d; ++k) n *= g->n[k];
  return n;
}

int or_stencil_halfwidth(const or_grid *g, const or_hill *hl, int k) {
  if (hl->method == OR_METHOD_MABP_COMPACT) return (int)floor(hl->a[k] / grid_spacing(g, k));
  return (int)ceil(hl->cutoff * hl->sigma[k] / grid_spacing(g, k));
}

/* Returns 0 if the grid and hill are usable, nonzero otherwise. */
int or_check(const or_grid *g, const or_hill *hl) {
  if (g->d < 1 || g->d > OR_MAXCV) return 1;
  const int mabp = hl->method == OR_METHOD_MABP_COMPACT;
  if (hl->method != OR_METHOD_WT_GAUSS && !mabp) return 6;
  if (mabp && (hl->p < 1 || !(hl->b > 0 && hl->b < 1) || !(hl->c > 0))) return 7;
  for (int k = 0; k < g->d; ++k) {
    if (g->n[k] < 2 || !(g->hi[k] > g->lo[k])) return 2;
    if (mabp ? !(hl->a[k] > 0) : !(hl->sigma[k] > 0)) return 3;
    /* a periodic stencil must not wrap onto itself */
    if (g->periodic[k] && 2 * or_stencil_halfwidth(g, hl, k) + 1 > g->n[k]) return 4;
  }
  if ((!mabp && !(hl->gamma > 1)) || !(hl->kT > 0) || hl->stride < 1) return 5;
  return 0;
}

/* wrap a fractional grid coordinate into [0, n) */
static double wrap_u(double u, int n) {
  u = fmod(u, (double)n);
  if (u < 0) u += n;
  if (u >= n) u -= n;
  return u;
}

/* ------------------------------------------------------------------ */
/* a1: collective variables and Jacobians                               */
/* ------------------------------------------------------------------ */

static void min_image(double *v, const or_cv *c) {
  if (!c->pbc) return;
  for (int k = 0; k < 3; ++k) v[k] -= c->box[k] * floor(v[k] / c->box[k] + 0.5);
}

/* s = |R_B - R_A|, R_G the mass-weighted mean of group G. */
static int cv_com_dist(const or_cv *c, const double *x, double *s, double *J) {
  double ra[3] = {0, 0, 0}, rb[3] = {0, 0, 0}, Ma = 0, Mb = 0;
  for (int i = 0; i < c->na; ++i) {
    double m = c->ma ? c->ma[i] : 1.0;
    for (int k = 0; k < 3; ++k) ra[k] += m * x[3 * c->ia[i] + k];
    Ma += m;
  }
  for (int i = 0; i < c->nb; ++i) {
    double m = c->mb ? c->mb[i] : 1.0;
    for (int k = 0; k < 3; ++k) rb[k] += m * x[3 * c->ib[i] + k];
    Mb += m;
  }
  double dv[3];
  for (int k = 0; k < 3; ++k) dv[k] = rb[k] / Mb - ra[k] / Ma;
  min_image(dv, c);
  double r = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  *s = r;
  if (r == 0.0) return OR_FLAG_SINGULAR;
  for (int i = 0; i < c->na; ++i) {
    double m = c->ma ? c->ma[i] : 1.0;
    for (int k = 0; k < 3; ++k) J[3 * c->ia[i] + k] -= (m / Ma) * dv[k] / r;
  }
  for (int i = 0; i < c->nb; ++i) {
    double m = c->mb ? c->mb[i] : 1.0;
    for (int k = 0; k < 3; ++k) J[3 * c->ib[i] + k] += (m / Mb) * dv[k] / r;
  }
  return 0;
}

static void cross(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Dihedral of atoms 1-2-3-4 (IUPAC sign), phi in [-pi, pi]:
 *   b1 = x2-x1, b2 = x3-x2, b3 = x4-x3, m = b1 x b2, n = b2 x b3,
 *   phi = atan2(|b2| b1.n, m.n),
 * gradient in the form of Blondel & Karplus, J. Comput. Chem. 17 (1996). */
static int cv_dihedral(const or_cv *c, const double *x, double *s, double *J) {
  const double *x1 = x + 3 * c->ia[0], *x2 = x + 3 * c->ia[1];
  const double *x3 = x + 3 * c->ia[2], *x4 = x + 3 * c->ia[3];
  double b1[3], b2[3], b3[3], m[3], n[3];
  for (int k = 0; k < 3; ++k) {
    b1[k] = x2[k] - x1[k];
    b2[k] = x3[k] - x2[k];
    b3[k] = x4[k] - x3[k];
  }
  min_image(b1, c);
  min_image(b2, c);
  min_image(b3, c);
  cross(b1, b2, m);
  cross(b2, b3, n);
  double lb2 = sqrt(dot(b2, b2));
  *s = atan2(lb2 * dot(b1, n), dot(m, n));
  double mm = dot(m, m), nn = dot(n, n);
  if (mm == 0.0 || nn == 0.0 || lb2 == 0.0) return OR_FLAG_SINGULAR;
  double g1[3], g4[3], g2[3], g3[3];
  double p = dot(b1, b2) / (lb2 * lb2), q = dot(b3, b2) / (lb2 * lb2);
  for (int k = 0; k < 3; ++k) {
    g1[k] = -lb2 / mm * m[k];
    g4[k] = lb2 / nn * n[k];
    /* dphi/dx2 = -(1 + p) dphi/dx1 + q dphi/dx4 ; dphi/dx3 = -(1 + q) dphi/dx4 + p dphi/dx1 */
    g2[k] = -(1.0 + p) * g1[k] + q * g4[k];
    g3[k] = -(1.0 + q) * g4[k] + p * g1[k];
  }
  for (int k = 0; k < 3; ++k) {
    J[3 * c->ia[0] + k] += g1[k];
    J[3 * c->ia[1] + k] += g2[k];
    J[3 * c->ia[2] + k] += g3[k];
    J[3 * c->ia[3] + k] += g4[k];
  }
  return 0;
}

/* Rational switching function sw(x) = (1 - x^n) / (1 - x^m), x = r / r0,
 * and its derivative dsw/dx. For m = 2n it equals 1 / (1 + x^n) exactly
 * (difference of squares), which also covers the removable point x = 1;
 * otherwise x = 1 takes the limit n/m. */
double or_switch(double x, int n, int m, double *dsdx) {
  if (m == 2 * n) {
    double xn = pow(x, n);
    double sw = 1.0 / (1.0 + xn);
    *dsdx = -n * pow(x, n - 1) * sw * sw;
    return sw;
  }
  if (x == 1.0) {
    *dsdx = 0.5 * n * (n - m) / (double)m;
    return (double)n / m;
  }
  double xn = pow(x, n), xm = pow(x, m);
  double num = 1.0 - xn, den = 1.0 - xm;
  *dsdx = (-n * pow(x, n - 1) * den + m * pow(x, m - 1) * num) / (den * den);
  return num / den;
}

/* s = sum_{i in A} sum_{j in B} sw(|x_i - x_j| / r0), all pairs, no cutoff. */
static int cv_coord(const or_cv *c, const double *x, double *s, double *J) {
  double acc = 0.0;
  int flag = 0;
  for (int a = 0; a < c->na; ++a) {
    const double *xi = x + 3 * c->ia[a];
    for (int b = 0; b < c->nb; ++b) {
      const double *xj = x + 3 * c->ib[b];
      double v[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
      min_image(v, c);
      double r = sqrt(dot(v, v));
      double dsdx;
      acc += or_switch(r / c->r0, c->nn, c->mm, &dsdx);
      if (r == 0.0) {
        flag = OR_FLAG_SINGULAR;
        continue;
      }
      for (int k = 0; k < 3; ++k) {
        double gk = dsdx / c->r0 * v[k] / r;
        J[3 * c->ia[a] + k] += gk;
        J[3 * c->ib[b] + k] -= gk;
      }
    }
  }
  *s = acc;
  return flag;
}

/* s = x coordinate of one atom (a test CV whose free energy equals the
 * potential acting on it). */
static int cv_pos_x(const or_cv *c, const double *x, double *s, double *J) {
  *s = x[3 * c->ia[0]];
  J[3 * c->ia[0]] += 1.0;
  return 0;
}

/* s = (sum_i |x_i - x0_i|^2 / N + 0.01)^(1/2) over the N atoms ia, no fit
 * (SI "Definition of the RMSD"); ds/dx_i = (x_i - x0_i) / (N s). */
static int cv_rmsd(const or_cv *c, const double *x, double *s, double *J) {
  double acc = 0.0;
  for (int i = 0; i < c->na; ++i)
    for (int k = 0; k < 3; ++k) {
      double dx = x[3 * c->ia[i] + k] - c->ref[3 * i + k];
      acc += dx * dx;
    }
  double r = sqrt(acc / c->na + 0.01);
  *s = r;
  for (int i = 0; i < c->na; ++i)
    for (int k = 0; k < 3; ++k) J[3 * c->ia[i] + k] += (x[3 * c->ia[i] + k] - c->ref[3 * i + k]) / (c->na * r);
  return 0;
}

/* Evaluate one CV; J (natoms x 3) is overwritten with ds/dx. */
int or_cv_eval(const or_cv *c, int natoms, const double *x, double *s, double *J) {
  memset(J, 0, sizeof(double) * 3 * (size_t)natoms);
  switch (c->type) {
    case OR_CV_COM_DIST: return cv_com_dist(c, x, s, J);
    case OR_CV_DIHEDRAL: return cv_dihedral(c, x, s, J);
    case OR_CV_COORD: return cv_coord(c, x, s, J);
    case OR_CV_POS_X: return cv_pos_x(c, x, s, J);
    case OR_CV_RMSD: return cv_rmsd(c, x, s, J);
  }
  *s = 0;
  return OR_FLAG_BADARG;
}

/* ------------------------------------------------------------------ */
/* a4: multilinear interpolation of V and of each dV/dxi_k              */
/* ------------------------------------------------------------------ */

/* field: [nodes][1+d], node = i0 + n0*(i1 + n1*i2). Writes V and dV[0..d-1].
 * Returns OR_FLAG_OOR if s left a non-periodic range. */
int or_interp(const or_grid *g, const double *field, const double *s, double *V, double *dV) {
  int d = g->d, nf = 1 + d, flag = 0;
  int i0[3] = {0, 0, 0}, i1[3] = {0, 0, 0}, clamped[3] = {0, 0, 0};
  double f[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) {
    double D = grid_spacing(g, k);
    double u = (s[k] - g->lo[k]) / D;
    if (g->periodic[k]) {
      u = wrap_u(u, g->n[k]);
      int a = (int)floor(u);
      if (a > g->n[k] - 1) a = g->n[k] - 1;
      i0[k] = a;
      i1[k] = (a + 1) % g->n[k];
      f[k] = u - a;
    } else {
      if (u < 0.0) { u = 0.0; clamped[k] = 1; flag = OR_FLAG_OOR; }
      if (u > g->n[k] - 1) { u = g->n[k] - 1; clamped[k] = 1; flag = OR_FLAG_OOR; }
      int a = (int)floor(u);
      if (a > g->n[k] - 2) a = g->n[k] - 2;
      i0[k] = a;
      i1[k] = a + 1;
      f[k] = u - a;
    }
  }
  double acc[1 + OR_MAXCV] = {0, 0, 0, 0};
  for (int corner = 0; corner < (1 << d); ++corner) {
    double wgt = 1.0;
    long node = 0, mul = 1;
    for (int k = 0; k < d; ++k) {
      int hi = (corner >> k) & 1;
      wgt *= hi ? f[k] : 1.0 - f[k];
      node += mul * (hi ? i1[k] : i0[k]);
      mul *= g->n[k];
    }
    for (int q = 0; q < nf; ++q) acc[q] += wgt * field[node * nf + q];
  }
  *V = acc[0];
  for (int k = 0; k < d; ++k) dV[k] = clamped[k] ? 0.0 : acc[1 + k];
  return flag;
}

/* Error-analysis companions of or_interp (test infrastructure: they scale
 * the tolerance of a per-step comparison, they are not part of the method).
 * At s, with the corners, weights and clamping of or_interp:
 *   H[3*k + j] = d(dV_k)/ds_j, the slope of the interpolated derivative field
 *                k along axis j (0 on a clamped axis j or for a clamped k);
 *   A[q]       = sum over corners of weight * the gross value of field q at
 *                the corner (the sum of the absolute values of every
 *                contribution deposited there, gross = NULL: |field|): the
 *                scale of the rounding error of a node value accumulated
 *                from single-precision contributions, and of the
 *                interpolation itself. */
void or_interp_aux(const or_grid *g, const double *field, const double *gross, const double *s, double *H,
                   double *A) {
  int d = g->d, nf = 1 + d;
  int i0[3] = {0, 0, 0}, i1[3] = {0, 0, 0}, clamped[3] = {0, 0, 0};
  double f[3] = {0, 0, 0}, D[3] = {1, 1, 1};
  for (int k = 0; k < d; ++k) {
    D[k] = grid_spacing(g, k);
    double u = (s[k] - g->lo[k]) / D[k];
    if (g->periodic[k]) {
      u = wrap_u(u, g->n[k]);
      int a = (int)floor(u);
      if (a > g->n[k] - 1) a = g->n[k] - 1;
      i0[k] = a;
      i1[k] = (a + 1) % g->n[k];
      f[k] = u - a;
    } else {
      if (u < 0.0) { u = 0.0; clamped[k] = 1; }
      if (u > g->n[k] - 1) { u = g->n[k] - 1; clamped[k] = 1; }
      int a = (int)floor(u);
      if (a > g->n[k] - 2) a = g->n[k] - 2;
      i0[k] = a;
      i1[k] = a + 1;
      f[k] = u - a;
    }
  }
  for (int q = 0; q < 9; ++q) H[q] = 0.0;
  for (int q = 0; q < 4; ++q) A[q] = 0.0;
  for (int corner = 0; corner < (1 << d); ++corner) {
    double wgt = 1.0, dw[3] = {1, 1, 1};
    long node = 0, mul = 1;
    for (int k = 0; k < d; ++k) {
      int hi = (corner >> k) & 1;
      double wk = hi ? f[k] : 1.0 - f[k];
      wgt *= wk;
      /* d(weight)/ds_j: the factor of axis j replaced by its derivative */
      for (int j = 0; j < d; ++j) dw[j] *= (j == k) ? (hi ? 1.0 : -1.0) / D[k] : wk;
      node += mul * (hi ? i1[k] : i0[k]);
      mul *= g->n[k];
    }
    for (int q = 0; q < nf; ++q) A[q] += wgt * (gross ? gross[node * nf + q] : fabs(field[node * nf + q]));
    for (int k = 0; k < d; ++k)
      for (int j = 0; j < d; ++j)
        if (!clamped[k] && !clamped[j]) H[3 * k + j] += dw[j] * field[node * nf + 1 + k];
  }
}

/* First-order bound on the rounding error of an evaluation of CV c at x in
 * a binary floating-point format of unit roundoff u, in units of u (multiply
 * by u). The evaluation forms coordinate differences first and then follows
 * the definition; every rounding of an operation is counted at the operands'
 * magnitude (test infrastructure: the tolerance of a CV comparison).
 *   COM distance: the group sums over offsets from each group's first atom
 *     (n + 3 roundings per term), the difference of the first atoms, the
 *     norm (6 |s|); a minimum image adds 3 L per axis;
 *   dihedral: bond vectors rounded (each a shift of 1/sin of the adjacent
 *     bond angle, twice for the middle bond), then the two atan2 arguments,
 *     each within 10 roundings of |b1| |b2|^2 |b3| while their norm is
 *     |m| |n| = |b1| |b2|^2 |b3| sin(theta1) sin(theta2);
 *   coordination number: per pair q = r^2 / r0^2 within (7 q + 2 sum_q |v_q|
 *     |dx_q| / r0^2) roundings (dx before and v after a minimum image), the
 *     switch within 5 more, dsw/dq = -3 q^2 sw^2; the partial sums 16 |s|;
 *   RMSD: the reference rounded (|x0|), each difference, the sum of 3N
 *     squares and the square root. */
double or_cv_round_bound(const or_cv *c, const double *x) {
  if (c->type == OR_CV_COM_DIST) {
    double ra[3] = {0, 0, 0}, rb[3] = {0, 0, 0}, Ma = 0, Mb = 0, ea = 0, eb = 0;
    for (int i = 0; i < c->na; ++i) Ma += c->ma ? c->ma[i] : 1.0;
    for (int i = 0; i < c->nb; ++i) Mb += c->mb ? c->mb[i] : 1.0;
    const double *xa0 = x + 3 * c->ia[0], *xb0 = x + 3 * c->ib[0];
    for (int i = 0; i < c->na; ++i) {
      double m = (c->ma ? c->ma[i] : 1.0) / Ma;
      for (int k = 0; k < 3; ++k) {
        ra[k] += m * x[3 * c->ia[i] + k];
        ea += m * fabs(x[3 * c->ia[i] + k] - xa0[k]);
      }
    }
    for (int i = 0; i < c->nb; ++i) {
      double m = (c->mb ? c->mb[i] : 1.0) / Mb;
      for (int k = 0; k < 3; ++k) {
        rb[k] += m * x[3 * c->ib[i] + k];
        eb += m * fabs(x[3 * c->ib[i] + k] - xb0[k]);
      }
    }
    double dv[3], d0 = 0.0;
    for (int k = 0; k < 3; ++k) {
      dv[k] = rb[k] - ra[k];
      d0 += fabs(xb0[k] - xa0[k]);
    }
    min_image(dv, c);
    double s = sqrt(dot(dv, dv));
    double b = (c->na + 3) * ea + (c->nb + 3) * eb + 3.0 * d0 + 6.0 * s;
    if (c->pbc) b += 3.0 * (c->box[0] + c->box[1] + c->box[2]);
    return b;
  }
  if (c->type == OR_CV_DIHEDRAL) {
    const double *x1 = x + 3 * c->ia[0], *x2 = x + 3 * c->ia[1];
    const double *x3 = x + 3 * c->ia[2], *x4 = x + 3 * c->ia[3];
    double b1[3], b2[3], b3[3], m[3], n[3];
    for (int k = 0; k < 3; ++k) {
      b1[k] = x2[k] - x1[k];
      b2[k] = x3[k] - x2[k];
      b3[k] = x4[k] - x3[k];
    }
    min_image(b1, c);
    min_image(b2, c);
    min_image(b3, c);
    cross(b1, b2, m);
    cross(b2, b3, n);
    double l1 = sqrt(dot(b1, b1)), l2 = sqrt(dot(b2, b2)), l3 = sqrt(dot(b3, b3));
    double lm = sqrt(dot(m, m)), ln = sqrt(dot(n, n));
    if (lm == 0.0 || ln == 0.0) return INFINITY;
    double i1 = l1 * l2 / lm, i2 = l2 * l3 / ln; /* 1/sin of the two bond angles */
    double b = 4.0 * (i1 + i2) + 20.0 * i1 * i2;
    /* with a minimum image a bond component is rounded at the magnitude of
     * the raw difference (up to the box edge); |d phi/d b1| = i1 / |b1|,
     * |d phi/d b3| = i2 / |b3|, |d phi/d b2| <= (i1 + i2) / |b2| */
    if (c->pbc) {
      double L = fmax(c->box[0], fmax(c->box[1], c->box[2]));
      b += 2.0 * sqrt(3.0) * L * (i1 / l1 + i2 / l3 + (i1 + i2) / l2);
    }
    return b;
  }
  if (c->type == OR_CV_COORD) {
    double k2 = 1.0 / (c->r0 * c->r0), acc = 0.0, s = 0.0;
    for (int a = 0; a < c->na; ++a) {
      const double *xi = x + 3 * c->ia[a];
      for (int bb = 0; bb < c->nb; ++bb) {
        const double *xj = x + 3 * c->ib[bb];
        double raw[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
        double v[3] = {raw[0], raw[1], raw[2]};
        min_image(v, c);
        double q = dot(v, v) * k2;
        double sw = 1.0 / (1.0 + q * q * q);
        double dq = 7.0 * q + 2.0 * k2 * (fabs(v[0] * raw[0]) + fabs(v[1] * raw[1]) + fabs(v[2] * raw[2]));
        acc += 3.0 * q * q * sw * sw * dq + 5.0 * sw;
        s += sw;
      }
    }
    return acc + 16.0 * s;
  }
  if (c->type == OR_CV_RMSD) {
    double acc = 0.0, e = 0.0;
    for (int i = 0; i < c->na; ++i)
      for (int k = 0; k < 3; ++k) {
        double xv = x[3 * c->ia[i] + k], x0 = c->ref[3 * i + k], dd = xv - x0;
        acc += dd * dd;
        e += 2.0 * fabs(dd) * (fabs(x0) + fabs(dd));
      }
    double s = sqrt(acc / c->na + 0.01);
    return (e / c->na + (3.0 * c->na + 3.0) * (acc / c->na + 0.01)) / (2.0 * s) + s;
  }
  return 0.0; /* OR_CV_POS_X: a coordinate, exact */
}

/* ------------------------------------------------------------------ */
/* a2 + a3: well-tempered height and Gaussian deposit in a cutoff box   */
/* ------------------------------------------------------------------ */

double or_height(const or_hill *hl, double Vb) {
  double dT = (hl->gamma - 1.0) * hl->kT;
  return hl->w * exp(-Vb / dT);
}

/* Adds h*G and h*dG/dxi_k at every node of the stencil box around s.
 * ic_out receives the box centre indices. */
void or_deposit_hill(const or_grid *g, const or_hill *hl, double *field, const double *s,
                     double h, int *ic_out, double *gross) {
  int d = g->d, nf = 1 + d;
  int ic[3] = {0, 0, 0}, R[3] = {0, 0, 0};
  double D[3] = {1, 1, 1}, L[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) {
    D[k] = grid_spacing(g, k);
    L[k] = g->hi[k] - g->lo[k];
    double u = (s[k] - g->lo[k]) / D[k];
    if (g->periodic[k]) u = wrap_u(u, g->n[k]);
    ic[k] = (int)floor(u + 0.5);
    if (g->periodic[k] && ic[k] >= g->n[k]) ic[k] -= g->n[k];
    R[k] = or_stencil_halfwidth(g, hl, k);
    ic_out[k] = ic[k];
  }
  for (int k = d; k < 3; ++k) ic_out[k] = 0;
  int span[3] = {1, 1, 1};
  for (int k = 0; k < d; ++k) span[k] = 2 * R[k] + 1;
  for (int c2 = 0; c2 < span[2]; ++c2)
    for (int c1 = 0; c1 < span[1]; ++c1)
      for (int c0 = 0; c0 < span[0]; ++c0) {
        int off[3] = {c0, c1, c2};
        long node = 0, mul = 1;
        double dist[3] = {0, 0, 0}, r2 = 0.0;
        int inside = 1;
        for (int k = 0; k < d; ++k) {
          int j = ic[k] - R[k] + off[k];
          if (g->periodic[k]) {
            j %= g->n[k];
            if (j < 0) j += g->n[k];
          } else if (j < 0 || j >= g->n[k]) {
            inside = 0;
            break;
          }
          double xi = g->lo[k] + j * D[k];
          double dk = xi - s[k];
          if (g->periodic[k]) dk -= L[k] * floor(dk / L[k] + 0.5);
          dist[k] = dk;
          r2 += dk * dk / (2.0 * hl->sigma[k] * hl->sigma[k]);
          node += mul * j;
          mul *= g->n[k];
        }
        if (!inside) continue;
        double hG = h * exp(-r2);
        field[node * nf] += hG;
        if (gross) gross[node * nf] += fabs(hG);
        for (int k = 0; k < d; ++k) {
          double v = hG * (-dist[k] / (hl->sigma[k] * hl->sigma[k]));
          field[node * nf + 1 + k] += v;
          if (gross) gross[node * nf + 1 + k] += fabs(v);
        }
      }
}

/* ------------------------------------------------------------------ */
/* mABP with compact hills                                              */
/* ------------------------------------------------------------------ */

/* The compact hill of Eq. (compacthill) along one CV, S = e^p e^(-p/(1-x^2))
 * for |x| = |u/a| < 1 (written as e^(-p x^2/(1-x^2)), the same number), else
 * 0; *dSdu receives dS/du. */
double or_compact(double u, double a, int p, double *dSdu) {
  double x = u / a;
  if (!(fabs(x) < 1.0)) {
    *dSdu = 0.0;
    return 0.0;
  }
  double om = 1.0 - x * x;
  double S = exp(-p * x * x / om);
  *dSdu = -2.0 * p * x * S / (a * om * om);
  return S;
}

/* Nearest grid node to s along every axis (limited to the grid on a
 * non-periodic axis, recorded in limited[k]). */
static void nearest_node(const or_grid *g, const double *s, int *ic, int *limited) {
  for (int k = 0; k < g->d; ++k) {
    double D = grid_spacing(g, k);
    double u = (s[k] - g->lo[k]) / D;
    limited[k] = 0;
    if (g->periodic[k]) {
      u = wrap_u(u, g->n[k]);
      int i = (int)floor(u + 0.5);
      ic[k] = i >= g->n[k] ? i - g->n[k] : i;
    } else {
      double i = floor(u + 0.5);
      if (i < 0) { i = 0; limited[k] = 1; }
      if (i > g->n[k] - 1) { i = g->n[k] - 1; limited[k] = 1; }
      ic[k] = (int)i;
    }
  }
}

/* Eq. (Cupdate) at the nearest node xi* to s: h += w S(xi* - xi) and
 * h'_i += w dS(xi* - xi)/dxi_i on every node within a of xi* (per axis),
 * S the product of the one-dimensional compact hills. */
void or_deposit_compact(const or_grid *g, const or_hill *hl, double *field, const double *s, double w,
                        int *ic_out, double *gross) {
  int d = g->d, nf = 1 + d;
  int ic[3] = {0, 0, 0}, R[3] = {0, 0, 0}, lim[3];
  double D[3] = {1, 1, 1};
  nearest_node(g, s, ic, lim);
  for (int k = 0; k < d; ++k) {
    D[k] = grid_spacing(g, k);
    R[k] = or_stencil_halfwidth(g, hl, k);
    ic_out[k] = ic[k];
  }
  for (int k = d; k < 3; ++k) ic_out[k] = 0;
  int span[3] = {1, 1, 1};
  for (int k = 0; k < d; ++k) span[k] = 2 * R[k] + 1;
  for (int c2 = 0; c2 < span[2]; ++c2)
    for (int c1 = 0; c1 < span[1]; ++c1)
      for (int c0 = 0; c0 < span[0]; ++c0) {
        int off[3] = {c0 - R[0], c1 - R[1], c2 - R[2]};
        long node = 0, mul = 1;
        double S[3] = {1, 1, 1}, dS[3] = {0, 0, 0};
        int inside = 1;
        for (int k = 0; k < d; ++k) {
          int j = ic[k] + off[k];
          if (g->periodic[k]) {
            j %= g->n[k];
            if (j < 0) j += g->n[k];
          } else if (j < 0 || j >= g->n[k]) {
            inside = 0;
            break;
          }
          /* u = xi*_k - xi_k, the node's offset from the centre */
          S[k] = or_compact(-off[k] * D[k], hl->a[k], hl->p, &dS[k]);
          node += mul * j;
          mul *= g->n[k];
        }
        if (!inside) continue;
        double prod = S[0] * S[1] * S[2];
        field[node * nf] += w * prod;
        if (gross) gross[node * nf] += fabs(w * prod);
        for (int k = 0; k < d; ++k) {
          double other = 1.0;
          for (int q = 0; q < d; ++q)
            if (q != k) other *= S[q];
          /* d S(xi* - xi) / d xi_k = - S'(u_k) * prod of the other axes */
          field[node * nf + 1 + k] += w * (-dS[k]) * other;
          if (gross) gross[node * nf + 1 + k] += fabs(w * dS[k] * other);
        }
      }
}

/* Eq. (apfm) and Eq. (btraj-grad) at the nearest node to s:
 *   V = kT b/(1-b) ln(c (1-b) h + 1),  dV/dxi_i = c b kT h'_i / (1 + c (1-b) h).
 * Returns OR_FLAG_OOR if s left a non-periodic range (that gradient is 0). */
int or_lookup_mabp(const or_grid *g, const or_hill *hl, const double *field, const double *s, double *V,
                   double *dV) {
  int d = g->d, nf = 1 + d, flag = 0;
  int ic[3] = {0, 0, 0}, lim[3] = {0, 0, 0};
  nearest_node(g, s, ic, lim);
  long node = 0, mul = 1;
  for (int k = 0; k < d; ++k) {
    node += mul * ic[k];
    mul *= g->n[k];
    if (lim[k]) flag = OR_FLAG_OOR;
  }
  double h = field[node * nf];
  double den = 1.0 + hl->c * (1.0 - hl->b) * h;
  *V = hl->kT * hl->b / (1.0 - hl->b) * log(den);
  for (int k = 0; k < d; ++k) dV[k] = lim[k] ? 0.0 : hl->c * hl->b * hl->kT * field[node * nf + 1 + k] / den;
  return flag;
}

/* dU/ds_k of the CV range limit: kwall (s - smax_k) above smax_k, else 0. */
double or_wall_grad(const or_hill *hl, int k, double s) {
  return (hl->kwall > 0 && s > hl->smax[k]) ? hl->kwall * (s - hl->smax[k]) : 0.0;
}

/* ------------------------------------------------------------------ */
/* closed-loop dynamics: counter-based noise, CV potentials, moves      */
/* ------------------------------------------------------------------ */

/* The model MD engine of the closed-loop workloads (not part of the paper's
 * method, which receives coordinates from an MD code and returns the bias
 * force): every CV atom moves by overdamped Langevin dynamics,
 *   x_i <- x_i + dt mu F_i + sqrt(2 mu kT dt) xi_i,
 *   F_i = -sum_k (dV_b/ds_k + dU/ds_k) ds_k/dx_i,
 * F_i the bias force of the step plus the force of a potential U(s) of the
 * walker's CVs, xi_i three standard normals per atom and step. */

/* Philox-4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11). A round multiplies counter
 * words 0 and 2 by the two round multipliers; the new counter is
 *   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
 * and the key advances by the two Weyl increments before every round but
 * the first. */
void or_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* A 32-bit word's top 24 bits as a uniform number in (0, 1): (j + 1/2) 2^-24,
 * exact in single and double precision. */
double or_uniform24(uint32_t r) { return ((double)(r >> 8) + 0.5) * (1.0 / 16777216.0); }

/* Three standard normals for one atom of one walker at one MD step:
 * Philox with counter (atom, step low word, step high word, stream) and key
 * (seed low word, seed high word); the four uniforms u0..u3 give
 *   n0 = r0 cos(2 pi u1), n1 = r0 sin(2 pi u1), n2 = r2 cos(2 pi u3),
 *   r = sqrt(-2 ln u) (Box and Muller, Ann. Math. Stat. 29 (1958)). */
void or_md_normals(uint64_t seed, uint32_t stream, int64_t step, int atom, double *n) {
  uint32_t ctr[4] = {(uint32_t)atom, (uint32_t)((uint64_t)step & 0xffffffffu), (uint32_t)((uint64_t)step >> 32),
                     stream};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t r[4];
  or_philox4x32_10(ctr, key, r);
  double u0 = or_uniform24(r[0]), u1 = or_uniform24(r[1]), u2 = or_uniform24(r[2]), u3 = or_uniform24(r[3]);
  const double two_pi = 6.283185307179586476925286766559;
  double r0 = sqrt(-2.0 * log(u0)), r2 = sqrt(-2.0 * log(u2));
  n[0] = r0 * cos(two_pi * u1);
  n[1] = r0 * sin(two_pi * u1);
  n[2] = r2 * cos(two_pi * u3);
}

/* U(s) of the walker's CVs and dU/ds_k (k < 3; unused entries 0):
 *   OR_POT_DOUBLE_WELL   U = A (s_0^2 - B^2)^2;
 *   OR_POT_MULLER_BROWN  U = scale sum_{i<4} A_i exp(a_i X'^2 + b_i X' Y' + c_i Y'^2),
 *                        X' = X - x0_i, Y' = Y - y0_i, X = mx s_0 + cx, Y = my s_1 + cy
 *                        (the four-term surface of Mueller and Brown,
 *                        Theor. Chim. Acta 53 (1979), on an affine image of
 *                        the CV box). */
double or_md_potential(const or_md *md, const double *s, double *dU) {
  dU[0] = dU[1] = dU[2] = 0.0;
  if (md->pot == OR_POT_DOUBLE_WELL) {
    double q = s[0] * s[0] - md->dw_b * md->dw_b;
    dU[0] = 4.0 * md->dw_a * s[0] * q;
    return md->dw_a * q * q;
  }
  if (md->pot == OR_POT_MULLER_BROWN) {
    double X = md->mb_map[0] * s[0] + md->mb_map[1], Y = md->mb_map[2] * s[1] + md->mb_map[3];
    double U = 0.0, dX = 0.0, dY = 0.0;
    for (int i = 0; i < 4; ++i) {
      double xp = X - md->mb_x0[i], yp = Y - md->mb_y0[i];
      double e = md->mb_A[i] * exp(md->mb_a[i] * xp * xp + md->mb_b[i] * xp * yp + md->mb_c[i] * yp * yp);
      U += e;
      dX += e * (2.0 * md->mb_a[i] * xp + md->mb_b[i] * yp);
      dY += e * (md->mb_b[i] * xp + 2.0 * md->mb_c[i] * yp);
    }
    dU[0] = md->mb_scale * md->mb_map[0] * dX;
    dU[1] = md->mb_scale * md->mb_map[2] * dY;
    return md->mb_scale * U;
  }
  return 0.0;
}

/* One move of one walker's atoms (see the section head): xn = x + dt mu
 * (Fb - sum_k dU/ds_k J_k) + sqrt(2 mu kT dt) xi, with Fb the step's bias
 * force and J_k = ds_k/dx at x. */
void or_md_move(const or_walker *wk, const or_md *md, uint32_t stream, int64_t step, const double *x,
                const double *Fb, const double *s, const double *const *J, double *xn) {
  double dU[3];
  or_md_potential(md, s, dU);
  double amp = sqrt(2.0 * md->mu * md->kT * md->dt);
  for (int i = 0; i < wk->natoms; ++i) {
    double nz[3];
    or_md_normals(md->seed, stream, step, i, nz);
    for (int q = 0; q < 3; ++q) {
      int a = 3 * i + q;
      double f = Fb[a];
      for (int k = 0; k < wk->g.d; ++k) f -= dU[k] * J[k][a];
      xn[a] = x[a] + md->dt * md->mu * f + amp * nz[q];
      if (md->state_f32) xn[a] = (double)(float)xn[a];
    }
  }
}

/* ------------------------------------------------------------------ */
/* one MD step for a batch of walkers                                   */
/* ------------------------------------------------------------------ */

/* fields[w] is walker w's grid; walkers whose pointers are equal share one
 * grid. x[w] holds walker w's atoms (natoms x 3). F[w] (natoms x 3) is
 * overwritten with the bias force. s/V/dV: per walker, 3 slots each for s
 * and dV. dep: one record per walker (valid where flags & DEPOSIT).
 * Returns 0, or OR_FLAG_BADARG on an unusable walker. */
int or_batch_step(int nw, const or_walker *wk, double *const *fields, const double *const *x,
                  int64_t step, double *s, double *V, double *dV, double *const *F, int *flags,
                  or_deposit *dep, const or_md *md, const uint32_t *streams, double *const *xn,
                  or_stepaux *aux, double *const *Jn, double *const *gross) {
  for (int w = 0; w < nw; ++w)
    if (or_check(&wk[w].g, &wk[w].hill)) return OR_FLAG_BADARG;

  /* a1: CVs for every walker; Jacobians kept for a5 */
  double **J = (double **)malloc(sizeof(double *) * (size_t)nw * OR_MAXCV);
  int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
  for (int w = 0; w < nw; ++w) {
    flags[w] = 0;
    for (int k = 0; k < wk[w].g.d; ++k) {
      J[w * OR_MAXCV + k] = (double *)malloc(sizeof(double) * 3 * (size_t)wk[w].natoms);
      int fl = or_cv_eval(&wk[w].cv[k], wk[w].natoms, x[w], &s[3 * w + k], J[w * OR_MAXCV + k]);
      if (fl & OR_FLAG_BADARG) bad = 1;
      flags[w] |= fl;
      if (aux) aux[w].sb[k] = or_cv_round_bound(&wk[w].cv[k], x[w]);
    }
    for (int k = wk[w].g.d; k < 3; ++k) s[3 * w + k] = 0.0;
  }

  /* a2: heights of this step's hills, all from the grids as they were
   * before any deposit of this step (mABP hills have height w) */
  double *h = (double *)calloc((size_t)nw, sizeof(double));
  for (int w = 0; w < nw; ++w) {
    if (step % wk[w].hill.stride != 0) continue;
    if (wk[w].hill.method == OR_METHOD_MABP_COMPACT) {
      h[w] = wk[w].hill.w;
      continue;
    }
    double Vb, g3[3];
    flags[w] |= or_interp(&wk[w].g, fields[w], &s[3 * w], &Vb, g3);
    h[w] = or_height(&wk[w].hill, Vb);
  }

  /* a3: deposits, in walker order */
  for (int w = 0; w < nw; ++w) {
    if (step % wk[w].hill.stride != 0) continue;
    dep[w].step = step;
    dep[w].walker = w;
    dep[w].height = h[w];
    for (int k = 0; k < 3; ++k) dep[w].s[k] = s[3 * w + k];
    double *gw = gross ? gross[w] : NULL;
    if (wk[w].hill.method == OR_METHOD_MABP_COMPACT)
      or_deposit_compact(&wk[w].g, &wk[w].hill, fields[w], &s[3 * w], h[w], dep[w].ic, gw);
    else
      or_deposit_hill(&wk[w].g, &wk[w].hill, fields[w], &s[3 * w], h[w], dep[w].ic, gw);
    flags[w] |= OR_FLAG_DEPOSIT;
  }

  /* a4 + a5: interpolation after all deposits, then the chain rule */
#pragma omp parallel for schedule(dynamic)
  for (int w = 0; w < nw; ++w) {
    int d = wk[w].g.d;
    double g3[3] = {0, 0, 0};
    if (wk[w].hill.method == OR_METHOD_MABP_COMPACT)
      flags[w] |= or_lookup_mabp(&wk[w].g, &wk[w].hill, fields[w], &s[3 * w], &V[w], g3);
    else
      flags[w] |= or_interp(&wk[w].g, fields[w], &s[3 * w], &V[w], g3);
    for (int k = 0; k < d; ++k) g3[k] += or_wall_grad(&wk[w].hill, k, s[3 * w + k]);
    if (aux) {
      for (int k = d; k < 3; ++k) aux[w].sb[k] = 0.0;
      if (wk[w].hill.method == OR_METHOD_MABP_COMPACT) {
        /* a node look-up: no slope inside a cell; the rounding scale is the
         * bias and its gradient themselves, and the gross histograms at the
         * node through dV/dh' = c b kT / (1 + c (1-b) h) */
        for (int q = 0; q < 9; ++q) aux[w].H[q] = 0.0;
        aux[w].A[0] = fabs(V[w]);
        int ic[3] = {0, 0, 0}, lim[3];
        nearest_node(&wk[w].g, &s[3 * w], ic, lim);
        long node = 0, mul = 1;
        for (int k = 0; k < d; ++k) {
          node += mul * ic[k];
          mul *= wk[w].g.n[k];
        }
        const double *fw = fields[w];
        const double den = 1.0 + wk[w].hill.c * (1.0 - wk[w].hill.b) * fw[node * (1 + d)];
        const double gfac = wk[w].hill.c * wk[w].hill.b * wk[w].hill.kT / den;
        for (int k = 0; k < 3; ++k)
          aux[w].A[1 + k] = k < d ? fabs(g3[k]) + (gross ? gfac * gross[w][node * (1 + d) + 1 + k] : 0.0) : 0.0;
      } else {
        or_interp_aux(&wk[w].g, fields[w], gross ? gross[w] : NULL, &s[3 * w], aux[w].H, aux[w].A);
      }
      for (int k = 0; k < d; ++k)
        if (or_wall_grad(&wk[w].hill, k, s[3 * w + k]) != 0.0) aux[w].H[4 * k] += wk[w].hill.kwall;
    }
    if (Jn && Jn[w])
      for (int i = 0; i < wk[w].natoms; ++i)
        for (int k = 0; k < 3; ++k) {
          double n2 = 0.0;
          if (k < d)
            for (int q = 0; q < 3; ++q) n2 += J[w * OR_MAXCV + k][3 * i + q] * J[w * OR_MAXCV + k][3 * i + q];
          Jn[w][3 * i + k] = sqrt(n2);
        }
    for (int k = 0; k < 3; ++k) dV[3 * w + k] = g3[k];
    double *Fw = F[w];
    for (int a = 0; a < 3 * wk[w].natoms; ++a) {
      double acc = 0.0;
      for (int k = 0; k < d; ++k) acc += g3[k] * J[w * OR_MAXCV + k][a];
      Fw[a] = -acc;
    }
    /* closed loop: the move of this step from x, the bias force and the
     * force of the CV potential (this step's CVs and Jacobians) */
    if (md) {
      const double *Jw[OR_MAXCV] = {NULL, NULL, NULL};
      for (int k = 0; k < d; ++k) Jw[k] = J[w * OR_MAXCV + k];
      or_md_move(&wk[w], md, streams ? streams[w] : 0u, step, x[w], Fw, &s[3 * w], Jw, xn[w]);
    }
    for (int k = 0; k < d; ++k) free(J[w * OR_MAXCV + k]);
  }
  free(J);
  free(h);
  return bad ? OR_FLAG_BADARG : 0;
}

/* ------------------------------------------------------------------ */
/* open-loop replay of a recorded trajectory                            */
/* ------------------------------------------------------------------ */

/* Runs T consecutive steps step0..step0+T-1. Walker w's atoms at step t are
 * frames[t*frame_stride + atom_off[w] + 3*i] (doubles). Optional outputs
 * (NULL to skip): s_hist [T][nw][3], V_hist [T][nw], dV_hist [T][nw][3],
 * F_hist [T][frame_stride] (forces at the same offsets as the frames),
 * flag_hist [T][nw], dep_log (capacity dep_cap; *n_dep receives the count).
 * With md (and Xn_hist [T][frame_stride]) the replay also predicts, for each
 * step, the coordinates after that step's closed-loop move from the recorded
 * ones (or_md_move; streams[w] is walker w's noise stream): a recorded
 * closed-loop trajectory is checked one step at a time against it.
 * aux_hist [T][nw] and Jn_hist [T][frame_stride] (optional) receive each
 * step's or_stepaux and, per atom, |ds_k/dx| of each CV k (error-analysis
 * outputs for per-step comparisons); gross (optional, laid out and shared
 * like fields) accumulates the absolute values of every deposited
 * contribution, the scale of the accumulated grid's rounding.
 * Returns 0 or OR_FLAG_BADARG. */
int or_run(int nw, const or_walker *wk, double *const *fields, const double *frames,
           const int64_t *atom_off, int64_t frame_stride, int64_t step0, int64_t T,
           double *s_hist, double *V_hist, double *dV_hist, double *F_hist, int *flag_hist,
           or_deposit *dep_log, int64_t dep_cap, int64_t *n_dep, const or_md *md, const uint32_t *streams,
           double *Xn_hist, or_stepaux *aux_hist, double *Jn_hist, double *const *gross) {
  const double **x = (const double **)malloc(sizeof(double *) * (size_t)nw);
  double **F = (double **)malloc(sizeof(double *) * (size_t)nw);
  double *s = (double *)malloc(sizeof(double) * 3 * (size_t)nw);
  double *V = (double *)malloc(sizeof(double) * (size_t)nw);
  double *dV = (double *)malloc(sizeof(double) * 3 * (size_t)nw);
  int *fl = (int *)malloc(sizeof(int) * (size_t)nw);
  or_deposit *dep = (or_deposit *)malloc(sizeof(or_deposit) * (size_t)nw);
  double *Fscratch = F_hist ? NULL : (double *)malloc(sizeof(double) * (size_t)frame_stride);
  int64_t nd = 0;
  int rc = 0;
  double **Xn = (double **)malloc(sizeof(double *) * (size_t)nw);
  double **Jn = (double **)malloc(sizeof(double *) * (size_t)nw);
  for (int64_t t = 0; t < T && rc == 0; ++t) {
    for (int w = 0; w < nw; ++w) {
      x[w] = frames + t * frame_stride + atom_off[w];
      F[w] = (F_hist ? F_hist + t * frame_stride : Fscratch) + atom_off[w];
      Xn[w] = (md && Xn_hist) ? Xn_hist + t * frame_stride + atom_off[w] : NULL;
      Jn[w] = Jn_hist ? Jn_hist + t * frame_stride + atom_off[w] : NULL;
    }
    rc = or_batch_step(nw, wk, fields, x, step0 + t, s, V, dV, F, fl, dep, (md && Xn_hist) ? md : NULL, streams,
                       Xn, aux_hist ? aux_hist + t * nw : NULL, Jn_hist ? Jn : NULL, gross);
    for (int w = 0; w < nw; ++w) {
      if (s_hist) for (int k = 0; k < 3; ++k) s_hist[(t * nw + w) * 3 + k] = s[3 * w + k];
      if (V_hist) V_hist[t * nw + w] = V[w];
      if (dV_hist) for (int k = 0; k < 3; ++k) dV_hist[(t * nw + w) * 3 + k] = dV[3 * w + k];
      if (flag_hist) flag_hist[t * nw + w] = fl[w];
      if ((fl[w] & OR_FLAG_DEPOSIT) && dep_log && nd < dep_cap) dep_log[nd] = dep[w];
      if (fl[w] & OR_FLAG_DEPOSIT) ++nd;
    }
  }
  if (n_dep) *n_dep = nd;
  free(Xn);
  free(Jn);
  free(x);
  free(F);
  free(s);
  free(V);
  free(dV);
  free(fl);
  free(dep);
  free(Fscratch);
  return rc;
}

/* Closed-loop run: steps step0..step0+T-1 of nw walkers whose atoms start
 * in x (one frame laid out as in or_run: walker w's atoms at atom_off[w],
 * frame_stride doubles), each step's move (or_md_move) applied in place.
 * Optional outputs (NULL to skip): X_hist [T][frame_stride], the coordinates
 * each step's bias was evaluated at; s_hist [T][nw][3]; V_hist [T][nw];
 * the deposit log as in or_run. Returns 0 or OR_FLAG_BADARG. */
int or_md_run(int nw, const or_walker *wk, double *const *fields, double *x, const int64_t *atom_off,
              int64_t frame_stride, const or_md *md, const uint32_t *streams, int64_t step0, int64_t T,
              double *X_hist, double *s_hist, double *V_hist, or_deposit *dep_log, int64_t dep_cap,
              int64_t *n_dep) {
  const double **xs = (const double **)malloc(sizeof(double *) * (size_t)nw);
  double **F = (double **)malloc(sizeof(double *) * (size_t)nw);
  double **Xn = (double **)malloc(sizeof(double *) * (size_t)nw);
  double *Fbuf = (double *)malloc(sizeof(double) * (size_t)frame_stride);
  double *xnext = (double *)malloc(sizeof(double) * (size_t)frame_stride);
  double *s = (double *)malloc(sizeof(double) * 3 * (size_t)nw);
  double *V = (double *)malloc(sizeof(double) * (size_t)nw);
  double *dV = (double *)malloc(sizeof(double) * 3 * (size_t)nw);
  int *fl = (int *)malloc(sizeof(int) * (size_t)nw);
  or_deposit *dep = (or_deposit *)malloc(sizeof(or_deposit) * (size_t)nw);
  int64_t nd = 0;
  int rc = 0;
  for (int w = 0; w < nw; ++w) {
    xs[w] = x + atom_off[w];
    F[w] = Fbuf + atom_off[w];
    Xn[w] = xnext + atom_off[w];
  }
  for (int64_t t = 0; t < T && rc == 0; ++t) {
    if (X_hist) memcpy(X_hist + t * frame_stride, x, sizeof(double) * (size_t)frame_stride);
    rc = or_batch_step(nw, wk, fields, xs, step0 + t, s, V, dV, F, fl, dep, md, streams, Xn, NULL, NULL, NULL);
    for (int w = 0; w < nw; ++w) {
      memcpy(x + atom_off[w], Xn[w], sizeof(double) * 3 * (size_t)wk[w].natoms);
      if (s_hist) for (int k = 0; k < 3; ++k) s_hist[(t * nw + w) * 3 + k] = s[3 * w + k];
      if (V_hist) V_hist[t * nw + w] = V[w];
      if ((fl[w] & OR_FLAG_DEPOSIT) && dep_log && nd < dep_cap) dep_log[nd] = dep[w];
      if (fl[w] & OR_FLAG_DEPOSIT) ++nd;
    }
  }
  if (n_dep) *n_dep = nd;
  free(xs);
  free(F);
  free(Xn);
  free(Fbuf);
  free(xnext);
  free(s);
  free(V);
  free(dV);
  free(fl);
  free(dep);
  return rc;
}

/* ------------------------------------------------------------------ */
/* closed-loop driver (used only to check the converged bias)           */
/* ------------------------------------------------------------------ */

/* Overdamped Langevin for one walker under U(s) = kw (s^2 - 1)^2 on its
 * first CV plus the bias:
 *   x += dt mu F + sqrt(2 mu kT dt) N(0,1),  F = -(U'(s) + dV_b/ds) ds/dx.
 * noise: [T][natoms*3] standard normals supplied by the caller. x (natoms*3)
 * is advanced in place; s_hist[T] (optional) records s before each move. */
int or_langevin_double_well(const or_walker *wk, double *field, double *x, int64_t T, double dt,
                            double mu, double kw, const double *noise, double *s_hist) {
  int na3 = 3 * wk->natoms;
  double *F = (double *)malloc(sizeof(double) * (size_t)na3);
  double *J = (double *)malloc(sizeof(double) * (size_t)na3);
  double *fields[1] = {field};
  const double *xs[1] = {x};
  double *Fs[1] = {F};
  double s[3], V, dV[3];
  int fl;
  or_deposit dep;
  int rc = 0;
  double amp = sqrt(2.0 * mu * wk->hill.kT * dt);
  for (int64_t t = 0; t < T && rc == 0; ++t) {
    rc = or_batch_step(1, wk, fields, xs, t, s, &V, dV, Fs, &fl, &dep, NULL, NULL, NULL, NULL, NULL, NULL);
    if (s_hist) s_hist[t] = s[0];
    double sv;
    or_cv_eval(&wk->cv[0], wk->natoms, x, &sv, J);
    double dU = 4.0 * kw * sv * (sv * sv - 1.0);
    for (int a = 0; a < na3; ++a)
      x[a] += dt * mu * (F[a] - dU * J[a]) + amp * noise[t * na3 + a];
  }
  free(F);
  free(J);
  return rc;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
