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
 * Conventions taken where the paper is silent (each also listed in the
 * design notes):
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
                     double h, int *ic_out) {
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
        for (int k = 0; k < d; ++k)
          field[node * nf + 1 + k] += hG * (-dist[k] / (hl->sigma[k] * hl->sigma[k]));
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
                        int *ic_out) {
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
        for (int k = 0; k < d; ++k) {
          double other = 1.0;
          for (int q = 0; q < d; ++q)
            if (q != k) other *= S[q];
          /* d S(xi* - xi) / d xi_k = - S'(u_k) * prod of the other axes */
          field[node * nf + 1 + k] += w * (-dS[k]) * other;
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
/* one MD step for a batch of walkers                                   */
/* ------------------------------------------------------------------ */

/* fields[w] is walker w's grid; walkers whose pointers are equal share one
 * grid. x[w] holds walker w's atoms (natoms x 3). F[w] (natoms x 3) is
 * overwritten with the bias force. s/V/dV: per walker, 3 slots each for s
 * and dV. dep: one record per walker (valid where flags & DEPOSIT).
 * Returns 0, or OR_FLAG_BADARG on an unusable walker. */
int or_batch_step(int nw, const or_walker *wk, double *const *fields, const double *const *x,
                  int64_t step, double *s, double *V, double *dV, double *const *F, int *flags,
                  or_deposit *dep) {
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
    if (wk[w].hill.method == OR_METHOD_MABP_COMPACT)
      or_deposit_compact(&wk[w].g, &wk[w].hill, fields[w], &s[3 * w], h[w], dep[w].ic);
    else
      or_deposit_hill(&wk[w].g, &wk[w].hill, fields[w], &s[3 * w], h[w], dep[w].ic);
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
    for (int k = 0; k < 3; ++k) dV[3 * w + k] = g3[k];
    double *Fw = F[w];
    for (int a = 0; a < 3 * wk[w].natoms; ++a) {
      double acc = 0.0;
      for (int k = 0; k < d; ++k) acc += g3[k] * J[w * OR_MAXCV + k][a];
      Fw[a] = -acc;
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
 * Returns 0 or OR_FLAG_BADARG. */
int or_run(int nw, const or_walker *wk, double *const *fields, const double *frames,
           const int64_t *atom_off, int64_t frame_stride, int64_t step0, int64_t T,
           double *s_hist, double *V_hist, double *dV_hist, double *F_hist, int *flag_hist,
           or_deposit *dep_log, int64_t dep_cap, int64_t *n_dep) {
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
  for (int64_t t = 0; t < T && rc == 0; ++t) {
    for (int w = 0; w < nw; ++w) {
      x[w] = frames + t * frame_stride + atom_off[w];
      F[w] = (F_hist ? F_hist + t * frame_stride : Fscratch) + atom_off[w];
    }
    rc = or_batch_step(nw, wk, fields, x, step0 + t, s, V, dV, F, fl, dep);
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
    rc = or_batch_step(1, wk, fields, xs, t, s, &V, dV, Fs, &fl, &dep);
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
