/*
 * pic_oracle.c -- plain, slow FP64 CPU oracle of the electromagnetic PIC step
 * of Hemker's OSIRIS thesis (arxiv 1503.00276), ch. 3 "PIC Algorithms for
 * 2D-Cartesian Simulations" and "3D-Cartesian ... Algorithms".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header or table with the CUDA library; the two meet only through the seeded
 * input generator.
 *
 * Units are the paper's normalised units (appendix, "Input File": frequency
 * w_p, mass m_e, charge e, speed c all 1), so the 4*pi and c factors of the
 * Gaussian-unit equations drop out:  dE/dt = curl B - J,  dB/dt = -curl E,
 * div E = rho,  du/dt = (q/m)(E + v x B).
 *
 * Grid arrays are [nz][ny][nx] doubles (nz = 1 in 2D) with no guard cells;
 * every index is wrapped periodically where it is used.  Array index (i,j,k) of
 * a component with stagger s sits at ((i+s1)dx1, (j+s2)dx2, (k+s3)dx3) relative
 * to xmin.  The staggering is read off the difference stencils of the field
 * equations (the grid figure itself is missing from the text):
 *   E1 (1/2,0,0)  E2 (0,1/2,0)  E3 (0,0,1/2)   J like E,  rho at nodes
 *   B1 (0,1/2,1/2) B2 (1/2,0,1/2) B3 (1/2,1/2,0)
 * In 2D the x3 stagger is dropped (E3 and rho at nodes, B1 at (0,1/2), ...).
 *
 * Order of one step n -> n+1 (the PIC loop figure; OSIRIS flow chart):
 *   for every particle: gather E^n,B^n -> Boris push u^{n-1/2} -> u^{n+1/2}
 *   -> move x^n -> x^{n+1} -> charge-conserving current deposit -> periodic wrap;
 *   then optional binomial smoothing of J; then the field solve
 *   B^n -> B^{n+1/2} -> E^{n+1} -> B^{n+1}.
 *
 * Pins (tests/test_oracle_*.py): gyration phase and radius, E x B drift,
 * |u| conserved in pure B, free streaming, linear-field gather exactness,
 * discrete continuity to rounding (2D and 3D, with face and corner crossings),
 * exact brute-force current from the time integral of the shape flux
 * (rational arithmetic), Gauss law preserved over many steps, Yee amplification
 * eigenvalues against the discrete vacuum dispersion relation, (1,2,1)
 * transfer function cos^2(k dx/2), cold-plasma oscillation frequency, tile
 * binning against brute force; ISIS deposit equal to TRISTAN for in-cell
 * moves, continuity to rounding, hand-worked crossing example.  No function
 * below is "parity unpinned".
 *
 * Compiled with -ffp-contract=off so that every product and sum rounds as
 * written.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "pic_oracle.h"

/* ------------------------------------------------------------------------ */
/* indexing                                                                   */
/* ------------------------------------------------------------------------ */

static long wrapi(long i, long n) {
  long r = i % n;
  return r < 0 ? r + n : r;
}

/* open x1 (moving window): a grid value beyond x1 reads as 0 and a deposit
   there is dropped; every other index wraps periodically */
static int outside(const ora_grid* g, long i) { return g->open_x1 && (i < 0 || i >= g->nx[0]); }

static long at(const ora_grid* g, long i, long j, long k);

static double rd(const ora_grid* g, const double* F, long i, long j, long k) {
  return outside(g, i) ? 0.0 : F[at(g, i, j, k)];
}

static void add_to(const ora_grid* g, double* F, long i, long j, long k, double v) {
  if (!outside(g, i)) F[at(g, i, j, k)] += v;
}

static long at(const ora_grid* g, long i, long j, long k) {
  long nx = g->nx[0], ny = g->nx[1], nz = g->nx[2];
  return (wrapi(k, nz) * ny + wrapi(j, ny)) * nx + wrapi(i, nx);
}

/* stagger of E1,E2,E3,B1,B2,B3 in units of the cell size */
static const double STAG[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};

static double cell_volume(const ora_grid* g) {
  double v = g->dx[0] * g->dx[1];
  if (g->ndim == 3) v = v * g->dx[2];
  return v;
}

/* ------------------------------------------------------------------------ */
/* field interpolation: eq. "2d-field-weighting-e3" and its 3D extension     */
/* ------------------------------------------------------------------------ */

/* Component F (0..5) at global position x: weight linearly from the nearest
 * 2^ndim points of F's own staggered lattice.  In each direction
 * g = (x - xmin)/dx - s, cell i = floor(g), epsilon = g - i. */
static double interp_component(const ora_grid* g, const double* F, int comp, const double x[3]) {
  long i[3] = {0, 0, 0};
  double eps[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < g->ndim; ++d) {
    double gd = (x[d] - g->xmin[d]) / g->dx[d] - STAG[comp][d];
    double fl = floor(gd);
    i[d] = (long)fl;
    eps[d] = gd - fl;
  }
  if (g->ndim == 2) {
    /* (1-e1)[(1-e2) F(i1,i2) + e2 F(i1,i2+1)] + e1[(1-e2) F(i1+1,i2) + e2 F(i1+1,i2+1)] */
    double lo = (1.0 - eps[1]) * rd(g, F, i[0], i[1], 0) + eps[1] * rd(g, F, i[0], i[1] + 1, 0);
    double hi = (1.0 - eps[1]) * rd(g, F, i[0] + 1, i[1], 0) + eps[1] * rd(g, F, i[0] + 1, i[1] + 1, 0);
    return (1.0 - eps[0]) * lo + eps[0] * hi;
  }
  double acc = 0.0;
  for (int c3 = 0; c3 < 2; ++c3)
    for (int c2 = 0; c2 < 2; ++c2)
      for (int c1 = 0; c1 < 2; ++c1) {
        double w = (c1 ? eps[0] : 1.0 - eps[0]) * (c2 ? eps[1] : 1.0 - eps[1]) * (c3 ? eps[2] : 1.0 - eps[2]);
        acc = acc + w * rd(g, F, i[0] + c1, i[1] + c2, i[2] + c3);
      }
  return acc;
}

void ora_gather(const ora_grid* g, double* const fld[6], const double x[3], double eb[6]) {
  for (int c = 0; c < 6; ++c) {
    double ext = c < 3 ? g->e0[c] : g->b0[c - 3];
    eb[c] = interp_component(g, fld[c], c, x) + ext;
  }
}

/* ------------------------------------------------------------------------ */
/* momentum update: eq. "momentum-update" (Boris push)                        */
/* ------------------------------------------------------------------------ */

static void cross(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* u = p/(m c).  q/m = 1/rqm.  Reading of the garbled printed form: the
 * standard relativistic Boris rotation with t = (q/m)(dt/2) B / gamma' and the
 * factor 1/(1 + B^2) of the third line read as 1/(1 + |t|^2). */
void ora_boris(double u[3], const double e[3], const double b[3], double rqm, double dt) {
  double alpha = dt / (2.0 * rqm); /* (q/m) dt/2 */
  double p1[3], p2[3], p3[3], t[3], s[3], c[3];
  for (int d = 0; d < 3; ++d) p1[d] = u[d] + alpha * e[d];                 /* p'   */
  double gam = sqrt(1.0 + p1[0] * p1[0] + p1[1] * p1[1] + p1[2] * p1[2]);
  for (int d = 0; d < 3; ++d) t[d] = alpha * b[d] / gam;
  cross(p1, t, c);
  for (int d = 0; d < 3; ++d) p2[d] = p1[d] + c[d];                        /* p''  */
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int d = 0; d < 3; ++d) s[d] = 2.0 * t[d] / (1.0 + t2);
  cross(p2, s, c);
  for (int d = 0; d < 3; ++d) p3[d] = p1[d] + c[d];                        /* p''' */
  for (int d = 0; d < 3; ++d) u[d] = p3[d] + alpha * e[d];                 /* p^{n+1/2} */
}

/* ------------------------------------------------------------------------ */
/* position update: eq. "2d-position-update" (the printed leading q is read as */
/* a typo), only in-plane components in 2D                                    */
/* ------------------------------------------------------------------------ */

double ora_gamma(const double u[3]) { return sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]); }

void ora_move(const ora_grid* g, double x[3], const double u[3]) {
  double gam = ora_gamma(u);
  for (int d = 0; d < g->ndim; ++d) x[d] = x[d] + g->dt * u[d] / gam;
}

/* periodic boundary (node configuration "communicates with its own opposite boundary") */
void ora_wrap(const ora_grid* g, double x[3]) {
  for (int d = 0; d < g->ndim; ++d) {
    if (d == 0 && g->open_x1) continue; /* open x1: removed by the caller instead */
    double L = g->nx[d] * g->dx[d];
    double xmax = g->xmin[d] + L;
    while (x[d] >= xmax) x[d] = x[d] - L;
    while (x[d] < g->xmin[d]) x[d] = x[d] + L;
    if (x[d] >= xmax) x[d] = g->xmin[d];
  }
}

/* ------------------------------------------------------------------------ */
/* charge-conserving deposit, TRISTAN / Villasenor-Buneman                    */
/* ------------------------------------------------------------------------ */

/* One straight in-cell segment of a particle path, deposited as the average
 * over every ordering of its orthogonal moves (the paper's description of the
 * 2D method; the 3D method is its extension, and 2D3V adds the x3 move, whose
 * length is v3 times the segment's share of dt).
 *   cell[]     global index of the cell holding the segment
 *   a[], b[]   segment ends in cell units relative to that cell (in [0,1])
 *   v3frac     2D3V only: v3 * (fraction of dt spent on this segment)
 * During a move along d the particle sits at fixed transverse coordinates p_t,
 * and its flux through face cell_d + 1/2 is shared among the transverse nodes
 * with the linear weights (1 - p_t, p_t). */
static void deposit_segment(const ora_grid* g, double* cur[3], const long cell[3], const double a[3],
                            const double b[3], double v3frac, double q, int only_out_of_plane) {
  const int nd = g->ndim;
  const int nmoves = 3; /* 2D3V: x1, x2 and the out-of-plane x3 move; 3D: x1, x2, x3 */
  static const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const double nperm = 6.0;
  double dvol = cell_volume(g);
  for (int pi = 0; pi < 6; ++pi) {
    double p[3] = {a[0], a[1], nd == 3 ? a[2] : 0.0};
    for (int m = 0; m < nmoves; ++m) {
      int d = PERM[pi][m];
      if (nd == 2 && d == 2) {
        /* out-of-plane move: current density at the four nodes around p */
        double amp = q * v3frac / dvol / nperm;
        for (int c2 = 0; c2 < 2; ++c2)
          for (int c1 = 0; c1 < 2; ++c1) {
            double w = (c1 ? p[0] : 1.0 - p[0]) * (c2 ? p[1] : 1.0 - p[1]);
            add_to(g, cur[2], cell[0] + c1, cell[1] + c2, 0, amp * w);
          }
        continue;
      }
      if (only_out_of_plane) {
        p[d] = b[d];
        continue;
      }
      double delta = b[d] - a[d]; /* move length in cell units */
      double amp = q * delta * g->dx[d] / (g->dt * dvol) / nperm;
      if (nd == 2) {
        int t = 1 - d; /* the one transverse in-plane direction */
        for (int ct = 0; ct < 2; ++ct) {
          double w = ct ? p[t] : 1.0 - p[t];
          long idx[3] = {cell[0], cell[1], 0};
          idx[t] += ct;
          add_to(g, cur[d], idx[0], idx[1], 0, amp * w);
        }
      } else {
        int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
        for (int c2 = 0; c2 < 2; ++c2)
          for (int c1 = 0; c1 < 2; ++c1) {
            double w = (c1 ? p[t1] : 1.0 - p[t1]) * (c2 ? p[t2] : 1.0 - p[t2]);
            long idx[3] = {cell[0], cell[1], cell[2]};
            idx[t1] += c1;
            idx[t2] += c2;
            add_to(g, cur[d], idx[0], idx[1], idx[2], amp * w);
          }
      }
      p[d] = b[d];
    }
  }
}

/* Split the straight path xold -> xnew (global, unwrapped) at the cell faces it
 * crosses -- at most one per direction since |dx_d| < one cell -- and deposit
 * each in-cell piece.  v3 = u3/gamma (used in 2D3V only). */
static void deposit_pieces(const ora_grid* g, double* cur[3], const double xold[3], const double xnew[3],
                           double v3, double q, int only_out_of_plane) {
  const int nd = g->ndim;
  long i0[3] = {0, 0, 0};
  double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
  for (int d = 0; d < nd; ++d) {
    double go = (xold[d] - g->xmin[d]) / g->dx[d];
    double gn = (xnew[d] - g->xmin[d]) / g->dx[d];
    double fl = floor(go);
    i0[d] = (long)fl;
    a[d] = go - fl;
    b[d] = gn - fl;
  }
  /* crossings: path parameter, direction, face side */
  double tc[3];
  int dc[3], sc[3], nc = 0;
  for (int d = 0; d < nd; ++d) {
    if (b[d] < 0.0) {
      tc[nc] = (0.0 - a[d]) / (b[d] - a[d]);
      dc[nc] = d;
      sc[nc] = -1;
      ++nc;
    } else if (b[d] >= 1.0) {
      tc[nc] = (1.0 - a[d]) / (b[d] - a[d]);
      dc[nc] = d;
      sc[nc] = +1;
      ++nc;
    }
  }
  /* order the crossings along the path (insertion sort, at most 3) */
  for (int m = 1; m < nc; ++m)
    for (int r = m; r > 0 && tc[r] < tc[r - 1]; --r) {
      double tt = tc[r]; tc[r] = tc[r - 1]; tc[r - 1] = tt;
      int td = dc[r]; dc[r] = dc[r - 1]; dc[r - 1] = td;
      int ts = sc[r]; sc[r] = sc[r - 1]; sc[r - 1] = ts;
    }
  long off[3] = {0, 0, 0};            /* current cell relative to i0 */
  double p0[3] = {a[0], a[1], a[2]};  /* start of the current piece, relative to i0 */
  double t0 = 0.0;
  for (int m = 0; m <= nc; ++m) {
    double t1 = m < nc ? tc[m] : 1.0;
    double p1[3];
    for (int d = 0; d < 3; ++d) p1[d] = m < nc ? a[d] + t1 * (b[d] - a[d]) : b[d];
    if (m < nc) p1[dc[m]] = sc[m] > 0 ? 1.0 + (double)off[dc[m]] : (double)off[dc[m]];
    long cell[3];
    double la[3], lb[3];
    for (int d = 0; d < 3; ++d) {
      cell[d] = i0[d] + off[d];
      la[d] = p0[d] - (double)off[d];
      lb[d] = p1[d] - (double)off[d];
    }
    deposit_segment(g, cur, cell, la, lb, v3 * (t1 - t0), q, only_out_of_plane);
    if (m < nc) off[dc[m]] += sc[m];
    for (int d = 0; d < 3; ++d) p0[d] = p1[d];
    t0 = t1;
  }
}

void ora_deposit_vb(const ora_grid* g, double* cur[3], const double xold[3], const double xnew[3],
                    double v3, double q) {
  deposit_pieces(g, cur, xold, xnew, v3, q, 0);
}

/* linear charge weight of node k for a particle at s (cell units, nodes at the
   integers) */
static double lin_weight(double s, long k) {
  double r = fabs(s - (double)k);
  return r < 1.0 ? 1.0 - r : 0.0;
}

/* Current of one straight move along direction d (2D) from s_a to s_b (cell
   units), at the fixed transverse coordinate s_t, with the given weight
   (1/2 for one of the two orders).  The current through face k + 1/2 is the
   charge weight that left the nodes at or below k:
   flux(k) = - sum_{k' <= k} [S(s_b - k') - S(s_a - k')]. */
static void isis_move(const ora_grid* g, double* cur[3], int d, double s_a, double s_b, double s_t, double share,
                      double q) {
  const int t = 1 - d;
  const double amp = share * q * g->dx[d] / (g->dt * cell_volume(g));
  const long lo = (long)floor(fmin(s_a, s_b)) - 1, hi = (long)floor(fmax(s_a, s_b)) + 1;
  double flux = 0.0;
  for (long k = lo; k <= hi; ++k) {
    flux -= lin_weight(s_b, k) - lin_weight(s_a, k);
    if (flux == 0.0) continue;
    const long jt = (long)floor(s_t);
    for (long m = jt; m <= jt + 1; ++m) {
      const double w = lin_weight(s_t, m);
      long idx[2];
      idx[d] = k;
      idx[t] = m;
      add_to(g, cur[d], idx[0], idx[1], 0, amp * flux * w);
    }
  }
}

/* ISIS deposit (2D3V): the in-plane current of the whole straight path
   xold -> xnew, not split at cell faces, is the average of the two orders of
   orthogonal moves -- x1 then x2, and x2 then x1 -- each move's current
   following from the change of the linear charge weights it causes.  The
   out-of-plane J3 is the time integral of v3 times the charge weights along
   the straight path, which the thesis' two methods share. */
void ora_deposit_isis(const ora_grid* g, double* cur[3], const double xold[3], const double xnew[3],
                      double v3, double q) {
  double a[2], b[2];
  for (int d = 0; d < 2; ++d) {
    a[d] = (xold[d] - g->xmin[d]) / g->dx[d];
    b[d] = (xnew[d] - g->xmin[d]) / g->dx[d];
  }
  /* order 1: x1 at x2 = a2, then x2 at x1 = b1 */
  isis_move(g, cur, 0, a[0], b[0], a[1], 0.5, q);
  isis_move(g, cur, 1, a[1], b[1], b[0], 0.5, q);
  /* order 2: x2 at x1 = a1, then x1 at x2 = b2 */
  isis_move(g, cur, 1, a[1], b[1], a[0], 0.5, q);
  isis_move(g, cur, 0, a[0], b[0], b[1], 0.5, q);
  deposit_pieces(g, cur, xold, xnew, v3, q, 1);
}

/* ------------------------------------------------------------------------ */
/* charge density with the same linear weights (diagnostics, Gauss law)      */
/* ------------------------------------------------------------------------ */

void ora_deposit_rho(const ora_grid* g, double* rho, const double* x, long long n, double q) {
  ora_deposit_rho_w(g, rho, x, NULL, n, q);
}

/* the same with per-particle charge weights w[p] (NULL: all 1) */
void ora_deposit_rho_w(const ora_grid* g, double* rho, const double* x, const double* wt, long long n, double q0) {
  double dvol = cell_volume(g);
  for (long long p = 0; p < n; ++p) {
    const double q = wt ? q0 * wt[p] : q0;
    long i[3] = {0, 0, 0};
    double e[3] = {0, 0, 0};
    for (int d = 0; d < g->ndim; ++d) {
      double gd = (x[3 * p + d] - g->xmin[d]) / g->dx[d];
      double fl = floor(gd);
      i[d] = (long)fl;
      e[d] = gd - fl;
    }
    int n3 = g->ndim == 3 ? 2 : 1;
    for (int c3 = 0; c3 < n3; ++c3)
      for (int c2 = 0; c2 < 2; ++c2)
        for (int c1 = 0; c1 < 2; ++c1) {
          double w = (c1 ? e[0] : 1.0 - e[0]) * (c2 ? e[1] : 1.0 - e[1]);
          if (g->ndim == 3) w = w * (c3 ? e[2] : 1.0 - e[2]);
          add_to(g, rho, i[0] + c1, i[1] + c2, i[2] + c3, q * w / dvol);
        }
  }
}

/* ------------------------------------------------------------------------ */
/* binomial smoothing (nl_smooth: smooth_level passes per direction, weights   */
/* swfj per pass, normalised by their sum; periodic)                          */
/* ------------------------------------------------------------------------ */

static void smooth_pass(const ora_grid* g, double* f, int d, const double w[3], double* tmp) {
  long nx = g->nx[0], ny = g->nx[1], nz = g->nx[2];
  double ws = w[0] + w[1] + w[2];
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long s[3] = {i, j, k};
        long lo[3] = {i, j, k}, hi[3] = {i, j, k};
        lo[d] -= 1;
        hi[d] += 1;
        tmp[at(g, s[0], s[1], s[2])] =
            (w[0] * rd(g, f, lo[0], lo[1], lo[2]) + w[1] * f[at(g, i, j, k)] + w[2] * rd(g, f, hi[0], hi[1], hi[2])) / ws;
      }
  memcpy(f, tmp, sizeof(double) * (size_t)(nx * ny * nz));
}

void ora_smooth(const ora_grid* g, double* f) {
  long n = (long)g->nx[0] * g->nx[1] * g->nx[2];
  double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
  for (int d = 0; d < g->ndim; ++d)
    for (int pass = 0; pass < g->smooth_level[d]; ++pass) smooth_pass(g, f, d, g->smooth_w[d][pass], tmp);
  free(tmp);
}

/* ------------------------------------------------------------------------ */
/* field solve: eqs. "2d-field-solve-b-part1", "-e", "-b-part2" and the 3D    */
/* extension (x3 derivatives added); the printed j1 of the E3 line is read as j3 */
/* ------------------------------------------------------------------------ */

static void advance_b_half(const ora_grid* g, double* const fld[6]) {
  double* E1 = fld[0]; double* E2 = fld[1]; double* E3 = fld[2];
  double* B1 = fld[3]; double* B2 = fld[4]; double* B3 = fld[5];
  double h = g->dt / 2.0;
  long nx = g->nx[0], ny = g->nx[1], nz = g->nx[2];
  int d3 = g->ndim == 3;
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long c = at(g, i, j, k);
        double dE3d2 = (E3[at(g, i, j + 1, k)] - E3[c]) / g->dx[1];
        double dE3d1 = (rd(g, E3, i + 1, j, k) - E3[c]) / g->dx[0];
        double dE2d1 = (rd(g, E2, i + 1, j, k) - E2[c]) / g->dx[0];
        double dE1d2 = (E1[at(g, i, j + 1, k)] - E1[c]) / g->dx[1];
        double dE2d3 = d3 ? (E2[at(g, i, j, k + 1)] - E2[c]) / g->dx[2] : 0.0;
        double dE1d3 = d3 ? (E1[at(g, i, j, k + 1)] - E1[c]) / g->dx[2] : 0.0;
        B1[c] = B1[c] - h * (dE3d2 - dE2d3);
        B2[c] = B2[c] - h * (dE1d3 - dE3d1);
        B3[c] = B3[c] - h * (dE2d1 - dE1d2);
      }
}

static void advance_e(const ora_grid* g, double* const fld[6], double* const cur[3]) {
  double* E1 = fld[0]; double* E2 = fld[1]; double* E3 = fld[2];
  double* B1 = fld[3]; double* B2 = fld[4]; double* B3 = fld[5];
  double dt = g->dt;
  long nx = g->nx[0], ny = g->nx[1], nz = g->nx[2];
  int d3 = g->ndim == 3;
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long c = at(g, i, j, k);
        double dB3d2 = (B3[c] - B3[at(g, i, j - 1, k)]) / g->dx[1];
        /* below an open lower x1 boundary: the entering pulse's B (or 0) */
        const int lower = g->open_x1 && i == 0;
        double b3m = lower ? (g->inc_b3 ? g->inc_b3[k * ny + j] : 0.0) : rd(g, B3, i - 1, j, k);
        double b2m = lower ? (g->inc_b2 ? g->inc_b2[k * ny + j] : 0.0) : rd(g, B2, i - 1, j, k);
        double dB3d1 = (B3[c] - b3m) / g->dx[0];
        double dB2d1 = (B2[c] - b2m) / g->dx[0];
        double dB1d2 = (B1[c] - B1[at(g, i, j - 1, k)]) / g->dx[1];
        double dB2d3 = d3 ? (B2[c] - B2[at(g, i, j, k - 1)]) / g->dx[2] : 0.0;
        double dB1d3 = d3 ? (B1[c] - B1[at(g, i, j, k - 1)]) / g->dx[2] : 0.0;
        E1[c] = E1[c] + dt * (dB3d2 - dB2d3) - dt * cur[0][c];
        E2[c] = E2[c] + dt * (dB1d3 - dB3d1) - dt * cur[1][c];
        E3[c] = E3[c] + dt * (dB2d1 - dB1d2) - dt * cur[2][c];
      }
}

void ora_field_solve(const ora_grid* g, double* const fld[6], double* const cur[3]) {
  advance_b_half(g, fld);   /* B^n     -> B^{n+1/2} with E^n     */
  advance_e(g, fld, cur);   /* E^n     -> E^{n+1}   with B^{n+1/2}, j^{n+1/2} */
  advance_b_half(g, fld);   /* B^{n+1/2} -> B^{n+1} with E^{n+1} */
}

/* ------------------------------------------------------------------------ */
/* one particle: gather + push + move (no deposit)                            */
/* ------------------------------------------------------------------------ */

void ora_advance_particle(const ora_grid* g, double* const fld[6], double rqm, double x[3], double u[3]) {
  double eb[6];
  ora_gather(g, fld, x, eb);
  ora_boris(u, eb, eb + 3, rqm, g->dt);
  ora_move(g, x, u);
}

void ora_advance_particles(const ora_grid* g, double* const fld[6], double rqm, long long n, double* x,
                           double* u, int wrap) {
  for (long long p = 0; p < n; ++p) {
    ora_advance_particle(g, fld, rqm, x + 3 * p, u + 3 * p);
    if (wrap) ora_wrap(g, x + 3 * p);
  }
}

/* ------------------------------------------------------------------------ */
/* whole step                                                                 */
/* ------------------------------------------------------------------------ */

void ora_particle_phase(const ora_grid* g, double* const fld[6], double* cur[3], const ora_species* sp, int nsp) {
  long n = (long)g->nx[0] * g->nx[1] * g->nx[2];
  for (int c = 0; c < 3; ++c) memset(cur[c], 0, sizeof(double) * (size_t)n);
  for (int s = 0; s < nsp; ++s) {
    for (long long p = 0; p < sp[s].n; ++p) {
      double* x = sp[s].x + 3 * p;
      double* u = sp[s].u + 3 * p;
      double xold[3] = {x[0], x[1], x[2]};
      ora_advance_particle(g, fld, sp[s].rqm, x, u);
      if (g->isis)
        ora_deposit_isis(g, cur, xold, x, u[2] / ora_gamma(u), sp[s].w ? sp[s].q * sp[s].w[p] : sp[s].q);
      else
        ora_deposit_vb(g, cur, xold, x, u[2] / ora_gamma(u), sp[s].w ? sp[s].q * sp[s].w[p] : sp[s].q);
      ora_wrap(g, x);
    }
  }
}

void ora_step(const ora_grid* g, double* const fld[6], double* cur[3], const ora_species* sp, int nsp,
              int nsteps) {
  for (int it = 0; it < nsteps; ++it) {
    ora_particle_phase(g, fld, cur, sp, nsp);
    for (int c = 0; c < 3; ++c) ora_smooth(g, cur[c]);
    ora_field_solve(g, fld, cur);
  }
}

/* ------------------------------------------------------------------------ */
/* diagnostics (FP64)                                                         */
/* ------------------------------------------------------------------------ */

/* rho of all species at the nodes plus the fixed background */
void ora_rho(const ora_grid* g, const ora_species* sp, int nsp, double* rho) {
  long n = (long)g->nx[0] * g->nx[1] * g->nx[2];
  for (long c = 0; c < n; ++c) rho[c] = g->rho_bg;
  for (int s = 0; s < nsp; ++s) ora_deposit_rho_w(g, rho, sp[s].x, sp[s].w, sp[s].n, sp[s].q);
}

/* max over nodes of |div E - rho|, div E by backward differences of the staggered E */
double ora_gauss_residual(const ora_grid* g, double* const fld[6], const double* rho) {
  long nx = g->nx[0], ny = g->nx[1], nz = g->nx[2];
  int d3 = g->ndim == 3;
  double r = 0.0;
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j)
      for (long i = 0; i < nx; ++i) {
        long c = at(g, i, j, k);
        double div = (fld[0][c] - rd(g, fld[0], i - 1, j, k)) / g->dx[0] +
                     (fld[1][c] - fld[1][at(g, i, j - 1, k)]) / g->dx[1];
        if (d3) div = div + (fld[2][c] - fld[2][at(g, i, j, k - 1)]) / g->dx[2];
        double e = fabs(div - rho[c]);
        if (e > r) r = e;
      }
  return r;
}

/* (1/2) sum (E^2 + B^2) dV over every grid value of the six components */
double ora_field_energy(const ora_grid* g, double* const fld[6]) {
  long n = (long)g->nx[0] * g->nx[1] * g->nx[2];
  double s = 0.0;
  for (int c = 0; c < 6; ++c)
    for (long m = 0; m < n; ++m) s = s + fld[c][m] * fld[c][m];
  return 0.5 * s * cell_volume(g);
}

/* sum of m_p (gamma - 1) with macroparticle mass m_p = q * rqm */
double ora_kinetic_energy(const ora_species* sp, int nsp) {
  double s = 0.0;
  for (int k = 0; k < nsp; ++k)
    for (long long p = 0; p < sp[k].n; ++p)
      s = s + (sp[k].w ? sp[k].q * sp[k].w[p] : sp[k].q) * sp[k].rqm * (ora_gamma(sp[k].u + 3 * p) - 1.0);
  return s;
}

/* Initial E1 from the discrete Gauss law along x1, column by column:
 * E1(i+1/2) - E1(i-1/2) = dx1 rho(i), with zero mean E1 per column.  Exact when
 * rho depends only on x1 within each column's neighbourhood (E2 = E3 = 0). */
void ora_init_e_gauss_x1(const ora_grid* g, const double* rho, double* E1) {
  long nx = g->nx[0], ny = g->nx[1], nz = g->nx[2];
  for (long k = 0; k < nz; ++k)
    for (long j = 0; j < ny; ++j) {
      double run = 0.0, mean = 0.0;
      for (long i = 0; i < nx; ++i) {
        run = run + g->dx[0] * rho[at(g, i, j, k)];
        E1[at(g, i, j, k)] = run;
        mean = mean + run;
      }
      mean = mean / (double)nx;
      for (long i = 0; i < nx; ++i) E1[at(g, i, j, k)] = E1[at(g, i, j, k)] - mean;
    }
}

/* ------------------------------------------------------------------------ */
/* tile binning (not in the paper; the order a tile-sorted particle store     */
/* must reproduce): tile id of each particle's cell, counts, stable order     */
/* ------------------------------------------------------------------------ */

void ora_tile_bin(const ora_grid* g, const int tile[3], long long n, const double* x, long long* tile_id,
                  long long* counts, long long* order) {
  long nt[3] = {1, 1, 1};
  for (int d = 0; d < g->ndim; ++d) nt[d] = g->nx[d] / tile[d];
  long ntiles = nt[0] * nt[1] * nt[2];
  for (long t = 0; t < ntiles; ++t) counts[t] = 0;
  for (long long p = 0; p < n; ++p) {
    long c[3] = {0, 0, 0};
    for (int d = 0; d < g->ndim; ++d) {
      c[d] = wrapi((long)floor((x[3 * p + d] - g->xmin[d]) / g->dx[d]), g->nx[d]);
    }
    long t = ((c[2] / tile[2]) * nt[1] + c[1] / tile[1]) * nt[0] + c[0] / tile[0];
    tile_id[p] = t;
    counts[t] += 1;
  }
  long long* start = (long long*)malloc(sizeof(long long) * (size_t)ntiles);
  long long run = 0;
  for (long t = 0; t < ntiles; ++t) {
    start[t] = run;
    run += counts[t];
  }
  for (long long p = 0; p < n; ++p) order[start[tile_id[p]]++] = p;
  free(start);
}
