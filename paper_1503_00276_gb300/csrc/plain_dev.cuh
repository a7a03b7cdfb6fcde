// plain_dev.cuh -- FP64 device helpers of the "plain" particle forms (Cartesian
// and r-z): Yee-staggered linear gather, relativistic Boris rotation and the
// Villasenor-Buneman current of a straight path.  Each including translation
// unit gets its own copy (internal linkage); they are built without
// multiply-add contraction so that every FP64 operation rounds as written.
#pragma once

#include "kernels.h"

namespace picgb {
namespace {

struct F6 {
  const double* c[6];
};
struct J3 {
  double* c[3];
};

// Yee staggering of E1,E2,E3,B1,B2,B3 in cell units (read off the difference
// stencils of the field equations).
__constant__ double kStag[6][3] = {{0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
                                    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};

// Linear weighting of one component from the nearest 2^NDIM points of its own
// lattice (eq. 2d-field-weighting-e3 and its 3D extension).
template <int NDIM>
__device__ inline double interp(const Layout& L, const PushConst& C, const double* F, int comp, const double x[3]) {
  int i[3] = {0, 0, 0};
  double e[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    double g = (x[d] - C.xmin[d]) / C.dx[d] - kStag[comp][d];
    double fl = floor(g);
    i[d] = (int)fl;
    e[d] = g - fl;
  }
  if (NDIM == 2) {
    double lo = (1.0 - e[1]) * F[L.idx(i[0], i[1], 0)] + e[1] * F[L.idx(i[0], i[1] + 1, 0)];
    double hi = (1.0 - e[1]) * F[L.idx(i[0] + 1, i[1], 0)] + e[1] * F[L.idx(i[0] + 1, i[1] + 1, 0)];
    return (1.0 - e[0]) * lo + e[0] * hi;
  }
  double acc = 0.0;
#pragma unroll
  for (int c3 = 0; c3 < 2; ++c3)
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
      for (int c1 = 0; c1 < 2; ++c1) {
        double w = (c1 ? e[0] : 1.0 - e[0]) * (c2 ? e[1] : 1.0 - e[1]) * (c3 ? e[2] : 1.0 - e[2]);
        acc = acc + w * F[L.idx(i[0] + c1, i[1] + c2, i[2] + c3)];
      }
  return acc;
}

__device__ inline void cross(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Relativistic Boris push (eq. momentum-update, read as the standard rotation).
__device__ inline void boris(double u[3], const double e[3], const double b[3], double rqm, double dt) {
  double alpha = dt / (2.0 * rqm);
  double p1[3], p2[3], t[3], s[3], c[3];
  for (int d = 0; d < 3; ++d) p1[d] = u[d] + alpha * e[d];
  double gam = sqrt(1.0 + p1[0] * p1[0] + p1[1] * p1[1] + p1[2] * p1[2]);
  for (int d = 0; d < 3; ++d) t[d] = alpha * b[d] / gam;
  cross(p1, t, c);
  for (int d = 0; d < 3; ++d) p2[d] = p1[d] + c[d];
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int d = 0; d < 3; ++d) s[d] = 2.0 * t[d] / (1.0 + t2);
  cross(p2, s, c);
  for (int d = 0; d < 3; ++d) u[d] = p1[d] + c[d] + alpha * e[d];
}

// Villasenor-Buneman current of one straight in-cell segment, closed form:
// for a move of length D_d (cell units) the flux through face cell_d+1/2 is
// shared among the transverse nodes with the path-averaged linear weights,
// i.e. the midpoint weights plus the covariance term D_t1 D_t2 / 12.
template <int NDIM>
__device__ inline void deposit_segment(const Layout& L, const PushConst& C, J3 J, const int cell[3],
                                       const double a[3], const double b[3], double v3frac, double q,
                                       bool only_j3 = false) {
  double dl[3], m[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dl[d] = b[d] - a[d];
    m[d] = 0.5 * (a[d] + b[d]);
  }
  if (NDIM == 2) {
    if (!only_j3) {
    double a1 = q * dl[0] * C.dx[0] / (C.dt * C.dvol);
    double a2 = q * dl[1] * C.dx[1] / (C.dt * C.dvol);
    atomicAdd(&J.c[0][L.idx(cell[0], cell[1], 0)], a1 * (1.0 - m[1]));
    atomicAdd(&J.c[0][L.idx(cell[0], cell[1] + 1, 0)], a1 * m[1]);
    atomicAdd(&J.c[1][L.idx(cell[0], cell[1], 0)], a2 * (1.0 - m[0]));
    atomicAdd(&J.c[1][L.idx(cell[0] + 1, cell[1], 0)], a2 * m[0]);
    }
    double a3 = q * v3frac / C.dvol;
    double cv = dl[0] * dl[1] / 12.0;
    atomicAdd(&J.c[2][L.idx(cell[0], cell[1], 0)], a3 * ((1.0 - m[0]) * (1.0 - m[1]) + cv));
    atomicAdd(&J.c[2][L.idx(cell[0] + 1, cell[1], 0)], a3 * (m[0] * (1.0 - m[1]) - cv));
    atomicAdd(&J.c[2][L.idx(cell[0], cell[1] + 1, 0)], a3 * ((1.0 - m[0]) * m[1] - cv));
    atomicAdd(&J.c[2][L.idx(cell[0] + 1, cell[1] + 1, 0)], a3 * (m[0] * m[1] + cv));
    return;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    double amp = q * dl[d] * C.dx[d] / (C.dt * C.dvol);
    double cv = dl[t1] * dl[t2] / 12.0;
    int id[3] = {cell[0], cell[1], cell[2]};
    atomicAdd(&J.c[d][L.idx(id[0], id[1], id[2])], amp * ((1.0 - m[t1]) * (1.0 - m[t2]) + cv));
    id[t1] += 1;
    atomicAdd(&J.c[d][L.idx(id[0], id[1], id[2])], amp * (m[t1] * (1.0 - m[t2]) - cv));
    id[t2] += 1;
    atomicAdd(&J.c[d][L.idx(id[0], id[1], id[2])], amp * (m[t1] * m[t2] + cv));
    id[t1] -= 1;
    atomicAdd(&J.c[d][L.idx(id[0], id[1], id[2])], amp * ((1.0 - m[t1]) * m[t2] - cv));
  }
}

// Split x_old -> x_new (global, unwrapped) at the faces it crosses (at most one
// per direction) and deposit each in-cell piece.
template <int NDIM>
__device__ inline void deposit_path(const Layout& L, const PushConst& C, J3 J, const double xo[3],
                                    const double xn[3], double v3, double q, bool only_j3 = false) {
  int i0[3] = {0, 0, 0};
  double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
  const int nn[3] = {L.nx, L.ny, L.nz};
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    double go = (xo[d] - C.xmin[d]) / C.dx[d];
    double gn = (xn[d] - C.xmin[d]) / C.dx[d];
    double fl = floor(go);
    int ic = (int)fl;
    a[d] = go - fl;
    b[d] = gn - fl;
    if (ic >= nn[d]) ic -= nn[d];  // x just below xmax rounding up to the last face
    i0[d] = ic;
  }
  double tc[3];
  int dc[3], sc[3], nc = 0;
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    if (b[d] < 0.0) {
      tc[nc] = (0.0 - a[d]) / (b[d] - a[d]);
      dc[nc] = d;
      sc[nc] = -1;
      ++nc;
    } else if (b[d] >= 1.0) {
      tc[nc] = (1.0 - a[d]) / (b[d] - a[d]);
      dc[nc] = d;
      sc[nc] = 1;
      ++nc;
    }
  }
  for (int m = 1; m < nc; ++m)
    for (int r = m; r > 0 && tc[r] < tc[r - 1]; --r) {
      double tt = tc[r];
      tc[r] = tc[r - 1];
      tc[r - 1] = tt;
      int td = dc[r];
      dc[r] = dc[r - 1];
      dc[r - 1] = td;
      int ts = sc[r];
      sc[r] = sc[r - 1];
      sc[r - 1] = ts;
    }
  int off[3] = {0, 0, 0};
  double p0[3] = {a[0], a[1], a[2]};
  double t0 = 0.0;
  for (int m = 0; m <= nc; ++m) {
    double t1 = m < nc ? tc[m] : 1.0;
    double p1[3];
    for (int d = 0; d < 3; ++d) p1[d] = m < nc ? a[d] + t1 * (b[d] - a[d]) : b[d];
    if (m < nc) p1[dc[m]] = sc[m] > 0 ? 1.0 + (double)off[dc[m]] : (double)off[dc[m]];
    int cell[3];
    double la[3], lb[3];
    for (int d = 0; d < 3; ++d) {
      cell[d] = i0[d] + off[d];
      la[d] = p0[d] - (double)off[d];
      lb[d] = p1[d] - (double)off[d];
    }
    deposit_segment<NDIM>(L, C, J, cell, la, lb, v3 * (t1 - t0), q, only_j3);
    if (m < nc) off[dc[m]] += sc[m];
    for (int d = 0; d < 3; ++d) p0[d] = p1[d];
    t0 = t1;
  }
}

}  // namespace
}  // namespace picgb
