// k_cyl.cu -- the 2D cylindrically symmetric (r-z) mode: the FP64 plain
// particle kernels, and the field, current and diagnostic kernels of both
// forms (templated on the stored precision; the FP32 form's particles move in
// the tile kernel's r-z instantiation).
//
// Thesis ch. 3, the 2D cylindrically symmetric algorithms: the Cartesian 2D
// grid with x1 -> z and x2 -> r (E1,E2,E3 -> Ez,Er,Etheta; B and j likewise),
// the axis through the middle of the first cell (node row j at r = (j - 1/2)
// dr, half row j + 1/2 at r = j dr), a conducting wall at node row nr.
//   * push: the Cartesian gather and Boris update of (pz, pr, ptheta); a
//     "pseudo" 3D move from (z, r, 0), then a rotation back into the r-z plane
//     (eqs. 2d-cyl-position-update-1..3), ptheta from the conservation of the
//     ring's angular momentum;
//   * deposit: the Cartesian 2D current deposit of the ring's current I, then
//     j = I / V(r) with V = r dr dz per radian at each component's radius, the
//     row below the axis folded back with the axial parity;
//   * field solve: the Cartesian stencils with the radius inside the
//     r-derivatives of the z components (eq. 2d-field-solve-cyl; the second
//     B_Theta of the printed Ez update is read as B_Theta,i1,i2-1), Bz on the
//     axis from the integral form of Faraday's law (eq.
//     2d-field-solve-cyl-b1-axis), parity rows at the axis.
// Particles are rings: x[1] = r >= 0 (FP64 form: r = -1 once absorbed at the
// wall), charge q * w per radian with w = (own weight) * r at loading.
// Compiled without multiply-add contraction, like the Cartesian plain form.
#include <algorithm>

#include "plain_dev.cuh"

namespace picgb {

namespace {

__device__ inline double r_node(const CylConst& K, int j) { return ((double)j - 0.5) * K.dr; }
__device__ inline double r_half(const CylConst& K, int j) { return (double)j * K.dr; }

// the six field planes / three current planes in the stored precision
template <typename T>
struct FT6 {
  T* c[6];
};
template <typename T>
struct JT3 {
  T* c[3];
};

// Lattice points of the first cell below the axis reflected to -r; ring
// weight w = (own weight, 1 without one) * r.  An explicit position below the
// axis is an error.
__global__ void k_cyl_load_fix(long long n, double* r, double* w, int lattice, int has_w0, int* status) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double v = r[k];
  if (v < 0.0) {
    if (!lattice) {
      atomicOr(status, ST_BADCELL);
      return;
    }
    v = -v;
    r[k] = v;
  }
  w[k] = (has_w0 ? w[k] : 1.0) * v;
}

__global__ void __launch_bounds__(256) k_cyl_push(Layout L, PushConst C, CylConst K, Plain p, F6 F, J3 J,
                                                  int* status) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  const double r = p.x[1][n];
  if (r < 0.0) return;  // absorbed at the wall in an earlier step
  double x[3] = {p.x[0][n], r, 0.0};
  double u[3] = {p.u[0][n], p.u[1][n], p.u[2][n]};
  double eb[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) eb[c] = interp<2>(L, C, F.c[c], c, x) + (c < 3 ? C.e0[c] : C.b0[c - 3]);
  boris(u, eb, eb + 3, C.rqm, C.dt);
  const double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  // eq. 2d-cyl-position-update-1: the move in 3D Cartesian space from (z, r, 0)
  const double zn = x[0] + C.dt * u[0] / gam;
  const double x2 = r + C.dt * u[1] / gam;
  const double x3 = C.dt * u[2] / gam;
  const double rn = hypot(x2, x3);  // eq. 2d-cyl-position-update-2
  if (!(isfinite(zn) && isfinite(rn) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]))) {
    atomicOr(status, ST_NONFINITE);
    return;
  }
  const double qp = C.q * p.w[n];
  const double v3 = u[2] / gam;  // the out-of-plane current uses ptheta before the rotation
  const double xo[3] = {x[0], r, 0.0};
  if (rn >= K.rmax) {  // absorbed: the path up to the wall, then the slot is emptied
    const double t = (K.rmax - r) / (rn - r);
    const double xc[3] = {x[0] + t * (zn - x[0]), K.rmax, 0.0};
    deposit_path<2>(L, C, J, xo, xc, v3 * t, qp);
    p.x[1][n] = -1.0;
    p.u[0][n] = 0.0;
    p.u[1][n] = 0.0;
    p.u[2][n] = 0.0;
    return;
  }
  const double xn[3] = {zn, rn, 0.0};
  deposit_path<2>(L, C, J, xo, xn, v3, qp);
  // eq. 2d-cyl-position-update-3: momenta in the rotated frame, ptheta from
  // r^n ptheta = r^{n+1} ptheta'
  double pr, pt;
  if (rn > 0.0) {
    pr = (u[1] * x2 + u[2] * x3) / rn;
    pt = u[2] * r / rn;
  } else {
    pr = hypot(u[1], u[2]);
    pt = 0.0;
  }
  double z = zn;
  const double zmax = C.xmin[0] + C.L[0];
  while (z >= zmax) z = z - C.L[0];
  while (z < C.xmin[0]) z = z + C.L[0];
  if (z >= zmax) z = C.xmin[0];
  p.x[0][n] = z;
  p.x[1][n] = rn;
  p.u[0][n] = u[0];
  p.u[1][n] = pr;
  p.u[2][n] = pt;
}

// Deposited current (Cartesian area units) to densities, one thread per (z
// column, node row 1 .. nr-1): the periodic guard columns folded in, the row
// below the axis folded onto row 1 with the parity sign (jz +, jtheta -; jr
// on the axis is 0), then divided by the radius of each component (node rows
// for jz, jtheta, half rows for jr).  The row-1 thread of a column is the only
// reader of its mirror row and clears it afterwards; the row nr-1 thread
// clears the wall row.
template <typename T>
__device__ inline T fold_z(const Layout& L, const CylConst& K, const T* A, int i, int j) {
  T v = A[L.idx(i, j, 0)];
  if (i == K.nz - 1) v = v + A[L.idx(-1, j, 0)];
  if (i < 3) v = v + A[L.idx(K.nz + i, j, 0)];
  return v;
}

template <typename T>
__global__ void k_cyl_current(Layout L, CylConst K, JT3<T> J) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)K.nz * (K.nr - 1)) return;
  const int i = (int)(q % K.nz), j = 1 + (int)(q / K.nz);
  for (int c = 0; c < 3; ++c) {
    T* A = J.c[c];
    T v = fold_z(L, K, A, i, j);
    if (j == 1) {
      const T v0 = fold_z(L, K, A, i, 0);
      v = c == 0 ? v + v0 : (c == 2 ? v - v0 : v);
      A[L.idx(i, 0, 0)] = T(0);
    }
    A[L.idx(i, j, 0)] = v / (T)(c == 1 ? r_half(K, j) : r_node(K, j));
    if (j == K.nr - 1) A[L.idx(i, K.nr, 0)] = T(0);
  }
}

// B advanced by h = dt/2 from E, one thread per (i, j), rows 0 .. nr-1 (eqs.
// 2d-field-solve-b-part1/-part2 with 2d-field-solve-cyl for Bz and the axis
// rule for Bz at j = 0: the loop of radius dr/2 about the axis encloses the
// disc pi (dr/2)^2 and runs along Etheta at r = dr/2, hence the factor 4).
// Arithmetic in the stored precision T.
template <typename T>
__global__ void k_cyl_b_half(Layout L, CylConst K, FT6<T> F, T h) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)K.nz * K.nr) return;
  const int i = (int)(q % K.nz), j = (int)(q / K.nz);
  const int ip = i + 1 == K.nz ? 0 : i + 1;
  const T* Ez = F.c[0];
  const T* Er = F.c[1];
  const T* Et = F.c[2];
  T* Bz = F.c[3];
  T* Br = F.c[4];
  T* Bt = F.c[5];
  const T dz = (T)K.dz, dr = (T)K.dr;
  const long long c = L.idx(i, j, 0);
  if (j == 0) {
    Bz[c] = Bz[c] - h * T(4) * Et[L.idx(i, 1, 0)] / dr;
    return;  // Br_0 mirrors row 1, Btheta_0 = 0 on the axis
  }
  Bz[c] = Bz[c] - h * ((T)r_node(K, j + 1) * Et[L.idx(i, j + 1, 0)] - (T)r_node(K, j) * Et[c]) / ((T)r_half(K, j) * dr);
  Br[c] = Br[c] + h * ((Et[L.idx(ip, j, 0)] - Et[c]) / dz);
  Bt[c] = Bt[c] - h * ((Er[L.idx(ip, j, 0)] - Er[c]) / dz - (Ez[L.idx(i, j + 1, 0)] - Ez[c]) / dr);
}

// E advanced by dt from B and j, rows 1 .. nr-1 (eq. 2d-field-solve-e with
// 2d-field-solve-cyl for Ez).
template <typename T>
__global__ void k_cyl_e(Layout L, CylConst K, FT6<T> F, JT3<T> J, T dt) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)K.nz * (K.nr - 1)) return;
  const int i = (int)(q % K.nz), j = 1 + (int)(q / K.nz);
  const int im = i == 0 ? K.nz - 1 : i - 1;
  T* Ez = F.c[0];
  T* Er = F.c[1];
  T* Et = F.c[2];
  const T* Bz = F.c[3];
  const T* Br = F.c[4];
  const T* Bt = F.c[5];
  const T dz = (T)K.dz, dr = (T)K.dr;
  const long long c = L.idx(i, j, 0), cd = L.idx(i, j - 1, 0), cm = L.idx(im, j, 0);
  Ez[c] = Ez[c] + dt * (((T)r_half(K, j) * Bt[c] - (T)r_half(K, j - 1) * Bt[cd]) / ((T)r_node(K, j) * dr) - J.c[0][c]);
  Er[c] = Er[c] + dt * (-((Bt[c] - Bt[cm]) / dz) - J.c[1][c]);
  Et[c] = Et[c] + dt * ((Br[c] - Br[cm]) / dz - (Bz[c] - Bz[cd]) / dr - J.c[2][c]);
}

// Axis and wall rows, one thread per z column: Ez_0 = Ez_1, Etheta_0 =
// -Etheta_1, Br_0 = -Br_1 (the mirror row at r = -dr/2), Er_0 = Btheta_0 = 0
// (odd, on the axis); at the wall (row nr) and beyond every field is 0.
template <typename T>
__global__ void k_cyl_rows(Layout L, CylConst K, FT6<T> F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K.nz) return;
  T* const* f = F.c;
  const long long r0 = L.idx(i, 0, 0), r1 = L.idx(i, 1, 0);
  f[0][r0] = f[0][r1];
  f[2][r0] = -f[2][r1];
  f[4][r0] = -f[4][r1];
  f[1][r0] = T(0);
  f[5][r0] = T(0);
  for (int j = K.nr; j <= K.nr + 1; ++j)
    for (int c = 0; c < 6; ++c) f[c][L.idx(i, j, 0)] = T(0);
}

// Periodic z guard columns (-1, nz .. nz+2) of rows 0 .. nr+1, for the gather.
template <typename T>
__global__ void k_cyl_zguards(Layout L, CylConst K, FT6<T> F) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > K.nr + 1) return;
  for (int c = 0; c < 6; ++c) {
    T* f = F.c[c];
    f[L.idx(-1, j, 0)] = f[L.idx(K.nz - 1, j, 0)];
    for (int g = 0; g < 3; ++g) f[L.idx(K.nz + g, j, 0)] = f[L.idx(g, j, 0)];
  }
}

// ring charge q w with the linear weights on the node rows (charge, not yet
// a density); absorbed particles skipped
__global__ void k_cyl_rho(Layout L, PushConst C, Plain p, double* rho) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  const double r = p.x[1][n];
  if (r < 0.0) return;
  const double g1 = (p.x[0][n] - C.xmin[0]) / C.dx[0], g2 = (r - C.xmin[1]) / C.dx[1];
  const double f1 = floor(g1), f2 = floor(g2);
  const int i0 = (int)f1, j0 = (int)f2;
  const double e1 = g1 - f1, e2 = g2 - f2;
  const double q = C.q * p.w[n];
  for (int c2 = 0; c2 < 2; ++c2)
    for (int c1 = 0; c1 < 2; ++c1)
      atomicAdd(&rho[L.idx(i0 + c1, j0 + c2, 0)], q * ((c1 ? e1 : 1.0 - e1) * (c2 ? e2 : 1.0 - e2)));
}

// charge to density, one thread per (z column, node row 1 .. nr-1): guards
// folded, row 0 folded onto row 1 (even), divided by V = r_j * area (area =
// dz dr for charges, 1 for a sum already per dz dr); the mirror and wall rows
// cleared by the row-1 and row nr-1 threads (their only readers)
__global__ void k_cyl_rho_finish(Layout L, CylConst K, double* rho, double area) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)K.nz * (K.nr - 1)) return;
  const int i = (int)(q % K.nz), j = 1 + (int)(q / K.nz);
  double v = fold_z(L, K, rho, i, j);
  if (j == 1) {
    v = v + fold_z(L, K, rho, i, 0);
    rho[L.idx(i, 0, 0)] = 0.0;
  }
  rho[L.idx(i, j, 0)] = v / (r_node(K, j) * area);
  if (j == K.nr - 1) rho[L.idx(i, K.nr, 0)] = 0.0;
}

__device__ inline double cyl_block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;  // valid in thread 0
}

__device__ inline double cyl_block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, red[w]);
  return s;
}

// Field energy sum F^2 V (per radian, halved and times 2 pi by the caller) and
// the Gauss maxima over the node rows 1 .. nr-1 with the cylindrical
// divergence (z difference plus (1/r_j) d(r Er)/dr).  Volumes: r dr dz at
// each component's radius, the axis disc (dr/2)^2/2 dz for the half row on
// the axis; the mirror row and the wall row are left out.
template <typename T>
__global__ void __launch_bounds__(256) k_cyl_diag_fields(Layout L, CylConst K, FT6<T> F, const double* rho,
                                                         double rho_bg, Diag64* acc) {
  __shared__ double red[32];
  const long long ncell = (long long)K.nz * K.nr;
  double s = 0.0, gm = 0.0, rm = 0.0, pm = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % K.nz), j = (int)(q / K.nz);
    const long long c = L.idx(i, j, 0);
    const double vh = j == 0 ? 0.125 * K.dr * K.dr * K.dz : r_half(K, j) * K.dr * K.dz;
    const double f1 = F.c[1][c], f3 = F.c[3][c], f5 = F.c[5][c];
    s = s + (f1 * f1 + f3 * f3 + f5 * f5) * vh;
    if (j == 0) continue;
    const double vn = r_node(K, j) * K.dr * K.dz;
    const double f0 = F.c[0][c], f2 = F.c[2][c], f4 = F.c[4][c];
    s = s + (f0 * f0 + f2 * f2 + f4 * f4) * vn;
    const int im = i == 0 ? K.nz - 1 : i - 1;
    const double div = (f0 - (double)F.c[0][L.idx(im, j, 0)]) / K.dz +
                       (r_half(K, j) * f1 - r_half(K, j - 1) * (double)F.c[1][L.idx(i, j - 1, 0)]) /
                           (r_node(K, j) * K.dr);
    const double rt = rho[c] + rho_bg;
    gm = fmax(gm, fabs(div - rt));
    rm = fmax(rm, fabs(rt));
    pm = fmax(pm, fabs(rho[c]));
  }
  s = cyl_block_sum(s, red);
  gm = cyl_block_max(gm, red);
  rm = cyl_block_max(rm, red);
  pm = cyl_block_max(pm, red);
  if (threadIdx.x == 0) {
    atomicAdd(&acc->field_energy, s);
    atomic_max_nonneg(&acc->gauss_max, gm);
    atomic_max_nonneg(&acc->rho_max, rm);
    atomic_max_nonneg(&acc->rho_part_max, pm);
  }
}

// sum over live rings of q w rqm (gamma - 1) and q w (per radian)
__global__ void __launch_bounds__(256) k_cyl_kinetic(PushConst C, Plain p, Diag64* acc) {
  __shared__ double red[32];
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double ke = 0.0, qs = 0.0;
  if (n < p.n && p.x[1][n] >= 0.0) {
    const double a = p.u[0][n], b = p.u[1][n], c = p.u[2][n];
    const double qw = C.q * p.w[n];
    ke = qw * C.rqm * (sqrt(1.0 + (a * a + b * b + c * c)) - 1.0);
    qs = qw;
  }
  ke = cyl_block_sum(ke, red);
  qs = cyl_block_sum(qs, red);
  if (threadIdx.x == 0) {
    atomicAdd(&acc->kinetic_energy, ke);
    atomicAdd(&acc->total_charge, qs);
  }
}

F6 f6(double* const* f) { return F6{{f[0], f[1], f[2], f[3], f[4], f[5]}}; }
unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void cyl_load_fix(long long n, double* r, double* w, bool lattice, bool has_w0, int* status, cudaStream_t s) {
  if (n <= 0) return;
  k_cyl_load_fix<<<blocks_for(n), 256, 0, s>>>(n, r, w, lattice ? 1 : 0, has_w0 ? 1 : 0, status);
}

void cyl_push(const Layout& L, const PushConst& C, const CylConst& K, Plain p, double* const* f, double* const* j,
              int* status, cudaStream_t s) {
  if (p.n == 0) return;
  J3 J{{j[0], j[1], j[2]}};
  k_cyl_push<<<blocks_for(p.n), 256, 0, s>>>(L, C, K, p, f6(f), J, status);
}

template <typename T>
void cyl_current(const Layout& L, const CylConst& K, T* const* j, cudaStream_t s) {
  JT3<T> J{{j[0], j[1], j[2]}};
  k_cyl_current<T><<<blocks_for((long long)K.nz * (K.nr - 1)), 256, 0, s>>>(L, K, J);
}

template <typename T>
void cyl_bound(const Layout& L, const CylConst& K, T* const* f, bool zguards, cudaStream_t s) {
  FT6<T> F{{f[0], f[1], f[2], f[3], f[4], f[5]}};
  k_cyl_rows<T><<<blocks_for(K.nz), 256, 0, s>>>(L, K, F);
  if (zguards) k_cyl_zguards<T><<<blocks_for(K.nr + 2), 256, 0, s>>>(L, K, F);
}

template <typename T>
int cyl_field_step(const Layout& L, const CylConst& K, T* const* f, T* const* j, cudaStream_t s) {
  JT3<T> J{{j[0], j[1], j[2]}};
  FT6<T> F{{f[0], f[1], f[2], f[3], f[4], f[5]}};
  const long long nb = (long long)K.nz * K.nr, ne = (long long)K.nz * (K.nr - 1);
  const T h = (T)(0.5 * K.dt), dt = (T)K.dt;
  k_cyl_b_half<T><<<blocks_for(nb), 256, 0, s>>>(L, K, F, h);
  k_cyl_rows<T><<<blocks_for(K.nz), 256, 0, s>>>(L, K, F);
  k_cyl_e<T><<<blocks_for(ne), 256, 0, s>>>(L, K, F, J, dt);
  k_cyl_rows<T><<<blocks_for(K.nz), 256, 0, s>>>(L, K, F);
  k_cyl_b_half<T><<<blocks_for(nb), 256, 0, s>>>(L, K, F, h);
  k_cyl_rows<T><<<blocks_for(K.nz), 256, 0, s>>>(L, K, F);
  k_cyl_zguards<T><<<blocks_for(K.nr + 2), 256, 0, s>>>(L, K, F);
  return 7;
}

void cyl_rho(const Layout& L, const PushConst& C, const CylConst& K, Plain p, double* rho, cudaStream_t s) {
  if (p.n > 0) k_cyl_rho<<<blocks_for(p.n), 256, 0, s>>>(L, C, p, rho);
}

void cyl_rho_finish(const Layout& L, const CylConst& K, double* rho, double area, cudaStream_t s) {
  k_cyl_rho_finish<<<blocks_for((long long)K.nz * (K.nr - 1)), 256, 0, s>>>(L, K, rho, area);
}

template <typename T>
void cyl_diag(const Layout& L, const CylConst& K, T* const* f, const double* rho, double rho_bg, Diag64* acc,
              cudaStream_t s) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = ((long long)K.nz * K.nr + 255) / 256;
  const int blocks = (int)std::min<long long>(want, 8ll * sms);
  FT6<T> F{{f[0], f[1], f[2], f[3], f[4], f[5]}};
  k_cyl_diag_fields<T><<<blocks, 256, 0, s>>>(L, K, F, rho, rho_bg, acc);
}

#define PICGB_CYL_INST(T)                                                                                \
  template void cyl_current<T>(const Layout&, const CylConst&, T* const*, cudaStream_t);                 \
  template void cyl_bound<T>(const Layout&, const CylConst&, T* const*, bool, cudaStream_t);             \
  template int cyl_field_step<T>(const Layout&, const CylConst&, T* const*, T* const*, cudaStream_t);    \
  template void cyl_diag<T>(const Layout&, const CylConst&, T* const*, const double*, double, Diag64*,   \
                            cudaStream_t);
PICGB_CYL_INST(float)
PICGB_CYL_INST(double)
#undef PICGB_CYL_INST

void cyl_kinetic(const PushConst& C, Plain p, Diag64* acc, cudaStream_t s) {
  if (p.n > 0) k_cyl_kinetic<<<blocks_for(p.n), 256, 0, s>>>(C, p, acc);
}

}  // namespace picgb
