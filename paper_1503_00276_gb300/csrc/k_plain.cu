// k_plain.cu -- FP64 "plain" form of the particle step and the FP64 loaders.
//
// One thread per particle: global FP64 positions and momenta, fields gathered
// from global memory, current deposited with FP64 global atomics.  This is the
// reference GPU form that the FP32 tiled form is measured against.  Compiled
// without multiply-add contraction so that every FP64 operation rounds as
// written.
#include "kernels.h"
#include "plain_dev.cuh"

namespace picgb {

namespace {

// ISIS deposit (2D3V): the in-plane current of the whole straight path is the
// average of the two orders of orthogonal moves, not split at cell faces.  A
// move along x puts, through the J1 face of column i0 + d (d = -1, 0, 1), the
// part of the move inside that column -- the change of the linear charge
// weights it causes -- with the transverse weights of its fixed coordinate
// (y_a in one order, y_b in the other, averaged).  J3 is TRISTAN's: the time
// integral along the straight path.
__device__ inline double lin_w(double s) { return fmax(0.0, 1.0 - fabs(s)); }

__device__ inline void deposit_isis(const Layout& L, const PushConst& C, J3 J, const double xo[3],
                                    const double xn[3], double v3, double q) {
  int i0[2];
  double a[2], b[2];
  const int nn[2] = {L.nx, L.ny};
  for (int d = 0; d < 2; ++d) {
    double go = (xo[d] - C.xmin[d]) / C.dx[d];
    double gn = (xn[d] - C.xmin[d]) / C.dx[d];
    double fl = floor(go);
    int ic = (int)fl;
    a[d] = go - fl;
    b[d] = gn - fl;
    if (ic >= nn[d]) ic -= nn[d];
    i0[d] = ic;
  }
  double f[2][3], w[2][4];
  for (int d = 0; d < 2; ++d) {
    f[d][0] = fmin(b[d], 0.0);
    f[d][1] = fmin(fmax(b[d], 0.0), 1.0) - a[d];
    f[d][2] = fmax(b[d] - 1.0, 0.0);
    for (int m = 0; m < 4; ++m) w[d][m] = 0.5 * (lin_w(a[d] - (double)(m - 1)) + lin_w(b[d] - (double)(m - 1)));
  }
  const double c1 = q * C.dx[0] / (C.dt * C.dvol), c2 = q * C.dx[1] / (C.dt * C.dvol);
  for (int d = 0; d < 3; ++d)
    for (int m = 0; m < 4; ++m) {
      if (f[0][d] != 0.0 && w[1][m] != 0.0)
        atomicAdd(&J.c[0][L.idx(i0[0] + d - 1, i0[1] + m - 1, 0)], c1 * f[0][d] * w[1][m]);
      if (f[1][d] != 0.0 && w[0][m] != 0.0)
        atomicAdd(&J.c[1][L.idx(i0[0] + m - 1, i0[1] + d - 1, 0)], c2 * f[1][d] * w[0][m]);
    }
  deposit_path<2>(L, C, J, xo, xn, v3, q, true);
}

template <int NDIM>
__global__ void __launch_bounds__(256) k_plain_push(Layout L, PushConst C, Plain p, F6 F, J3 J, int* status) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  double x[3] = {p.x[0][n], p.x[1][n], NDIM == 3 ? p.x[2][n] : 0.0};
  double u[3] = {p.u[0][n], p.u[1][n], p.u[2][n]};
  double eb[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) eb[c] = interp<NDIM>(L, C, F.c[c], c, x) + (c < 3 ? C.e0[c] : C.b0[c - 3]);
  boris(u, eb, eb + 3, C.rqm, C.dt);
  double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double xo[3] = {x[0], x[1], x[2]};
#pragma unroll
  for (int d = 0; d < NDIM; ++d) x[d] = x[d] + C.dt * u[d] / gam;
  bool ok = isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) && isfinite(x[0]) && isfinite(x[1]) &&
            isfinite(x[2]);
  if (!ok) {
    atomicOr(status, ST_NONFINITE);
    return;
  }
  const double qp = p.w ? C.q * p.w[n] : C.q;  // charge of this particle (density profile)
  if (NDIM == 2 && C.isis)
    deposit_isis(L, C, J, xo, x, u[2] / gam, qp);
  else
    deposit_path<NDIM>(L, C, J, xo, x, u[2] / gam, qp);
  // periodic wrap
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    double xmax = C.xmin[d] + C.L[d];
    while (x[d] >= xmax) x[d] = x[d] - C.L[d];
    while (x[d] < C.xmin[d]) x[d] = x[d] + C.L[d];
    if (x[d] >= xmax) x[d] = C.xmin[d];
  }
  p.x[0][n] = x[0];
  p.x[1][n] = x[1];
  if (NDIM == 3) p.x[2][n] = x[2];
  p.u[0][n] = u[0];
  p.u[1][n] = u[1];
  p.u[2][n] = u[2];
}

template <int NDIM>
__global__ void k_plain_rho(Layout L, PushConst C, Plain p, double* rho) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  int i[3] = {0, 0, 0};
  double e[3] = {0, 0, 0};
  const int nn[3] = {L.nx, L.ny, L.nz};
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    double g = (p.x[d][n] - C.xmin[d]) / C.dx[d];
    double fl = floor(g);
    i[d] = (int)fl;
    if (i[d] >= nn[d]) i[d] -= nn[d];
    e[d] = g - fl;
  }
#pragma unroll
  for (int c3 = 0; c3 < (NDIM == 3 ? 2 : 1); ++c3)
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
      for (int c1 = 0; c1 < 2; ++c1) {
        double w = (c1 ? e[0] : 1.0 - e[0]) * (c2 ? e[1] : 1.0 - e[1]);
        if (NDIM == 3) w = w * (c3 ? e[2] : 1.0 - e[2]);
        atomicAdd(&rho[L.idx(i[0] + c1, i[1] + c2, i[2] + c3)], (p.w ? C.q * p.w[n] : C.q) * w / C.dvol);
      }
}

__global__ void k_plain_kinetic(PushConst C, Plain p, double* ke, double* qsum) {
  __shared__ double red[8];
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0, qn = 0.0;
  if (n < p.n) {
    double u0 = p.u[0][n], u1 = p.u[1][n], u2 = p.u[2][n];
    qn = p.w ? C.q * p.w[n] : C.q;
    v = qn * C.rqm * (sqrt(1.0 + u0 * u0 + u1 * u1 + u2 * u2) - 1.0);
  }
  __shared__ double redq[8];
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_down_sync(0xffffffffu, v, o);
    qn += __shfl_down_sync(0xffffffffu, qn, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = v;
    redq[threadIdx.x >> 5] = qn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, sq = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s += red[w];
      sq += redq[w];
    }
    atomicAdd(ke, s);
    atomicAdd(qsum, sq);
  }
}

// Lattice loader (nl_species num_par_x / vth / vfl): particle p is sub-lattice
// point s of cell c, p = c*ppc + s, both in x1-fastest order; position
// xmin + (cell + (s + 1/2)/npx) dx; u = vfl + vth * normal(seed, 3p + d).
__global__ void k_lattice(LatticeSpec S, long long first, long long count, double* x0, double* x1, double* x2,
                          double* u0, double* u1, double* u2, int* id) {
  double* x[3] = {x0, x1, x2};
  double* u[3] = {u0, u1, u2};
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  long long p = first + t;
  long long ppc = (long long)S.ppc[0] * S.ppc[1] * S.ppc[2];
  long long cell = p / ppc;
  long long sub = p - cell * ppc;
  long long ci[3], si[3];
  ci[0] = cell % S.nx[0];
  ci[1] = (cell / S.nx[0]) % S.nx[1];
  ci[2] = cell / ((long long)S.nx[0] * S.nx[1]);
  si[0] = sub % S.ppc[0];
  si[1] = (sub / S.ppc[0]) % S.ppc[1];
  si[2] = sub / ((long long)S.ppc[0] * S.ppc[1]);
  for (int d = 0; d < 3; ++d) {
    double v = 0.0;
    if (d < S.ndim) {
      double off = ((double)si[d] + 0.5) / (double)S.ppc[d];
      v = S.xmin[d] + ((double)ci[d] + off) * S.dx[d];
    }
    if (x[d]) x[d][t] = v;
  }
  for (int d = 0; d < 3; ++d) {
    double v = S.ufl[d];
    if (S.uth[d] != 0.0) v = S.ufl[d] + S.uth[d] * normal_dev(S.seed, 3ull * (unsigned long long)p + d);
    u[d][t] = v;
  }
  if (id) id[t] = (int)p;
}

}  // namespace

void plain_push(int ndim, const Layout& L, const PushConst& C, Plain p, double* const* f, double* const* j,
                int* status, cudaStream_t s) {
  if (p.n == 0) return;
  F6 F{{f[0], f[1], f[2], f[3], f[4], f[5]}};
  J3 J{{j[0], j[1], j[2]}};
  unsigned blocks = (unsigned)((p.n + 255) / 256);
  if (ndim == 2)
    k_plain_push<2><<<blocks, 256, 0, s>>>(L, C, p, F, J, status);
  else
    k_plain_push<3><<<blocks, 256, 0, s>>>(L, C, p, F, J, status);
}

void plain_rho(int ndim, const Layout& L, const PushConst& C, Plain p, double* rho, cudaStream_t s) {
  if (p.n == 0) return;
  unsigned blocks = (unsigned)((p.n + 255) / 256);
  if (ndim == 2)
    k_plain_rho<2><<<blocks, 256, 0, s>>>(L, C, p, rho);
  else
    k_plain_rho<3><<<blocks, 256, 0, s>>>(L, C, p, rho);
}

void plain_kinetic(const PushConst& C, Plain p, Diag64* acc, cudaStream_t s) {
  if (p.n == 0) return;
  unsigned blocks = (unsigned)((p.n + 255) / 256);
  k_plain_kinetic<<<blocks, 256, 0, s>>>(C, p, &acc->kinetic_energy, &acc->total_charge);
}

namespace {
// weight and keep flag of every loaded particle
__global__ void k_profile_keep(int ndim, ProfileDev P, long long n, const double* x0, const double* x1,
                               const double* x2, double* w, int* keep) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double x[3] = {x0[k], x1[k], ndim == 3 ? x2[k] : 0.0};
  const double v = profile_weight(P, x);
  w[k] = v;
  keep[k] = P.density * v > P.den_min ? 1 : 0;
}

// the kept particles, in order, to their compacted places
__global__ void k_profile_scatter(long long n, const int* keep, const long long* pos, const double* x0,
                                  const double* x1, const double* x2, const double* u0, const double* u1,
                                  const double* u2, const int* id, const double* w, double* dx0, double* dx1,
                                  double* dx2, double* du0, double* du1, double* du2, int* did, double* dw) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || !keep[k]) return;
  const long long j = pos[k];
  dx0[j] = x0[k];
  dx1[j] = x1[k];
  if (dx2) dx2[j] = x2[k];
  du0[j] = u0[k];
  du1[j] = u1[k];
  du2[j] = u2[k];
  if (did) did[j] = id[k];
  dw[j] = w[k];
}
}  // namespace

size_t profile_scratch_bytes(long long count) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  return al(8 * (size_t)count) + al(4 * (size_t)count) + al(8 * (size_t)count) + al(scan_scratch_bytes(count));
}

long long profile_compact(int ndim, const ProfileDev& P, long long count, double* const x[3], double* const u[3],
                          const int* id, double* const dx[3], double* const du[3], int* did, double* dw,
                          void* scratch, cudaStream_t s) {
  if (count <= 0) return 0;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  char* c = reinterpret_cast<char*>(scratch);
  double* w = reinterpret_cast<double*>(c);
  c += al(8 * (size_t)count);
  int* keep = reinterpret_cast<int*>(c);
  c += al(4 * (size_t)count);
  long long* pos = reinterpret_cast<long long*>(c);
  c += al(8 * (size_t)count);
  const unsigned blocks = (unsigned)((count + 255) / 256);
  k_profile_keep<<<blocks, 256, 0, s>>>(ndim, P, count, x[0], x[1], x[2], w, keep);
  exclusive_scan_i32(keep, pos, count, c, s);
  k_profile_scatter<<<blocks, 256, 0, s>>>(count, keep, pos, x[0], x[1], x[2], u[0], u[1], u[2], id, w, dx[0],
                                           dx[1], dx[2], du[0], du[1], du[2], did, dw);
  long long last_pos = 0;
  int last_keep = 0;
  cudaMemcpyAsync(&last_pos, pos + count - 1, 8, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&last_keep, keep + count - 1, 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  return last_pos + last_keep;
}

void lattice_load(const LatticeSpec& S, long long first, long long count, double* const x[3], double* const u[3],
                  int* id, cudaStream_t s) {
  if (count == 0) return;
  k_lattice<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(S, first, count, x[0], x[1], x[2], u[0], u[1], u[2],
                                                             id);
}

}  // namespace picgb
