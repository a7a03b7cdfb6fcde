// k_field.cu -- grid kernels: Yee field solve, periodic guards, current fold,
// binomial smoothing, and the FP64 diagnostics (field energy, Gauss residual).
//
// Compiled without multiply-add contraction so that the FP64 instantiation
// rounds every operation exactly as written; the FP32 instantiation is
// bandwidth-bound, so the contraction would buy nothing there.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "kernels.h"

namespace picgb {

namespace {

__device__ inline int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

inline dim3 interior_grid(const Layout& L) { return dim3((L.nx + 31) / 32, (L.ny + 7) / 8, L.nz); }
const dim3 kBlock(32, 8, 1);

template <typename T>
struct Ptr3 {
  T* c[3];
};
template <typename T>
struct Ptr6 {
  T* c[6];
};

// ---------------------------------------------------------------- guards
// Flat enumeration of the guard cells only: the z slabs (all y, x), then the
// y slabs of interior z (all x), then the x slabs of interior z and y.
__device__ inline bool guard_xyz(const Layout& L, long long g, int& X, int& Y, int& Z) {
  const long long nzs = (long long)(L.NZ - L.nz) * L.NY * L.NX;
  if (g < nzs) {
    const long long plane = (long long)L.NY * L.NX;
    int zi = (int)(g / plane);
    const long long r = g - (long long)zi * plane;
    Z = zi < L.gz ? zi : zi + L.nz;
    Y = (int)(r / L.NX);
    X = (int)(r - (long long)Y * L.NX);
    return true;
  }
  g -= nzs;
  const long long nys = (long long)L.nz * (L.NY - L.ny) * L.NX;
  if (g < nys) {
    const long long slab = (long long)(L.NY - L.ny) * L.NX;
    Z = (int)(g / slab) + L.gz;
    const long long r = g - (long long)(Z - L.gz) * slab;
    int yi = (int)(r / L.NX);
    X = (int)(r - (long long)yi * L.NX);
    Y = yi < L.gy ? yi : yi + L.ny;
    return true;
  }
  g -= nys;
  const int gw = L.NX - L.nx;
  const long long nxs = (long long)L.nz * L.ny * gw;
  if (g < nxs) {
    const long long row = gw;
    const long long zy = g / row;
    int xi = (int)(g - zy * row);
    Z = (int)(zy / L.ny) + L.gz;
    Y = (int)(zy - (long long)(Z - L.gz) * L.ny) + L.gy;
    X = xi < L.gx ? xi : xi + L.nx;
    return true;
  }
  return false;
}

inline long long guard_count(const Layout& L) {
  return (long long)(L.NZ - L.nz) * L.NY * L.NX + (long long)L.nz * (L.NY - L.ny) * L.NX +
         (long long)L.nz * L.ny * (L.NX - L.nx);
}

template <typename T, int NC>
struct PtrN {
  T* c[NC];
};

template <typename T>
__device__ inline void fill_guard_at(const Layout& L, const PtrN<T, 6>& P, int ncomp, long long g) {
  int X, Y, Z;
  if (!guard_xyz(L, g, X, Y, Z)) return;
  const int i = X - L.gx, j = Y - L.gy, k = Z - L.gz;
  const long long dst = ((long long)Z * L.NY + Y) * L.NX + X;
  if (L.open_x && (i < 0 || i >= L.nx)) {  // beyond an open x1 boundary: no field
    for (int c = 0; c < ncomp; ++c) P.c[c][dst] = T(0);
    return;
  }
  const long long src = L.idx(wrapi(i, L.nx), wrapi(j, L.ny), wrapi(k, L.nz));
  for (int c = 0; c < ncomp; ++c) P.c[c][dst] = P.c[c][src];
}

template <typename T>
__global__ void k_fill_guards(Layout L, PtrN<T, 6> P, int ncomp) {
  fill_guard_at<T>(L, P, ncomp, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// Periodic boundary for the current: what the deposit put into a guard cell
// belongs to the interior cell at the wrapped index (the node "communicates
// with its own opposite boundary").  Several guard cells can map to one
// interior cell (edges, corners), hence the atomics.
template <typename T>
__device__ inline void fold_guard_at(const Layout& L, const PtrN<T, 6>& P, int ncomp, long long g) {
  int X, Y, Z;
  if (!guard_xyz(L, g, X, Y, Z)) return;
  const int i = X - L.gx, j = Y - L.gy, k = Z - L.gz;
  const long long src = ((long long)Z * L.NY + Y) * L.NX + X;
  const bool drop = L.open_x && (i < 0 || i >= L.nx);  // deposited beyond an open x1 boundary
  const long long dst = L.idx(wrapi(i, L.nx), wrapi(j, L.ny), wrapi(k, L.nz));
  for (int c = 0; c < ncomp; ++c) {
    const T v = P.c[c][src];
    if (v != T(0) && !drop) atomicAdd(&P.c[c][dst], v);
    P.c[c][src] = T(0);
  }
}

template <typename T>
__global__ void k_fold_guards(Layout L, PtrN<T, 6> P, int ncomp) {
  fold_guard_at<T>(L, P, ncomp, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------- smoothing
// One pass of (w0, w1, w2)/(w0+w1+w2) along `dim`, periodic, out of place.
template <typename T>
__global__ void k_smooth(Layout L, const T* __restrict__ f, T* __restrict__ out, int dim, T w0, T w1, T w2, T ws) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= L.nx || j >= L.ny) return;
  int lo[3] = {i, j, k}, hi[3] = {i, j, k};
  int n[3] = {L.nx, L.ny, L.nz};
  const bool lo_out = L.open_x && dim == 0 && lo[0] == 0, hi_out = L.open_x && dim == 0 && hi[0] == n[0] - 1;
  lo[dim] = lo[dim] == 0 ? n[dim] - 1 : lo[dim] - 1;
  hi[dim] = hi[dim] == n[dim] - 1 ? 0 : hi[dim] + 1;
  long long c = L.idx(i, j, k);
  const T fl = lo_out ? T(0) : f[L.idx(lo[0], lo[1], lo[2])];  // beyond an open x1 boundary: 0
  const T fh = hi_out ? T(0) : f[L.idx(hi[0], hi[1], hi[2])];
  out[c] = (w0 * fl + w1 * f[c] + w2 * fh) / ws;
}

// ---------------------------------------------------------------- Yee solve
// Faraday half step (eq. 2d-field-solve-b-part1 / -part2; 3D adds the x3
// derivatives): B -= (dt/2) curl E with forward differences of E.
template <typename T>
__global__ void k_yee_b_half(Layout L, Ptr3<T> E, Ptr3<T> B, T h, T dx1, T dx2, T dx3) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= L.nx || j >= L.ny) return;
  // forward neighbours, wrapped periodically (no guard cells read)
  const long long c = L.idx(i, j, k);
  const long long cx = L.idx(i + 1 == L.nx ? 0 : i + 1, j, k);
  const long long cy = L.idx(i, j + 1 == L.ny ? 0 : j + 1, k);
  const T* E1 = E.c[0];
  const T* E2 = E.c[1];
  const T* E3 = E.c[2];
  T dE3d2 = (E3[cy] - E3[c]) / dx2;
  T dE3d1 = (E3[cx] - E3[c]) / dx1;
  T dE2d1 = (E2[cx] - E2[c]) / dx1;
  T dE1d2 = (E1[cy] - E1[c]) / dx2;
  T dE2d3 = T(0), dE1d3 = T(0);
  if (L.ndim == 3) {
    const long long cz = L.idx(i, j, k + 1 == L.nz ? 0 : k + 1);
    dE2d3 = (E2[cz] - E2[c]) / dx3;
    dE1d3 = (E1[cz] - E1[c]) / dx3;
  }
  B.c[0][c] = B.c[0][c] - h * (dE3d2 - dE2d3);
  B.c[1][c] = B.c[1][c] - h * (dE1d3 - dE3d1);
  B.c[2][c] = B.c[2][c] - h * (dE2d1 - dE1d2);
}

// Ampere step (eq. 2d-field-solve-e; the printed j1 of the E3 line read as j3):
// E += dt (curl B - J) with backward differences of B.
template <typename T>
__global__ void k_yee_e(Layout L, Ptr3<T> E, Ptr3<T> B, Ptr3<T> J, T dt, T dx1, T dx2, T dx3) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= L.nx || j >= L.ny) return;
  // backward neighbours, wrapped periodically (no guard cells read)
  const long long c = L.idx(i, j, k);
  const long long cx = L.idx(i == 0 ? L.nx - 1 : i - 1, j, k);
  const long long cy = L.idx(i, j == 0 ? L.ny - 1 : j - 1, k);
  const T* B1 = B.c[0];
  const T* B2 = B.c[1];
  const T* B3 = B.c[2];
  T dB3d2 = (B3[c] - B3[cy]) / dx2;
  T dB3d1 = (B3[c] - B3[cx]) / dx1;
  T dB2d1 = (B2[c] - B2[cx]) / dx1;
  T dB1d2 = (B1[c] - B1[cy]) / dx2;
  T dB2d3 = T(0), dB1d3 = T(0);
  if (L.ndim == 3) {
    const long long cz = L.idx(i, j, k == 0 ? L.nz - 1 : k - 1);
    dB2d3 = (B2[c] - B2[cz]) / dx3;
    dB1d3 = (B1[c] - B1[cz]) / dx3;
  }
  E.c[0][c] = E.c[0][c] + dt * (dB3d2 - dB2d3) - dt * J.c[0][c];
  E.c[1][c] = E.c[1][c] + dt * (dB1d3 - dB3d1) - dt * J.c[1][c];
  E.c[2][c] = E.c[2][c] + dt * (dB2d1 - dB1d2) - dt * J.c[2][c];
}

// FP32 forms of the two sweeps (the FP32 cell-offset path): multiplication by
// 1/dx and explicit fused multiply-adds.  The FP64 sweeps above keep the
// oracle's operation order (divisions, no contraction) for the FP64 parity.
__device__ inline void yee_b_f32_at(const Layout& L, const Ptr3<float>& E, const Ptr3<float>& B, float h, float i1,
                                    float i2, float i3, int i, int j, int k) {
  if (i >= L.nx || j >= L.ny) return;
  const long long c = L.idx(i, j, k);
  const long long cx = c + (i + 1 == L.nx ? 1 - L.nx : 1);
  const long long cy = c + (j + 1 == L.ny ? (long long)(1 - L.ny) * L.NX : L.NX);
  const float* __restrict__ E1 = E.c[0];
  const float* __restrict__ E2 = E.c[1];
  const float* __restrict__ E3 = E.c[2];
  const float e1 = __ldg(E1 + c), e2 = __ldg(E2 + c), e3 = __ldg(E3 + c);
  const bool front = L.open_x && i + 1 == L.nx;  // beyond an open x1 boundary: E = 0
  const float dE3d2 = (__ldg(E3 + cy) - e3) * i2;
  const float dE3d1 = ((front ? 0.f : __ldg(E3 + cx)) - e3) * i1;
  const float dE2d1 = ((front ? 0.f : __ldg(E2 + cx)) - e2) * i1;
  const float dE1d2 = (__ldg(E1 + cy) - e1) * i2;
  float dE2d3 = 0.f, dE1d3 = 0.f;
  if (L.ndim == 3) {
    const long long cz = c + (k + 1 == L.nz ? (long long)(1 - L.nz) * L.NX * L.NY : (long long)L.NX * L.NY);
    dE2d3 = (__ldg(E2 + cz) - e2) * i3;
    dE1d3 = (__ldg(E1 + cz) - e1) * i3;
  }
  B.c[0][c] = fmaf(-h, dE3d2 - dE2d3, B.c[0][c]);
  B.c[1][c] = fmaf(-h, dE1d3 - dE3d1, B.c[1][c]);
  B.c[2][c] = fmaf(-h, dE2d1 - dE1d2, B.c[2][c]);
}

__global__ void k_yee_b_half_f32(Layout L, Ptr3<float> E, Ptr3<float> B, float h, float i1, float i2, float i3) {
  yee_b_f32_at(L, E, B, h, i1, i2, i3, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y,
               blockIdx.z);
}

__device__ inline void yee_e_f32_at(const Layout& L, const Ptr3<float>& E, const Ptr3<float>& B, const Ptr3<float>& J,
                                    float dt, float i1, float i2, float i3, const float* inc, int i, int j, int k) {
  if (i >= L.nx || j >= L.ny) return;
  const long long c = L.idx(i, j, k);
  const long long cx = c - (i == 0 ? 1 - L.nx : 1);
  const long long cy = c - (j == 0 ? (long long)(1 - L.ny) * L.NX : L.NX);
  const float* __restrict__ B1 = B.c[0];
  const float* __restrict__ B2 = B.c[1];
  const float* __restrict__ B3 = B.c[2];
  const float b1 = __ldg(B1 + c), b2 = __ldg(B2 + c), b3 = __ldg(B3 + c);
  // beyond an open x1 boundary: B = 0, or that of a pulse entering there
  const bool back = L.open_x && i == 0;
  const long long p = (long long)k * L.ny + j;  // this row in the incident planes
  const float b3m = back ? (inc ? inc[(long long)L.ny * L.nz + p] : 0.f) : __ldg(B3 + cx);
  const float b2m = back ? (inc ? inc[p] : 0.f) : __ldg(B2 + cx);
  const float dB3d2 = (b3 - __ldg(B3 + cy)) * i2;
  const float dB3d1 = (b3 - b3m) * i1;
  const float dB2d1 = (b2 - b2m) * i1;
  const float dB1d2 = (b1 - __ldg(B1 + cy)) * i2;
  float dB2d3 = 0.f, dB1d3 = 0.f;
  if (L.ndim == 3) {
    const long long cz = c - (k == 0 ? (long long)(1 - L.nz) * L.NX * L.NY : (long long)L.NX * L.NY);
    dB2d3 = (b2 - __ldg(B2 + cz)) * i3;
    dB1d3 = (b1 - __ldg(B1 + cz)) * i3;
  }
  E.c[0][c] = fmaf(dt, dB3d2 - dB2d3 - __ldg(J.c[0] + c), E.c[0][c]);
  E.c[1][c] = fmaf(dt, dB1d3 - dB3d1 - __ldg(J.c[1] + c), E.c[1][c]);
  E.c[2][c] = fmaf(dt, dB2d1 - dB1d2 - __ldg(J.c[2] + c), E.c[2][c]);
}

__global__ void k_yee_e_f32(Layout L, Ptr3<float> E, Ptr3<float> B, Ptr3<float> J, float dt, float i1, float i2,
                            float i3, const float* inc) {
  yee_e_f32_at(L, E, B, J, dt, i1, i2, i3, inc, blockIdx.x * blockDim.x + threadIdx.x,
               blockIdx.y * blockDim.y + threadIdx.y, blockIdx.z);
}

// 3D forms of the two FP32 sweeps that walk kZM planes of x3 per thread and
// carry the x3 neighbour of one plane into the next in registers (the B half
// step reads E at k + 1, the E step B at k - 1).  Every value is computed with
// the expressions of yee_b_f32_at / yee_e_f32_at.
constexpr int kZM = 8;

__global__ void k_yee_b_half_f32_z(Layout L, Ptr3<float> E, Ptr3<float> B, float h, float i1, float i2, float i3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * kZM;
  if (i >= L.nx || j >= L.ny) return;
  const long long pz = (long long)L.NX * L.NY;
  const float* __restrict__ E1 = E.c[0];
  const float* __restrict__ E2 = E.c[1];
  const float* __restrict__ E3 = E.c[2];
  const bool front = L.open_x && i + 1 == L.nx;
  const long long dx1 = i + 1 == L.nx ? 1 - L.nx : 1;
  const long long dy1 = j + 1 == L.ny ? (long long)(1 - L.ny) * L.NX : L.NX;
  long long c = L.idx(i, j, k0);
  float e1 = __ldg(E1 + c), e2 = __ldg(E2 + c);
  const int k1 = min(k0 + kZM, L.nz);
  for (int k = k0; k < k1; ++k) {
    const long long cx = c + dx1, cy = c + dy1;
    const long long cz = c + (k + 1 == L.nz ? (long long)(1 - L.nz) * pz : pz);
    const float e3 = __ldg(E3 + c);
    const float z1 = __ldg(E1 + cz), z2 = __ldg(E2 + cz);  // the next plane's e1, e2
    const float dE3d2 = (__ldg(E3 + cy) - e3) * i2;
    const float dE3d1 = ((front ? 0.f : __ldg(E3 + cx)) - e3) * i1;
    const float dE2d1 = ((front ? 0.f : __ldg(E2 + cx)) - e2) * i1;
    const float dE1d2 = (__ldg(E1 + cy) - e1) * i2;
    const float dE2d3 = (z2 - e2) * i3;
    const float dE1d3 = (z1 - e1) * i3;
    B.c[0][c] = fmaf(-h, dE3d2 - dE2d3, B.c[0][c]);
    B.c[1][c] = fmaf(-h, dE1d3 - dE3d1, B.c[1][c]);
    B.c[2][c] = fmaf(-h, dE2d1 - dE1d2, B.c[2][c]);
    e1 = z1;
    e2 = z2;
    c += pz;
  }
}

__global__ void k_yee_e_f32_z(Layout L, Ptr3<float> E, Ptr3<float> B, Ptr3<float> J, float dt, float i1, float i2,
                              float i3, const float* inc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * kZM;
  if (i >= L.nx || j >= L.ny) return;
  const long long pz = (long long)L.NX * L.NY;
  const float* __restrict__ B1 = B.c[0];
  const float* __restrict__ B2 = B.c[1];
  const float* __restrict__ B3 = B.c[2];
  const bool back = L.open_x && i == 0;
  const long long dx1 = i == 0 ? 1 - L.nx : 1;
  const long long dy1 = j == 0 ? (long long)(1 - L.ny) * L.NX : L.NX;
  long long c = L.idx(i, j, k0);
  const long long cz0 = c - (k0 == 0 ? (long long)(1 - L.nz) * pz : pz);
  float m1 = __ldg(B1 + cz0), m2 = __ldg(B2 + cz0);  // the previous plane's b1, b2
  const int k1 = min(k0 + kZM, L.nz);
  for (int k = k0; k < k1; ++k) {
    const long long cx = c - dx1, cy = c - dy1;
    const float b1 = __ldg(B1 + c), b2 = __ldg(B2 + c), b3 = __ldg(B3 + c);
    const long long p = (long long)k * L.ny + j;  // this row in the incident planes
    const float b3m = back ? (inc ? inc[(long long)L.ny * L.nz + p] : 0.f) : __ldg(B3 + cx);
    const float b2m = back ? (inc ? inc[p] : 0.f) : __ldg(B2 + cx);
    const float dB3d2 = (b3 - __ldg(B3 + cy)) * i2;
    const float dB3d1 = (b3 - b3m) * i1;
    const float dB2d1 = (b2 - b2m) * i1;
    const float dB1d2 = (b1 - __ldg(B1 + cy)) * i2;
    const float dB2d3 = (b2 - m2) * i3;
    const float dB1d3 = (b1 - m1) * i3;
    E.c[0][c] = fmaf(dt, dB3d2 - dB2d3 - __ldg(J.c[0] + c), E.c[0][c]);
    E.c[1][c] = fmaf(dt, dB1d3 - dB3d1 - __ldg(J.c[1] + c), E.c[1][c]);
    E.c[2][c] = fmaf(dt, dB2d1 - dB1d2 - __ldg(J.c[2] + c), E.c[2][c]);
    m1 = b1;
    m2 = b2;
    c += pz;
  }
}

// Moving window: every field value one cell back in x1 (value at i <- value
// at i + 1), zero in the new front column.  One warp per row, 256 values per
// round with every load of the round before its stores; a row is read
// ahead of where it is written.
template <typename T>
__device__ inline void shift_row(const Layout& L, const PtrN<T, 6>& P, int ncomp, long long row) {
  const int lane = threadIdx.x & 31;
  const long long rows = (long long)ncomp * L.ny * L.nz;
  if (row >= rows) return;
  const int c = (int)(row / ((long long)L.ny * L.nz));
  const long long r = row - (long long)c * L.ny * L.nz;
  const int j = (int)(r % L.ny), k = (int)(r / L.ny);
  T* f = P.c[c] + L.idx(0, j, k);
  // 256 values per round: all loads of a round are in flight before its
  // stores, which only touch values the later rounds no longer read
  constexpr int kR = 8;
  for (int b = 0; b < L.nx; b += 32 * kR) {
    T v[kR];
#pragma unroll
    for (int m = 0; m < kR; ++m) {
      const int i = b + 32 * m + lane;
      v[m] = i + 1 < L.nx ? f[i + 1] : T(0);
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < kR; ++m) {
      const int i = b + 32 * m + lane;
      if (i < L.nx) f[i] = v[m];
    }
    __syncwarp();
  }
}

template <typename T>
__global__ void k_shift_x(Layout L, PtrN<T, 6> P, int ncomp) {
  shift_row<T>(L, P, ncomp, (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
}

// Laser pulse added to the fields, each component at its staggered position.
// The pulse moves in +x_a (a = 0: wavetype 1, along x1; a = 1: wavetype 2,
// along x2) with the vector potential A = vosc f(xi) g T cos(psi) along
// p = cos(pol) e_t + sin(pol) e_3 (e_t the in-plane transverse axis); in the
// slowly varying envelope form E = -dA/dt = -vosc k f g T sin(psi) p and
// B = e_a x E.  xi = x_front - x_a; f rises as 10 s^3 - 15 s^4 + 6 s^5
// (s = xi / rise), stays 1 over `length` and falls as the mirror image over
// `fall` (the thesis' temporal profile).  With a focal plane (focus_on) the
// transverse profile is the lowest Hermite-Gaussian beam of the thesis'
// laser-beam section: z = x_a - x_focus, z_R = k w0^2 / 2, w = w0 sqrt(1 +
// (z/z_R)^2), T = exp(-r^2 / w^2), g = w0 / w (3D; sqrt(w0 / w) for the 2D
// slab beam), psi = k (x_a - x_front) + k r^2 / (2 R) - G + phase with
// R = z + z_R^2 / z and the Gouy phase G = atan(z / z_R) (half of it in 2D).
// Without a focal plane g = 1, w = w0, psi = k (x_a - x_front) + phase.
struct LaserDev {
  double vosc, k, w0, rise, length, fall, xfront, ct, c3, cpol, spol, phase;
  double xmin[3], dx[3];
  int axis, focus_on;
  double xfocus;
};

__device__ inline double laser_profile(double s) { return s * s * s * (10.0 + s * (-15.0 + 6.0 * s)); }

__device__ inline double laser_amp(const LaserDev& P, int ndim, const double x[3]) {
  const int a = P.axis, t = 1 - P.axis;
  const double xi = P.xfront - x[a];
  double f = 0.0;
  if (xi >= 0.0 && xi < P.rise)
    f = laser_profile(xi / P.rise);
  else if (xi >= P.rise && xi < P.rise + P.length)
    f = 1.0;
  else if (xi >= P.rise + P.length && xi < P.rise + P.length + P.fall)
    f = laser_profile(1.0 - (xi - P.rise - P.length) / P.fall);
  if (f == 0.0) return 0.0;
  double r2 = (x[t] - P.ct) * (x[t] - P.ct);
  if (ndim == 3) r2 += (x[2] - P.c3) * (x[2] - P.c3);
  double w2 = P.w0 * P.w0, g = 1.0, psi = P.k * (x[a] - P.xfront) + P.phase;
  if (P.focus_on) {
    const double zr = 0.5 * P.k * P.w0 * P.w0, z = x[a] - P.xfocus, q = 1.0 + (z / zr) * (z / zr);
    w2 *= q;
    g = ndim == 3 ? 1.0 / sqrt(q) : 1.0 / sqrt(sqrt(q));
    const double gouy = atan(z / zr);
    psi += (z != 0.0 ? P.k * r2 / (2.0 * (z + zr * zr / z)) : 0.0) - (ndim == 3 ? gouy : 0.5 * gouy);
  }
  return -P.vosc * P.k * f * g * exp(-r2 / w2) * sin(psi);
}

template <typename T>
__global__ void k_laser_add(Layout L, Ptr6<T> F, LaserDev P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= L.nx || j >= L.ny) return;
  const long long c = L.idx(i, j, k);
  const double h3 = L.ndim == 3 ? 0.5 : 0.0;
  // position of a component with stagger (s1, s2, s3)
  auto A = [&](double s1, double s2, double s3) {
    const double x[3] = {P.xmin[0] + (i + s1) * P.dx[0], P.xmin[1] + (j + s2) * P.dx[1],
                         P.xmin[2] + (k + s3) * P.dx[2]};
    return laser_amp(P, L.ndim, x);
  };
  if (P.axis == 0) {  // along x1: E2, E3; B3 = E2, B2 = -E3
    F.c[1][c] = (T)((double)F.c[1][c] + A(0.0, 0.5, 0.0) * P.cpol);
    F.c[2][c] = (T)((double)F.c[2][c] + A(0.0, 0.0, h3) * P.spol);
    F.c[4][c] = (T)((double)F.c[4][c] - A(0.5, 0.0, h3) * P.spol);
    F.c[5][c] = (T)((double)F.c[5][c] + A(0.5, 0.5, 0.0) * P.cpol);
  } else {  // along x2: E1, E3; B1 = E3, B3 = -E1
    F.c[0][c] = (T)((double)F.c[0][c] + A(0.5, 0.0, 0.0) * P.cpol);
    F.c[2][c] = (T)((double)F.c[2][c] + A(0.0, 0.0, h3) * P.spol);
    F.c[3][c] = (T)((double)F.c[3][c] + A(0.0, 0.5, h3) * P.spol);
    F.c[5][c] = (T)((double)F.c[5][c] - A(0.5, 0.5, 0.0) * P.cpol);
  }
}

// ---------------------------------------------------------------- diagnostics
__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int nw = (blockDim.x * blockDim.y + 31) / 32;
  double s = 0.0;
  if (warp == 0) {
    s = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;
}

__device__ inline double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int nw = (blockDim.x * blockDim.y + 31) / 32;
  double s = 0.0;
  if (warp == 0) {
    s = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
  }
  __syncthreads();
  return s;
}

template <typename T>
__global__ void k_field_energy(Layout L, Ptr6<T> F, double* acc) {
  __shared__ double red[32];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  double s = 0.0;
  if (i < L.nx && j < L.ny) {
    long long c = L.idx(i, j, k);
    for (int m = 0; m < 6; ++m) {
      double v = (double)F.c[m][c];
      s = s + v * v;
    }
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(acc, s);
}

// Field energy and Gauss-law diagnostics of the FP32 fields in one pass over
// the cells, a fixed number of blocks striding over them (one atomic per block
// and quantity): the sum of E^2 + B^2 (FP32 squares of four cells, summed in
// FP64), and the maxima of |div E - rho_total|, |rho_total| and
// |rho_particles| as k_gauss.  The divergence terms are differences of FP32
// values taken in FP32 (their rounding is of the order of the fields' own);
// rho_total and the residual are FP64.  The maxima are kept as the bit
// patterns of non-negative doubles, whose integer order is their order.
constexpr int kDiagThreads = 256;
constexpr int kDiagUnroll = 4;

__global__ void __launch_bounds__(kDiagThreads) k_diag_fields(Layout L, Ptr6<float> F, const double* __restrict__ rho,
                                                              double rho_bg, float i1, float i2, float i3,
                                                              Diag64* acc) {
  __shared__ double red[32];
  const int ncell = L.nx * L.ny * L.nz;  // < 2^31 (checked by the launcher)
  const int stride = gridDim.x * blockDim.x;
  const int sy = L.NX, sz = L.NX * L.NY;
  double s = 0.0;
  long long g = 0, r = 0, p = 0;
  for (int q0 = blockIdx.x * blockDim.x + threadIdx.x; q0 < ncell; q0 += kDiagUnroll * stride) {
    float es = 0.f;
#pragma unroll
    for (int u = 0; u < kDiagUnroll; ++u) {
      const int q = q0 + u * stride;
      if (q >= ncell) break;
      const int i = q % L.nx, rest = q / L.nx;
      const int j = rest % L.ny, k = rest / L.ny;
      const long long c = L.idx(i, j, k);
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        const float v = F.c[m][c];
        es = fmaf(v, v, es);
      }
      float div = (F.c[0][c] - F.c[0][c - 1]) * i1 + (F.c[1][c] - F.c[1][c - sy]) * i2;
      if (L.ndim == 3) div += (F.c[2][c] - F.c[2][c - sz]) * i3;
      const double rp = rho[c], rt = rp + rho_bg;
      g = max(g, __double_as_longlong(fabs((double)div - rt)));
      r = max(r, __double_as_longlong(fabs(rt)));
      p = max(p, __double_as_longlong(fabs(rp)));
    }
    s += (double)es;
  }
  s = block_sum(s, red);
  const double gm = block_max(__longlong_as_double(g), red);
  const double rm = block_max(__longlong_as_double(r), red);
  const double pm = block_max(__longlong_as_double(p), red);
  if (threadIdx.x == 0) {
    atomicAdd(&acc->field_energy, s);
    atomic_max_nonneg(&acc->gauss_max, gm);
    atomic_max_nonneg(&acc->rho_max, rm);
    atomic_max_nonneg(&acc->rho_part_max, pm);
  }
}

template <typename T>
// dx1..dx3: the reciprocal cell sizes
__global__ void k_gauss(Layout L, Ptr3<T> E, const double* __restrict__ rho, double rho_bg, double dx1, double dx2,
                        double dx3, double* gmax, double* rmax, double* pmax) {
  __shared__ double red[32];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  double g = 0.0, r = 0.0, p = 0.0;
  if (i < L.nx && j < L.ny) {
    const long long sx = 1, sy = L.NX, sz = (long long)L.NX * L.NY;
    long long c = L.idx(i, j, k);
    // FP64 differences (exact for FP32 E) times 1/dx: the residual is itself
    // ~1e-7 of rho, so the divergence stays in FP64
    double div = ((double)E.c[0][c] - (double)E.c[0][c - sx]) * dx1 + ((double)E.c[1][c] - (double)E.c[1][c - sy]) * dx2;
    if (L.ndim == 3) div = div + ((double)E.c[2][c] - (double)E.c[2][c - sz]) * dx3;
    double rt = rho[c] + rho_bg;
    g = fabs(div - rt);
    r = fabs(rt);
    p = fabs(rho[c]);
  }
  g = block_max(g, red);
  r = block_max(r, red);
  p = block_max(p, red);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    atomic_max_nonneg(gmax, g);
    atomic_max_nonneg(rmax, r);
    atomic_max_nonneg(pmax, p);
  }
}

template <typename T>
__global__ void k_pack(Layout L, const T* __restrict__ f, double* __restrict__ dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= L.nx || j >= L.ny) return;
  dst[((long long)k * L.ny + j) * L.nx + i] = (double)f[L.idx(i, j, k)];
}

template <typename T>
__global__ void k_unpack(Layout L, const double* __restrict__ src, T* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= L.nx || j >= L.ny) return;
  f[L.idx(i, j, k)] = (T)src[((long long)k * L.ny + j) * L.nx + i];
}

// E1(i+1/2) - E1(i-1/2) = dx1 * rho(i), zero mean per column.
template <typename T>
__global__ void k_gauss_x1(Layout L, const double* __restrict__ rho, double rho_bg, double dx1, T* e1) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (j >= L.ny) return;
  double run = 0.0, mean = 0.0;
  for (int i = 0; i < L.nx; ++i) {
    long long c = L.idx(i, j, k);
    run = run + dx1 * (rho[c] + rho_bg);
    mean = mean + run;
  }
  mean = mean / (double)L.nx;
  run = 0.0;
  for (int i = 0; i < L.nx; ++i) {
    long long c = L.idx(i, j, k);
    run = run + dx1 * (rho[c] + rho_bg);
    e1[c] = (T)(run - mean);
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers
template <typename T>
void fill_guards(const Layout& L, T* const* comps, int ncomp, cudaStream_t s) {
  const long long n = guard_count(L);
  if (n == 0) return;
  for (int c0 = 0; c0 < ncomp; c0 += 6) {
    PtrN<T, 6> P{};
    const int m = ncomp - c0 < 6 ? ncomp - c0 : 6;
    for (int c = 0; c < m; ++c) P.c[c] = comps[c0 + c];
    k_fill_guards<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, P, m);
  }
}

template <typename T>
void fold_guards(const Layout& L, T* const* comps, int ncomp, cudaStream_t s) {
  const long long n = guard_count(L);
  if (n == 0) return;
  for (int c0 = 0; c0 < ncomp; c0 += 6) {
    PtrN<T, 6> P{};
    const int m = ncomp - c0 < 6 ? ncomp - c0 : 6;
    for (int c = 0; c < m; ++c) P.c[c] = comps[c0 + c];
    k_fold_guards<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, P, m);
  }
}

template <typename T>
void smooth_pass(const Layout& L, T* comp, T* tmp, int dim, double w0, double w1, double w2, cudaStream_t s) {
  k_smooth<T><<<interior_grid(L), kBlock, 0, s>>>(L, comp, tmp, dim, (T)w0, (T)w1, (T)w2, (T)(w0 + w1 + w2));
  cudaMemcpyAsync(comp, tmp, sizeof(T) * (size_t)L.plane, cudaMemcpyDeviceToDevice, s);
}

template <typename T>
void yee_b_half(const Layout& L, T* const* e, T* const* b, double dt, const double dx[3], cudaStream_t s) {
  Ptr3<T> E{{e[0], e[1], e[2]}}, B{{b[0], b[1], b[2]}};
  if constexpr (sizeof(T) == 4) {
    if (L.ndim == 3)
      k_yee_b_half_f32_z<<<dim3((L.nx + 31) / 32, (L.ny + 7) / 8, (L.nz + kZM - 1) / kZM), kBlock, 0, s>>>(
          L, E, B, (float)(dt / 2.0), (float)(1.0 / dx[0]), (float)(1.0 / dx[1]), (float)(1.0 / dx[2]));
    else
      k_yee_b_half_f32<<<interior_grid(L), kBlock, 0, s>>>(L, E, B, (float)(dt / 2.0), (float)(1.0 / dx[0]),
                                                           (float)(1.0 / dx[1]), (float)(1.0 / dx[2]));
  }
  else
    k_yee_b_half<T><<<interior_grid(L), kBlock, 0, s>>>(L, E, B, (T)(dt / 2.0), (T)dx[0], (T)dx[1], (T)dx[2]);
}

template <typename T>
void yee_e(const Layout& L, T* const* e, T* const* b, T* const* j, double dt, const double dx[3], cudaStream_t s,
           const float* inc) {
  Ptr3<T> E{{e[0], e[1], e[2]}}, B{{b[0], b[1], b[2]}}, J{{j[0], j[1], j[2]}};
  if constexpr (sizeof(T) == 4) {
    if (L.ndim == 3)
      k_yee_e_f32_z<<<dim3((L.nx + 31) / 32, (L.ny + 7) / 8, (L.nz + kZM - 1) / kZM), kBlock, 0, s>>>(
          L, E, B, J, (float)dt, (float)(1.0 / dx[0]), (float)(1.0 / dx[1]), (float)(1.0 / dx[2]), inc);
    else
      k_yee_e_f32<<<interior_grid(L), kBlock, 0, s>>>(L, E, B, J, (float)dt, (float)(1.0 / dx[0]),
                                                      (float)(1.0 / dx[1]), (float)(1.0 / dx[2]), inc);
  }
  else
    k_yee_e<T><<<interior_grid(L), kBlock, 0, s>>>(L, E, B, J, (T)dt, (T)dx[0], (T)dx[1], (T)dx[2]);
}

template <typename T>
void shift_x(const Layout& L, T* const* comps, int ncomp, cudaStream_t s) {
  PtrN<T, 6> P{};
  for (int c = 0; c < ncomp; ++c) P.c[c] = comps[c];
  const long long rows = (long long)ncomp * L.ny * L.nz;
  k_shift_x<T><<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(L, P, ncomp);
}

// B2 and B3 of the antenna pulses just below the lower x1 boundary (x1 =
// xlo1 - dx1/2) at time t, summed into inc[2][ny nz]: each pulse's front is
// at xlo1 + (t - start); B3 = E2, B2 = -E3 of laser_amp at the B positions.
__global__ void k_antenna_plane(Layout L, const LaserDev* P, int n, double t, double xlo1, const double* txlo,
                                float* inc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (j >= L.ny) return;
  if (txlo) {  // read on the device (a step replayed from a graph)
    t = txlo[0];
    xlo1 = txlo[1];
  }
  const double h3 = L.ndim == 3 ? 0.5 : 0.0;
  double b2 = 0.0, b3 = 0.0;
  for (int a = 0; a < n; ++a) {
    LaserDev Q = P[a];
    Q.xfront = xlo1 + (t - Q.xfront);  // xfront holds `start` for an antenna
    const double x1 = xlo1 - 0.5 * Q.dx[0];
    const double xb2[3] = {x1, Q.xmin[1] + j * Q.dx[1], Q.xmin[2] + (k + h3) * Q.dx[2]};
    const double xb3[3] = {x1, Q.xmin[1] + (j + 0.5) * Q.dx[1], Q.xmin[2] + k * Q.dx[2]};
    b2 -= laser_amp(Q, L.ndim, xb2) * Q.spol;
    b3 += laser_amp(Q, L.ndim, xb3) * Q.cpol;
  }
  const long long p = (long long)k * L.ny + j;
  inc[p] = (float)b2;
  inc[(long long)L.ny * L.nz + p] = (float)b3;
}

LaserDev laser_dev(const double* p) {
  LaserDev P;
  P.vosc = p[0];
  P.k = p[1];
  P.w0 = p[2];
  P.rise = p[3];
  P.length = p[4];
  P.fall = p[5];
  P.xfront = p[6];
  P.ct = p[7];
  P.c3 = p[8];
  P.cpol = p[9];
  P.spol = p[10];
  P.phase = p[11];
  for (int d = 0; d < 3; ++d) {
    P.xmin[d] = p[12 + d];
    P.dx[d] = p[15 + d];
  }
  P.axis = (int)p[18];
  P.focus_on = p[19] != 0.0;
  P.xfocus = p[20];
  return P;
}

size_t antenna_bytes() { return sizeof(LaserDev); }

void antenna_store(const double* p, void* dst) {
  const LaserDev P = laser_dev(p);
  std::memcpy(dst, &P, sizeof(P));
}

void antenna_plane(const Layout& L, const void* ants, int n, double t, double xlo1, float* inc, cudaStream_t s,
                   const double* txlo) {
  k_antenna_plane<<<dim3((L.ny + 127) / 128, L.nz), 128, 0, s>>>(L, static_cast<const LaserDev*>(ants), n, t, xlo1,
                                                                 txlo, inc);
}

template <typename T>
void laser_add(const Layout& L, T* const* f, const double* p, cudaStream_t s) {
  Ptr6<T> F{{f[0], f[1], f[2], f[3], f[4], f[5]}};
  LaserDev P;
  P.vosc = p[0];
  P.k = p[1];
  P.w0 = p[2];
  P.rise = p[3];
  P.length = p[4];
  P.fall = p[5];
  P.xfront = p[6];
  P.ct = p[7];
  P.c3 = p[8];
  P.cpol = p[9];
  P.spol = p[10];
  P.phase = p[11];
  for (int d = 0; d < 3; ++d) {
    P.xmin[d] = p[12 + d];
    P.dx[d] = p[15 + d];
  }
  P.axis = (int)p[18];
  P.focus_on = p[19] != 0.0;
  P.xfocus = p[20];
  k_laser_add<T><<<interior_grid(L), kBlock, 0, s>>>(L, F, P);
}

template <typename T>
void field_energy(const Layout& L, T* const* f, Diag64* acc, cudaStream_t s) {
  Ptr6<T> F{{f[0], f[1], f[2], f[3], f[4], f[5]}};
  k_field_energy<T><<<interior_grid(L), kBlock, 0, s>>>(L, F, &acc->field_energy);
}

void diag_fields(const Layout& L, float* const* f, const double* rho, double rho_bg, const double dx[3], Diag64* acc,
                 cudaStream_t s) {
  Ptr6<float> F{{f[0], f[1], f[2], f[3], f[4], f[5]}};
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ncell = (long long)L.nx * L.ny * L.nz;
  if (ncell <= 0 || ncell >= (1ll << 31)) {  // int32 cell index in the kernel
    gauss_residual<float>(L, f, rho, rho_bg, dx, acc, s);
    field_energy<float>(L, f, acc, s);
    return;
  }
  const long long want = (ncell + kDiagThreads * kDiagUnroll - 1) / (kDiagThreads * kDiagUnroll);
  const int blocks = (int)std::min<long long>(want, 8ll * sms);
  k_diag_fields<<<blocks, kDiagThreads, 0, s>>>(L, F, rho, rho_bg, (float)(1.0 / dx[0]), (float)(1.0 / dx[1]),
                                               (float)(1.0 / dx[2]), acc);
}

template <typename T>
void gauss_residual(const Layout& L, T* const* e, const double* rho, double rho_bg, const double dx[3], Diag64* acc,
                    cudaStream_t s) {
  Ptr3<T> E{{e[0], e[1], e[2]}};
  k_gauss<T><<<interior_grid(L), kBlock, 0, s>>>(L, E, rho, rho_bg, 1.0 / dx[0], 1.0 / dx[1], 1.0 / dx[2],
                                                 &acc->gauss_max,
                                                 &acc->rho_max, &acc->rho_part_max);
}

template <typename T>
void pack_interior(const Layout& L, const T* comp, double* dst, cudaStream_t s) {
  k_pack<T><<<interior_grid(L), kBlock, 0, s>>>(L, comp, dst);
}

template <typename T>
void unpack_interior(const Layout& L, const double* src, T* comp, cudaStream_t s) {
  k_unpack<T><<<interior_grid(L), kBlock, 0, s>>>(L, src, comp);
}

template <typename T>
void init_e_gauss_x1(const Layout& L, const double* rho, double rho_bg, double dx1, T* e1, cudaStream_t s) {
  k_gauss_x1<T><<<dim3((L.ny + 127) / 128, L.nz), 128, 0, s>>>(L, rho, rho_bg, dx1, e1);
}

// ------------------------------------------------------- batched field step
// Every stage of the FP32 field step of many simulations in one launch: block
// b belongs to the member m with blk[m] <= b < blk[m + 1] and runs the same
// per-element code as the single-simulation kernels on its block of member m.
__device__ inline int batch_member(const int* blk, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(blk + mid) <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// interior blocks of 32 x 8 cells (one x3 plane), as interior_grid
__device__ inline void batch_cell(const Layout& L, int lb, int& i, int& j, int& k) {
  const int gx = (L.nx + 31) / 32, gy = (L.ny + 7) / 8;
  const int bx = lb % gx, by = (lb / gx) % gy;
  k = lb / (gx * gy);
  i = bx * 32 + (threadIdx.x & 31);
  j = by * 8 + (threadIdx.x >> 5);
}

__global__ void k_batch_zero(const BatchZeroSeg* seg, const int* blk, int n) {
  const int m = batch_member(blk, n, blockIdx.x);
  const BatchZeroSeg z = seg[m];
  const long long w0 = ((long long)(blockIdx.x - blk[m]) * blockDim.x + threadIdx.x) * 4;
  uint32_t* p = static_cast<uint32_t*>(z.p);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (w0 + q < z.words) p[w0 + q] = 0u;
}

__global__ void k_batch_fold(BatchFieldTable T) {
  const int m = batch_member(T.blk_guard, T.n, blockIdx.x);
  const BatchFieldMember& M = T.m[m];
  PtrN<float, 6> P{};
  for (int c = 0; c < 3; ++c) P.c[c] = M.j[c];
  fold_guard_at<float>(M.L, P, 3, (long long)(blockIdx.x - T.blk_guard[m]) * blockDim.x + threadIdx.x);
}

__global__ void k_batch_fill(BatchFieldTable T) {
  const int m = batch_member(T.blk_guard, T.n, blockIdx.x);
  const BatchFieldMember& M = T.m[m];
  PtrN<float, 6> P{};
  for (int c = 0; c < 6; ++c) P.c[c] = M.f[c];
  fill_guard_at<float>(M.L, P, 6, (long long)(blockIdx.x - T.blk_guard[m]) * blockDim.x + threadIdx.x);
}

__global__ void k_batch_yee_b(BatchFieldTable T) {
  const int m = batch_member(T.blk_int, T.n, blockIdx.x);
  const BatchFieldMember& M = T.m[m];
  int i, j, k;
  batch_cell(M.L, blockIdx.x - T.blk_int[m], i, j, k);
  const Ptr3<float> E{{M.f[0], M.f[1], M.f[2]}}, B{{M.f[3], M.f[4], M.f[5]}};
  yee_b_f32_at(M.L, E, B, M.h, M.i1, M.i2, M.i3, i, j, k);
}

__global__ void k_batch_yee_e(BatchFieldTable T) {
  const int m = batch_member(T.blk_int, T.n, blockIdx.x);
  const BatchFieldMember& M = T.m[m];
  int i, j, k;
  batch_cell(M.L, blockIdx.x - T.blk_int[m], i, j, k);
  const Ptr3<float> E{{M.f[0], M.f[1], M.f[2]}}, B{{M.f[3], M.f[4], M.f[5]}}, J{{M.j[0], M.j[1], M.j[2]}};
  yee_e_f32_at(M.L, E, B, J, M.dt, M.i1, M.i2, M.i3, M.inc, i, j, k);
}

__global__ void k_batch_shift(BatchFieldTable T) {
  const int m = batch_member(T.blk_rows, T.n, blockIdx.x);
  if (!T.shift[m]) return;  // this member does not move this step
  const BatchFieldMember& M = T.m[m];
  PtrN<float, 6> P{};
  for (int c = 0; c < 6; ++c) P.c[c] = M.f[c];
  shift_row<float>(M.L, P, 6, (long long)(blockIdx.x - T.blk_rows[m]) * (blockDim.x >> 5) + (threadIdx.x >> 5));
}

int batch_interior_blocks(const Layout& L) { return ((L.nx + 31) / 32) * ((L.ny + 7) / 8) * L.nz; }
int batch_guard_blocks(const Layout& L) { return (int)((guard_count(L) + 255) / 256); }
int batch_row_blocks(const Layout& L) { return (int)((6LL * L.ny * L.nz + 7) / 8); }
int batch_zero_blocks(long long words) { return (int)((words + 1023) / 1024); }

void batch_zero(const BatchZeroSeg* seg, const int* blk, int n, int nblk, cudaStream_t s) {
  if (nblk > 0) k_batch_zero<<<nblk, 256, 0, s>>>(seg, blk, n);
}
void batch_fold(const BatchFieldTable& T, int nblk, cudaStream_t s) {
  if (nblk > 0) k_batch_fold<<<nblk, 256, 0, s>>>(T);
}
void batch_fill(const BatchFieldTable& T, int nblk, cudaStream_t s) {
  if (nblk > 0) k_batch_fill<<<nblk, 256, 0, s>>>(T);
}
void batch_yee_b(const BatchFieldTable& T, int nblk, cudaStream_t s) {
  if (nblk > 0) k_batch_yee_b<<<nblk, 256, 0, s>>>(T);
}
void batch_yee_e(const BatchFieldTable& T, int nblk, cudaStream_t s) {
  if (nblk > 0) k_batch_yee_e<<<nblk, 256, 0, s>>>(T);
}
void batch_shift(const BatchFieldTable& T, int nblk, cudaStream_t s) {
  if (nblk > 0) k_batch_shift<<<nblk, 256, 0, s>>>(T);
}

#define PICGB_INST(T)                                                                                         \
  template void fill_guards<T>(const Layout&, T* const*, int, cudaStream_t);                                  \
  template void fold_guards<T>(const Layout&, T* const*, int, cudaStream_t);                                  \
  template void smooth_pass<T>(const Layout&, T*, T*, int, double, double, double, cudaStream_t);             \
  template void yee_b_half<T>(const Layout&, T* const*, T* const*, double, const double[3], cudaStream_t);     \
  template void yee_e<T>(const Layout&, T* const*, T* const*, T* const*, double, const double[3], cudaStream_t,   \
                         const float*);                                                                       \
  template void field_energy<T>(const Layout&, T* const*, Diag64*, cudaStream_t);                             \
  template void shift_x<T>(const Layout&, T* const*, int, cudaStream_t);                                      \
  template void laser_add<T>(const Layout&, T* const*, const double*, cudaStream_t);                          \
  template void gauss_residual<T>(const Layout&, T* const*, const double*, double, const double[3], Diag64*,   \
                                  cudaStream_t);                                                              \
  template void pack_interior<T>(const Layout&, const T*, double*, cudaStream_t);                             \
  template void unpack_interior<T>(const Layout&, const double*, T*, cudaStream_t);                           \
  template void init_e_gauss_x1<T>(const Layout&, const double*, double, double, T*, cudaStream_t);

PICGB_INST(float)
PICGB_INST(double)

}  // namespace picgb
