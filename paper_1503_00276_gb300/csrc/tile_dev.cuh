// tile_dev.cuh -- device helpers of the tile kernels of the FP32 cell-offset
// form (the sorting, compacting, batched and small-tile kernels of k_tiled.cu).
// Internal, not part of the ABI.
#pragma once

#include "kernels.h"

namespace picgb {

struct TileArgs {
  int nt[3];
  int ntiles;
  const long long* base;
  const int* cap;
  const int* res;
  TileSide in;
  TileSide out;
  Flat32 spill;
  int* spill_count;
  long long spill_cap;
  int* work;            // dynamic tile counter
  float qmdt2;          // (q/m) dt/2 = dt / (2 rqm)
  float dt_dx[3];       // dt / dx_d
  float cf[3];          // q dx_d / (dt dV): current density per cell-unit of displacement
  float j3f;            // q / dV (2D3V out-of-plane current per unit v3 and time share)
  int isis;             // 1: ISIS deposit (2D3V): a crossing path's in-plane current is
                        // that of its whole straight path, not split at faces
  float e0[3], b0[3];
  int ext;              // 1: some e0 / b0 component is non-zero
  int* status;
  const int* nslice;    // [ntiles] slices of each tile (nullptr: one work item per tile)
  const int2* extra;    // (tile, slice) of the work items after the first ntiles
  const int* nextra;    // entries of `extra`
  int extra_cap;
  int shift_x;          // moving window: this step ends with a one-cell shift back in x1
  const int* shift_ptr; // batched runs: the member's shift flag of this step in device memory (else null)
  int open_x;           // x1 open: a particle leaving the box in x1 is dropped
  int* lost;            // count of dropped particles
  int cyl;              // 2D r-z mode: x2 = r, rings rotated back into the r-z plane
  int nrow;             // r-z: cell rows; the conducting wall is the upper face of row nrow-1
  float dr, dt;         // r-z: dx2 and dt
};

// Shapes of the general kernel (any particle count per tile) ...
#define PICGB_TILE_SHAPES(X) \
  X(3, 8, 8, 8)              \
  X(3, 16, 8, 4)             \
  X(2, 32, 16, 1)            \
  X(2, 16, 16, 1)            \
  X(2, 8, 8, 1)

namespace {

constexpr int kThreads = 256;
constexpr int kPPT = 2;                      // consecutive particles per thread per chunk
constexpr int kChunk = kThreads * kPPT;      // 512
constexpr int kQCap = 192;                   // crossing queue entries
constexpr uint32_t kHoleCell = 0xFFFFFFFFu;  // cell word of an empty slot
constexpr long long kWaitLimit = 2000000000ll;  // mbarrier waits give up after 2 s
constexpr int kSliceChunks = 8;                // chunks per work item of a heavy tile
constexpr int kDensePerCell = 32;              // particles per cell above which a tile counts as dense



// Shared-memory tiles: fields and current cover local cells [-1, T+3) in x
// (TMA boxes start 16-byte aligned one cell left of the tile), fields
// [-1, T+1) and current [-1, T+2) in y and z.
template <int NDIM, int TX, int TY, int TZ>
struct Geo {
  static constexpr int NC = TX * TY * TZ;
  static constexpr int NK = NC + 1;  // keys: new cell of a stayer, or NC = left the tile
  static constexpr int FX = TX + 4, FY = TY + 2, FZ = NDIM == 3 ? TZ + 2 : 1;
  static constexpr int JX = TX + 4, JY = TY + 3, JZ = NDIM == 3 ? TZ + 3 : 1;
  static constexpr int FPL = FX * FY * FZ;
  static constexpr int JPL = JX * JY * JZ;
  static constexpr int FBYTES = 6 * FPL * 4;
  static constexpr int JBYTES = 3 * JPL * 4;
  static constexpr int QW = NDIM == 3 ? 8 : 7;  // words per queue entry (last: charge weight)
  static constexpr int FOFF = 0;
  static constexpr int JOFF = ((FBYTES + 127) / 128) * 128;
  static constexpr int HOFF = JOFF + ((JBYTES + 127) / 128) * 128;   // hist[NK]
  static constexpr int QOFF = HOFF + ((NK * 4 + 15) / 16) * 16;      // queue
  static constexpr int MOFF = QOFF + ((kQCap * QW * 4 + 15) / 16) * 16;
  static constexpr int NOFF = MOFF + 256;  // the 27 neighbour tiles' regions (Nbr)
  static constexpr int SMEM = NOFF + 27 * 24;
};

struct P {
  uint32_t cell;
  float o0, o1, o2;
  float u0, u1, u2;
  int id;
  float w;  // charge weight (density profile; 1 without one)
};

__device__ inline float lerp(float a, float b, float w) { return fmaf(w, b - a, a); }

// N consecutive 32-bit words from a 4N-byte aligned address, one vector load
template <typename T, int N>
__device__ inline void load_vec(const T* p, T (&v)[N]) {
  static_assert(sizeof(T) == 4 && (N == 1 || N == 2 || N == 4), "32-bit words, 1, 2 or 4 of them");
  if constexpr (N == 4) {
    const uint4 w = *reinterpret_cast<const uint4*>(p);
    v[0] = __builtin_bit_cast(T, w.x);
    v[1] = __builtin_bit_cast(T, w.y);
    v[2] = __builtin_bit_cast(T, w.z);
    v[3] = __builtin_bit_cast(T, w.w);
  } else if constexpr (N == 2) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    v[0] = __builtin_bit_cast(T, w.x);
    v[1] = __builtin_bit_cast(T, w.y);
  } else {
    v[0] = *p;
  }
}

// Trilinear (bilinear in 2D) weighting of one staged component.
template <int NDIM, int FX, int FY>
__device__ inline float interp(const float* F, int ix, int iy, int iz, float wx, float wy, float wz) {
  if (NDIM == 2) {
    const float* r = F + (iy + 1) * FX + (ix + 1);
    return lerp(lerp(r[0], r[1], wx), lerp(r[FX], r[FX + 1], wx), wy);
  } else {
    const float* r = F + ((iz + 1) * FY + (iy + 1)) * FX + (ix + 1);
    constexpr int PL = FX * FY;
    const float a0 = lerp(r[0], r[1], wx);
    const float a1 = lerp(r[FX], r[FX + 1], wx);
    const float b0 = lerp(r[PL], r[PL + 1], wx);
    const float b1 = lerp(r[PL + FX], r[PL + FX + 1], wx);
    return lerp(lerp(a0, a1, wy), lerp(b0, b1, wy), wz);
  }
}

// Villasenor-Buneman weights of one straight in-cell piece a -> b (cell units
// relative to its cell): the flux of the move along d through face cell_d+1/2
// is shared among the transverse nodes with the path-averaged linear weights,
// i.e. the midpoint weights plus the covariance term D_t1 D_t2 / 12.  Order of
// the 12 (3D) / 8 (2D) values: J1 (n,n+y,n+z,n+y+z) J2 (n,n+z,n+x,n+z+x)
// J3 (n,n+x,n+y,n+x+y) in 3D; J1 (n,n+y) J2 (n,n+x) J3 (n,n+x,n+y,n+x+y) in 2D.
template <int NDIM>
__device__ inline void seg_weights(const TileArgs& A, float ax, float ay, float az, float bx, float by, float bz,
                                   float v3frac, float w[12], float q = 1.f) {
  const float dx = bx - ax, dy = by - ay;
  const float mx = 0.5f * (ax + bx), my = 0.5f * (ay + by);
  if (NDIM == 2) {
    const float a1 = A.cf[0] * q * dx, a2 = A.cf[1] * q * dy;
    w[0] = a1 * (1.f - my);
    w[1] = a1 * my;
    w[2] = a2 * (1.f - mx);
    w[3] = a2 * mx;
    const float a3 = A.j3f * q * v3frac;
    const float cv = dx * dy * (1.f / 12.f);
    w[4] = a3 * ((1.f - mx) * (1.f - my) + cv);
    w[5] = a3 * (mx * (1.f - my) - cv);
    w[6] = a3 * ((1.f - mx) * my - cv);
    w[7] = a3 * (mx * my + cv);
  } else {
    // a ((1 - m1)(1 - m2) + c) etc. as fused products: a (1 - m1), a m1 and
    // a c once per component, then one FMA per weight
    const float dz = bz - az, mz = 0.5f * (az + bz);
    const float nx = 1.f - mx, ny = 1.f - my, nz = 1.f - mz;
    const float c12 = 1.f / 12.f;
    float a = A.cf[0] * q * dx, an = a * ny, am = a * my, ac = a * (dy * dz * c12);
    w[0] = fmaf(an, nz, ac);
    w[1] = fmaf(am, nz, -ac);
    w[2] = fmaf(an, mz, -ac);
    w[3] = fmaf(am, mz, ac);
    a = A.cf[1] * q * dy;
    an = a * nz;
    am = a * mz;
    ac = a * (dz * dx * c12);
    w[4] = fmaf(an, nx, ac);
    w[5] = fmaf(am, nx, -ac);
    w[6] = fmaf(an, mx, -ac);
    w[7] = fmaf(am, mx, ac);
    a = A.cf[2] * q * dz;
    an = a * nx;
    am = a * mx;
    ac = a * (dx * dy * c12);
    w[8] = fmaf(an, ny, ac);
    w[9] = fmaf(am, ny, -ac);
    w[10] = fmaf(an, my, -ac);
    w[11] = fmaf(am, my, ac);
  }
}

// Shared-memory atomics of one piece's values at cell (cx,cy,cz) of the tile.
template <int NDIM, int JX, int JY, int JPL>
__device__ inline void flush_cell(float* J, int cx, int cy, int cz, const float w[12]) {
  if (NDIM == 2) {
    const int c = (cy + 1) * JX + (cx + 1);
    atomicAdd(&J[c], w[0]);
    atomicAdd(&J[c + JX], w[1]);
    atomicAdd(&J[JPL + c], w[2]);
    atomicAdd(&J[JPL + c + 1], w[3]);
    atomicAdd(&J[2 * JPL + c], w[4]);
    atomicAdd(&J[2 * JPL + c + 1], w[5]);
    atomicAdd(&J[2 * JPL + c + JX], w[6]);
    atomicAdd(&J[2 * JPL + c + JX + 1], w[7]);
  } else {
    constexpr int SY = JX, SZ = JX * JY;
    const int c = (cz + 1) * SZ + (cy + 1) * SY + (cx + 1);
    atomicAdd(&J[c], w[0]);
    atomicAdd(&J[c + SY], w[1]);
    atomicAdd(&J[c + SZ], w[2]);
    atomicAdd(&J[c + SY + SZ], w[3]);
    atomicAdd(&J[JPL + c], w[4]);
    atomicAdd(&J[JPL + c + SZ], w[5]);
    atomicAdd(&J[JPL + c + 1], w[6]);
    atomicAdd(&J[JPL + c + SZ + 1], w[7]);
    atomicAdd(&J[2 * JPL + c], w[8]);
    atomicAdd(&J[2 * JPL + c + 1], w[9]);
    atomicAdd(&J[2 * JPL + c + SY], w[10]);
    atomicAdd(&J[2 * JPL + c + SY + 1], w[11]);
  }
}

// Face crossings of the path a -> b (cell units): parameter along the path
// (2 = none) and side (+1 / -1) per direction; |b - a| < 1 so at most one
// crossing per direction.
template <int NDIM>
__device__ inline void crossings(float ax, float ay, float az, float bx, float by, float bz, float& tx, float& ty,
                                 float& tz, int& sx, int& sy, int& sz) {
  tx = ty = tz = 2.f;
  sx = sy = sz = 0;
  if (bx < 0.f) { tx = ax / (ax - bx); sx = -1; } else if (bx >= 1.f) { tx = (1.f - ax) / (bx - ax); sx = 1; }
  if (by < 0.f) { ty = ay / (ay - by); sy = -1; } else if (by >= 1.f) { ty = (1.f - ay) / (by - ay); sy = 1; }
  if (NDIM == 3) {
    if (bz < 0.f) { tz = az / (az - bz); sz = -1; } else if (bz >= 1.f) { tz = (1.f - az) / (bz - az); sz = 1; }
  }
}

// Walk the in-cell pieces of a -> b in path order, calling f(k, ox, oy, oz,
// piece start, piece end, time share) for piece k in cell (start cell + o).
template <int NDIM, typename Fn>
__device__ inline void walk(float ax, float ay, float az, float bx, float by, float bz, Fn f) {
  float tcx, tcy, tcz;
  int scx, scy, scz;
  crossings<NDIM>(ax, ay, az, bx, by, bz, tcx, tcy, tcz, scx, scy, scz);
  int ox = 0, oy = 0, oz = 0;
  float p0x = ax, p0y = ay, p0z = az, t0 = 0.f;
#pragma unroll
  for (int m = 0; m <= NDIM; ++m) {
    const float tm = fminf(tcx, fminf(tcy, tcz));
    const bool last = tm >= 1.f;
    float p1x, p1y, p1z, t1;
    int w = -1;
    if (last) {
      t1 = 1.f;
      p1x = bx;
      p1y = by;
      p1z = bz;
    } else {
      t1 = tm;
      w = (tm == tcx) ? 0 : ((tm == tcy) ? 1 : 2);
      p1x = fmaf(t1, bx - ax, ax);
      p1y = fmaf(t1, by - ay, ay);
      p1z = fmaf(t1, bz - az, az);
      if (w == 0) p1x = (float)(ox + (scx > 0));
      if (w == 1) p1y = (float)(oy + (scy > 0));
      if (w == 2) p1z = (float)(oz + (scz > 0));
    }
    f(m, ox, oy, oz, p0x - ox, p0y - oy, p0z - oz, p1x - ox, p1y - oy, p1z - oz, t1 - t0);
    if (last) break;
    if (w == 0) { ox += scx; tcx = 2.f; }
    if (w == 1) { oy += scy; tcy = 2.f; }
    if (w == 2) { oz += scz; tcz = 2.f; }
    p0x = p1x;
    p0y = p1y;
    p0z = p1z;
    t0 = t1;
  }
}

// ISIS deposit (2D3V) of a whole straight path a -> b that starts in tile cell
// (lx, ly) (a, b in cell units relative to that cell): the in-plane current is
// the average of the two orders of orthogonal moves.  A move along x from a_x to
// b_x puts, through the J1 face of column lx + d (d = -1, 0, 1), the part of
// the move inside that column (the change of the linear charge weights it
// causes); the transverse weights are those of the fixed coordinate of the
// move, a_y in one order and b_y in the other, averaged.  Likewise for y.  J3 is
// the time integral along the straight path, the same as TRISTAN's (its pieces).
__device__ inline float lin_w(float s) { return fmaxf(0.f, 1.f - fabsf(s)); }

template <int TX, int TY>
__device__ inline void isis_path(float* J, const TileArgs& A, int lx, int ly, float ax, float ay, float bx,
                                 float by, float v3, float q) {
  using G = Geo<2, TX, TY, 1>;
  const float fx[3] = {fminf(bx, 0.f), fminf(fmaxf(bx, 0.f), 1.f) - ax, fmaxf(bx - 1.f, 0.f)};
  const float fy[3] = {fminf(by, 0.f), fminf(fmaxf(by, 0.f), 1.f) - ay, fmaxf(by - 1.f, 0.f)};
  float wx[4], wy[4];  // nodes -1 .. 2 relative to the start cell
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    wx[m] = 0.5f * (lin_w(ax - (float)(m - 1)) + lin_w(bx - (float)(m - 1)));
    wy[m] = 0.5f * (lin_w(ay - (float)(m - 1)) + lin_w(by - (float)(m - 1)));
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (fx[d] != 0.f && wy[m] != 0.f)  // J1 at (lx + d - 1, ly + m - 1)
        atomicAdd(&J[(ly + m) * G::JX + (lx + d)], A.cf[0] * q * fx[d] * wy[m]);
      if (fy[d] != 0.f && wx[m] != 0.f)  // J2 at (lx + m - 1, ly + d - 1)
        atomicAdd(&J[G::JPL + (ly + d) * G::JX + (lx + m)], A.cf[1] * q * fy[d] * wx[m]);
    }
  }
  walk<2>(ax, ay, 0.f, bx, by, 0.f,
          [&](int k, int ox, int oy, int oz, float sx0, float sy0, float sz0, float sx1, float sy1, float sz1,
              float frac) {
            float w[12];
            seg_weights<2>(A, sx0, sy0, 0.f, sx1, sy1, 0.f, v3 * frac, w, q);
            const int c = 2 * G::JPL + (ly + oy + 1) * G::JX + (lx + ox + 1);
            atomicAdd(&J[c], w[4]);
            atomicAdd(&J[c + 1], w[5]);
            atomicAdd(&J[c + G::JX], w[6]);
            atomicAdd(&J[c + G::JX + 1], w[7]);
          });
}

// Per-thread accumulator of first pieces that start in the same cell.
struct Acc {
  float w[12];
  int cell;  // packed local cell, -1 = empty
};

template <int NDIM, int TX, int TY, int TZ>
__device__ inline void acc_flush(float* J, Acc& a) {
  using G = Geo<NDIM, TX, TY, TZ>;
  if (a.cell >= 0) {
    flush_cell<NDIM, G::JX, G::JY, G::JPL>(J, a.cell & 255, (a.cell >> 8) & 255, (a.cell >> 16) & 255, a.w);
#pragma unroll
    for (int k = 0; k < 12; ++k) a.w[k] = 0.f;
  }
  a.cell = -1;
}

// Adds each active lane's 12 values at its cell, given as the code
// (x + 1) | (y + 1) << 8 | (z + 1) << 16 of tile-local cell coordinates (a
// piece may lie in the halo cells -1 and T).  Called by all 32 lanes of the
// warp.  A shared-memory FP32 add is a compare-and-swap loop that
// retries once per lane on the same word, so where several lanes hold the same
// cell (a dense beam puts a whole warp on one cell) their values are first
// summed across the warp and one lane adds them; lanes alone or in pairs on a
// cell add directly.
constexpr int kAggMin = 3;  // lanes on one cell from which the warp sums first

template <int NDIM, int TX, int TY, int TZ>
__device__ inline void flush_warp(float* J, bool act, int cell, const float (&w)[12]) {
  using G = Geo<NDIM, TX, TY, TZ>;
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(kFull, act ? cell : -1);
  const bool big = act && __popc(peers) >= kAggMin;
  if (act && !big)
    flush_cell<NDIM, G::JX, G::JY, G::JPL>(J, (cell & 255) - 1, ((cell >> 8) & 255) - 1, ((cell >> 16) & 255) - 1, w);
  unsigned lead = __ballot_sync(kFull, big && (__ffs(peers) - 1) == lane);
  while (lead) {  // one round per crowded cell
    const int L = __ffs(lead) - 1;
    lead &= lead - 1;
    const int c = __shfl_sync(kFull, cell, L);
    const bool mine = big && cell == c;
    float v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = mine ? w[k] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < (NDIM == 3 ? 12 : 8); ++k) v[k] += __shfl_xor_sync(kFull, v[k], o);
    }
    if (lane == L)
      flush_cell<NDIM, G::JX, G::JY, G::JPL>(J, (c & 255) - 1, ((c >> 8) & 255) - 1, ((c >> 16) & 255) - 1, v);
  }
}

// Lanes hold runs of equal cells (stayers arrive sorted by cell): each lane's
// accumulator is summed into the first lane of its run (segmented suffix sums
// in log steps, as many as the longest run needs); the other lanes are emptied.
template <int NDIM>
__device__ inline void acc_merge_runs(Acc& a) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int up1 = __shfl_down_sync(kFull, a.cell, 1);
  const int dn1 = __shfl_up_sync(kFull, a.cell, 1);
  const unsigned ends = __ballot_sync(kFull, lane == 31 || a.cell < 0 || up1 != a.cell);
  const int e = __ffs(ends & (kFull << lane)) - 1;  // last lane of my run
  const bool head = lane == 0 || a.cell < 0 || dn1 != a.cell;
  const int maxlen = (int)__reduce_max_sync(kFull, head ? (unsigned)(e - lane + 1) : 1u);
  for (int s = 1; s < maxlen; s <<= 1) {
#pragma unroll
    for (int k = 0; k < (NDIM == 3 ? 12 : 8); ++k) {
      const float v = __shfl_down_sync(kFull, a.w[k], s);
      if (lane + s <= e) a.w[k] += v;
    }
  }
  if (!head) a.cell = -1;
}

// acc_flush for a whole warp (all lanes call it)
template <int NDIM, int TX, int TY, int TZ>
__device__ inline void acc_flush_warp(float* J, Acc& a) {
  flush_warp<NDIM, TX, TY, TZ>(J, a.cell >= 0, a.cell + 0x010101, a.w);
#pragma unroll
  for (int k = 0; k < 12; ++k) a.w[k] = 0.f;
  a.cell = -1;
}

// Gather + push + move of one particle, deposit of its first in-cell piece into
// the accumulator, crossing pieces queued.  Rewrites p in the coordinates of
// the tile it ends in; returns its key: new cell (stayers) or NC + direction.
// The first half of a particle's step: gather (eq. 2d-field-weighting-e3 and
// its 3D extension), relativistic Boris push (eq. momentum-update) and
// position update (eq. 2d-position-update; r-z: the ring move of ch. 3), in
// straight-line code without memory writes, so that a thread's particles can
// be advanced side by side before any of them deposits.  A particle whose cell
// word is corrupt is gathered at a clamped cell and flagged; the flags are
// reported by deposit_one.
struct Adv {
  float ax, ay, az, bx, by, bz;  // path in cell units relative to the start cell
  float ux, uy, uz;              // u^{n+1/2} (r-z: Cartesian at the start, before the rotation)
  float un1, un2;                // r-z: momenta after the rotation into the new r-z plane
  float v3;                      // out-of-plane velocity times the time share up to the wall (r-z)
  int lx, ly, lz;
  int bad;                       // 1: corrupt cell word, 2: non-finite result
  bool absorbed;                 // r-z: the ring reached the wall
};

template <int NDIM, int TX, int TY, int TZ, bool CYL = false>
__device__ inline Adv advance_one(const float* F, const TileArgs& A, const P& p, int row0 = 0) {
  using G = Geo<NDIM, TX, TY, TZ>;
  Adv a;
  int lx = p.cell & 255, ly = (p.cell >> 8) & 255, lz = NDIM == 3 ? (p.cell >> 16) & 255 : 0;
  a.bad = (lx >= TX || ly >= TY || lz >= TZ) ? 1 : 0;
  lx = min(lx, TX - 1);  // keeps the stencil reads inside the staged tile
  ly = min(ly, TY - 1);
  lz = min(lz, TZ - 1);
  a.lx = lx;
  a.ly = ly;
  a.lz = lz;
  const bool hx = p.o0 < 0.5f, hy = p.o1 < 0.5f, hz = p.o2 < 0.5f;
  const int x1 = lx - hx, y1 = ly - hy, z1 = lz - hz;
  const float wx1 = hx ? p.o0 + 0.5f : p.o0 - 0.5f;
  const float wy1 = hy ? p.o1 + 0.5f : p.o1 - 0.5f;
  const float wz1 = hz ? p.o2 + 0.5f : p.o2 - 0.5f;
  constexpr int FX = G::FX, FY = G::FY, FP = G::FPL;
  float e1, e2, e3, b1, b2, b3;
  if (NDIM == 3) {
    e1 = interp<3, FX, FY>(F + 0 * FP, x1, ly, lz, wx1, p.o1, p.o2);
    e2 = interp<3, FX, FY>(F + 1 * FP, lx, y1, lz, p.o0, wy1, p.o2);
    e3 = interp<3, FX, FY>(F + 2 * FP, lx, ly, z1, p.o0, p.o1, wz1);
    b1 = interp<3, FX, FY>(F + 3 * FP, lx, y1, z1, p.o0, wy1, wz1);
    b2 = interp<3, FX, FY>(F + 4 * FP, x1, ly, z1, wx1, p.o1, wz1);
    b3 = interp<3, FX, FY>(F + 5 * FP, x1, y1, lz, wx1, wy1, p.o2);
  } else {
    e1 = interp<2, FX, FY>(F + 0 * FP, x1, ly, 0, wx1, p.o1, 0.f);
    e2 = interp<2, FX, FY>(F + 1 * FP, lx, y1, 0, p.o0, wy1, 0.f);
    e3 = interp<2, FX, FY>(F + 2 * FP, lx, ly, 0, p.o0, p.o1, 0.f);
    b1 = interp<2, FX, FY>(F + 3 * FP, lx, y1, 0, p.o0, wy1, 0.f);
    b2 = interp<2, FX, FY>(F + 4 * FP, x1, ly, 0, wx1, p.o1, 0.f);
    b3 = interp<2, FX, FY>(F + 5 * FP, x1, y1, 0, wx1, wy1, 0.f);
  }
  if (A.ext) {  // constant external fields (uniform branch)
    e1 += A.e0[0];
    e2 += A.e0[1];
    e3 += A.e0[2];
    b1 += A.b0[0];
    b2 += A.b0[1];
    b3 += A.b0[2];
  }
  // Boris push
  const float al = A.qmdt2;
  const float p1x = fmaf(al, e1, p.u0), p1y = fmaf(al, e2, p.u1), p1z = fmaf(al, e3, p.u2);
  const float ig = rsqrtf(1.f + p1x * p1x + p1y * p1y + p1z * p1z);
  const float tx = al * b1 * ig, ty = al * b2 * ig, tz = al * b3 * ig;
  const float p2x = p1x + (p1y * tz - p1z * ty);
  const float p2y = p1y + (p1z * tx - p1x * tz);
  const float p2z = p1z + (p1x * ty - p1y * tx);
  const float sf = __fdividef(2.f, 1.f + tx * tx + ty * ty + tz * tz);
  const float sx = tx * sf, sy = ty * sf, sz = tz * sf;
  const float ux = p1x + (p2y * sz - p2z * sy) + al * e1;
  const float uy = p1y + (p2z * sx - p2x * sz) + al * e2;
  const float uz = p1z + (p2x * sy - p2y * sx) + al * e3;
  // position update in cell units
  const float ig2 = rsqrtf(1.f + ux * ux + uy * uy + uz * uz);
  const float ax = p.o0, ay = p.o1, az = NDIM == 3 ? p.o2 : 0.f;
  float bx = ax + ux * ig2 * A.dt_dx[0];
  float by = ay + uy * ig2 * A.dt_dx[1];
  const float bz = NDIM == 3 ? az + uz * ig2 * A.dt_dx[2] : 0.f;
  // r-z (thesis ch. 3, 2D cylindrically symmetric position update): the ring
  // moves in 3D from (r, 0) by (dt v_r, dt v_theta) and is rotated back into
  // the r-z plane; p_r is the momentum along the new radius and r p_theta is
  // conserved.  The radial step r' - r is formed without cancellation.  A
  // ring reaching the wall (upper face of the last row) is absorbed: its path
  // is cut there.
  float un1 = uy, un2 = uz, tclip = 1.f;
  bool absorbed = false;
  if constexpr (CYL) {
    const float r = ((float)(row0 + ly) + ay - 0.5f) * A.dr;
    const float d2 = uy * ig2 * A.dt, d3 = uz * ig2 * A.dt;
    const float x2 = r + d2, rn = sqrtf(x2 * x2 + d3 * d3);
    if (rn > 0.f) {
      by = ay + (d2 * (r + x2) + d3 * d3) / ((r + rn) * A.dr);
      un1 = (uy * x2 + uz * d3) / rn;
      un2 = uz * r / rn;
    } else {
      by = ay - r / A.dr;
      un1 = sqrtf(uy * uy + uz * uz);
      un2 = 0.f;
    }
    const float top = (float)(A.nrow - row0 - ly);  // the wall, in this cell's units
    if (by >= top) {
      tclip = (top - ay) / (by - ay);
      bx = fmaf(tclip, bx - ax, ax);
      by = top;
      absorbed = true;
    }
  }
  // one test for all six: a NaN or an infinity in any of them makes the sum non-finite
  if (!isfinite(((bx + by) + bz) + ((ux + uy) + uz)) && !a.bad) a.bad = 2;
  a.ax = ax;
  a.ay = ay;
  a.az = az;
  a.bx = bx;
  a.by = by;
  a.bz = bz;
  a.ux = ux;
  a.uy = uy;
  a.uz = uz;
  a.un1 = un1;
  a.un2 = un2;
  a.v3 = uz * ig2 * tclip;  // r-z: v_theta before the rotation, for the time up to the wall
  a.absorbed = absorbed;
  return a;
}

// The second half: report flags, deposit the first in-cell piece of the path
// into the accumulator and queue the rest, new cell and offset; rewrites p in
// the coordinates of the tile it ends in and returns its key (new cell for
// stayers, NC for leavers, NK when dropped).
template <int NDIM, int TX, int TY, int TZ, int QCAP = kQCap, bool CYL = false>
__device__ inline int deposit_one(float* J, const TileArgs& A, P& p, const Adv& ad, Acc& acc, float* Q, int* qn) {
  using G = Geo<NDIM, TX, TY, TZ>;
  const int lx = ad.lx, ly = ad.ly, lz = ad.lz;
  const int cellp = lx | (ly << 8) | (lz << 16);
  if (ad.bad == 1) {
    atomicOr(A.status, ST_BADCELL);
    p.cell = kHoleCell;
    return G::NK;  // dropped
  }
  if (ad.bad == 2) {
    atomicOr(A.status, ST_NONFINITE);
    p.cell = cellp | ((uint32_t)DIR_STAY << 24);
    return lx + TX * (ly + TY * lz);  // kept in place, not advanced
  }
  const float ax = ad.ax, ay = ad.ay, az = ad.az, bx = ad.bx, by = ad.by, bz = ad.bz;
  const float ux = ad.ux, uy = ad.uy, uz = ad.uz, un1 = ad.un1, un2 = ad.un2;
  const bool absorbed = ad.absorbed;
  const float v3 = ad.v3;
  // first in-cell piece into the accumulator; later pieces to the queue
  float tcx, tcy, tcz;
  int scx, scy, scz;
  crossings<NDIM>(ax, ay, az, bx, by, bz, tcx, tcy, tcz, scx, scy, scz);
  const float tm = fminf(tcx, fminf(tcy, tcz));
  {
    float p1x = bx, p1y = by, p1z = bz, t1 = 1.f;
    if (tm < 1.f) {
      t1 = tm;
      const int w = (tm == tcx) ? 0 : ((tm == tcy) ? 1 : 2);
      p1x = fmaf(t1, bx - ax, ax);
      p1y = fmaf(t1, by - ay, ay);
      p1z = fmaf(t1, bz - az, az);
      if (w == 0) p1x = (float)(scx > 0);
      if (w == 1) p1y = (float)(scy > 0);
      if (w == 2) p1z = (float)(scz > 0);
    }
    if (!(NDIM == 2 && A.isis && tm < 1.f)) {  // an ISIS crossing path is deposited whole below
      if (acc.cell != cellp) {
        acc_flush<NDIM, TX, TY, TZ>(J, acc);
        acc.cell = cellp;
      }
      float w[12];
      seg_weights<NDIM>(A, ax, ay, az, p1x, p1y, p1z, v3 * t1, w, p.w);
#pragma unroll
      for (int k = 0; k < (NDIM == 3 ? 12 : 8); ++k) acc.w[k] += w[k];
    }
  }
  if (tm < 1.f) {
    const int q = atomicAdd(qn, 1);
    if (q < QCAP) {
      float* e = Q + q * G::QW;
      e[0] = __int_as_float(cellp);
      e[1] = ax;
      e[2] = ay;
      e[3] = bx;
      e[4] = by;
      if (NDIM == 3) {
        e[5] = az;
        e[6] = bz;
      } else {
        e[5] = v3;
      }
      e[G::QW - 1] = p.w;
    } else {
      // queue full: deposit the remaining pieces here
      const float pw = p.w;
      if (NDIM == 2 && A.isis)
        isis_path<TX, TY>(J, A, lx, ly, ax, ay, bx, by, v3, pw);
      else
      walk<NDIM>(ax, ay, az, bx, by, bz,
                 [&](int k, int ox, int oy, int oz, float sx0, float sy0, float sz0, float sx1, float sy1, float sz1,
                     float frac) {
                   if (k == 0) return;
                   float w[12];
                   seg_weights<NDIM>(A, sx0, sy0, sz0, sx1, sy1, sz1, v3 * frac, w, pw);
                   flush_cell<NDIM, G::JX, G::JY, G::JPL>(J, lx + ox, ly + oy, lz + oz, w);
                 });
    }
  }
  if constexpr (CYL) {
    if (absorbed) {
      atomicAdd(A.lost, 1);
      p.cell = kHoleCell;
      return G::NK;  // absorbed at the wall
    }
  }
  // new cell and offset
  int cx = 0, cy = 0, cz = 0;
  float nx = bx, ny = by, nz = bz;
  if (nx < 0.f) { nx += 1.f; cx = -1; } else if (nx >= 1.f) { nx -= 1.f; cx = 1; }
  if (nx >= 1.f) { nx = 0.f; cx += 1; }
  if (ny < 0.f) { ny += 1.f; cy = -1; } else if (ny >= 1.f) { ny -= 1.f; cy = 1; }
  if (ny >= 1.f) { ny = 0.f; cy += 1; }
  if (NDIM == 3) {
    if (nz < 0.f) { nz += 1.f; cz = -1; } else if (nz >= 1.f) { nz -= 1.f; cz = 1; }
    if (nz >= 1.f) { nz = 0.f; cz += 1; }
  }
  cx -= A.shift_ptr ? *A.shift_ptr : A.shift_x;  // moving window: the cell grid moves one cell forward
  int gx = lx + cx, gy = ly + cy, gz = lz + cz;
  const int dx_ = gx < 0 ? -1 : (gx >= TX ? 1 : 0);
  const int dy_ = gy < 0 ? -1 : (gy >= TY ? 1 : 0);
  const int dz_ = NDIM == 3 ? (gz < 0 ? -1 : (gz >= TZ ? 1 : 0)) : 0;
  gx -= dx_ * TX;
  gy -= dy_ * TY;
  gz -= dz_ * TZ;
  const int dir = (dx_ + 1) + 3 * (dy_ + 1) + 9 * (dz_ + 1);
  p.cell = (uint32_t)gx | ((uint32_t)gy << 8) | ((uint32_t)gz << 16) | ((uint32_t)dir << 24);
  p.o0 = nx;
  p.o1 = ny;
  p.o2 = NDIM == 3 ? nz : 0.f;
  p.u0 = ux;
  p.u1 = CYL ? un1 : uy;
  p.u2 = CYL ? un2 : uz;
  return dir == DIR_STAY ? gx + TX * (gy + TY * gz) : G::NC;
}

// Gather + push + move of one particle, deposit of its first in-cell piece into
// the accumulator, crossing pieces queued (advance_one then deposit_one).
template <int NDIM, int TX, int TY, int TZ, int QCAP = kQCap, bool CYL = false>
__device__ inline int push_one(const float* F, float* J, const TileArgs& A, P& p, Acc& acc, float* Q, int* qn,
                               int row0 = 0) {
  const Adv a = advance_one<NDIM, TX, TY, TZ, CYL>(F, A, p, row0);
  return deposit_one<NDIM, TX, TY, TZ, QCAP, CYL>(J, A, p, a, acc, Q, qn);
}

// Deposit the queued crossing pieces (all but the first of each path).  All
// threads of the block call it, one entry per thread and round.  AGG (dense
// tiles, where the paths queued together share their cells): the second piece
// of each path goes through flush_warp; otherwise every piece is added
// directly.
template <int NDIM, int TX, int TY, int TZ, bool AGG = false>
__device__ inline void drain_queue(float* J, const TileArgs& A, const float* Q, int n) {
  using G = Geo<NDIM, TX, TY, TZ>;
  for (int q0 = 0; q0 < n; q0 += kThreads) {
    const int q = q0 + threadIdx.x;
    float w1[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) w1[k] = 0.f;
    int c1 = -1;
    if (q < n) {
      const float* e = Q + q * G::QW;
      const int c = __float_as_int(e[0]);
      const int lx = c & 255, ly = (c >> 8) & 255, lz = (c >> 16) & 255;
      const float ax = e[1], ay = e[2], bx = e[3], by = e[4];
      const float az = NDIM == 3 ? e[5] : 0.f, bz = NDIM == 3 ? e[6] : 0.f;
      const float v3 = NDIM == 3 ? 0.f : e[5];
      const float pw = e[G::QW - 1];
      if (NDIM == 2 && A.isis)
        isis_path<TX, TY>(J, A, lx, ly, ax, ay, bx, by, v3, pw);
      else
      walk<NDIM>(ax, ay, az, bx, by, bz,
                 [&](int k, int ox, int oy, int oz, float sx0, float sy0, float sz0, float sx1, float sy1, float sz1,
                     float frac) {
                   if (k == 0) return;
                   if (AGG && k == 1) {
                     seg_weights<NDIM>(A, sx0, sy0, sz0, sx1, sy1, sz1, v3 * frac, w1, pw);
                     c1 = (lx + ox + 1) | ((ly + oy + 1) << 8) | ((lz + oz + 1) << 16);
                     return;
                   }
                   float w[12];
                   seg_weights<NDIM>(A, sx0, sy0, sz0, sx1, sy1, sz1, v3 * frac, w, pw);
                   flush_cell<NDIM, G::JX, G::JY, G::JPL>(J, lx + ox, ly + oy, lz + oz, w);
                 });
    }
    if (AGG) flush_warp<NDIM, TX, TY, TZ>(J, c1 >= 0, c1, w1);
  }
}

__device__ inline void spill_put(const TileArgs& A, int tile, const P& q) {
  atomicOr(A.status, ST_SPILL);
  const int k = atomicAdd(A.spill_count, 1);
  if (k >= A.spill_cap) {
    atomicOr(A.status, ST_SPILL_LOST);
    return;
  }
  A.spill.tile[k] = tile;
  A.spill.cell[k] = (q.cell & 0x00FFFFFFu) | ((uint32_t)DIR_STAY << 24);
  A.spill.o[0][k] = q.o0;
  A.spill.o[1][k] = q.o1;
  A.spill.o[2][k] = q.o2;
  A.spill.u[0][k] = q.u0;
  A.spill.u[1][k] = q.u1;
  A.spill.u[2][k] = q.u2;
  if (A.spill.id) A.spill.id[k] = q.id;
  if (A.spill.w) A.spill.w[k] = q.w;
}

template <int NDIM>
__device__ inline void store_particle(const Part32& o, long long s, const P& q) {
  o.cell[s] = q.cell;
  o.o[0][s] = q.o0;
  o.o[1][s] = q.o1;
  if (NDIM == 3) o.o[2][s] = q.o2;
  o.u[0][s] = q.u0;
  o.u[1][s] = q.u1;
  o.u[2][s] = q.u2;
  if (o.id) o.id[s] = q.id;
  if (o.w) o.w[s] = q.w;
}

// Region of one of the 27 tiles around (and including) the current one, by
// direction code (dx+1) + 3(dy+1) + 9(dz+1).
struct Nbr {
  long long base;
  int cap, res, tile, pad;
};

// Thread d < 27 of the block: the region of neighbour d of tile (tix, tiy, tiz).
__device__ inline void load_neighbour(const TileArgs& A, int tix, int tiy, int tiz, Nbr* nb) {
  const int d = threadIdx.x;
  if (d < 27) {
    if (A.open_x && (tix + d % 3 - 1 < 0 || tix + d % 3 - 1 >= A.nt[0])) {
      nb[d].tile = -1;  // beyond an open x1 boundary
      return;
    }
    const int ix = (tix + d % 3 - 1 + A.nt[0]) % A.nt[0];
    const int iy = (tiy + (d / 3) % 3 - 1 + A.nt[1]) % A.nt[1];
    const int iz = (tiz + d / 9 - 1 + A.nt[2]) % A.nt[2];
    const int dt_ = (iz * A.nt[1] + iy) * A.nt[0] + ix;
    nb[d].tile = dt_;
    nb[d].base = A.base[dt_];
    nb[d].cap = A.cap[dt_];
    nb[d].res = A.res[dt_];
  }
}

// A particle that left tile (tix, tiy, tiz): appended, with one global atomic,
// to the arrival slots at the back of its new tile's output region (spill
// list when they are full).  nb: the neighbour regions in shared memory, or
// nullptr to look them up in global memory.
template <int NDIM>
__device__ inline void store_leaver(const TileArgs& A, int tix, int tiy, int tiz, const P& q,
                                    const Nbr* nb = nullptr) {
  const int dir = (int)(q.cell >> 24);
  P q2 = q;
  q2.cell = (q.cell & 0x00FFFFFFu) | ((uint32_t)DIR_STAY << 24);
  if (nb) {
    const Nbr& n = nb[dir];
    if (n.tile < 0) {  // left through an open x1 boundary
      atomicAdd(A.lost, 1);
      return;
    }
    const int slot = atomicAdd(&A.out.inc[n.tile], 1);
    if (slot < n.res)
      store_particle<NDIM>(A.out.p, n.base + n.cap - 1 - slot, q2);
    else
      spill_put(A, n.tile, q2);
    return;
  }
  if (A.open_x && (tix + dir % 3 - 1 < 0 || tix + dir % 3 - 1 >= A.nt[0])) {
    atomicAdd(A.lost, 1);
    return;
  }
  const int ix = (tix + dir % 3 - 1 + A.nt[0]) % A.nt[0];
  const int iy = (tiy + (dir / 3) % 3 - 1 + A.nt[1]) % A.nt[1];
  const int iz = (tiz + dir / 9 - 1 + A.nt[2]) % A.nt[2];
  const int dt_ = (iz * A.nt[1] + iy) * A.nt[0] + ix;
  const int slot = atomicAdd(&A.out.inc[dt_], 1);
  if (slot < A.res[dt_])
    store_particle<NDIM>(A.out.p, A.base[dt_] + A.cap[dt_] - 1 - slot, q2);
  else
    spill_put(A, dt_, q2);
}

// base pointer of staged array a of a particle buffer: cell, o1..o3, u1..u3, id, w
__device__ inline void* arr_ptr(const Part32& p, int a) {
  switch (a) {
    case 0: return p.cell;
    case 1: return p.o[0];
    case 2: return p.o[1];
    case 3: return p.o[2];
    case 4: return p.u[0];
    case 5: return p.u[1];
    case 6: return p.u[2];
    case 7: return p.id;
    default: return p.w;
  }
}

}  // namespace
}  // namespace picgb
