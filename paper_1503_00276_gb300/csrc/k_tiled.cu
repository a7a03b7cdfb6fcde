// k_tiled.cu -- FP32 cell-offset form of the particle step, one CTA per tile.
//
// Particles live in per-tile regions of a slot array (structure of arrays):
// a tile's particles that stayed in it during the last step sit at the front
// of its region, those that left it sit at the back, each tagged with the
// direction it left in and its cell relative to the tile it entered.  One
// launch of k_tile_push advances every particle of a tile -- its own stayers
// plus the movers its 26 (3D) or 8 (2D) neighbours tagged for it -- and writes
// them, binned the same way, into the other (ping-pong) slot array.  So the
// per-tile sort costs no separate pass.
//
// Per tile:
//   * one TMA copy stages the E/B stencil of the tile plus halo in shared memory;
//   * gather (eq. 2d-field-weighting-e3, 3D extension), Boris push
//     (eq. momentum-update), position update (eq. 2d-position-update) and the
//     TRISTAN / Villasenor-Buneman deposit run in FP32 on int cell + FP32 offset;
//   * the deposit goes to a shared-memory current tile with shared atomics;
//   * one TMA reduce-add flushes that current tile (with halo) into HBM.
#include "kernels.h"

namespace picgb {

namespace {

constexpr int kThreads = 256;
constexpr int kPPT = 4;                      // particles per thread per chunk
constexpr int kChunk = kThreads * kPPT;      // 1024
constexpr int kIncMax = kChunk;              // incoming-mover list capacity
constexpr long long kWaitLimit = 1ll << 26;  // bounded mbarrier poll

struct TileArgs {
  int nt[3];
  int ntiles;
  const long long* base;
  const int* cap;
  Part32 in;
  const int* in_stay;
  const int* in_move;
  Part32 out;
  int* out_stay;
  int* out_move;
  Flat32 spill;
  int* spill_count;
  long long spill_cap;
  float qmdt2;     // (q/m) dt/2 = dt / (2 rqm)
  float dt_dx[3];  // dt / dx_d
  float cf[3];     // q dx_d / (dt dV): current density per cell-unit of displacement
  float j3f;       // q / dV (2D3V out-of-plane current per unit v3 and time share)
  float e0[3], b0[3];
  int* status;
};

template <int NDIM, int TX, int TY, int TZ>
struct Geo {
  static constexpr int FX = TX + 8, FY = TY + 2, FZ = NDIM == 3 ? TZ + 2 : 1;
  static constexpr int JX = TX + 8, JY = TY + 3, JZ = NDIM == 3 ? TZ + 3 : 1;
  static constexpr int FPL = FX * FY * FZ;
  static constexpr int JPL = JX * JY * JZ;
  static constexpr int FBYTES = 6 * FPL * 4;
  static constexpr int JBYTES = 3 * JPL * 4;
  static constexpr int FOFF = 0;
  static constexpr int JOFF = ((FBYTES + 1023) / 1024) * 1024;
  static constexpr int INCOFF = JOFF + ((JBYTES + 127) / 128) * 128;
  static constexpr int MISCOFF = INCOFF + kIncMax * 8;
  static constexpr int SMEM = MISCOFF + 1024;
};

struct P {
  uint32_t cell;
  float o0, o1, o2;
  float u0, u1, u2;
  int id;
};

__device__ inline float lerp(float a, float b, float w) { return fmaf(w, b - a, a); }

// Trilinear (bilinear in 2D) weighting of one staged component.
template <int NDIM, int FX, int FY>
__device__ inline float interp(const float* F, int ix, int iy, int iz, float wx, float wy, float wz) {
  if (NDIM == 2) {
    const float* r = F + (iy + 1) * FX + (ix + 4);
    float lo = lerp(r[0], r[1], wx);
    float hi = lerp(r[FX], r[FX + 1], wx);
    return lerp(lo, hi, wy);
  } else {
    const float* r = F + ((iz + 1) * FY + (iy + 1)) * FX + (ix + 4);
    constexpr int PL = FX * FY;
    float a0 = lerp(r[0], r[1], wx);
    float a1 = lerp(r[FX], r[FX + 1], wx);
    float b0 = lerp(r[PL], r[PL + 1], wx);
    float b1 = lerp(r[PL + FX], r[PL + FX + 1], wx);
    return lerp(lerp(a0, a1, wy), lerp(b0, b1, wy), wz);
  }
}

// Villasenor-Buneman current of one in-cell segment into the shared tile, 2D3V.
// (cx,cy): the segment's cell relative to the tile; (ax,ay)->(bx,by): its ends
// in cell units relative to that cell; v3frac: v3 times its share of dt.
template <int JX, int JY>
__device__ inline void deposit_seg2(float* J, const TileArgs& A, int cx, int cy, float ax, float ay, float bx,
                                    float by, float v3frac) {
  constexpr int JP = JX * JY;
  float* J1 = J;
  float* J2 = J + JP;
  float* J3 = J + 2 * JP;
  const float dx = bx - ax, dy = by - ay;
  const float mx = 0.5f * (ax + bx), my = 0.5f * (ay + by);
  const int c = (cy + 1) * JX + (cx + 4);
  const float a1 = A.cf[0] * dx, a2 = A.cf[1] * dy;
  atomicAdd(&J1[c], a1 * (1.f - my));
  atomicAdd(&J1[c + JX], a1 * my);
  atomicAdd(&J2[c], a2 * (1.f - mx));
  atomicAdd(&J2[c + 1], a2 * mx);
  const float a3 = A.j3f * v3frac;
  const float cv = dx * dy * (1.f / 12.f);
  atomicAdd(&J3[c], a3 * ((1.f - mx) * (1.f - my) + cv));
  atomicAdd(&J3[c + 1], a3 * (mx * (1.f - my) - cv));
  atomicAdd(&J3[c + JX], a3 * ((1.f - mx) * my - cv));
  atomicAdd(&J3[c + JX + 1], a3 * (mx * my + cv));
}

template <int NDIM, int TX, int TY, int TZ>
__device__ inline void deposit_seg3(float* J, const TileArgs& A, int cx, int cy, int cz, float ax, float ay,
                                    float az, float bx, float by, float bz) {
  using G = Geo<NDIM, TX, TY, TZ>;
  constexpr int SY = G::JX, SZ = G::JX * G::JY;
  float* J1 = J;
  float* J2 = J + G::JPL;
  float* J3 = J + 2 * G::JPL;
  const float dx = bx - ax, dy = by - ay, dz = bz - az;
  const float mx = 0.5f * (ax + bx), my = 0.5f * (ay + by), mz = 0.5f * (az + bz);
  const int c = (cz + 1) * SZ + (cy + 1) * SY + (cx + 4);
  {  // J1: face cx, nodes (cy, cz)
    const float a = A.cf[0] * dx, cv = dy * dz * (1.f / 12.f);
    atomicAdd(&J1[c], a * ((1.f - my) * (1.f - mz) + cv));
    atomicAdd(&J1[c + SY], a * (my * (1.f - mz) - cv));
    atomicAdd(&J1[c + SZ], a * ((1.f - my) * mz - cv));
    atomicAdd(&J1[c + SY + SZ], a * (my * mz + cv));
  }
  {  // J2: face cy, nodes (cz, cx)
    const float a = A.cf[1] * dy, cv = dz * dx * (1.f / 12.f);
    atomicAdd(&J2[c], a * ((1.f - mz) * (1.f - mx) + cv));
    atomicAdd(&J2[c + SZ], a * (mz * (1.f - mx) - cv));
    atomicAdd(&J2[c + 1], a * ((1.f - mz) * mx - cv));
    atomicAdd(&J2[c + SZ + 1], a * (mz * mx + cv));
  }
  {  // J3: face cz, nodes (cx, cy)
    const float a = A.cf[2] * dz, cv = dx * dy * (1.f / 12.f);
    atomicAdd(&J3[c], a * ((1.f - mx) * (1.f - my) + cv));
    atomicAdd(&J3[c + 1], a * (mx * (1.f - my) - cv));
    atomicAdd(&J3[c + SY], a * ((1.f - mx) * my - cv));
    atomicAdd(&J3[c + SY + 1], a * (mx * my + cv));
  }
}

// Gather + push + move + deposit of one particle.  Returns the direction code
// of the tile it ends in (DIR_STAY or a neighbour) and rewrites p in the
// coordinates of that tile.
template <int NDIM, int TX, int TY, int TZ>
__device__ inline int push_one(const float* F, float* J, const TileArgs& A, P& p) {
  using G = Geo<NDIM, TX, TY, TZ>;
  const int lx = p.cell & 255, ly = (p.cell >> 8) & 255, lz = NDIM == 3 ? (p.cell >> 16) & 255 : 0;
  if (lx >= TX || ly >= TY || lz >= TZ) {
    atomicOr(A.status, ST_BADCELL);
    return DIR_STAY;
  }
  // lattice indices and weights for stagger 0 and 1/2 in each direction
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
  e1 += A.e0[0];
  e2 += A.e0[1];
  e3 += A.e0[2];
  b1 += A.b0[0];
  b2 += A.b0[1];
  b3 += A.b0[2];
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
  const float bx = ax + ux * ig2 * A.dt_dx[0];
  const float by = ay + uy * ig2 * A.dt_dx[1];
  const float bz = NDIM == 3 ? az + uz * ig2 * A.dt_dx[2] : 0.f;
  if (!(isfinite(bx) && isfinite(by) && isfinite(bz) && isfinite(ux) && isfinite(uy) && isfinite(uz))) {
    atomicOr(A.status, ST_NONFINITE);
    return DIR_STAY;
  }
  // split the path at the faces it crosses (at most one per direction) and
  // deposit each in-cell piece
  float tcx = 2.f, tcy = 2.f, tcz = 2.f;
  int scx = 0, scy = 0, scz = 0;
  if (bx < 0.f) { tcx = ax / (ax - bx); scx = -1; } else if (bx >= 1.f) { tcx = (1.f - ax) / (bx - ax); scx = 1; }
  if (by < 0.f) { tcy = ay / (ay - by); scy = -1; } else if (by >= 1.f) { tcy = (1.f - ay) / (by - ay); scy = 1; }
  if (NDIM == 3) {
    if (bz < 0.f) { tcz = az / (az - bz); scz = -1; } else if (bz >= 1.f) { tcz = (1.f - az) / (bz - az); scz = 1; }
  }
  const float v3 = uz * ig2;
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
    if (NDIM == 3)
      deposit_seg3<NDIM, TX, TY, TZ>(J, A, lx + ox, ly + oy, lz + oz, p0x - ox, p0y - oy, p0z - oz, p1x - ox,
                                     p1y - oy, p1z - oz);
    else
      deposit_seg2<G::JX, G::JY>(J, A, lx + ox, ly + oy, p0x - ox, p0y - oy, p1x - ox, p1y - oy, v3 * (t1 - t0));
    if (last) break;
    if (w == 0) { ox += scx; tcx = 2.f; }
    if (w == 1) { oy += scy; tcy = 2.f; }
    if (w == 2) { oz += scz; tcz = 2.f; }
    p0x = p1x;
    p0y = p1y;
    p0z = p1z;
    t0 = t1;
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
  p.u1 = uy;
  p.u2 = uz;
  return dir;
}

// Block-wide exclusive scan of one int per thread; returns the total.
__device__ inline int block_excl_scan(int v, int* scratch, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = lane < (kThreads / 32) ? scratch[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < (kThreads / 32)) scratch[lane] = s;
  }
  __syncthreads();
  const int before = warp > 0 ? scratch[warp - 1] : 0;
  total = scratch[kThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

template <int NDIM, int TX, int TY, int TZ>
__device__ inline void store_chunk(const TileArgs& A, int t, long long base, int cap, P (&pp)[kPPT],
                                   int (&dir)[kPPT], int nvalid, int& ws, int& wm, int* scr) {
  int ns = 0, nm = 0;
#pragma unroll
  for (int r = 0; r < kPPT; ++r) {
    if (r < nvalid) {
      if (dir[r] == DIR_STAY)
        ++ns;
      else
        ++nm;
    }
  }
  int S, M;
  int rs = block_excl_scan(ns, scr, S);
  int rm = block_excl_scan(nm, scr + 16, M);
  const int free_slots = cap - ws - wm;
  const int putS = S < free_slots ? S : free_slots;
  const int putM = M < free_slots - putS ? M : free_slots - putS;
#pragma unroll
  for (int r = 0; r < kPPT; ++r) {
    if (r >= nvalid) continue;
    long long slot = -1;
    if (dir[r] == DIR_STAY) {
      if (rs < putS) slot = base + ws + rs;
      ++rs;
    } else {
      if (rm < putM) slot = base + cap - 1 - (wm + rm);
      ++rm;
    }
    const P& q = pp[r];
    if (slot >= 0) {
      A.out.cell[slot] = q.cell;
      A.out.o[0][slot] = q.o0;
      A.out.o[1][slot] = q.o1;
      if (NDIM == 3) A.out.o[2][slot] = q.o2;
      A.out.u[0][slot] = q.u0;
      A.out.u[1][slot] = q.u1;
      A.out.u[2][slot] = q.u2;
      if (A.out.id) A.out.id[slot] = q.id;
    } else {
      // tile region full: park the particle in the spill list, tagged with the
      // tile it belongs to; the host re-bins before the next step
      atomicOr(A.status, ST_SPILL);
      int k = atomicAdd(A.spill_count, 1);
      if (k >= A.spill_cap) {
        atomicOr(A.status, ST_SPILL_LOST);
        continue;
      }
      const int d = dir[r];
      int ti[3] = {t % A.nt[0], (t / A.nt[0]) % A.nt[1], t / (A.nt[0] * A.nt[1])};
      ti[0] = (ti[0] + (d % 3) - 1 + A.nt[0]) % A.nt[0];
      ti[1] = (ti[1] + (d / 3) % 3 - 1 + A.nt[1]) % A.nt[1];
      ti[2] = (ti[2] + d / 9 - 1 + A.nt[2]) % A.nt[2];
      A.spill.tile[k] = (ti[2] * A.nt[1] + ti[1]) * A.nt[0] + ti[0];
      A.spill.cell[k] = (q.cell & 0x00FFFFFFu) | ((uint32_t)DIR_STAY << 24);
      A.spill.o[0][k] = q.o0;
      A.spill.o[1][k] = q.o1;
      A.spill.o[2][k] = q.o2;
      A.spill.u[0][k] = q.u0;
      A.spill.u[1][k] = q.u1;
      A.spill.u[2][k] = q.u2;
      if (A.spill.id) A.spill.id[k] = q.id;
    }
  }
  ws += putS;
  wm += putM;
}

template <int NDIM, int TX, int TY, int TZ>
__global__ void __launch_bounds__(kThreads, 2)
    k_tile_push(const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap jmap, TileArgs A) {
  using G = Geo<NDIM, TX, TY, TZ>;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* F = reinterpret_cast<float*>(smem + G::FOFF);
  float* J = reinterpret_cast<float*>(smem + G::JOFF);
  long long* inc = reinterpret_cast<long long*>(smem + G::INCOFF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + G::MISCOFF);
  int* scr = reinterpret_cast<int*>(smem + G::MISCOFF + 16);        // 32 ints
  int* nbm = reinterpret_cast<int*>(smem + G::MISCOFF + 16 + 128);  // 27 ints: mover counts
  int* nbp = nbm + 32;                                              // 28 ints: prefix
  long long* nbs = reinterpret_cast<long long*>(smem + G::MISCOFF + 512);  // 27 starts

  const int t = blockIdx.x;
  const int tix = t % A.nt[0], tiy = (t / A.nt[0]) % A.nt[1], tiz = t / (A.nt[0] * A.nt[1]);
  const int x0 = tix * TX, y0 = tiy * TY, z0 = tiz * TZ;

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)G::FBYTES);
    if (NDIM == 3)
      tma_load_4d(F, &fmap, bar, x0, y0, z0, 0);
    else
      tma_load_3d(F, &fmap, bar, x0, y0, 0);
  }
  for (int k = threadIdx.x; k < 3 * G::JPL; k += kThreads) J[k] = 0.f;
  // neighbour mover lists: who sends to this tile
  if (threadIdx.x < 27) {
    const int d = threadIdx.x;  // direction from the neighbour to this tile
    int cnt = 0;
    long long start = 0;
    const int ddx = d % 3 - 1, ddy = (d / 3) % 3 - 1, ddz = d / 9 - 1;
    const bool valid = d != DIR_STAY && (NDIM == 3 || ddz == 0);
    if (valid) {
      const int nx_ = (tix - ddx + A.nt[0]) % A.nt[0];
      const int ny_ = (tiy - ddy + A.nt[1]) % A.nt[1];
      const int nz_ = NDIM == 3 ? (tiz - ddz + A.nt[2]) % A.nt[2] : 0;
      const int nb = (nz_ * A.nt[1] + ny_) * A.nt[0] + nx_;
      cnt = A.in_move[nb];
      start = A.base[nb] + A.cap[nb] - cnt;
    }
    nbm[d] = cnt;
    nbs[d] = start;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int d = 0; d < 27; ++d) {
      nbp[d] = run;
      run += nbm[d];
    }
    nbp[27] = run;
  }
  // wait for the staged fields (bounded)
  if (!mbar_wait_bounded(bar, 0, kWaitLimit)) {
    if (threadIdx.x == 0) atomicOr(A.status, ST_TIMEOUT);
    // give the copy a second bounded chance to land before the CTA exits
    mbar_wait_bounded(bar, 0, kWaitLimit);
    return;
  }
  __syncthreads();

  const long long base = A.base[t];
  const int cap = A.cap[t];
  int ws = 0, wm = 0;

  // (1) own stayers: vectorised loads, 4 consecutive particles per thread
  const int nstay = A.in_stay[t];
  for (int c0 = 0; c0 < nstay; c0 += kChunk) {
    P pp[kPPT];
    int dir[kPPT];
    const int first = c0 + threadIdx.x * kPPT;
    int nvalid = nstay - first;
    nvalid = nvalid < 0 ? 0 : (nvalid > kPPT ? kPPT : nvalid);
    if (nvalid > 0) {
      const long long s = base + first;
      const uint4 cl = *reinterpret_cast<const uint4*>(A.in.cell + s);
      const float4 q0 = *reinterpret_cast<const float4*>(A.in.o[0] + s);
      const float4 q1 = *reinterpret_cast<const float4*>(A.in.o[1] + s);
      float4 q2 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (NDIM == 3) q2 = *reinterpret_cast<const float4*>(A.in.o[2] + s);
      const float4 v0 = *reinterpret_cast<const float4*>(A.in.u[0] + s);
      const float4 v1 = *reinterpret_cast<const float4*>(A.in.u[1] + s);
      const float4 v2 = *reinterpret_cast<const float4*>(A.in.u[2] + s);
      int4 idv = make_int4(0, 0, 0, 0);
      if (A.in.id) idv = *reinterpret_cast<const int4*>(A.in.id + s);
      pp[0] = P{cl.x, q0.x, q1.x, q2.x, v0.x, v1.x, v2.x, idv.x};
      pp[1] = P{cl.y, q0.y, q1.y, q2.y, v0.y, v1.y, v2.y, idv.y};
      pp[2] = P{cl.z, q0.z, q1.z, q2.z, v0.z, v1.z, v2.z, idv.z};
      pp[3] = P{cl.w, q0.w, q1.w, q2.w, v0.w, v1.w, v2.w, idv.w};
    }
#pragma unroll
    for (int r = 0; r < kPPT; ++r) dir[r] = r < nvalid ? push_one<NDIM, TX, TY, TZ>(F, J, A, pp[r]) : DIR_STAY;
    store_chunk<NDIM, TX, TY, TZ>(A, t, base, cap, pp, dir, nvalid, ws, wm, scr);
  }

  // (2) incoming movers from the neighbours' lists, compacted into `inc`
  const int ncand = nbp[27];
  int ninc = 0;
  for (int c0 = 0; c0 < ncand; c0 += kThreads) {
    const int k = c0 + threadIdx.x;
    int match = 0;
    long long slot = 0;
    if (k < ncand) {
      int d = 0;
      while (d < 26 && nbp[d + 1] <= k) ++d;
      slot = nbs[d] + (k - nbp[d]);
      match = (int)(A.in.cell[slot] >> 24) == d;
    }
    int tot;
    const int pos = block_excl_scan(match, scr, tot);
    if (ninc + tot > kIncMax) {
      // flush the list before it overflows: process what is queued
      // (all threads take part; the scan above is repeated for this batch)
      __syncthreads();
      for (int c1 = 0; c1 < ninc; c1 += kChunk) {
        P pp[kPPT];
        int dir[kPPT];
        const int first = c1 + threadIdx.x * kPPT;
        int nvalid = ninc - first;
        nvalid = nvalid < 0 ? 0 : (nvalid > kPPT ? kPPT : nvalid);
#pragma unroll
        for (int r = 0; r < kPPT; ++r) {
          if (r < nvalid) {
            const long long s = inc[first + r];
            pp[r] = P{A.in.cell[s] & 0x00FFFFFFu, A.in.o[0][s], A.in.o[1][s], NDIM == 3 ? A.in.o[2][s] : 0.f,
                      A.in.u[0][s], A.in.u[1][s], A.in.u[2][s], A.in.id ? A.in.id[s] : 0};
          }
        }
#pragma unroll
        for (int r = 0; r < kPPT; ++r) dir[r] = r < nvalid ? push_one<NDIM, TX, TY, TZ>(F, J, A, pp[r]) : DIR_STAY;
        store_chunk<NDIM, TX, TY, TZ>(A, t, base, cap, pp, dir, nvalid, ws, wm, scr);
      }
      ninc = 0;
      __syncthreads();
    }
    if (match) inc[ninc + pos] = slot;
    ninc += tot;
    __syncthreads();
  }
  for (int c1 = 0; c1 < ninc; c1 += kChunk) {
    P pp[kPPT];
    int dir[kPPT];
    const int first = c1 + threadIdx.x * kPPT;
    int nvalid = ninc - first;
    nvalid = nvalid < 0 ? 0 : (nvalid > kPPT ? kPPT : nvalid);
#pragma unroll
    for (int r = 0; r < kPPT; ++r) {
      if (r < nvalid) {
        const long long s = inc[first + r];
        pp[r] = P{A.in.cell[s] & 0x00FFFFFFu, A.in.o[0][s], A.in.o[1][s], NDIM == 3 ? A.in.o[2][s] : 0.f,
                  A.in.u[0][s], A.in.u[1][s], A.in.u[2][s], A.in.id ? A.in.id[s] : 0};
      }
    }
#pragma unroll
    for (int r = 0; r < kPPT; ++r) dir[r] = r < nvalid ? push_one<NDIM, TX, TY, TZ>(F, J, A, pp[r]) : DIR_STAY;
    store_chunk<NDIM, TX, TY, TZ>(A, t, base, cap, pp, dir, nvalid, ws, wm, scr);
  }

  if (threadIdx.x == 0) {
    A.out_stay[t] = ws;
    A.out_move[t] = wm;
  }
  // flush the current tile: every thread orders its shared-memory atomics
  // before the async proxy reads them; one thread issues the TMA reduce-add
  fence_proxy_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (NDIM == 3)
      tma_reduce_add_4d(&jmap, J, x0, y0, z0, 0);
    else
      tma_reduce_add_3d(&jmap, J, x0, y0, 0);
    tma_commit();
    tma_wait_read0();
  }
}

// ------------------------------------------------------------ support kernels
__device__ inline void tile_origin(const Tiles& tg, int t, int o[3]) {
  o[0] = (t % tg.nt[0]) * tg.T[0];
  o[1] = ((t / tg.nt[0]) % tg.nt[1]) * tg.T[1];
  o[2] = (t / (tg.nt[0] * tg.nt[1])) * tg.T[2];
}

// tile a packed cell belongs to: the tile itself, or the neighbour its
// direction code names
__device__ inline int dest_tile(const Tiles& tg, int t, uint32_t cell) {
  const int d = (int)(cell >> 24);
  if (d == DIR_STAY) return t;
  int ix = t % tg.nt[0], iy = (t / tg.nt[0]) % tg.nt[1], iz = t / (tg.nt[0] * tg.nt[1]);
  ix = (ix + d % 3 - 1 + tg.nt[0]) % tg.nt[0];
  iy = (iy + (d / 3) % 3 - 1 + tg.nt[1]) % tg.nt[1];
  iz = (iz + d / 9 - 1 + tg.nt[2]) % tg.nt[2];
  return (iz * tg.nt[1] + iy) * tg.nt[0] + ix;
}

__global__ void k_flatten(Tiles tg, Part32 in, const int* stay, const int* move, const long long* out_off,
                          Flat32 out) {
  const int t = blockIdx.x;
  const int ns = stay[t], nm = move[t];
  const long long base = tg.base[t];
  const int cap = tg.cap[t];
  const long long o = out_off[t];
  for (int k = threadIdx.x; k < ns + nm; k += blockDim.x) {
    const long long s = k < ns ? base + k : base + cap - nm + (k - ns);
    const uint32_t c = in.cell[s];
    const long long w = o + k;
    out.tile[w] = dest_tile(tg, t, c);
    out.cell[w] = (c & 0x00FFFFFFu) | ((uint32_t)DIR_STAY << 24);
    out.o[0][w] = in.o[0][s];
    out.o[1][w] = in.o[1][s];
    out.o[2][w] = tg.ndim == 3 ? in.o[2][s] : 0.f;
    out.u[0][w] = in.u[0][s];
    out.u[1][w] = in.u[1][s];
    out.u[2][w] = in.u[2][s];
    if (out.id) out.id[w] = in.id ? in.id[s] : 0;
  }
}

__global__ void k_flat_count(Flat32 f, long long n, int ntiles, int* counts) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int t = f.tile[k];
  if (t >= 0 && t < ntiles) atomicAdd(&counts[t], 1);
}

__global__ void k_flat_scatter(Flat32 f, long long n, Tiles tg, int* cursor, Part32 out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int t = f.tile[k];
  if (t < 0 || t >= tg.ntiles) return;
  const int r = atomicAdd(&cursor[t], 1);
  if (r >= tg.cap[t]) return;  // capacities are sized from the same counts
  const long long s = tg.base[t] + r;
  out.cell[s] = f.cell[k];
  out.o[0][s] = f.o[0][k];
  out.o[1][s] = f.o[1][k];
  if (tg.ndim == 3) out.o[2][s] = f.o[2][k];
  out.u[0][s] = f.u[0][k];
  out.u[1][s] = f.u[1][k];
  out.u[2][s] = f.u[2][k];
  if (out.id) out.id[s] = f.id ? f.id[k] : 0;
}

__global__ void k_flat_to_global(int ndim, Tiles tg, PushConst C, Flat32 f, long long n, double* x, double* u) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int o[3];
  tile_origin(tg, f.tile[k], o);
  const uint32_t c = f.cell[k];
  const int l[3] = {(int)(c & 255), (int)((c >> 8) & 255), (int)((c >> 16) & 255)};
  for (int d = 0; d < 3; ++d) {
    double v = 0.0;
    if (d < ndim) v = C.xmin[d] + ((double)(o[d] + l[d]) + (double)f.o[d][k]) * C.dx[d];
    if (x) x[3 * k + d] = v;
    if (u) u[3 * k + d] = (double)f.u[d][k];
  }
}

// global FP64 position -> tile, packed local cell, FP32 offset
__global__ void k_global_to_flat(int ndim, Layout L, Tiles tg, PushConst C, const double* x0, const double* x1,
                                 const double* x2, const double* u0, const double* u1, const double* u2,
                                 const int* id, long long n, Flat32 out, int* status) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double* xs[3] = {x0, x1, x2};
  const int nn[3] = {L.nx, L.ny, L.nz};
  int cell[3] = {0, 0, 0};
  float off[3] = {0.f, 0.f, 0.f};
  bool ok = true;
  for (int d = 0; d < ndim; ++d) {
    const double v = xs[d][k];
    if (!(v >= C.xmin[d] && v < C.xmin[d] + C.L[d])) {  // outside the box or NaN
      ok = false;
      break;
    }
    const double g = (v - C.xmin[d]) / C.dx[d];
    const double fl = floor(g);
    long long c = (long long)fl;
    float o = (float)(g - fl);
    if (o >= 1.f) {  // FP32 offset rounded up to the next face
      o = 0.f;
      c += 1;
    }
    if (c >= nn[d]) c -= nn[d];
    cell[d] = (int)c;
    off[d] = o;
  }
  if (!ok) {
    atomicOr(status, ST_BADCELL);
    out.tile[k] = -1;
    return;
  }
  const int ti[3] = {cell[0] / tg.T[0], cell[1] / tg.T[1], ndim == 3 ? cell[2] / tg.T[2] : 0};
  const int l[3] = {cell[0] - ti[0] * tg.T[0], cell[1] - ti[1] * tg.T[1], ndim == 3 ? cell[2] - ti[2] * tg.T[2] : 0};
  out.tile[k] = (ti[2] * tg.nt[1] + ti[1]) * tg.nt[0] + ti[0];
  out.cell[k] = (uint32_t)l[0] | ((uint32_t)l[1] << 8) | ((uint32_t)l[2] << 16) | ((uint32_t)DIR_STAY << 24);
  out.o[0][k] = off[0];
  out.o[1][k] = off[1];
  out.o[2][k] = off[2];
  out.u[0][k] = (float)u0[k];
  out.u[1][k] = (float)u1[k];
  out.u[2][k] = (float)u2[k];
  if (out.id) out.id[k] = id ? id[k] : (int)k;
}

// charge density with linear weights (FP64 atomics) of every particle in the store
__global__ void k_tiled_rho(Layout L, PushConst C, Tiles tg, Part32 in, const int* stay, const int* move,
                            double* rho) {
  const int t = blockIdx.x;
  const int ns = stay[t], nm = move[t];
  const long long base = tg.base[t];
  const int cap = tg.cap[t];
  for (int k = threadIdx.x; k < ns + nm; k += blockDim.x) {
    const long long s = k < ns ? base + k : base + cap - nm + (k - ns);
    const uint32_t c = in.cell[s];
    int o[3];
    tile_origin(tg, dest_tile(tg, t, c), o);
    const int i = o[0] + (int)(c & 255), j = o[1] + (int)((c >> 8) & 255), kk = o[2] + (int)((c >> 16) & 255);
    const double e0 = in.o[0][s], e1 = in.o[1][s], e2 = tg.ndim == 3 ? (double)in.o[2][s] : 0.0;
    const double qv = C.q / C.dvol;
    for (int c3 = 0; c3 < (tg.ndim == 3 ? 2 : 1); ++c3)
      for (int c2 = 0; c2 < 2; ++c2)
        for (int c1 = 0; c1 < 2; ++c1) {
          double w = (c1 ? e0 : 1.0 - e0) * (c2 ? e1 : 1.0 - e1);
          if (tg.ndim == 3) w *= (c3 ? e2 : 1.0 - e2);
          atomicAdd(&rho[L.idx(i + c1, j + c2, kk + c3)], qv * w);
        }
  }
}

__global__ void k_tiled_kinetic(PushConst C, Tiles tg, Part32 in, const int* stay, const int* move, double* ke,
                                double* qsum) {
  __shared__ double red[32];
  const int t = blockIdx.x;
  const int ns = stay[t], nm = move[t];
  const long long base = tg.base[t];
  const int cap = tg.cap[t];
  double v = 0.0;
  for (int k = threadIdx.x; k < ns + nm; k += blockDim.x) {
    const long long s = k < ns ? base + k : base + cap - nm + (k - ns);
    const double a = in.u[0][s], b = in.u[1][s], c = in.u[2][s];
    v += C.q * C.rqm * (sqrt(1.0 + a * a + b * b + c * c) - 1.0);
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(ke, s);
    atomicAdd(qsum, C.q * (double)(ns + nm));
  }
}

template <int NDIM, int TX, int TY, int TZ>
void launch_push(const CUtensorMap* fmap, const CUtensorMap* jmap, const TileArgs& A, int ntiles, cudaStream_t s) {
  using G = Geo<NDIM, TX, TY, TZ>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_tile_push<NDIM, TX, TY, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    attr_set = true;
  }
  k_tile_push<NDIM, TX, TY, TZ><<<ntiles, kThreads, G::SMEM, s>>>(*fmap, *jmap, A);
}

}  // namespace

int tiled_push_smem_bytes(int ndim, const int T[3]) {
  if (ndim == 3 && T[0] == 8 && T[1] == 8 && T[2] == 8) return Geo<3, 8, 8, 8>::SMEM;
  if (ndim == 3 && T[0] == 16 && T[1] == 8 && T[2] == 4) return Geo<3, 16, 8, 4>::SMEM;
  if (ndim == 3 && T[0] == 4 && T[1] == 4 && T[2] == 4) return Geo<3, 4, 4, 4>::SMEM;
  if (ndim == 2 && T[0] == 32 && T[1] == 16) return Geo<2, 32, 16, 1>::SMEM;
  if (ndim == 2 && T[0] == 16 && T[1] == 16) return Geo<2, 16, 16, 1>::SMEM;
  if (ndim == 2 && T[0] == 8 && T[1] == 8) return Geo<2, 8, 8, 1>::SMEM;
  return -1;
}

void tiled_push(const Layout& L, const PushConst& C, const Tiles& tg, const Part32& in, const int* in_stay,
                const int* in_move, const Part32& out, int* out_stay, int* out_move, Flat32 spill,
                int* spill_count, long long spill_cap, const CUtensorMap* fmap, const CUtensorMap* jmap,
                int* status, cudaStream_t s) {
  (void)L;
  TileArgs A;
  for (int d = 0; d < 3; ++d) A.nt[d] = tg.nt[d];
  A.ntiles = tg.ntiles;
  A.base = tg.base;
  A.cap = tg.cap;
  A.in = in;
  A.in_stay = in_stay;
  A.in_move = in_move;
  A.out = out;
  A.out_stay = out_stay;
  A.out_move = out_move;
  A.spill = spill;
  A.spill_count = spill_count;
  A.spill_cap = spill_cap;
  A.qmdt2 = (float)(C.dt / (2.0 * C.rqm));
  for (int d = 0; d < 3; ++d) {
    A.dt_dx[d] = (float)(C.dt / C.dx[d]);
    A.cf[d] = (float)(C.q * C.dx[d] / (C.dt * C.dvol));
    A.e0[d] = (float)C.e0[d];
    A.b0[d] = (float)C.b0[d];
  }
  A.j3f = (float)(C.q / C.dvol);
  A.status = status;
  const int* T = tg.T;
  if (tg.ndim == 3 && T[0] == 8 && T[1] == 8 && T[2] == 8)
    launch_push<3, 8, 8, 8>(fmap, jmap, A, tg.ntiles, s);
  else if (tg.ndim == 3 && T[0] == 16 && T[1] == 8 && T[2] == 4)
    launch_push<3, 16, 8, 4>(fmap, jmap, A, tg.ntiles, s);
  else if (tg.ndim == 3 && T[0] == 4 && T[1] == 4 && T[2] == 4)
    launch_push<3, 4, 4, 4>(fmap, jmap, A, tg.ntiles, s);
  else if (tg.ndim == 2 && T[0] == 32 && T[1] == 16)
    launch_push<2, 32, 16, 1>(fmap, jmap, A, tg.ntiles, s);
  else if (tg.ndim == 2 && T[0] == 16 && T[1] == 16)
    launch_push<2, 16, 16, 1>(fmap, jmap, A, tg.ntiles, s);
  else if (tg.ndim == 2 && T[0] == 8 && T[1] == 8)
    launch_push<2, 8, 8, 1>(fmap, jmap, A, tg.ntiles, s);
}

void tiled_flatten(const Tiles& tg, const Part32& in, const int* stay, const int* move, const long long* out_off,
                   Flat32 out, cudaStream_t s) {
  k_flatten<<<tg.ntiles, 256, 0, s>>>(tg, in, stay, move, out_off, out);
}

void flat_count(const Flat32& f, long long n, int ntiles, int* counts, cudaStream_t s) {
  if (n == 0) return;
  k_flat_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, n, ntiles, counts);
}

void flat_scatter(const Flat32& f, long long n, const Tiles& tg, int* cursor, Part32 out, cudaStream_t s) {
  if (n == 0) return;
  k_flat_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, n, tg, cursor, out);
}

void flat_to_global(int ndim, const Tiles& tg, const PushConst& C, const Flat32& f, long long n, double* x, double* u,
                    cudaStream_t s) {
  if (n == 0) return;
  k_flat_to_global<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ndim, tg, C, f, n, x, u);
}

void global_to_flat(int ndim, const Layout& L, const Tiles& tg, const PushConst& C, double* const x[3],
                    double* const u[3], const int* id, long long n, Flat32 out, int* status, cudaStream_t s) {
  if (n == 0) return;
  k_global_to_flat<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ndim, L, tg, C, x[0], x[1], x[2], u[0], u[1], u[2],
                                                                id, n, out, status);
}

void tiled_rho(const Layout& L, const PushConst& C, const Tiles& tg, const Part32& in, const int* stay,
               const int* move, double* rho, cudaStream_t s) {
  k_tiled_rho<<<tg.ntiles, 256, 0, s>>>(L, C, tg, in, stay, move, rho);
}

void tiled_kinetic(const PushConst& C, const Tiles& tg, const Part32& in, const int* stay, const int* move,
                   Diag64* acc, cudaStream_t s) {
  k_tiled_kinetic<<<tg.ntiles, 256, 0, s>>>(C, tg, in, stay, move, &acc->kinetic_energy, &acc->total_charge);
}

}  // namespace picgb
