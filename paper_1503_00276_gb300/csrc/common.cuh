// common.cuh -- internal device/host helpers of libpicgb (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/pic.h"

namespace picgb {

// ---------------------------------------------------------------------------
// Field storage: one component = a padded [NZ][NY][NX] plane with guard cells.
// Interior cell (i,j,k), 0 <= i < nx, lives at ((k+gz)*NY + (j+gy))*NX + (i+gx).
// Guards: x 1 below / 3 above, y and z 1 below / 2 above (the deposit reaches
// one node beyond the first neighbour cell).  With one guard cell below, the
// TMA box of a tile starting at cell x0 - 1 starts at padded column x0, a
// multiple of 4 floats, as a TMA copy requires; the 3 cells above make the
// padded row a multiple of 4 floats too.  2D: no z guards, NZ = 1.
// ---------------------------------------------------------------------------
constexpr int GX_LO = 1, GX_HI = 3, GY_LO = 1, GY_HI = 2;

struct Layout {
  int ndim;
  int nx, ny, nz;
  int gx, gy, gz;         // guard widths below
  int NX, NY, NZ;         // padded extents
  long long plane;        // elements per component
  int open_x;             // 1: x1 is open (moving window): guards beyond x1 hold 0, no wrap

  __host__ __device__ inline long long idx(int i, int j, int k) const {
    return ((long long)(k + gz) * NY + (j + gy)) * NX + (i + gx);
  }
};

inline Layout make_layout(int ndim, const int nx[3]) {
  Layout L;
  L.ndim = ndim;
  L.nx = nx[0];
  L.ny = nx[1];
  L.nz = ndim == 3 ? nx[2] : 1;
  L.gx = GX_LO;
  L.gy = GY_LO;
  L.gz = ndim == 3 ? GY_LO : 0;
  L.NX = L.nx + GX_LO + GX_HI;
  L.NY = L.ny + GY_LO + GY_HI;
  L.NZ = ndim == 3 ? L.nz + GY_LO + GY_HI : 1;
  L.plane = (long long)L.NX * L.NY * L.NZ;
  L.open_x = 0;
  return L;
}

// Status word bits shared by every kernel (device int, polled by the host).
enum : int { ST_NONFINITE = 1, ST_SPILL = 2, ST_SPILL_LOST = 4, ST_TIMEOUT = 8, ST_BADCELL = 16 };

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood 2014): draw c of stream `seed`.
// ---------------------------------------------------------------------------
__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ inline double uniform01(uint64_t seed, uint64_t c) {
  return (double)(splitmix64(seed, c) >> 11) * (1.0 / 9007199254740992.0);
}

// Box-Muller, cos branch, draws 2c and 2c+1.
__device__ inline double normal_dev(uint64_t seed, uint64_t c) {
  double u1 = 1.0 - uniform01(seed, 2ull * c);
  double u2 = uniform01(seed, 2ull * c + 1ull);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
}

// ---------------------------------------------------------------------------
// TMA / mbarrier wrappers (inline PTX, sm_90+ forms that sm_103a keeps).
// ---------------------------------------------------------------------------
__device__ inline uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ inline uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: gives up after limit_ns nanoseconds and returns false.
__device__ inline bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((long long)(global_ns() - t0) > limit_ns) return false;
  }
}

__device__ inline void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ inline void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ inline void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ inline void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                   int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ inline void tma_reduce_add_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
      : "memory");
}

__device__ inline void tma_reduce_add_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.4d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
      : "memory");
}

// 1D bulk copies (no tensor map): both addresses 16-byte aligned, size a
// multiple of 16 bytes.
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ inline void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}

// L2 prefetch of `bytes` bytes at `src` (both multiples of 16)
__device__ inline void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// 4-byte global -> shared copy without a register round trip (LDGSTS); many
// may be in flight per thread until cp_async_wait0
__device__ inline void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ inline void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ inline void tma_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ inline void tma_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ inline void tma_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ inline void tma_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Atomic max of a non-negative double through its bit pattern.
__device__ inline void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), static_cast<unsigned long long>(__double_as_longlong(v)));
}

}  // namespace picgb
