// k_sort.cu -- prefix sums and the stateless tile binning entry point.
#include <mutex>
#include <string>

#include "kernels.h"

namespace picgb {

void set_error(const std::string& msg);  // api.cu

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

// Exclusive scan of one 2048-element tile per block; block totals to `sums`.
template <typename Tin>
__global__ void k_scan_tile(const Tin* in, long long* out, long long n, long long* sums) {
  __shared__ long long warp_tot[kScanThreads / 32];
  const long long b0 = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  long long v[kScanItems];
  long long run = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    const long long k = b0 + r;
    v[r] = k < n ? (long long)in[k] : 0;
    run += v[r];
  }
  // inclusive scan of per-thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long s = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = s;
  }
  __syncthreads();
  long long pre = (warp > 0 ? warp_tot[warp - 1] : 0) + x - run;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    const long long k = b0 + r;
    if (k < n) out[k] = pre;
    pre += v[r];
  }
  if (threadIdx.x == kScanThreads - 1 && sums) sums[blockIdx.x] = warp_tot[kScanThreads / 32 - 1];
}

__global__ void k_add_offsets(long long* out, long long n, const long long* offs) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] += offs[k / kScanTile];
}

long long nblocks(long long n) { return (n + kScanTile - 1) / kScanTile; }

template <typename Tin>
void scan_rec(const Tin* in, long long* out, long long n, long long* scratch, cudaStream_t s) {
  if (n <= 0) return;
  const long long nb = nblocks(n);
  if (nb == 1) {
    k_scan_tile<Tin><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    return;
  }
  long long* sums = scratch;
  k_scan_tile<Tin><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  scan_rec<long long>(sums, sums, nb, scratch + nb, s);
  k_add_offsets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums);
}

// tile of each particle; counts by atomics; cells out of range are counted in err
__global__ void k_bin_count(int nx0, int nx1, int nx2, int T0, int T1, int T2, int nt0, int nt1, long long n,
                            const int* cell, int* counts, int* tile_of, int* err) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int c0 = cell[3 * p], c1 = cell[3 * p + 1], c2 = cell[3 * p + 2];
  if (c0 < 0 || c0 >= nx0 || c1 < 0 || c1 >= nx1 || c2 < 0 || c2 >= nx2) {
    atomicAdd(err, 1);
    tile_of[p] = -1;
    return;
  }
  const int t = ((c2 / T2) * nt1 + c1 / T1) * nt0 + c0 / T0;
  tile_of[p] = t;
  atomicAdd(&counts[t], 1);
}

__global__ void k_bin_scatter(long long n, const int* tile_of, const long long* start, int* cursor,
                              long long* perm) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int t = tile_of[p];
  if (t < 0) return;
  perm[start[t] + atomicAdd(&cursor[t], 1)] = p;
}

}  // namespace

size_t scan_scratch_bytes(long long n) {
  size_t total = 0;
  long long m = n;
  while (m > kScanTile) {
    m = nblocks(m);
    total += (size_t)m * sizeof(long long);
  }
  return total + 64;
}

void exclusive_scan_i32(const int* in, long long* out, long long n, void* scratch, cudaStream_t s) {
  scan_rec<int>(in, out, n, reinterpret_cast<long long*>(scratch), s);
}

// Shared body of the stateless binning: scratch layout is
// [tile_of: n int32][cursor: ntiles int32][err: int32][scan scratch].
size_t bin_scratch_bytes(long long n, long long ntiles) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  return al((size_t)n * 4) + al((size_t)ntiles * 4) + al(4) + al(scan_scratch_bytes(ntiles));
}

pic_status bin_tiles_run(const int nx[3], const int tile[3], long long n, const int* cell, int* tile_count,
                         long long* tile_start, long long* perm, void* scratch, cudaStream_t s) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  int nt[3];
  for (int d = 0; d < 3; ++d) nt[d] = nx[d] / tile[d];
  const long long ntiles = (long long)nt[0] * nt[1] * nt[2];
  char* p = reinterpret_cast<char*>(scratch);
  int* tile_of = reinterpret_cast<int*>(p);
  p += al((size_t)n * 4);
  int* cursor = reinterpret_cast<int*>(p);
  p += al((size_t)ntiles * 4);
  int* err = reinterpret_cast<int*>(p);
  p += al(4);
  long long* sscr = reinterpret_cast<long long*>(p);
  cudaMemsetAsync(tile_count, 0, sizeof(int) * (size_t)ntiles, s);
  cudaMemsetAsync(cursor, 0, sizeof(int) * (size_t)ntiles, s);
  cudaMemsetAsync(err, 0, sizeof(int), s);
  if (n > 0)
    k_bin_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nx[0], nx[1], nx[2], tile[0], tile[1], tile[2], nt[0],
                                                             nt[1], n, cell, tile_count, tile_of, err);
  exclusive_scan_i32(tile_count, tile_start, ntiles, sscr, s);
  if (n > 0)
    k_bin_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, tile_of, tile_start, cursor, perm);
  int herr = 0;
  cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("pic_bin_tiles: ") + cudaGetErrorString(e));
    return PIC_ECUDA;
  }
  if (herr != 0) {
    set_error("pic_bin_tiles: " + std::to_string(herr) + " cell coordinates outside [0, nx)");
    return PIC_EINVAL;
  }
  return PIC_OK;
}

pic_status bin_tiles_check(const int nx[3], const int tile[3], long long n, const int* cell, int* tile_count,
                           long long* tile_start, long long* perm) {
  if (!nx || !tile || n < 0 || !tile_count || !tile_start || (n > 0 && (!cell || !perm))) {
    set_error("pic_bin_tiles: null pointer or negative count");
    return PIC_EINVAL;
  }
  long long ntiles = 1;
  for (int d = 0; d < 3; ++d) {
    if (nx[d] <= 0 || tile[d] <= 0 || nx[d] % tile[d] != 0) {
      set_error("pic_bin_tiles: every nx[d] must be a positive multiple of tile[d]");
      return PIC_EINVAL;
    }
    ntiles *= nx[d] / tile[d];
  }
  if (ntiles > (1ll << 30)) {
    set_error("pic_bin_tiles: too many tiles");
    return PIC_EINVAL;
  }
  return PIC_OK;
}

}  // namespace picgb

using namespace picgb;

extern "C" pic_status pic_bin_tiles(const int nx[3], const int tile[3], long long n, const int* cell,
                                    int* tile_count, long long* tile_start, long long* perm,
                                    const pic_allocator* alloc, void* stream) {
  pic_status st = bin_tiles_check(nx, tile, n, cell, tile_count, tile_start, perm);
  if (st != PIC_OK) return st;
  const long long ntiles = (long long)(nx[0] / tile[0]) * (nx[1] / tile[1]) * (nx[2] / tile[2]);
  const size_t bytes = bin_scratch_bytes(n, ntiles);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  if (alloc && alloc->alloc) {
    scratch = alloc->alloc(alloc->ctx, bytes);
  } else if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
    scratch = nullptr;
  }
  if (!scratch) {
    set_error("pic_bin_tiles: scratch allocation of " + std::to_string(bytes) + " bytes failed");
    return PIC_ENOMEM;
  }
  st = bin_tiles_run(nx, tile, n, cell, tile_count, tile_start, perm, scratch, s);
  if (alloc && alloc->alloc) {
    if (alloc->free) alloc->free(alloc->ctx, scratch, bytes);
  } else {
    cudaFree(scratch);
  }
  return st;
}

// ---------------------------------------------------------------------------
// pic_bin_tiles_noalloc: the same binning with its scratch in a fixed device
// array instead of memory obtained from an allocator.
//
// The array lives in this library's module image, so every GPU that loads the
// library keeps PIC_BIN_NOALLOC_SCRATCH_BYTES of device memory reserved until
// the process exits.  Host code must not use the array's name as a device
// address; its address is looked up per device with cudaGetSymbolAddress the
// first time the entry point runs on that device (with that device current),
// then cached.
// ---------------------------------------------------------------------------
namespace picgb {
namespace {

constexpr size_t kNoAllocBytes = PIC_BIN_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_bin_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_bin_scratch_addr[kMaxDevices] = {};
std::mutex g_bin_scratch_mu;

pic_status bin_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("pic_bin_tiles_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return PIC_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("pic_bin_tiles_noalloc: device ordinal out of range");
    return PIC_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_bin_scratch_mu);
  if (!g_bin_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_bin_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("pic_bin_tiles_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return PIC_ECUDA;
    }
    g_bin_scratch_addr[dev] = p;
  }
  *out = g_bin_scratch_addr[dev];
  return PIC_OK;
}

}  // namespace
}  // namespace picgb

extern "C" pic_status pic_bin_tiles_noalloc(const int nx[3], const int tile[3], long long n, const int* cell,
                                            int* tile_count, long long* tile_start, long long* perm, void* stream) {
  pic_status st = bin_tiles_check(nx, tile, n, cell, tile_count, tile_start, perm);
  if (st != PIC_OK) return st;
  const long long ntiles = (long long)(nx[0] / tile[0]) * (nx[1] / tile[1]) * (nx[2] / tile[2]);
  const size_t bytes = bin_scratch_bytes(n, ntiles);
  if (bytes > kNoAllocBytes) {
    set_error("pic_bin_tiles_noalloc: " + std::to_string(n) + " particles on " + std::to_string(ntiles) +
              " tiles need " + std::to_string(bytes) + " bytes of scratch, more than the fixed " +
              std::to_string(kNoAllocBytes) + "; use pic_bin_tiles");
    return PIC_EINVAL;
  }
  void* scratch = nullptr;
  st = bin_scratch_address(&scratch);
  if (st != PIC_OK) return st;
  return bin_tiles_run(nx, tile, n, cell, tile_count, tile_start, perm, scratch,
                       reinterpret_cast<cudaStream_t>(stream));
}
