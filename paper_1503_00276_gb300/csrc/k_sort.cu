// k_sort.cu -- prefix sums and the stateless tile binning entry point.
#include <algorithm>
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

// Tile of each particle and the count of every tile (atomics; counts do not
// depend on their order).  A cell out of range is counted in err and gets the
// key ntiles, which sorts after every tile.
__global__ void k_bin_count(int nx0, int nx1, int nx2, int T0, int T1, int T2, int nt0, int nt1, int ntiles,
                            long long n, const int* cell, int* counts, int* tile_of, int* err) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int c0 = cell[3 * p], c1 = cell[3 * p + 1], c2 = cell[3 * p + 2];
  if (c0 < 0 || c0 >= nx0 || c1 < 0 || c1 >= nx1 || c2 < 0 || c2 >= nx2) {
    atomicAdd(err, 1);
    tile_of[p] = ntiles;
    return;
  }
  const int t = ((c2 / T2) * nt1 + c1 / T1) * nt0 + c0 / T0;
  tile_of[p] = t;
  atomicAdd(&counts[t], 1);
}

// Stable order of the particles by tile: a least-significant-digit radix sort
// of the particle indices on the tile key, 8 bits per pass.  Every pass is a
// stable counting sort, so after the last one the particles of a tile are in
// increasing index.  A block takes kRxBlock consecutive elements of the pass's
// input, in kRxRounds rounds of kRxThreads; within a round an element's rank
// among equal digits is the count of equal digits in earlier warps of the
// round plus those in lower lanes of its own warp, so the block keeps the
// input order.
constexpr int kRxThreads = 256;  // one thread per digit value in the per-round bookkeeping
constexpr int kRxRounds = 16;
constexpr int kRxBlock = kRxThreads * kRxRounds;
constexpr int kRxWarps = kRxThreads / 32;

// per-block digit counts, digit-major: hist[d * nb + b]
__global__ void __launch_bounds__(kRxThreads) k_rx_hist(long long n, const int* vin, const int* tile_of, int shift,
                                                        int nb, int* hist) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long b0 = (long long)blockIdx.x * kRxBlock;
  for (int j = 0; j < kRxRounds; ++j) {
    const long long k = b0 + (long long)j * kRxThreads + threadIdx.x;
    if (k < n) {
      const int v = vin ? vin[k] : (int)k;
      atomicAdd(&h[(tile_of[v] >> shift) & 255], 1);
    }
  }
  __syncthreads();
  hist[(long long)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// stable scatter of one pass: offs[d * nb + b] is where block b's first
// element of digit d goes; vout (int32) or, on the last pass, pout (int64)
__global__ void __launch_bounds__(kRxThreads) k_rx_scatter(long long n, const int* vin, const int* tile_of,
                                                           int shift, int nb, const long long* offs, int* vout,
                                                           long long* pout) {
  __shared__ int wc[kRxWarps][256];
  __shared__ long long base[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offs[(long long)tid * nb + blockIdx.x];
  for (int w = 0; w < kRxWarps; ++w) wc[w][tid] = 0;
  __syncthreads();
  const long long b0 = (long long)blockIdx.x * kRxBlock;
  for (int j = 0; j < kRxRounds; ++j) {
    const long long k = b0 + (long long)j * kRxThreads + tid;
    int dg = 256, v = 0;
    if (k < n) {
      v = vin ? vin[k] : (int)k;
      dg = (tile_of[v] >> shift) & 255;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, dg);
    const int lr = __popc(peers & ((1u << lane) - 1u));
    if (dg < 256 && lr == 0) wc[warp][dg] = __popc(peers);
    __syncthreads();
    if (dg < 256) {
      long long pos = base[dg] + lr;
      for (int w = 0; w < warp; ++w) pos += wc[w][dg];
      if (pout)
        pout[pos] = v;
      else
        vout[pos] = v;
    }
    __syncthreads();
    int s = 0;
    for (int w = 0; w < kRxWarps; ++w) {
      s += wc[w][tid];
      wc[w][tid] = 0;
    }
    base[tid] += s;
    __syncthreads();
  }
}

// radix passes needed for keys 0 .. ntiles (ntiles itself marks a bad cell)
int rx_passes(long long ntiles) {
  int bits = 1;
  while ((1ll << bits) <= ntiles) ++bits;
  return (bits + 7) / 8;
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

// Shared body of the stateless binning.  Scratch layout:
// [tile_of: n int32][err: int32][hist: 256 nb int32][offs: 256 nb int64]
// [scan scratch][values A: n int32 (2+ passes)][values B: n int32 (3+ passes)]
// with nb = ceil(n / kRxBlock) blocks per radix pass.
struct BinScratch {
  int* tile_of;
  int* err;
  int* hist;
  long long* offs;
  long long* sscr;
  int* vals[2];
};

size_t bin_scratch_layout(long long n, long long ntiles, void* base, BinScratch* out) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const long long nb = (n + kRxBlock - 1) / kRxBlock;
  const int passes = rx_passes(ntiles);
  const size_t parts[7] = {al((size_t)n * 4), al(4), al((size_t)nb * 256 * 4), al((size_t)nb * 256 * 8),
                           al(std::max(scan_scratch_bytes(ntiles), scan_scratch_bytes(nb * 256))),
                           passes >= 2 ? al((size_t)n * 4) : 0, passes >= 3 ? al((size_t)n * 4) : 0};
  size_t off[7], total = 0;
  for (int k = 0; k < 7; ++k) {
    off[k] = total;
    total += parts[k];
  }
  if (out) {
    char* p = reinterpret_cast<char*>(base);
    out->tile_of = reinterpret_cast<int*>(p + off[0]);
    out->err = reinterpret_cast<int*>(p + off[1]);
    out->hist = reinterpret_cast<int*>(p + off[2]);
    out->offs = reinterpret_cast<long long*>(p + off[3]);
    out->sscr = reinterpret_cast<long long*>(p + off[4]);
    out->vals[0] = passes >= 2 ? reinterpret_cast<int*>(p + off[5]) : nullptr;
    out->vals[1] = passes >= 3 ? reinterpret_cast<int*>(p + off[6]) : nullptr;
  }
  return total;
}

size_t bin_scratch_bytes(long long n, long long ntiles) { return bin_scratch_layout(n, ntiles, nullptr, nullptr); }

pic_status bin_tiles_run(const int nx[3], const int tile[3], long long n, const int* cell, int* tile_count,
                         long long* tile_start, long long* perm, void* scratch, cudaStream_t s) {
  int nt[3];
  for (int d = 0; d < 3; ++d) nt[d] = nx[d] / tile[d];
  const long long ntiles = (long long)nt[0] * nt[1] * nt[2];
  BinScratch B;
  bin_scratch_layout(n, ntiles, scratch, &B);
  cudaMemsetAsync(tile_count, 0, sizeof(int) * (size_t)ntiles, s);
  cudaMemsetAsync(B.err, 0, sizeof(int), s);
  if (n > 0)
    k_bin_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nx[0], nx[1], nx[2], tile[0], tile[1], tile[2], nt[0],
                                                             nt[1], (int)ntiles, n, cell, tile_count, B.tile_of,
                                                             B.err);
  exclusive_scan_i32(tile_count, tile_start, ntiles, B.sscr, s);
  if (n > 0) {
    const long long nb = (n + kRxBlock - 1) / kRxBlock;
    const int passes = rx_passes(ntiles);
    const int* vin = nullptr;  // first pass: the particle indices themselves
    for (int ps = 0; ps < passes; ++ps) {
      const bool last = ps == passes - 1;
      int* vout = last ? nullptr : B.vals[ps & 1];
      k_rx_hist<<<(unsigned)nb, kRxThreads, 0, s>>>(n, vin, B.tile_of, 8 * ps, (int)nb, B.hist);
      exclusive_scan_i32(B.hist, B.offs, nb * 256, B.sscr, s);
      k_rx_scatter<<<(unsigned)nb, kRxThreads, 0, s>>>(n, vin, B.tile_of, 8 * ps, (int)nb, B.offs, vout,
                                                        last ? perm : nullptr);
      vin = vout;
    }
  }
  int herr = 0;
  cudaMemcpyAsync(&herr, B.err, sizeof(int), cudaMemcpyDeviceToHost, s);
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
  if (n > 0x7fffffffll) {
    set_error("pic_bin_tiles: more than 2^31 - 1 particles");
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
// address; its address is looked up with cudaGetSymbolAddress (with the device
// current) the first time the entry point runs in a CUDA context, and cached
// under that context's unique id, so a device reset (which makes a new
// context and loads the module again) leads to a fresh look-up.
// ---------------------------------------------------------------------------
namespace picgb {
namespace {

constexpr size_t kNoAllocBytes = PIC_BIN_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_bin_scratch[kNoAllocBytes];

// driver calls reached through the runtime's entry-point query (the library
// does not link libcuda)
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

constexpr int kMaxCtx = 64;
struct ScratchSlot {
  unsigned long long ctx_id;
  void* addr;
};
ScratchSlot g_bin_scratch_addr[kMaxCtx] = {};
int g_bin_scratch_n = 0;
std::mutex g_bin_scratch_mu;

void* driver_fn(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return p;
}

pic_status bin_scratch_address(void** out) {
  // make the device's context current (the runtime does this on first use)
  cudaError_t e = cudaFree(nullptr);
  if (e != cudaSuccess) {
    set_error(std::string("pic_bin_tiles_noalloc: no usable device: ") + cudaGetErrorString(e));
    return PIC_ECUDA;
  }
  static CtxGetCurrentFn get_current = reinterpret_cast<CtxGetCurrentFn>(driver_fn("cuCtxGetCurrent"));
  static CtxGetIdFn get_id = reinterpret_cast<CtxGetIdFn>(driver_fn("cuCtxGetId"));
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) {
    set_error("pic_bin_tiles_noalloc: the current CUDA context could not be identified");
    return PIC_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_bin_scratch_mu);
  for (int k = 0; k < g_bin_scratch_n; ++k)
    if (g_bin_scratch_addr[k].ctx_id == id) {
      *out = g_bin_scratch_addr[k].addr;
      return PIC_OK;
    }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_bin_scratch);
  if (e != cudaSuccess || !p) {
    set_error(std::string("pic_bin_tiles_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return PIC_ECUDA;
  }
  // a full table (more contexts than kMaxCtx in one process) recycles the oldest slot
  const int k = g_bin_scratch_n < kMaxCtx ? g_bin_scratch_n++ : (int)(id % kMaxCtx);
  g_bin_scratch_addr[k] = ScratchSlot{id, p};
  *out = p;
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
