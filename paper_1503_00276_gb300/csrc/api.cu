// api.cu -- the C ABI of libpicgb (include/pic.h): simulation state, loading,
// the step schedule, copy-out and diagnostics.  All numerical work runs in the
// kernels of k_*.cu; this file only allocates, orders launches and checks status.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <functional>
#include <vector>

#include "kernels.h"

namespace picgb {

static thread_local std::string g_err = "no error";
void set_error(const std::string& msg) { g_err = msg; }

// the counters of every (member, species) of a batch into one array, and
// reset them (batched moving windows)
__global__ void k_batch_gather_counts(int* const* src, int* dst, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    dst[k] = *src[k];
    *src[k] = 0;
  }
}

namespace {

// ------------------------------------------------------------- small kernels
__global__ void k_aos3_to_soa(const double* a, long long n, double* x0, double* x1, double* x2) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  x0[k] = a[3 * k];
  x1[k] = a[3 * k + 1];
  x2[k] = a[3 * k + 2];
}

__global__ void k_soa_to_aos3(const double* x0, const double* x1, const double* x2, long long n, double* a) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  a[3 * k] = x0[k];
  a[3 * k + 1] = x1[k];
  a[3 * k + 2] = x2 ? x2[k] : 0.0;
}

// Explicit positions must lie in the periodic box [xmin, xmin + nx dx).
__global__ void k_check_box(int ndim, PushConst C, const double* x0, const double* x1, const double* x2, long long n,
                            int* status) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double* xs[3] = {x0, x1, x2};
  for (int d = 0; d < ndim; ++d) {
    const double v = xs[d][k];
    if (!(v >= C.xmin[d] && v < C.xmin[d] + C.L[d])) atomicOr(status, ST_BADCELL);
  }
}

// FP32 weights to FP64 (null: all 1)
__global__ void k_widen(const float* w, double* out, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = w ? (double)w[k] : 1.0;
}

struct StatusWord {  // status bits of every kernel of one simulation (ST_*); spill counts are per species
  int status;
  int pad;
};

// ------------------------------------------------------------- allocation
struct Allocator {
  pic_allocator user{};
  bool has_user = false;
  std::vector<std::pair<void*, size_t>> live;

  void* get(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (has_user) {
      p = user.alloc(user.ctx, bytes);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) live.emplace_back(p, bytes);
    return p;
  }
  void put(void* p) {
    if (!p) return;
    for (size_t k = 0; k < live.size(); ++k) {
      if (live[k].first == p) {
        if (has_user) {
          if (user.free) user.free(user.ctx, p, live[k].second);
        } else {
          cudaFree(p);
        }
        live.erase(live.begin() + (long)k);
        return;
      }
    }
  }
  void release_all() {
    while (!live.empty()) put(live.back().first);
  }
};

struct SpeciesState {
  double rqm = -1.0, q = 0.0;
  long long n = 0;
  long long np_max = 0;
  bool ids = false;
  // FP64 plain
  Plain plain{};
  // FP32 tiled
  Tiles tg{};
  TileSide side[2]{};
  int cur = 0;
  long long slots = 0;
  Flat32 spill{};
  long long spill_cap = 0;
  int grid = 0;             // persistent CTAs of the tile kernel
  int* work = nullptr;      // its dynamic tile counter
  // lattice description (moving-window injection continues the loader)
  int ppc[3] = {0, 0, 0};
  double uth[3] = {0, 0, 0}, ufl[3] = {0, 0, 0};
  unsigned long long seed = 0;
  long long created = 0;    // particles ever created (ids and draw indices continue from here)
  int* d_lost = nullptr;    // particles dropped through an open x1 boundary in the last step
  int* d_spill = nullptr;   // records in this species' spill list
  SliceScratch slices{};    // work items of the tile kernel (heavy tiles split)
  double slack = 0.25;      // region growth room; raised after each spill
  // density profile / explicit weights: per-particle charge weights
  bool weighted = false;
  bool has_prof = false;
  ProfileDev prof{};        // device copy of the profile tables (lattice species)
  double* prof_mem = nullptr;
  int* d_kept = nullptr;    // particles the last injection created
};

constexpr int kTimingSlots = 5;
constexpr int kLaunchSlot = 5;

}  // namespace
}  // namespace picgb

using namespace picgb;

struct pic_sim {
  pic_grid g{};
  Layout L{};
  int ndim = 0;
  pic_precision prec = PIC_FP64_PLAIN;
  cudaStream_t s = nullptr;
  Allocator al;
  void* fld = nullptr;  // 6 planes E1..B3
  void* cur = nullptr;  // 3 planes J1..J3
  void* tmp = nullptr;  // 1 plane (smoothing)
  double* rho = nullptr;
  double* dense = nullptr;  // 1 dense FP64 grid (copy-out staging)
  Diag64* dacc = nullptr;
  StatusWord* dstat = nullptr;
  StatusWord* hstat = nullptr;  // pinned
  int* hcnt = nullptr;          // pinned: dropped / created particles per species, read with the status
  std::vector<SpeciesState> sp;
  CUtensorMap fmap{}, jmap{};
  long long step = 0;
  int T[3] = {1, 1, 1};
  double slack = 0.25;
  int sort_period = 1;
  int minb = 4;  // CTAs per SM the general tile kernel is built for (2 or 4)
  bool timing = false;
  double t_ms[kTimingSlots] = {0, 0, 0, 0, 0};
  long long t_n[kTimingSlots] = {0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  int sticky_flags = 0;
  long long nlaunch = 0;  // kernels launched by pic_step since the last reset
  bool no_small = false;  // member of a batch or moving window: the general tile kernel only
  // laser antennas (pulses entering through the lower x1 boundary)
  std::vector<unsigned char> h_ants;  // antenna_bytes() per pulse
  void* d_ants = nullptr;
  int n_ants = 0;
  float* d_inc = nullptr;             // [2][ny nz] incident B2, B3 below the boundary
  bool moving = false;    // window moving at c in +x1
  long long shifts = 0;   // one-cell shifts of the window so far
  bool in_batch = false;  // stepped by its batch; pic_step refuses it
  bool cyl = false;       // 2D cylindrically symmetric (r-z) mode
  CylConst K{};
};

namespace {

size_t elem_bytes(const pic_sim* S) { return S->prec == PIC_FP32_CELLOFF ? 4 : 8; }

template <typename T>
T* fld_ptr(pic_sim* S, int c) {
  return reinterpret_cast<T*>(S->fld) + (long long)c * S->L.plane;
}
template <typename T>
T* cur_ptr(pic_sim* S, int c) {
  return reinterpret_cast<T*>(S->cur) + (long long)c * S->L.plane;
}

pic_status cuda_check(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return PIC_ECUDA;
  }
  return PIC_OK;
}

PushConst make_const(const pic_sim* S, const SpeciesState& sp) {
  PushConst C{};
  const pic_grid& g = S->g;
  double dvol = 1.0;
  for (int d = 0; d < 3; ++d) {
    C.xmin[d] = g.xmin[d];
    C.dx[d] = d < S->ndim ? g.dx[d] : 1.0;
    C.inv_dx[d] = 1.0 / C.dx[d];
    C.e0[d] = g.e0[d];
    C.b0[d] = g.b0[d];
    C.L[d] = d < S->ndim ? g.nx[d] * g.dx[d] : 1.0;
    if (d < S->ndim) dvol *= g.dx[d];
  }
  C.dt = g.dt;
  C.rqm = sp.rqm;
  C.q = sp.q;
  C.dvol = dvol;
  C.isis = g.deposit == PIC_DEPOSIT_ISIS ? 1 : 0;
  C.cyl = S->cyl ? 1 : 0;
  return C;
}

// ------------------------------------------------------------- timing
cudaEvent_t ev_get(pic_sim* S) {
  if (!S->ev_pool.empty()) {
    cudaEvent_t e = S->ev_pool.back();
    S->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct Span {
  pic_sim* S;
  int slot;
  cudaEvent_t a = nullptr;
  Span(pic_sim* s_, int slot_) : S(s_), slot(slot_) {
    if (S->timing) {
      a = ev_get(S);
      cudaEventRecord(a, S->s);
    }
  }
  ~Span() {
    if (S->timing) {
      cudaEvent_t b = ev_get(S);
      cudaEventRecord(b, S->s);
      S->ev_pending.push_back({slot, {a, b}});
    }
  }
};

void timing_collect(pic_sim* S) {
  if (S->ev_pending.empty()) return;
  cudaStreamSynchronize(S->s);
  for (auto& p : S->ev_pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.second.first, p.second.second);
    S->t_ms[p.first] += ms;
    S->t_n[p.first] += 1;
    S->ev_pool.push_back(p.second.first);
    S->ev_pool.push_back(p.second.second);
  }
  S->ev_pending.clear();
}

// ------------------------------------------------------------- tensor maps
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

pic_status make_maps(pic_sim* S) {
  auto enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled not available from the driver");
    return PIC_ECUDA;
  }
  const Layout& L = S->L;
  const cuuint64_t ps = (cuuint64_t)L.plane * 4;
  CUresult r1, r2;
  if (S->ndim == 3) {
    cuuint64_t gdim[4] = {(cuuint64_t)L.NX, (cuuint64_t)L.NY, (cuuint64_t)L.NZ, 6};
    cuuint64_t gstr[3] = {(cuuint64_t)L.NX * 4, (cuuint64_t)L.NX * L.NY * 4, ps};
    cuuint32_t box[4] = {(cuuint32_t)S->T[0] + 4, (cuuint32_t)S->T[1] + 2, (cuuint32_t)S->T[2] + 2, 6};
    cuuint32_t es[4] = {1, 1, 1, 1};
    r1 = enc(&S->fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, S->fld, gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    cuuint64_t jdim[4] = {(cuuint64_t)L.NX, (cuuint64_t)L.NY, (cuuint64_t)L.NZ, 3};
    cuuint32_t jbox[4] = {(cuuint32_t)S->T[0] + 4, (cuuint32_t)S->T[1] + 3, (cuuint32_t)S->T[2] + 3, 3};
    r2 = enc(&S->jmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, S->cur, jdim, gstr, jbox, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint64_t gdim[3] = {(cuuint64_t)L.NX, (cuuint64_t)L.NY, 6};
    cuuint64_t gstr[2] = {(cuuint64_t)L.NX * 4, ps};
    cuuint32_t box[3] = {(cuuint32_t)S->T[0] + 4, (cuuint32_t)S->T[1] + 2, 6};
    cuuint32_t es[3] = {1, 1, 1};
    r1 = enc(&S->fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, S->fld, gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    cuuint64_t jdim[3] = {(cuuint64_t)L.NX, (cuuint64_t)L.NY, 3};
    cuuint32_t jbox[3] = {(cuuint32_t)S->T[0] + 4, (cuuint32_t)S->T[1] + 3, 3};
    r2 = enc(&S->jmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, S->cur, jdim, gstr, jbox, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r1) + ", " + std::to_string((int)r2) + ")");
    return PIC_ECUDA;
  }
  return PIC_OK;
}

// ------------------------------------------------------------- tiled store
Part32 alloc_part(pic_sim* S, long long slots, bool ids, bool& ok, bool weights = false) {
  Part32 p{};
  p.cell = (uint32_t*)S->al.get(4 * (size_t)slots);
  for (int d = 0; d < 3; ++d) {
    p.o[d] = (d < S->ndim) ? (float*)S->al.get(4 * (size_t)slots) : nullptr;
    p.u[d] = (float*)S->al.get(4 * (size_t)slots);
  }
  if (S->ndim == 2) p.o[2] = nullptr;
  p.id = ids ? (int*)S->al.get(4 * (size_t)slots) : nullptr;
  p.w = weights ? (float*)S->al.get(4 * (size_t)slots) : nullptr;
  ok = p.cell && p.o[0] && p.o[1] && (S->ndim == 2 || p.o[2]) && p.u[0] && p.u[1] && p.u[2] && (!ids || p.id) &&
       (!weights || p.w);
  return p;
}

void free_part(pic_sim* S, Part32& p) {
  S->al.put(p.cell);
  for (int d = 0; d < 3; ++d) {
    S->al.put(p.o[d]);
    S->al.put(p.u[d]);
  }
  S->al.put(p.id);
  S->al.put(p.w);
  p = Part32{};
}

Flat32 alloc_flat(pic_sim* S, long long n, bool ids, bool& ok, bool weights = false) {
  Flat32 f{};
  size_t m = (size_t)std::max<long long>(n, 1);
  f.tile = (int*)S->al.get(4 * m);
  f.cell = (uint32_t*)S->al.get(4 * m);
  for (int d = 0; d < 3; ++d) {
    f.o[d] = (float*)S->al.get(4 * m);
    f.u[d] = (float*)S->al.get(4 * m);
  }
  f.id = ids ? (int*)S->al.get(4 * m) : nullptr;
  f.w = weights ? (float*)S->al.get(4 * m) : nullptr;
  ok = f.tile && f.cell && f.o[0] && f.o[1] && f.o[2] && f.u[0] && f.u[1] && f.u[2] && (!ids || f.id) &&
       (!weights || f.w);
  return f;
}

void free_flat(pic_sim* S, Flat32& f) {
  S->al.put(f.tile);
  S->al.put(f.cell);
  for (int d = 0; d < 3; ++d) {
    S->al.put(f.o[d]);
    S->al.put(f.u[d]);
  }
  S->al.put(f.id);
  S->al.put(f.w);
  f = Flat32{};
}

// Bin a flat particle list into buffer `cur` of the store, sizing every tile
// region from its count (plus slack).  Regrows the store when needed.
pic_status bin_flat(pic_sim* S, SpeciesState& sp, Flat32& flat, long long n) {
  const int nt = sp.tg.ntiles;
  int* counts = (int*)S->al.get(4 * (size_t)nt);
  if (!counts) {
    set_error("out of device memory (tile counts)");
    return PIC_ENOMEM;
  }
  cudaMemsetAsync(counts, 0, 4 * (size_t)nt, S->s);
  flat_count(flat, n, nt, counts, S->s);
  std::vector<int> hc(nt);
  cudaMemcpyAsync(hc.data(), counts, 4 * (size_t)nt, cudaMemcpyDeviceToHost, S->s);
  if (cudaStreamSynchronize(S->s) != cudaSuccess) {
    S->al.put(counts);
    return cuda_check("binning");
  }
  long long total = 0;
  for (int t = 0; t < nt; ++t) total += hc[t];
  if (total != n) {
    S->al.put(counts);
    set_error("binning: " + std::to_string(n - total) + " particles outside the grid");
    return PIC_EINVAL;
  }
  // Region of tile t: its count plus slack for growth, of which the back
  // part `res` receives the particles entering the tile during a step.  The
  // arrivals come from the neighbours, so `res` follows the fullest of the 27
  // tiles around (a tile ahead of a dense beam is empty until the beam enters
  // it); with a moving window a shift step also brings the whole first cell
  // column of the tile ahead in x1.
  std::vector<int> hcap(nt), hres(nt);
  std::vector<long long> hbase(nt);
  const int* ntd = sp.tg.nt;
  std::vector<long long> nbmax(nt, 0);
  for (int t = 0; t < nt; ++t) {
    const int ix = t % ntd[0], iy = (t / ntd[0]) % ntd[1], iz = t / (ntd[0] * ntd[1]);
    long long m = 0;
    for (int dz = (ntd[2] > 1 ? -1 : 0); dz <= (ntd[2] > 1 ? 1 : 0); ++dz)
      for (int dy = (ntd[1] > 1 ? -1 : 0); dy <= (ntd[1] > 1 ? 1 : 0); ++dy)
        for (int dx = (ntd[0] > 1 ? -1 : 0); dx <= (ntd[0] > 1 ? 1 : 0); ++dx) {
          const int jx = (ix + dx + ntd[0]) % ntd[0], jy = (iy + dy + ntd[1]) % ntd[1];
          const int jz = (iz + dz + ntd[2]) % ntd[2];
          m = std::max<long long>(m, hc[(jz * ntd[1] + jy) * ntd[0] + jx]);
        }
    nbmax[t] = m;
  }
  long long slots = 0;
  for (int t = 0; t < nt; ++t) {
    const long long c = hc[t];
    long long res = std::max<long long>(32, (long long)std::ceil(0.5 * sp.slack * nbmax[t]));
    if (S->moving) {
      // a shift step brings the first cell column of the tile ahead; the
      // front tile column gets the fresh plasma of the new front cells instead
      const int ix = t % ntd[0];
      const long long lattice = (long long)sp.ppc[0] * sp.ppc[1] * sp.ppc[2] * S->T[0] * S->T[1] *
                                (S->ndim == 3 ? S->T[2] : 1);
      const long long ahead = ix + 1 < ntd[0] ? hc[t + 1] : lattice;
      res = std::max<long long>(res, (long long)std::ceil(1.25 * ahead / S->T[0]) + 32);
    }
    res = (res + 3) / 4 * 4;  // a multiple of 4, so that the stayer part ends 16-byte aligned
    const long long extra = std::max<long long>({64, (long long)std::ceil(c * sp.slack), 2 * res});
    long long cap = (c + extra + 3) / 4 * 4;
    if (cap > (1ll << 30)) cap = 1ll << 30;
    hcap[t] = (int)cap;
    hres[t] = (int)(std::min<long long>(cap - c, res) & ~3ll);
    hbase[t] = slots;
    slots += cap;
  }
  if (sp.np_max > 0 && n > sp.np_max) {
    S->al.put(counts);
    set_error("species holds " + std::to_string(n) + " particles, more than np_max");
    return PIC_EOVERFLOW;
  }
  if (slots > sp.slots) {
    for (int b = 0; b < 2; ++b) free_part(S, sp.side[b].p);
    bool ok0, ok1;
    sp.side[0].p = alloc_part(S, slots, sp.ids, ok0, sp.weighted);
    sp.side[1].p = alloc_part(S, slots, sp.ids, ok1, sp.weighted);
    if (!ok0 || !ok1) {
      S->al.put(counts);
      set_error("out of device memory (particle store of " + std::to_string(slots) + " slots)");
      return PIC_ENOMEM;
    }
    sp.slots = slots;
    S->al.put(sp.slices.extra);
    const long long ecap = slice_list_capacity(slots, nt);
    sp.slices.extra = (int2*)S->al.get(sizeof(int2) * (size_t)ecap);
    sp.slices.cap = (int)std::min<long long>(ecap, 1ll << 30);
    if (!sp.slices.extra) {
      S->al.put(counts);
      set_error("out of device memory (slice list)");
      return PIC_ENOMEM;
    }
  }
  long long max_cap = 0;
  for (int t = 0; t < nt; ++t) max_cap = std::max<long long>(max_cap, hcap[t]);
  sp.tg.small = !S->no_small && !sp.weighted && tiled_has_small(S->ndim, S->T) &&
                (max_cap <= tiled_small_capacity() || !tiled_has_general(S->ndim, S->T));
  if (!sp.tg.small && !tiled_has_general(S->ndim, S->T)) {
    S->al.put(counts);
    set_error("this tile shape has only the small-tile kernel, which a moving window, a batch member or a "
              "species with charge weights does not use (or a tile holds too many particles for it)");
    return PIC_EUNSUPPORTED;
  }
  sp.grid = tiled_push_grid(S->ndim, S->T, nt, sp.tg.small != 0, S->minb);
  cudaMemcpyAsync(sp.tg.cap, hcap.data(), 4 * (size_t)nt, cudaMemcpyHostToDevice, S->s);
  cudaMemcpyAsync(sp.tg.res, hres.data(), 4 * (size_t)nt, cudaMemcpyHostToDevice, S->s);
  cudaMemcpyAsync(sp.tg.base, hbase.data(), 8 * (size_t)nt, cudaMemcpyHostToDevice, S->s);
  int* cursor = (int*)S->al.get(4 * (size_t)nt);
  if (!cursor) {
    S->al.put(counts);
    set_error("out of device memory (cursor)");
    return PIC_ENOMEM;
  }
  cudaMemsetAsync(cursor, 0, 4 * (size_t)nt, S->s);
  flat_scatter(flat, n, sp.tg, cursor, sp.side[sp.cur].p, S->s);
  cudaMemcpyAsync(sp.side[sp.cur].stay, counts, 4 * (size_t)nt, cudaMemcpyDeviceToDevice, S->s);
  cudaMemsetAsync(sp.side[sp.cur].inc, 0, 4 * (size_t)nt, S->s);
  cudaError_t e = cudaStreamSynchronize(S->s);
  S->al.put(cursor);
  S->al.put(counts);
  if (e != cudaSuccess) return cuda_check("binning scatter");
  sp.n = n;
  return PIC_OK;
}

// Flatten the current buffer of a tiled species (+ spill list) into `flat`.
pic_status flatten(pic_sim* S, SpeciesState& sp, Flat32& flat, long long& n, bool include_spill, int spill_n,
                   bool& allocated) {
  const int nt = sp.tg.ntiles;
  int* tot = (int*)S->al.get(4 * (size_t)nt);
  long long* off = (long long*)S->al.get(8 * (size_t)nt + 8);
  void* scr = S->al.get(scan_scratch_bytes(nt));
  if (!tot || !off || !scr) {
    S->al.put(tot);
    S->al.put(off);
    S->al.put(scr);
    set_error("out of device memory (flatten)");
    return PIC_ENOMEM;
  }
  tiled_live(sp.tg, sp.side[sp.cur], tot, S->s);
  exclusive_scan_i32(tot, off, nt, scr, S->s);
  long long last_off = 0;
  int last_cnt = 0;
  cudaMemcpyAsync(&last_off, off + nt - 1, 8, cudaMemcpyDeviceToHost, S->s);
  cudaMemcpyAsync(&last_cnt, tot + nt - 1, 4, cudaMemcpyDeviceToHost, S->s);
  if (cudaStreamSynchronize(S->s) != cudaSuccess) return cuda_check("flatten");
  const long long nstore = last_off + last_cnt;
  n = nstore + (include_spill ? spill_n : 0);
  bool ok = true;
  flat = alloc_flat(S, n, sp.ids, ok, sp.weighted);
  allocated = true;
  if (!ok) {
    S->al.put(tot);
    S->al.put(off);
    S->al.put(scr);
    free_flat(S, flat);
    allocated = false;
    set_error("out of device memory (flat copy of " + std::to_string(n) + " particles)");
    return PIC_ENOMEM;
  }
  tiled_flatten(sp.tg, sp.side[sp.cur], off, flat, S->s);
  if (include_spill && spill_n > 0) {
    auto cp = [&](void* dst, const void* src) {
      cudaMemcpyAsync((char*)dst + 4 * (size_t)nstore, src, 4 * (size_t)spill_n, cudaMemcpyDeviceToDevice, S->s);
    };
    cp(flat.tile, sp.spill.tile);
    cp(flat.cell, sp.spill.cell);
    for (int d = 0; d < 3; ++d) {
      cp(flat.o[d], sp.spill.o[d]);
      cp(flat.u[d], sp.spill.u[d]);
    }
    if (flat.id && sp.spill.id) cp(flat.id, sp.spill.id);
    if (flat.w && sp.spill.w) cp(flat.w, sp.spill.w);
  }
  cudaError_t e = cudaStreamSynchronize(S->s);
  S->al.put(tot);
  S->al.put(off);
  S->al.put(scr);
  if (e != cudaSuccess) return cuda_check("flatten");
  return PIC_OK;
}

pic_status rebuild(pic_sim* S, SpeciesState& sp, int spill_n) {
  Flat32 flat{};
  long long n = 0;
  bool alloc = false;
  pic_status st = flatten(S, sp, flat, n, true, spill_n, alloc);
  if (st == PIC_OK) st = bin_flat(S, sp, flat, n);
  if (alloc) free_flat(S, flat);
  return st;
}

// Every species whose spill list holds records is re-binned (its records
// merged back into the store); the counters restart from zero.
pic_status rebuild_spilled(pic_sim* S) {
  for (auto& s : S->sp) {
    if (!s.d_spill) continue;
    int n = 0;
    if (cudaMemcpyAsync(&n, s.d_spill, sizeof(int), cudaMemcpyDeviceToHost, S->s) != cudaSuccess ||
        cudaStreamSynchronize(S->s) != cudaSuccess)
      return cuda_check("spill count");
    if (n <= 0) continue;
    // regions sized afresh from the new counts, with more growth room than
    // the last time (a beam keeps filling the tiles ahead of it)
    s.slack = std::min(1.0, std::max(s.slack, 0.25) * 1.5);
    const pic_status st = rebuild(S, s, (int)std::min<long long>(n, s.spill_cap));
    if (st != PIC_OK) return st;
    cudaMemsetAsync(s.d_spill, 0, sizeof(int), S->s);
  }
  return PIC_OK;
}

// ------------------------------------------------------------- loading
pic_status load_species(pic_sim* S, const pic_species& in, SpeciesState& sp) {
  const pic_grid& g = S->g;
  const int nd = S->ndim;
  double dvol = 1.0;
  long long ncells = 1;
  for (int d = 0; d < nd; ++d) {
    dvol *= g.dx[d];
    ncells *= g.nx[d];
  }
  sp.rqm = in.rqm;
  sp.ids = in.track_ids != 0;
  sp.np_max = in.np_max;
  for (int d = 0; d < 3; ++d) {
    sp.ppc[d] = d < S->ndim ? in.ppc[d] : 1;
    sp.uth[d] = in.uth[d];
    sp.ufl[d] = in.ufl[d];
  }
  sp.seed = in.seed;
  if (in.rqm == 0.0 || !std::isfinite(in.rqm)) {
    set_error("species rqm must be finite and non-zero");
    return PIC_EINVAL;
  }
  long long n;
  long long ppc = 1;
  if (in.n_explicit > 0) {
    if (!in.x0 || !in.u0) {
      set_error("explicit species needs x0 and u0");
      return PIC_EINVAL;
    }
    n = in.n_explicit;
  } else {
    for (int d = 0; d < 3; ++d) {
      const int v = d < nd ? in.ppc[d] : 1;
      if (d < nd && v <= 0) {
        set_error("species ppc must be positive");
        return PIC_EINVAL;
      }
      ppc *= (d < nd ? v : 1);
    }
    n = ncells * ppc;
  }
  if (in.np_max > 0 && n > in.np_max) {
    set_error("species has " + std::to_string(n) + " particles, more than np_max");
    return PIC_EOVERFLOW;
  }
  if (n > (1ll << 31) - 1 && sp.ids) {
    set_error("particle ids are int32: too many particles");
    return PIC_EINVAL;
  }
  // macroparticle charge: density * cell volume / ppc with the sign of q;
  // an explicit list gives it directly (q_explicit), else one particle per cell
  const double sign = in.rqm < 0 ? -1.0 : 1.0;
  if (in.n_explicit > 0)
    sp.q = in.q_explicit != 0.0 ? in.q_explicit : sign * in.density * dvol;
  else
    sp.q = sign * in.density * dvol / (double)ppc;
  sp.n = n;

  // density profile (lattice species) or explicit weights: per-particle charge weights
  sp.has_prof = false;
  sp.prof = ProfileDev{};
  if (in.n_explicit <= 0) {
    size_t tot = 0;
    for (int d = 0; d < nd; ++d) {
      const int np = in.prof_n[d];
      if (np <= 0) continue;
      if (!in.prof_x[d] || !in.prof_f[d]) {
        set_error("density profile: prof_x / prof_f missing");
        return PIC_EINVAL;
      }
      for (int k = 0; k < np; ++k)
        if (!std::isfinite(in.prof_x[d][k]) || !std::isfinite(in.prof_f[d][k]) || in.prof_f[d][k] < 0.0 ||
            (k > 0 && !(in.prof_x[d][k] >= in.prof_x[d][k - 1]))) {
          set_error("density profile: points must be finite and ascending, values >= 0");
          return PIC_EINVAL;
        }
      tot += 2 * (size_t)np;
    }
    if (tot > 0) {
      std::vector<double> h;
      h.reserve(tot);
      for (int d = 0; d < nd; ++d)
        for (int a = 0; a < 2 && in.prof_n[d] > 0; ++a)
          for (int k = 0; k < in.prof_n[d]; ++k) h.push_back(a == 0 ? in.prof_x[d][k] : in.prof_f[d][k]);
      sp.prof_mem = (double*)S->al.get(8 * tot);
      if (!sp.prof_mem) {
        set_error("out of device memory (density profile)");
        return PIC_ENOMEM;
      }
      cudaMemcpyAsync(sp.prof_mem, h.data(), 8 * tot, cudaMemcpyHostToDevice, S->s);
      size_t o = 0;
      for (int d = 0; d < nd; ++d) {
        const int np = in.prof_n[d];
        if (np <= 0) continue;
        sp.prof.n[d] = np;
        sp.prof.x[d] = sp.prof_mem + o;
        sp.prof.f[d] = sp.prof_mem + o + np;
        o += 2 * (size_t)np;
      }
      sp.prof.density = in.density;
      sp.prof.den_min = in.den_min;
      sp.has_prof = true;
      cudaStreamSynchronize(S->s);
    }
  }
  if (S->cyl && sp.has_prof) {
    set_error("the r-z mode takes no density profile");
    return PIC_EUNSUPPORTED;
  }
  sp.weighted = sp.has_prof || (in.n_explicit > 0 && in.w0 != nullptr) || S->cyl;  // r-z: ring weights
  sp.created = n;  // lattice places (ids and draw indices), kept or not

  // FP64 SoA of the initial state, in chunks (device); with a profile the
  // loader's output is staged and only the kept particles are moved on
  const long long chunk = S->prec == PIC_FP64_PLAIN && !sp.has_prof ? std::max<long long>(n, 1)
                                                                    : std::min<long long>(std::max<long long>(n, 1),
                                                                                          1ll << 25);
  double* xs[3] = {nullptr, nullptr, nullptr};
  double* us[3] = {nullptr, nullptr, nullptr};
  int* ids = nullptr;
  double* ws = nullptr;      // weights of the staged chunk
  double* cx[3] = {nullptr, nullptr, nullptr};  // FP32 form with a profile: the kept particles
  double* cu[3] = {nullptr, nullptr, nullptr};
  int* cid = nullptr;
  void* pscr = nullptr;      // profile_compact scratch
  double* aos = nullptr;
  auto fail = [&](const char* what) {
    set_error(std::string("out of device memory (") + what + ")");
    return PIC_ENOMEM;
  };
  if (S->prec == PIC_FP64_PLAIN) {
    for (int d = 0; d < 3; ++d) {
      sp.plain.x[d] = (d < nd) ? (double*)S->al.get(8 * (size_t)std::max<long long>(n, 1)) : nullptr;
      sp.plain.u[d] = (double*)S->al.get(8 * (size_t)std::max<long long>(n, 1));
      if ((d < nd && !sp.plain.x[d]) || !sp.plain.u[d]) return fail("particles");
    }
    sp.plain.id = sp.ids ? (int*)S->al.get(4 * (size_t)std::max<long long>(n, 1)) : nullptr;
    if (sp.ids && !sp.plain.id) return fail("ids");
    sp.plain.w = sp.weighted ? (double*)S->al.get(8 * (size_t)std::max<long long>(n, 1)) : nullptr;
    if (sp.weighted && !sp.plain.w) return fail("weights");
    sp.plain.n = n;
  }
  Flat32 flat{};
  bool flat_ok = true;
  if (S->prec == PIC_FP32_CELLOFF) {
    flat = alloc_flat(S, n, sp.ids, flat_ok, sp.weighted);
    if (!flat_ok) {
      free_flat(S, flat);
      return fail("flat staging");
    }
  }
  const bool staged = S->prec == PIC_FP32_CELLOFF || sp.has_prof;
  if (staged) {
    for (int d = 0; d < 3; ++d) {
      xs[d] = (double*)S->al.get(8 * (size_t)chunk);
      us[d] = (double*)S->al.get(8 * (size_t)chunk);
      if (!xs[d] || !us[d]) return fail("staging");
    }
    ids = sp.ids ? (int*)S->al.get(4 * (size_t)chunk) : nullptr;
    if (sp.ids && !ids) return fail("staging");
  }
  if (sp.weighted && S->prec == PIC_FP32_CELLOFF) {
    ws = (double*)S->al.get(8 * (size_t)chunk);
    if (!ws) return fail("staging");
  }
  if (sp.has_prof) {
    pscr = S->al.get(profile_scratch_bytes(chunk));
    if (!pscr) return fail("profile scratch");
    if (S->prec == PIC_FP32_CELLOFF) {
      for (int d = 0; d < 3; ++d) {
        cx[d] = (double*)S->al.get(8 * (size_t)chunk);
        cu[d] = (double*)S->al.get(8 * (size_t)chunk);
        if (!cx[d] || !cu[d]) return fail("staging");
      }
      cid = sp.ids ? (int*)S->al.get(4 * (size_t)chunk) : nullptr;
      if (sp.ids && !cid) return fail("staging");
    }
  }
  double* scratch_x2 = nullptr;
  long long kept = 0;  // particles created so far: where the next ones go
  for (long long first = 0; first < n; first += chunk) {
    const long long cnt = std::min(chunk, n - first);
    if (!staged) {  // FP64 plain, no profile: straight into the particle arrays
      for (int d = 0; d < 3; ++d) {
        xs[d] = sp.plain.x[d] ? sp.plain.x[d] + first : nullptr;
        us[d] = sp.plain.u[d] + first;
      }
      ids = sp.plain.id ? sp.plain.id + first : nullptr;
      if (!xs[2]) {
        if (!scratch_x2) scratch_x2 = (double*)S->al.get(8 * (size_t)chunk);
        if (!scratch_x2) return fail("staging");
        xs[2] = scratch_x2;
      }
    }
    if (in.n_explicit > 0) {
      if (!aos) aos = (double*)S->al.get(24 * (size_t)chunk);
      if (!aos) return fail("staging");
      cudaMemcpyAsync(aos, in.x0 + 3 * first, 24 * (size_t)cnt, cudaMemcpyHostToDevice, S->s);
      k_aos3_to_soa<<<(unsigned)((cnt + 255) / 256), 256, 0, S->s>>>(aos, cnt, xs[0], xs[1], xs[2]);
      k_check_box<<<(unsigned)((cnt + 255) / 256), 256, 0, S->s>>>(nd, make_const(S, sp), xs[0], xs[1], xs[2], cnt,
                                                                   &S->dstat->status);
      cudaMemcpyAsync(aos, in.u0 + 3 * first, 24 * (size_t)cnt, cudaMemcpyHostToDevice, S->s);
      k_aos3_to_soa<<<(unsigned)((cnt + 255) / 256), 256, 0, S->s>>>(aos, cnt, us[0], us[1], us[2]);
      if (ids) {
        std::vector<int> h((size_t)cnt);
        for (long long k = 0; k < cnt; ++k) h[(size_t)k] = (int)(first + k);
        cudaMemcpyAsync(ids, h.data(), 4 * (size_t)cnt, cudaMemcpyHostToDevice, S->s);
        cudaStreamSynchronize(S->s);
      }
      if (in.w0)  // explicit weights
        cudaMemcpyAsync(S->prec == PIC_FP64_PLAIN ? sp.plain.w + first : ws, in.w0 + first, 8 * (size_t)cnt,
                        cudaMemcpyHostToDevice, S->s);
    } else {
      LatticeSpec L{};
      L.ndim = nd;
      for (int d = 0; d < 3; ++d) {
        L.nx[d] = d < nd ? g.nx[d] : 1;
        L.xmin[d] = g.xmin[d];
        L.dx[d] = d < nd ? g.dx[d] : 1.0;
        L.ppc[d] = d < nd ? in.ppc[d] : 1;
        L.uth[d] = in.uth[d];
        L.ufl[d] = in.ufl[d];
      }
      L.seed = in.seed;
      lattice_load(L, first, cnt, xs, us, ids, S->s);
    }
    long long got = cnt;  // particles of this chunk that are created
    double* const* gx = xs;
    double* const* gu = us;
    const int* gid = ids;
    if (sp.has_prof) {
      if (S->prec == PIC_FP64_PLAIN) {
        double* dxp[3] = {sp.plain.x[0] + kept, sp.plain.x[1] + kept, nd == 3 ? sp.plain.x[2] + kept : nullptr};
        double* dup[3] = {sp.plain.u[0] + kept, sp.plain.u[1] + kept, sp.plain.u[2] + kept};
        got = profile_compact(nd, sp.prof, cnt, xs, us, ids, dxp, dup, sp.plain.id ? sp.plain.id + kept : nullptr,
                              sp.plain.w + kept, pscr, S->s);
      } else {
        got = profile_compact(nd, sp.prof, cnt, xs, us, ids, cx, cu, cid, ws, pscr, S->s);
        gx = cx;
        gu = cu;
        gid = cid;
      }
      if (got < 0) return cuda_check("density profile");
    }
    if (S->prec == PIC_FP32_CELLOFF) {
      Flat32 part = flat;
      part.tile += kept;
      part.cell += kept;
      for (int d = 0; d < 3; ++d) {
        part.o[d] += kept;
        part.u[d] += kept;
      }
      if (part.id) part.id += kept;
      if (part.w) part.w += kept;
      PushConst C = make_const(S, sp);
      if (S->cyl)  // rings: lattice points below the axis reflected, w = own weight * r
        cyl_load_fix(got, gx[1], ws, in.n_explicit <= 0, in.n_explicit > 0 && in.w0 != nullptr, &S->dstat->status,
                     S->s);
      global_to_flat(nd, S->L, sp.tg, C, gx, gu, gid, sp.weighted ? ws : nullptr, got, part, &S->dstat->status,
                     S->s);
    }
    kept += got;
    cudaError_t e = cudaStreamSynchronize(S->s);
    if (e != cudaSuccess) return cuda_check("loading particles");
  }
  n = kept;
  sp.n = n;
  if (S->prec == PIC_FP64_PLAIN) sp.plain.n = n;
  if (S->cyl && S->prec == PIC_FP64_PLAIN)  // rings: lattice points below the axis reflected, w = own weight * r
    cyl_load_fix(n, sp.plain.x[1], sp.plain.w, in.n_explicit <= 0, in.n_explicit > 0 && in.w0 != nullptr,
                 &S->dstat->status, S->s);
  if (aos) S->al.put(aos);
  if (scratch_x2) S->al.put(scratch_x2);
  if (staged) {
    for (int d = 0; d < 3; ++d) {
      S->al.put(xs[d]);
      S->al.put(us[d]);
      S->al.put(cx[d]);
      S->al.put(cu[d]);
    }
    S->al.put(ids);
    S->al.put(cid);
  }
  S->al.put(ws);
  S->al.put(pscr);
  if (S->prec == PIC_FP32_CELLOFF) {
    pic_status st = bin_flat(S, sp, flat, n);
    free_flat(S, flat);
    if (st != PIC_OK) return st;
  }
  return cuda_check("loading particles");
}

pic_status setup_tiles(pic_sim* S, SpeciesState& sp) {
  Tiles& tg = sp.tg;
  tg.ndim = S->ndim;
  tg.ntiles = 1;
  for (int d = 0; d < 3; ++d) {
    tg.T[d] = d < S->ndim ? S->T[d] : 1;
    tg.nt[d] = d < S->ndim ? S->g.nx[d] / S->T[d] : 1;
    tg.ntiles *= tg.nt[d];
  }
  tg.base = (long long*)S->al.get(8 * (size_t)tg.ntiles);
  tg.cap = (int*)S->al.get(4 * (size_t)tg.ntiles);
  tg.res = (int*)S->al.get(4 * (size_t)tg.ntiles);
  bool ok = tg.base && tg.cap && tg.res;
  for (int b = 0; b < 2; ++b) {
    TileSide& sd = sp.side[b];
    sd.stay = (int*)S->al.get(4 * (size_t)tg.ntiles);
    sd.inc = (int*)S->al.get(4 * (size_t)tg.ntiles);
    ok = ok && sd.stay && sd.inc;
  }
  sp.work = (int*)S->al.get(sizeof(int));
  sp.slices.nslice = (int*)S->al.get(4 * (size_t)tg.ntiles);
  sp.slices.nextra = (int*)S->al.get(sizeof(int));
  if (!ok || !sp.work || !sp.slices.nslice || !sp.slices.nextra) {
    set_error("out of device memory (tile tables)");
    return PIC_ENOMEM;
  }
  for (int b = 0; b < 2; ++b) {
    cudaMemsetAsync(sp.side[b].stay, 0, 4 * (size_t)tg.ntiles, S->s);
    cudaMemsetAsync(sp.side[b].inc, 0, 4 * (size_t)tg.ntiles, S->s);
  }
  return PIC_OK;
}

pic_status alloc_spill(pic_sim* S, SpeciesState& sp) {
  sp.spill_cap = std::max<long long>(1 << 16, sp.n / 64);
  bool ok = true;
  sp.spill = alloc_flat(S, sp.spill_cap, sp.ids, ok, sp.weighted);
  sp.d_lost = (int*)S->al.get(sizeof(int));
  sp.d_spill = (int*)S->al.get(sizeof(int));
  sp.d_kept = (int*)S->al.get(sizeof(int));
  if (!ok || !sp.d_lost || !sp.d_spill || !sp.d_kept) {
    set_error("out of device memory (spill list)");
    return PIC_ENOMEM;
  }
  cudaMemsetAsync(sp.d_lost, 0, sizeof(int), S->s);
  cudaMemsetAsync(sp.d_spill, 0, sizeof(int), S->s);
  cudaMemsetAsync(sp.d_kept, 0, sizeof(int), S->s);
  if (sp.created < sp.n) sp.created = sp.n;
  return PIC_OK;
}

// rho of every species into S->rho (padded FP64), guards folded; acc
// non-null (FP32 form): the kinetic energy and charge summed in the same pass
void compute_rho(pic_sim* S, Diag64* acc = nullptr) {
  cudaMemsetAsync(S->rho, 0, 8 * (size_t)S->L.plane, S->s);
  if (S->cyl) {  // ring charges (FP64: charges; FP32 tiles: per dz dr), then / V(r)
    for (auto& sp : S->sp) {
      PushConst C = make_const(S, sp);
      if (S->prec == PIC_FP64_PLAIN)
        cyl_rho(S->L, C, S->K, sp.plain, S->rho, S->s);
      else
        tiled_rho(S->L, C, sp.tg, sp.side[sp.cur], S->rho, acc, S->s);
    }
    cyl_rho_finish(S->L, S->K, S->rho, S->prec == PIC_FP64_PLAIN ? S->g.dx[0] * S->g.dx[1] : 1.0, S->s);
    return;
  }
  for (auto& sp : S->sp) {
    PushConst C = make_const(S, sp);
    if (S->prec == PIC_FP64_PLAIN)
      plain_rho(S->ndim, S->L, C, sp.plain, S->rho, S->s);
    else
      tiled_rho(S->L, C, sp.tg, sp.side[sp.cur], S->rho, acc, S->s);
  }
  double* r[1] = {S->rho};
  fold_guards<double>(S->L, r, 1, S->s);
}

// r-z: current to densities, then the r-z field solve
template <typename T>
void cyl_fields(pic_sim* S) {
  T* f[6];
  T* j[3];
  for (int c = 0; c < 6; ++c) f[c] = fld_ptr<T>(S, c);
  for (int c = 0; c < 3; ++c) j[c] = cur_ptr<T>(S, c);
  {
    Span sp(S, 1);
    cyl_current<T>(S->L, S->K, j, S->s);
  }
  Span sp(S, 2);
  S->nlaunch += 1 + cyl_field_step<T>(S->L, S->K, f, j, S->s);
}

template <typename T>
void field_step(pic_sim* S) {
  const Layout& L = S->L;
  T* e[3] = {fld_ptr<T>(S, 0), fld_ptr<T>(S, 1), fld_ptr<T>(S, 2)};
  T* b[3] = {fld_ptr<T>(S, 3), fld_ptr<T>(S, 4), fld_ptr<T>(S, 5)};
  T* j[3] = {cur_ptr<T>(S, 0), cur_ptr<T>(S, 1), cur_ptr<T>(S, 2)};
  {
    Span sp(S, 1);
    fold_guards<T>(L, j, 3, S->s);
    S->nlaunch += 1;
    for (int d = 0; d < S->ndim; ++d)
      for (int pass = 0; pass < S->g.smooth_level[d]; ++pass) {
        const double* w = S->g.smooth_w[d][pass];
        for (int c = 0; c < 3; ++c) smooth_pass<T>(L, j[c], reinterpret_cast<T*>(S->tmp), d, w[0], w[1], w[2], S->s);
        S->nlaunch += 3;
      }
  }
  {
    Span sp(S, 2);
    double dx[3] = {S->g.dx[0], S->g.dx[1], S->ndim == 3 ? S->g.dx[2] : 1.0};
    // the sweeps wrap their neighbours periodically; the guard cells (read by
    // the particle kernels) are refreshed once at the end
    yee_b_half<T>(L, e, b, S->g.dt, dx, S->s);
    const float* inc = nullptr;
    if (S->n_ants > 0) {  // the entering pulses' B below the lower x1 boundary at t = (n + 1/2) dt
      antenna_plane(L, S->d_ants, S->n_ants, ((double)S->step + 0.5) * S->g.dt, S->g.xmin[0], S->d_inc, S->s);
      inc = S->d_inc;
      S->nlaunch += 1;
    }
    yee_e<T>(L, e, b, j, S->g.dt, dx, S->s, inc);
    yee_b_half<T>(L, e, b, S->g.dt, dx, S->s);
    T* eb[6] = {e[0], e[1], e[2], b[0], b[1], b[2]};
    fill_guards<T>(L, eb, 6, S->s);
    S->nlaunch += 4;
  }
}

pic_status one_step(pic_sim* S, bool check_now) {
  Span whole(S, 4);
  // moving window: shift by one cell at the end of the step that brings c t a
  // full cell past the last shift
  // the window moves at c from window_start on
  const double lag = (double)(S->step + 1) * S->g.dt - S->g.window_start;
  const bool shift = S->moving && lag > 0.0 && (long long)std::floor(lag / S->g.dx[0]) > S->shifts;
  cudaMemsetAsync(S->cur, 0, 3 * elem_bytes(S) * (size_t)S->L.plane, S->s);
  {
    Span sp(S, 0);
    for (auto& s : S->sp) {
      PushConst C = make_const(S, s);
      if (S->prec == PIC_FP64_PLAIN) {
        double* f[6];
        double* j[3];
        for (int c = 0; c < 6; ++c) f[c] = fld_ptr<double>(S, c);
        for (int c = 0; c < 3; ++c) j[c] = cur_ptr<double>(S, c);
        if (S->cyl)
          cyl_push(S->L, C, S->K, s.plain, f, j, &S->dstat->status, S->s);
        else
          plain_push(S->ndim, S->L, C, s.plain, f, j, &S->dstat->status, S->s);
      } else {
        const int in = s.cur, out = 1 - s.cur;
        // the last step of every sort_period steps re-sorts each tile by cell;
        // the steps before it keep the order they find (blocks compacted)
        const bool stream = S->sort_period > 1 && !s.tg.small && (S->step + 1) % S->sort_period != 0;
        const int nk = tiled_push(S->L, C, s.tg, s.side[in], s.side[out], s.spill, s.d_spill, s.spill_cap, s.grid,
                                  s.work, &S->fmap, &S->jmap, &S->dstat->status, stream, S->minb, shift ? 1 : 0,
                                  s.d_lost, &s.slices, S->s);
        if (nk == 0) {
          set_error("no tile kernel for this tile shape");
          return PIC_EUNSUPPORTED;
        }
        S->nlaunch += nk - 1;  // the tile kernel itself is counted below
        s.cur = out;
        if (shift) {  // fresh plasma for the new front column
          const long long cnt = (long long)S->L.ny * S->L.nz * s.ppc[0] * s.ppc[1] * s.ppc[2];
          const int nxs[3] = {S->L.nx, S->L.ny, S->L.nz};
          tiled_inject(C, s.tg, s.side[out], s.spill, s.d_spill, s.spill_cap, &S->dstat->status, nxs,
                       s.ppc, s.uth, s.ufl, s.seed, s.created, cnt, s.has_prof ? &s.prof : nullptr, s.d_kept,
                       S->s);
          s.created += cnt;  // lattice places; the particles created are counted on the device
          S->nlaunch += cnt > 0 ? 1 : 0;
        }
      }
      S->nlaunch += s.n > 0 || S->prec == PIC_FP32_CELLOFF ? 1 : 0;
    }
  }
  if (S->cyl && S->prec == PIC_FP64_PLAIN) {
    cyl_fields<double>(S);
  } else if (S->cyl) {
    cyl_fields<float>(S);
  } else if (S->prec == PIC_FP64_PLAIN) {
    field_step<double>(S);
  } else {
    field_step<float>(S);
  }
  if (shift) {  // every field value one cell back; zero front column
    float* eb[6];
    for (int c = 0; c < 6; ++c) eb[c] = fld_ptr<float>(S, c);
    shift_x<float>(S->L, eb, 6, S->s);
    fill_guards<float>(S->L, eb, 6, S->s);
    S->g.xmin[0] += S->g.dx[0];
    ++S->shifts;
    S->nlaunch += 2;
  }
  ++S->step;
  pic_status st = cuda_check("step launch");
  if (st != PIC_OK) return st;
  if (!check_now) return PIC_OK;
  cudaMemcpyAsync(S->hstat, S->dstat, sizeof(StatusWord), cudaMemcpyDeviceToHost, S->s);
  // dropped (and injected) particles, read back with the status word
  const bool counted = S->moving || (S->cyl && S->prec == PIC_FP32_CELLOFF);
  if (counted)
    for (size_t k = 0; k < S->sp.size(); ++k) {
      cudaMemcpyAsync(S->hcnt + 2 * k, S->sp[k].d_lost, sizeof(int), cudaMemcpyDeviceToHost, S->s);
      cudaMemcpyAsync(S->hcnt + 2 * k + 1, S->sp[k].d_kept, sizeof(int), cudaMemcpyDeviceToHost, S->s);
      cudaMemsetAsync(S->sp[k].d_lost, 0, sizeof(int), S->s);
      cudaMemsetAsync(S->sp[k].d_kept, 0, sizeof(int), S->s);
    }
  if (cudaStreamSynchronize(S->s) != cudaSuccess) return cuda_check("step");
  const int flags = S->hstat->status;
  S->sticky_flags |= flags;
  if (counted)
    for (size_t k = 0; k < S->sp.size(); ++k) S->sp[k].n += S->hcnt[2 * k + 1] - S->hcnt[2 * k];
  if (flags & ST_SPILL) {
    if (flags & ST_SPILL_LOST) {
      set_error("particle spill list overflowed: particles were lost");
      return PIC_EOVERFLOW;
    }
    // the spilled particles were fully advanced; re-bin before the next step
    Span rb(S, 3);
    if ((st = rebuild_spilled(S)) != PIC_OK) return st;
    cudaMemsetAsync(S->dstat, 0, sizeof(StatusWord), S->s);
  }
  if (flags & ST_TIMEOUT) {
    set_error("a bounded device wait gave up (TMA copy did not complete)");
    return PIC_ETIMEOUT;
  }
  if (flags & (ST_NONFINITE | ST_BADCELL)) {
    set_error("non-finite particle or field value");
    return PIC_ENONFINITE;
  }
  return PIC_OK;
}

pic_status validate_grid(const pic_grid* g) {
  if (!g) {
    set_error("grid is NULL");
    return PIC_EINVAL;
  }
  if (g->ndim != 2 && g->ndim != 3) {
    set_error("ndim must be 2 or 3");
    return PIC_EINVAL;
  }
  double s = 0.0;
  for (int d = 0; d < g->ndim; ++d) {
    if (g->nx[d] < 4 || !(g->dx[d] > 0.0) || !std::isfinite(g->dx[d])) {
      set_error("nx must be >= 4 and dx > 0 in every direction");
      return PIC_EINVAL;
    }
    s += 1.0 / (g->dx[d] * g->dx[d]);
    for (int side = 0; side < 2; ++side)
      if (g->bc[d][side] != PIC_BC_PERIODIC && !(g->coords == PIC_COORDS_CYLINDRICAL && d == 1)) {
        set_error("only periodic boundaries are implemented");
        return PIC_EUNSUPPORTED;
      }
    if (g->smooth_level[d] < 0 || g->smooth_level[d] > PIC_MAX_SMOOTH) {
      set_error("smooth_level out of range");
      return PIC_EINVAL;
    }
  }
  if (!(g->dt > 0.0) || !std::isfinite(g->dt)) {
    set_error("dt must be positive");
    return PIC_EINVAL;
  }
  if (g->deposit != PIC_DEPOSIT_TRISTAN && g->deposit != PIC_DEPOSIT_ISIS) {
    set_error("deposit must be PIC_DEPOSIT_TRISTAN or PIC_DEPOSIT_ISIS");
    return PIC_EINVAL;
  }
  if (g->deposit == PIC_DEPOSIT_ISIS && g->ndim != 2) {
    set_error("the ISIS deposit is defined for 2D3V only");
    return PIC_EUNSUPPORTED;
  }
  if (g->coords != PIC_COORDS_CARTESIAN && g->coords != PIC_COORDS_CYLINDRICAL) {
    set_error("coords must be PIC_COORDS_CARTESIAN or PIC_COORDS_CYLINDRICAL");
    return PIC_EINVAL;
  }
  if (g->coords == PIC_COORDS_CYLINDRICAL) {
    if (g->ndim != 2 || g->deposit != PIC_DEPOSIT_TRISTAN || g->move_window || g->init_e_gauss_x1 ||
        g->smooth_level[0] || g->smooth_level[1]) {
      set_error("the r-z mode needs ndim 2 and the TRISTAN deposit, without smoothing, move_window or "
                "init_e_gauss_x1");
      return PIC_EUNSUPPORTED;
    }
    if (g->bc[1][0] != PIC_BC_AXIAL || g->bc[1][1] != PIC_BC_CONDUCT_ABSORB) {
      set_error("the r-z mode's r boundaries are bc[1] = {PIC_BC_AXIAL, PIC_BC_CONDUCT_ABSORB}");
      return PIC_EINVAL;
    }
    if (std::fabs(g->xmin[1] + 0.5 * g->dx[1]) > 1e-12 * g->dx[1]) {
      set_error("the r-z mode puts the axis through the middle of the first cell: xmin[1] must be -dx[1]/2");
      return PIC_EINVAL;
    }
    // the radial operator's largest eigenvalue with the axis rule is 1.2105 x 4/dr^2
    if (g->dt >= 1.0 / std::sqrt(1.0 / (g->dx[0] * g->dx[0]) + 1.2105 / (g->dx[1] * g->dx[1]))) {
      set_error("Courant condition of the r-z mode violated: dt >= 1/sqrt(1/dz^2 + 1.2105/dr^2)");
      return PIC_ECOURANT;
    }
  }
  if (g->dt >= 1.0 / std::sqrt(s)) {
    set_error("Courant condition violated: dt >= 1/sqrt(sum dx^-2)");
    return PIC_ECOURANT;
  }
  if (g->precision != PIC_FP64_PLAIN && g->precision != PIC_FP32_CELLOFF) {
    set_error("unknown precision");
    return PIC_EINVAL;
  }
  return PIC_OK;
}

}  // namespace

// ============================================================= the C ABI
extern "C" {

const char* pic_last_error(void) { return g_err.c_str(); }

pic_status pic_destroy(pic_sim* S) {
  if (!S) return PIC_OK;
  cudaStreamSynchronize(S->s);
  timing_collect(S);
  for (auto e : S->ev_pool) cudaEventDestroy(e);
  S->al.release_all();
  if (S->hstat) cudaFreeHost(S->hstat);
  if (S->hcnt) cudaFreeHost(S->hcnt);
  delete S;
  return PIC_OK;
}

namespace {
// Loads species k of a simulation being set up from a checkpoint instead of
// the pic_species description.
using RestoreFn = std::function<pic_status(pic_sim*, int, SpeciesState&)>;

pic_status init_sim(const pic_grid* grid, const pic_species* species, int nspecies, const pic_allocator* alloc,
                    void* stream, bool no_small, pic_sim** out, const RestoreFn* restore = nullptr);
}

pic_status pic_init(const pic_grid* grid, const pic_species* species, int nspecies, const pic_allocator* alloc,
                    void* stream, pic_sim** out) {
  return init_sim(grid, species, nspecies, alloc, stream, false, out);
}

namespace {
pic_status init_sim(const pic_grid* grid, const pic_species* species, int nspecies, const pic_allocator* alloc,
                    void* stream, bool no_small, pic_sim** out, const RestoreFn* restore) {
  if (!out) {
    set_error("out is NULL");
    return PIC_EINVAL;
  }
  *out = nullptr;
  pic_status st = validate_grid(grid);
  if (st != PIC_OK) return st;
  if (nspecies < 0 || (nspecies > 0 && !species && !restore)) {
    set_error("bad species list");
    return PIC_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    set_error("no CUDA device");
    return PIC_ECUDA;
  }
  if (grid->move_window && grid->precision != PIC_FP32_CELLOFF) {
    set_error("move_window needs the FP32 cell-offset form");
    return PIC_EUNSUPPORTED;
  }
  pic_sim* S = new pic_sim();
  S->moving = grid->move_window != 0;
  // r-z rings are weighted: the general tile kernel (the small one has no weights)
  S->no_small = no_small || S->moving || grid->coords == PIC_COORDS_CYLINDRICAL;
  S->g = *grid;
  S->ndim = grid->ndim;
  S->prec = grid->precision;
  S->s = reinterpret_cast<cudaStream_t>(stream);
  if (alloc && alloc->alloc) {
    S->al.user = *alloc;
    S->al.has_user = true;
  }
  // a moving window compresses and drags plasma through the tiles: more growth room
  S->slack = grid->slack > 0.0 ? grid->slack : (grid->move_window ? 0.75 : 0.25);
  S->sort_period = grid->sort_period > 0 ? grid->sort_period : 1;
  int nxv[3] = {grid->nx[0], grid->nx[1], grid->ndim == 3 ? grid->nx[2] : 1};
  S->L = make_layout(S->ndim, nxv);
  S->L.open_x = S->moving ? 1 : 0;
  S->cyl = grid->coords == PIC_COORDS_CYLINDRICAL;
  S->K = CylConst{grid->nx[0], grid->nx[1], grid->dx[0], grid->dx[1], grid->dt, ((double)grid->nx[1] - 0.5) * grid->dx[1]};
  if (S->prec == PIC_FP32_CELLOFF) {
    for (int d = 0; d < 3; ++d) S->T[d] = d < S->ndim ? grid->tile[d] : 1;
    if (S->T[0] <= 0 || S->T[1] <= 0 || (S->ndim == 3 && S->T[2] <= 0)) {
      // defaults: 3D 8x8x8, 2D 32x16 (the first shape that divides the grid)
      static const int c3[][3] = {{8, 8, 8}, {16, 8, 4}, {8, 4, 4}, {4, 4, 4}};
      static const int c2[][3] = {{32, 16, 1}, {16, 16, 1}, {16, 8, 1}, {8, 8, 1}};
      S->T[0] = 0;
      for (int k = 0; k < 4 && S->T[0] == 0; ++k) {
        const int* c = S->ndim == 3 ? c3[k] : c2[k];
        bool fits = true;
        for (int d = 0; d < S->ndim; ++d) fits = fits && grid->nx[d] % c[d] == 0;
        if (fits)
          for (int d = 0; d < 3; ++d) S->T[d] = c[d];
      }
      if (S->T[0] == 0) {
        set_error("no supported tile shape divides the grid");
        delete S;
        return PIC_EINVAL;
      }
    }
    int ctas = grid->ctas_per_sm;
    if (ctas == 0)
      if (const char* e = getenv("PICGB_TILE_CTAS")) ctas = atoi(e);
    if (ctas != 0 && ctas != 2 && ctas != 4) {
      set_error("ctas_per_sm must be 0 (default), 2 or 4");
      delete S;
      return PIC_EINVAL;
    }
    S->minb = ctas == 2 ? 2 : 4;
    if (tiled_push_smem_bytes(S->ndim, S->T) < 0) {
      set_error("unsupported tile shape (3D: 4x4x4, 4x4x2, 8x4x4, 8x8x8, 16x8x4; 2D: 8x4, 8x8, 16x8, 16x16, 32x16)");
      delete S;
      return PIC_EUNSUPPORTED;
    }
    for (int d = 0; d < S->ndim; ++d)
      if (grid->nx[d] % S->T[d] != 0) {
        set_error("nx must be a multiple of the tile size in every direction");
        delete S;
        return PIC_EINVAL;
      }
  }
  auto bail = [&](pic_status code) {
    pic_destroy(S);
    return code;
  };
  const size_t eb = elem_bytes(S);
  S->fld = S->al.get(6 * eb * (size_t)S->L.plane);
  S->cur = S->al.get(3 * eb * (size_t)S->L.plane);
  S->tmp = S->al.get(eb * (size_t)S->L.plane);
  S->rho = (double*)S->al.get(8 * (size_t)S->L.plane);
  S->dense = (double*)S->al.get(8 * (size_t)S->L.nx * S->L.ny * S->L.nz);
  S->dacc = (Diag64*)S->al.get(sizeof(Diag64));
  S->dstat = (StatusWord*)S->al.get(sizeof(StatusWord));
  if (!S->fld || !S->cur || !S->tmp || !S->rho || !S->dense || !S->dacc || !S->dstat) {
    set_error("out of device memory (grid arrays)");
    return bail(PIC_ENOMEM);
  }
  if (cudaMallocHost(&S->hcnt, sizeof(int) * 2 * (size_t)std::max(nspecies, 1)) != cudaSuccess) {
    S->hcnt = nullptr;
    set_error("pinned host allocation failed");
    return bail(PIC_ENOMEM);
  }
  if (cudaMallocHost(&S->hstat, sizeof(StatusWord)) != cudaSuccess) {
    S->hstat = nullptr;
    set_error("pinned host allocation failed");
    return bail(PIC_ENOMEM);
  }
  cudaMemsetAsync(S->fld, 0, 6 * eb * (size_t)S->L.plane, S->s);
  cudaMemsetAsync(S->cur, 0, 3 * eb * (size_t)S->L.plane, S->s);
  cudaMemsetAsync(S->tmp, 0, eb * (size_t)S->L.plane, S->s);
  cudaMemsetAsync(S->dstat, 0, sizeof(StatusWord), S->s);
  if ((st = cuda_check("pic_init")) != PIC_OK) return bail(st);
  S->sp.resize((size_t)nspecies);
  for (auto& s : S->sp) s.slack = S->slack;
  for (int k = 0; k < nspecies; ++k) {
    if (S->prec == PIC_FP32_CELLOFF) {
      if ((st = setup_tiles(S, S->sp[k])) != PIC_OK) return bail(st);
    }
    if (restore)
      st = (*restore)(S, k, S->sp[k]);
    else
      st = load_species(S, species[k], S->sp[k]);
    if (st != PIC_OK) return bail(st);
    if (S->prec == PIC_FP32_CELLOFF) {
      if ((st = alloc_spill(S, S->sp[k])) != PIC_OK) return bail(st);
    }
  }
  // explicit positions were checked on the device; nothing may read them
  // before that check is known to have passed
  if (cudaStreamSynchronize(S->s) != cudaSuccess) return bail(cuda_check("pic_init"));
  cudaMemcpy(S->hstat, S->dstat, sizeof(StatusWord), cudaMemcpyDeviceToHost);
  if (S->hstat->status & ST_BADCELL) {
    set_error("initial particle position outside the box or not finite");
    return bail(PIC_EINVAL);
  }
  if (S->prec == PIC_FP32_CELLOFF) {
    if ((st = make_maps(S)) != PIC_OK) return bail(st);
  }
  if (grid->init_e_gauss_x1 && !restore) {
    compute_rho(S);
    if (S->prec == PIC_FP64_PLAIN)
      init_e_gauss_x1<double>(S->L, S->rho, grid->rho_bg, grid->dx[0], fld_ptr<double>(S, 0), S->s);
    else
      init_e_gauss_x1<float>(S->L, S->rho, grid->rho_bg, grid->dx[0], fld_ptr<float>(S, 0), S->s);
  }
  if (S->prec == PIC_FP64_PLAIN) {
    double* f[6];
    for (int c = 0; c < 6; ++c) f[c] = fld_ptr<double>(S, c);
    if (S->cyl)
      cyl_bound<double>(S->L, S->K, f, true, S->s);
    else
      fill_guards<double>(S->L, f, 6, S->s);
  } else {
    float* f[6];
    for (int c = 0; c < 6; ++c) f[c] = fld_ptr<float>(S, c);
    if (S->cyl)
      cyl_bound<float>(S->L, S->K, f, true, S->s);
    else
      fill_guards<float>(S->L, f, 6, S->s);
  }
  if (cudaStreamSynchronize(S->s) != cudaSuccess) return bail(cuda_check("pic_init"));
  if ((st = cuda_check("pic_init")) != PIC_OK) return bail(st);
  cudaMemcpy(S->hstat, S->dstat, sizeof(StatusWord), cudaMemcpyDeviceToHost);
  if (S->hstat->status & ST_BADCELL) {
    set_error("initial particle position outside the box or not finite");
    return bail(PIC_EINVAL);
  }
  *out = S;
  return PIC_OK;
}
}  // namespace

pic_status pic_step(pic_sim* S, int nsteps) {
  if (!S || nsteps < 0) {
    set_error("pic_step: bad arguments");
    return PIC_EINVAL;
  }
  if (S->in_batch) {
    set_error("pic_step: this simulation belongs to a batch; step it with pic_batch_step");
    return PIC_EINVAL;
  }
  pic_status st = PIC_OK;
  const bool tiled = S->prec == PIC_FP32_CELLOFF;
  for (int k = 0; k < nsteps && st == PIC_OK; ++k) st = one_step(S, tiled);
  if (st == PIC_OK && !tiled) {
    cudaMemcpyAsync(S->hstat, S->dstat, sizeof(StatusWord), cudaMemcpyDeviceToHost, S->s);
    if (cudaStreamSynchronize(S->s) != cudaSuccess) return cuda_check("pic_step");
    S->sticky_flags |= S->hstat->status;
    if (S->hstat->status & ST_NONFINITE) {
      set_error("non-finite particle value");
      st = PIC_ENONFINITE;
    }
  }
  if (S->timing) timing_collect(S);
  return st;
}

pic_status pic_fields(pic_sim* S, int which, void* dst, size_t dst_bytes, int dst_on_device) {
  if (!S || !dst || which < PIC_E1 || which > PIC_RHO) {
    set_error("pic_fields: bad arguments");
    return PIC_EINVAL;
  }
  const size_t cells = (size_t)S->L.nx * S->L.ny * S->L.nz;
  if (dst_bytes < 8 * cells) {
    set_error("pic_fields: destination too small");
    return PIC_EINVAL;
  }
  double* target = dst_on_device ? reinterpret_cast<double*>(dst) : S->dense;
  if (which == PIC_RHO) {
    compute_rho(S);
    pack_interior<double>(S->L, S->rho, target, S->s);
  } else if (S->prec == PIC_FP64_PLAIN) {
    const double* src = which <= PIC_B3 ? fld_ptr<double>(S, which) : cur_ptr<double>(S, which - PIC_J1);
    pack_interior<double>(S->L, src, target, S->s);
  } else {
    const float* src = which <= PIC_B3 ? fld_ptr<float>(S, which) : cur_ptr<float>(S, which - PIC_J1);
    pack_interior<float>(S->L, src, target, S->s);
  }
  if (!dst_on_device) cudaMemcpyAsync(dst, S->dense, 8 * cells, cudaMemcpyDeviceToHost, S->s);
  if (cudaStreamSynchronize(S->s) != cudaSuccess) return cuda_check("pic_fields");
  return cuda_check("pic_fields");
}

pic_status pic_set_field(pic_sim* S, int which, const void* src, size_t src_bytes, int src_on_device) {
  if (!S || !src || which < PIC_E1 || which > PIC_B3) {
    set_error("pic_set_field: bad arguments");
    return PIC_EINVAL;
  }
  const size_t cells = (size_t)S->L.nx * S->L.ny * S->L.nz;
  if (src_bytes < 8 * cells) {
    set_error("pic_set_field: source too small");
    return PIC_EINVAL;
  }
  const double* from = reinterpret_cast<const double*>(src);
  if (!src_on_device) {
    cudaMemcpyAsync(S->dense, src, 8 * cells, cudaMemcpyHostToDevice, S->s);
    from = S->dense;
  }
  if (S->prec == PIC_FP64_PLAIN) {
    double* f = fld_ptr<double>(S, which);
    unpack_interior<double>(S->L, from, f, S->s);
    double* all[6];
    for (int c = 0; c < 6; ++c) all[c] = fld_ptr<double>(S, c);
    if (S->cyl)
      cyl_bound<double>(S->L, S->K, all, true, S->s);
    else
      fill_guards<double>(S->L, all, 6, S->s);
  } else {
    float* f = fld_ptr<float>(S, which);
    unpack_interior<float>(S->L, from, f, S->s);
    float* all[6];
    for (int c = 0; c < 6; ++c) all[c] = fld_ptr<float>(S, c);
    if (S->cyl)
      cyl_bound<float>(S->L, S->K, all, true, S->s);
    else
      fill_guards<float>(S->L, all, 6, S->s);
  }
  if (cudaStreamSynchronize(S->s) != cudaSuccess) return cuda_check("pic_set_field");
  return cuda_check("pic_set_field");
}

pic_status pic_particles(pic_sim* S, int species, double* x, double* u, long long cap, long long* n_out,
                         int dst_on_device) {
  if (!S || species < 0 || species >= (int)S->sp.size() || !n_out) {
    set_error("pic_particles: bad arguments");
    return PIC_EINVAL;
  }
  SpeciesState& sp = S->sp[(size_t)species];
  if (S->prec == PIC_FP64_PLAIN) {
    const long long n = sp.plain.n;
    *n_out = n;
    if (n > cap) {
      set_error("pic_particles: capacity too small");
      return PIC_EOVERFLOW;
    }
    if (n == 0) return PIC_OK;
    double* tmp = dst_on_device ? nullptr : (double*)S->al.get(24 * (size_t)n);
    if (!dst_on_device && !tmp) {
      set_error("out of device memory (copy-out)");
      return PIC_ENOMEM;
    }
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (x) {
      double* d = dst_on_device ? x : tmp;
      k_soa_to_aos3<<<nb, 256, 0, S->s>>>(sp.plain.x[0], sp.plain.x[1], S->ndim == 3 ? sp.plain.x[2] : nullptr, n,
                                          d);
      if (!dst_on_device) cudaMemcpyAsync(x, tmp, 24 * (size_t)n, cudaMemcpyDeviceToHost, S->s);
      cudaStreamSynchronize(S->s);
    }
    if (u) {
      double* d = dst_on_device ? u : tmp;
      k_soa_to_aos3<<<nb, 256, 0, S->s>>>(sp.plain.u[0], sp.plain.u[1], sp.plain.u[2], n, d);
      if (!dst_on_device) cudaMemcpyAsync(u, tmp, 24 * (size_t)n, cudaMemcpyDeviceToHost, S->s);
      cudaStreamSynchronize(S->s);
    }
    S->al.put(tmp);
    return cuda_check("pic_particles");
  }
  Flat32 flat{};
  long long n = 0;
  bool allocated = false;
  pic_status st = flatten(S, sp, flat, n, false, 0, allocated);
  if (st != PIC_OK) {
    if (allocated) free_flat(S, flat);
    return st;
  }
  *n_out = n;
  if (n > cap) {
    free_flat(S, flat);
    set_error("pic_particles: capacity too small");
    return PIC_EOVERFLOW;
  }
  PushConst C = make_const(S, sp);
  double* tx = (x && !dst_on_device) ? (double*)S->al.get(24 * (size_t)std::max<long long>(n, 1)) : x;
  double* tu = (u && !dst_on_device) ? (double*)S->al.get(24 * (size_t)std::max<long long>(n, 1)) : u;
  if ((x && !tx) || (u && !tu)) {
    free_flat(S, flat);
    set_error("out of device memory (copy-out)");
    return PIC_ENOMEM;
  }
  flat_to_global(S->ndim, sp.tg, C, flat, n, tx, tu, S->s);
  if (x && !dst_on_device) cudaMemcpyAsync(x, tx, 24 * (size_t)n, cudaMemcpyDeviceToHost, S->s);
  if (u && !dst_on_device) cudaMemcpyAsync(u, tu, 24 * (size_t)n, cudaMemcpyDeviceToHost, S->s);
  cudaStreamSynchronize(S->s);
  if (x && !dst_on_device) S->al.put(tx);
  if (u && !dst_on_device) S->al.put(tu);
  free_flat(S, flat);
  return cuda_check("pic_particles");
}

pic_status pic_particle_ids(pic_sim* S, int species, int* ids, long long cap, long long* n_out, int dst_on_device) {
  if (!S || species < 0 || species >= (int)S->sp.size() || !n_out || !ids) {
    set_error("pic_particle_ids: bad arguments");
    return PIC_EINVAL;
  }
  SpeciesState& sp = S->sp[(size_t)species];
  if (!sp.ids) {
    set_error("pic_particle_ids: species was created without track_ids");
    return PIC_EINVAL;
  }
  if (S->prec == PIC_FP64_PLAIN) {
    *n_out = sp.plain.n;
    if (sp.plain.n > cap) {
      set_error("pic_particle_ids: capacity too small");
      return PIC_EOVERFLOW;
    }
    cudaMemcpyAsync(ids, sp.plain.id, 4 * (size_t)sp.plain.n,
                    dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, S->s);
    cudaStreamSynchronize(S->s);
    return cuda_check("pic_particle_ids");
  }
  Flat32 flat{};
  long long n = 0;
  bool allocated = false;
  pic_status st = flatten(S, sp, flat, n, false, 0, allocated);
  if (st != PIC_OK) {
    if (allocated) free_flat(S, flat);
    return st;
  }
  *n_out = n;
  if (n > cap) {
    free_flat(S, flat);
    set_error("pic_particle_ids: capacity too small");
    return PIC_EOVERFLOW;
  }
  cudaMemcpyAsync(ids, flat.id, 4 * (size_t)n, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                  S->s);
  cudaStreamSynchronize(S->s);
  free_flat(S, flat);
  return cuda_check("pic_particle_ids");
}

pic_status pic_particle_weights(pic_sim* S, int species, double* w, long long cap, long long* n_out,
                                int dst_on_device) {
  if (!S || species < 0 || species >= (int)S->sp.size() || !n_out || !w) {
    set_error("pic_particle_weights: bad arguments");
    return PIC_EINVAL;
  }
  SpeciesState& sp = S->sp[(size_t)species];
  Flat32 flat{};
  long long n = sp.n;
  bool allocated = false;
  if (S->prec == PIC_FP32_CELLOFF) {
    const pic_status st = flatten(S, sp, flat, n, false, 0, allocated);
    if (st != PIC_OK) {
      if (allocated) free_flat(S, flat);
      return st;
    }
  } else {
    n = sp.plain.n;
  }
  *n_out = n;
  if (n > cap) {
    if (allocated) free_flat(S, flat);
    set_error("pic_particle_weights: capacity too small");
    return PIC_EOVERFLOW;
  }
  double* d = (double*)S->al.get(8 * (size_t)std::max<long long>(n, 1));
  if (!d) {
    if (allocated) free_flat(S, flat);
    set_error("out of device memory (weights)");
    return PIC_ENOMEM;
  }
  if (n > 0) {
    if (S->prec == PIC_FP64_PLAIN && sp.plain.w)
      cudaMemcpyAsync(d, sp.plain.w, 8 * (size_t)n, cudaMemcpyDeviceToDevice, S->s);
    else
      k_widen<<<(unsigned)((n + 255) / 256), 256, 0, S->s>>>(S->prec == PIC_FP32_CELLOFF ? flat.w : nullptr, d, n);
    cudaMemcpyAsync(w, d, 8 * (size_t)n, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, S->s);
  }
  cudaStreamSynchronize(S->s);
  S->al.put(d);
  if (allocated) free_flat(S, flat);
  return cuda_check("pic_particle_weights");
}

pic_status pic_tile_counts(pic_sim* S, int species, long long* counts, long long cap, long long* ntiles_out) {
  if (!S || species < 0 || species >= (int)S->sp.size() || !ntiles_out) {
    set_error("pic_tile_counts: bad arguments");
    return PIC_EINVAL;
  }
  if (S->prec != PIC_FP32_CELLOFF) {
    set_error("pic_tile_counts: only the FP32 cell-offset form stores particles by tile");
    return PIC_EINVAL;
  }
  SpeciesState& sp = S->sp[(size_t)species];
  const int nt = sp.tg.ntiles;
  *ntiles_out = nt;
  if (!counts || cap < nt) {
    set_error("pic_tile_counts: capacity too small");
    return PIC_EOVERFLOW;
  }
  Flat32 flat{};
  long long n = 0;
  bool allocated = false;
  pic_status st = flatten(S, sp, flat, n, false, 0, allocated);
  if (st != PIC_OK) {
    if (allocated) free_flat(S, flat);
    return st;
  }
  int* dc = (int*)S->al.get(4 * (size_t)nt);
  if (!dc) {
    free_flat(S, flat);
    set_error("out of device memory");
    return PIC_ENOMEM;
  }
  cudaMemsetAsync(dc, 0, 4 * (size_t)nt, S->s);
  flat_count(flat, n, nt, dc, S->s);
  std::vector<int> h((size_t)nt);
  cudaMemcpyAsync(h.data(), dc, 4 * (size_t)nt, cudaMemcpyDeviceToHost, S->s);
  cudaStreamSynchronize(S->s);
  for (int t = 0; t < nt; ++t) counts[t] = h[(size_t)t];
  S->al.put(dc);
  free_flat(S, flat);
  return cuda_check("pic_tile_counts");
}

pic_status pic_diag(pic_sim* S, pic_diag_t* out) {
  if (!S || !out) {
    set_error("pic_diag: bad arguments");
    return PIC_EINVAL;
  }
  cudaMemsetAsync(S->dacc, 0, sizeof(Diag64), S->s);
  compute_rho(S, S->prec == PIC_FP64_PLAIN ? nullptr : S->dacc);
  double dx[3] = {S->g.dx[0], S->g.dx[1], S->ndim == 3 ? S->g.dx[2] : 1.0};
  long long n = 0;
  if (S->cyl && S->prec == PIC_FP64_PLAIN) {
    double* f[6];
    for (int c = 0; c < 6; ++c) f[c] = fld_ptr<double>(S, c);
    cyl_diag<double>(S->L, S->K, f, S->rho, S->g.rho_bg, S->dacc, S->s);
  } else if (S->cyl) {
    float* f[6];
    for (int c = 0; c < 6; ++c) f[c] = fld_ptr<float>(S, c);
    cyl_diag<float>(S->L, S->K, f, S->rho, S->g.rho_bg, S->dacc, S->s);
  } else if (S->prec == PIC_FP64_PLAIN) {
    double* f[6];
    for (int c = 0; c < 6; ++c) f[c] = fld_ptr<double>(S, c);
    gauss_residual<double>(S->L, f, S->rho, S->g.rho_bg, dx, S->dacc, S->s);
    field_energy<double>(S->L, f, S->dacc, S->s);
  } else {
    float* f[6];
    for (int c = 0; c < 6; ++c) f[c] = fld_ptr<float>(S, c);
    diag_fields(S->L, f, S->rho, S->g.rho_bg, dx, S->dacc, S->s);
  }
  for (auto& sp : S->sp) {
    PushConst C = make_const(S, sp);
    if (S->cyl && S->prec == PIC_FP64_PLAIN)
      cyl_kinetic(C, sp.plain, S->dacc, S->s);
    else if (S->prec == PIC_FP64_PLAIN && !S->cyl)
      plain_kinetic(C, sp.plain, S->dacc, S->s);
    n += sp.n;
  }
  Diag64 h{};
  cudaMemcpyAsync(&h, S->dacc, sizeof(Diag64), cudaMemcpyDeviceToHost, S->s);
  cudaMemcpyAsync(S->hstat, S->dstat, sizeof(StatusWord), cudaMemcpyDeviceToHost, S->s);
  if (cudaStreamSynchronize(S->s) != cudaSuccess) return cuda_check("pic_diag");
  double dvol = 1.0;
  for (int d = 0; d < S->ndim; ++d) dvol *= S->g.dx[d];
  out->step = S->step;
  out->time = (double)S->step * S->g.dt;
  out->field_energy = 0.5 * h.field_energy * dvol;
  out->kinetic_energy = h.kinetic_energy;
  out->total_charge = h.total_charge;
  if (S->cyl) {  // per-radian sums (field energy already volume-weighted) over the full 2 pi
    const double two_pi = 2.0 * 3.141592653589793;
    out->field_energy = 0.5 * h.field_energy * two_pi;
    out->kinetic_energy = h.kinetic_energy * two_pi;
    out->total_charge = h.total_charge * two_pi;
  }
  out->gauss_resid_max = h.gauss_max;
  out->rho_abs_max = h.rho_max;
  out->rho_particles_abs_max = h.rho_part_max;
  out->n_particles = n;
  const int f = S->sticky_flags | S->hstat->status;
  out->error_flags = ((f & (ST_NONFINITE | ST_BADCELL)) ? 1 : 0) | ((f & ST_SPILL) ? 2 : 0);
  return cuda_check("pic_diag");
}

pic_status pic_timing_enable(pic_sim* S, int enable) {
  if (!S) {
    set_error("pic_timing_enable: NULL handle");
    return PIC_EINVAL;
  }
  S->timing = enable != 0;
  return PIC_OK;
}

pic_status pic_timing_read(pic_sim* S, double* ms, long long* launches, int nslots, int reset) {
  if (!S || nslots < 0) {
    set_error("pic_timing_read: bad arguments");
    return PIC_EINVAL;
  }
  timing_collect(S);
  for (int k = 0; k < nslots && k < kTimingSlots; ++k) {
    if (ms) ms[k] = S->t_ms[k];
    if (launches) launches[k] = S->t_n[k];
  }
  if (nslots > kLaunchSlot) {
    if (ms) ms[kLaunchSlot] = 0.0;
    if (launches) launches[kLaunchSlot] = S->nlaunch;
  }
  if (reset) {
    for (int k = 0; k < kTimingSlots; ++k) {
      S->t_ms[k] = 0.0;
      S->t_n[k] = 0;
    }
    S->nlaunch = 0;
  }
  return PIC_OK;
}


// ------------------------------------------------------------- batched scan

struct pic_batch {
  std::vector<pic_sim*> sims;
  std::vector<std::pair<int, int>> ent;  // (simulation, species) of each table entry
  cudaStream_t s = nullptr;      // the batch's own stream (capturable): all member work after set-up
  cudaStream_t user = nullptr;   // the caller's stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  Allocator al;
  int ndim = 0;
  int T[3] = {1, 1, 1};
  void* d_args[2] = {nullptr, nullptr};  // entry tables for store side 0 / 1 as input
  CUtensorMap* d_fmaps = nullptr;
  CUtensorMap* d_jmaps = nullptr;
  int* d_tile0 = nullptr;
  int* d_work = nullptr;
  StatusWord* d_stat = nullptr;  // one per simulation
  StatusWord* h_stat = nullptr;  // pinned mirror
  int grid = 0;
  int minb = 4;
  bool use_graph = true;
  bool dirty = true;  // tables / graphs must be rebuilt before the next step
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  long long step = 0;
  long long nlaunch = 0;
  // moving windows (members with move_window): the dropped / created
  // particle counters of every (member, species) gathered into one array per
  // step
  bool moving = false;
  int** d_cnt_src = nullptr;  // [2 nent]: each entry's d_lost, d_kept
  int* d_cnt = nullptr;       // [2 nent]
  int* h_cnt = nullptr;       // pinned mirror
  // the field step of all members, one launch per stage
  BatchFieldTable ft{};
  BatchFieldMember* d_fm = nullptr;
  int* d_blk = nullptr;  // first blocks per member: interior, guard, shift-row launches ([nsims + 1] each)
  int nblk_int = 0, nblk_guard = 0, nblk_rows = 0;
  BatchZeroSeg* d_zseg[2] = {nullptr, nullptr};  // per input side: every current, every arrival counter
  int* d_zblk[2] = {nullptr, nullptr};
  int nzseg = 0;
  int nzblk[2] = {0, 0};
  void* d_ispec = nullptr;  // front-column injection records (moving windows)
  int* d_iblk = nullptr;
  int ninj_blk = 0;
  // values of the next step read on the device (so that a captured step can
  // be replayed): shift flag per member, the window's x1 corner after its
  // shift per member, antenna time and x1 corner per member, first fresh
  // particle index per entry; filled on the host before each step
  unsigned char* h_dyn = nullptr;  // pinned
  unsigned char* d_dyn = nullptr;
  size_t dyn_bytes = 0, off_xinj = 0, off_ant = 0, off_first = 0;
  long long ants_built = -1;  // antenna pulses of all members when the step was built
  int* shift_flags() const { return reinterpret_cast<int*>(d_dyn); }
  int* h_shift_flags() const { return reinterpret_cast<int*>(h_dyn); }
};

namespace {

// the moving-window decision of one member for the step it is about to take
// (the same rule as one_step: the step whose end brings c t a full cell past
// the last shift ends with a shift; the window moves from window_start on)
bool window_shift_due(const pic_sim* S) {
  if (!S->moving) return false;
  const double lag = (double)(S->step + 1) * S->g.dt - S->g.window_start;
  return lag > 0.0 && (long long)std::floor(lag / S->g.dx[0]) > S->shifts;
}

void batch_drop_graphs(pic_batch* B) {
  for (int p = 0; p < 2; ++p)
    if (B->exec[p]) {
      cudaGraphExecDestroy(B->exec[p]);
      B->exec[p] = nullptr;
    }
}

long long batch_antennas(const pic_batch* B) {
  long long n = 0;
  for (const pic_sim* S : B->sims) n += S->n_ants;
  return n;
}

// The next step's per-member values into the pinned block (read on the
// device after the step's first copy): the moving-window decision as in
// one_step, the window corner the fresh column is created at, the antenna time
// and corner, and every entry's first fresh particle index.
void batch_prepare(pic_batch* B) {
  const int nsims = (int)B->sims.size();
  int* shift = B->h_shift_flags();
  double* xinj = reinterpret_cast<double*>(B->h_dyn + B->off_xinj);
  double* ant = reinterpret_cast<double*>(B->h_dyn + B->off_ant);
  long long* first = reinterpret_cast<long long*>(B->h_dyn + B->off_first);
  for (int i = 0; i < nsims; ++i) {
    const pic_sim* S = B->sims[i];
    shift[i] = window_shift_due(S) ? 1 : 0;
    xinj[i] = S->g.xmin[0] + S->g.dx[0];
    ant[2 * i] = ((double)S->step + 0.5) * S->g.dt;
    ant[2 * i + 1] = S->g.xmin[0];
  }
  for (size_t k = 0; k < B->ent.size(); ++k) first[k] = B->sims[B->ent[k].first]->sp[B->ent[k].second].created;
}

// The host's record of the step just taken: members that shifted moved their
// window and used up their lattice places of the front column.
void batch_after_step(pic_batch* B) {
  const int* shift = B->h_shift_flags();
  for (int i = 0; i < (int)B->sims.size(); ++i) {
    if (!shift[i]) continue;
    pic_sim* S = B->sims[i];
    for (auto& sp : S->sp) sp.created += (long long)S->L.ny * S->L.nz * sp.ppc[0] * sp.ppc[1] * sp.ppc[2];
    S->g.xmin[0] += S->g.dx[0];
    ++S->shifts;
  }
}

// Everything one step enqueues for all simulations, store side p as input:
// the step's values to the device, then one launch per stage for all members
// (currents and arrival counters cleared, the batched tile kernel, fresh front
// columns, current fold, B half step, E step, B half step, window shift,
// guards), per-member launches only for smoothing passes and antenna planes.
// It reads nothing from the host after the first copy, so it can be captured.
void batch_enqueue(pic_batch* B, int p) {
  const int nsims = (int)B->sims.size();
  const int nent = (int)B->ent.size();
  cudaMemcpyAsync(B->d_dyn, B->h_dyn, B->dyn_bytes, cudaMemcpyHostToDevice, B->s);
  batch_zero(B->d_zseg[p], B->d_zblk[p], B->nzseg, B->nzblk[p], B->s);
  tiled_push_batch(B->ndim, B->T, B->d_args[p], B->d_fmaps, B->d_jmaps, B->d_tile0, nent, B->d_work, B->grid,
                   B->minb, B->s);
  if (B->moving)
    tiled_inject_batch(B->d_args[p], B->d_ispec, B->d_iblk, nent, B->ninj_blk, B->shift_flags(),
                       reinterpret_cast<const double*>(B->d_dyn + B->off_xinj),
                       reinterpret_cast<const long long*>(B->d_dyn + B->off_first), B->s);
  batch_fold(B->ft, B->nblk_guard, B->s);
  for (pic_sim* S : B->sims)  // smoothing passes, as field_step
    for (int d = 0; d < S->ndim; ++d)
      for (int pass = 0; pass < S->g.smooth_level[d]; ++pass) {
        const double* w = S->g.smooth_w[d][pass];
        for (int c = 0; c < 3; ++c)
          smooth_pass<float>(S->L, cur_ptr<float>(S, c), reinterpret_cast<float*>(S->tmp), d, w[0], w[1], w[2],
                             B->s);
      }
  batch_yee_b(B->ft, B->nblk_int, B->s);
  for (int i = 0; i < nsims; ++i) {
    pic_sim* S = B->sims[i];
    if (S->n_ants > 0)
      antenna_plane(S->L, S->d_ants, S->n_ants, 0.0, 0.0, S->d_inc, B->s,
                    reinterpret_cast<const double*>(B->d_dyn + B->off_ant) + 2 * i);
  }
  batch_yee_e(B->ft, B->nblk_int, B->s);
  batch_yee_b(B->ft, B->nblk_int, B->s);
  if (B->moving) batch_shift(B->ft, B->nblk_rows, B->s);
  batch_fill(B->ft, B->nblk_guard, B->s);
  if (B->moving)
    k_batch_gather_counts<<<(unsigned)((2 * nent + 127) / 128), 128, 0, B->s>>>(B->d_cnt_src, B->d_cnt, 2 * nent);
}

long long batch_launches_per_step(const pic_batch* B) {
  long long n = 6;  // clear, tile kernel, fold, B half, E, B half
  n += B->nblk_guard > 0 ? 1 : 0;  // guards
  if (B->moving) n += (B->ninj_blk > 0 ? 1 : 0) + 2;  // fresh columns, shift, counter gather
  for (const pic_sim* S : B->sims) {
    for (int d = 0; d < S->ndim; ++d) n += 3 * (long long)S->g.smooth_level[d];
    if (S->n_ants > 0) n += 1;  // the antenna plane
  }
  return n;
}

pic_status batch_build(pic_batch* B) {
  batch_drop_graphs(B);
  const int n = (int)B->ent.size();
  const size_t ab = tiled_args_bytes();
  std::vector<unsigned char> args(ab * n);
  std::vector<CUtensorMap> fm(B->sims.size()), jm(B->sims.size());
  std::vector<CUtensorMap> fme(n), jme(n);
  std::vector<int> tile0(n + 1, 0);
  for (int p = 0; p < 2; ++p) {
    for (int k = 0; k < n; ++k) {
      pic_sim* S = B->sims[B->ent[k].first];
      SpeciesState& sp = S->sp[B->ent[k].second];
      if (sp.tg.small) {
        set_error("pic_batch: a member simulation uses the small-tile kernel");
        return PIC_EUNSUPPORTED;
      }
      PushConst C = make_const(S, sp);
      StatusWord* st = S->dstat;
      tiled_fill_args(args.data() + ab * k, C, sp.tg, sp.side[p], sp.side[1 - p], sp.spill, sp.d_spill,
                      sp.spill_cap, &st->status, S->L.open_x, S->moving ? sp.d_lost : nullptr,
                      S->moving ? B->shift_flags() + B->ent[k].first : nullptr);
      if (p == 0) {
        fme[k] = S->fmap;
        jme[k] = S->jmap;
        tile0[k + 1] = tile0[k] + sp.tg.ntiles;
      }
    }
    cudaMemcpyAsync(B->d_args[p], args.data(), ab * n, cudaMemcpyHostToDevice, B->s);
  }
  cudaMemcpyAsync(B->d_fmaps, fme.data(), sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice, B->s);
  cudaMemcpyAsync(B->d_jmaps, jme.data(), sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice, B->s);
  cudaMemcpyAsync(B->d_tile0, tile0.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, B->s);
  B->grid = tiled_batch_grid(B->ndim, B->T, tile0[n], B->minb);
  if (B->grid <= 0) {
    set_error("pic_batch: tile shape not supported by the batched kernel");
    return PIC_EUNSUPPORTED;
  }
  // the batched field step: one record and the first blocks per member
  const int nsims = (int)B->sims.size();
  std::vector<BatchFieldMember> fmem(nsims);
  std::vector<int> blk(3 * (size_t)(nsims + 1), 0);
  int* bi = blk.data();
  int* bg = bi + nsims + 1;
  int* br = bg + nsims + 1;
  for (int i = 0; i < nsims; ++i) {
    pic_sim* S = B->sims[i];
    BatchFieldMember& m = fmem[i];
    m.L = S->L;
    for (int c = 0; c < 6; ++c) m.f[c] = fld_ptr<float>(S, c);
    for (int c = 0; c < 3; ++c) m.j[c] = cur_ptr<float>(S, c);
    const double dx3 = S->ndim == 3 ? S->g.dx[2] : 1.0;  // the constants yee_b_half / yee_e pass
    m.h = (float)(S->g.dt / 2.0);
    m.dt = (float)S->g.dt;
    m.i1 = (float)(1.0 / S->g.dx[0]);
    m.i2 = (float)(1.0 / S->g.dx[1]);
    m.i3 = (float)(1.0 / dx3);
    m.inc = S->n_ants > 0 ? S->d_inc : nullptr;
    bi[i + 1] = bi[i] + batch_interior_blocks(S->L);
    bg[i + 1] = bg[i] + batch_guard_blocks(S->L);
    br[i + 1] = br[i] + batch_row_blocks(S->L);
  }
  B->nblk_int = bi[nsims];
  B->nblk_guard = bg[nsims];
  B->nblk_rows = br[nsims];
  cudaMemcpyAsync(B->d_fm, fmem.data(), sizeof(BatchFieldMember) * nsims, cudaMemcpyHostToDevice, B->s);
  cudaMemcpyAsync(B->d_blk, blk.data(), sizeof(int) * blk.size(), cudaMemcpyHostToDevice, B->s);
  B->ft.m = B->d_fm;
  B->ft.blk_int = B->d_blk;
  B->ft.blk_guard = B->d_blk + nsims + 1;
  B->ft.blk_rows = B->d_blk + 2 * (nsims + 1);
  B->ft.shift = B->shift_flags();
  B->ft.n = nsims;
  // what each step clears, per input side: the currents, then the arrival
  // counters of the output side
  std::vector<BatchZeroSeg> zs(B->nzseg);
  std::vector<int> zb(B->nzseg + 1);
  for (int p = 0; p < 2; ++p) {
    for (int i = 0; i < nsims; ++i) zs[i] = BatchZeroSeg{B->sims[i]->cur, 3 * (long long)B->sims[i]->L.plane};
    for (int k = 0; k < n; ++k) {
      SpeciesState& sp = B->sims[B->ent[k].first]->sp[B->ent[k].second];
      zs[nsims + k] = BatchZeroSeg{sp.side[1 - p].inc, (long long)sp.tg.ntiles};
    }
    zb[0] = 0;
    for (int q = 0; q < B->nzseg; ++q) zb[q + 1] = zb[q] + batch_zero_blocks(zs[q].words);
    B->nzblk[p] = zb[B->nzseg];
    cudaMemcpyAsync(B->d_zseg[p], zs.data(), sizeof(BatchZeroSeg) * zs.size(), cudaMemcpyHostToDevice, B->s);
    cudaMemcpyAsync(B->d_zblk[p], zb.data(), sizeof(int) * zb.size(), cudaMemcpyHostToDevice, B->s);
    if (cudaStreamSynchronize(B->s) != cudaSuccess) return cuda_check("pic_batch tables");  // zs reused
  }
  // the fresh front column of every entry of a moving member
  if (B->moving) {
    const size_t rb = tiled_inject_spec_bytes();
    std::vector<unsigned char> rec(rb * n);
    std::vector<int> ib(n + 1, 0);
    for (int k = 0; k < n; ++k) {
      pic_sim* S = B->sims[B->ent[k].first];
      SpeciesState& sp = S->sp[B->ent[k].second];
      const long long cnt = S->moving ? (long long)S->L.ny * S->L.nz * sp.ppc[0] * sp.ppc[1] * sp.ppc[2] : 0;
      const int nxs[3] = {S->L.nx, S->L.ny, S->L.nz};
      tiled_fill_inject(rec.data() + rb * k, make_const(S, sp), sp.tg, nxs, sp.ppc, sp.uth, sp.ufl, sp.seed,
                        sp.has_prof ? &sp.prof : nullptr, sp.d_kept, B->ent[k].first, cnt);
      ib[k + 1] = ib[k] + (int)((cnt + 255) / 256);
    }
    B->ninj_blk = ib[n];
    cudaMemcpyAsync(B->d_ispec, rec.data(), rec.size(), cudaMemcpyHostToDevice, B->s);
    cudaMemcpyAsync(B->d_iblk, ib.data(), sizeof(int) * ib.size(), cudaMemcpyHostToDevice, B->s);
    if (cudaStreamSynchronize(B->s) != cudaSuccess) return cuda_check("pic_batch tables");
  }
  B->ants_built = batch_antennas(B);
  if (cudaStreamSynchronize(B->s) != cudaSuccess) return cuda_check("pic_batch tables");
  if (B->use_graph) {
    for (int p = 0; p < 2; ++p) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(B->s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cuda_check("pic_batch capture");
      batch_enqueue(B, p);
      if (cudaStreamEndCapture(B->s, &g) != cudaSuccess) return cuda_check("pic_batch capture");
      const cudaError_t e = cudaGraphInstantiate(&B->exec[p], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_check("pic_batch graph");
    }
  }
  B->dirty = false;
  return cuda_check("pic_batch build");
}

}  // namespace

pic_status pic_batch_init(int nsims, const pic_grid* grids, const pic_species* species, int nspecies,
                          const pic_allocator* alloc, void* stream, pic_batch** out) {
  if (!out || nsims < 1 || !grids || nspecies < 1 || !species) {
    set_error("pic_batch_init: bad arguments");
    return PIC_EINVAL;
  }
  *out = nullptr;
  const int ndim = grids[0].ndim;
  for (int i = 0; i < nsims; ++i) {
    if (grids[i].coords != PIC_COORDS_CARTESIAN) {
      // the batched step has no r-z field solve: such a member is refused, not mis-stepped
      set_error("pic_batch_init: simulation " + std::to_string(i) +
                " asks for the r-z mode, which the batched step does not do");
      return PIC_EUNSUPPORTED;
    }
    if (grids[i].precision != PIC_FP32_CELLOFF || grids[i].ndim != ndim) {
      set_error("pic_batch_init: every simulation must be FP32 cell-offset, with the same ndim");
      return PIC_EINVAL;
    }
    for (int d = 0; d < 3; ++d)
      if (grids[i].tile[d] != grids[0].tile[d]) {
        set_error("pic_batch_init: every simulation must use the same tile shape");
        return PIC_EINVAL;
      }
    if (grids[i].ctas_per_sm != grids[0].ctas_per_sm) {
      set_error("pic_batch_init: every simulation must use the same ctas_per_sm");
      return PIC_EINVAL;
    }
  }
  // tile shape: the given one, else the first general shape dividing every grid
  int T[3] = {grids[0].tile[0], grids[0].tile[1], ndim == 3 ? grids[0].tile[2] : 1};
  if (T[0] <= 0) {
    static const int c3[][3] = {{8, 8, 8}, {16, 8, 4}};
    static const int c2[][3] = {{32, 16, 1}, {16, 16, 1}, {8, 8, 1}};
    const int nc = ndim == 3 ? 2 : 3;
    T[0] = 0;
    for (int k = 0; k < nc && T[0] == 0; ++k) {
      const int* c = ndim == 3 ? c3[k] : c2[k];
      bool fits = true;
      for (int i = 0; i < nsims; ++i)
        for (int d = 0; d < ndim; ++d) fits = fits && grids[i].nx[d] % c[d] == 0;
      if (fits)
        for (int d = 0; d < 3; ++d) T[d] = c[d];
    }
    if (T[0] == 0) {
      set_error("pic_batch_init: no batched tile shape divides every grid");
      return PIC_EINVAL;
    }
  }
  pic_batch* B = new pic_batch();
  B->user = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    set_error("pic_batch_init: stream or event creation failed");
    pic_batch_destroy(B);
    return PIC_ECUDA;
  }
  B->ndim = ndim;
  B->minb = grids[0].ctas_per_sm == 2 ? 2 : 4;
  for (int d = 0; d < 3; ++d) B->T[d] = T[d];
  if (alloc && alloc->alloc) {
    B->al.user = *alloc;
    B->al.has_user = true;
  }
  if (const char* e = getenv("PICGB_BATCH_GRAPH")) B->use_graph = atoi(e) != 0;
  auto bail = [&](pic_status code) {
    pic_batch_destroy(B);
    return code;
  };
  for (int i = 0; i < nsims; ++i) {
    pic_grid g = grids[i];
    for (int d = 0; d < 3; ++d) g.tile[d] = T[d];
    g.sort_period = 1;
    pic_sim* S = nullptr;
    const pic_status st = init_sim(&g, species + (size_t)i * nspecies, nspecies, alloc, stream, true, &S);
    if (st != PIC_OK) {
      const std::string msg = "simulation " + std::to_string(i) + ": " + g_err;
      set_error(msg);
      return bail(st);
    }
    B->sims.push_back(S);
    for (int k = 0; k < nspecies; ++k) B->ent.push_back({i, k});
  }
  // the particle launch takes work items in entry order: the densest entries
  // (most particles per tile) first, so that their heavy tiles start early
  // and the small tiles of sparse members fill the end of the launch
  std::stable_sort(B->ent.begin(), B->ent.end(), [&](const std::pair<int, int>& a, const std::pair<int, int>& b) {
    const SpeciesState& sa = B->sims[a.first]->sp[a.second];
    const SpeciesState& sb = B->sims[b.first]->sp[b.second];
    return (double)sa.n * sb.tg.ntiles > (double)sb.n * sa.tg.ntiles;
  });
  const int n = (int)B->ent.size();
  B->d_args[0] = B->al.get(tiled_args_bytes() * n);
  B->d_args[1] = B->al.get(tiled_args_bytes() * n);
  B->d_fmaps = (CUtensorMap*)B->al.get(sizeof(CUtensorMap) * n);
  B->d_jmaps = (CUtensorMap*)B->al.get(sizeof(CUtensorMap) * n);
  B->d_tile0 = (int*)B->al.get(sizeof(int) * (n + 1));
  B->d_work = (int*)B->al.get(sizeof(int));
  B->d_stat = (StatusWord*)B->al.get(sizeof(StatusWord) * nsims);
  if (!B->d_args[0] || !B->d_args[1] || !B->d_fmaps || !B->d_jmaps || !B->d_tile0 || !B->d_work || !B->d_stat) {
    set_error("pic_batch_init: out of device memory (tables)");
    return bail(PIC_ENOMEM);
  }
  if (cudaMallocHost(&B->h_stat, sizeof(StatusWord) * nsims) != cudaSuccess) {
    B->h_stat = nullptr;
    set_error("pic_batch_init: pinned host allocation failed");
    return bail(PIC_ENOMEM);
  }
  for (pic_sim* S : B->sims) B->moving = B->moving || S->moving;
  // batched field step tables and the per-step block (pinned mirror)
  B->nzseg = nsims + n;
  B->off_xinj = ((sizeof(int) * nsims + 7) / 8) * 8;
  B->off_ant = B->off_xinj + sizeof(double) * nsims;
  B->off_first = B->off_ant + 2 * sizeof(double) * nsims;
  B->dyn_bytes = B->off_first + sizeof(long long) * n;
  B->d_fm = (BatchFieldMember*)B->al.get(sizeof(BatchFieldMember) * nsims);
  B->d_blk = (int*)B->al.get(sizeof(int) * 3 * (nsims + 1));
  B->d_dyn = (unsigned char*)B->al.get(B->dyn_bytes);
  bool ok = B->d_fm && B->d_blk && B->d_dyn;
  for (int p = 0; p < 2; ++p) {
    B->d_zseg[p] = (BatchZeroSeg*)B->al.get(sizeof(BatchZeroSeg) * B->nzseg);
    B->d_zblk[p] = (int*)B->al.get(sizeof(int) * (B->nzseg + 1));
    ok = ok && B->d_zseg[p] && B->d_zblk[p];
  }
  if (B->moving) {
    B->d_ispec = B->al.get(tiled_inject_spec_bytes() * n);
    B->d_iblk = (int*)B->al.get(sizeof(int) * (n + 1));
    B->d_cnt_src = (int**)B->al.get(sizeof(int*) * 2 * n);
    B->d_cnt = (int*)B->al.get(sizeof(int) * 2 * n);
    ok = ok && B->d_ispec && B->d_iblk && B->d_cnt_src && B->d_cnt;
  }
  if (!ok) {
    set_error("pic_batch_init: out of device memory (field and window tables)");
    return bail(PIC_ENOMEM);
  }
  if (cudaMallocHost(&B->h_dyn, B->dyn_bytes) != cudaSuccess ||
      (B->moving && cudaMallocHost(&B->h_cnt, sizeof(int) * 2 * n) != cudaSuccess)) {
    set_error("pic_batch_init: pinned host allocation failed");
    return bail(PIC_ENOMEM);
  }
  memset(B->h_dyn, 0, B->dyn_bytes);
  if (B->moving) {
    std::vector<int*> src(2 * (size_t)n);
    for (int k = 0; k < n; ++k) {
      SpeciesState& sp = B->sims[B->ent[k].first]->sp[B->ent[k].second];
      src[2 * k] = sp.d_lost;
      src[2 * k + 1] = sp.d_kept;
    }
    cudaMemcpyAsync(B->d_cnt_src, src.data(), sizeof(int*) * 2 * n, cudaMemcpyHostToDevice, B->s);
    if (cudaStreamSynchronize(B->s) != cudaSuccess) return bail(cuda_check("pic_batch_init"));
  }
  cudaMemsetAsync(B->d_stat, 0, sizeof(StatusWord) * nsims, B->s);
  // every member reports into the batch's status array and runs on the
  // batch's stream from now on (the members were set up on the caller's
  // stream, which pic_init synchronised)
  for (int i = 0; i < nsims; ++i) {
    pic_sim* S = B->sims[i];
    if (S->hstat) cudaFreeHost(S->hstat);
    S->hstat = B->h_stat + i;
    S->dstat = B->d_stat + i;
    S->s = B->s;
    S->in_batch = true;
  }
  const pic_status st = batch_build(B);
  if (st != PIC_OK) return bail(st);
  *out = B;
  return PIC_OK;
}

pic_status pic_batch_step(pic_batch* B, int nsteps) {
  if (!B || nsteps < 0) {
    set_error("pic_batch_step: bad arguments");
    return PIC_EINVAL;
  }
  const int nsims = (int)B->sims.size();
  // order after the caller's earlier work; the caller's stream waits for the batch at the end
  cudaEventRecord(B->ev_in, B->user);
  cudaStreamWaitEvent(B->s, B->ev_in, 0);
  struct Join {
    pic_batch* B;
    ~Join() {
      cudaEventRecord(B->ev_out, B->s);
      cudaStreamWaitEvent(B->user, B->ev_out, 0);
    }
  } join{B};
  for (int k = 0; k < nsteps; ++k) {
    if (B->dirty || batch_antennas(B) != B->ants_built) {  // re-bin, or a pulse added through a member
      const pic_status st = batch_build(B);
      if (st != PIC_OK) return st;
    }
    const int p = B->sims[0]->sp[0].cur;
    batch_prepare(B);  // the previous step has completed: the block is free
    if (B->use_graph) {
      if (cudaGraphLaunch(B->exec[p], B->s) != cudaSuccess) return cuda_check("pic_batch_step graph launch");
    } else {
      batch_enqueue(B, p);
    }
    B->nlaunch += batch_launches_per_step(B);
    for (pic_sim* S : B->sims) {
      for (auto& sp : S->sp) sp.cur = 1 - sp.cur;
      ++S->step;
    }
    ++B->step;
    cudaMemcpyAsync(B->h_stat, B->d_stat, sizeof(StatusWord) * nsims, cudaMemcpyDeviceToHost, B->s);
    if (B->moving)
      cudaMemcpyAsync(B->h_cnt, B->d_cnt, sizeof(int) * 2 * B->ent.size(), cudaMemcpyDeviceToHost, B->s);
    if (cudaStreamSynchronize(B->s) != cudaSuccess) return cuda_check("pic_batch_step");
    batch_after_step(B);
    if (B->moving)  // particles dropped through the open x1 side and created at the front
      for (size_t k = 0; k < B->ent.size(); ++k)
        B->sims[B->ent[k].first]->sp[B->ent[k].second].n += B->h_cnt[2 * k + 1] - B->h_cnt[2 * k];
    for (int i = 0; i < nsims; ++i) {
      pic_sim* S = B->sims[i];
      const int flags = B->h_stat[i].status;
      S->sticky_flags |= flags;
      if (flags & ST_SPILL) {
        if (flags & ST_SPILL_LOST) {
          set_error("pic_batch_step: simulation " + std::to_string(i) + ": spill list overflowed");
          return PIC_EOVERFLOW;
        }
        const pic_status st = rebuild_spilled(S);
        if (st != PIC_OK) return st;
        cudaMemsetAsync(S->dstat, 0, sizeof(StatusWord), B->s);
        B->dirty = true;
      }
      if (flags & ST_TIMEOUT) {
        set_error("pic_batch_step: simulation " + std::to_string(i) + ": a bounded device wait gave up");
        return PIC_ETIMEOUT;
      }
      if (flags & (ST_NONFINITE | ST_BADCELL)) {
        set_error("pic_batch_step: simulation " + std::to_string(i) + ": non-finite particle or field value");
        return PIC_ENONFINITE;
      }
    }
  }
  return cuda_check("pic_batch_step");
}

pic_status pic_batch_sim(pic_batch* B, int i, pic_sim** out) {
  if (!B || !out || i < 0 || i >= (int)B->sims.size()) {
    set_error("pic_batch_sim: bad arguments");
    return PIC_EINVAL;
  }
  *out = B->sims[i];
  return PIC_OK;
}

pic_status pic_batch_info(const pic_batch* B, long long* steps, long long* launches, int tile[3]) {
  if (!B) {
    set_error("pic_batch_info: bad arguments");
    return PIC_EINVAL;
  }
  if (steps) *steps = B->step;
  if (launches) *launches = B->nlaunch;
  if (tile)
    for (int d = 0; d < 3; ++d) tile[d] = B->T[d];
  return PIC_OK;
}

pic_status pic_batch_destroy(pic_batch* B) {
  if (!B) return PIC_OK;
  if (B->s) cudaStreamSynchronize(B->s);
  batch_drop_graphs(B);
  for (pic_sim* S : B->sims) {
    S->hstat = nullptr;  // the batch's pinned array
    S->s = B->user;      // the allocator frees on the caller's stream
    pic_destroy(S);
  }
  B->al.release_all();
  if (B->h_stat) cudaFreeHost(B->h_stat);
  if (B->h_dyn) cudaFreeHost(B->h_dyn);
  if (B->h_cnt) cudaFreeHost(B->h_cnt);
  if (B->ev_in) cudaEventDestroy(B->ev_in);
  if (B->ev_out) cudaEventDestroy(B->ev_out);
  if (B->s) cudaStreamDestroy(B->s);
  delete B;
  return PIC_OK;
}


// ------------------------------------------------------------- autotuner

namespace {

// tile shapes of the general kernel and of the small-tile kernel, largest first
const int kShapes3[][3] = {{8, 8, 8}, {16, 8, 4}, {8, 4, 4}, {4, 4, 4}, {4, 4, 2}};
const int kShapes2[][3] = {{32, 16, 1}, {16, 16, 1}, {8, 8, 1}, {16, 8, 1}, {8, 4, 1}};
constexpr int kGeneral3 = 2, kGeneral2 = 3;  // the first ones are the general kernel's

struct TuneCand {
  int T[3];
  int ctas, sort;
};

std::vector<TuneCand> tune_candidates(int nsims, const pic_grid* grids, bool batch) {
  std::vector<TuneCand> out;
  const int ndim = grids[0].ndim;
  const int ns = 5, ngen = ndim == 3 ? kGeneral3 : kGeneral2;
  for (int k = 0; k < ns; ++k) {
    const int* c = ndim == 3 ? kShapes3[k] : kShapes2[k];
    bool fits = true;
    for (int i = 0; i < nsims; ++i)
      for (int d = 0; d < ndim; ++d) fits = fits && grids[i].nx[d] % c[d] == 0;
    if (!fits) continue;
    const bool general = k < ngen;
    if (batch && !general) continue;
    for (int ctas : {4, 2}) {
      if (!general && ctas == 2) continue;  // the small-tile kernel has one build
      for (int sort : {1, 4}) {
        if ((batch || !general) && sort != 1) continue;
        out.push_back({{c[0], c[1], ndim == 3 ? c[2] : 1}, ctas, sort});
      }
    }
  }
  return out;
}

// Device time per step of `steps` steps after `warmup` (events on `st`).
double time_steps(cudaStream_t st, int warmup, int steps, const std::function<pic_status(int)>& step) {
  if (step(warmup) != PIC_OK) return -1.0;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, st);
  const pic_status rc = step(steps);
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = -1.f;
  if (rc == PIC_OK) cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc == PIC_OK && steps > 0 ? ms / steps : -1.0;
}

pic_status tune_run(int nsims, const pic_grid* grids, const pic_species* species, int nspecies,
                    const pic_allocator* alloc, void* stream, int warmup, int steps, bool batch,
                    pic_tune_choice* best, pic_tune_choice* tried, int max_tried, int* n_tried) {
  if (nsims < 1 || !grids || !species || nspecies < 1 || !best || warmup < 0 || steps < 1) {
    set_error("autotune: bad arguments");
    return PIC_EINVAL;
  }
  for (int i = 0; i < nsims; ++i)
    if (grids[i].precision != PIC_FP32_CELLOFF || grids[i].ndim != grids[0].ndim) {
      set_error("autotune: every grid must be PIC_FP32_CELLOFF with the same ndim");
      return PIC_EINVAL;
    }
  const std::vector<TuneCand> cand = tune_candidates(nsims, grids, batch);
  if (cand.empty()) {
    set_error("autotune: no tile shape divides every grid");
    return PIC_EINVAL;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int nt = 0;
  best->ms_per_step = -1.0;
  for (const TuneCand& c : cand) {
    std::vector<pic_grid> g(grids, grids + nsims);
    for (auto& x : g) {
      for (int d = 0; d < 3; ++d) x.tile[d] = c.T[d];
      x.ctas_per_sm = c.ctas;
      x.sort_period = c.sort;
    }
    double ms = -1.0;
    if (batch) {
      pic_batch* B = nullptr;
      if (pic_batch_init(nsims, g.data(), species, nspecies, alloc, stream, &B) == PIC_OK) {
        ms = time_steps(st, warmup, steps, [&](int n) { return pic_batch_step(B, n); });
        pic_batch_destroy(B);
      }
    } else {
      pic_sim* S = nullptr;
      if (init_sim(g.data(), species, nspecies, alloc, stream, false, &S) == PIC_OK) {
        ms = time_steps(st, warmup, steps, [&](int n) { return pic_step(S, n); });
        pic_destroy(S);
      }
    }
    cudaGetLastError();
    pic_tune_choice r;
    for (int d = 0; d < 3; ++d) r.tile[d] = c.T[d];
    r.ctas_per_sm = c.ctas;
    r.sort_period = c.sort;
    r.ms_per_step = ms;
    if (tried && nt < max_tried) tried[nt] = r;
    ++nt;
    if (ms > 0.0 && (best->ms_per_step < 0.0 || ms < best->ms_per_step)) *best = r;
  }
  if (n_tried) *n_tried = nt;
  if (best->ms_per_step < 0.0) {
    set_error("autotune: no candidate ran");
    return PIC_ECUDA;
  }
  return PIC_OK;
}

}  // namespace

pic_status pic_autotune(const pic_grid* grid, const pic_species* species, int nspecies, const pic_allocator* alloc,
                        void* stream, int warmup, int steps, pic_tune_choice* best, pic_tune_choice* tried,
                        int max_tried, int* n_tried) {
  return tune_run(1, grid, species, nspecies, alloc, stream, warmup, steps, false, best, tried, max_tried, n_tried);
}

pic_status pic_batch_autotune(int nsims, const pic_grid* grids, const pic_species* species, int nspecies,
                              const pic_allocator* alloc, void* stream, int warmup, int steps, pic_tune_choice* best,
                              pic_tune_choice* tried, int max_tried, int* n_tried) {
  return tune_run(nsims, grids, species, nspecies, alloc, stream, warmup, steps, true, best, tried, max_tried,
                  n_tried);
}


// ------------------------------------------------------------- checkpoint

namespace {

const char kCkptMagic[8] = {'P', 'I', 'C', 'G', 'B', 'C', 'K', '1'};
constexpr uint32_t kCkptVersion = 3;  // 3: the antenna pulse table follows the fields
constexpr size_t kIoChunk = size_t(64) << 20;  // host staging per copy

struct CkptSpecies {
  double rqm, q;
  long long n, np_max;
  int ids, ppc[3];
  double uth[3], ufl[3];
  unsigned long long seed;
  long long created;
  int weighted, prof_n[3];  // charge weights stored; profile tables that follow the particles
  double density, den_min;
};

bool write_dev(FILE* f, const void* dev, size_t bytes, cudaStream_t s, std::vector<unsigned char>& buf) {
  for (size_t o = 0; o < bytes; o += kIoChunk) {
    const size_t m = std::min(kIoChunk, bytes - o);
    if (cudaMemcpyAsync(buf.data(), static_cast<const char*>(dev) + o, m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || fwrite(buf.data(), 1, m, f) != m)
      return false;
  }
  return true;
}

bool read_dev(FILE* f, void* dev, size_t bytes, cudaStream_t s, std::vector<unsigned char>& buf) {
  for (size_t o = 0; o < bytes; o += kIoChunk) {
    const size_t m = std::min(kIoChunk, bytes - o);
    if (fread(buf.data(), 1, m, f) != m ||
        cudaMemcpyAsync(static_cast<char*>(dev) + o, buf.data(), m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return false;
  }
  return true;
}

pic_grid effective_grid(const pic_sim* S) {
  pic_grid g = S->g;
  for (int d = 0; d < 3; ++d) g.tile[d] = S->prec == PIC_FP32_CELLOFF ? S->T[d] : 0;
  g.sort_period = S->sort_period;
  g.ctas_per_sm = S->minb;
  g.slack = S->slack;
  g.init_e_gauss_x1 = 0;
  return g;
}

// the arrays of one species' records, in file order
std::vector<std::pair<void*, size_t>> species_arrays(const pic_sim* S, const SpeciesState& sp, const Flat32& fl,
                                                     long long n) {
  std::vector<std::pair<void*, size_t>> a;
  const size_t m = (size_t)n;
  if (S->prec == PIC_FP32_CELLOFF) {
    a.push_back({fl.tile, 4 * m});
    a.push_back({fl.cell, 4 * m});
    for (int d = 0; d < 3; ++d) a.push_back({fl.o[d], 4 * m});
    for (int d = 0; d < 3; ++d) a.push_back({fl.u[d], 4 * m});
    if (sp.ids) a.push_back({fl.id, 4 * m});
    if (sp.weighted) a.push_back({fl.w, 4 * m});
  } else {
    for (int d = 0; d < S->ndim; ++d) a.push_back({sp.plain.x[d], 8 * m});
    for (int d = 0; d < 3; ++d) a.push_back({sp.plain.u[d], 8 * m});
    if (sp.ids) a.push_back({sp.plain.id, 4 * m});
    if (sp.weighted) a.push_back({sp.plain.w, 8 * m});
  }
  size_t tab = 0;  // the profile tables (x then f per direction)
  for (int d = 0; d < 3; ++d) tab += 2 * (size_t)sp.prof.n[d];
  if (sp.has_prof && tab) a.push_back({sp.prof_mem, 8 * tab});
  return a;
}

}  // namespace

pic_status pic_checkpoint_save(pic_sim* S, const char* path) {
  if (!S || !path) {
    set_error("pic_checkpoint_save: bad arguments");
    return PIC_EINVAL;
  }
  if (cudaStreamSynchronize(S->s) != cudaSuccess) return cuda_check("pic_checkpoint_save");
  FILE* f = fopen(path, "wb");
  if (!f) {
    set_error(std::string("pic_checkpoint_save: cannot open ") + path);
    return PIC_EINVAL;
  }
  std::vector<unsigned char> buf(kIoChunk);
  bool ok = true;
  auto put = [&](const void* p, size_t n) { ok = ok && fwrite(p, 1, n, f) == n; };
  const uint32_t hdr[4] = {kCkptVersion, (uint32_t)sizeof(pic_grid), (uint32_t)sizeof(CkptSpecies), 0};
  put(kCkptMagic, 8);
  put(hdr, sizeof(hdr));
  const pic_grid g = effective_grid(S);
  put(&g, sizeof(g));
  const long long step = S->step, shifts = S->shifts;
  const int nsp = (int)S->sp.size(), pad = 0;
  put(&step, 8);
  put(&shifts, 8);
  put(&nsp, 4);
  put(&pad, 4);
  pic_status st = PIC_OK;
  for (auto& sp : S->sp) {
    Flat32 fl{};
    long long n = sp.n;
    bool alloc = false;
    if (S->prec == PIC_FP32_CELLOFF && (st = flatten(S, sp, fl, n, false, 0, alloc)) != PIC_OK) break;
    CkptSpecies h{};
    h.rqm = sp.rqm;
    h.q = sp.q;
    h.n = n;
    h.np_max = sp.np_max;
    h.ids = sp.ids ? 1 : 0;
    for (int d = 0; d < 3; ++d) {
      h.ppc[d] = sp.ppc[d];
      h.uth[d] = sp.uth[d];
      h.ufl[d] = sp.ufl[d];
    }
    h.seed = sp.seed;
    h.created = sp.created;
    h.weighted = sp.weighted ? 1 : 0;
    for (int d = 0; d < 3; ++d) h.prof_n[d] = sp.has_prof ? sp.prof.n[d] : 0;
    h.density = sp.prof.density;
    h.den_min = sp.prof.den_min;
    put(&h, sizeof(h));
    for (auto& a : species_arrays(S, sp, fl, n)) ok = ok && write_dev(f, a.first, a.second, S->s, buf);
    if (alloc) free_flat(S, fl);
    if (!ok) break;
  }
  const size_t eb = elem_bytes(S);
  for (int c = 0; c < 6 && ok && st == PIC_OK; ++c)
    ok = write_dev(f, static_cast<char*>(S->fld) + (size_t)c * eb * (size_t)S->L.plane, eb * (size_t)S->L.plane,
                   S->s, buf);
  // pulses entering through the lower x1 boundary (their records are in the
  // lab frame: start time, focal plane), so a restored moving-window run
  // keeps driving them
  const int nants = S->n_ants;
  const uint32_t rb = (uint32_t)antenna_bytes();
  put(&nants, 4);
  put(&rb, 4);
  if (nants > 0) put(S->h_ants.data(), (size_t)rb * (size_t)nants);
  ok = (fclose(f) == 0) && ok;
  if (st != PIC_OK) return st;
  if (!ok) {
    set_error(std::string("pic_checkpoint_save: write failed: ") + path);
    return PIC_EINVAL;
  }
  return cuda_check("pic_checkpoint_save");
}

pic_status pic_checkpoint_load(const char* path, const pic_allocator* alloc, void* stream, pic_sim** out) {
  if (!path || !out) {
    set_error("pic_checkpoint_load: bad arguments");
    return PIC_EINVAL;
  }
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) {
    set_error(std::string("pic_checkpoint_load: cannot open ") + path);
    return PIC_EINVAL;
  }
  struct Closer {
    FILE* f;
    ~Closer() { fclose(f); }
  } closer{f};
  char magic[8];
  uint32_t hdr[4];
  pic_grid g{};
  long long step = 0, shifts = 0;
  int nsp = 0, pad = 0;
  if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kCkptMagic, 8) != 0 || fread(hdr, 1, sizeof(hdr), f) != sizeof(hdr) ||
      hdr[0] != kCkptVersion || hdr[1] != sizeof(pic_grid) || hdr[2] != sizeof(CkptSpecies) ||
      fread(&g, 1, sizeof(g), f) != sizeof(g) || fread(&step, 1, 8, f) != 8 || fread(&shifts, 1, 8, f) != 8 ||
      fread(&nsp, 1, 4, f) != 4 ||
      fread(&pad, 1, 4, f) != 4 || nsp < 0 || nsp > 64) {
    set_error(std::string("pic_checkpoint_load: not a checkpoint of this library version: ") + path);
    return PIC_EINVAL;
  }
  std::vector<unsigned char> buf(kIoChunk);
  RestoreFn restore = [&](pic_sim* S, int, SpeciesState& sp) -> pic_status {
    CkptSpecies h{};
    if (fread(&h, 1, sizeof(h), f) != sizeof(h) || h.n < 0) {
      set_error("pic_checkpoint_load: truncated species record");
      return PIC_EINVAL;
    }
    sp.rqm = h.rqm;
    sp.q = h.q;
    sp.n = h.n;
    sp.np_max = h.np_max;
    sp.ids = h.ids != 0;
    for (int d = 0; d < 3; ++d) {
      sp.ppc[d] = h.ppc[d];
      sp.uth[d] = h.uth[d];
      sp.ufl[d] = h.ufl[d];
    }
    sp.seed = h.seed;
    sp.created = h.created;
    sp.weighted = h.weighted != 0;
    size_t tab = 0;
    for (int d = 0; d < 3; ++d) tab += 2 * (size_t)std::max(h.prof_n[d], 0);
    sp.has_prof = tab > 0;
    sp.prof = ProfileDev{};
    if (sp.has_prof) {
      sp.prof_mem = (double*)S->al.get(8 * tab);
      if (!sp.prof_mem) {
        set_error("out of device memory (density profile)");
        return PIC_ENOMEM;
      }
      size_t o = 0;
      for (int d = 0; d < 3; ++d) {
        sp.prof.n[d] = h.prof_n[d];
        if (h.prof_n[d] <= 0) continue;
        sp.prof.x[d] = sp.prof_mem + o;
        sp.prof.f[d] = sp.prof_mem + o + h.prof_n[d];
        o += 2 * (size_t)h.prof_n[d];
      }
      sp.prof.density = h.density;
      sp.prof.den_min = h.den_min;
    }
    const size_t m = (size_t)std::max<long long>(h.n, 1);
    Flat32 fl{};
    if (S->prec == PIC_FP32_CELLOFF) {
      bool okf = true;
      fl = alloc_flat(S, h.n, sp.ids, okf, sp.weighted);
      if (!okf) {
        free_flat(S, fl);
        set_error("out of device memory (checkpoint particles)");
        return PIC_ENOMEM;
      }
    } else {
      for (int d = 0; d < 3; ++d) {
        sp.plain.x[d] = d < S->ndim ? (double*)S->al.get(8 * m) : nullptr;
        sp.plain.u[d] = (double*)S->al.get(8 * m);
        if ((d < S->ndim && !sp.plain.x[d]) || !sp.plain.u[d]) {
          set_error("out of device memory (checkpoint particles)");
          return PIC_ENOMEM;
        }
      }
      sp.plain.id = sp.ids ? (int*)S->al.get(4 * m) : nullptr;
      sp.plain.w = sp.weighted ? (double*)S->al.get(8 * m) : nullptr;
      if (sp.weighted && !sp.plain.w) {
        set_error("out of device memory (checkpoint particles)");
        return PIC_ENOMEM;
      }
      sp.plain.n = h.n;
    }
    for (auto& a : species_arrays(S, sp, fl, h.n))
      if (!read_dev(f, a.first, a.second, S->s, buf)) {
        if (S->prec == PIC_FP32_CELLOFF) free_flat(S, fl);
        set_error("pic_checkpoint_load: truncated particle data");
        return PIC_EINVAL;
      }
    if (S->prec == PIC_FP32_CELLOFF) {
      const pic_status st = bin_flat(S, sp, fl, h.n);
      free_flat(S, fl);
      return st;
    }
    return PIC_OK;
  };
  pic_sim* S = nullptr;
  pic_status st = init_sim(&g, nullptr, nsp, alloc, stream, false, &S, &restore);
  if (st != PIC_OK) return st;
  const size_t eb = elem_bytes(S);
  for (int c = 0; c < 6; ++c)
    if (!read_dev(f, static_cast<char*>(S->fld) + (size_t)c * eb * (size_t)S->L.plane, eb * (size_t)S->L.plane, S->s,
                  buf)) {
      pic_destroy(S);
      set_error("pic_checkpoint_load: truncated field data");
      return PIC_EINVAL;
    }
  S->step = step;
  S->shifts = shifts;
  int nants = 0;
  uint32_t rb = 0;
  if (fread(&nants, 1, 4, f) != 4 || fread(&rb, 1, 4, f) != 4 || nants < 0 || nants > (1 << 20) ||
      (nants > 0 && rb != (uint32_t)antenna_bytes())) {
    pic_destroy(S);
    set_error("pic_checkpoint_load: truncated or foreign antenna table");
    return PIC_EINVAL;
  }
  if (nants > 0) {
    S->h_ants.resize((size_t)rb * (size_t)nants);
    S->d_ants = S->al.get(S->h_ants.size());
    S->d_inc = (float*)S->al.get(2 * sizeof(float) * (size_t)S->L.ny * (size_t)S->L.nz);
    if (fread(S->h_ants.data(), 1, S->h_ants.size(), f) != S->h_ants.size() || !S->d_ants || !S->d_inc) {
      pic_destroy(S);
      set_error("pic_checkpoint_load: antenna table truncated or out of device memory");
      return PIC_EINVAL;
    }
    cudaMemcpyAsync(S->d_ants, S->h_ants.data(), S->h_ants.size(), cudaMemcpyHostToDevice, S->s);
    if (cudaStreamSynchronize(S->s) != cudaSuccess) {
      pic_destroy(S);
      return cuda_check("pic_checkpoint_load");
    }
    S->n_ants = nants;
  }
  *out = S;
  return cuda_check("pic_checkpoint_load");
}

pic_status pic_laser_add(pic_sim* S, const pic_laser* L) {
  if (!S || !L || !(L->rkkp > 0.0) || !(L->w0 > 0.0) || L->rise < 0.0 || L->fall < 0.0 || L->length < 0.0 ||
      (L->wavetype != 0 && L->wavetype != 1 && L->wavetype != 2)) {
    set_error("pic_laser_add: bad arguments");
    return PIC_EINVAL;
  }
  if (S->cyl) {
    set_error("pic_laser_add: no laser in the r-z mode");
    return PIC_EUNSUPPORTED;
  }
  if (L->antenna && (!S->moving || S->prec != PIC_FP32_CELLOFF || L->wavetype == 2)) {
    set_error("pic_laser_add: an antenna needs the open x1 boundary of a move_window simulation (FP32) and "
              "wavetype 1");
    return PIC_EUNSUPPORTED;
  }
  const pic_grid& g = S->g;
  const double nxr[3] = {(double)S->L.nx, (double)S->L.ny, (double)S->L.nz};
  const int a = L->wavetype == 2 ? 1 : 0, tr = 1 - a;  // propagation and in-plane transverse axes
  const double pol = L->pol * 3.141592653589793 / 180.0;
  const double upper = g.xmin[a] + nxr[a] * g.dx[a];  // the side the pulse moves towards
  double p[21];
  p[0] = L->vosc;
  p[1] = L->rkkp;
  p[2] = L->w0;
  p[3] = L->rise;
  p[4] = L->length;
  p[5] = L->fall;
  p[6] = upper - L->start;  // pulse front
  p[7] = g.xmin[tr] + 0.5 * nxr[tr] * g.dx[tr] + L->offset[0];
  p[8] = S->ndim == 3 ? g.xmin[2] + 0.5 * nxr[2] * g.dx[2] + L->offset[1] : 0.0;
  p[9] = cos(pol);
  p[10] = sin(pol);
  p[11] = L->phase;
  for (int d = 0; d < 3; ++d) {
    p[12 + d] = g.xmin[d];
    p[15 + d] = d < S->ndim ? g.dx[d] : 1.0;
  }
  p[18] = a;
  p[19] = L->focus_on ? 1.0 : 0.0;
  p[20] = upper - L->focus;  // focal plane
  if (L->antenna) {  // driven at the lower x1 boundary from the next step on
    p[6] = L->start;                   // time at which the front crosses the boundary
    p[20] = g.xmin[0] + L->focus;      // focal plane, into the box from that boundary
    const size_t rb = antenna_bytes();
    S->h_ants.resize(rb * (size_t)(S->n_ants + 1));
    antenna_store(p, S->h_ants.data() + rb * (size_t)S->n_ants);
    void* d = S->al.get(S->h_ants.size());
    if (!S->d_inc) S->d_inc = (float*)S->al.get(2 * sizeof(float) * (size_t)S->L.ny * (size_t)S->L.nz);
    if (!d || !S->d_inc) {
      S->al.put(d);
      set_error("out of device memory (antenna)");
      return PIC_ENOMEM;
    }
    cudaMemcpyAsync(d, S->h_ants.data(), S->h_ants.size(), cudaMemcpyHostToDevice, S->s);
    if (cudaStreamSynchronize(S->s) != cudaSuccess) return cuda_check("pic_laser_add");
    S->al.put(S->d_ants);
    S->d_ants = d;
    S->n_ants += 1;
    return PIC_OK;
  }
  if (S->prec == PIC_FP64_PLAIN) {
    double* f[6];
    for (int c = 0; c < 6; ++c) f[c] = fld_ptr<double>(S, c);
    laser_add<double>(S->L, f, p, S->s);
    fill_guards<double>(S->L, f, 6, S->s);
  } else {
    float* f[6];
    for (int c = 0; c < 6; ++c) f[c] = fld_ptr<float>(S, c);
    laser_add<float>(S->L, f, p, S->s);
    fill_guards<float>(S->L, f, 6, S->s);
  }
  if (cudaStreamSynchronize(S->s) != cudaSuccess) return cuda_check("pic_laser_add");
  return cuda_check("pic_laser_add");
}

pic_status pic_info(const pic_sim* S, pic_grid* grid, int* nspecies, long long* step) {
  if (!S) {
    set_error("pic_info: bad arguments");
    return PIC_EINVAL;
  }
  if (grid) *grid = effective_grid(S);
  if (nspecies) *nspecies = (int)S->sp.size();
  if (step) *step = S->step;
  return PIC_OK;
}

}  // extern "C"
