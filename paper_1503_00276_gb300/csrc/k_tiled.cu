// k_tiled.cu -- FP32 cell-offset form of the particle step on tiles of cells.
//
// Store: per tile a region of slots (structure of arrays).  At the start of a
// step a region holds, at its front, the tile's stayers in runs sorted by cell
// and, at its back, the particles that entered the tile during the last step
// (their cell already relative to this tile).
//
// k_tile_push (persistent CTAs, one tile at a time) advances every particle of
// its tile:
//   * one TMA copy stages the E/B stencil of the tile + halo in shared memory;
//   * gather (eq. 2d-field-weighting-e3, 3D extension), Boris push
//     (eq. momentum-update), position update (eq. 2d-position-update) and the
//     TRISTAN / Villasenor-Buneman deposit run in FP32 on int cell + FP32 offset;
//   * the tile's particles are read in chunks of 512 as one sequence, the
//     stayers continued by the arrivals;
//   * the current goes to a shared-memory tile: each thread adds the first
//     in-cell pieces of its two particles in registers, each warp then sums
//     its lanes over runs of equal cells, and one lane per cell flushes;
//     pieces after a face crossing (a few % of particles) are queued in
//     shared memory and deposited by full warps;
//   * each chunk of 512 advanced particles is counting-sorted by new cell in
//     shared memory (keys only -- the particles stay in registers) and written
//     to the front of the tile's region on the other store side; particles that
//     left the tile are appended, with one global atomic each (one per warp
//     and destination when a window shifts), to the back of their new tile's
//     region there;
//   * one TMA reduce-add flushes the shared current tile (with halo) into HBM.
// The store is therefore re-binned by tile and re-sorted by cell every step
// without a separate pass over HBM.
#include <cstring>

#include "tile_dev.cuh"

namespace picgb {

namespace {

// Counting sort of one chunk of advanced particles (still in registers) by key
// and write-out: stayers to the front of this tile's output region in cell
// order, leavers to the back of their new tile's output region.
template <int NDIM, int TX, int TY, int TZ, int PPT = kPPT>
__device__ inline void sort_and_store(const TileArgs& A, int t, int tix, int tiy, int tiz, long long base, int room,
                                      P (&pp)[PPT], int (&key)[PPT], int nvalid, int& ws, int* hist, int* misc,
                                      const Nbr* nb = nullptr, int* stay_ctr = nullptr) {
  using G = Geo<NDIM, TX, TY, TZ>;
  const int tid = threadIdx.x;
  __syncthreads();  // previous chunk's ranks read
  for (int k = tid; k < G::NK; k += kThreads) hist[k] = 0;
  __syncthreads();
  {
    int hk = -1, hc = 0;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      if (r < nvalid && key[r] < G::NK) {
        if (key[r] != hk) {
          if (hk >= 0) atomicAdd(&hist[hk], hc);
          hk = key[r];
          hc = 0;
        }
        ++hc;
      }
    }
    if (hk >= 0) atomicAdd(&hist[hk], hc);
  }
  __syncthreads();
  // every push of the chunk is done: snapshot of the crossing-queue count, read
  // by every thread after the caller's next barrier
  if (tid == 0) misc[5] = misc[1];
  // exclusive scan of hist in place
  {
    constexpr int PER = (G::NK + kThreads - 1) / kThreads;
    int v[PER];
    int run = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int k = tid * PER + r;
      v[r] = k < G::NK ? hist[k] : 0;
      run += v[r];
    }
    const int lane = tid & 31, warp = tid >> 5;
    int x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) misc[8 + warp] = x;
    __syncthreads();
    if (tid == 0) {
      int s = 0;
      for (int w = 0; w < kThreads / 32; ++w) {
        const int tmp = misc[8 + w];
        misc[8 + w] = s;
        s += tmp;
      }
      misc[7] = s;  // chunk total
    }
    __syncthreads();
    int pre = misc[8 + warp] + x - run;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int k = tid * PER + r;
      if (k < G::NK) hist[k] = pre;
      if (k == G::NC) {
        misc[6] = pre;  // stayers in this chunk (hist[NC] moves during ranking)
        // a tile split over several blocks reserves its chunk's output slots
        if (stay_ctr) misc[4] = atomicAdd(stay_ctr, pre);
      }
      pre += v[r];
    }
  }
  __syncthreads();
  const int nst = misc[6];
  const int wsb = stay_ctr ? misc[4] : ws;
  // rank within key (a run of equal keys takes one atomic) and write; every
  // index into pp/key is a compile-time constant, so the chunk stays in
  // registers
  {
    int p0 = 0, rs = 0;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      if (r < nvalid) {
        const int k = key[r];
        if (r == 0 || key[r > 0 ? r - 1 : 0] != k) {  // first of a run of equal keys
          int n = 1;
#pragma unroll
          for (int m = r + 1; m < PPT; ++m)
            if (m < nvalid && n == m - r && key[m] == k) ++n;
          if (k < G::NK) p0 = atomicAdd(&hist[k], n);
          rs = r;
        }
        if (k < G::NC) {
          const int pos = wsb + p0 + (r - rs);
          if (pos < room)
            store_particle<NDIM>(A.out.p, base + pos, pp[r]);
          else
            spill_put(A, t, pp[r]);
        } else if (k < G::NK) {
          store_leaver<NDIM>(A, tix, tiy, tiz, pp[r], nb);
        }
      }
    }
  }
  ws += nst;
}

// The counting sort of the general kernel with three block barriers per chunk
// (sort_and_store takes six).  Only stayers are ranked (leavers go to their new
// tile through store_leaver), so the histogram has NC bins.  It is kept in two
// buffers used by alternate chunks, so one is cleared while the other is in
// use, and packed two 16-bit counts per word (a chunk holds at most kChunk <
// 65536 particles).  Every thread adds up the earlier warps' totals itself
// instead of one thread scanning them.  Returns the crossing-queue count
// snapshot taken when every push of the chunk was done (misc[5]).
template <int NDIM, int TX, int TY, int TZ>
__device__ inline int sort_and_store_lean(const TileArgs& A, int t, int tix, int tiy, int tiz, long long base,
                                          int room, P (&pp)[kPPT], int (&key)[kPPT], int nvalid, int& ws,
                                          uint32_t* h2, uint32_t* h2next, int* misc, const Nbr* nb,
                                          int* stay_ctr) {
  using G = Geo<NDIM, TX, TY, TZ>;
  static_assert(kChunk < 65536, "16-bit histogram counts");
  constexpr int PER = ((G::NC + kThreads - 1) / kThreads + 1) & ~1;  // bins per thread, even
  static_assert(PER * kThreads >= G::NC, "every bin owned by a thread");
  constexpr int NW = G::NC / 2;  // words per histogram buffer
  static_assert(G::NC % 2 == 0 && G::NC * 4 <= G::QOFF - G::HOFF, "two packed buffers in the histogram space");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    int hk = -1, hc = 0;
#pragma unroll
    for (int r = 0; r < kPPT; ++r) {
      if (r < nvalid && key[r] < G::NC) {
        if (key[r] != hk) {
          if (hk >= 0) atomicAdd(&h2[hk >> 1], (uint32_t)hc << (16 * (hk & 1)));
          hk = key[r];
          hc = 0;
        }
        ++hc;
      }
    }
    if (hk >= 0) atomicAdd(&h2[hk >> 1], (uint32_t)hc << (16 * (hk & 1)));
  }
  __syncthreads();  // every push and count of the chunk is done
  if (tid == 0) misc[5] = misc[1];
  uint32_t v[PER];
  int run = 0;
#pragma unroll
  for (int r = 0; r < PER; r += 2) {
    const int k = tid * PER + r;
    const uint32_t w = k < G::NC ? h2[k >> 1] : 0u;
    v[r] = w & 0xFFFFu;
    v[r + 1] = w >> 16;
    run += (int)(v[r] + v[r + 1]);
  }
  int x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) misc[8 + warp] = x;
  // the other buffer's last use (the previous chunk's ranking) ended before the barrier above
  for (int k = tid; k < NW; k += kThreads) h2next[k] = 0u;
  __syncthreads();
  int pre = x - run, nst = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) {
    const int c = misc[8 + w];
    pre += w < warp ? c : 0;
    nst += c;  // stayers of the chunk
  }
#pragma unroll
  for (int r = 0; r < PER; r += 2) {
    const int k = tid * PER + r;
    if (k < G::NC) {
      const uint32_t lo = (uint32_t)pre;
      pre += (int)v[r];
      h2[k >> 1] = lo | ((uint32_t)pre << 16);
      pre += (int)v[r + 1];
    }
  }
  // a tile split over several blocks reserves its chunk's output slots
  if (stay_ctr && tid == 0) misc[4] = atomicAdd(stay_ctr, nst);
  const int nq = misc[5];
  __syncthreads();
  const int wsb = stay_ctr ? misc[4] : ws;
  const bool agg = A.shift_ptr != nullptr || A.shift_x != 0;  // a window shift: many leavers
  {
    int p0 = 0, rs = 0;
#pragma unroll
    for (int r = 0; r < kPPT; ++r) {
      if (r < nvalid) {
        const int k = key[r];
        if (k < G::NC && (r == 0 || key[r > 0 ? r - 1 : 0] != k)) {  // first of a run of equal keys
          int n = 1;
#pragma unroll
          for (int m = r + 1; m < kPPT; ++m)
            if (m < nvalid && n == m - r && key[m] == k) ++n;
          const int sh = 16 * (k & 1);
          p0 = (int)((atomicAdd(&h2[k >> 1], (uint32_t)n << sh) >> sh) & 0xFFFFu);
          rs = r;
        }
        if (k < G::NC) {
          const int pos = wsb + p0 + (r - rs);
          if (pos < room)
            store_particle<NDIM>(A.out.p, base + pos, pp[r]);
          else
            spill_put(A, t, pp[r]);
        } else if (k < G::NK && !agg) {
          store_leaver<NDIM>(A, tix, tiy, tiz, pp[r], nb);
        }
      }
    }
  }
  // leavers: the lanes bound for one neighbour tile take their arrival slots
  // with one atomic (a window shift sends a tile's whole first cell column
  // to the tile behind)
  if (agg) {
#pragma unroll
    for (int r = 0; r < kPPT; ++r) {
      const bool lv = r < nvalid && key[r] == G::NC;
      const int dir = lv ? (int)(pp[r].cell >> 24) : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, dir);
      if (lv) {
        const int leader = __ffs(peers) - 1;
        const int cnt = __popc(peers), rank = __popc(peers & ((1u << lane) - 1u));
        const Nbr& nbr = nb[dir];
        if (nbr.tile < 0) {  // left through an open x1 boundary
          if (lane == leader) atomicAdd(A.lost, cnt);
        } else {
          int slot0 = 0;
          if (lane == leader) slot0 = atomicAdd(&A.out.inc[nbr.tile], cnt);
          slot0 = __shfl_sync(peers, slot0, leader);
          const int slot = slot0 + rank;
          P q2 = pp[r];
          q2.cell = (q2.cell & 0x00FFFFFFu) | ((uint32_t)DIR_STAY << 24);
          if (slot < nbr.res)
            store_particle<NDIM>(A.out.p, nbr.base + nbr.cap - 1 - slot, q2);
          else
            spill_put(A, nbr.tile, q2);
        }
      }
    }
  }
  ws += nst;
  return nq;
}

// The step between two re-sorts: the chunk's stayers go to the front of the
// tile's output region in the order they were read (one block scan instead of
// the counting sort), leavers to their new tile as in sort_and_store.
template <int NDIM, int TX, int TY, int TZ>
__device__ inline void compact_and_store(const TileArgs& A, int t, int tix, int tiy, int tiz, long long base, int room,
                                         P (&pp)[kPPT], int (&key)[kPPT], int nvalid, int& ws, int* misc,
                                         const Nbr* nb) {
  using G = Geo<NDIM, TX, TY, TZ>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int cnt = 0;
#pragma unroll
  for (int r = 0; r < kPPT; ++r) cnt += r < nvalid && key[r] < G::NC;
  int x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) misc[8 + warp] = x;
  __syncthreads();
  // every push of the chunk is done: snapshot of the crossing-queue count,
  // read by every thread after the caller's next barrier
  if (tid == 0) misc[5] = misc[1];
  int pre = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) {
    const int v = misc[8 + w];
    pre += w < warp ? v : 0;
    total += v;
  }
  int pos = ws + pre + x - cnt;
#pragma unroll
  for (int r = 0; r < kPPT; ++r) {
    if (r >= nvalid || key[r] >= G::NK) continue;  // empty slot or dropped particle
    const P& q = pp[r];
    if (key[r] < G::NC) {
      if (pos < room)
        store_particle<NDIM>(A.out.p, base + pos, q);
      else
        spill_put(A, t, q);
      ++pos;
    } else {
      store_leaver<NDIM>(A, tix, tiy, tiz, q, nb);
    }
  }
  ws += total;
}

// Everything the sorting kernel does for tile t of one simulation (A): stage
// the fields, advance, sort and store every particle of the tile, flush the
// current.  Called by all threads of the block; false if a bounded wait gave
// up (the block then stops).
// IDW = false: the store carries neither ids nor charge weights (every
// particle's id is 0 and weight 1 at compile time, which frees registers)
template <int NDIM, int TX, int TY, int TZ, bool SORT, bool CYL = false, bool IDW = true>
__device__ inline bool sort_tile(const TileArgs& A, const CUtensorMap* fmap, const CUtensorMap* jmap, int t,
                                 int slice, unsigned char* smem, uint32_t& phase) {
  using G = Geo<NDIM, TX, TY, TZ>;
  float* F = reinterpret_cast<float*>(smem + G::FOFF);
  float* J = reinterpret_cast<float*>(smem + G::JOFF);
  int* hist = reinterpret_cast<int*>(smem + G::HOFF);
  float* Q = reinterpret_cast<float*>(smem + G::QOFF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + G::MOFF);
  // misc: [0] tile [1] queue count [2] table entry or slice [4] stayer base of
  // the chunk (sliced tile) [5] queue-count snapshot [6] stayers of the chunk
  // [7] chunk total [8..15] scan
  int* misc = reinterpret_cast<int*>(smem + G::MOFF + 16);
  Nbr* nb = reinterpret_cast<Nbr*>(smem + G::NOFF);
  const int tid = threadIdx.x;
  const int tix = t % A.nt[0], tiy = (t / A.nt[0]) % A.nt[1], tiz = t / (A.nt[0] * A.nt[1]);
  const int x0 = tix * TX, y0 = tiy * TY, z0 = tiz * TZ;
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, (uint32_t)G::FBYTES);
    if (NDIM == 3)
      tma_load_4d(F, fmap, bar, x0, y0, z0, 0);
    else
      tma_load_3d(F, fmap, bar, x0, y0, 0);
  }
  for (int k = tid; k < 3 * G::JPL; k += kThreads) J[k] = 0.f;
  if (SORT)  // both buffers of sort_and_store_lean's packed histogram
    for (int k = tid; k < G::NC; k += kThreads) hist[k] = 0;
  load_neighbour(A, tix, tiy, tiz, nb);
  const long long base = A.base[t];
  const int cap = A.cap[t];
  const int res = A.res[t];
  const int room = cap - res;  // stayer slots of the output region
  int nstay = A.in.stay[t];
  nstay = nstay < room ? nstay : room;  // a sliced tile's count includes what it spilled
  int ninc = A.in.inc[t];
  ninc = ninc < res ? ninc : res;
  // a heavy tile is split into slices of kSliceChunks chunks (separate work
  // items); their stayers reserve output slots with an atomic per chunk
  const int nslices = A.nslice ? A.nslice[t] : 1;
  int* stay_ctr = (SORT && nslices > 1) ? A.out.stay + t : nullptr;
  // A dense tile (a beam: many lanes of a warp on one cell) takes one particle
  // per thread and pass, so that a pass queues at most kThreads crossing paths
  // and the queue never overflows; its current is summed across each warp
  // before the shared-memory adds.
  const bool dense = nstay + ninc > kDensePerCell * G::NC;
  const int per = dense ? 1 : kPPT;  // particles per thread and chunk
  const int csz = kThreads * per;
  const bool ok = mbar_wait_bounded(bar, phase, kWaitLimit);
  if (__syncthreads_or(!ok)) {  // every thread takes the same decision
    if (tid == 0) atomicOr(A.status, ST_TIMEOUT);
    mbar_wait_bounded(bar, phase, kWaitLimit);
    return false;
  }
  phase ^= 1u;

  int ws = 0;
  int nch = 0;  // chunks done: picks the histogram buffer
  // chunks over the tile's particles read as one sequence, the stayers (front,
  // 16-byte aligned) followed by the arrivals (back), so that the arrivals
  // fill the last stayer chunk instead of taking a pass of their own
  const int ntot = nstay + ninc;
  const int nchunk = (ntot + csz - 1) / csz;
  const int spc = kSliceChunks * (kPPT / per);  // chunks per slice (a slice is kSliceChunks * kChunk particles)
  const int ch_end = nslices > 1 ? min(nchunk, (slice + 1) * spc) : nchunk;
  for (int ch = nslices > 1 ? slice * spc : 0; ch < ch_end; ++ch) {
    P pp[kPPT];
    int key[kPPT];
    const int first = ch * csz + tid * per;
    int nvalid = ntot - first;
    nvalid = nvalid < 0 ? 0 : (nvalid > per ? per : nvalid);
    if (!dense && first + kPPT <= nstay) {  // a whole pair of stayers: vector loads
      const long long s = base + first;
      uint32_t cl[kPPT];
      float q0[kPPT], q1[kPPT], q2[kPPT] = {}, v0[kPPT], v1[kPPT], v2[kPPT];
      int idv[kPPT] = {};
      float wv[kPPT];
#pragma unroll
      for (int r = 0; r < kPPT; ++r) wv[r] = 1.f;
      load_vec(A.in.p.cell + s, cl);
      load_vec(A.in.p.o[0] + s, q0);
      load_vec(A.in.p.o[1] + s, q1);
      if (NDIM == 3) load_vec(A.in.p.o[2] + s, q2);
      load_vec(A.in.p.u[0] + s, v0);
      load_vec(A.in.p.u[1] + s, v1);
      load_vec(A.in.p.u[2] + s, v2);
      if (IDW && A.in.p.id) load_vec(A.in.p.id + s, idv);
      if (IDW && A.in.p.w) load_vec(A.in.p.w + s, wv);
#pragma unroll
      for (int r = 0; r < kPPT; ++r) pp[r] = P{cl[r], q0[r], q1[r], q2[r], v0[r], v1[r], v2[r], idv[r], wv[r]};
    } else {  // one at a time: the last stayers, the arrivals, a dense tile
#pragma unroll
      for (int r = 0; r < kPPT; ++r) {
        if (r < nvalid) {
          const int v = first + r;
          const long long s = v < nstay ? base + v : base + cap - ninc + (v - nstay);
          pp[r] = P{A.in.p.cell[s], A.in.p.o[0][s], A.in.p.o[1][s], NDIM == 3 ? A.in.p.o[2][s] : 0.f,
                    A.in.p.u[0][s], A.in.p.u[1][s], A.in.p.u[2][s], IDW && A.in.p.id ? A.in.p.id[s] : 0,
                    IDW && A.in.p.w ? A.in.p.w[s] : 1.f};
        }
      }
    }
    {
      Acc acc;
#pragma unroll
      for (int k = 0; k < 12; ++k) acc.w[k] = 0.f;
      acc.cell = -1;
#pragma unroll
      for (int r = 0; r < kPPT; ++r)
        key[r] = r < nvalid ? push_one<NDIM, TX, TY, TZ, kQCap, CYL>(F, J, A, pp[r], acc, Q, misc + 1, tiy * TY)
                            : Geo<NDIM, TX, TY, TZ>::NK;
      if (dense) {
        acc_flush_warp<NDIM, TX, TY, TZ>(J, acc);
      } else {
        acc_merge_runs<NDIM>(acc);
        acc_flush<NDIM, TX, TY, TZ>(J, acc);
      }
    }
    int nq;  // the same value in every thread
    if constexpr (SORT) {
      uint32_t* h2 = reinterpret_cast<uint32_t*>(hist) + (nch & 1) * (G::NC / 2);
      uint32_t* h2next = reinterpret_cast<uint32_t*>(hist) + ((nch + 1) & 1) * (G::NC / 2);
      nq = sort_and_store_lean<NDIM, TX, TY, TZ>(A, t, tix, tiy, tiz, base, room, pp, key, nvalid, ws, h2, h2next,
                                                 misc, nb, stay_ctr);
    } else {
      compact_and_store<NDIM, TX, TY, TZ>(A, t, tix, tiy, tiz, base, room, pp, key, nvalid, ws, misc, nb);
      __syncthreads();
      nq = misc[5];
    }
    ++nch;
    // drain when another chunk's typical crossings might not fit (fuller
    // drains keep more of the block busy; an overflow falls back to direct
    // deposits, so this is a cost question only)
    if (nq > (dense ? kQCap - kThreads : kQCap - 64)) {  // entries [0, nq) are complete since the snapshot
      if (dense)
        drain_queue<NDIM, TX, TY, TZ, true>(J, A, Q, nq < kQCap ? nq : kQCap);
      else
        drain_queue<NDIM, TX, TY, TZ>(J, A, Q, nq < kQCap ? nq : kQCap);
      __syncthreads();
      if (tid == 0) misc[1] = 0;
      __syncthreads();  // the reset lands before the next chunk queues anything
    }
  }
  __syncthreads();
  {
    const int nq = misc[1];
    if (nq > 0 && dense)
      drain_queue<NDIM, TX, TY, TZ, true>(J, A, Q, nq < kQCap ? nq : kQCap);
    else if (nq > 0)
      drain_queue<NDIM, TX, TY, TZ>(J, A, Q, nq < kQCap ? nq : kQCap);
  }
  if (tid == 0 && !stay_ctr) A.out.stay[t] = ws < room ? ws : room;
  // flush the current tile: every thread orders its shared atomics before the
  // async proxy reads them; one thread issues the TMA reduce-add and waits
  // until the TMA has read the tile before the next tile reuses it
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0) {
    if (NDIM == 3)
      tma_reduce_add_4d(jmap, J, x0, y0, z0, 0);
    else
      tma_reduce_add_3d(jmap, J, x0, y0, 0);
    tma_commit();
    tma_wait_read0();
  }
  return true;
}

template <int NDIM, int TX, int TY, int TZ, int MINB, bool SORT = true, bool CYL = false, bool IDW = true>
__global__ void __launch_bounds__(kThreads, MINB)
    k_tile_push(const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap jmap, TileArgs A) {
  using G = Geo<NDIM, TX, TY, TZ>;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + G::MOFF);
  int* misc = reinterpret_cast<int*>(smem + G::MOFF + 16);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  uint32_t phase = 0;
  // work items: slice 0 of every tile, then the further slices of heavy tiles
  int nextra = 0;
  if (A.nslice) {
    nextra = *A.nextra;
    nextra = nextra < A.extra_cap ? nextra : A.extra_cap;
  }
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const int w = atomicAdd(A.work, 1);
      int t = w, slice = 0;
      if (w >= A.ntiles) {
        t = A.ntiles;  // no work left
        for (int e = w - A.ntiles; e < nextra; e = atomicAdd(A.work, 1) - A.ntiles) {
          const int2 x = A.extra[e];
          if (x.x >= 0) {  // entries of a tile whose reservation did not fit are -1
            t = x.x;
            slice = x.y;
            break;
          }
        }
      }
      misc[0] = t;
      misc[2] = slice;
      misc[1] = 0;
    }
    __syncthreads();
    const int t = misc[0];
    if (t >= A.ntiles) break;
    if (!sort_tile<NDIM, TX, TY, TZ, SORT, CYL, IDW>(A, &fmap, &jmap, t, misc[2], smem, phase)) return;
  }
}

// Many independent simulations in one launch: work item w is tile
// w - tile0[s] of table entry s (one entry per simulation and species), whose
// arguments and tensor maps live in device memory.
struct BatchTable {
  const TileArgs* args;
  const CUtensorMap* fmaps;
  const CUtensorMap* jmaps;
  const int* tile0;  // [n + 1] first work item of each entry
  int n;
  int* work;
};

template <int NDIM, int TX, int TY, int TZ, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_tile_push_batch(const BatchTable B) {
  using G = Geo<NDIM, TX, TY, TZ>;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + G::MOFF);
  int* misc = reinterpret_cast<int*>(smem + G::MOFF + 16);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  const int total = B.tile0[B.n];
  uint32_t phase = 0;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const int w = atomicAdd(B.work, 1);
      int s = 0;
      if (w < total) {  // last entry whose first work item is <= w
        int lo = 0, hi = B.n - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (B.tile0[mid] <= w)
            lo = mid;
          else
            hi = mid - 1;
        }
        s = lo;
      }
      misc[0] = w;
      misc[2] = s;
      misc[1] = 0;
    }
    __syncthreads();
    const int w = misc[0];
    if (w >= total) break;
    const int s = misc[2];
    if (!sort_tile<NDIM, TX, TY, TZ, true>(B.args[s], B.fmaps + s, B.jmaps + s, w - B.tile0[s], 0, smem, phase))
      return;
  }
}

// ============================================================================
// Small-tile kernel: every tile holds at most kCapS particles, so one CTA
// stages a whole tile in shared memory and the pipeline runs on TMA:
//   tile t computes while the tile it takes next streams in (fields into the
//   other field buffer, particles into the input stage, by 1D bulk copies);
//   the stayers leave cell-sorted through an output stage by bulk stores; the
//   current tiles are double-buffered so a tile's reduce-add drains while the
//   next tile deposits.  Tiles with more particles (density far from the mean)
//   are processed straight from global memory in chunks.
// ============================================================================
constexpr int kCapS = 768;                // particles per staged tile
constexpr int kPPTS = kCapS / kThreads;  // 3
constexpr int kQCapS = 96;
constexpr int kNA = 8;                    // staged arrays: cell, o1..o3, u1..u3, id

template <int NDIM, int TX, int TY, int TZ>
struct GeoS {
  using G = Geo<NDIM, TX, TY, TZ>;
  static constexpr int FB = ((6 * G::FPL * 4 + 127) / 128) * 128;
  static constexpr int JB = ((3 * G::JPL * 4 + 127) / 128) * 128;
  static constexpr int SB = kNA * kCapS * 4;
  static constexpr int F0 = 0, F1 = FB, J0 = 2 * FB, J1 = 2 * FB + JB;
  static constexpr int IN = 2 * FB + 2 * JB;
  static constexpr int OUT = IN + SB;
  static constexpr int H = OUT + SB;
  static constexpr int QO = H + ((G::NK * 4 + 15) / 16) * 16;
  static constexpr int MO = QO + ((kQCapS * G::QW * 4 + 15) / 16) * 16;
  static constexpr int SMEM = MO + 256;
  // misc ints (after 3 mbarriers): sort scratch 6..15, then the tile pipeline
  static constexpr int M_TILE = 16, M_NEXT = 17, M_QN = 18, M_NS = 19, M_NI = 20, M_AOFF = 21, M_BIG = 22,
                       M_NST = 23;
};


// Thread 0: start the copies of tile t's fields and particles; record where
// the particles land in the input stage.
template <int NDIM, int TX, int TY, int TZ>
__device__ inline void issue_tile(const TileArgs& A, const CUtensorMap* fmap, int t, float* F, uint64_t* fbar,
                                  float* IN, uint64_t* inbar, int* misc) {
  using S = GeoS<NDIM, TX, TY, TZ>;
  using G = Geo<NDIM, TX, TY, TZ>;
  const int tix = t % A.nt[0], tiy = (t / A.nt[0]) % A.nt[1], tiz = t / (A.nt[0] * A.nt[1]);
  mbar_arrive_expect_tx(fbar, (uint32_t)G::FBYTES);
  if (NDIM == 3)
    tma_load_4d(F, fmap, fbar, tix * TX, tiy * TY, tiz * TZ, 0);
  else
    tma_load_3d(F, fmap, fbar, tix * TX, tiy * TY, 0);
  const int ns = A.in.stay[t];
  int ni = A.in.inc[t];
  ni = ni < A.res[t] ? ni : A.res[t];
  const long long base = A.base[t];
  const int cap = A.cap[t];
  misc[S::M_NS] = ns;
  misc[S::M_NI] = ni;
  if (ns + ni + 9 > kCapS) {  // over-full tile: processed from global memory
    misc[S::M_BIG] = 1;
    mbar_arrive_expect_tx(inbar, 0);
    return;
  }
  misc[S::M_BIG] = 0;
  const int ns4 = (ns + 3) & ~3;
  const int a0 = (cap - ni) & ~3;          // aligned start of the arrivals
  const int delta = (cap - ni) - a0;
  const int ni4 = (ni + delta + 3) & ~3;
  misc[S::M_AOFF] = ns4 + delta;
  int na = 0;
  for (int a = 0; a < kNA; ++a)
    if (arr_ptr(A.in.p, a) && !(NDIM == 2 && a == 3)) ++na;
  mbar_arrive_expect_tx(inbar, (uint32_t)(na * (ns4 + (ni > 0 ? ni4 : 0)) * 4));
  for (int a = 0; a < kNA; ++a) {
    const float* src = reinterpret_cast<const float*>(arr_ptr(A.in.p, a));
    if (!src || (NDIM == 2 && a == 3)) continue;
    float* dst = IN + a * kCapS;
    if (ns4 > 0) bulk_g2s(dst, src + base, (uint32_t)ns4 * 4, inbar);
    if (ni > 0) bulk_g2s(dst + ns4, src + base + a0, (uint32_t)ni4 * 4, inbar);
  }
}

template <int NDIM>
__device__ inline P stage_get(const float* IN, int i) {
  P p;
  p.cell = __float_as_uint(IN[i]);
  p.o0 = IN[kCapS + i];
  p.o1 = IN[2 * kCapS + i];
  p.o2 = NDIM == 3 ? IN[3 * kCapS + i] : 0.f;
  p.u0 = IN[4 * kCapS + i];
  p.u1 = IN[5 * kCapS + i];
  p.u2 = IN[6 * kCapS + i];
  p.id = __float_as_int(IN[7 * kCapS + i]);
  p.w = 1.f;  // weighted species do not use the small-tile kernel
  return p;
}

template <int NDIM, int TX, int TY, int TZ>
__global__ void __launch_bounds__(kThreads, 3)
    k_tile_push_s(const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap jmap, TileArgs A) {
  using G = Geo<NDIM, TX, TY, TZ>;
  using S = GeoS<NDIM, TX, TY, TZ>;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* Fb[2] = {reinterpret_cast<float*>(smem + S::F0), reinterpret_cast<float*>(smem + S::F1)};
  float* Jb[2] = {reinterpret_cast<float*>(smem + S::J0), reinterpret_cast<float*>(smem + S::J1)};
  float* IN = reinterpret_cast<float*>(smem + S::IN);
  float* OUT = reinterpret_cast<float*>(smem + S::OUT);
  int* hist = reinterpret_cast<int*>(smem + S::H);
  float* Q = reinterpret_cast<float*>(smem + S::QO);
  uint64_t* fbar = reinterpret_cast<uint64_t*>(smem + S::MO);  // [2]
  uint64_t* inbar = fbar + 2;
  int* misc = reinterpret_cast<int*>(smem + S::MO + 32);
  const int tid = threadIdx.x;
  const bool has_id = A.in.p.id != nullptr;

  if (tid == 0) {
    mbar_init(&fbar[0], 1);
    mbar_init(&fbar[1], 1);
    mbar_init(inbar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    const int t0 = atomicAdd(A.work, 1);
    misc[S::M_TILE] = t0;
    if (t0 < A.ntiles) issue_tile<NDIM, TX, TY, TZ>(A, &fmap, t0, Fb[0], &fbar[0], IN, inbar, misc);
  }
  __syncthreads();
  uint32_t fph0 = 0, fph1 = 0, iph = 0;
  for (int it = 0;; ++it) {
    const int t = misc[S::M_TILE];
    if (t >= A.ntiles) break;
    const int fb = it & 1;
    const int tix = t % A.nt[0], tiy = (t / A.nt[0]) % A.nt[1], tiz = t / (A.nt[0] * A.nt[1]);
    const long long base = A.base[t];
    const int cap = A.cap[t];
    const int room = cap - A.res[t];
    const uint32_t fph = fb ? fph1 : fph0;
    bool ok = mbar_wait_bounded(&fbar[fb], fph, kWaitLimit);
    ok = mbar_wait_bounded(inbar, iph, kWaitLimit) && ok;
    if (__syncthreads_or(!ok)) {  // every thread takes the same decision
      if (tid == 0) atomicOr(A.status, ST_TIMEOUT);
      mbar_wait_bounded(&fbar[fb], fph, kWaitLimit);
      mbar_wait_bounded(inbar, iph, kWaitLimit);
      break;
    }
    if (fb) fph1 ^= 1u; else fph0 ^= 1u;
    iph ^= 1u;
    const int ns = misc[S::M_NS], ni = misc[S::M_NI], aoff = misc[S::M_AOFF], big = misc[S::M_BIG];
    const int n = ns + ni;
    P pp[kPPTS];
    int nvalid = 0;
    if (!big) {
      const int first = tid * kPPTS;
      nvalid = n - first;
      nvalid = nvalid < 0 ? 0 : (nvalid > kPPTS ? kPPTS : nvalid);
#pragma unroll
      for (int r = 0; r < kPPTS; ++r) {
        if (r < nvalid) {
          const int i = first + r;
          pp[r] = stage_get<NDIM>(IN, i < ns ? i : aoff + (i - ns));
          if (!has_id) pp[r].id = 0;
        }
      }
    }
    if (tid == 0) tma_wait_read1();  // current tile Jb[fb] of two tiles ago has been read
    __syncthreads();                  // the input stage and the tile's metadata are consumed
    if (tid == 0) {
      const int tn = atomicAdd(A.work, 1);
      misc[S::M_NEXT] = tn;
      misc[S::M_QN] = 0;
      if (tn < A.ntiles) issue_tile<NDIM, TX, TY, TZ>(A, &fmap, tn, Fb[fb ^ 1], &fbar[fb ^ 1], IN, inbar, misc);
    }
    float* F = Fb[fb];
    float* J = Jb[fb];
    for (int k = tid; k < 3 * G::JPL; k += kThreads) J[k] = 0.f;
    for (int k = tid; k < G::NK; k += kThreads) hist[k] = 0;
    __syncthreads();

    if (!big) {
      int key[kPPTS];
      {
        Acc acc;
#pragma unroll
        for (int k = 0; k < 12; ++k) acc.w[k] = 0.f;
        acc.cell = -1;
#pragma unroll
        for (int r = 0; r < kPPTS; ++r)
          key[r] = r < nvalid ? push_one<NDIM, TX, TY, TZ, kQCapS>(F, J, A, pp[r], acc, Q, misc + S::M_QN) : 0;
        acc_flush<NDIM, TX, TY, TZ>(J, acc);
      }
      {
        int hk = -1, hc = 0;
#pragma unroll
        for (int r = 0; r < kPPTS; ++r) {
          if (r < nvalid) {
            if (key[r] != hk) {
              if (hk >= 0) atomicAdd(&hist[hk], hc);
              hk = key[r];
              hc = 0;
            }
            ++hc;
          }
        }
        if (hk >= 0) atomicAdd(&hist[hk], hc);
      }
      __syncthreads();
      {
        const int nq = misc[S::M_QN];
        drain_queue<NDIM, TX, TY, TZ>(J, A, Q, nq < kQCapS ? nq : kQCapS);
      }
      if (tid < 32) {  // exclusive scan of the key histogram by one warp
        constexpr int PW = (G::NK + 31) / 32;
        int v[PW];
        int run = 0;
#pragma unroll
        for (int r = 0; r < PW; ++r) {
          const int k = tid * PW + r;
          v[r] = k < G::NK ? hist[k] : 0;
          run += v[r];
        }
        int x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, x, o);
          if (tid >= o) x += y;
        }
        int pre = x - run;
#pragma unroll
        for (int r = 0; r < PW; ++r) {
          const int k = tid * PW + r;
          if (k < G::NK) hist[k] = pre;
          if (k == G::NC) misc[S::M_NST] = pre;
          pre += v[r];
        }
      }
      if (tid == 0) tma_wait_read0();  // the output stage's previous bulk stores have read it
      __syncthreads();
      // rank within key (a run of equal keys takes one atomic); stayers to the
      // output stage in cell order, leavers straight to their new tile
      {
        int r = 0;
        while (r < nvalid) {
          const int k = key[r];
          int m = 1;
          while (r + m < nvalid && key[r + m] == k) ++m;
          const int p0 = atomicAdd(&hist[k], m);
          for (int j = 0; j < m; ++j) {
            const P& q = pp[r + j];
            if (k < G::NC) {
              const int pos = p0 + j;
              if (pos < room) {
                OUT[pos] = __uint_as_float(q.cell);
                OUT[kCapS + pos] = q.o0;
                OUT[2 * kCapS + pos] = q.o1;
                if (NDIM == 3) OUT[3 * kCapS + pos] = q.o2;
                OUT[4 * kCapS + pos] = q.u0;
                OUT[5 * kCapS + pos] = q.u1;
                OUT[6 * kCapS + pos] = q.u2;
                OUT[7 * kCapS + pos] = __int_as_float(q.id);
              } else {
                spill_put(A, t, q);
              }
            } else {
              const int dir = (int)(q.cell >> 24);
              const int ix = (tix + dir % 3 - 1 + A.nt[0]) % A.nt[0];
              const int iy = (tiy + (dir / 3) % 3 - 1 + A.nt[1]) % A.nt[1];
              const int iz = (tiz + dir / 9 - 1 + A.nt[2]) % A.nt[2];
              const int dt_ = (iz * A.nt[1] + iy) * A.nt[0] + ix;
              P q2 = q;
              q2.cell = (q.cell & 0x00FFFFFFu) | ((uint32_t)DIR_STAY << 24);
              const int slot = atomicAdd(&A.out.inc[dt_], 1);
              if (slot < A.res[dt_])
                store_particle<NDIM>(A.out.p, A.base[dt_] + A.cap[dt_] - 1 - slot, q2);
              else
                spill_put(A, dt_, q2);
            }
          }
          r += m;
        }
      }
    } else {
      // over-full tile: chunks straight from global memory, each sorted by cell
      int ws = 0;
      for (int c0 = 0; c0 < n; c0 += kCapS) {
        P qq[kPPTS];
        int key[kPPTS];
        const int first = c0 + tid * kPPTS;
        int nv = n - first;
        nv = nv < 0 ? 0 : (nv > kPPTS ? kPPTS : nv);
#pragma unroll
        for (int r = 0; r < kPPTS; ++r) {
          if (r < nv) {
            const int i = first + r;
            const long long s = i < ns ? base + i : base + cap - ni + (i - ns);
            qq[r] = P{A.in.p.cell[s], A.in.p.o[0][s], A.in.p.o[1][s], NDIM == 3 ? A.in.p.o[2][s] : 0.f,
                      A.in.p.u[0][s], A.in.p.u[1][s], A.in.p.u[2][s], has_id ? A.in.p.id[s] : 0, 1.f};
          }
        }
        Acc acc;
#pragma unroll
        for (int k = 0; k < 12; ++k) acc.w[k] = 0.f;
        acc.cell = -1;
#pragma unroll
        for (int r = 0; r < kPPTS; ++r)
          key[r] = r < nv ? push_one<NDIM, TX, TY, TZ, kQCapS>(F, J, A, qq[r], acc, Q, misc + S::M_QN) : 0;
        acc_flush<NDIM, TX, TY, TZ>(J, acc);
        sort_and_store<NDIM, TX, TY, TZ, kPPTS>(A, t, tix, tiy, tiz, base, room, qq, key, nv, ws, hist, misc);
        __syncthreads();
        const int nq = misc[S::M_QN];
        drain_queue<NDIM, TX, TY, TZ>(J, A, Q, nq < kQCapS ? nq : kQCapS);
        __syncthreads();
        if (tid == 0) misc[S::M_QN] = 0;
        __syncthreads();
      }
      if (tid == 0) misc[S::M_NST] = -1 - (ws < room ? ws : room);  // already stored
    }
    // flush: current tile by TMA reduce-add, stayers by bulk stores
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      if (NDIM == 3)
        tma_reduce_add_4d(&jmap, J, tix * TX, tiy * TY, tiz * TZ, 0);
      else
        tma_reduce_add_3d(&jmap, J, tix * TX, tiy * TY, 0);
      int nst = misc[S::M_NST];
      if (nst >= 0) {
        nst = nst < room ? nst : room;
        const int n4 = (nst + 3) & ~3;  // room is a multiple of 4, so n4 <= room
        if (n4 > 0)
          for (int a = 0; a < kNA; ++a) {
            float* dst = reinterpret_cast<float*>(arr_ptr(A.out.p, a));
            if (!dst || (NDIM == 2 && a == 3)) continue;
            bulk_s2g(dst + base, OUT + a * kCapS, (uint32_t)n4 * 4);
          }
      } else {
        nst = -1 - nst;
      }
      A.out.stay[t] = nst;
      tma_commit();
      misc[S::M_TILE] = misc[S::M_NEXT];
    }
    __syncthreads();
  }
  if (tid == 0) tma_wait0();
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

// slot of the k-th particle of tile t: stayers from the front, arrivals at the back
__device__ inline long long tile_slot(const Tiles& tg, const TileSide& in, int t, int k, int& n) {
  int ns = in.stay[t];
  ns = ns < tg.cap[t] - tg.res[t] ? ns : tg.cap[t] - tg.res[t];  // a sliced tile counts its overflow too
  int ni = in.inc[t];
  ni = ni < tg.res[t] ? ni : tg.res[t];
  n = ns + ni;
  return k < ns ? tg.base[t] + k : tg.base[t] + tg.cap[t] - ni + (k - ns);
}

// live (non-empty) slots of every tile
__global__ void k_tile_live(Tiles tg, TileSide in, int* live) {
  const int t = blockIdx.x;
  int n;
  tile_slot(tg, in, t, 0, n);
  int c = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) c += in.p.cell[tile_slot(tg, in, t, k, n)] != kHoleCell;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  __shared__ int red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    live[t] = s;
  }
}

// every live particle of tile t to out[out_off[t] ...], in slot order (so two
// flattenings of the same store agree particle by particle)
__global__ void k_flatten(Tiles tg, TileSide in, const long long* out_off, Flat32 out) {
  __shared__ int wsum[32];
  __shared__ int done;
  const int t = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) done = 0;
  __syncthreads();
  int n;
  tile_slot(tg, in, t, 0, n);
  const long long o = out_off[t];
  for (int k0 = 0; k0 < n; k0 += blockDim.x) {
    const int k = k0 + threadIdx.x;
    long long s = 0;
    uint32_t c = kHoleCell;
    if (k < n) {
      s = tile_slot(tg, in, t, k, n);
      c = in.p.cell[s];
    }
    const bool v = c != kHoleCell;
    const unsigned m = __ballot_sync(0xffffffffu, v);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int pre = done, tot = 0;
    for (int w = 0; w < nw; ++w) {
      pre += w < warp ? wsum[w] : 0;
      tot += wsum[w];
    }
    if (v) {
      const long long w = o + pre + __popc(m & ((1u << lane) - 1u));
      out.tile[w] = dest_tile(tg, t, c);
      out.cell[w] = (c & 0x00FFFFFFu) | ((uint32_t)DIR_STAY << 24);
      out.o[0][w] = in.p.o[0][s];
      out.o[1][w] = in.p.o[1][s];
      out.o[2][w] = tg.ndim == 3 ? in.p.o[2][s] : 0.f;
      out.u[0][w] = in.p.u[0][s];
      out.u[1][w] = in.p.u[1][s];
      out.u[2][w] = in.p.u[2][s];
      if (out.id) out.id[w] = in.p.id ? in.p.id[s] : 0;
      if (out.w) out.w[w] = in.p.w ? in.p.w[s] : 1.f;
    }
    __syncthreads();
    if (threadIdx.x == 0) done += tot;
    __syncthreads();
  }
}

// Tile counts and the scatter into the tile regions.  The flat input is
// mostly grouped by tile (the loader's lattice order, a flattened store), so
// the lanes of a warp that share a tile take their slots with one atomic
// (match, then the leader adds the group's size and shares the base).  Every
// block is a whole number of warps; lanes past n carry tile -1.
__global__ void k_flat_count(Flat32 f, long long n, int ntiles, int* counts) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int t = k < n ? f.tile[k] : -1;
  if (t >= ntiles) t = -1;
  const unsigned peers = __match_any_sync(0xffffffffu, t);
  if (t >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&counts[t], __popc(peers));
}
__global__ void k_flat_scatter(Flat32 f, long long n, Tiles tg, int* cursor, Part32 out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int t = k < n ? f.tile[k] : -1;
  if (t >= tg.ntiles) t = -1;
  const unsigned peers = __match_any_sync(0xffffffffu, t);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (t >= 0 && lane == leader) base = atomicAdd(&cursor[t], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (t < 0) return;
  const int r = base + __popc(peers & ((1u << lane) - 1u));
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
  if (out.w) out.w[s] = f.w ? f.w[k] : 1.f;
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
                                 const int* id, const double* w, long long n, Flat32 out, int* status) {
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
    if (c >= nn[d]) {
      if (d == 0 && L.open_x) {  // open x1: stay in the last cell, just below its far face
        c = nn[d] - 1;
        o = 0.99999994f;
      } else {
        c -= nn[d];
      }
    }
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
  if (out.w) out.w[k] = w ? (float)w[k] : 1.f;
}

// Charge density of one tile's particles (one block per tile).  Every stored
// particle's cell is local to its tile, so its weights land on the tile's
// (T+1)^d nodes.  A warp takes kRhoWarp consecutive slots; each lane takes
// kRhoRun consecutive ones (cell-sorted runs after the last sort), read as two
// groups of four with one 128-bit load per array (four stayers: regions are
// 16-byte aligned) or one by one (the last stayers, the arrivals), and sums
// the weights of consecutive same-cell particles in registers (FP32).  Each run goes into a shared node
// tile of 64-bit fixed-point sums in units of 2^-32, so the node sums do not
// depend on the order of the adds (a node's sum must stay below 2^31 particle
// weights).  The sums are kept as two 32-bit words added by 32-bit atomics: the
// low word's carry goes into the high word with the high part of the add.  The
// node tile is then added to the FP64 grid once: plain adds for the nodes no
// other tile touches, atomics on the tile's faces.
// KIN: the same pass also sums the kinetic energy m c^2 (gamma - 1) and the
// charge of the tile's particles into acc; gamma - 1 = u^2 / (1 + gamma) in
// FP32 from the FP32 momenta (no cancellation at small u), summed per run in
// FP32 and across runs in FP64.
constexpr int kRhoRun = 8;
constexpr int kRhoWarp = 32 * kRhoRun;
constexpr int kRhoThreads = 128;

template <bool KIN>
__global__ void __launch_bounds__(kRhoThreads, 8) k_tiled_rho(Layout L, PushConst C, Tiles tg, TileSide in, double* rho,
                                                           Diag64* acc) {
  // node sums, fixed point in units of 2^-32: low words Rlo[nr], high words Rhi[nr]
  extern __shared__ unsigned int Rlo[];
  const int t = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int R0 = tg.T[0] + 1, R1 = tg.T[1] + 1, R2 = tg.ndim == 3 ? tg.T[2] + 1 : 1;
  const int nr = R0 * R1 * R2;
  int* Rhi = reinterpret_cast<int*>(Rlo + nr);
  for (int q = threadIdx.x; q < nr; q += blockDim.x) {
    Rlo[q] = 0u;
    Rhi[q] = 0;
  }
  int ns = in.stay[t];
  ns = ns < tg.cap[t] - tg.res[t] ? ns : tg.cap[t] - tg.res[t];  // a sliced tile counts its overflow too
  int ni = in.inc[t];
  ni = ni < tg.res[t] ? ni : tg.res[t];
  const int n = ns + ni;
  const long long base = tg.base[t], back = tg.base[t] + tg.cap[t] - ni - ns;
  const bool d3 = tg.ndim == 3, has_w = in.p.w != nullptr;
  int o[3];
  tile_origin(tg, t, o);
  __syncthreads();
  double kin = 0.0, live = 0.0;
  for (int k0 = warp * kRhoWarp; k0 < n; k0 += (kRhoThreads / 32) * kRhoWarp) {
    float accw[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float kp = 0.f, lp = 0.f;  // this run's kinetic energy and charge
    int cur = -1;
    auto flush = [&]() {
      const int a = cur & 255, b = (cur >> 8) & 255, c = (cur >> 16) & 255;
      for (int c3 = 0; c3 < (d3 ? 2 : 1); ++c3)
        for (int c2 = 0; c2 < 2; ++c2)
          for (int c1 = 0; c1 < 2; ++c1) {
            // x = hi + lo 2^-32 exactly: floor and fraction of an FP32 value are
            // exact, and the fraction's 2^32 multiple rounds to the nearest unit
            const float x = accw[c3 * 4 + c2 * 2 + c1], fl = floorf(x);
            const int hi = (int)fl;
            const unsigned lo = __float2uint_rn((x - fl) * 4294967296.f);
            const int q = ((c + c3) * R1 + (b + c2)) * R0 + (a + c1);
            const unsigned old = atomicAdd(&Rlo[q], lo);
            const int carry = old + lo < old ? 1 : 0;
            if (hi + carry != 0) atomicAdd(&Rhi[q], hi + carry);
          }
    };
#pragma unroll
    for (int h = 0; h < kRhoRun / 4; ++h) {
      const int kb = k0 + kRhoRun * lane + 4 * h;  // this lane's next four slots
      uint32_t cw[4];
      float e0[4], e1[4], e2[4] = {0.f, 0.f, 0.f, 0.f}, pw[4] = {1.f, 1.f, 1.f, 1.f};
      float ua[4] = {}, ub[4] = {}, uc[4] = {};
      if (kb + 4 <= ns) {  // four stayers
        const long long s = base + kb;
        load_vec(in.p.cell + s, cw);
        load_vec(in.p.o[0] + s, e0);
        load_vec(in.p.o[1] + s, e1);
        if (d3) load_vec(in.p.o[2] + s, e2);
        if (has_w) load_vec(in.p.w + s, pw);
        if constexpr (KIN) {
          load_vec(in.p.u[0] + s, ua);
          load_vec(in.p.u[1] + s, ub);
          load_vec(in.p.u[2] + s, uc);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = kb + j;
          cw[j] = kHoleCell;
          e0[j] = e1[j] = 0.f;
          if (k < n) {
            const long long s = k < ns ? base + k : back + k;
            cw[j] = in.p.cell[s];
            e0[j] = in.p.o[0][s];
            e1[j] = in.p.o[1][s];
            if (d3) e2[j] = in.p.o[2][s];
            if (has_w) pw[j] = in.p.w[s];
            if constexpr (KIN) {
              ua[j] = in.p.u[0][s];
              ub[j] = in.p.u[1][s];
              uc[j] = in.p.u[2][s];
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (cw[j] == kHoleCell) continue;
        const int cell = (int)(cw[j] & 0x00FFFFFFu);
        if (cell != cur) {
          if (cur >= 0) flush();
          cur = cell;
#pragma unroll
          for (int q = 0; q < 8; ++q) accw[q] = 0.f;
        }
        if constexpr (KIN) {
          const float u2 = fmaf(ua[j], ua[j], fmaf(ub[j], ub[j], uc[j] * uc[j]));
          kp = fmaf(pw[j], __fdividef(u2, 1.f + sqrtf(1.f + u2)), kp);  // 2 ulp: far below the gates
          lp += pw[j];
        }
        const float f1[2] = {1.f - e0[j], e0[j]}, f2[2] = {1.f - e1[j], e1[j]}, f3[2] = {1.f - e2[j], e2[j]};
#pragma unroll
        for (int c3 = 0; c3 < 2; ++c3)
#pragma unroll
          for (int c2 = 0; c2 < 2; ++c2) {
            const float w23 = f2[c2] * (d3 ? f3[c3] : 1.f) * pw[j];
#pragma unroll
            for (int c1 = 0; c1 < 2; ++c1)
              accw[c3 * 4 + c2 * 2 + c1] = fmaf(f1[c1], w23, accw[c3 * 4 + c2 * 2 + c1]);
          }
      }
    }
    if (cur >= 0) flush();
    if constexpr (KIN) {
      kin += (double)kp;
      live += (double)lp;
    }
  }
  if constexpr (KIN) {
    __shared__ double red[2][kRhoThreads / 32];
    double dk = kin, dl = live;
    for (int m = 16; m > 0; m >>= 1) {
      dk += __shfl_down_sync(0xffffffffu, dk, m);
      dl += __shfl_down_sync(0xffffffffu, dl, m);
    }
    if (lane == 0) {
      red[0][warp] = dk;
      red[1][warp] = dl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < kRhoThreads / 32; ++w) {
        a += red[0][w];
        b += red[1][w];
      }
      atomicAdd(&acc->kinetic_energy, C.q * C.rqm * a);
      atomicAdd(&acc->total_charge, C.q * b);
    }
  }
  __syncthreads();
  const double qv = C.q / C.dvol;
  for (int q = threadIdx.x; q < nr; q += blockDim.x) {
    const unsigned long long fx = ((unsigned long long)(unsigned)Rhi[q] << 32) + Rlo[q];
    if (fx == 0ull) continue;
    const double v = (double)(long long)fx * (1.0 / 4294967296.0);
    const int a = q % R0, b = (q / R0) % R1, c = q / (R0 * R1);
    const long long g = L.idx(o[0] + a, o[1] + b, o[2] + c);
    const bool face = a == 0 || a == R0 - 1 || b == 0 || b == R1 - 1 || (d3 && (c == 0 || c == R2 - 1));
    if (face)
      atomicAdd(&rho[g], qv * v);
    else
      rho[g] += qv * v;  // no other tile of this launch reaches this node
  }
}

// Moving window: fresh plasma for the new front column (cell index nx1 - 1)
// -- the column's cells in cell order (x3 slowest), the loader's sub-lattice
// in each cell, momenta from the loader's draws for global particle indices
// first, first + 1, ... -- appended to the arrival slots of the last tile
// column on the output side (spill list when full).
struct InjectSpec {
  int ndim;
  int nx[3], ppc[3];
  double uth[3], ufl[3];
  unsigned long long seed;
  long long first;
  double xlo[3], dx[3];  // lower corner of the window after the shift (lab frame), cell size
  ProfileDev prof;
  int has_prof;
  int* kept;             // particles created
};

// Fresh particle k of the front column: first = global index of particle 0
// (the lattice places created so far), xlo0 = the window's lower x1 corner
// after its shift.
__device__ inline void inject_one(const TileArgs& A, const int* T, const int* nt, const InjectSpec& J,
                                  long long first, double xlo0, long long k) {
  const int ppc = J.ppc[0] * J.ppc[1] * J.ppc[2];
  const long long col = k / ppc;
  const int sub = (int)(k - col * ppc);
  const int cj = (int)(col % J.nx[1]), ck = (int)(col / J.nx[1]);
  const int si = sub % J.ppc[0], sj = (sub / J.ppc[0]) % J.ppc[1], sk = sub / (J.ppc[0] * J.ppc[1]);
  const int ix = nt[0] - 1, iy = cj / T[1], iz = J.ndim == 3 ? ck / T[2] : 0;
  const int t = (iz * nt[1] + iy) * nt[0] + ix;
  const int lx = J.nx[0] - 1 - ix * T[0], ly = cj - iy * T[1], lz = J.ndim == 3 ? ck - iz * T[2] : 0;
  P q;
  q.cell = (uint32_t)lx | ((uint32_t)ly << 8) | ((uint32_t)lz << 16) | ((uint32_t)DIR_STAY << 24);
  q.o0 = (float)((si + 0.5) / J.ppc[0]);
  q.o1 = (float)((sj + 0.5) / J.ppc[1]);
  q.o2 = J.ndim == 3 ? (float)((sk + 0.5) / J.ppc[2]) : 0.f;
  const unsigned long long g = (unsigned long long)(first + k);
  float uu[3];
  for (int d = 0; d < 3; ++d)
    uu[d] = (float)(J.uth[d] != 0.0 ? J.ufl[d] + J.uth[d] * normal_dev(J.seed, 3ull * g + d) : J.ufl[d]);
  q.u0 = uu[0];
  q.u1 = uu[1];
  q.u2 = uu[2];
  q.id = (int)g;
  q.w = 1.f;
  if (J.has_prof) {  // the profile at the particle's lab-frame position
    const double x[3] = {xlo0 + (J.nx[0] - 1 + (si + 0.5) / J.ppc[0]) * J.dx[0],
                         J.xlo[1] + (cj + (sj + 0.5) / J.ppc[1]) * J.dx[1],
                         J.ndim == 3 ? J.xlo[2] + (ck + (sk + 0.5) / J.ppc[2]) * J.dx[2] : 0.0};
    const double w = profile_weight(J.prof, x);
    if (!(J.prof.density * w > J.prof.den_min)) return;  // no particle where the density is this low
    q.w = (float)w;
  }
  // the lanes still here are created; a warp's lanes mostly share a tile (a
  // column's cells are consecutive), so each group takes its slots and adds to
  // the count with one atomic
  const unsigned act = __activemask();
  const int lane = threadIdx.x & 31;
  if (lane == __ffs(act) - 1) atomicAdd(J.kept, __popc(act));
  const unsigned peers = __match_any_sync(act, t);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&A.out.inc[t], __popc(peers));
  base = __shfl_sync(peers, base, leader);
  const int slot = base + __popc(peers & ((1u << lane) - 1u));
  if (slot < A.res[t]) {
    const long long s = A.base[t] + A.cap[t] - 1 - slot;
    if (J.ndim == 3)
      store_particle<3>(A.out.p, s, q);
    else
      store_particle<2>(A.out.p, s, q);  // 2D stores have no third offset array
  } else {
    spill_put(A, t, q);
  }
}

__global__ void k_inject(TileArgs A, Tiles tg, InjectSpec J, long long count) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) inject_one(A, tg.T, tg.nt, J, J.first, J.xlo[0], k);
}

// Batched form: entry e (a member and species) owns blocks [blk[e],
// blk[e + 1]); a member that does not shift this step creates nothing.  The
// per-step values (shift flag, window corner, first index) are read from
// device memory, so the launch can be replayed from a graph.
struct InjectBatchSpec {
  InjectSpec J;
  int T[3], nt[3];
  int member;
  long long count;
};

__global__ void k_inject_batch(const TileArgs* args, const InjectBatchSpec* spec, const int* blk, int n,
                               const int* shift, const double* xlo0, const long long* first) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (blk[mid] <= (int)blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  const InjectBatchSpec& S = spec[lo];
  if (!shift[S.member]) return;
  const long long k = (long long)(blockIdx.x - blk[lo]) * blockDim.x + threadIdx.x;
  if (k < S.count) inject_one(args[lo], S.T, S.nt, S.J, first[lo], xlo0[S.member], k);
}

template <int NDIM, int TX, int TY, int TZ, int MINB, bool SORT = true, bool CYL = false, bool IDW = true>
int occupancy() {
  using G = Geo<NDIM, TX, TY, TZ>;
  static int occ = -1;
  if (occ < 0) {
    cudaFuncSetAttribute(k_tile_push<NDIM, TX, TY, TZ, MINB, SORT, CYL, IDW>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_tile_push<NDIM, TX, TY, TZ, MINB, SORT, CYL, IDW>,
                                                      kThreads, G::SMEM) != cudaSuccess ||
        o < 1)
      o = 1;
    occ = o;
  }
  return occ;
}

template <int NDIM, int TX, int TY, int TZ>
int occupancy_s() {
  using S = GeoS<NDIM, TX, TY, TZ>;
  static int occ = -1;
  if (occ < 0) {
    cudaFuncSetAttribute(k_tile_push_s<NDIM, TX, TY, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_tile_push_s<NDIM, TX, TY, TZ>, kThreads, S::SMEM) !=
            cudaSuccess ||
        o < 1)
      o = 1;
    occ = o;
  }
  return occ;
}

// The sorting step of a store without ids and weights (the common case) runs
// the IDW = false instantiation; every other case the general one.
template <int NDIM, int TX, int TY, int TZ, int MINB, bool SORT, bool CYL = false>
void launch_push(const CUtensorMap* fmap, const CUtensorMap* jmap, const TileArgs& A, int grid, cudaStream_t s) {
  using G = Geo<NDIM, TX, TY, TZ>;
  if constexpr (SORT && !CYL) {
    if (!A.in.p.id && !A.in.p.w) {
      occupancy<NDIM, TX, TY, TZ, MINB, SORT, CYL, false>();
      k_tile_push<NDIM, TX, TY, TZ, MINB, SORT, CYL, false><<<grid, kThreads, G::SMEM, s>>>(*fmap, *jmap, A);
      return;
    }
  }
  occupancy<NDIM, TX, TY, TZ, MINB, SORT, CYL>();
  k_tile_push<NDIM, TX, TY, TZ, MINB, SORT, CYL><<<grid, kThreads, G::SMEM, s>>>(*fmap, *jmap, A);
}

// r-z rings (2D shapes only, 4 blocks per SM): the general kernel with the
// ring move; false for a shape it is not built for
template <int NDIM, int TX, int TY, int TZ>
bool launch_push_cyl(const CUtensorMap* fmap, const CUtensorMap* jmap, const TileArgs& A, int grid, bool stream,
                     cudaStream_t s) {
  if constexpr (NDIM == 2) {
    if (stream)
      launch_push<NDIM, TX, TY, TZ, 4, false, true>(fmap, jmap, A, grid, s);
    else
      launch_push<NDIM, TX, TY, TZ, 4, true, true>(fmap, jmap, A, grid, s);
    return true;
  }
  return false;
}

template <int NDIM, int TX, int TY, int TZ>
void launch_push_s(const CUtensorMap* fmap, const CUtensorMap* jmap, const TileArgs& A, int grid, cudaStream_t s) {
  using S = GeoS<NDIM, TX, TY, TZ>;
  occupancy_s<NDIM, TX, TY, TZ>();
  k_tile_push_s<NDIM, TX, TY, TZ><<<grid, kThreads, S::SMEM, s>>>(*fmap, *jmap, A);
}


// ... and of the small-tile kernel (at most kCapS - 9 particles per tile region)
#define PICGB_SMALL_SHAPES(X) \
  X(3, 4, 4, 4)               \
  X(3, 4, 4, 2)               \
  X(3, 8, 4, 4)               \
  X(2, 8, 8, 1)               \
  X(2, 8, 4, 1)               \
  X(2, 16, 8, 1)

}  // namespace

static bool shape_is(int ndim, const int T[3], int n, int a, int b, int c) {
  return ndim == n && T[0] == a && T[1] == b && (n == 2 || T[2] == c);
}

int tiled_push_smem_bytes(int ndim, const int T[3]) {
#define X(N, A_, B_, C_) \
  if (shape_is(ndim, T, N, A_, B_, C_)) return Geo<N, A_, B_, C_>::SMEM;
  PICGB_TILE_SHAPES(X)
#undef X
#define X(N, A_, B_, C_) \
  if (shape_is(ndim, T, N, A_, B_, C_)) return GeoS<N, A_, B_, C_>::SMEM;
  PICGB_SMALL_SHAPES(X)
#undef X
  return -1;
}

bool tiled_has_general(int ndim, const int T[3]) {
#define X(N, A_, B_, C_) \
  if (shape_is(ndim, T, N, A_, B_, C_)) return true;
  PICGB_TILE_SHAPES(X)
#undef X
  return false;
}

bool tiled_has_small(int ndim, const int T[3]) {
#define X(N, A_, B_, C_) \
  if (shape_is(ndim, T, N, A_, B_, C_)) return true;
  PICGB_SMALL_SHAPES(X)
#undef X
  return false;
}

int tiled_small_capacity() { return kCapS - 9; }




int tiled_push_grid(int ndim, const int T[3], int ntiles, bool small, int minb) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int occ = 1;
  if (small) {
#define X(N, A_, B_, C_) \
  if (shape_is(ndim, T, N, A_, B_, C_)) occ = occupancy_s<N, A_, B_, C_>();
    PICGB_SMALL_SHAPES(X)
#undef X
  } else {
#define X(N, A_, B_, C_)                  \
  if (shape_is(ndim, T, N, A_, B_, C_)) \
    occ = minb == 2 ? occupancy<N, A_, B_, C_, 2>() : occupancy<N, A_, B_, C_, 4>();
    PICGB_TILE_SHAPES(X)
#undef X
  }
  const int g = sms * occ;
  return g < ntiles ? g : ntiles;
}

namespace {
TileArgs make_args(const PushConst& C, const Tiles& tg, const TileSide& in, const TileSide& out, Flat32 spill,
                   int* spill_count, long long spill_cap, int* work, int* status) {
  TileArgs A;
  for (int d = 0; d < 3; ++d) A.nt[d] = tg.nt[d];
  A.ntiles = tg.ntiles;
  A.base = tg.base;
  A.cap = tg.cap;
  A.res = tg.res;
  A.in = in;
  A.out = out;
  A.spill = spill;
  A.spill_count = spill_count;
  A.spill_cap = spill_cap;
  A.work = work;
  A.qmdt2 = (float)(C.dt / (2.0 * C.rqm));
  for (int d = 0; d < 3; ++d) {
    A.dt_dx[d] = (float)(C.dt / C.dx[d]);
    A.cf[d] = (float)(C.q * C.dx[d] / (C.dt * C.dvol));
    A.e0[d] = (float)C.e0[d];
    A.b0[d] = (float)C.b0[d];
  }
  A.ext = C.e0[0] != 0.0 || C.e0[1] != 0.0 || C.e0[2] != 0.0 || C.b0[0] != 0.0 || C.b0[1] != 0.0 || C.b0[2] != 0.0;
  A.j3f = (float)(C.q / C.dvol);
  A.isis = C.isis;
  A.status = status;
  A.nslice = nullptr;
  A.extra = nullptr;
  A.nextra = nullptr;
  A.extra_cap = 0;
  A.shift_x = 0;
  A.shift_ptr = nullptr;
  A.open_x = 0;
  A.lost = nullptr;
  A.cyl = 0;
  A.nrow = 0;
  A.dr = 0.f;
  A.dt = 0.f;
  return A;
}

template <int NDIM, int TX, int TY, int TZ, int MINB>
int occupancy_b() {
  using G = Geo<NDIM, TX, TY, TZ>;
  static int occ = -1;
  if (occ < 0) {
    cudaFuncSetAttribute(k_tile_push_batch<NDIM, TX, TY, TZ, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         G::SMEM);
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_tile_push_batch<NDIM, TX, TY, TZ, MINB>, kThreads,
                                                      G::SMEM) != cudaSuccess ||
        o < 1)
      o = 1;
    occ = o;
  }
  return occ;
}
}  // namespace

size_t tiled_args_bytes() { return sizeof(TileArgs); }

void tiled_fill_args(void* dst, const PushConst& C, const Tiles& tg, const TileSide& in, const TileSide& out,
                     Flat32 spill, int* spill_count, long long spill_cap, int* status, int open_x, int* lost,
                     const int* shift_ptr) {
  TileArgs A = make_args(C, tg, in, out, spill, spill_count, spill_cap, nullptr, status);
  A.open_x = open_x;
  A.lost = lost;
  A.shift_ptr = shift_ptr;
  memcpy(dst, &A, sizeof(A));
}

int tiled_batch_grid(int ndim, const int T[3], int total_tiles, int minb) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int occ = 0;
#define X(N, A_, B_, C_) \
  if (shape_is(ndim, T, N, A_, B_, C_)) \
    occ = minb == 2 ? occupancy_b<N, A_, B_, C_, 2>() : occupancy_b<N, A_, B_, C_, 4>();
  PICGB_TILE_SHAPES(X)
#undef X
  if (occ < 1) return 0;
  const int g = sms * occ;
  return g < total_tiles ? g : total_tiles;
}

bool tiled_push_batch(int ndim, const int T[3], const void* args, const CUtensorMap* fmaps, const CUtensorMap* jmaps,
                      const int* tile0, int n, int* work, int grid, int minb, cudaStream_t s) {
  BatchTable B;
  B.args = static_cast<const TileArgs*>(args);
  B.fmaps = fmaps;
  B.jmaps = jmaps;
  B.tile0 = tile0;
  B.n = n;
  B.work = work;
  cudaMemsetAsync(work, 0, sizeof(int), s);
#define X(N, A_, B_, C_)                                                      \
  if (shape_is(ndim, T, N, A_, B_, C_)) {                                     \
    using G = Geo<N, A_, B_, C_>;                                             \
    if (minb == 2) {                                                          \
      occupancy_b<N, A_, B_, C_, 2>();                                        \
      k_tile_push_batch<N, A_, B_, C_, 2><<<grid, kThreads, G::SMEM, s>>>(B); \
    } else {                                                                  \
      occupancy_b<N, A_, B_, C_, 4>();                                        \
      k_tile_push_batch<N, A_, B_, C_, 4><<<grid, kThreads, G::SMEM, s>>>(B); \
    }                                                                         \
    return true;                                                              \
  }
  PICGB_TILE_SHAPES(X)
#undef X
  return false;
}

// Slices of every tile (one per kSliceChunks chunks of its particles); the
// slices after the first are appended to the extra list.  The list is sized
// so that every tile fits (see slice_list_capacity); a tile whose reservation
// would not fit all the same stays whole and marks its entries -1.
__global__ void k_slices(Tiles tg, TileSide in, int* nslice, int2* extra, int* nextra, int cap) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tg.ntiles) return;
  int n;
  tile_slot(tg, in, t, 0, n);
  int ns = in.stay[t];
  const int room = tg.cap[t] - tg.res[t];
  ns = ns < room ? ns : room;
  const int chunks = (ns + (n - ns) + kChunk - 1) / kChunk;  // stayers and arrivals read as one sequence
  int s = (chunks + kSliceChunks - 1) / kSliceChunks;
  s = s > 1 ? s : 1;
  if (s > 1) {
    const int e0 = atomicAdd(nextra, s - 1);
    const bool fits = e0 + (s - 1) <= cap;
    for (int k = 1; k < s && e0 + k - 1 < cap; ++k) extra[e0 + k - 1] = fits ? make_int2(t, k) : make_int2(-1, 0);
    if (!fits) s = 1;
  }
  nslice[t] = s;
}

// A tile region of c slots holds at most c / kChunk + 1 chunks, so it adds at
// most c / (kChunk kSliceChunks) + 1/8 slices to the list.
long long slice_list_capacity(long long slots, int ntiles) {
  return slots / (kChunk * kSliceChunks) + ntiles / 4 + 64;
}

int tiled_push(const Layout& L, const PushConst& C, const Tiles& tg, const TileSide& in, const TileSide& out,
                Flat32 spill, int* spill_count, long long spill_cap, int grid, int* work, const CUtensorMap* fmap,
                const CUtensorMap* jmap, int* status, bool stream, int minb, int shift_x, int* lost,
                const SliceScratch* slices, cudaStream_t s) {
  TileArgs A = make_args(C, tg, in, out, spill, spill_count, spill_cap, work, status);
  A.shift_x = shift_x;
  A.open_x = L.open_x;
  A.lost = lost;
  A.cyl = C.cyl;
  A.nrow = L.ny;
  A.dr = (float)C.dx[1];
  A.dt = (float)C.dt;
  int launches = 1;
  if (slices && slices->extra && !stream && !tg.small) {  // heavy tiles are split over several blocks
    cudaMemsetAsync(slices->nextra, 0, sizeof(int), s);
    cudaMemsetAsync(out.stay, 0, sizeof(int) * (size_t)tg.ntiles, s);
    k_slices<<<(tg.ntiles + 255) / 256, 256, 0, s>>>(tg, in, slices->nslice, slices->extra, slices->nextra,
                                                     slices->cap);
    A.nslice = slices->nslice;
    A.extra = slices->extra;
    A.nextra = slices->nextra;
    A.extra_cap = slices->cap;
    launches += 1;
  }
  cudaMemsetAsync(work, 0, sizeof(int), s);
  cudaMemsetAsync(out.inc, 0, sizeof(int) * (size_t)tg.ntiles, s);
  const int* T = tg.T;
  if (tg.small) {
#define X(N, A_, B_, C_)                                \
  if (shape_is(tg.ndim, T, N, A_, B_, C_)) {            \
    launch_push_s<N, A_, B_, C_>(fmap, jmap, A, grid, s); \
    return launches;                                    \
  }
    PICGB_SMALL_SHAPES(X)
#undef X
  }
  // the general kernel: counting sort by cell, or (between re-sorts) the
  // order-keeping compaction
#define X(N, A_, B_, C_)                                                    \
  if (shape_is(tg.ndim, T, N, A_, B_, C_)) {                                \
    if (A.cyl)                                                              \
      return launch_push_cyl<N, A_, B_, C_>(fmap, jmap, A, grid, stream, s) ? launches : 0; \
    if (minb == 2)                                                          \
      stream ? launch_push<N, A_, B_, C_, 2, false>(fmap, jmap, A, grid, s) \
             : launch_push<N, A_, B_, C_, 2, true>(fmap, jmap, A, grid, s); \
    else                                                                    \
      stream ? launch_push<N, A_, B_, C_, 4, false>(fmap, jmap, A, grid, s) \
             : launch_push<N, A_, B_, C_, 4, true>(fmap, jmap, A, grid, s); \
    return launches;                                                        \
  }
  PICGB_TILE_SHAPES(X)
#undef X
  return 0;
}

void tiled_inject(const PushConst& C, const Tiles& tg, const TileSide& out, Flat32 spill, int* spill_count,
                  long long spill_cap, int* status, const int nx[3], const int ppc[3], const double uth[3],
                  const double ufl[3], unsigned long long seed, long long first, long long count,
                  const ProfileDev* prof, int* kept, cudaStream_t s) {
  if (count <= 0) return;
  const TileArgs A = make_args(C, tg, out, out, spill, spill_count, spill_cap, nullptr, status);
  InjectSpec J;
  J.ndim = tg.ndim;
  for (int d = 0; d < 3; ++d) {
    J.nx[d] = nx[d];
    J.ppc[d] = ppc[d];
    J.uth[d] = uth[d];
    J.ufl[d] = ufl[d];
  }
  J.seed = seed;
  J.first = first;
  for (int d = 0; d < 3; ++d) {
    J.xlo[d] = C.xmin[d] + (d == 0 ? C.dx[0] : 0.0);  // the window after its one-cell shift
    J.dx[d] = C.dx[d];
  }
  J.has_prof = prof != nullptr;
  if (prof) J.prof = *prof;
  J.kept = kept;
  k_inject<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(A, tg, J, count);
}

size_t tiled_inject_spec_bytes() { return sizeof(InjectBatchSpec); }

void tiled_fill_inject(void* dst, const PushConst& C, const Tiles& tg, const int nx[3], const int ppc[3],
                       const double uth[3], const double ufl[3], unsigned long long seed, const ProfileDev* prof,
                       int* kept, int member, long long count) {
  InjectBatchSpec S{};
  S.J.ndim = tg.ndim;
  for (int d = 0; d < 3; ++d) {
    S.J.nx[d] = nx[d];
    S.J.ppc[d] = ppc[d];
    S.J.uth[d] = uth[d];
    S.J.ufl[d] = ufl[d];
    S.J.xlo[d] = C.xmin[d];  // x1 is replaced by the step's value
    S.J.dx[d] = C.dx[d];
    S.T[d] = tg.T[d];
    S.nt[d] = tg.nt[d];
  }
  S.J.seed = seed;
  S.J.has_prof = prof != nullptr;
  if (prof) S.J.prof = *prof;
  S.J.kept = kept;
  S.member = member;
  S.count = count;
  memcpy(dst, &S, sizeof(S));
}

void tiled_inject_batch(const void* args, const void* specs, const int* blk, int n, int nblk, const int* shift,
                        const double* xlo0, const long long* first, cudaStream_t s) {
  if (nblk > 0)
    k_inject_batch<<<nblk, 256, 0, s>>>(static_cast<const TileArgs*>(args),
                                        static_cast<const InjectBatchSpec*>(specs), blk, n, shift, xlo0, first);
}

void tiled_flatten(const Tiles& tg, const TileSide& in, const long long* out_off, Flat32 out, cudaStream_t s) {
  k_flatten<<<tg.ntiles, 256, 0, s>>>(tg, in, out_off, out);
}

void tiled_live(const Tiles& tg, const TileSide& in, int* live, cudaStream_t s) {
  k_tile_live<<<tg.ntiles, 256, 0, s>>>(tg, in, live);
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
                    double* const u[3], const int* id, const double* w, long long n, Flat32 out, int* status,
                    cudaStream_t s) {
  if (n == 0) return;
  k_global_to_flat<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ndim, L, tg, C, x[0], x[1], x[2], u[0], u[1], u[2],
                                                                id, w, n, out, status);
}

void tiled_rho(const Layout& L, const PushConst& C, const Tiles& tg, const TileSide& in, double* rho, Diag64* acc,
               cudaStream_t s) {
  const size_t nodes = (size_t)(tg.T[0] + 1) * (tg.T[1] + 1) * (tg.ndim == 3 ? tg.T[2] + 1 : 1);
  if (acc)
    k_tiled_rho<true><<<tg.ntiles, kRhoThreads, 8 * nodes, s>>>(L, C, tg, in, rho, acc);
  else
    k_tiled_rho<false><<<tg.ntiles, kRhoThreads, 8 * nodes, s>>>(L, C, tg, in, rho, nullptr);
}

}  // namespace picgb
