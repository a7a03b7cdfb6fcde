// kernels.h -- internal launchers of libpicgb (host side, C++; not part of the ABI).
#pragma once

#include "common.cuh"

namespace picgb {

// ----------------------------------------------------------------- grid fields
struct Diag64 {           // device accumulators of one diagnostic pass (FP64)
  double field_energy;
  double kinetic_energy;
  double total_charge;
  double gauss_max;
  double rho_max;
  double rho_part_max;
};

template <typename T> void fill_guards(const Layout& L, T* const* comps, int ncomp, cudaStream_t s);
template <typename T> void fold_guards(const Layout& L, T* const* comps, int ncomp, cudaStream_t s);
template <typename T>
void smooth_pass(const Layout& L, T* comp, T* tmp, int dim, double w0, double w1, double w2, cudaStream_t s);
template <typename T>
void yee_b_half(const Layout& L, T* const* e, T* const* b, double dt, const double dx[3], cudaStream_t s);
// inc (FP32 form, open x1): B2 and B3 just below the lower x1 boundary,
// [2][ny nz], read there instead of 0 (antenna pulses); null: 0
template <typename T>
void yee_e(const Layout& L, T* const* e, T* const* b, T* const* j, double dt, const double dx[3], cudaStream_t s,
           const float* inc = nullptr);
template <typename T> void field_energy(const Layout& L, T* const* f, Diag64* acc, cudaStream_t s);
// field energy and the Gauss-law maxima of the FP32 fields in one pass (f:
// E1..E3, B1..B3)
void diag_fields(const Layout& L, float* const* f, const double* rho, double rho_bg, const double dx[3], Diag64* acc,
                 cudaStream_t s);
// moving window: every E/B value one cell back in x1, zero front column
template <typename T> void shift_x(const Layout& L, T* const* comps, int ncomp, cudaStream_t s);
// laser pulse added to the fields; p: vosc, k, w0, rise, length, fall,
// x_front, transverse axis position (in-plane), axis x3, cos pol, sin pol,
// phase, xmin[3], dx[3], propagation axis (0: x1, 1: x2), focus on, x_focus
template <typename T> void laser_add(const Layout& L, T* const* f, const double* p, cudaStream_t s);
// antenna pulses: a record of antenna_bytes() bytes per pulse, written by
// antenna_store from the same parameters as laser_add (with `start` in
// place of x_front and the lab focal plane); antenna_plane sums their B2, B3
// just below the lower x1 boundary at lab position xlo1 and time t into inc
size_t antenna_bytes();
void antenna_store(const double* p, void* dst);
// txlo non-null: t and xlo1 are read from txlo[0], txlo[1] on the device
void antenna_plane(const Layout& L, const void* ants, int n, double t, double xlo1, float* inc, cudaStream_t s,
                   const double* txlo = nullptr);
template <typename T>
void gauss_residual(const Layout& L, T* const* e, const double* rho, double rho_bg, const double dx[3], Diag64* acc,
                    cudaStream_t s);
template <typename T> void pack_interior(const Layout& L, const T* comp, double* dst, cudaStream_t s);
template <typename T> void unpack_interior(const Layout& L, const double* src, T* comp, cudaStream_t s);
// E1 from the discrete Gauss law along x1, column by column (rho padded FP64).
template <typename T> void init_e_gauss_x1(const Layout& L, const double* rho, double rho_bg, double dx1, T* e1,
                                           cudaStream_t s);

// Batched FP32 field step (pic_batch): one launch per stage for all members.
// Each table lists, per member, the first block of that member in the launch
// (blk_*[n] = the total); the block counts per member are batch_*_blocks.
struct BatchFieldMember {
  Layout L;
  float* f[6];            // E1..E3, B1..B3
  float* j[3];
  float h, dt, i1, i2, i3;  // dt / 2, dt and 1 / dx, as the single-simulation sweeps take them
  const float* inc;       // antenna B plane below the lower x1 boundary, or null
};
struct BatchFieldTable {
  const BatchFieldMember* m;
  const int* blk_int;     // interior sweeps: blocks of 32 x 8 cells
  const int* blk_guard;   // guard fill / fold: 256 guard cells per block
  const int* blk_rows;    // window shift: 8 rows per block
  const int* shift;       // [n] this step's shift flags (device)
  int n;
};
struct BatchZeroSeg {     // words to clear: 4 per thread, 1024 per block
  void* p;
  long long words;
};
int batch_interior_blocks(const Layout& L);
int batch_guard_blocks(const Layout& L);
int batch_row_blocks(const Layout& L);
int batch_zero_blocks(long long words);
void batch_zero(const BatchZeroSeg* seg, const int* blk, int n, int nblk, cudaStream_t s);
void batch_fold(const BatchFieldTable& T, int nblk, cudaStream_t s);
void batch_fill(const BatchFieldTable& T, int nblk, cudaStream_t s);
void batch_yee_b(const BatchFieldTable& T, int nblk, cudaStream_t s);
void batch_yee_e(const BatchFieldTable& T, int nblk, cudaStream_t s);
void batch_shift(const BatchFieldTable& T, int nblk, cudaStream_t s);

// ----------------------------------------------------------------- particles
struct PushConst {        // per-species constants of one step
  double xmin[3], dx[3], inv_dx[3], dt;
  double e0[3], b0[3];
  double rqm, q, dvol;
  double L[3];            // box length per direction
  int isis;               // 1: ISIS deposit (2D3V), 0: TRISTAN / Villasenor-Buneman
  int cyl;                // 1: r-z mode (x2 = r, rings), 0: Cartesian
};

// FP64 plain form
struct Plain {
  double* x[3];
  double* u[3];
  int* id;
  double* w;              // charge weights (density profile); null: all 1
  long long n;
};
void plain_push(int ndim, const Layout& L, const PushConst& C, Plain p, double* const* f, double* const* j,
                int* status, cudaStream_t s);
void plain_rho(int ndim, const Layout& L, const PushConst& C, Plain p, double* rho, cudaStream_t s);
void plain_kinetic(const PushConst& C, Plain p, Diag64* acc, cudaStream_t s);

// FP32 cell-offset form, particles stored by tile
struct Part32 {           // one particle buffer (structure of arrays)
  uint32_t* cell;         // packed local cell lx | ly<<8 | lz<<16 | dir<<24
  float* o[3];            // in-cell offsets in [0,1)
  float* u[3];
  int* id;                // may be null
  float* w;               // charge weights (density profile); null: all 1
};
struct Flat32 {           // unsorted staging form (load, rebuild, copy-out)
  int* tile;
  uint32_t* cell;         // packed local cell within `tile`, dir = 13
  float* o[3];
  float* u[3];
  int* id;
  float* w;
};
struct Tiles {
  int ndim;
  int T[3];               // tile size in cells
  int nt[3];              // tiles per direction
  int ntiles;
  long long* base;        // [ntiles] first slot of each tile region
  int* cap;               // [ntiles] slots of each tile region
  int* res;               // [ntiles] slots at the back of each region kept for arrivals
  int small;              // 1: every region fits the small-tile kernel's stage
};
constexpr int DIR_STAY = 13;

// One side of the ping-pong particle store.  Region of tile t: slots
// [base[t], base[t] + cap[t]).  Its front holds the tile's stayers (stay[t]
// of them, sorted by cell in runs); its back holds the particles that entered
// the tile in the last step (inc[t] of them, at most res[t]), written there
// by the neighbouring tiles.
struct TileSide {
  Part32 p;
  int* stay;
  int* inc;
};

// Work items of the tile kernel beyond one per tile: a tile with more than
// kSliceChunks chunks of particles is split into slices that separate blocks
// take.  nslice[ntiles] counts each tile's slices; extra[cap] lists the
// (tile, slice >= 1) items, nextra[0] of them.
struct SliceScratch {
  int* nslice;
  int2* extra;
  int* nextra;
  int cap;
};
// capacity of the extra list for a particle store of `slots` slots in ntiles regions
long long slice_list_capacity(long long slots, int ntiles);

// stream = true: the step between re-sorts (stayers keep the order they were
// read in, compacted); false: the step that counting-sorts every tile by cell.
// Returns the number of kernels it launched.
int tiled_push(const Layout& L, const PushConst& C, const Tiles& tg, const TileSide& in, const TileSide& out,
                Flat32 spill, int* spill_count, long long spill_cap, int grid, int* work, const CUtensorMap* fmap,
                const CUtensorMap* jmap, int* status, bool stream, int minb, int shift_x, int* lost,
                const SliceScratch* slices, cudaStream_t s);
// moving window: `count` fresh particles of the front column appended to the
// last tile column of side `out` (global particle indices first, ...)
// A density profile on the device: per direction n[d] points (0: flat), at
// x[d][0..n-1] with values f[d][...]; the weight is the product of the
// piecewise-linear functions (constant beyond the ends), and no particle is
// created where density * weight is not above den_min.
struct ProfileDev {
  int n[3];
  const double* x[3];
  const double* f[3];
  double density, den_min;
};
// weight of the profile at position x (piecewise linear per direction,
// constant beyond the ends; product over the directions)
__device__ inline double profile_weight(const ProfileDev& P, const double x[3]) {
  double w = 1.0;
  for (int d = 0; d < 3; ++d) {
    const int n = P.n[d];
    if (n <= 0) continue;
    const double* xs = P.x[d];
    const double* fs = P.f[d];
    double f;
    if (x[d] <= xs[0]) {
      f = fs[0];
    } else if (x[d] >= xs[n - 1]) {
      f = fs[n - 1];
    } else {
      int lo = 0, hi = n - 1;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (xs[mid] <= x[d])
          lo = mid;
        else
          hi = mid;
      }
      const double slope = (fs[hi] - fs[lo]) / (xs[hi] - xs[lo]);
      f = slope * (x[d] - xs[lo]) + fs[lo];
    }
    w *= f;
  }
  return w;
}

// `kept`: count of the particles created (those the profile keeps)
void tiled_inject(const PushConst& C, const Tiles& tg, const TileSide& out, Flat32 spill, int* spill_count,
                  long long spill_cap, int* status, const int nx[3], const int ppc[3], const double uth[3],
                  const double ufl[3], unsigned long long seed, long long first, long long count,
                  const ProfileDev* prof, int* kept, cudaStream_t s);
// Batched form: many simulations (one table entry per simulation and species)
// in one launch of the sorting kernel.  tiled_fill_args writes one entry
// (tiled_args_bytes bytes) on the host; tile0[n] is the exclusive prefix of
// the entries' tile counts.  tiled_push_batch returns false for a tile shape
// the kernel is not built for.
size_t tiled_args_bytes();
// open_x, lost, shift_ptr: a member with a moving window (open x1, its count
// of dropped particles, its per-step shift flag in device memory); 0 / null
// otherwise
void tiled_fill_args(void* dst, const PushConst& C, const Tiles& tg, const TileSide& in, const TileSide& out,
                     Flat32 spill, int* spill_count, long long spill_cap, int* status, int open_x, int* lost,
                     const int* shift_ptr);
int tiled_batch_grid(int ndim, const int T[3], int total_tiles, int minb);
// Batched front-column injection (moving windows): one record per table entry
// (tiled_inject_spec_bytes bytes, written by tiled_fill_inject with the entry's
// member index and lattice count); entry e owns blocks [blk[e], blk[e + 1]) of
// 256 particles.  Per step, read on the device: shift[member], xlo0[member]
// (the window's lower x1 corner after the shift) and first[e] (global index of
// the entry's first fresh particle).  args: the entries' tile-kernel records
// of the step (their output side receives the particles).
size_t tiled_inject_spec_bytes();
void tiled_fill_inject(void* dst, const PushConst& C, const Tiles& tg, const int nx[3], const int ppc[3],
                       const double uth[3], const double ufl[3], unsigned long long seed, const ProfileDev* prof,
                       int* kept, int member, long long count);
void tiled_inject_batch(const void* args, const void* specs, const int* blk, int n, int nblk, const int* shift,
                        const double* xlo0, const long long* first, cudaStream_t s);
bool tiled_push_batch(int ndim, const int T[3], const void* args, const CUtensorMap* fmaps, const CUtensorMap* jmaps,
                      const int* tile0, int n, int* work, int grid, int minb, cudaStream_t s);
void tiled_live(const Tiles& tg, const TileSide& in, int* live, cudaStream_t s);
int tiled_push_smem_bytes(int ndim, const int T[3]);
int tiled_push_grid(int ndim, const int T[3], int ntiles, bool small, int minb);  // persistent CTAs
bool tiled_has_general(int ndim, const int T[3]);
bool tiled_has_small(int ndim, const int T[3]);
int tiled_small_capacity();  // largest tile region the small-tile kernel stages
void tiled_flatten(const Tiles& tg, const TileSide& in, const long long* out_off, Flat32 out, cudaStream_t s);
void flat_count(const Flat32& f, long long n, int ntiles, int* counts, cudaStream_t s);
void flat_scatter(const Flat32& f, long long n, const Tiles& tg, int* cursor, Part32 out, cudaStream_t s);
void flat_to_global(int ndim, const Tiles& tg, const PushConst& C, const Flat32& f, long long n, double* x, double* u,
                    cudaStream_t s);
void global_to_flat(int ndim, const Layout& L, const Tiles& tg, const PushConst& C, double* const x[3],
                    double* const u[3], const int* id, const double* w, long long n, Flat32 out, int* status,
                    cudaStream_t s);
// acc non-null: the kinetic energy and charge of the particles summed into it
// in the same pass
void tiled_rho(const Layout& L, const PushConst& C, const Tiles& tg, const TileSide& in, double* rho, Diag64* acc,
               cudaStream_t s);

// ----------------------------------------------------------------- r-z mode
// 2D cylindrically symmetric form (FP64 plain particles as rings: x[1] = r,
// r = -1 once absorbed at the wall; w = own weight * r at loading).  Field
// rows: node row j at r = (j - 1/2) dr, half rows at r = j dr, row 0 the
// mirror / axis row, row nr the conducting wall.
struct CylConst {
  int nz, nr;
  double dz, dr, dt;
  double rmax;  // (nr - 1/2) dr
};
// lattice: reflect r < 0 (first cell below the axis); explicit: r < 0 flags
// ST_BADCELL.  Then w = (has_w0 ? w : 1) * r.
void cyl_load_fix(long long n, double* r, double* w, bool lattice, bool has_w0, int* status, cudaStream_t s);
void cyl_push(const Layout& L, const PushConst& C, const CylConst& K, Plain p, double* const* f, double* const* j,
              int* status, cudaStream_t s);
// deposited current -> densities (guards and the mirror row folded, / V(r))
template <typename T> void cyl_current(const Layout& L, const CylConst& K, T* const* j, cudaStream_t s);
// axis / wall rows (and, with zguards, the periodic z guard columns)
template <typename T> void cyl_bound(const Layout& L, const CylConst& K, T* const* f, bool zguards, cudaStream_t s);
// B half step, E step, B half step with the boundary rows; returns launches
template <typename T>
int cyl_field_step(const Layout& L, const CylConst& K, T* const* f, T* const* j, cudaStream_t s);
// ring charges on the node rows (rho zeroed by the caller), then to density
void cyl_rho(const Layout& L, const PushConst& C, const CylConst& K, Plain p, double* rho, cudaStream_t s);
// (area: dz dr when rho holds charges, 1 when it holds charge per dz dr)
void cyl_rho_finish(const Layout& L, const CylConst& K, double* rho, double area, cudaStream_t s);
// field energy sum (per radian, not halved) and the Gauss maxima
template <typename T>
void cyl_diag(const Layout& L, const CylConst& K, T* const* f, const double* rho, double rho_bg, Diag64* acc,
              cudaStream_t s);
// kinetic energy and charge of the live rings (per radian)
void cyl_kinetic(const PushConst& C, Plain p, Diag64* acc, cudaStream_t s);

// ----------------------------------------------------------------- loading
// Lattice loader (nl_species num_par_x, vth, vfl) on the device, FP64 output.
struct LatticeSpec {
  int ndim;
  int nx[3];
  double xmin[3], dx[3];
  int ppc[3];
  double uth[3], ufl[3];
  unsigned long long seed;
};
void lattice_load(const LatticeSpec& S, long long first, long long count, double* const x[3], double* const u[3],
                  int* id, cudaStream_t s);
// Weights of `count` FP64 particles from the profile and the keep flags
// (density * weight > den_min); then the kept ones moved, in order, to
// dst (x, u, id, w) from index dst_first on.  Returns the number kept (syncs).
long long profile_compact(int ndim, const ProfileDev& P, long long count, double* const x[3], double* const u[3],
                          const int* id, double* const dx[3], double* const du[3], int* did, double* dw,
                          void* scratch, cudaStream_t s);
size_t profile_scratch_bytes(long long count);

// ----------------------------------------------------------------- sorting
// Exclusive prefix sum of n int32 counts into int64 starts; `scratch` holds at
// least scan_scratch_bytes(n) bytes.
size_t scan_scratch_bytes(long long n);
void exclusive_scan_i32(const int* in, long long* out, long long n, void* scratch, cudaStream_t s);

}  // namespace picgb
