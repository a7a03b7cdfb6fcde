/*
 * pic.h -- C ABI of libpicgb, the GB300 (sm_103a) electromagnetic particle-in-cell
 * hot path of Hemker's OSIRIS thesis (arxiv 1503.00276).
 *
 * One simulation step (thesis ch. 3, the PIC loop figure and the OSIRIS flow
 * chart, where gather, push and deposit form one combined particle algorithm):
 *   1. interpolate E^n, B^n linearly to every particle from each component's own
 *      staggered lattice (eq. "2d-field-weighting-e3", 3D extension);
 *   2. relativistic Boris push u^{n-1/2} -> u^{n+1/2} (eq. "momentum-update");
 *   3. position update x^{n+1} = x^n + dt u/gamma (eq. "2d-position-update");
 *   4. charge-conserving TRISTAN / Villasenor-Buneman current deposit from the
 *      straight path x^n -> x^{n+1}, split at cell faces (sect. "PIC Algorithms for
 *      2D-Cartesian Simulations"; 3D extension in sect. "3D-Cartesian ...");
 *   5. periodic wrap of particles and fold of current guard cells (appendix,
 *      nl_node_conf if_periodic);
 *   6. optional binomial smoothing of J (appendix, nl_smooth);
 *   7. field solve B -> B^{n+1/2} -> E^{n+1} -> B^{n+1}
 *      (eqs. "2d-field-solve-b-part1", "-e", "-b-part2" and the 3D extension).
 *
 * Units are the thesis' normalised units (appendix "Input File"): t in 1/w_p,
 * x in c/w_p, u = p/(m_e c), E and B in m_e c w_p / e, J in e n0 c, rho in e n0.
 * Every quantity crossing this ABI is in these units.
 *
 * Conventions for every function below:
 *  - Return value: PIC_OK or a negative pic_status; nothing aborts or exits.
 *    pic_last_error() gives a one-line message for the last failure.
 *  - Device work is enqueued on the CUDA stream passed to pic_init; functions that
 *    hand data to the host synchronise that stream.
 *  - Ownership: the library owns every device buffer it allocates (through the
 *    caller's pic_allocator, or cudaMalloc when that is NULL) and frees them in
 *    pic_destroy.  Caller arrays are only read or written during the call.
 *  - Calls on one handle are not thread-safe; distinct handles are independent.
 *  - Grid arrays crossing the ABI are dense [nz][ny][nx] (x1 fastest; nz = 1 in
 *    2D) without guard cells.  Array index (i,j,k) of a component sits at
 *    xmin + ((i,j,k) + stagger) * dx with the Yee staggering read off the
 *    difference stencils of the field equations:
 *      E1 (1/2,0,0)  E2 (0,1/2,0)  E3 (0,0,1/2)  B1 (0,1/2,1/2)  B2 (1/2,0,1/2)
 *      B3 (1/2,1/2,0)  J like E  rho at the nodes (0,0,0)   (x3 entry dropped in 2D).
 */
#ifndef PICGB_PIC_H
#define PICGB_PIC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PIC_OK = 0,
  PIC_EINVAL = -1,        /* bad argument or unsupported combination */
  PIC_ENOMEM = -2,        /* device allocation failed */
  PIC_ECUDA = -3,         /* a CUDA call failed (message in pic_last_error) */
  PIC_ECOURANT = -4,      /* dt >= 1/sqrt(sum dx_d^-2): the Courant condition
                             c dt < dx (sect. on moving boundaries), multi-D form */
  PIC_EOVERFLOW = -5,     /* particle storage exhausted (np_max, appendix nl_species) */
  PIC_ENONFINITE = -6,    /* a NaN or Inf appeared in particles or fields */
  PIC_ETIMEOUT = -7,      /* a bounded device-side wait gave up */
  PIC_EUNSUPPORTED = -8,  /* valid request that this build does not implement */
  PIC_ENOTBUILT = -9      /* the library was built without a GPU code path */
} pic_status;

/* Numerical form of the particle data and of the whole step. */
typedef enum {
  /* Reference form: global FP64 positions, FP64 momenta, FP64 fields and
   * current, gather from global memory, deposit with FP64 global atomics. */
  PIC_FP64_PLAIN = 0,
  /* Fast form: int32 cell index within a tile + FP32 in-cell offsets in [0,1),
   * FP32 momenta and fields; particles stored by tile; each tile's E/B stencil
   * staged in shared memory by TMA and its current accumulated in shared memory
   * before one TMA reduce-add into HBM. */
  PIC_FP32_CELLOFF = 1
} pic_precision;

/* Boundary types (appendix nl_emf_bound / nl_spe_bound).  This build
 * implements periodic boundaries (nl_node_conf if_periodic) only. */
/* boundary types (appendix nl_emf_bound): periodic; 5 = conducting boundary
 * with particle absorption and 20 = axial boundary, the two r boundaries of
 * the 2D cylindrically symmetric mode (lower r: 20, upper r: 5) */
enum { PIC_BC_PERIODIC = 0, PIC_BC_CONDUCT_ABSORB = 5, PIC_BC_AXIAL = 20 };

/* Field selectors for pic_fields / pic_set_field. */
enum { PIC_E1 = 0, PIC_E2, PIC_E3, PIC_B1, PIC_B2, PIC_B3, PIC_J1, PIC_J2, PIC_J3, PIC_RHO };

#define PIC_MAX_SMOOTH 8

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns a device pointer aligned to at least 256 bytes, or NULL on failure;
 * free releases it.  ctx is passed back unchanged. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes);
  void (*free)(void* ctx, void* ptr, size_t bytes);
} pic_allocator;

/* Grid, time step, fields and numerical options
 * (appendix sections nl_grid, nl_space, nl_time_step, nl_el_mag_fld, nl_smooth). */
typedef struct {
  int ndim;                 /* 2 (2D3V: x1,x2 in the plane, three u components) or 3 */
  int nx[3];                /* cells per direction (nx_p); nx[2] ignored in 2D */
  double xmin[3];           /* lower corner of the box (nl_space xmin) */
  double dx[3];             /* cell size */
  double dt;                /* time step; must satisfy dt < 1/sqrt(sum_d dx_d^-2) */
  int bc[3][2];             /* boundary type per direction and side: PIC_BC_PERIODIC; in the
                               r-z mode bc[1] = {PIC_BC_AXIAL, PIC_BC_CONDUCT_ABSORB} */
  double e0[3], b0[3];      /* constant external fields added at the gather (nl_el_mag_fld) */
  int smooth_level[3];      /* smoothing passes of J per direction (0 = off) */
  double smooth_w[3][PIC_MAX_SMOOTH][3];  /* weights (swfj) per direction and pass;
                                             each pass is normalised by the weight sum */
  double rho_bg;            /* fixed neutralising background charge density */
  int init_e_gauss_x1;      /* 1: set the initial E1 from the discrete Gauss law
                               along x1, column by column (exact for charge
                               densities that vary only along x1); 0: E = 0 */
  pic_precision precision;
  int tile[3];              /* PIC_FP32_CELLOFF tile size in cells (0 = default:
                               2D 32x16, 3D 8x8x8); nx must be a multiple */
  double slack;             /* per-tile storage slack fraction (0 = default: 0.25, or
                               0.75 with a moving window) */
  int sort_period;          /* PIC_FP32_CELLOFF: every sort_period-th step re-sorts each
                               tile by cell; the steps between update particles in
                               place (0 = default 1: sort every step) */
  int ctas_per_sm;          /* PIC_FP32_CELLOFF: thread blocks per SM the general tile
                               kernel is built for: 4 (64 registers per thread) or 2
                               (128); 0 = default 4 */
  int move_window;          /* 1: the window moves at c in +x1 (thesis: dynamic simulation
                               space, if_move): x1 is open -- fields beyond it are 0, particles
                               leaving through it are dropped -- and whenever c t runs a full
                               cell ahead of the window, every field value and particle moves
                               one cell back, the back column is discarded and the front column
                               gets zero fields and fresh plasma of every species (its lattice,
                               u_th, u_fl and draw stream continued; explicit species need
                               ppc set).  PIC_FP32_CELLOFF only (else PIC_EUNSUPPORTED). */
  int deposit;              /* current deposit (thesis ch. 3, "ISIS or TRISTAN methods"):
                               PIC_DEPOSIT_TRISTAN (0, default; Villasenor-Buneman: the path
                               is split at cell faces and each piece is the average of its
                               orthogonal-move orders) or PIC_DEPOSIT_ISIS (1; the average of
                               the two orders of orthogonal moves of the whole path, not
                               split; 2D3V only, else PIC_EUNSUPPORTED).  Both conserve
                               charge exactly; they differ by a divergence-free current. */
  double window_start;      /* move_window: time from which the window moves (before it
                               the box is still, x1 open); 0 = from the start */
  int coords;               /* PIC_COORDS_CARTESIAN (0, default) or PIC_COORDS_CYLINDRICAL (1):
                               the 2D cylindrically symmetric mode (thesis ch. 3).  x1 = z
                               (periodic), x2 = r with the axis through the middle of the first
                               cell (xmin[1] must be -dx[1]/2) and a perfectly conducting wall at
                               r = (nx[1] - 1/2) dx[1]; E1,E2,E3 are Ez,Er,Etheta (B, J likewise).
                               The field solve weights the r-derivatives of the z components by
                               the radius and advances Bz on the axis from Faraday's law on the
                               disc of radius dx[1]/2; field rows at the axis follow the axial
                               parity.  Particles are rings: x2 = r >= 0, u = (pz, pr, ptheta),
                               charge q * w * r per radian (w the own weight, 1 without one),
                               moved in 3D and rotated back into the r-z plane; lattice points
                               below the axis are reflected; a particle reaching the wall is
                               absorbed (PIC_FP64_PLAIN: its slot stays, with r = -1 and u = 0;
                               PIC_FP32_CELLOFF: it is removed).  J and RHO are densities
                               (current or charge per r dr dz); pic_diag totals are over the full
                               2 pi.  Needs ndim 2 and the TRISTAN deposit, no smoothing,
                               move_window, init_e_gauss_x1 or density profile, no laser, not in a
                               batch (else PIC_EUNSUPPORTED); bc[1] must be {PIC_BC_AXIAL,
                               PIC_BC_CONDUCT_ABSORB} (else PIC_EINVAL).
                               Time step: dt < 1/sqrt(1/dx1^2 + 1.2105/dx2^2) (PIC_ECOURANT), the
                               radial factor being the largest eigenvalue of the discrete radial
                               operator with the axis rule, in units of 4/dx2^2. */
} pic_grid;

enum { PIC_DEPOSIT_TRISTAN = 0, PIC_DEPOSIT_ISIS = 1 };
enum { PIC_COORDS_CARTESIAN = 0, PIC_COORDS_CYLINDRICAL = 1 };

/* One particle species (appendix nl_species / nl_profile).  Either loaded on the
 * device from the num_par_x lattice and a seed, or given explicitly. */
typedef struct {
  double rqm;               /* m/q in units of m_e/e (electrons: -1) */
  int ppc[3];               /* num_par_x: particles per cell direction (lattice) */
  double uth[3];            /* vth: standard deviation of each u component */
  double ufl[3];            /* vfl: fluid momentum */
  double density;           /* uniform density in units of n0 (macroparticle charge
                               q = sign(1/rqm) * density * cell volume / ppc) */
  unsigned long long seed;  /* SplitMix64 stream for the thermal momenta */
  /* Explicit particles instead of the lattice (n_explicit > 0): host arrays of
   * n_explicit rows [x1 x2 x3] (global positions, x3 ignored in 2D) and
   * [u1 u2 u3], FP64, copied during pic_init; every position must lie in the
   * periodic box [xmin, xmin + nx dx) (else PIC_EINVAL).  q_explicit is the
   * charge per macroparticle (0: density times the cell volume). */
  long long n_explicit;
  const double* x0;
  const double* u0;
  double q_explicit;
  long long np_max;         /* storage limit in particles (0 = no limit) */
  int track_ids;            /* 1: keep an int32 particle id (lattice index or explicit
                               row) alongside each particle, for pic_particle_ids */
  /* Density profile (nl_num_x / nl_profile), lattice species only: per
   * direction prof_n[d] points (0 = flat) at prof_x[d][0..n-1] (ascending) with
   * values prof_f[d][...]; the density is `density` times the product of the
   * piecewise-linear functions (constant beyond the end points).  Each
   * particle's charge is q times the profile at its initial position (for a
   * moving window, at the lab-frame position where it is injected); no
   * particle is created where density times the profile is not above den_min.
   * Host arrays, copied during pic_init. */
  int prof_n[3];
  const double* prof_x[3];
  const double* prof_f[3];
  double den_min;
  const double* w0;         /* explicit species: per-particle charge weights (n_explicit
                               values; NULL = all 1) */
} pic_species;

typedef struct pic_sim pic_sim;   /* opaque; owns all device state */

typedef struct {
  long long step;           /* steps taken */
  double time;              /* step * dt */
  double field_energy;      /* (1/2) sum over grid values of (E^2 + B^2) * cell volume */
  double kinetic_energy;    /* sum over particles of q*rqm*(gamma - 1), u at the last half step */
  double total_charge;      /* sum of macroparticle charges (background excluded) */
  double gauss_resid_max;   /* max over nodes |div E - rho - rho_bg|, backward differences */
  double rho_abs_max;       /* max over nodes |rho + rho_bg| */
  double rho_particles_abs_max; /* max over nodes |rho| of the particles alone */
  long long n_particles;
  int error_flags;          /* bit 0: non-finite value seen; bit 1: tile storage spill */
} pic_diag_t;

/* Create a simulation (thesis: global -> local object set-up).  Validates the
 * Courant condition (PIC_ECOURANT), sizes and tile divisibility (PIC_EINVAL),
 * allocates every device buffer, loads the particles and sets the initial fields
 * (zero, or Gauss-consistent E1 when init_e_gauss_x1).  `stream` is a
 * cudaStream_t (NULL = the legacy default stream).  On failure *out is NULL and
 * nothing is leaked. */
pic_status pic_init(const pic_grid* grid, const pic_species* species, int nspecies,
                    const pic_allocator* alloc, void* stream, pic_sim** out);

/* Advance nsteps full steps (the seven stages in the header comment).  Returns
 * after the work is enqueued and the per-step device status has been checked;
 * PIC_ENONFINITE if a NaN/Inf was flagged. */
pic_status pic_step(pic_sim* sim, int nsteps);

/* The grid data dumps of the thesis' diagnostics (appendix, input blocks
 * nl_diag_emf for the full E and B data and nl_diag_phy_field for the current
 * and the charge density), returned to the caller instead of written to files.
 * Copy one grid quantity (PIC_E1 .. PIC_RHO) as a dense FP64 [nz][ny][nx] array
 * into dst (dst_bytes >= 8 * cells; device pointer if dst_on_device), each
 * component at its own staggered position (ch. 3, Yee grid).  J is the
 * (folded, smoothed) current of the last step; RHO is computed on demand from the
 * current particle positions with the linear weights, background excluded.
 * Errors: PIC_EINVAL (null sim or dst, which out of range, dst_bytes too
 * small); PIC_ECUDA.  Synchronises the stream. */
pic_status pic_fields(pic_sim* sim, int which, void* dst, size_t dst_bytes, int dst_on_device);

/* Overwrite one field component (PIC_E1 .. PIC_B3) from a dense FP64
 * [nz][ny][nx] array (device pointer if src_on_device). */
pic_status pic_set_field(pic_sim* sim, int which, const void* src, size_t src_bytes, int src_on_device);

/* The particle data dumps of the thesis' diagnostics (appendix, input block
 * nl_diag_particles: each particle's position and momentum), without the
 * gamma filter, returned to the caller.  Copy the particles of one species as
 * global FP64 positions x[n][3] (x in c/w_p; 2D: x[.][2] = 0; r-z: (z, r, 0))
 * and momenta u[n][3] = p/(m_e c) (either pointer may be NULL).  cap is the
 * row capacity of the destination; *n_out receives the particle count
 * (PIC_EOVERFLOW when it exceeds cap, nothing copied).  Rows come in the
 * library's storage order (pic_particle_ids gives the matching ids).
 * Errors: PIC_EINVAL (null sim or n_out, species out of range); PIC_ECUDA.
 * Synchronises the stream. */
pic_status pic_particles(pic_sim* sim, int species, double* x, double* u, long long cap,
                         long long* n_out, int dst_on_device);

/* Particle ids (species with track_ids) in the same order as pic_particles. */
pic_status pic_particle_ids(pic_sim* sim, int species, int* ids, long long cap, long long* n_out,
                            int dst_on_device);

/* Charge weights of a species' particles (1 without a profile or explicit
 * weights), in the order of pic_particles / pic_particle_ids; same arguments
 * and errors as pic_particle_ids. */
pic_status pic_particle_weights(pic_sim* S, int species, double* w, long long cap, long long* n_out,
                                int dst_on_device);

/* Number of tiles of the PIC_FP32_CELLOFF store and the particle count of each
 * (tiles in x1-fastest order), host array of ntiles entries. */
pic_status pic_tile_counts(pic_sim* sim, int species, long long* counts, long long cap,
                           long long* ntiles_out);

/* Global numbers of the state, reduced in FP64 on the device: the residual
 * of Gauss's law (ch. 3, Maxwell's equations, eq. maxwell-1: div E = 4 pi rho,
 * div E = rho in normalised units) as max |div E - rho - rho_bg| over nodes
 * with div E from the backward differences of the staggered E; the field
 * energy (1/2) sum (E^2 + B^2) dV; the particles' kinetic energy
 * sum |q| |rqm| (gamma - 1); their total charge and count; the largest |rho|
 * (net, and of the particles alone).  These condense what the thesis'
 * diagnostics dump (appendix, nl_diag_* blocks) into the checks that the
 * scheme conserves charge and energy.  Synchronises the stream.  Errors:
 * PIC_EINVAL (null arguments); PIC_ECUDA. */
pic_status pic_diag(pic_sim* sim, pic_diag_t* out);

/* Per-stage device time accumulated with CUDA events on the simulation's stream
 * while timing is enabled.  Slots: 0 particle kernel (gather+push+deposit),
 * 1 current fold/smoothing, 2 field solve, 3 tile rebuilds, 4 whole steps;
 * pic_timing_read returns milliseconds and the number of timed spans per slot
 * since the last reset.  Slot 5 (when nslots > 5) counts every kernel that
 * pic_step launched since the last reset, timing enabled or not (ms[5] = 0). */
pic_status pic_timing_enable(pic_sim* sim, int enable);
pic_status pic_timing_read(pic_sim* sim, double* ms, long long* launches, int nslots, int reset);

/* End of a run (the end of the thesis' main loop, ch. 4, high level
 * description and flow chart): release every device buffer, stream event and
 * table the simulation owns (through the allocator it was created with).
 * NULL is accepted.  sim must not be used afterwards; a borrowed batch member
 * (pic_batch_sim) must not be passed. */
pic_status pic_destroy(pic_sim* sim);

/* Message of the last failure on this thread (never NULL; "no error" before
 * the first one).  The thesis' code reports failures of its input and run
 * phases by messages; here every call returns a pic_status and leaves the
 * message here, valid until the next failing call on the same thread. */
const char* pic_last_error(void);

/* Stateless tile binning (not in the thesis: the supporting per-tile sort;
 * the thesis keeps each node's particles in one unsorted array, appendix
 * nl_species num_par_max).
 * For n particles with integer cell coordinates cell[n][3] (device, int32,
 * each in [0, nx_d)), computes the tile of each particle
 * t = ((c3/T3)*nt2 + c2/T2)*nt1 + c1/T1 (nt_d = nx_d/T_d), the count of every
 * tile (tile_count[ntiles], device int32), the exclusive prefix sum of the counts
 * (tile_start[ntiles], device int64) and a permutation perm[n] (device int64)
 * that lists particles tile by tile, in increasing particle index within each
 * tile (a stable sort by tile: the result is unique and does not depend on
 * scheduling).  n must be below 2^31.  Scratch memory (about 5 bytes per
 * particle, 9 with more than 255 tiles, 13 with more than 65535) comes from
 * `alloc` (NULL = cudaMalloc) and is released before returning.  `stream` is a
 * cudaStream_t.  In 2D pass nx[2] = tile[2] = 1 and cell[.][2] = 0.  A cell
 * outside [0, nx) returns PIC_EINVAL (the outputs are then unspecified). */
pic_status pic_bin_tiles(const int nx[3], const int tile[3], long long n, const int* cell,
                         int* tile_count, long long* tile_start, long long* perm,
                         const pic_allocator* alloc, void* stream);

/* Bytes of the fixed device scratch behind pic_bin_tiles_noalloc. */
#define PIC_BIN_NOALLOC_SCRATCH_BYTES (16u << 20)

/* pic_bin_tiles without any device allocation (the thesis has no counterpart;
 * this entry point exists for callers).  Some callers cannot call cudaMalloc
 * or take an allocator callback: code that runs where allocation is forbidden
 * or unsafe -- inside a framework that owns every byte of device memory through
 * its own pool and accounting, in latency-critical paths where a cudaMalloc or
 * cudaFree (which may synchronise the device) is not allowed, or where an
 * allocation failure mid-run cannot be handled.  They get the same result as
 * pic_bin_tiles (same arguments, same output: particles tile by tile, in
 * increasing particle index within each tile) with the scratch taken from a
 * fixed array compiled into the library:
 *  - its size is PIC_BIN_NOALLOC_SCRATCH_BYTES (16 MiB), reserved on every GPU
 *    that loads the library until the process exits;
 *  - the scratch a call needs is about 5 bytes per particle with up to 255
 *    tiles, 9 with up to 65535 and 13 beyond (e.g. 1.8 million particles on
 *    32 thousand tiles take 15 MiB); requests needing more than the array
 *    return PIC_EINVAL with a message, and nothing runs;
 *  - the first call in a CUDA context (the device current) looks the array's
 *    device address up with cudaGetSymbolAddress and keeps it for that
 *    context (a device reset makes a new context, which looks it up again);
 *    make that first call before any stream capture;
 *  - every call in one process shares the array on a device (each process has
 *    its own copy of the library's device memory) and the function clears
 *    what must start at zero, so calls whose GPU work overlaps (different
 *    streams or threads of one process on one device) race and must be
 *    serialised by the caller;
 *  - like pic_bin_tiles it synchronises `stream` before returning.
 * It calls no cudaMalloc, cudaFree or other allocating routine. */
pic_status pic_bin_tiles_noalloc(const int nx[3], const int tile[3], long long n, const int* cell,
                                 int* tile_count, long long* tile_start, long long* perm, void* stream);


/* ---- Batched parameter scan ------------------------------------------------
 * The thesis runs one simulation at a time; a parameter scan (many independent
 * 2D/3D runs of uneven grid sizes and particle counts) is advanced here as one
 * batch, so that small runs share the GPU instead of each leaving most SMs
 * idle.  Every step of every member is the same step pic_step takes (gather,
 * Boris push, move and Villasenor-Buneman deposit of section 2.2, current fold,
 * smoothing and Yee solve of section 2.1), but the particle step of all members
 * is ONE launch of the persistent sorting tile kernel, whose work items are the
 * tiles of all members, each stage of the field step (current fold, the two
 * B half steps and the E step, guard cells, window shift) is one launch over
 * all members, and the whole step of the batch is one CUDA graph launch
 * (captured once per store side; re-captured after a member re-bins or gains
 * an antenna pulse).
 */
typedef struct pic_batch pic_batch;

/* nsims simulations: grids[i] with species[i*nspecies .. i*nspecies+nspecies-1].
 * Every grid must be PIC_FP32_CELLOFF with the same ndim and the same tile
 * field; tile {0,0,0} picks the first shape that divides every grid (3D 8x8x8,
 * 16x8x4; 2D 32x16, 16x16, 8x8).  sort_period is forced to 1.  Device memory
 * comes from `alloc` (NULL: cudaMalloc); all work is enqueued on `stream`.
 * Members may have a moving window (move_window, open x1, front injection,
 * lasers and antennas added through their pic_batch_sim handles): each
 * shifts on its own steps, exactly as pic_step would move it.  The values that
 * change from step to step (shift flags, window corners, antenna times, first
 * indices of fresh particles) are written on the host before each step into a
 * pinned block that the step's first node copies to the device, so the same
 * graph serves every step.
 * Errors: PIC_EINVAL for mismatched grids (message names the member),
 * PIC_EUNSUPPORTED for an r-z member (the batched step has no r-z solve),
 * PIC_ENOMEM, PIC_ECUDA, plus every error pic_init reports for a member. */
pic_status pic_batch_init(int nsims, const pic_grid* grids, const pic_species* species, int nspecies,
                          const pic_allocator* alloc, void* stream, pic_batch** out);

/* Advance every member nsteps steps.  After each step the members' device
 * status words are read back once (one synchronisation per step): a member
 * whose tile storage spilled is re-binned before the next step; PIC_ETIMEOUT /
 * PIC_ENONFINITE / PIC_EOVERFLOW name the member. */
pic_status pic_batch_step(pic_batch* B, int nsteps);

/* Borrowed handle of member i for pic_fields, pic_particles, pic_particle_ids,
 * pic_tile_counts and pic_diag.  pic_step and pic_destroy must not be called on
 * it (pic_step returns PIC_EINVAL); it lives until pic_batch_destroy. */
pic_status pic_batch_sim(pic_batch* B, int i, pic_sim** out);

/* Steps taken, kernel launches enqueued by pic_batch_step (every graph node
 * that is a kernel), and the tile shape in use; any pointer may be NULL. */
pic_status pic_batch_info(const pic_batch* B, long long* steps, long long* launches, int tile[3]);

/* Frees every member and the batch; synchronises its stream first. */
pic_status pic_batch_destroy(pic_batch* B);


/* ---- Autotuner --------------------------------------------------------------
 * Chooses the launch parameters of the FP32 particle step by running them: the
 * tile shape (3D 8x8x8, 16x8x4, 8x4x4, 4x4x4, 4x4x2; 2D 32x16, 16x16, 8x8,
 * 16x8, 8x4 -- those dividing every grid), the thread blocks per SM of the
 * general tile kernel (4 or 2: its particles in flight per SM), and the sort
 * period (1 or 4).  Each candidate is set up from the same grid/species,
 * stepped `warmup` steps, then `steps` steps are timed with CUDA events on
 * `stream`; the candidate is freed before the next.  The thesis tunes nothing
 * of this kind (its particle loop runs on CPUs).
 * best: the fastest candidate; tried[0 .. min(max_tried, *n_tried) - 1]: every
 * candidate with its time (ms_per_step < 0: it could not run, e.g. no memory).
 * PIC_EINVAL for bad arguments or grids no shape divides; PIC_ECUDA if no
 * candidate ran. */
typedef struct {
  int tile[3];
  int ctas_per_sm;
  int sort_period;
  double ms_per_step;
} pic_tune_choice;

pic_status pic_autotune(const pic_grid* grid, const pic_species* species, int nspecies, const pic_allocator* alloc,
                        void* stream, int warmup, int steps, pic_tune_choice* best, pic_tune_choice* tried,
                        int max_tried, int* n_tried);

/* The same for a batch (pic_batch_init arguments): general tile shapes that
 * divide every member's grid, 4 or 2 blocks per SM, sort period 1; each
 * candidate is a whole batch. */
pic_status pic_batch_autotune(int nsims, const pic_grid* grids, const pic_species* species, int nspecies,
                              const pic_allocator* alloc, void* stream, int warmup, int steps, pic_tune_choice* best,
                              pic_tune_choice* tried, int max_tried, int* n_tried);


/* ---- Checkpoint / restart ---------------------------------------------------
 * The restart files of the thesis' code (its restart section: dump the full
 * state every n steps, resume from it) for this library's state.
 * pic_checkpoint_save writes one self-describing binary file: magic
 * "PICGBCK1", version, sizeof(pic_grid), the effective grid (tile shape, sort
 * period, blocks per SM and slack as in use), the step count, then per species
 * its macro-charge, rqm, count and id flag followed by its particles in the
 * stored precision (FP32 form: tile index, packed cell, 3 offsets, 3 momenta,
 * ids; FP64 form: positions, momenta, ids), then the six E/B planes as stored
 * (guard cells included), then the table of pulses driven through the lower
 * x1 boundary (pic_laser.antenna; lab-frame records).  A moving window's
 * state travels in the effective grid (x1 origin after its shifts), the step
 * and shift counts and each species' count of injected lattice places, so a
 * restored window keeps shifting, injecting and driving its pulses as the
 * uninterrupted run would.  The current and charge are not stored: the next
 * step recomputes them.  It synchronises S's stream and streams through a
 * 64 MiB host buffer.  Errors: PIC_EINVAL (bad arguments, file cannot be
 * written), PIC_ENOMEM, PIC_ECUDA.
 * pic_checkpoint_load creates a new simulation from such a file (on `stream`,
 * memory from `alloc`): the restored particles, fields and step count are the
 * saved ones bit for bit (the order of particles within a tile may differ).
 * Errors: PIC_EINVAL for a missing, truncated or foreign file (nothing is
 * allocated), plus those of pic_init. */
pic_status pic_checkpoint_save(pic_sim* S, const char* path);
pic_status pic_checkpoint_load(const char* path, const pic_allocator* alloc, void* cuda_stream, pic_sim** out);

/* The effective grid of S (tile shape etc. as in use), its species count and
 * step count; any output pointer may be NULL. */
pic_status pic_info(const pic_sim* S, pic_grid* grid, int* nspecies, long long* step);


/* ---- Laser pulses ------------------------------------------------------------
 * A pulse added to the current fields (the thesis' pulse input): wavetype 1
 * (or 0) moves in +x1, wavetype 2 in +x2.  vosc = peak normalised vector
 * potential a0; rkkp = its wavenumber k (= omega0 / omega_p); w0 = spot size
 * (field 1/e radius in the focal plane); rise / length / fall = envelope
 * distances behind the front (rise 10 s^3 - 15 s^4 + 6 s^5 with s the
 * fraction of the rise, flat, then the mirror image -- the thesis' temporal
 * profile); start = distance of the front from the side of the box the pulse
 * moves towards; pol = polarisation angle in degrees from the in-plane
 * transverse axis (x2 for wavetype 1, x1 for wavetype 2) towards x3; phase;
 * offset = transverse offset of the axis from the box centre (in-plane axis,
 * x3).  focus_on: 1 = the lowest Hermite-Gaussian beam of the thesis' laser-beam
 * section with its focal plane at distance `focus` from that same side (spot
 * size w0 sqrt(1 + (z/z_R)^2), curvature and Gouy phase; 2D: slab beam with
 * amplitude sqrt(w0 / w) and half the Gouy phase); 0 = waist profile w0
 * everywhere.  A along the polarisation gives E = -dA/dt and B = e_k x E in
 * the slowly varying envelope form, each component at its own staggered
 * position.  The thesis' `time` is the step at which the caller adds the
 * pulse.  Synchronises S's stream. */
typedef struct {
  double vosc, rkkp, w0, rise, fall, length, start, pol, phase;
  double offset[2];
  int wavetype;             /* 1 (or 0): along x1; 2: along x2 */
  int focus_on;
  double focus;
  int antenna;              /* 1: the pulse enters through the lower x1 boundary instead
                               of being set up in the box (move_window simulations, whose
                               x1 is open; wavetype 1): below that boundary the E update
                               reads the pulse's B, its front crossing the boundary at time
                               `start`; `focus` is then measured into the box from that
                               boundary.  Every later pic_step drives it (not stored in
                               checkpoints). */
} pic_laser;

pic_status pic_laser_add(pic_sim* S, const pic_laser* laser);

#ifdef __cplusplus
}
#endif

#endif /* PICGB_PIC_H */
