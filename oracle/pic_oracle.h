/*
 * pic_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure only;
 * see pic_oracle.c).  This header belongs to the oracle alone: the CUDA library
 * neither includes it nor shares any of its types.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#define ORA_MAX_PASS 8

typedef struct {
  int ndim;                              /* 2 (2D3V) or 3 */
  int nx[3];                             /* cells per direction, nx[2] = 1 in 2D */
  double dx[3];
  double xmin[3];
  double dt;
  double e0[3];                          /* constant external fields */
  double b0[3];
  int smooth_level[3];                   /* passes per direction */
  double smooth_w[3][ORA_MAX_PASS][3];   /* weights per direction and pass */
  double rho_bg;                         /* fixed background charge density */
  int open_x1;                           /* 1: x1 is open (moving window): values beyond
                                            x1 read as 0, deposits there are dropped,
                                            particles are not wrapped in x1 */
  int isis;                              /* 1: ISIS current deposit (2D3V) instead of
                                            TRISTAN / Villasenor-Buneman */
  /* open x1: B2 and B3 just below the lower x1 boundary ([nz][ny], at
     x1 = xmin - dx1/2 and time n + 1/2), read by the E update there instead
     of 0 -- a pulse entering through that boundary; NULL: 0 */
  const double* inc_b2;
  const double* inc_b3;
} ora_grid;

typedef struct {
  double rqm;        /* m/q */
  double q;          /* charge per macroparticle */
  long long n;
  double* x;         /* [n][3] global positions */
  double* u;         /* [n][3] momenta p/(m c) */
  const double* w;   /* [n] charge weights (density profile), NULL: all 1;
                        particle p carries charge q w[p] */
} ora_species;

void ora_gather(const ora_grid* g, double* const fld[6], const double x[3], double eb[6]);
void ora_boris(double u[3], const double e[3], const double b[3], double rqm, double dt);
double ora_gamma(const double u[3]);
void ora_move(const ora_grid* g, double x[3], const double u[3]);
void ora_wrap(const ora_grid* g, double x[3]);
void ora_deposit_vb(const ora_grid* g, double* cur[3], const double xold[3], const double xnew[3], double v3,
                    double q);
void ora_deposit_isis(const ora_grid* g, double* cur[3], const double xold[3], const double xnew[3], double v3,
                      double q);
void ora_deposit_rho(const ora_grid* g, double* rho, const double* x, long long n, double q);
void ora_deposit_rho_w(const ora_grid* g, double* rho, const double* x, const double* w, long long n, double q);
void ora_smooth(const ora_grid* g, double* f);
void ora_field_solve(const ora_grid* g, double* const fld[6], double* const cur[3]);
void ora_advance_particle(const ora_grid* g, double* const fld[6], double rqm, double x[3], double u[3]);
void ora_advance_particles(const ora_grid* g, double* const fld[6], double rqm, long long n, double* x,
                           double* u, int wrap);
void ora_particle_phase(const ora_grid* g, double* const fld[6], double* cur[3], const ora_species* sp, int nsp);
void ora_step(const ora_grid* g, double* const fld[6], double* cur[3], const ora_species* sp, int nsp,
              int nsteps);
void ora_rho(const ora_grid* g, const ora_species* sp, int nsp, double* rho);
double ora_gauss_residual(const ora_grid* g, double* const fld[6], const double* rho);
double ora_field_energy(const ora_grid* g, double* const fld[6]);
double ora_kinetic_energy(const ora_species* sp, int nsp);
void ora_init_e_gauss_x1(const ora_grid* g, const double* rho, double* E1);
void ora_tile_bin(const ora_grid* g, const int tile[3], long long n, const double* x, long long* tile_id,
                  long long* counts, long long* order);

#endif
