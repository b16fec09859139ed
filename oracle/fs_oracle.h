/*
 * fs_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, single-threaded FP64 CPU implementation of the faux-shock hybrid
 * particle-in-cell step (Simon, Caprioli, Haggerty & Reville, "A 'Faux-Shock'
 * Method for Hybrid Simulations of Astrophysical Shocks", Sec. 2, Eq. 1).
 * It exists to check the CUDA path; only tests/, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header,
 * constant table or helper with the CUDA library.
 *
 * Normalised units (Sec. 2): x in d_i, t in 1/Omega_ci, v in v_A, B in B0,
 * n in n_g, E in v_A B0 / c, energy in m v_A^2, ion q/m = 1.
 * Canonical frame (Sec. 2): the faux shock sits at x = 0, plasma enters at
 * x = L and drifts in -x at u_sh = M_A.
 */
#ifndef FS_ORACLE_H
#define FS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BC_FAUXSHOCK = 0, OR_BC_PERIODIC = 1 };
enum { OR_FS_OPEN = 0, OR_FS_SHOCK = 1 };
enum { OR_FRAME_SHOCK = 0, OR_FRAME_DOWNSTREAM = 1 };

typedef struct {
  int dim, nx, ny;            /* dim 1: ny must be 1 */
  double dx, dy, dt;
  double mach_a;              /* u_sh / v_A in the shock (simulation) frame */
  double theta_bn_deg;        /* B0 = (cos, sin, 0) */
  double beta_i, beta_e;      /* T_i = beta_i / 2, T_e = beta_e / 2 */
  int ppc;                    /* thermal macroparticles per cell */
  int bc_x;                   /* OR_BC_FAUXSHOCK or OR_BC_PERIODIC */
  int fs_mode_thermal;        /* OR_FS_OPEN (paper) or OR_FS_SHOCK */
  int fs_speed_frame;         /* speed used in Eq. 1 */
  double r_comp;              /* compression ratio r */
  double u2;                  /* downstream speed; <= 0 -> mach_a / r_comp */
  int inject_thermal;         /* inflow at x = L (faux-shock box only) */
  int cr_enable;              /* cosmic-ray source at the faux shock */
  double n_cr_ratio, p_iso, u_cr; /* u_cr <= 0 -> u2 */
  int n_sub;                  /* RK4 substeps per particle step */
  double n_floor, eta;
  double j_cr_ext;            /* prescribed uniform x-current (Bell test) */
  int init_plasma;            /* load the uniform drifting plasma at t = 0 */
  uint64_t seed;
  int hist_nx, hist_np;       /* x-p_x histogram shape */
  double hist_pmin, hist_pmax;
  double c_light;             /* c / v_A; 0: non-relativistic ions. With c > 0
                                 the stored velocity is u = gamma v (momentum
                                 per mass), as in the relativistic dHybridR */
  int spec_np;                /* momentum spectrum n(p): log bins of |u| */
  double spec_pmin, spec_pmax;
} or_params;

typedef struct {
  long long step, n_particles, next_id;
  long long incident, transmitted, reflected, escaped, injected;
  double kinetic, magnetic, px, py, pz;
  double fs_energy;           /* cumulative sum of w * dE at reflections */
  double injected_energy, removed_energy;
  double push_work;           /* cumulative work of E on the ions in the Boris
                                 pushes: with the three energies above it
                                 closes the kinetic-energy budget */
} or_diag_t;

typedef struct or_sim or_sim;

/* what codes for or_get_grid */
enum {
  OR_GRID_B = 0,      /* centres, [ny][nx][3] */
  OR_GRID_E = 1,      /* nodes, [ny][nxn][3] */
  OR_GRID_BBAR = 2,   /* nodes, [ny][nxn][3] */
  OR_GRID_N = 3,      /* nodes, [ny][nxn] */
  OR_GRID_J = 4,      /* nodes, [ny][nxn][3] */
  OR_GRID_U = 5,      /* nodes, [ny][nxn][3] */
  OR_GRID_PROFILE_N = 6,  /* [nxn] y-averaged n */
  OR_GRID_PROFILE_DB2 = 7 /* [nx] y-averaged |B - B0|^2 */
};

or_sim* or_create(const or_params* p);
void or_destroy(or_sim* s);
int or_nxn(const or_sim* s);
int or_step(or_sim* s, int nsteps);
long long or_num_particles(const or_sim* s);
int or_get_particles(const or_sim* s, int32_t* ci, int32_t* cj, double* fx,
                     double* fy, double* vx, double* vy, double* vz,
                     uint32_t* id);
int or_get_grid(const or_sim* s, int what, double* out);
int or_set_B(or_sim* s, const double* B);
int or_set_node_fields(or_sim* s, const double* E, const double* Bbar);
int or_inject(or_sim* s, long long n, const int32_t* ci, const int32_t* cj,
              const double* fx, const double* fy, const double* vx,
              const double* vy, const double* vz, const uint32_t* ids);
int or_diag(const or_sim* s, or_diag_t* out);
int or_histogram(const or_sim* s, int species, long long* out);
/* Momentum spectrum of one species (-1: all, 0: thermal, 1: cosmic rays):
   counts of |u| in spec_np bins between log-spaced edges
   e_k = spec_pmin exp((k / spec_np) ln(spec_pmax / spec_pmin)), bin k for
   e_k <= |u| < e_{k+1}; out [spec_np]. */
int or_spectrum_p(const or_sim* s, int species, long long* out);
void or_gather(const or_sim* s, int i, int j, double fx, double fy,
               double* out6);

/* building blocks, exported for the pin tests */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                      uint32_t out[4]);
double or_u01(uint32_t k);
double or_log(double x);
void or_sincos2pi(double u, double* c, double* s);
void or_boris(double* v, const double* E, const double* B, double dt);
/* relativistic Boris step of u = gamma v (c_light = c / v_A) */
void or_boris_rel(double* u, const double* E, const double* B, double dt,
                  double c_light);
int or_fs_rule(const or_params* p, double* v, uint32_t pid, long long step,
               double* mu_out);

#ifdef __cplusplus
}
#endif
#endif
