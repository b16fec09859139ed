/*
 * fs.h -- C ABI of the GB300 faux-shock hybrid particle-in-cell engine.
 *
 * The engine advances a hybrid plasma (kinetic ions, massless isothermal
 * electron fluid) in a box whose x = 0 wall is the "faux shock" of Simon,
 * Caprioli, Haggerty & Reville (arXiv 2507.14282, Sec. 2): a particle that
 * crosses it leaves the box or is returned upstream with a momentum kick that
 * mimics scattering in the downstream, with the return probability of Eq. 1.
 * Plasma enters continuously through the far wall x = L drifting toward the
 * faux shock at u_sh = M_A (Sec. 2); the far wall is open; y is periodic.
 *
 * Normalised units (Sec. 2): x in d_i, t in 1/Omega_ci, v in v_A, B in B0,
 * n in n_g, E in v_A B0 / c, energy in m v_A^2, ion charge-to-mass 1.
 *
 * Conventions for every entry point:
 *  - Every function returns an int status: FS_OK (0) or a negative FS_E*
 *    code; fs_strerror() names it. No C++ exception crosses the ABI.
 *  - Device memory is owned by the caller: fs_query() reports how many bytes
 *    one simulation needs, the caller allocates one device buffer of that size
 *    (any allocator, e.g. a torch uint8 tensor) and passes it to fs_init().
 *    The library never allocates or frees device memory. The buffer must stay
 *    valid until fs_destroy(). Host arrays passed in are copied before return.
 *  - Work is enqueued on the CUDA stream given to fs_init() (NULL = legacy
 *    default stream). Entry points documented "synchronises" wait for that
 *    stream; the others only enqueue.
 *  - Device-side error conditions (capacity exhausted, non-finite motion, id
 *    overflow) are sticky: kernels record them in a device status word, and
 *    the next synchronising call returns the corresponding code. A handle that
 *    has reported an error keeps returning it.
 *  - One handle is not thread-safe; distinct handles are independent.
 */
#ifndef FS_H
#define FS_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FS_OK 0
#define FS_EINVAL (-1)        /* bad parameter, size, pointer or argument */
#define FS_ECAPACITY (-2)     /* particle, tile or mover capacity exhausted */
#define FS_ENAN (-3)          /* non-finite particle motion */
#define FS_EIDOVERFLOW (-4)   /* more than 2^30 particle ids issued */
#define FS_ECUDA (-5)         /* a CUDA call or kernel launch failed */
#define FS_ETIMEOUT (-6)      /* a bounded device wait ran out */
#define FS_EUNSTABLE (-7)     /* fs_diag: field integrator beyond its RK4 stability bound */
#define FS_ENOMEM (-8)        /* a host memory allocation failed */
#define FS_EBADCELL (-9)      /* a particle found outside its tile (corrupted state) */

/* precision of particle and field arithmetic */
#define FS_FP64 0
#define FS_FP32 1

/* x boundary: the faux-shock box (Sec. 2) or a periodic box (tests) */
#define FS_BC_FAUXSHOCK 0
#define FS_BC_PERIODIC 1

/* what the faux shock does to a species crossing it (Sec. 2) */
#define FS_OPEN 0   /* always leaves the box (the paper's thermal plasma) */
#define FS_SHOCK 1  /* passes or returns with Eq. 1's probability */

/* frame of the speed v in Eq. 1 */
#define FS_FRAME_SHOCK 0       /* the paper's wording: shock-frame speed */
#define FS_FRAME_DOWNSTREAM 1  /* downstream-frame speed (flux-ratio form) */

/*
 * Simulation parameters. fs_params_default() fills every field; callers then
 * change what they need. Physical parameters follow the columns of the
 * paper's Table 1 (M_A, Delta x, Delta t, theta_Bn, n_cr/n_g, p_iso) and the
 * faux-shock description of Sec. 2 (r, u2 = u_sh / r, Eq. 1).
 */
typedef struct fs_params {
  int dim;                 /* 1 or 2 */
  int nx, ny;              /* cells; ny = 1 when dim = 1; nx < 65536, ny < 32768 */
  double dx, dy, dt;       /* cell size in d_i, step in 1/Omega_ci */
  int precision;           /* FS_FP64 or FS_FP32 */
  double mach_a;           /* u_sh / v_A in the shock (simulation) frame */
  double theta_bn_deg;     /* B0 = (cos, sin, 0) */
  double beta_i, beta_e;   /* T_i = beta_i / 2, T_e = beta_e / 2 (isothermal) */
  int ppc;                 /* thermal macroparticles per cell; weight 1/ppc */
  int bc_x;                /* FS_BC_FAUXSHOCK or FS_BC_PERIODIC */
  int fs_mode_thermal;     /* FS_OPEN (paper) or FS_SHOCK */
  int fs_speed_frame;      /* FS_FRAME_SHOCK or FS_FRAME_DOWNSTREAM */
  double r_comp;           /* compression ratio r (default 4) */
  double u2;               /* downstream speed; <= 0 means mach_a / r_comp */
  int inject_thermal;      /* thermal inflow at x = L (faux-shock box) */
  int cr_enable;           /* cosmic-ray source at the faux shock (Sec. 2) */
  double n_cr_ratio;       /* n_cr / n_g (0.01 in Table 1) */
  double p_iso;            /* cosmic-ray speed in the downstream frame */
  double u_cr;             /* cosmic-ray bulk drift; <= 0 means u2 */
  int n_sub;               /* RK4 field substeps per particle step */
  double n_floor;          /* density floor used in Ohm's law */
  double eta;              /* resistivity (default 0) */
  double j_cr_ext;         /* prescribed uniform x-current in Ohm's law */
  int init_plasma;         /* load the uniform drifting plasma at t = 0 */
  unsigned long long seed; /* Philox key */
  double capacity_factor;  /* particle slots per tile / (ppc * cells per tile) */
  double mover_fraction;   /* mover-list slots / particle slots */
  int tile_x, tile_y;      /* cells per tile (0: chosen by the library) */
  int hist_nx, hist_np;    /* x - p_x histogram bins */
  double hist_pmin, hist_pmax;
  int use_graph;           /* replay fs_step as a captured CUDA graph (default 1;
                              the first step runs directly, later ones replay;
                              steps with fs_profile enabled run directly) */
  double c_light;          /* c / v_A; 0 (default): non-relativistic ions. With
                              c > 0 (the relativistic code of Sec. 2) particles
                              carry u = gamma v (momentum per mass, in the vx,
                              vy, vz slots and in fs_inject / fs_get_particles),
                              the Boris rotation uses B dt / (2 gamma), moves and
                              currents use v = u / gamma, the faux shock acts on
                              v, and p_iso is the CRs' momentum */
  int spec_np;             /* momentum spectrum n(p) (FS_SPECTRUM_P_*): bins of */
  double spec_pmin, spec_pmax; /* |u| between log-spaced edges pmin..pmax */
  /* launch shape of the particle push (a tuning choice; results do not
     depend on it in FP64): */
  int push_chunk;          /* particles per shared-memory chunk: 0 (library
                              choice), 512 (three stages in FP32) or 576 (two
                              stages; FP32 only) */
  int push_ctas_per_sm;    /* persistent CTAs per SM: 0 (as many as fit) or a
                              cap >= 1 */
} fs_params;

/* sizes reported by fs_query */
typedef struct fs_sizes {
  size_t device_bytes;          /* one device buffer of this many bytes */
  size_t device_alignment;      /* its required alignment in bytes */
  long long particle_capacity;  /* total particle slots */
  long long tiles;              /* number of tiles */
  int tile_x, tile_y;           /* tile shape in cells */
  int nxn;                      /* node columns: nx + 1, or nx when periodic */
} fs_sizes;

/* diagnostics (fs_diag) */
typedef struct fs_diag_t {
  long long step, n_particles, next_id;
  long long incident, transmitted, reflected, escaped, injected;
  double kinetic, magnetic;       /* energies, m v_A^2 n_g d_i^dim units */
  double px, py, pz;              /* total momentum */
  double fs_energy;               /* cumulative w dE of returned particles */
  double injected_energy, removed_energy;
  int status;                     /* sticky device status bits */
  long long launches;             /* kernels this handle has launched */
  /* Stability number of the field integrator: z = h omega_max, h = dt/n_sub
     the RK4 substep and omega_max = max over nodes of
     (4/dx^2 + 4/dy^2) |Bbar| / n + (2/dx + 2/dy) |u| (no dy terms in 1D), an
     upper estimate of the fastest discrete mode (grid-scale whistler plus
     advection). RK4 is stable on the imaginary axis for z <= FS_RK4_Z_MAX;
     above it fs_diag returns FS_EUNSTABLE (with *out filled in). */
  double max_z;
} fs_diag_t;

#define FS_RK4_Z_MAX 2.8284271247461903 /* 2 sqrt 2 */

/* what codes for fs_moments */
#define FS_B 0            /* B at cell centres: [ny][nx][3] doubles */
#define FS_E 1            /* E at nodes: [ny][nxn][3] */
#define FS_BBAR 2         /* B averaged to nodes: [ny][nxn][3] */
#define FS_N 3            /* ion density at nodes (after floor): [ny][nxn] */
#define FS_J 4            /* ion current at nodes: [ny][nxn][3] */
#define FS_U 5            /* ion bulk velocity J/n at nodes: [ny][nxn][3] */
#define FS_PROFILE_N 6    /* y-averaged n: [nxn] */
#define FS_PROFILE_DB2 7  /* y-averaged |B - B0|^2 / B0^2: [nx] */
#define FS_HIST_XPX 8     /* x - p_x histogram, all species: [hist_nx][hist_np] int64 */
#define FS_HIST_XPX_CR 9  /* the same for the cosmic-ray species only */
#define FS_PROFILE_B 10   /* y-averaged B (lineouts of Bx, By, Bz, Sec. 3.1): [nx][3] */
/* Perpendicular magnetic power spectrum averaged over y (Sec. 3.1, Fig. 3
   caption): P[k] = (1/ny) sum_y (|F[By](k, y)|^2 + |F[Bz](k, y)|^2) with
   F[f](k, y) = (1/nx) sum_x f(x, y) exp(-2 pi i k x / nx), for
   k = 0 .. nx/2 (wavenumber 2 pi k / (nx dx)): [nx/2 + 1] doubles. Computed
   in FP64 in every precision. */
#define FS_SPECTRUM_BPERP 11
/* Momentum spectra n(p): counts of particles with e_k <= |u| < e_{k+1},
   e_k = spec_pmin exp((k / spec_np) ln(spec_pmax / spec_pmin)) (edges
   computed once on the host), k = 0 .. spec_np - 1: [spec_np] int64. */
#define FS_SPECTRUM_P_CR 12   /* cosmic-ray species */
#define FS_SPECTRUM_P_ALL 13  /* all particles */

/* Run state beyond the particles and the field, for checkpoint / restart:
   fs_moments(FS_STATE) copies it out, fs_restore_state() puts it back. The
   step counter keys the random draws of the faux-shock return and of the
   inflow (Philox counter = (particle number, step, purpose), Sec. 2 draws);
   the row accumulators carry each transverse row's fractional inflow
   particle (ppc u_sh dt / dx per step, Sec. 2's continuous injection) to
   the next step. With them, a run saved after N steps (fs_get_particles,
   fs_moments(FS_B), fs_moments(FS_STATE)) and restored into a fresh handle
   (init_plasma = 0; fs_load_fields, fs_inject with the saved ids,
   fs_restore_state) continues as the straight run does: in FP64 bit for bit
   (the deposit sums do not depend on particle order); the energy sums
   only to FP64 rounding, their later additions being order dependent. */
typedef struct fs_run_state {
  long long step;          /* steps taken */
  long long next_id;       /* next particle number to issue */
  long long incident, transmitted, reflected, escaped, injected;  /* flux counters */
  double fs_energy, injected_energy, removed_energy;  /* energy budget sums */
  int ny;                  /* rows: entries of the accumulators that follow */
  int reserved;            /* 0 */
  /* followed in the same buffer by double row_acc[ny] */
} fs_run_state;
#define FS_STATE 14       /* fs_run_state then row_acc[ny]: sizeof(fs_run_state) + 8 ny bytes */

typedef struct fs_handle fs_handle;
typedef struct fs_batch fs_batch;   /* ensemble of handles stepped together */

/* Fills *out with defaults for a dim-dimensional faux-shock box.
   Returns FS_EINVAL if out is NULL or dim is not 1 or 2. */
int fs_params_default(int dim, fs_params* out);

/* Validates *p -- the problem statement of Sec. 2 (box, inflow speed u_sh =
   M_A, faux-shock parameters r and u2 of Eq. 1) and the run columns of
   Table 1 (Delta x, Delta t, M_A, theta_Bn, n_cr/n_g, p_iso) -- and reports
   the device buffer size it needs in *out: the particle buckets (capacity
   factor x ppc per cell), the grids, the moments and the counters.
   Allocates nothing. Returns FS_EINVAL for an inconsistent parameter set. */
int fs_query(const fs_params* p, fs_sizes* out);

/* Creates a simulation in the caller's device buffer (device_mem, of
   device_bytes >= fs_query's size, aligned to device_alignment) on the given
   CUDA stream (a cudaStream_t, or NULL). Loads B0 and, when init_plasma is
   set, ppc particles per cell (uniform positions, drifting Maxwellian,
   Sec. 2), deposits the moments and computes E^0. Enqueues only. */
int fs_init(const fs_params* p, void* device_mem, size_t device_bytes,
            void* cuda_stream, fs_handle** out);

/* Appends n kinetic ions given on the host (the particle species of the
   hybrid model, Sec. 2: a test population, a custom upstream, or a saved
   run being restored): cell indices (ci, cj), in-cell
   offsets (fx, fy) in [0, 1), velocities (vx, vy, vz); fy/cj ignored in 1D.
   Layout: n entries per array, x = (ci + fx) dx, y = (cj + fy) dy.
   ids: NULL assigns fresh thermal ids; otherwise each id word (bits 0-29
   particle number, bit 30 cosmic ray, bit 31 returned) is kept. Re-deposits
   the moments and recomputes E from the current B. Synchronises.
   FS_EINVAL on an out-of-range cell or offset; FS_ECAPACITY when a tile is
   full. */
int fs_inject(fs_handle* h, long long n, const int* ci, const int* cj,
              const double* fx, const double* fy, const double* vx,
              const double* vy, const double* vz, const unsigned* ids);

/* Replaces B at the cell centres ([ny][nx][3] doubles on the host, copied
   before return) -- e.g. seeded transverse modes like the perturbations the
   Bell instability of Sec. 3.1 grows from, or a saved field -- and
   recomputes E from Ohm's law with the massless-electron closure of Sec. 2
   and B at the nodes, from the current moments. Values are not checked:
   a non-finite B surfaces as FS_ENAN once particles move through it.
   Synchronises. */
int fs_load_fields(fs_handle* h, const double* B_host);

/* Advances nsteps particle steps (Sec. 2's boundary, the hybrid step).
   Enqueues only; errors found on the device surface at the next
   synchronising call. */
int fs_step(fs_handle* h, int nsteps);

/* Copies an output (what = FS_*) to dst (dst_bytes large enough:
   doubles, or int64 for the histograms), on the host or (dst_on_device)
   in device memory, converted to FP64 in either precision: the fields and
   ion moments of the hybrid model (Sec. 2: B, E, n, J, u), the y-averaged
   profiles and B lineouts (Sec. 3.1, Fig. 2), the x - p_x phase space
   (Fig. 1), the perpendicular power spectrum (Fig. 3 caption), the
   momentum spectra (Fig. 1 bottom panels) and the run state (FS_STATE).
   FS_EINVAL for an unknown code or a short buffer. Synchronises. */
int fs_moments(fs_handle* h, int what, void* dst, size_t dst_bytes,
               int dst_on_device);

/* Restores the run state saved by fs_moments(FS_STATE) from host memory
   (state, state_bytes >= sizeof(fs_run_state) + 8 ny): the step counter,
   next particle number, flux counters, energy sums and inflow row
   accumulators. Particles and field are not touched (fs_inject,
   fs_load_fields restore them). Synchronises. FS_EINVAL for a NULL or short
   buffer, a row count other than the handle's, negative counts or a
   non-finite accumulator. */
int fs_restore_state(fs_handle* h, const void* state, size_t state_bytes);

/* Number of live particles. Synchronises. */
int fs_num_particles(fs_handle* h, long long* n);

/* Copies every live particle to host arrays of length cap (order
   unspecified: sort by id to compare). *n receives the count.
   FS_EINVAL if cap is too small. Synchronises. */
int fs_get_particles(fs_handle* h, long long cap, int* ci, int* cj,
                     double* fx, double* fy, double* vx, double* vy,
                     double* vz, unsigned* id, long long* n);

/* Diagnostics: FP64 energy/momentum sums, int64 faux-shock flux counters
   (incident = transmitted + reflected: each crossing either passes or is
   returned with Eq. 1's probability, Sec. 2), the energy the returns add
   (the downstream-frame kick of Sec. 2), injected and removed energy,
   particle count, the sticky status bits and the field integrator's
   stability number. Synchronises; returns the sticky device error, if any,
   and FS_EUNSTABLE (with *out filled) above the RK4 bound. */
int fs_diag(fs_handle* h, fs_diag_t* out);

/* Per-phase timing of fs_step with CUDA events on the handle's stream
   (tracing). Phases: FS_PHASE_PUSH (fused gather/push/faux shock/sort/
   deposit kernel), FS_PHASE_MOVERS, FS_PHASE_INJECT, FS_PHASE_MOMENTS,
   FS_PHASE_FIELDS (RK4 Ohm + Faraday and the node packing).
   fs_profile(h, 1) starts recording (events are created on the host, no
   device memory); fs_profile_read() synchronises and writes, per phase, the
   summed milliseconds ms[k] and the number of steps timed counts[k] since the
   last read (arrays of nphases <= FS_NPHASES entries), then restarts the
   sums. fs_profile(h, 0) stops and releases the events. */
#define FS_PHASE_PUSH 0
#define FS_PHASE_MOVERS 1
#define FS_PHASE_INJECT 2
#define FS_PHASE_MOMENTS 3
#define FS_PHASE_FIELDS 4
#define FS_NPHASES 5
int fs_profile(fs_handle* h, int enable);
int fs_profile_read(fs_handle* h, double* ms, long long* counts, int nphases);

/* Allocation-free field advance (no counterpart in the paper: an addition
   of this library). Advances B by one particle step -- p->n_sub classical
   RK4 substeps of dB/dt = -curl E(B), E from Ohm's law with the moments n,
   u held fixed -- and writes E at the nodes from the advanced B: the same
   arithmetic fs_step applies after its deposit, for a caller that holds the
   moments and the field itself.
   Meant for callers that cannot allocate device memory and cannot lend the
   library scratch either: a host framework that owns every device byte
   through its own fixed pool, or a time-critical loop that must not trigger
   the implicit device synchronisation an allocation can cause. The RK4
   stage buffers live in one static device array of 2^20 doubles (8 MiB)
   that every GPU loading the library holds until the process exits; the
   function allocates and frees nothing, and the caller passes all inputs and
   outputs as device pointers on the current device:
     B_in, B_out  [3][ny][nx]   centre field, one plane per component
                                (B_out may equal B_in: advanced in place)
     n            [ny][nxn]     ion density at the nodes (after the floor)
     u            [3][ny][nxn]  ion bulk velocity at the nodes
     E_out        [3][ny][nxn]  electric field at the nodes
   nxn = nx + 1 (faux-shock box) or nx (periodic box). FP64 only. Apart
   from B_out == B_in, no output may share a byte with another output or an
   input (FS_EINVAL).
   Returns FS_EINVAL for a NULL pointer, FS_FP32, an invalid parameter set,
   overlapping buffers, or a grid whose stage buffers (6 nx ny + 3 nxn ny
   doubles) exceed the static array; FS_ECUDA when a CUDA call fails.
   Enqueues on cuda_stream. A call made while cuda_stream is not being
   captured looks up the array's device address on the current device (a
   host-side lookup, no synchronisation) and remembers it; a call made during
   stream capture uses the address remembered from an earlier call on that
   device, so make the first call on a device before any stream capture (a
   first call under capture returns FS_EINVAL). Every call on a device
   shares the one array, and it keeps the last call's contents (each call
   writes the stages before reading them): calls that overlap on the GPU --
   on different streams, or from different threads -- race. */
int fs_field_advance_noalloc(const fs_params* p, const double* B_in,
                             const double* n, const double* u, double* B_out,
                             double* E_out, void* cuda_stream);

/* ---- Batched ensembles: independent runs stepped together (Sec. 2 setup
   per run; the batch is an execution schedule, not a different method).
   A batch steps several handles -- faux-shock runs of any size, one
   precision and dimension, created on one CUDA stream -- with one push
   launch per step for each class of runs (1D FP32 runs of tile width 4, 8
   or 16 cells each form a class with that width compiled in; all other runs
   one class; the classes' launches run side by side): each run gets a group
   of CTAs about proportional to its particles (a (run, tile) work list, each
   run's pointers, geometry and physics read from a device table). When every run
   is 1D with x walls (the one-launch field advance), the rest of the step --
   movers, injection, moments, field advance, step counter -- is one launch
   per kernel over all runs too (each block works for one run, found from
   per-run block prefixes in the table): about seven launches per step
   whatever the number of runs. Otherwise each run's remaining kernels run in
   parallel branches. Either way the step is captured as a CUDA graph. The
   push's launch shape is the runs' push_chunk and push_ctas_per_sm when all
   runs agree on them, else the library's choice. Each
   run's results are those of fs_step on that handle alone (bit-identical in
   FP64).

   fs_batch_plan: host-only planner of the CTA groups. Runs of
   n_particles[r] particles in ntiles[r] tiles share ncta_max CTAs:
   ncta_out[r] is at least 1 and at most ntiles[r], the sum is at most
   ncta_max, and ncta_out[r] / n_particles[r] is as even as integer
   counts allow. FS_EINVAL for NULL arrays, nruns < 1, nruns > ncta_max, a
   negative count or a tile count < 1. */
int fs_batch_plan(int nruns, const long long* n_particles, const int* ntiles,
                  int ncta_max, int* ncta_out);

/* Device bytes of the run table of a batch of nruns runs of the given
   precision (FS_FP32 / FS_FP64). The caller allocates them (256-byte
   aligned) and keeps them until fs_batch_destroy. FS_EINVAL for nruns < 1
   or an unknown precision. */
int fs_batch_query(int nruns, int precision, size_t* table_bytes);

/* Creates a batch over runs[0..nruns-1]. The handles are not owned: each
   stays valid, and is not stepped on its own, until fs_batch_destroy.
   Synchronises the stream and sizes the CTA groups from the current
   particle counts (for each class of runs, four CTAs per CTA slot the GPU
   holds at once, at most 16384 over all classes). FS_EINVAL: NULL
   arguments, handles of mixed precision, dimension or stream, a table
   smaller than fs_batch_query's size, or more runs in a class than its
   CTAs; a handle's sticky error is returned as it is. */
int fs_batch_init(fs_handle* const* runs, int nruns, void* table_dev,
                  size_t table_bytes, fs_batch** out);

/* Advances every run of the batch by nsteps, asynchronously on the runs'
   stream. The first step is launched directly; later ones replay a
   captured CUDA graph (two, one per particle-buffer parity). Device
   conditions surface per run through fs_diag and the other synchronising
   calls; a failed launch marks every run with FS_ECUDA. */
int fs_batch_step(fs_batch* b, int nsteps);

/* Releases the batch (host state, its streams, events and graphs). The
   handles and the table buffer stay the caller's. */
int fs_batch_destroy(fs_batch* b);

/* Releases the handle (host memory only). The device buffer stays the
   caller's. */
int fs_destroy(fs_handle* h);

/* Name of a status code. */
const char* fs_strerror(int status);

/* Failure-detection self-test (an addition of this library, with no
   counterpart in the paper). Every device wait of the particle push is
   bounded: after a fixed number of tries it gives up, records a timeout bit
   in the simulation's device status word and returns, and the next
   synchronising call reports FS_ETIMEOUT, so a lost copy cannot hang the
   GPU. This call exercises that path on purpose without a fault: it launches
   one CTA that waits with the same bounded wait, at most `limit` tries
   (1 <= limit <= 2^20), on an mbarrier that nothing arrives on and no copy
   targets. The wait runs out, the CTA sets the timeout bit in *status_dev
   (one int of device memory owned by the caller; the call zeroes it first)
   and returns with nothing in flight. Synchronises cuda_stream and returns
   the code of the status word: FS_ETIMEOUT when the wait ran out (the
   expected result), FS_OK if it completed, FS_EINVAL for a NULL pointer or
   a limit out of range, FS_ECUDA for a failed launch or copy. */
int fs_selftest_wait(int limit, int* status_dev, void* cuda_stream);

/* Measurement utility (not part of the method): this GPU's FP64
   fused multiply-add rate, the denominator of the FP64 push's roofline.
   Runs a kernel of independent FP64 FMA chains on every SM at full
   occupancy, `iters` FMAs per chain (1 <= iters <= 2^24), on `cuda_stream`
   (0: the legacy default stream); returns FMA lane operations per second
   in *ops_per_s (an FMA counted once: FLOP/s is twice this). Synchronises
   the stream. FS_EINVAL for a bad argument, FS_ECUDA for a launch error. */
int fs_fp64_fma_rate(int iters, void* cuda_stream, double* ops_per_s);

/* ------------------------------------------------------------------------
   Differentiable window (1D faux-shock box): the gradient of a loss at the
   end of `steps` hybrid steps with respect to
     theta = (a_1 .. a_M, u_cr, u2),
   the amplitudes of M seeded transverse-B modes
     B_y = B0_y + sum_m a_m cos(2 pi m x / L + phi_m),
     B_z = B0_z + sum_m a_m sin(2 pi m x / L + phi_m)   (x at cell centres),
   the drift speed u_cr of the cosmic-ray source at the faux shock (Sec. 2;
   its ions start with speed p_iso, flux-weighted in the frame drifting at
   u_cr) and the faux shock's downstream speed u2 (the kick of the return,
   Eq. 1). The loss is the upstream magnetic fluctuation energy at the
   window's end, sum over cells i >= loss_i0 of |B_perp - B0_perp|^2 dx.
   The step is fs_step's scheme (CIC gather, Boris push, faux-shock return,
   inflow at x = L, CR source, CIC deposit, RK4 Ohm + Faraday with the
   moments frozen), on particles kept in fixed slots. The backward is the
   discrete adjoint along the forward's branches: crossings, returns,
   escapes, the density floor and every random draw are frozen. Checkpoints
   every ckpt_every steps; each segment is recomputed once in the backward
   (deterministic int64 fixed-point deposit sums, so a recomputed segment
   repeats the forward exactly).
   Parameters come from fs_params with dim = 1, the faux-shock box and no
   relativistic ions (c_light = 0); precision FS_FP32 or FS_FP64; p->u2 and
   p->u_cr are ignored (theta holds them).

   fs_window_query: device bytes for the window (no allocation).
   fs_window_init: x_init[n_init] positions in cells (X = i + f, 0 <= X <
   nx), v_init[n_init][3] velocities (v_A), host arrays copied before return;
   mode_phase[n_modes] the phases phi_m; dev_buf (256-byte aligned, >= the
   queried bytes, owned by the caller, outliving the handle). The initial
   ions get ids 0 .. n_init - 1; injected ions continue from n_init.
   fs_window_forward: runs the window for theta[n_modes + 2] and writes the
   loss; synchronises. FS_EINVAL for u2 <= 0 or u_cr outside [0, p_iso).
   fs_window_backward: d loss / d theta (times dloss) into grad[n_modes + 2];
   needs a forward just before it (the backward reuses and overwrites the
   forward's state; FS_EINVAL otherwise); synchronises.
   fs_window_counts: incident, returned, transmitted, escaped, injected of
   the last forward. */
typedef struct fs_window fs_window;
int fs_window_query(const fs_params* p, int steps, int ckpt_every, long long n_init,
                    int n_modes, size_t* bytes);
int fs_window_init(const fs_params* p, int steps, int ckpt_every, long long n_init,
                   const double* x_init, const double* v_init, int n_modes,
                   const double* mode_phase, int loss_i0, void* dev_buf, size_t bytes,
                   void* cuda_stream, fs_window** out);
int fs_window_forward(fs_window* w, const double* theta, double* loss);
int fs_window_backward(fs_window* w, double dloss, double* grad);
int fs_window_counts(fs_window* w, long long* out5);
int fs_window_destroy(fs_window* w);

#ifdef __cplusplus
}
#endif
#endif
