// fs_internal.h -- host-side state shared by the C ABI (fs_api.cu) and the
// per-precision kernel translation units (fs_f32.cu, fs_f64.cu).
#pragma once
#include <new>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fs.h"

namespace fsx {

// particle id word: bits 0-29 particle number, bit 30 cosmic-ray species,
// bit 31 set once the faux shock has returned the particle
constexpr uint32_t kIdMask = 0x3FFFFFFFu;
constexpr uint32_t kIdCR = 0x40000000u;
constexpr uint32_t kIdReturned = 0x80000000u;

// sticky device status bits
enum : int {
  kStatusCapacity = 1,
  kStatusNaN = 2,
  kStatusIdOverflow = 4,
  kStatusBadCell = 8,
  kStatusTimeout = 16
};

// Device-resident counters of one simulation (zeroed by fs_init).
struct Counters {
  unsigned long long incident, transmitted, reflected, escaped, injected;
  unsigned long long next_id;
  double fs_energy, injected_energy, removed_energy;
  double sums[8];        // diagnostics: kinetic, px, py, pz, magnetic
  int status;            // kStatus* bits
  int mover_count;       // unused
  long long step;        // step being taken (the Philox step counter)
};

// Structure-of-arrays particle buffer. cell packs (j << 16) | i.
template <typename T>
struct Parts {
  int* cell;
  T* ox;
  T* oy;
  T* vx;
  T* vy;
  T* vz;
  uint32_t* id;
};

// Geometry of the grid and of the tile decomposition.
struct Geo {
  int dim, nx, ny, nxn;     // nxn node columns: nx + 1, or nx when periodic
  int TX, TY, ntx, nty, ntiles;
  int bc_x;
  int chunk;                // particles per shared-memory chunk in the push
  int tile_cap;             // particle slots per tile
  long long cap_total;      // ntiles * tile_cap
  int mover_per_tile;       // mover-list slots of each tile
  int mover_cap;            // mover-list slots: ntiles * mover_per_tile
  int staging_cap;          // host-injection staging slots
  int na;                   // accumulator nodes per tile: (TX+3)*(TY+3) or TX+3
  int nk;                   // sort keys per tile
  int push_ctas;            // cap on the push's persistent CTAs per SM (0: none)
};

// Constants derived once on the host from fs_params (FP64; kernels cast).
struct Phys {
  double dtdx, dtdy, hdt, hdx, hdy, idx, h, hh, h6, te, vth, w_th, w_cr;
  double u2, u_cr, p_iso, mach_a, n_floor, eta, jcr, rate, cellvol;
  double b0x, b0y, b0z;
  int fs_mode_thermal, fs_frame, inject_thermal, cr_enable;
  unsigned long long seed;
  int hist_nx, hist_np;
  double hist_pmin, hist_pmax;
  double c2inv;    // 1 / c^2 (0: non-relativistic ions)
  double p_iso_v;  // CR injection speed p_iso / gamma(p_iso)
  int spec_np;     // momentum-spectrum bins
};

// Byte offsets of every region inside the caller's device buffer.
struct Layout {
  size_t part[2][7], mov[7], stg[7];
  size_t tile_base, cnt[2], mcnt;
  size_t B, Bs, Bsum, E, Es, Bb, G, n, u, J, pre;
  size_t partial, far, acc, inj, ctr, hist, prof, spec;
  size_t total;
};

// Typed device pointers (resolved from the layout).
template <typename T>
struct DevPtrs {
  Parts<T> P[2], M, S;
  int* tile_base;
  int* cnt[2];
  int* mcnt;      // movers written by each tile this step
  T *B, *Bs, *Bsum, *E, *Es, *Bb, *G, *n, *u, *J;
  T* pre;          // FP64: 1/n and the two pressure terms per node, per step
  void* partial;   // float accumulators (FP32) or int64 fixed point (FP64)
  void* far;
  double* acc;
  int* inj;        // injection row counts [ny] and offsets [ny + 1]
  Counters* ctr;
  unsigned long long* hist;
  double* prof;
};

// One run of a batched ensemble as the batched push reads it (device table,
// records sizeof(BatchRun) apart: 16-byte aligned, so host and device agree
// on the stride).
// The push's per-step constants in the run's precision, formed on the host:
// kernel parameters of that type are operands the push reads as they are,
// with no FP64 conversion on the device.
// Body guard of every C entry point: no C++ exception leaves the library
// (a failed host allocation returns FS_ENOMEM, anything else FS_ECUDA).
#define FS_GUARD_BEGIN try {
#define FS_GUARD_END                     \
  }                                      \
  catch (const std::bad_alloc&) {        \
    return FS_ENOMEM;                    \
  }                                      \
  catch (...) {                          \
    return FS_ECUDA;                     \
  }

template <typename T>
struct PushConst {
  T dtdx, dtdy, hdt;  // dt/dx, dt/dy, dt/2
  T wth, wcr;         // deposit weights (x 2^40 in FP64: the fixed-point scale)
  T c2inv;            // 1/c^2 (0: non-relativistic)
};
template <typename T>
inline PushConst<T> push_const(const Phys& ph) {
  const double ws = sizeof(T) == 8 ? 0x1p40 : 1.0;
  return PushConst<T>{(T)ph.dtdx, (T)ph.dtdy, (T)ph.hdt, (T)(ph.w_th * ws), (T)(ph.w_cr * ws),
                      (T)ph.c2inv};
}

template <typename T>
struct alignas(16) BatchRun {
  DevPtrs<T> d;
  Geo g;
  Phys ph;
  PushConst<T> pc;
  int in, out;  // particle buffers read and written this step
  int ncta;     // CTAs of the run's group
  int n_sub;    // RK4 field substeps per step
};
static_assert(sizeof(BatchRun<float>) % 16 == 0 && sizeof(BatchRun<double>) % 16 == 0,
              "batch records must tile the table at their own size");

struct Sim;

// Per-precision kernel launchers. Each returns cudaSuccess or the launch
// error; none allocates memory.
struct Ops {
  cudaError_t (*init_particles)(Sim*);
  cudaError_t (*deposit_all)(Sim*, int buf);
  cudaError_t (*moments)(Sim*);
  cudaError_t (*ohm_final)(Sim*);
  // ev: NULL, or FS_NPHASES + 1 events recorded at the phase boundaries
  cudaError_t (*step)(Sim*, int in_buf, long long step, cudaEvent_t* ev);
  cudaError_t (*step_rest)(Sim*, int in_buf, cudaEvent_t* ev);  // all but the push
  // batched ensembles (k_push_batch)
  size_t (*batch_run_bytes)();
  void (*fill_batch_run)(const Sim*, int in_buf, int ncta, void* dst);
  // chunk: the batch's push chunk (every run's push_chunk when they agree,
  // else 0: the large chunk)
  size_t (*batch_smem)(int dim, int tx, int ty, int chunk);
  // rel: the push variant with the relativistic terms (some run has c > 0)
  // txc: the tile width of every run of the launch (1D FP32 widths 4, 8, 16
  // have a kernel with the width compiled in; else 0)
  cudaError_t (*batch_setup)(int dim, int rel, int chunk, int txc, size_t smem, int* occ);
  cudaError_t (*push_batch)(int dim, int rel, int chunk, int txc, const void* runs,
                            const int2* cta_map, int ncta, size_t smem, cudaStream_t st);
  // the rest of a batched step in one launch per kernel over every run (1D
  // runs with x walls): pre holds three block prefixes over the runs (movers,
  // moments, field tiles; nruns + 1 entries each), nblk their totals
  // (the movers on stream side, between events fork and join, beside the
  // injection, moments and field advance on st)
  cudaError_t (*batch_rest)(const void* runs, const int* pre, int nruns, const int* nblk,
                            int n_sub_max, cudaStream_t st, cudaStream_t side,
                            cudaEvent_t fork, cudaEvent_t join);
  cudaError_t (*fields)(Sim*);
  cudaError_t (*insert_staged)(Sim*, int buf, int n, bool from_movers);
  cudaError_t (*diag)(Sim*, int buf);
  cudaError_t (*hist)(Sim*, int buf, int species);
  cudaError_t (*profiles)(Sim*);
  cudaError_t (*profile_B)(Sim*);       // y-averaged B into the profile region
  cudaError_t (*spectrum_bperp)(Sim*);  // B-perp power spectrum into the profile region
  cudaError_t (*spectrum_p)(Sim*, int buf, int species);  // n(p) counts
  cudaError_t (*export_grid)(Sim*, int what, double* dst_dev);
  cudaError_t (*import_B)(Sim*, const double* src_dev);
  cudaError_t (*export_particles)(Sim*, int buf, double* dst_dev, int* cell_dev,
                                  uint32_t* id_dev, int* count_dev);
};

const Ops& ops_f32();
const Ops& ops_f64();
size_t push_smem_bytes_f32(int dim, int tx, int ty, int chunk);
size_t push_smem_bytes_f64(int dim, int tx, int ty, int chunk);
int derive_geometry(const fs_params* p, Geo* g, Phys* ph);
// one CTA of the bounded-wait self-test (k_wait_selftest) on st
cudaError_t launch_wait_selftest(int* status, int limit, cudaStream_t st);

struct Sim {
  fs_params p;
  Geo g;
  Phys ph;
  Layout L;
  char* base;          // caller's device buffer
  cudaStream_t stream;
  int cur;             // ping-pong buffer holding the current particles
  long long step;
  int sticky;          // first error code reported
  long long launches;  // kernels launched through this handle
  const Ops* ops;
  // one captured step per ping-pong parity (replayed by fs_step)
  cudaGraphExec_t graph[2];
  cudaStream_t cap_stream;
  // a second stream for the captured step: the movers run on it beside the
  // injection, moments and field advance (fork / join events)
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  // a third stream: the FP32 2D field substep's wall tile columns beside its
  // interior launch
  cudaStream_t side2;
  cudaEvent_t ev_fork2, ev_join2;
  bool graphs_ready;
  int steps_direct;    // steps launched directly (graphs are captured after one)
  template <typename T>
  DevPtrs<T> ptrs(int dummy = 0) const;
};

template <typename T>
inline Parts<T> parts_at(char* base, const size_t off[7]) {
  Parts<T> r;
  r.cell = (int*)(base + off[0]);
  r.ox = (T*)(base + off[1]);
  r.oy = (T*)(base + off[2]);
  r.vx = (T*)(base + off[3]);
  r.vy = (T*)(base + off[4]);
  r.vz = (T*)(base + off[5]);
  r.id = (uint32_t*)(base + off[6]);
  return r;
}

template <typename T>
inline DevPtrs<T> Sim::ptrs(int) const {
  DevPtrs<T> d;
  d.P[0] = parts_at<T>(base, L.part[0]);
  d.P[1] = parts_at<T>(base, L.part[1]);
  d.M = parts_at<T>(base, L.mov);
  d.S = parts_at<T>(base, L.stg);
  d.tile_base = (int*)(base + L.tile_base);
  d.cnt[0] = (int*)(base + L.cnt[0]);
  d.cnt[1] = (int*)(base + L.cnt[1]);
  d.mcnt = (int*)(base + L.mcnt);
  d.B = (T*)(base + L.B);
  d.Bs = (T*)(base + L.Bs);
  d.Bsum = (T*)(base + L.Bsum);
  d.E = (T*)(base + L.E);
  d.Es = (T*)(base + L.Es);
  d.Bb = (T*)(base + L.Bb);
  d.G = (T*)(base + L.G);
  d.n = (T*)(base + L.n);
  d.u = (T*)(base + L.u);
  d.J = (T*)(base + L.J);
  d.pre = (T*)(base + L.pre);
  d.partial = (void*)(base + L.partial);
  d.far = (void*)(base + L.far);
  d.acc = (double*)(base + L.acc);
  d.inj = (int*)(base + L.inj);
  d.ctr = (Counters*)(base + L.ctr);
  d.hist = (unsigned long long*)(base + L.hist);
  d.prof = (double*)(base + L.prof);
  return d;
}

}  // namespace fsx
