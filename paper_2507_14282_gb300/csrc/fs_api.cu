// fs_api.cu -- the C ABI declared in include/fs.h: parameter validation,
// tile decomposition, layout of the caller's device buffer, and the host
// orchestration of the kernels (fs_ops.cuh) on the caller's stream.
//
// The library allocates no device memory: every device region below is a
// slice of the single buffer the caller passes to fs_init().
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <thread>
#include <vector>

#include "fs.h"
#include "fs_internal.h"

using namespace fsx;

namespace {

constexpr size_t kAlign = 256;

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool divides(int a, int b) { return a > 0 && b % a == 0; }

// The push's shared memory for a tx x ty tile fits one CTA.
// The push's chunk: the caller's choice, else 576 particles in FP32 (a
// 512-particle mean tile in one chunk, four CTAs per SM) unless the mean tile
// holds at most 256, and 512 in FP64 (two CTAs per SM with its wider
// particles).
int push_chunk_of(const fs_params* p, int tx, int ty) {
  if (p->push_chunk) return p->push_chunk;
  return (p->precision == FS_FP32 && (long long)tx * ty * p->ppc > 256) ? 576 : 512;
}

bool push_tile_fits(const fs_params* p, int tx, int ty) {
  const int chunk = push_chunk_of(p, tx, ty);
  const size_t smem = (p->precision == FS_FP64) ? push_smem_bytes_f64(p->dim, tx, ty, chunk)
                                                : push_smem_bytes_f32(p->dim, tx, ty, chunk);
  return smem <= 227 * 1024 - 1024;
}

// Tile shape: the most cells (then the squarest tile) whose mean particle
// count stays within 512 and whose push fits shared memory; tile sides
// divide the box.
void choose_tile(const fs_params* p, int* tx, int* ty) {
  if (p->dim == 1) {
    if (p->tile_x > 0) { *tx = p->tile_x; *ty = 1; return; }
    int best = 0;
    for (int c = 2; c <= 256 && c <= p->nx; ++c) {
      if (!divides(c, p->nx)) continue;
      if ((long long)c * p->ppc <= 512 || best == 0) best = c;
    }
    *tx = best ? best : p->nx;
    *ty = 1;
    return;
  }
  if (p->tile_x > 0 && p->tile_y > 0) { *tx = p->tile_x; *ty = p->tile_y; return; }
  int bx = 0, by = 0;
  long long bestc = -1;
  for (int cy = 1; cy <= 32 && cy <= p->ny; ++cy) {
    if (!divides(cy, p->ny)) continue;
    for (int cx = 2; cx <= 64 && cx <= p->nx; ++cx) {
      if (!divides(cx, p->nx)) continue;
      const long long cells = (long long)cx * cy;
      if (cells * p->ppc > 512) continue;
      if (!push_tile_fits(p, cx, cy)) continue;  // node block + accumulators in smem
      // prefer more cells, then squarer tiles
      const long long score = cells * 1000 - (long long)abs(cx - 2 * cy);
      if (score > bestc) { bestc = score; bx = cx; by = cy; }
    }
  }
  if (bestc < 0) {  // ppc very large: smallest legal tile
    bx = 0;
    for (int cx = 2; cx <= p->nx; ++cx) if (divides(cx, p->nx)) { bx = cx; break; }
    by = 1;
  }
  *tx = bx;
  *ty = by;
}

int validate(const fs_params* p) {
  if (!p) return FS_EINVAL;
  if (p->dim != 1 && p->dim != 2) return FS_EINVAL;
  if (p->nx < 2 || p->nx > 65535) return FS_EINVAL;
  if (p->ny < 1 || p->ny > 32767) return FS_EINVAL;
  if (p->dim == 1 && p->ny != 1) return FS_EINVAL;
  if (!(p->dx > 0) || !(p->dt > 0) || (p->dim == 2 && !(p->dy > 0))) return FS_EINVAL;
  if (p->precision != FS_FP64 && p->precision != FS_FP32) return FS_EINVAL;
  if (p->ppc < 1 || p->n_sub < 1) return FS_EINVAL;
  if (p->bc_x != FS_BC_FAUXSHOCK && p->bc_x != FS_BC_PERIODIC) return FS_EINVAL;
  if (p->fs_mode_thermal != FS_OPEN && p->fs_mode_thermal != FS_SHOCK) return FS_EINVAL;
  if (p->fs_speed_frame != FS_FRAME_SHOCK && p->fs_speed_frame != FS_FRAME_DOWNSTREAM)
    return FS_EINVAL;
  if (!(p->r_comp > 1.0) && !(p->u2 > 0)) return FS_EINVAL;
  if (!(p->beta_i >= 0) || !(p->beta_e >= 0)) return FS_EINVAL;
  if (!(p->n_floor > 0)) return FS_EINVAL;
  if (!(p->capacity_factor >= 1.0) || !(p->mover_fraction > 0)) return FS_EINVAL;
  if (p->cr_enable) {
    const double u2 = p->u2 > 0 ? p->u2 : p->mach_a / p->r_comp;
    const double ucr = p->u_cr > 0 ? p->u_cr : u2;
    if (!(p->p_iso > ucr)) return FS_EINVAL;
  }
  if (p->hist_nx < 1 || p->hist_np < 1 || !(p->hist_pmax > p->hist_pmin)) return FS_EINVAL;
  if (!(p->c_light >= 0)) return FS_EINVAL;
  if (p->c_light > 0 && !(p->mach_a < p->c_light)) return FS_EINVAL;
  if (p->spec_np < 1 || !(p->spec_pmin > 0) || !(p->spec_pmax > p->spec_pmin)) return FS_EINVAL;
  if (p->mach_a < 0) return FS_EINVAL;
  if (p->push_chunk != 0 && p->push_chunk != 512 &&
      !(p->push_chunk == 576 && p->precision == FS_FP32))
    return FS_EINVAL;
  if (p->push_ctas_per_sm < 0) return FS_EINVAL;
  return FS_OK;
}

int derive(const fs_params* p, Geo* g, Phys* ph, Layout* L) {
  int r = validate(p);
  if (r) return r;
  memset(g, 0, sizeof(*g));
  memset(ph, 0, sizeof(*ph));
  memset(L, 0, sizeof(*L));
  int tx, ty;
  choose_tile(p, &tx, &ty);
  if (tx < 2 || !divides(tx, p->nx)) return FS_EINVAL;
  if (p->dim == 2) {
    if (ty < 1 || !divides(ty, p->ny)) return FS_EINVAL;
  } else {
    ty = 1;
  }
  g->dim = p->dim;
  g->nx = p->nx;
  g->ny = p->ny;
  g->bc_x = p->bc_x;
  g->nxn = (p->bc_x == FS_BC_PERIODIC) ? p->nx : p->nx + 1;
  g->TX = tx;
  g->TY = ty;
  g->ntx = p->nx / tx;
  g->nty = p->ny / ty;
  g->ntiles = g->ntx * g->nty;
  const long long cells_per_tile = (long long)tx * ty;
  long long cap = (long long)ceil(p->capacity_factor * (double)(cells_per_tile * p->ppc)) + 64;
  cap = (cap + 31) / 32 * 32;
  if (cap > (1LL << 30)) return FS_EINVAL;
  g->tile_cap = (int)cap;
  g->cap_total = cap * g->ntiles;
  if (g->cap_total >= (1LL << 31) - 1) return FS_EINVAL;
  long long mpt = (long long)ceil(p->mover_fraction * (double)cap) + 32;
  mpt = (mpt + 31) / 32 * 32;
  if (mpt * g->ntiles >= (1LL << 31) - 1) return FS_EINVAL;
  g->mover_per_tile = (int)mpt;
  g->mover_cap = (int)(mpt * g->ntiles);
  g->staging_cap = 1 << 16;
  g->chunk = push_chunk_of(p, tx, ty);
  g->push_ctas = p->push_ctas_per_sm;
  g->na = (tx + 3) * (p->dim == 2 ? ty + 3 : 1);
  g->nk = (tx + 2) * (p->dim == 2 ? ty + 2 : 1) + 2;
  const size_t smem = (p->precision == FS_FP64)
                          ? push_smem_bytes_f64(p->dim, tx, ty, g->chunk)
                          : push_smem_bytes_f32(p->dim, tx, ty, g->chunk);
  if (smem > 227 * 1024 - 1024) return FS_EINVAL;
  if (g->nk > 32 * 1024) return FS_EINVAL;

  // physics constants (the same FP64 expressions the scheme is written in)
  ph->dtdx = p->dt / p->dx;
  ph->dtdy = (p->dim == 2) ? p->dt / p->dy : 0.0;
  ph->hdt = 0.5 * p->dt;
  ph->hdx = 0.5 / p->dx;
  ph->hdy = (p->dim == 2) ? 0.5 / p->dy : 0.0;
  ph->idx = 1.0 / p->dx;
  ph->h = p->dt / (double)p->n_sub;
  ph->hh = 0.5 * ph->h;
  ph->h6 = ph->h / 6.0;
  ph->te = 0.5 * p->beta_e;
  ph->vth = sqrt(0.5 * p->beta_i);
  ph->w_th = 1.0 / (double)p->ppc;
  ph->w_cr = p->n_cr_ratio / (double)p->ppc;
  ph->u2 = p->u2 > 0.0 ? p->u2 : p->mach_a / p->r_comp;
  ph->u_cr = p->u_cr > 0.0 ? p->u_cr : ph->u2;
  ph->p_iso = p->p_iso;
  ph->mach_a = p->mach_a;
  ph->n_floor = p->n_floor;
  ph->eta = p->eta;
  ph->jcr = p->j_cr_ext;
  ph->rate = (((double)p->ppc * p->mach_a) * p->dt) / p->dx;
  ph->cellvol = (p->dim == 2) ? p->dx * p->dy : p->dx;
  const double th = p->theta_bn_deg * (3.14159265358979323846264338327950288 / 180.0);
  ph->b0x = cos(th);
  ph->b0y = sin(th);
  ph->b0z = 0.0;
  ph->fs_mode_thermal = p->fs_mode_thermal;
  ph->fs_frame = p->fs_speed_frame;
  ph->inject_thermal = p->inject_thermal ? 1 : 0;
  ph->cr_enable = p->cr_enable ? 1 : 0;
  ph->seed = p->seed;
  ph->hist_nx = p->hist_nx;
  ph->hist_np = p->hist_np;
  ph->hist_pmin = p->hist_pmin;
  ph->hist_pmax = p->hist_pmax;
  ph->c2inv = (p->c_light > 0.0) ? 1.0 / (p->c_light * p->c_light) : 0.0;
  ph->p_iso_v = (ph->c2inv > 0.0) ? p->p_iso / sqrt(1.0 + (p->p_iso * p->p_iso) * ph->c2inv)
                                  : p->p_iso;
  ph->spec_np = p->spec_np;

  // device buffer layout
  const size_t T = (p->precision == FS_FP64) ? 8 : 4;
  const size_t A = (p->precision == FS_FP64) ? 8 : 4;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    o = up(o, kAlign);
    const size_t r = o;
    o += bytes;
    return r;
  };
  auto parts = [&](size_t* dst, size_t n) {
    dst[0] = take(4 * n);
    dst[1] = take(T * n);
    dst[2] = take(p->dim == 2 ? T * n : 0);
    dst[3] = take(T * n);
    dst[4] = take(T * n);
    dst[5] = take(T * n);
    dst[6] = take(4 * n);
  };
  parts(L->part[0], g->cap_total);
  parts(L->part[1], g->cap_total);
  parts(L->mov, g->mover_cap);
  parts(L->stg, g->staging_cap);
  L->tile_base = take(4 * (size_t)g->ntiles);
  L->cnt[0] = take(4 * (size_t)g->ntiles);
  L->cnt[1] = take(4 * (size_t)g->ntiles);
  L->mcnt = take(4 * (size_t)g->ntiles);
  const size_t nc = (size_t)p->nx * p->ny, nn = (size_t)g->nxn * p->ny;
  L->B = take(3 * T * nc);
  L->Bs = take(3 * T * nc);
  L->Bsum = take(3 * T * nc);
  L->E = take(3 * T * nn);
  L->Es = take(3 * T * nn);
  L->Bb = take(3 * T * nn);
  L->G = take(8 * T * (size_t)(p->nx + 1) * (p->ny + 1));
  L->n = take(T * nn);
  L->u = take(3 * T * nn);
  L->J = take(3 * T * nn);
  // FP64 only: per-step Ohm's-law terms that depend on n alone
  L->pre = take(p->precision == FS_FP64 ? 3 * T * nn : 0);
  L->partial = take(A * 4 * (size_t)g->na * g->ntiles);
  L->far = take(A * 4 * nn);
  L->acc = take(8 * (size_t)p->ny);
  L->inj = take(4 * (2 * (size_t)p->ny + 2));
  L->ctr = take(sizeof(Counters));
  L->hist = take(8 * (size_t)p->hist_nx * p->hist_np);
  L->spec = take(8 * (2 * (size_t)p->spec_np + 1));  // edges [np + 1], counts [np]
  // profiles: n [nxn], dB^2 [nx], B [nx][3], B-perp spectrum [nx/2 + 1]
  L->prof = take(8 * ((size_t)g->nxn + p->nx + 3 * (size_t)p->nx + (size_t)p->nx / 2 + 1));
  L->total = up(o, kAlign);
  return FS_OK;
}

int status_to_code(int st) {
  if (st & kStatusTimeout) return FS_ETIMEOUT;
  if (st & kStatusNaN) return FS_ENAN;
  if (st & kStatusIdOverflow) return FS_EIDOVERFLOW;
  if (st & kStatusCapacity) return FS_ECAPACITY;
  if (st & kStatusBadCell) return FS_EBADCELL;
  return FS_OK;
}

__global__ void k_fill_tiles(int* base, int* cnt, int ntiles, int cap, int init) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles;
       t += gridDim.x * blockDim.x) {
    base[t] = t * cap;
    cnt[t] = init;
  }
}

template <typename T>
__global__ void k_fill_B(T* B, int nc, double bx, double by, double bz) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc;
       c += gridDim.x * blockDim.x) {
    B[c] = (T)bx;
    B[(size_t)nc + c] = (T)by;
    B[(size_t)2 * nc + c] = (T)bz;
  }
}

// Synchronise the stream, then fold the device status word into the handle.
int sync_and_check(Sim* s) {
  if (s->sticky) return s->sticky;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return s->sticky = FS_ECUDA;
  int st = 0;
  e = cudaMemcpy(&st, s->base + s->L.ctr + offsetof(Counters, status), sizeof(int),
                 cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return s->sticky = FS_ECUDA;
  const int code = status_to_code(st);
  if (code) s->sticky = code;
  return code;
}

int grid_blocks(long long n) {
  long long g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return (int)g;
}

// Capture one step for each ping-pong parity on a private stream (the legacy
// default stream cannot be captured); the graphs replay on the caller's stream.
// Kernels one step launches: push, movers, injection (3), moments, the field
// advance, step end. The field advance is one tiled launch in 1D boxes with
// x walls, one per substep in FP32 2D boxes with x walls, else [FP64: Ohm
// density terms], 2 x 4 x n_sub stage passes and the final Ohm (the same
// choice as the field launcher makes).
long long launches_per_step(const Sim* s) {
  const bool inj = s->g.bc_x == FS_BC_FAUXSHOCK && (s->ph.inject_thermal || s->ph.cr_enable);
  const bool walls = s->g.bc_x != FS_BC_PERIODIC;
  long long fields;
  if (s->g.dim == 1 && walls && s->p.n_sub <= 16)
    fields = 1;
  else if (s->p.precision == FS_FP32 && s->g.dim == 2 && walls)
    fields = s->p.n_sub;
  else
    fields = (s->p.precision == FS_FP64 ? 1 : 0) + 8LL * s->p.n_sub + 1;
  return 1 + 1 + (inj ? 3 : 0) + 1 + fields + 1;
}

int build_graphs(Sim* s) {
  if (!s->cap_stream &&
      cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return FS_ECUDA;
  if (!s->side && cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess)
    return FS_ECUDA;
  if ((!s->ev_fork && cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess) ||
      (!s->ev_join && cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess))
    return FS_ECUDA;
  if (!s->side2 && cudaStreamCreateWithFlags(&s->side2, cudaStreamNonBlocking) != cudaSuccess)
    return FS_ECUDA;
  if ((!s->ev_fork2 && cudaEventCreateWithFlags(&s->ev_fork2, cudaEventDisableTiming) != cudaSuccess) ||
      (!s->ev_join2 && cudaEventCreateWithFlags(&s->ev_join2, cudaEventDisableTiming) != cudaSuccess))
    return FS_ECUDA;
  // the captured work must follow everything already queued on the caller's stream
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return FS_ECUDA;
  cudaStream_t user = s->stream;
  s->stream = s->cap_stream;
  int rc = FS_OK;
  for (int par = 0; par < 2 && rc == FS_OK; ++par) {
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = FS_ECUDA;
      break;
    }
    const cudaError_t e = s->ops->step(s, par, 0, nullptr);
    const cudaError_t e2 = cudaStreamEndCapture(s->stream, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess || !gr) {
      rc = FS_ECUDA;
      if (gr) cudaGraphDestroy(gr);
      break;
    }
    if (cudaGraphInstantiate(&s->graph[par], gr, 0) != cudaSuccess) rc = FS_ECUDA;
    cudaGraphDestroy(gr);
  }
  s->stream = user;
  cudaGetLastError();
  if (rc == FS_OK) s->graphs_ready = true;
  return rc;
}

void release_graphs(Sim* s) {
  for (int par = 0; par < 2; ++par)
    if (s->graph[par]) {
      cudaGraphExecDestroy(s->graph[par]);
      s->graph[par] = nullptr;
    }
  if (s->cap_stream) {
    cudaStreamDestroy(s->cap_stream);
    s->cap_stream = nullptr;
  }
  if (s->side) {
    cudaStreamDestroy(s->side);
    s->side = nullptr;
  }
  if (s->ev_fork) {
    cudaEventDestroy(s->ev_fork);
    s->ev_fork = nullptr;
  }
  if (s->ev_join) {
    cudaEventDestroy(s->ev_join);
    s->ev_join = nullptr;
  }
  if (s->side2) {
    cudaStreamDestroy(s->side2);
    s->side2 = nullptr;
  }
  if (s->ev_fork2) {
    cudaEventDestroy(s->ev_fork2);
    s->ev_fork2 = nullptr;
  }
  if (s->ev_join2) {
    cudaEventDestroy(s->ev_join2);
    s->ev_join2 = nullptr;
  }
  s->graphs_ready = false;
}

int redeposit(Sim* s) {
  cudaError_t e = cudaMemsetAsync(s->base + s->L.far, 0,
                                  (s->p.precision == FS_FP64 ? 8 : 4) * 4 *
                                      (size_t)s->g.nxn * s->g.ny,
                                  s->stream);
  if (e != cudaSuccess) return FS_ECUDA;
  if ((e = s->ops->deposit_all(s, s->cur)) != cudaSuccess) return FS_ECUDA;
  if ((e = s->ops->moments(s)) != cudaSuccess) return FS_ECUDA;
  if ((e = s->ops->ohm_final(s)) != cudaSuccess) return FS_ECUDA;
  return FS_OK;
}

}  // namespace

namespace fsx {
// Geometry and derived constants of a parameter set, without a handle (used
// by the allocation-free field entry point).
int derive_geometry(const fs_params* p, Geo* g, Phys* ph) {
  Layout L;
  return derive(p, g, ph, &L);
}
}  // namespace fsx

struct fs_handle {
  Sim sim;
  // phase timing (fs_profile): one set of FS_NPHASES + 1 events per step
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  size_t used = 0;  // event sets recorded since the last read
  double ms[FS_NPHASES] = {0};
  long long counts[FS_NPHASES] = {0};
};

namespace {
void release_events(fs_handle* h) {
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  h->events.clear();
  h->used = 0;
}
}  // namespace

namespace {
// Runs f(lo, hi) over [0, n) in slices on up to 16 host threads. If a
// thread cannot be started, the slices it would have taken run on the
// calling thread (no exception leaves this function).
template <typename F>
void parallel_slices(long long n, F f) {
  const unsigned hw = std::thread::hardware_concurrency();
  long long nt = std::min<long long>(hw ? hw : 1, 16);
  nt = std::max<long long>(1, std::min<long long>(nt, n / (1 << 16)));
  std::vector<std::thread> th;
  long long k = 1;  // slice 0 runs here
  try {
    th.reserve((size_t)nt);
    for (; k < nt; ++k) th.emplace_back(f, n * k / nt, n * (k + 1) / nt);
  } catch (...) {
  }
  f(0LL, n / nt);
  for (long long r = k; r < nt; ++r) f(n * r / nt, n * (r + 1) / nt);
  for (auto& x : th) x.join();
}

// Staged copies of the caller's columns: cell = (j << 16) | i from the i
// column (in `cell`) and the j column (in `id`, 2D), then the ids first,
// first + 1, ... in input order.
__global__ void k_pack_staged(int* cell, uint32_t* id, int m, int dim,
                              unsigned long long first) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const int j = (dim == 2) ? (int)id[k] : 0;
    cell[k] = (j << 16) | cell[k];
    id[k] = (uint32_t)(first + (unsigned long long)k);
  }
}
}  // namespace

namespace {
// Independent FP64 FMA chains (8 per thread) for fs_fp64_fma_rate: x <- x a + b
// with a = b = 1/2 converges to 1, so the values stay finite; the sink write
// never happens but keeps the chains.
constexpr int kFmaChains = 8;
__global__ void __launch_bounds__(256) k_fp64_fma(double* sink, int iters, double a, double b) {
  double x[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) x[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) x[k] = __fma_rn(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += x[k];
  if (s == -1.0) sink[blockIdx.x] = s;
}
}  // namespace

extern "C" {

int fs_params_default(int dim, fs_params* out) {
  FS_GUARD_BEGIN
  if (!out || (dim != 1 && dim != 2)) return FS_EINVAL;
  memset(out, 0, sizeof(*out));
  out->dim = dim;
  out->nx = 512;
  out->ny = (dim == 2) ? 64 : 1;
  out->dx = 0.5;
  out->dy = 0.5;
  out->dt = 0.005;
  out->precision = FS_FP64;
  out->mach_a = 10.0;
  out->theta_bn_deg = 0.0;
  out->beta_i = 1.0;
  out->beta_e = 1.0;
  out->ppc = 32;
  out->bc_x = FS_BC_FAUXSHOCK;
  out->fs_mode_thermal = FS_SHOCK;
  out->fs_speed_frame = FS_FRAME_SHOCK;
  out->r_comp = 4.0;
  out->u2 = 0.0;
  out->inject_thermal = 1;
  out->cr_enable = 0;
  out->n_cr_ratio = 0.01;
  out->p_iso = 100.0;
  out->u_cr = 0.0;
  out->n_sub = 2;
  out->n_floor = 0.05;
  out->eta = 0.0;
  out->j_cr_ext = 0.0;
  out->init_plasma = 1;
  out->seed = 1;
  out->use_graph = 1;
  out->capacity_factor = 3.0;
  out->mover_fraction = 0.25;
  out->tile_x = 0;
  out->tile_y = 0;
  out->hist_nx = 64;
  out->hist_np = 64;
  out->hist_pmin = -40.0;
  out->hist_pmax = 40.0;
  out->c_light = 0.0;
  out->spec_np = 64;
  out->spec_pmin = 1.0;
  out->spec_pmax = 1.0e4;
  return FS_OK;
  FS_GUARD_END
}

int fs_query(const fs_params* p, fs_sizes* out) {
  FS_GUARD_BEGIN
  if (!out) return FS_EINVAL;
  Geo g;
  Phys ph;
  Layout L;
  const int r = derive(p, &g, &ph, &L);
  if (r) return r;
  out->device_bytes = L.total;
  out->device_alignment = kAlign;
  out->particle_capacity = g.cap_total;
  out->tiles = g.ntiles;
  out->tile_x = g.TX;
  out->tile_y = g.TY;
  out->nxn = g.nxn;
  return FS_OK;
  FS_GUARD_END
}

int fs_init(const fs_params* p, void* device_mem, size_t device_bytes,
            void* cuda_stream, fs_handle** out) {
  FS_GUARD_BEGIN
  if (!out) return FS_EINVAL;
  *out = nullptr;
  fs_handle* h = new (std::nothrow) fs_handle();
  if (!h) return FS_EINVAL;
  Sim* s = &h->sim;
  int r = derive(p, &s->g, &s->ph, &s->L);
  if (r) { delete h; return r; }
  if (!device_mem || device_bytes < s->L.total || ((uintptr_t)device_mem % kAlign) != 0) {
    delete h;
    return FS_EINVAL;
  }
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, device_mem) != cudaSuccess ||
      attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    delete h;
    return FS_EINVAL;
  }
  s->p = *p;
  s->base = (char*)device_mem;
  s->stream = (cudaStream_t)cuda_stream;
  s->cur = 0;
  s->step = 0;
  s->sticky = 0;
  s->ops = (p->precision == FS_FP64) ? &ops_f64() : &ops_f32();
  const long long nc = (long long)p->nx * p->ny;
  const size_t Tsz = (p->precision == FS_FP64) ? 8 : 4;
  cudaError_t e = cudaSuccess;
  auto zero = [&](size_t off, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemsetAsync(s->base + off, 0, bytes, s->stream);
  };
  zero(s->L.ctr, sizeof(Counters));
  zero(s->L.acc, 8 * (size_t)p->ny);
  zero(s->L.far, (s->L.acc > s->L.far) ? s->L.acc - s->L.far : 0);
  zero(s->L.G, 8 * Tsz * (size_t)(p->nx + 1) * (p->ny + 1));
  zero(s->L.cnt[1], 4 * (size_t)s->g.ntiles);
  if (e != cudaSuccess) { delete h; return FS_ECUDA; }
  const int init_cnt = p->init_plasma ? s->g.TX * s->g.TY * p->ppc : 0;
  if (init_cnt > s->g.tile_cap) { delete h; return FS_EINVAL; }
  if (p->init_plasma && nc * (long long)p->ppc > (long long)kIdMask) { delete h; return FS_EIDOVERFLOW; }
  k_fill_tiles<<<grid_blocks(s->g.ntiles), 256, 0, s->stream>>>(
      (int*)(s->base + s->L.tile_base), (int*)(s->base + s->L.cnt[0]), s->g.ntiles,
      s->g.tile_cap, init_cnt);
  if (p->precision == FS_FP64)
    k_fill_B<double><<<grid_blocks(nc), 256, 0, s->stream>>>(
        (double*)(s->base + s->L.B), (int)nc, s->ph.b0x, s->ph.b0y, s->ph.b0z);
  else
    k_fill_B<float><<<grid_blocks(nc), 256, 0, s->stream>>>(
        (float*)(s->base + s->L.B), (int)nc, s->ph.b0x, s->ph.b0y, s->ph.b0z);
  if (cudaGetLastError() != cudaSuccess) { delete h; return FS_ECUDA; }
  if (p->init_plasma) {
    if (s->ops->init_particles(s) != cudaSuccess) { delete h; return FS_ECUDA; }
    const unsigned long long next = (unsigned long long)nc * p->ppc;
    if (cudaMemcpyAsync(s->base + s->L.ctr + offsetof(Counters, next_id), &next, 8,
                        cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
      delete h;
      return FS_ECUDA;
    }
    // the copy reads a host stack value: wait for it before returning
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) { delete h; return FS_ECUDA; }
  }
  {
    // momentum-spectrum bin edges, computed once on the host
    std::vector<double> edges(p->spec_np + 1);
    const double lr = log(p->spec_pmax / p->spec_pmin);
    for (int k = 0; k <= p->spec_np; ++k)
      edges[k] = p->spec_pmin * exp(((double)k / (double)p->spec_np) * lr);
    if (cudaMemcpyAsync(s->base + s->L.spec, edges.data(), 8 * edges.size(),
                        cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess) {
      delete h;
      return FS_ECUDA;
    }
  }
  r = redeposit(s);
  if (r) { delete h; return r; }
  *out = h;
  return FS_OK;
  FS_GUARD_END
}

int fs_step(fs_handle* h, int nsteps) {
  FS_GUARD_BEGIN
  if (!h || nsteps < 0) return FS_EINVAL;
  Sim* s = &h->sim;
  if (s->sticky) return s->sticky;
  const long long per_step = launches_per_step(s);
  constexpr int kSet = FS_NPHASES + 1;
  if (!h->profiling && s->p.use_graph && s->steps_direct > 0 && !s->graphs_ready) {
    int r = build_graphs(s);
    if (r) return s->sticky = r;
  }
  if (!h->profiling && s->graphs_ready) {
    for (int k = 0; k < nsteps; ++k) {
      if (cudaGraphLaunch(s->graph[s->cur], s->stream) != cudaSuccess)
        return s->sticky = FS_ECUDA;
      s->cur = 1 - s->cur;
      s->step++;
      s->launches += per_step;
    }
    return FS_OK;
  }
  for (int k = 0; k < nsteps; ++k) {
    cudaEvent_t* ev = nullptr;
    if (h->profiling) {
      while (h->events.size() < (h->used + 1) * kSet) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return s->sticky = FS_ECUDA;
        h->events.push_back(e);
      }
      ev = &h->events[h->used * kSet];
      h->used++;
    }
    if (s->ops->step(s, s->cur, s->step, ev) != cudaSuccess) return s->sticky = FS_ECUDA;
    s->cur = 1 - s->cur;
    s->step++;
    s->launches += per_step;
    s->steps_direct++;
  }
  return FS_OK;
  FS_GUARD_END
}

int fs_inject(fs_handle* h, long long n, const int* ci, const int* cj,
              const double* fx, const double* fy, const double* vx,
              const double* vy, const double* vz, const unsigned* ids) {
  FS_GUARD_BEGIN
  if (!h || n < 0) return FS_EINVAL;
  Sim* s = &h->sim;
  if (n == 0) return FS_OK;
  if (!ci || !fx || !vx || !vy || !vz) return FS_EINVAL;
  if (s->g.dim == 2 && (!cj || !fy)) return FS_EINVAL;
  // every input is checked before anything reaches the device
  const int dim = s->g.dim, nx = s->g.nx, ny = s->g.ny;
  std::atomic<bool> bad(false);
  parallel_slices(n, [&](long long lo, long long hi) {
    for (long long k = lo; k < hi && !bad.load(std::memory_order_relaxed); ++k) {
      const int j = (dim == 2) ? cj[k] : 0;
      if (ci[k] < 0 || ci[k] >= nx || j < 0 || j >= ny || !(fx[k] >= 0.0 && fx[k] < 1.0) ||
          (dim == 2 && !(fy[k] >= 0.0 && fy[k] < 1.0)) || !isfinite(vx[k]) ||
          !isfinite(vy[k]) || !isfinite(vz[k]))
        bad.store(true, std::memory_order_relaxed);
    }
  });
  if (bad.load()) return FS_EINVAL;
  int r = sync_and_check(s);
  if (r) return r;
  unsigned long long next = 0;
  if (cudaMemcpy(&next, s->base + s->L.ctr + offsetof(Counters, next_id), 8,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return s->sticky = FS_ECUDA;
  if (!ids && next + (unsigned long long)n - 1 > kIdMask) return s->sticky = FS_EIDOVERFLOW;
  const bool dbl = (s->p.precision == FS_FP64);
  const size_t Tsz = dbl ? 8 : 4;
  // stage through the mover list (unused between steps) in large chunks
  const int chunk = s->g.mover_cap > s->g.staging_cap ? s->g.mover_cap : s->g.staging_cap;
  const size_t* stg = s->g.mover_cap > s->g.staging_cap ? s->L.mov : s->L.stg;
  char* base = s->base;
  auto h2d = [&](size_t off, const void* src, size_t bytes) {
    return cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, s->stream);
  };
  if (dbl && !ids) {
    // FP64 without caller ids: the caller's columns go to the staging area as
    // they are (a pinned caller's arrays take the DMA path), the cell index
    // and the ids are formed on the device; the stream orders the chunks
    for (long long k0 = 0; k0 < n; k0 += chunk) {
      const int m = (int)((n - k0) < chunk ? (n - k0) : chunk);
      cudaError_t e = h2d(stg[0], ci + k0, 4 * (size_t)m);
      if (e == cudaSuccess && dim == 2) e = h2d(stg[6], cj + k0, 4 * (size_t)m);
      if (e == cudaSuccess) e = h2d(stg[1], fx + k0, 8 * (size_t)m);
      if (e == cudaSuccess && dim == 2) e = h2d(stg[2], fy + k0, 8 * (size_t)m);
      if (e == cudaSuccess) e = h2d(stg[3], vx + k0, 8 * (size_t)m);
      if (e == cudaSuccess) e = h2d(stg[4], vy + k0, 8 * (size_t)m);
      if (e == cudaSuccess) e = h2d(stg[5], vz + k0, 8 * (size_t)m);
      if (e == cudaSuccess) {
        k_pack_staged<<<std::min(1024, (m + 255) / 256), 256, 0, s->stream>>>(
            (int*)(base + stg[0]), (uint32_t*)(base + stg[6]), m, dim, next + (unsigned long long)k0);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = s->ops->insert_staged(s, s->cur, m, stg == s->L.mov);
      if (e != cudaSuccess) return s->sticky = FS_ECUDA;
    }
    next += (unsigned long long)n;
  } else {
    std::vector<int> cell(chunk);
    std::vector<uint32_t> id(chunk);
    std::vector<char> buf(5 * Tsz * (size_t)chunk);
    for (long long k0 = 0; k0 < n; k0 += chunk) {
      const int m = (int)((n - k0) < chunk ? (n - k0) : chunk);
      char* cols[5];
      for (int c = 0; c < 5; ++c) cols[c] = buf.data() + (size_t)c * Tsz * chunk;
      std::atomic<unsigned long long> top(next);
      parallel_slices(m, [&](long long lo, long long hi) {
        unsigned long long mx = 0;
        for (long long k = lo; k < hi; ++k) {
          const long long q = k0 + k;
          const int j = (dim == 2) ? cj[q] : 0;
          cell[k] = (j << 16) | ci[q];
          uint32_t w;
          if (ids) {
            w = ids[q];
            const unsigned long long num = w & kIdMask;
            if (num + 1 > mx) mx = num + 1;
          } else {
            w = (uint32_t)(next + (unsigned long long)q);
          }
          id[k] = w;
          const double vals[5] = {fx[q], dim == 2 ? fy[q] : 0.0, vx[q], vy[q], vz[q]};
          for (int c = 0; c < 5; ++c) {
            if (dbl) {
              ((double*)cols[c])[k] = vals[c];
            } else {
              float f = (float)vals[c];
              if (c < 2 && f >= 1.0f) f = 0x1.fffffep-1f;
              ((float*)cols[c])[k] = f;
            }
          }
        }
        unsigned long long cur = top.load();
        while (mx > cur && !top.compare_exchange_weak(cur, mx)) {
        }
      });
      cudaError_t e = h2d(stg[0], cell.data(), 4 * (size_t)m);
      for (int c = 0; c < 5 && e == cudaSuccess; ++c) {
        if (c == 1 && dim == 1) continue;
        e = h2d(stg[1 + c], cols[c], Tsz * (size_t)m);
      }
      if (e == cudaSuccess) e = h2d(stg[6], id.data(), 4 * (size_t)m);
      if (e == cudaSuccess) e = s->ops->insert_staged(s, s->cur, m, stg == s->L.mov);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // host buffers reused
      if (e != cudaSuccess) return s->sticky = FS_ECUDA;
      next = ids ? top.load() : next;
    }
    if (!ids) next += (unsigned long long)n;
  }
  if (cudaMemcpyAsync(s->base + s->L.ctr + offsetof(Counters, next_id), &next, 8,
                      cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return s->sticky = FS_ECUDA;
  r = redeposit(s);
  if (r) return s->sticky = r;
  return sync_and_check(s);
  FS_GUARD_END
}

int fs_load_fields(fs_handle* h, const double* B_host) {
  FS_GUARD_BEGIN
  if (!h || !B_host) return FS_EINVAL;
  Sim* s = &h->sim;
  int r = sync_and_check(s);
  if (r) return r;
  const size_t nc = (size_t)s->g.nx * s->g.ny;
  const bool dbl = (s->p.precision == FS_FP64);
  std::vector<char> tmp(3 * nc * (dbl ? 8 : 4));
  for (size_t q = 0; q < nc; ++q)
    for (int c = 0; c < 3; ++c) {
      if (dbl) ((double*)tmp.data())[c * nc + q] = B_host[q * 3 + c];
      else ((float*)tmp.data())[c * nc + q] = (float)B_host[q * 3 + c];
    }
  if (cudaMemcpyAsync(s->base + s->L.B, tmp.data(), tmp.size(), cudaMemcpyHostToDevice,
                      s->stream) != cudaSuccess)
    return s->sticky = FS_ECUDA;
  if (s->ops->ohm_final(s) != cudaSuccess) return s->sticky = FS_ECUDA;
  return sync_and_check(s);
  FS_GUARD_END
}

int fs_moments(fs_handle* h, int what, void* dst, size_t dst_bytes, int dst_on_device) {
  FS_GUARD_BEGIN
  if (!h || !dst) return FS_EINVAL;
  Sim* s = &h->sim;
  int r = sync_and_check(s);
  if (r) return r;
  const Geo& g = s->g;
  const bool dbl = (s->p.precision == FS_FP64);
  const size_t Tsz = dbl ? 8 : 4;
  if (what == FS_STATE) {
    const size_t need = sizeof(fs_run_state) + 8 * (size_t)g.ny;
    if (dst_bytes < need) return FS_EINVAL;
    Counters c;
    std::vector<char> blob(need);
    if (cudaMemcpyAsync(&c, s->base + s->L.ctr, sizeof(c), cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess ||
        cudaMemcpyAsync(blob.data() + sizeof(fs_run_state), s->base + s->L.acc,
                        8 * (size_t)g.ny, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
      return s->sticky = FS_ECUDA;
    r = sync_and_check(s);
    if (r) return r;
    fs_run_state st;
    memset(&st, 0, sizeof st);
    st.step = s->step;
    st.next_id = (long long)c.next_id;
    st.incident = (long long)c.incident;
    st.transmitted = (long long)c.transmitted;
    st.reflected = (long long)c.reflected;
    st.escaped = (long long)c.escaped;
    st.injected = (long long)c.injected;
    st.fs_energy = c.fs_energy;
    st.injected_energy = c.injected_energy;
    st.removed_energy = c.removed_energy;
    st.ny = g.ny;
    memcpy(blob.data(), &st, sizeof st);
    if (!dst_on_device) {
      memcpy(dst, blob.data(), need);
      return FS_OK;
    }
    if (cudaMemcpyAsync(dst, blob.data(), need, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
      return s->sticky = FS_ECUDA;
    return sync_and_check(s);
  }
  if (what == FS_HIST_XPX || what == FS_HIST_XPX_CR) {
    const size_t need = 8 * (size_t)s->ph.hist_nx * s->ph.hist_np;
    if (dst_bytes < need) return FS_EINVAL;
    if (s->ops->hist(s, s->cur, what == FS_HIST_XPX ? -1 : 1) != cudaSuccess)
      return s->sticky = FS_ECUDA;
    if (cudaMemcpyAsync(dst, s->base + s->L.hist, need,
                        dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess)
      return s->sticky = FS_ECUDA;
    return sync_and_check(s);
  }
  if (what == FS_PROFILE_N || what == FS_PROFILE_DB2) {
    const size_t cnt = (what == FS_PROFILE_N) ? g.nxn : g.nx;
    if (dst_bytes < 8 * cnt) return FS_EINVAL;
    if (s->ops->profiles(s) != cudaSuccess) return s->sticky = FS_ECUDA;
    const size_t off = s->L.prof + (what == FS_PROFILE_N ? 0 : 8 * (size_t)g.nxn);
    if (cudaMemcpyAsync(dst, s->base + off, 8 * cnt,
                        dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess)
      return s->sticky = FS_ECUDA;
    return sync_and_check(s);
  }
  if (what == FS_SPECTRUM_P_CR || what == FS_SPECTRUM_P_ALL) {
    const size_t np = (size_t)s->p.spec_np;
    if (dst_bytes < 8 * np) return FS_EINVAL;
    if (s->ops->spectrum_p(s, s->cur, what == FS_SPECTRUM_P_CR ? 1 : -1) != cudaSuccess)
      return s->sticky = FS_ECUDA;
    if (cudaMemcpyAsync(dst, s->base + s->L.spec + 8 * (np + 1), 8 * np,
                        dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess)
      return s->sticky = FS_ECUDA;
    return sync_and_check(s);
  }
  if (what == FS_PROFILE_B || what == FS_SPECTRUM_BPERP) {
    const bool spec = (what == FS_SPECTRUM_BPERP);
    const size_t cnt = spec ? (size_t)g.nx / 2 + 1 : 3 * (size_t)g.nx;
    if (dst_bytes < 8 * cnt) return FS_EINVAL;
    const cudaError_t e = spec ? s->ops->spectrum_bperp(s) : s->ops->profile_B(s);
    if (e != cudaSuccess) return s->sticky = FS_ECUDA;
    const size_t off = s->L.prof + 8 * ((size_t)g.nxn + g.nx + (spec ? 3 * (size_t)g.nx : 0));
    if (cudaMemcpyAsync(dst, s->base + off, 8 * cnt,
                        dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess)
      return s->sticky = FS_ECUDA;
    return sync_and_check(s);
  }
  size_t planes = 3, cols = g.nxn, src = 0;
  switch (what) {
    case FS_B: src = s->L.B; cols = g.nx; break;
    case FS_E: src = s->L.E; break;
    case FS_BBAR: src = s->L.Bb; break;
    case FS_N: src = s->L.n; planes = 1; break;
    case FS_J: src = s->L.J; break;
    case FS_U: src = s->L.u; break;
    default: return FS_EINVAL;
  }
  const size_t npts = cols * g.ny;
  if (dst_bytes < 8 * planes * npts) return FS_EINVAL;
  if (dst_on_device) {
    if (s->ops->export_grid(s, what, (double*)dst) != cudaSuccess) return s->sticky = FS_ECUDA;
    return sync_and_check(s);
  }
  std::vector<char> tmp(planes * npts * Tsz);
  if (cudaMemcpyAsync(tmp.data(), s->base + src, tmp.size(), cudaMemcpyDeviceToHost,
                      s->stream) != cudaSuccess)
    return s->sticky = FS_ECUDA;
  r = sync_and_check(s);
  if (r) return r;
  double* o = (double*)dst;
  for (size_t q = 0; q < npts; ++q)
    for (size_t c = 0; c < planes; ++c)
      o[q * planes + c] = dbl ? ((double*)tmp.data())[c * npts + q]
                              : (double)((float*)tmp.data())[c * npts + q];
  return FS_OK;
  FS_GUARD_END
}

int fs_restore_state(fs_handle* h, const void* state, size_t state_bytes) {
  FS_GUARD_BEGIN
  if (!h || !state || state_bytes < sizeof(fs_run_state)) return FS_EINVAL;
  Sim* s = &h->sim;
  fs_run_state st;
  memcpy(&st, state, sizeof st);
  if (st.ny != s->g.ny || state_bytes < sizeof(fs_run_state) + 8 * (size_t)s->g.ny)
    return FS_EINVAL;
  if (st.step < 0 || st.next_id < 0 || st.next_id > (long long)kIdMask + 1 || st.incident < 0 ||
      st.transmitted < 0 || st.reflected < 0 || st.escaped < 0 || st.injected < 0 ||
      st.incident != st.transmitted + st.reflected)
    return FS_EINVAL;
  std::vector<double> acc(s->g.ny);
  memcpy(acc.data(), (const char*)state + sizeof(fs_run_state), 8 * (size_t)s->g.ny);
  for (double a : acc)
    if (!(a >= 0.0 && a < 1.0)) return FS_EINVAL;
  int r = sync_and_check(s);
  if (r) return r;
  Counters c;
  if (cudaMemcpy(&c, s->base + s->L.ctr, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
    return s->sticky = FS_ECUDA;
  c.step = st.step;
  c.next_id = (unsigned long long)st.next_id;
  c.incident = (unsigned long long)st.incident;
  c.transmitted = (unsigned long long)st.transmitted;
  c.reflected = (unsigned long long)st.reflected;
  c.escaped = (unsigned long long)st.escaped;
  c.injected = (unsigned long long)st.injected;
  c.fs_energy = st.fs_energy;
  c.injected_energy = st.injected_energy;
  c.removed_energy = st.removed_energy;
  if (cudaMemcpy(s->base + s->L.ctr, &c, sizeof(c), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->base + s->L.acc, acc.data(), 8 * acc.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return s->sticky = FS_ECUDA;
  s->step = st.step;
  return sync_and_check(s);
  FS_GUARD_END
}

int fs_num_particles(fs_handle* h, long long* n) {
  FS_GUARD_BEGIN
  if (!h || !n) return FS_EINVAL;
  Sim* s = &h->sim;
  int r = sync_and_check(s);
  if (r) return r;
  std::vector<int> cnt(s->g.ntiles);
  if (cudaMemcpy(cnt.data(), s->base + s->L.cnt[s->cur], 4 * (size_t)s->g.ntiles,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return s->sticky = FS_ECUDA;
  long long tot = 0;
  for (int c : cnt) tot += (c < s->g.tile_cap ? c : s->g.tile_cap);
  *n = tot;
  return FS_OK;
  FS_GUARD_END
}

int fs_get_particles(fs_handle* h, long long cap, int* ci, int* cj, double* fx,
                     double* fy, double* vx, double* vy, double* vz, unsigned* id,
                     long long* n) {
  FS_GUARD_BEGIN
  if (!h || !n) return FS_EINVAL;
  Sim* s = &h->sim;
  long long tot = 0;
  int r = fs_num_particles(h, &tot);
  if (r) return r;
  *n = tot;
  if (cap < tot) return FS_EINVAL;
  if (tot > 0 && (!ci || !cj || !fx || !fy || !vx || !vy || !vz || !id)) return FS_EINVAL;
  const Geo& g = s->g;
  const bool dbl = (s->p.precision == FS_FP64);
  const size_t Tsz = dbl ? 8 : 4;
  std::vector<int> cnt(g.ntiles), base(g.ntiles);
  cudaMemcpy(cnt.data(), s->base + s->L.cnt[s->cur], 4 * (size_t)g.ntiles, cudaMemcpyDeviceToHost);
  cudaMemcpy(base.data(), s->base + s->L.tile_base, 4 * (size_t)g.ntiles, cudaMemcpyDeviceToHost);
  const size_t* off = s->L.part[s->cur];
  long long o = 0;
  std::vector<char> tb(7 * 8 * (size_t)g.tile_cap);
  for (int t = 0; t < g.ntiles; ++t) {
    const int c = cnt[t] < g.tile_cap ? cnt[t] : g.tile_cap;
    if (c <= 0) continue;
    const size_t b = (size_t)base[t];
    cudaError_t e = cudaSuccess;
    char* p[7];
    for (int k = 0; k < 7; ++k) p[k] = tb.data() + (size_t)k * 8 * g.tile_cap;
    e = cudaMemcpy(p[0], s->base + off[0] + 4 * b, 4 * (size_t)c, cudaMemcpyDeviceToHost);
    for (int k = 1; k <= 5 && e == cudaSuccess; ++k) {
      if (k == 2 && g.dim == 1) continue;
      e = cudaMemcpy(p[k], s->base + off[k] + Tsz * b, Tsz * (size_t)c, cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess)
      e = cudaMemcpy(p[6], s->base + off[6] + 4 * b, 4 * (size_t)c, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return s->sticky = FS_ECUDA;
    for (int k = 0; k < c; ++k, ++o) {
      const int cell = ((int*)p[0])[k];
      ci[o] = cell & 0xFFFF;
      cj[o] = cell >> 16;
      auto getT = [&](int col) {
        return dbl ? ((double*)p[col])[k] : (double)((float*)p[col])[k];
      };
      fx[o] = getT(1);
      fy[o] = (g.dim == 2) ? getT(2) : 0.0;
      vx[o] = getT(3);
      vy[o] = getT(4);
      vz[o] = getT(5);
      id[o] = ((uint32_t*)p[6])[k];
    }
  }
  return FS_OK;
  FS_GUARD_END
}

int fs_diag(fs_handle* h, fs_diag_t* out) {
  FS_GUARD_BEGIN
  if (!h || !out) return FS_EINVAL;
  Sim* s = &h->sim;
  int r = sync_and_check(s);
  if (r) return r;
  if (s->ops->diag(s, s->cur) != cudaSuccess) return s->sticky = FS_ECUDA;
  Counters c;
  if (cudaMemcpyAsync(&c, s->base + s->L.ctr, sizeof(c), cudaMemcpyDeviceToHost,
                      s->stream) != cudaSuccess)
    return s->sticky = FS_ECUDA;
  r = sync_and_check(s);
  if (r) return r;
  long long np = 0;
  r = fs_num_particles(h, &np);
  if (r) return r;
  memset(out, 0, sizeof(*out));
  out->step = s->step;
  out->n_particles = np;
  out->next_id = (long long)c.next_id;
  out->incident = (long long)c.incident;
  out->transmitted = (long long)c.transmitted;
  out->reflected = (long long)c.reflected;
  out->escaped = (long long)c.escaped;
  out->injected = (long long)c.injected;
  out->kinetic = c.sums[0];
  out->px = c.sums[1];
  out->py = c.sums[2];
  out->pz = c.sums[3];
  out->magnetic = c.sums[4];
  out->fs_energy = c.fs_energy;
  out->injected_energy = c.injected_energy;
  out->removed_energy = c.removed_energy;
  out->status = c.status;
  out->launches = s->launches;
  out->max_z = c.sums[5];
  return out->max_z > FS_RK4_Z_MAX ? FS_EUNSTABLE : FS_OK;
  FS_GUARD_END
}

int fs_profile(fs_handle* h, int enable) {
  FS_GUARD_BEGIN
  if (!h) return FS_EINVAL;
  if (enable) {
    h->profiling = true;
    return FS_OK;
  }
  cudaStreamSynchronize(h->sim.stream);
  h->profiling = false;
  release_events(h);
  return FS_OK;
  FS_GUARD_END
}

int fs_profile_read(fs_handle* h, double* ms, long long* counts, int nphases) {
  FS_GUARD_BEGIN
  if (!h || !ms || !counts || nphases < 1 || nphases > FS_NPHASES) return FS_EINVAL;
  Sim* s = &h->sim;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return s->sticky = FS_ECUDA;
  constexpr int kSet = FS_NPHASES + 1;
  for (size_t u = 0; u < h->used; ++u) {
    for (int k = 0; k < FS_NPHASES; ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, h->events[u * kSet + k], h->events[u * kSet + k + 1]) !=
          cudaSuccess)
        return s->sticky = FS_ECUDA;
      h->ms[k] += t;
      h->counts[k] += 1;
    }
  }
  h->used = 0;
  for (int k = 0; k < nphases; ++k) {
    ms[k] = h->ms[k];
    counts[k] = h->counts[k];
  }
  for (int k = 0; k < FS_NPHASES; ++k) {
    h->ms[k] = 0;
    h->counts[k] = 0;
  }
  return FS_OK;
  FS_GUARD_END
}

int fs_destroy(fs_handle* h) {
  FS_GUARD_BEGIN
  if (!h) return FS_EINVAL;
  cudaStreamSynchronize(h->sim.stream);
  release_events(h);
  release_graphs(&h->sim);
  delete h;
  return FS_OK;
  FS_GUARD_END
}


}  // extern "C"

// ---------------------------------------------------------------- batches
// (definitions keep the C linkage of their declarations in fs.h)

namespace {
constexpr int kBatchMaxCtas = 16384;  // CTA map entries the table holds
constexpr int kBatchOversubscribe = 4;  // batched-push CTAs per resident CTA slot
#ifndef FS_BATCH_BRANCHES
#define FS_BATCH_BRANCHES 32
#endif
constexpr int kBatchBranches = FS_BATCH_BRANCHES;  // parallel graph branches, per-run work

// the kernel indexes the table by record, so the stride is the record size
size_t batch_rec_bytes(int precision) {
  const Ops& o = (precision == FS_FP64) ? ops_f64() : ops_f32();
  return o.batch_run_bytes();
}
size_t batch_map_offset(int nruns, int precision) {
  return up(2 * (size_t)nruns * batch_rec_bytes(precision), kAlign);
}
// the block prefixes of the batched step tail (movers, moments, field tiles)
size_t batch_pre_offset(int nruns, int precision) {
  return up(batch_map_offset(nruns, precision) + sizeof(int2) * (size_t)kBatchMaxCtas, kAlign);
}
size_t batch_table_bytes(int nruns, int precision) {
  return batch_pre_offset(nruns, precision) + 3 * sizeof(int) * ((size_t)nruns + 1);
}
// blocks of the per-run step kernels the batched tail replaces (as step_rest
// and the 1D field launcher size them)
int movers_blocks(const Sim& s) { return std::min((s.g.ntiles + 7) / 8, 152 * 16); }
int moments_blocks(const Sim& s) {
  const long long nn = (long long)s.g.nxn * s.g.ny;
  return (int)std::max(1LL, std::min((nn + 255) / 256, 152LL * 16));
}
int field1_blocks(const Sim& s) { return (s.g.nx + 63) / 64; }
// runs whose whole step tail the batched kernels cover: 1D boxes with x
// walls and the one-launch field advance
bool tail_batchable(const Sim& s) {
  return s.g.dim == 1 && s.g.bc_x != FS_BC_PERIODIC && s.p.n_sub <= 16;
}
}  // namespace

struct fs_batch {
  std::vector<fs_handle*> runs;
  std::vector<int> cur0;  // each run's particle buffer when the batch was made
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private capture stream
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  char* table = nullptr;
  size_t rec = 0;
  int2* map = nullptr;
  int ncta = 0;
  size_t smem = 0;
  // one push launch per class of runs: its tile width (0: any), its CTAs'
  // range of the map, its shared memory
  struct Class { int txc, map0, ncta; size_t smem; };
  std::vector<Class> classes;
  int dim = 1;
  int rel = 0;  // some run has relativistic ions (c > 0)
  int chunk = 0;  // the batch push's chunk (0: the large chunk)
  const Ops* ops = nullptr;
  int parity = 0;  // steps taken, mod 2
  bool tail_batched = false;  // the step tail runs as one launch per kernel
  int nblk[3] = {0, 0, 0};    // blocks of the batched movers, moments, field tiles
  int n_sub_max = 1;
  int* pre = nullptr;         // their block prefixes in the table
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graphs_ready = false;
  int steps_direct = 0;
};

namespace {
// One batched step on stream st for table half p: the push of every run in
// one launch, then each run's remaining kernels on its branch.
cudaError_t batch_enqueue(fs_batch* b, int p, cudaStream_t st) {
  const int nr = (int)b->runs.size();
  cudaError_t e = cudaSuccess;
  const int nc = (int)b->classes.size();
  if (nc > 1 && (int)b->branch.size() >= nc) {
    // the classes' push launches side by side (one branch each), so that one
    // launch's last CTAs overlap the others'
    if ((e = cudaEventRecord(b->fork, st)) != cudaSuccess) return e;
    for (int k = 0; k < nc; ++k) {
      const auto& c = b->classes[k];
      cudaStream_t bs = b->branch[k];
      if ((e = cudaStreamWaitEvent(bs, b->fork, 0)) != cudaSuccess) return e;
      e = b->ops->push_batch(b->dim, b->rel, b->chunk, c.txc,
                             b->table + (size_t)p * nr * b->rec, b->map + c.map0, c.ncta, c.smem,
                             bs);
      if (e != cudaSuccess) return e;
      if ((e = cudaEventRecord(b->join[k], bs)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(st, b->join[k], 0)) != cudaSuccess) return e;
    }
  } else {
    for (const auto& c : b->classes) {
      e = b->ops->push_batch(b->dim, b->rel, b->chunk, c.txc,
                             b->table + (size_t)p * nr * b->rec, b->map + c.map0, c.ncta, c.smem,
                             st);
      if (e != cudaSuccess) return e;
    }
  }
  if (b->tail_batched)
    return b->ops->batch_rest(b->table + (size_t)p * nr * b->rec, b->pre, nr, b->nblk,
                              b->n_sub_max, st, b->branch[0], b->fork, b->join[0]);
  if ((e = cudaEventRecord(b->fork, st)) != cudaSuccess) return e;
  const int K = (int)b->branch.size();
  for (int k = 0; k < K; ++k)
    if ((e = cudaStreamWaitEvent(b->branch[k], b->fork, 0)) != cudaSuccess) return e;
  for (int r = 0; r < nr; ++r) {
    Sim* s = &b->runs[r]->sim;
    cudaStream_t user = s->stream;
    s->stream = b->branch[r % K];
    e = s->ops->step_rest(s, (b->cur0[r] + p) & 1, nullptr);
    s->stream = user;
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k < K; ++k) {
    if ((e = cudaEventRecord(b->join[k], b->branch[k])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, b->join[k], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int batch_build_graphs(fs_batch* b) {
  if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return FS_ECUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return FS_ECUDA;
  int rc = FS_OK;
  for (int par = 0; par < 2 && rc == FS_OK; ++par) {
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = FS_ECUDA;
      break;
    }
    const cudaError_t e = batch_enqueue(b, par, b->cap);
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess || !gr) {
      rc = FS_ECUDA;
      if (gr) cudaGraphDestroy(gr);
      break;
    }
    if (cudaGraphInstantiate(&b->graph[par], gr, 0) != cudaSuccess) rc = FS_ECUDA;
    cudaGraphDestroy(gr);
  }
  cudaGetLastError();
  if (rc == FS_OK) b->graphs_ready = true;
  return rc;
}

void batch_fail(fs_batch* b, int code) {
  for (fs_handle* h : b->runs)
    if (!h->sim.sticky) h->sim.sticky = code;
}
}  // namespace

int fs_batch_plan(int nruns, const long long* n_particles, const int* ntiles, int ncta_max,
                  int* ncta_out) {
  FS_GUARD_BEGIN
  if (nruns < 1 || !n_particles || !ntiles || !ncta_out || nruns > ncta_max) return FS_EINVAL;
  long double total = 0;
  for (int r = 0; r < nruns; ++r) {
    if (n_particles[r] < 0 || ntiles[r] < 1) return FS_EINVAL;
    total += (long double)n_particles[r];
  }
  long long sum = 0;
  for (int r = 0; r < nruns; ++r) {
    long long a = 1;
    if (total > 0) a = (long long)((long double)n_particles[r] * ncta_max / total);
    a = std::max(1LL, std::min<long long>(a, ntiles[r]));
    ncta_out[r] = (int)a;
    sum += a;
  }
  // load of a run per CTA; equal loads are broken by the lower run index
  auto load = [&](int r, int a) { return (long double)n_particles[r] / a; };
  while (sum > ncta_max) {  // take from the lightest group that has more than one CTA
    int best = -1;
    for (int r = 0; r < nruns; ++r)
      if (ncta_out[r] > 1 && (best < 0 || load(r, ncta_out[r] - 1) < load(best, ncta_out[best] - 1)))
        best = r;
    if (best < 0) return FS_EINVAL;
    --ncta_out[best];
    --sum;
  }
  while (sum < ncta_max) {  // give to the heaviest group that can still grow
    int best = -1;
    for (int r = 0; r < nruns; ++r)
      if (ncta_out[r] < ntiles[r] && (best < 0 || load(r, ncta_out[r]) > load(best, ncta_out[best])))
        best = r;
    if (best < 0) break;
    ++ncta_out[best];
    ++sum;
  }
  return FS_OK;
  FS_GUARD_END
}

int fs_batch_query(int nruns, int precision, size_t* table_bytes) {
  FS_GUARD_BEGIN
  if (nruns < 1 || !table_bytes || (precision != FS_FP32 && precision != FS_FP64))
    return FS_EINVAL;
  *table_bytes = batch_table_bytes(nruns, precision);
  return FS_OK;
  FS_GUARD_END
}

int fs_batch_init(fs_handle* const* runs, int nruns, void* table_dev, size_t table_bytes,
                  fs_batch** out) {
  FS_GUARD_BEGIN
  if (!runs || nruns < 1 || !table_dev || !out) return FS_EINVAL;
  *out = nullptr;
  for (int r = 0; r < nruns; ++r) {
    if (!runs[r]) return FS_EINVAL;
    if (runs[r]->sim.sticky) return runs[r]->sim.sticky;
  }
  const Sim& s0 = runs[0]->sim;
  for (int r = 1; r < nruns; ++r) {
    const Sim& s = runs[r]->sim;
    if (s.p.precision != s0.p.precision || s.g.dim != s0.g.dim || s.stream != s0.stream)
      return FS_EINVAL;
  }
  size_t need = 0;
  fs_batch_query(nruns, s0.p.precision, &need);
  if (table_bytes < need || ((uintptr_t)table_dev % kAlign) != 0) return FS_EINVAL;
  const Ops* ops = s0.ops;
  size_t smem = 0;
  int rel = 0;
  // launch shape: every run's push_chunk and CTA cap when they agree, else
  // the library's choice
  int chunk = s0.p.push_chunk, cap = s0.p.push_ctas_per_sm;
  for (int r = 1; r < nruns; ++r) {
    if (runs[r]->sim.p.push_chunk != chunk) chunk = 0;
    if (runs[r]->sim.p.push_ctas_per_sm != cap) cap = 0;
  }
  for (int r = 0; r < nruns; ++r) {
    smem = std::max(smem, ops->batch_smem(s0.g.dim, runs[r]->sim.g.TX, runs[r]->sim.g.TY, chunk));
    if (runs[r]->sim.ph.c2inv > 0.0) rel = 1;
  }
  if (smem > 227 * 1024 - 2048) return FS_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FS_ECUDA;
  std::vector<long long> np(nruns);
  std::vector<int> nt(nruns), ncta(nruns), cls(nruns);
  for (int r = 0; r < nruns; ++r) {
    const int rc = fs_num_particles(runs[r], &np[r]);  // synchronises
    if (rc) return rc;
    nt[r] = runs[r]->sim.g.ntiles;
  }
  // classes: runs of one compiled-in tile width each, the rest together; one
  // push launch per class after another, each planned over the whole GPU
  std::vector<int> widths;  // class c's width (0: any)
  for (int r = 0; r < nruns; ++r) {
    const int tx = runs[r]->sim.g.TX;
    const int w = (s0.g.dim == 1 && s0.p.precision == FS_FP32 && !rel && chunk != 512 &&
                   (tx == 4 || tx == 8 || tx == 16)) ? tx : 0;
    int c = -1;
    for (size_t k = 0; k < widths.size(); ++k) if (widths[k] == w) c = (int)k;
    if (c < 0) { c = (int)widths.size(); widths.push_back(w); }
    cls[r] = c;
  }
  std::vector<fs_batch::Class> classes;
  int map_used = 0;
  for (size_t c = 0; c < widths.size(); ++c) {
    std::vector<int> idx;
    size_t sm_c = 0;
    for (int r = 0; r < nruns; ++r)
      if (cls[r] == (int)c) {
        idx.push_back(r);
        sm_c = std::max(sm_c, ops->batch_smem(s0.g.dim, runs[r]->sim.g.TX, runs[r]->sim.g.TY, chunk));
      }
    int occ = 0;
    if (ops->batch_setup(s0.g.dim, rel, chunk, widths[c], sm_c, &occ) != cudaSuccess || occ < 1)
      return FS_ECUDA;
    if (cap > 0) occ = std::min(occ, cap);
    // four CTAs per resident slot: the runs' groups are whole CTAs, and with
    // more, smaller CTAs than fit at once the hardware starts a waiting CTA
    // wherever one finishes, which evens out the groups' unequal loads
    const int ncta_max = std::min(nsm * occ * kBatchOversubscribe,
                                  kBatchMaxCtas / (int)widths.size());
    std::vector<long long> npc;
    std::vector<int> ntc, nc(idx.size());
    for (int r : idx) { npc.push_back(np[r]); ntc.push_back(nt[r]); }
    const int rc = fs_batch_plan((int)idx.size(), npc.data(), ntc.data(), ncta_max, nc.data());
    if (rc) return rc;
    int tot = 0;
    for (size_t k = 0; k < idx.size(); ++k) { ncta[idx[k]] = nc[k]; tot += nc[k]; }
    classes.push_back({widths[c], map_used, tot, sm_c});
    map_used += tot;
  }
  fs_batch* b = new fs_batch();
  b->runs.assign(runs, runs + nruns);
  b->stream = s0.stream;
  b->ops = ops;
  b->dim = s0.g.dim;
  b->rel = rel;
  b->chunk = chunk;
  b->smem = smem;
  b->classes = classes;
  b->rec = batch_rec_bytes(s0.p.precision);
  b->table = (char*)table_dev;
  b->map = (int2*)(b->table + batch_map_offset(nruns, s0.p.precision));
  b->pre = (int*)(b->table + batch_pre_offset(nruns, s0.p.precision));
  std::vector<char> host(need, 0);
  std::vector<int2> map;
  std::vector<int> pre(3 * ((size_t)nruns + 1), 0);
  b->tail_batched = true;
  for (int r = 0; r < nruns; ++r) {
    const Sim& s = runs[r]->sim;
    b->cur0.push_back(s.cur);
    for (int p = 0; p < 2; ++p)
      ops->fill_batch_run(&s, (s.cur + p) & 1, ncta[r],
                          host.data() + ((size_t)p * nruns + r) * b->rec);

    b->tail_batched = b->tail_batched && tail_batchable(s);
    b->n_sub_max = std::max(b->n_sub_max, s.p.n_sub);
    const int n1 = nruns + 1;
    pre[r + 1] = pre[r] + movers_blocks(s);
    pre[n1 + r + 1] = pre[n1 + r] + moments_blocks(s);
    pre[2 * n1 + r + 1] = pre[2 * n1 + r] + field1_blocks(s);
  }
  for (int k = 0; k < 3; ++k) b->nblk[k] = pre[(size_t)k * (nruns + 1) + nruns];
  for (size_t c = 0; c < classes.size(); ++c)  // the map in class order
    for (int r = 0; r < nruns; ++r)
      if (cls[r] == (int)c)
        for (int k = 0; k < ncta[r]; ++k) map.push_back(make_int2(r, k));
  b->ncta = (int)map.size();
  memcpy(host.data() + batch_map_offset(nruns, s0.p.precision), map.data(),
         sizeof(int2) * map.size());
  memcpy(host.data() + batch_pre_offset(nruns, s0.p.precision), pre.data(),
         sizeof(int) * pre.size());
  bool ok = cudaMemcpyAsync(table_dev, host.data(), need, cudaMemcpyHostToDevice, b->stream) ==
                cudaSuccess &&
            cudaStreamSynchronize(b->stream) == cudaSuccess;
  const int K = std::min(nruns, kBatchBranches);
  ok = ok && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < K; ++k) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    if (st) b->branch.push_back(st);
    if (ev) b->join.push_back(ev);
  }
  if (!ok) {
    fs_batch_destroy(b);
    return FS_ECUDA;
  }
  *out = b;
  return FS_OK;
  FS_GUARD_END
}

int fs_batch_step(fs_batch* b, int nsteps) {
  FS_GUARD_BEGIN
  if (!b || nsteps < 0) return FS_EINVAL;
  for (fs_handle* h : b->runs)
    if (h->sim.sticky) return h->sim.sticky;
  bool use_graph = true;
  for (fs_handle* h : b->runs) use_graph = use_graph && h->sim.p.use_graph;
  for (int k = 0; k < nsteps; ++k) {
    if (use_graph && b->steps_direct > 0 && !b->graphs_ready) {
      const int rc = batch_build_graphs(b);
      if (rc) {
        batch_fail(b, rc);
        return rc;
      }
    }
    cudaError_t e;
    if (b->graphs_ready) {
      e = cudaGraphLaunch(b->graph[b->parity], b->stream);
    } else {
      e = batch_enqueue(b, b->parity, b->stream);
      b->steps_direct++;
    }
    if (e != cudaSuccess) {
      batch_fail(b, FS_ECUDA);
      return FS_ECUDA;
    }
    b->parity ^= 1;
    for (fs_handle* h : b->runs) {
      Sim* s = &h->sim;
      s->cur = 1 - s->cur;
      s->step++;
      s->launches += launches_per_step(s);  // the shared push counted in each run
    }
  }
  return FS_OK;
  FS_GUARD_END
}

int fs_batch_destroy(fs_batch* b) {
  FS_GUARD_BEGIN
  if (!b) return FS_EINVAL;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int p = 0; p < 2; ++p)
    if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
  for (cudaStream_t st : b->branch) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaGetLastError();
  delete b;
  return FS_OK;
  FS_GUARD_END
}

extern "C" {

int fs_fp64_fma_rate(int iters, void* cuda_stream, double* ops_per_s) {
  FS_GUARD_BEGIN
  if (!ops_per_s || iters < 1 || iters > (1 << 24)) return FS_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fp64_fma, 256, 0) != cudaSuccess ||
      nsm < 1 || occ < 1)
    return FS_ECUDA;
  const int grid = nsm * occ;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return FS_ECUDA;
  }
  k_fp64_fma<<<grid, 256, 0, st>>>(nullptr, iters < 64 ? iters : 64, 0.5, 0.5);  // warm-up
  cudaEventRecord(e0, st);
  k_fp64_fma<<<grid, 256, 0, st>>>(nullptr, iters, 0.5, 0.5);
  cudaEventRecord(e1, st);
  float ms = 0.0f;
  const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return FS_ECUDA;
  *ops_per_s = (double)grid * 256.0 * kFmaChains * (double)iters / (ms * 1e-3);
  return FS_OK;
  FS_GUARD_END
}

int fs_selftest_wait(int limit, int* status_dev, void* cuda_stream) {
  FS_GUARD_BEGIN
  if (!status_dev || limit < 1 || limit > (1 << 20)) return FS_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int word = 0;
  if (cudaMemsetAsync(status_dev, 0, sizeof(int), st) != cudaSuccess) return FS_ECUDA;
  if (launch_wait_selftest(status_dev, limit, st) != cudaSuccess) return FS_ECUDA;
  if (cudaMemcpyAsync(&word, status_dev, sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FS_ECUDA;
  return status_to_code(word);
  FS_GUARD_END
}

const char* fs_strerror(int status) {
  switch (status) {
    case FS_OK: return "ok";
    case FS_EINVAL: return "invalid argument";
    case FS_ECAPACITY: return "particle capacity exhausted";
    case FS_ENAN: return "non-finite particle motion";
    case FS_EIDOVERFLOW: return "particle id overflow";
    case FS_ECUDA: return "CUDA error";
    case FS_ETIMEOUT: return "device wait timed out";
    case FS_EUNSTABLE: return "field solve unstable";
    case FS_ENOMEM: return "host memory exhausted";
    case FS_EBADCELL: return "particle outside its tile";
  }
  return "unknown status";
}

}  // extern "C"
