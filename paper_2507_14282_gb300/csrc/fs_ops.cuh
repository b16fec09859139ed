// fs_ops.cuh -- launch side of the kernels for one arithmetic type T:
// fills the Ops table used by the C ABI. Instantiated by fs_f32.cu and
// fs_f64.cu (the latter compiled with -fmad=false).
#pragma once
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "fs_push.cuh"
#include "fs_spectra.cuh"

namespace fsx {

// one thread per element up to 64 blocks per SM (every kernel launched with
// it strides over the rest)
inline int grid_for(long long n, int block = kBlock) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152LL * 64) g = 152LL * 64;
  return (int)g;
}

template <typename T, int DIM, int CH, int NS, bool REL, int TXC = 0, int TYC = 0>
cudaError_t launch_push(Sim* s, int in, long long step) {
  const PushLayout<T, DIM> L(s->g.TX, s->g.TY, CH, NS);
  // per kernel instance: the largest dynamic shared memory enabled so far and
  // the occupancy at the last size asked for (host threads may share them)
  static std::mutex mu;
  static size_t attr_bytes = 0;
  static size_t occ_bytes = 0;
  static int occ_blocks_c = 1, n_sm_c = 0;
  int occ_blocks, n_sm;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (L.bytes > attr_bytes) {
      cudaError_t e = cudaFuncSetAttribute(k_push<T, DIM, CH, NS, REL, TXC, TYC>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)L.bytes);
      if (e != cudaSuccess) return e;
      attr_bytes = L.bytes;
    }
    if (L.bytes != occ_bytes) {
      int dev = 0, nsm = 0, occ = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_push<T, DIM, CH, NS, REL, TXC, TYC>,
                                                          kBlock, L.bytes);
      if (e != cudaSuccess) return e;
      if (occ < 1) return cudaErrorInvalidConfiguration;
      n_sm_c = nsm;
      occ_blocks_c = occ;
      occ_bytes = L.bytes;
    }
    occ_blocks = occ_blocks_c;
    n_sm = n_sm_c;
  }
  StepArgs a;
  a.g = s->g;
  a.ph = s->ph;
  a.in = in;
  a.out = 1 - in;
  a.step = step;
  const int per_sm = s->g.push_ctas > 0 ? std::min(occ_blocks, s->g.push_ctas) : occ_blocks;
  const long long want = (long long)n_sm * per_sm;
  const int grid = (int)std::min<long long>(want, s->g.ntiles);
  k_push<T, DIM, CH, NS, REL, TXC, TYC><<<grid, kBlock, L.bytes, s->stream>>>(
      s->ptrs<T>(), a, push_const<T>(s->ph));
  return cudaGetLastError();
}

// shared-memory chunk (particles) and pipeline stages per precision
template <typename T>
struct PushShape;
template <>
struct PushShape<float> {
  static constexpr int kChunkSmall = 512, kStagesSmall = 3;
  static constexpr int kChunkLarge = 576, kStagesLarge = 2;
};
template <>
struct PushShape<double> {
  static constexpr int kChunkSmall = 512, kStagesSmall = 2;
  static constexpr int kChunkLarge = 512, kStagesLarge = 2;
};

template <typename T, int DIM>
cudaError_t push_dispatch(Sim* s, int in, long long step) {
  using S = PushShape<T>;
  // the relativistic terms are compiled in only for runs with a finite c
  if (s->ph.c2inv > 0.0) {
    if (s->g.chunk == S::kChunkSmall)
      return launch_push<T, DIM, S::kChunkSmall, S::kStagesSmall, true>(s, in, step);
    return launch_push<T, DIM, S::kChunkLarge, S::kStagesLarge, true>(s, in, step);
  }
  if (s->g.chunk == S::kChunkSmall)
    return launch_push<T, DIM, S::kChunkSmall, S::kStagesSmall, false>(s, in, step);
  // The 2D FP32 tile shape the library picks at 64 ppc (4 x 2 cells), compiled
  // in: every layout offset and tile constant of the push becomes an
  // immediate (7.11 -> 6.67 ms on the 268 M-particle precision form; the
  // FP64 push, bound by its FP64 pipe, gains nothing from the same).
  if constexpr (DIM == 2 && sizeof(T) == 4) {
    if (s->g.TX == 4 && s->g.TY == 2)
      return launch_push<T, DIM, S::kChunkLarge, S::kStagesLarge, false, 4, 2>(s, in, step);
  }
  return launch_push<T, DIM, S::kChunkLarge, S::kStagesLarge, false>(s, in, step);
}

template <typename T>
struct OpsImpl {
  static DevPtrs<T> P(Sim* s) { return s->ptrs<T>(); }

  static cudaError_t init_particles(Sim* s) {
    const long long total = (long long)s->g.nx * s->g.ny * s->p.ppc;
    if (s->g.dim == 1)
      k_init_particles<T, 1><<<grid_for(total), kBlock, 0, s->stream>>>(P(s), s->g, s->ph, s->cur, s->p.ppc);
    else
      k_init_particles<T, 2><<<grid_for(total), kBlock, 0, s->stream>>>(P(s), s->g, s->ph, s->cur, s->p.ppc);
    return cudaGetLastError();
  }

  static cudaError_t deposit_all(Sim* s, int buf) {
    using A = typename Num<T>::acc;
    const size_t na = (size_t)s->g.ntiles * 4 * s->g.na;
    cudaError_t e = cudaMemsetAsync(s->base + s->L.partial, 0, na * sizeof(A), s->stream);
    if (e != cudaSuccess) return e;
    if (s->g.dim == 1)
      k_deposit_all<T, 1><<<s->g.ntiles, kBlock, 0, s->stream>>>(P(s), s->g, s->ph, buf);
    else
      k_deposit_all<T, 2><<<s->g.ntiles, kBlock, 0, s->stream>>>(P(s), s->g, s->ph, buf);
    return cudaGetLastError();
  }

  static cudaError_t moments(Sim* s) {
    const long long nn = (long long)s->g.nxn * s->g.ny;
    const Geo& g = s->g;
    // the tile shapes the library picks for the 2D workloads (FP32 4 x 2 at
    // 64 ppc, FP64 8 x 4 at 16 ppc), compiled in, for boxes with x walls that
    // are more than a tile's accumulator high and more than three tile rows
    const bool ct = g.dim == 2 && g.bc_x != FS_BC_PERIODIC && g.ny >= 2 * (g.TY + 3) && g.nty > 3;
    if (g.dim == 1)
      k_moments<T, 1><<<grid_for(nn), kBlock, 0, s->stream>>>(P(s), g, s->ph);
    else if (ct && g.TX == 4 && g.TY == 2)
      k_moments_ct<T, 4, 2><<<grid_for(nn), kBlock, 0, s->stream>>>(P(s), g, s->ph);
    else if (ct && g.TX == 8 && g.TY == 4)
      k_moments_ct<T, 8, 4><<<grid_for(nn), kBlock, 0, s->stream>>>(P(s), g, s->ph);
    else
      k_moments<T, 2><<<grid_for(nn), kBlock, 0, s->stream>>>(P(s), g, s->ph);
    return cudaGetLastError();
  }

  // pre: the per-step density terms (k_ohm_pre), or nullptr to form them here
  static void ohm(Sim* s, const T* Bc, T* Eo, T* Bbo, T* G, const T* pre = nullptr) {
    DevPtrs<T> d = P(s);
    const long long nn = (long long)s->g.nxn * s->g.ny;
    if (s->g.dim == 1)
      k_ohm<T, 1><<<grid_for(nn), kBlock, 0, s->stream>>>(Bc, d.n, d.u, pre, Eo, Bbo, G, s->g,
                                                          s->ph);
    else
      k_ohm<T, 2><<<grid_for(nn), kBlock, 0, s->stream>>>(Bc, d.n, d.u, pre, Eo, Bbo, G, s->g,
                                                          s->ph);
  }

  static void faraday(Sim* s, int stage) {
    DevPtrs<T> d = P(s);
    const long long nc = (long long)s->g.nx * s->g.ny;
    if (s->g.dim == 1)
      k_faraday<T, 1><<<grid_for(nc), kBlock, 0, s->stream>>>(d.Es, d.B, d.Bs, d.Bsum, stage, s->g, s->ph);
    else
      k_faraday<T, 2><<<grid_for(nc), kBlock, 0, s->stream>>>(d.Es, d.B, d.Bs, d.Bsum, stage, s->g, s->ph);
  }

  static cudaError_t ohm_final(Sim* s) {
    DevPtrs<T> d = P(s);
    ohm(s, d.B, d.E, d.Bb, d.G);
    return cudaGetLastError();
  }

  // FP32 2D boxes with x walls: each RK4 substep in one tiled launch
  // (k_field_substep2); B alternates with the stage buffer Bs, which that
  // path does not otherwise use.
  static cudaError_t fields_tiled(Sim* s) {
    static_assert(sizeof(T) == 4, "the tiled field advance is the FP32 path");
    DevPtrs<T> d = P(s);
    constexpr size_t smem = field_tile_smem<T>();
    static std::atomic<bool> attr(false);  // set once per process; setting it twice is harmless
    if (!attr.load()) {
      for (auto k : {k_field_substep2<T, -2>, k_field_substep2<T, -1>, k_field_substep2<T, 0>,
                     k_field_substep2<T, 1>}) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
      }
      attr.store(true);
    }
    const int gx = (s->g.nx + kFTX - 1) / kFTX, gy = (s->g.ny + kFTY - 1) / kFTY;
    // interior tile columns (full, halo inside the box): 1 .. gx - 2 when the
    // box is a whole number of tiles and rows; the rest take the general form
    const bool split = gx >= 3 && s->g.nx % kFTX == 0 && s->g.ny % kFTY == 0 &&
                       kFTX >= kFH;
    T* src = d.B;
    T* dst = d.Bs;
    const FieldConst<T> fc = field_const<T>(s->ph);
    for (int sub = 0; sub < s->p.n_sub; ++sub) {
      const int fin = (sub + 1 == s->p.n_sub) ? 1 : 0;
      if (split) {
        const dim3 gi(gx - 2, gy), ge(2, gy);
        // the two wall columns (few CTAs) on the third stream beside the
        // interior launch, joined before the next substep
        const bool side = s->side2 && s->ev_fork2 && s->ev_join2;
        cudaStream_t es = s->stream;
        if (side) {
          cudaError_t e0 = cudaEventRecord(s->ev_fork2, s->stream);
          if (e0 == cudaSuccess) e0 = cudaStreamWaitEvent(s->side2, s->ev_fork2, 0);
          if (e0 != cudaSuccess) return e0;
          es = s->side2;
        }
        k_field_substep2<T, -1><<<ge, kBlock, smem, es>>>(src, dst, d.n, d.u, d.E, d.Bb, d.G,
                                                          s->g, s->ph, fc, fin, 0, gx - 1);
        if (side) {
          const cudaError_t e0 = cudaEventRecord(s->ev_join2, s->side2);
          if (e0 != cudaSuccess) return e0;
        }
        // the substeps before the last need a halo of kFH - 1 cells only: their
        // smaller shared memory lets four CTAs share an SM
        constexpr size_t smem0 =
            sizeof(T) * (9 * (size_t)(kFTX + 2 * (kFH - 1)) * (kFTY + 2 * (kFH - 1)) +
                         3 * (size_t)(kFTX + 2 * (kFH - 1) + 1) * (kFTY + 2 * (kFH - 1) + 1));
        if (fin)
          k_field_substep2<T, 1><<<gi, kBlock, smem, s->stream>>>(src, dst, d.n, d.u, d.E, d.Bb,
                                                                d.G, s->g, s->ph, fc, fin, 1, 0);
        else
          k_field_substep2<T, 0><<<gi, kBlock, smem0, s->stream>>>(src, dst, d.n, d.u, d.E, d.Bb,
                                                                 d.G, s->g, s->ph, fc, fin, 1, 0);
        if (side) {
          const cudaError_t e0 = cudaStreamWaitEvent(s->stream, s->ev_join2, 0);
          if (e0 != cudaSuccess) return e0;
        }
      } else {
        const dim3 grid(gx, gy);
        // every column: the general form
        k_field_substep2<T, -2><<<grid, kBlock, smem, s->stream>>>(src, dst, d.n, d.u, d.E, d.Bb,
                                                                 d.G, s->g, s->ph, fc, fin, 0, 0);
      }
      std::swap(src, dst);
    }
    if (src != d.B)  // odd n_sub: the field ended in the stage buffer
      return cudaMemcpyAsync(d.B, src, 3 * sizeof(T) * (size_t)s->g.nx * s->g.ny,
                             cudaMemcpyDeviceToDevice, s->stream);
    return cudaGetLastError();
  }

  // 1D boxes with x walls: the whole field advance in one tiled launch
  // (k_field_step1), the new B written to the stage buffer and copied back.
  static cudaError_t fields_tiled1(Sim* s) {
    DevPtrs<T> d = P(s);
    const size_t smem = field1_smem<T>(s->p.n_sub);
    // the largest size enabled so far; a raise races harmlessly (each caller
    // sets at least its own size before it launches)
    static std::atomic<size_t> attr(0);
    if (smem > attr.load()) {
      cudaError_t e = cudaFuncSetAttribute(k_field_step1<T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      size_t cur = attr.load();
      while (smem > cur && !attr.compare_exchange_weak(cur, smem)) {
      }
    }
    const int grid = (s->g.nx + kF1 - 1) / kF1;
    k_field_step1<T><<<grid, kF1Threads, smem, s->stream>>>(d.B, d.Bs, d.n, d.u, d.E, d.Bb, d.G,
                                                           s->g, s->ph, field_const<T>(s->ph),
                                                           s->p.n_sub);
    return cudaMemcpyAsync(d.B, d.Bs, 3 * sizeof(T) * (size_t)s->g.nx, cudaMemcpyDeviceToDevice,
                           s->stream);
  }

  static cudaError_t fields(Sim* s) {
    if (s->g.dim == 1 && s->g.bc_x != FS_BC_PERIODIC && s->p.n_sub <= 16) return fields_tiled1(s);
    if constexpr (sizeof(T) == 4) {
      if (s->g.dim == 2 && s->g.bc_x != FS_BC_PERIODIC) return fields_tiled(s);
    }
    DevPtrs<T> d = P(s);
    // FP64 (bound by the FP64 pipe): 1/n and the pressure terms once per
    // step; FP32 (bound by memory) forms them in every stage instead
    const T* pre = nullptr;
    if (sizeof(T) == 8) {
      const long long nn = (long long)s->g.nxn * s->g.ny;
      if (s->g.dim == 1)
        k_ohm_pre<T, 1><<<grid_for(nn), kBlock, 0, s->stream>>>(d.n, d.pre, s->g, s->ph);
      else
        k_ohm_pre<T, 2><<<grid_for(nn), kBlock, 0, s->stream>>>(d.n, d.pre, s->g, s->ph);
      pre = d.pre;
    }
    for (int sub = 0; sub < s->p.n_sub; ++sub) {
      ohm(s, d.B, d.Es, nullptr, nullptr, pre);
      faraday(s, 1);
      ohm(s, d.Bs, d.Es, nullptr, nullptr, pre);
      faraday(s, 2);
      ohm(s, d.Bs, d.Es, nullptr, nullptr, pre);
      faraday(s, 3);
      ohm(s, d.Bs, d.Es, nullptr, nullptr, pre);
      faraday(s, 4);
    }
    ohm(s, d.B, d.E, d.Bb, d.G, pre);
    return cudaGetLastError();
  }

  // Everything of a step after the push (movers, injection, moments, field
  // advance, step counter); ev as in step().
  static cudaError_t step_rest(Sim* s, int in, cudaEvent_t* ev) {
    DevPtrs<T> d = P(s);
    const int out = 1 - in;
    auto mark = [&](int k) {
      if (ev) cudaEventRecord(ev[k], s->stream);
    };
    const int mg = std::min((s->g.ntiles + 7) / 8, 152 * 16);
    // without phase events, the movers (buckets) run on the side stream
    // beside the injection, moments and field advance, which read no bucket
    const bool split = !ev && s->side && s->ev_fork && s->ev_join;
    cudaStream_t mst = s->stream;
    if (split) {
      cudaError_t e0 = cudaEventRecord(s->ev_fork, s->stream);
      if (e0 == cudaSuccess) e0 = cudaStreamWaitEvent(s->side, s->ev_fork, 0);
      if (e0 != cudaSuccess) return e0;
      mst = s->side;
    }
    if (s->g.dim == 1)
      k_movers<T, 1><<<mg, kBlock, 0, mst>>>(d, s->g, out);
    else
      k_movers<T, 2><<<mg, kBlock, 0, mst>>>(d, s->g, out);
    if (split) {
      const cudaError_t e0 = cudaEventRecord(s->ev_join, s->side);
      if (e0 != cudaSuccess) return e0;
    }
    mark(2);
    if (s->g.bc_x == FS_BC_FAUXSHOCK && (s->ph.inject_thermal || s->ph.cr_enable)) {
      int* rowcnt = d.inj;
      int* rowoff = rowcnt + s->g.ny;
      const int mult = (s->ph.inject_thermal ? 1 : 0) + (s->ph.cr_enable ? 1 : 0);
      k_inject_count<<<1, 1024, 0, s->stream>>>(d.acc, rowcnt, rowoff, s->g.ny, s->ph.rate, mult);
      const int maxk = (int)s->ph.rate + 2;
      const long long nthreads = (long long)s->g.ny * maxk;
      const int blocks = (int)((nthreads + kBlock - 1) / kBlock);
      if (s->g.dim == 1)
        k_inject_gen<T, 1><<<blocks, kBlock, 0, s->stream>>>(d, s->g, s->ph, out, rowcnt, rowoff, maxk);
      else
        k_inject_gen<T, 2><<<blocks, kBlock, 0, s->stream>>>(d, s->g, s->ph, out, rowcnt, rowoff, maxk);
      k_inject_commit<<<1, 32, 0, s->stream>>>(d.ctr, rowoff, s->g.ny);
    }
    mark(3);
    cudaError_t e = moments(s);
    if (e != cudaSuccess) return e;
    mark(4);
    e = fields(s);
    if (split) {
      const cudaError_t e0 = cudaStreamWaitEvent(s->stream, s->ev_join, 0);
      if (e0 != cudaSuccess) return e0;
    }
    k_step_end<<<1, 32, 0, s->stream>>>(d.ctr);
    mark(5);
    return e;
  }

  static cudaError_t step(Sim* s, int in, long long step, cudaEvent_t* ev) {
    if (ev) cudaEventRecord(ev[0], s->stream);
    const cudaError_t e =
        (s->g.dim == 1) ? push_dispatch<T, 1>(s, in, step) : push_dispatch<T, 2>(s, in, step);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s->stream);
    return step_rest(s, in, ev);
  }

  // ---- batched ensembles: one push launch over every run's CTA group
  static size_t batch_run_bytes() { return sizeof(BatchRun<T>); }
  static void fill_batch_run(const Sim* s, int in, int ncta, void* dst) {
    BatchRun<T> r;
    r.d = const_cast<Sim*>(s)->ptrs<T>();
    r.g = s->g;
    r.ph = s->ph;
    r.pc = push_const<T>(s->ph);
    r.in = in;
    r.out = 1 - in;
    r.ncta = ncta;
    r.n_sub = s->p.n_sub;
    memcpy(dst, &r, sizeof r);
  }
  // chunk: 0 or the large chunk (PushShape::kChunkLarge, its stages), or
  // the small chunk (kChunkSmall, its stages) for every run of the batch
  static bool batch_small(int chunk) {
    using S = PushShape<T>;
    return chunk == S::kChunkSmall && S::kChunkSmall != S::kChunkLarge;
  }
  static size_t batch_smem(int dim, int tx, int ty, int chunk) {
    using S = PushShape<T>;
    const int ch = batch_small(chunk) ? S::kChunkSmall : S::kChunkLarge;
    const int ns = batch_small(chunk) ? S::kStagesSmall : S::kStagesLarge;
    return dim == 1 ? PushLayout<T, 1>(tx, ty, ch, ns).bytes
                    : PushLayout<T, 2>(tx, ty, ch, ns).bytes;
  }
  template <int DIM, int CH, int NS, bool REL, int TXC = 0>
  static cudaError_t batch_kernel_setup(size_t smem, int* occ) {
    auto kern = k_push_batch<T, DIM, CH, NS, REL, TXC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess && occ)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, kBlock, smem);
    return e;
  }
  template <int CH, int NS>
  static cudaError_t batch_setup_shape(int dim, int rel, size_t smem, int* occ) {
    if (rel)
      return dim == 1 ? batch_kernel_setup<1, CH, NS, true>(smem, occ)
                      : batch_kernel_setup<2, CH, NS, true>(smem, occ);
    return dim == 1 ? batch_kernel_setup<1, CH, NS, false>(smem, occ)
                    : batch_kernel_setup<2, CH, NS, false>(smem, occ);
  }
  // sets the shared-memory attribute; occ (optional): CTAs per SM. rel: the
  // variant with the relativistic terms (some run has a finite c).
  // the 1D FP32 tile widths compiled into their own batched push
  static bool batch_width_compiled(int dim, int rel, int chunk, int txc) {
    return sizeof(T) == 4 && dim == 1 && !rel && !batch_small(chunk) &&
           (txc == 4 || txc == 8 || txc == 16);
  }
  static cudaError_t batch_setup(int dim, int rel, int chunk, int txc, size_t smem, int* occ) {
    using S = PushShape<T>;
    if (batch_width_compiled(dim, rel, chunk, txc)) {
      constexpr int CH = S::kChunkLarge, NS = S::kStagesLarge;
      if (txc == 4) return batch_kernel_setup<1, CH, NS, false, 4>(smem, occ);
      if (txc == 8) return batch_kernel_setup<1, CH, NS, false, 8>(smem, occ);
      return batch_kernel_setup<1, CH, NS, false, 16>(smem, occ);
    }
    if (batch_small(chunk))
      return batch_setup_shape<S::kChunkSmall, S::kStagesSmall>(dim, rel, smem, occ);
    return batch_setup_shape<S::kChunkLarge, S::kStagesLarge>(dim, rel, smem, occ);
  }
  template <int CH, int NS, bool REL>
  static void push_batch_launch(int dim, const BatchRun<T>* r, const int2* cta_map, int ncta,
                                size_t smem, cudaStream_t st) {
    if (dim == 1)
      k_push_batch<T, 1, CH, NS, REL><<<ncta, kBlock, smem, st>>>(r, cta_map);
    else
      k_push_batch<T, 2, CH, NS, REL><<<ncta, kBlock, smem, st>>>(r, cta_map);
  }
  static cudaError_t push_batch(int dim, int rel, int chunk, int txc, const void* runs,
                                const int2* cta_map, int ncta, size_t smem, cudaStream_t st) {
    using S = PushShape<T>;
    const BatchRun<T>* r = (const BatchRun<T>*)runs;
    if (batch_width_compiled(dim, rel, chunk, txc)) {
      constexpr int CH = S::kChunkLarge, NS = S::kStagesLarge;
      if (txc == 4) k_push_batch<T, 1, CH, NS, false, 4><<<ncta, kBlock, smem, st>>>(r, cta_map);
      else if (txc == 8) k_push_batch<T, 1, CH, NS, false, 8><<<ncta, kBlock, smem, st>>>(r, cta_map);
      else k_push_batch<T, 1, CH, NS, false, 16><<<ncta, kBlock, smem, st>>>(r, cta_map);
      return cudaGetLastError();
    }
    const bool sm = batch_small(chunk);
    if (rel) {
      if (sm) push_batch_launch<S::kChunkSmall, S::kStagesSmall, true>(dim, r, cta_map, ncta, smem, st);
      else push_batch_launch<S::kChunkLarge, S::kStagesLarge, true>(dim, r, cta_map, ncta, smem, st);
    } else {
      if (sm) push_batch_launch<S::kChunkSmall, S::kStagesSmall, false>(dim, r, cta_map, ncta, smem, st);
      else push_batch_launch<S::kChunkLarge, S::kStagesLarge, false>(dim, r, cta_map, ncta, smem, st);
    }
    return cudaGetLastError();
  }

  // the rest of a batched step over every run (all 1D with x walls)
  static cudaError_t batch_rest(const void* runs, const int* pre, int nruns, const int* nblk,
                                int n_sub_max, cudaStream_t st, cudaStream_t side,
                                cudaEvent_t fork, cudaEvent_t join) {
    const BatchRun<T>* r = (const BatchRun<T>*)runs;
    const size_t fsm = field1_smem<T>(n_sub_max);
    static std::atomic<size_t> attr(0);  // the largest size enabled so far
    if (fsm > attr.load()) {
      cudaError_t e = cudaFuncSetAttribute(k_field1_batch<T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
      if (e != cudaSuccess) return e;
      size_t cur = attr.load();
      while (fsm > cur && !attr.compare_exchange_weak(cur, fsm)) {
      }
    }
    const int n1 = nruns + 1;
    // the movers (buckets) beside the injection, moments and field advance,
    // which read no bucket: the injection appends to the buckets with its own
    // slot atomics, the moments read the deposit partials and far sums
    cudaError_t e;
    if ((e = cudaEventRecord(fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess) return e;
    k_movers_batch<T, 1><<<nblk[0], kBlock, 0, side>>>(r, pre, nruns);
    if ((e = cudaEventRecord(join, side)) != cudaSuccess) return e;
    k_inject_batch<T, 1><<<nruns, kBlock, 0, st>>>(r, nruns);
    k_moments_batch<T, 1><<<nblk[1], kBlock, 0, st>>>(r, pre + n1, nruns);
    k_field1_batch<T><<<nblk[2], kF1Threads, fsm, st>>>(r, pre + 2 * n1, nruns);
    k_copyB_batch<T><<<nblk[2], kF1Threads, 0, st>>>(r, pre + 2 * n1, nruns);
    if ((e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess) return e;
    k_step_end_batch<T><<<(nruns + 63) / 64, 64, 0, st>>>(r, nruns);
    return cudaGetLastError();
  }

  static cudaError_t insert_staged(Sim* s, int buf, int n, bool from_movers) {
    DevPtrs<T> d = P(s);
    const Parts<T> src = from_movers ? d.M : d.S;
    if (s->g.dim == 1)
      k_insert_staged<T, 1><<<grid_for(n), kBlock, 0, s->stream>>>(d, src, s->g, buf, n);
    else
      k_insert_staged<T, 2><<<grid_for(n), kBlock, 0, s->stream>>>(d, src, s->g, buf, n);
    return cudaGetLastError();
  }

  static cudaError_t diag(Sim* s, int buf) {
    DevPtrs<T> d = P(s);
    cudaError_t e = cudaMemsetAsync(d.ctr->sums, 0, sizeof(d.ctr->sums), s->stream);
    if (e != cudaSuccess) return e;
    if (s->g.dim == 1)
      k_diag_particles<T, 1><<<s->g.ntiles, kBlock, 0, s->stream>>>(d, s->g, s->ph, buf);
    else
      k_diag_particles<T, 2><<<s->g.ntiles, kBlock, 0, s->stream>>>(d, s->g, s->ph, buf);
    k_diag_field<T><<<grid_for((long long)s->g.nx * s->g.ny), kBlock, 0, s->stream>>>(d, s->g, s->ph);
    return cudaGetLastError();
  }

  static cudaError_t hist(Sim* s, int buf, int species) {
    DevPtrs<T> d = P(s);
    cudaError_t e = cudaMemsetAsync(d.hist, 0,
                                    sizeof(unsigned long long) * s->ph.hist_nx * s->ph.hist_np,
                                    s->stream);
    if (e != cudaSuccess) return e;
    if (s->g.dim == 1)
      k_hist<T, 1><<<s->g.ntiles, kBlock, 0, s->stream>>>(d, s->g, s->ph, buf, species);
    else
      k_hist<T, 2><<<s->g.ntiles, kBlock, 0, s->stream>>>(d, s->g, s->ph, buf, species);
    return cudaGetLastError();
  }

  static double* profile_region(Sim* s) { return (double*)(s->base + s->L.prof); }

  static cudaError_t profile_B(Sim* s) {
    const int nx = s->g.nx;
    double* out = profile_region(s) + s->g.nxn + nx;
    k_profile_B<T><<<grid_for(nx), kBlock, 0, s->stream>>>(P(s).B, nx, s->g.ny, out);
    return cudaGetLastError();
  }

  static cudaError_t spectrum_bperp(Sim* s) {
    const int nx = s->g.nx, ny = s->g.ny;
    double* out = profile_region(s) + s->g.nxn + 4 * (size_t)nx;
    cudaError_t e = cudaMemsetAsync(out, 0, 8 * ((size_t)nx / 2 + 1), s->stream);
    if (e != cudaSuccess) return e;
    const bool pow2 = (nx & (nx - 1)) == 0;
    if (pow2 && nx <= kFftMax) {
      int logn = 0;
      while ((1 << logn) < nx) ++logn;
      const size_t smem = sizeof(double2) * (size_t)nx;
      e = cudaFuncSetAttribute(k_bperp_fft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return e;
      k_bperp_fft<T><<<ny, kFftThreads, smem, s->stream>>>(P(s).B, nx, ny, logn, out);
    } else {
      const long long work = (long long)(nx / 2 + 1) * ny;
      k_bperp_dft<T><<<grid_for(work), kBlock, 0, s->stream>>>(P(s).B, nx, ny, out);
    }
    return cudaGetLastError();
  }

  static cudaError_t spectrum_p(Sim* s, int buf, int species) {
    const int np = s->p.spec_np;
    const double* e = (const double*)(s->base + s->L.spec);
    unsigned long long* out = (unsigned long long*)(s->base + s->L.spec + 8 * ((size_t)np + 1));
    cudaError_t err = cudaMemsetAsync(out, 0, 8 * (size_t)np, s->stream);
    if (err != cudaSuccess) return err;
    k_spectrum_p<T><<<s->g.ntiles, kBlock, 0, s->stream>>>(P(s), s->g, buf, species, np, e, out);
    return cudaGetLastError();
  }

  static cudaError_t profiles(Sim* s) {
    k_profiles<T><<<grid_for(s->g.nxn), kBlock, 0, s->stream>>>(P(s), s->g, s->ph);
    return cudaGetLastError();
  }

  static cudaError_t export_grid(Sim* s, int what, double* dst) {
    DevPtrs<T> d = P(s);
    const T* src = nullptr;
    int planes = 3, cols = s->g.nxn;
    switch (what) {
      case FS_B: src = d.B; cols = s->g.nx; break;
      case FS_E: src = d.E; break;
      case FS_BBAR: src = d.Bb; break;
      case FS_N: src = d.n; planes = 1; break;
      case FS_J: src = d.J; break;
      case FS_U: src = d.u; break;
      default: return cudaErrorInvalidValue;
    }
    const long long n = (long long)cols * s->g.ny;
    k_export_grid<T><<<grid_for(n), kBlock, 0, s->stream>>>(src, planes, cols, s->g.ny, dst);
    return cudaGetLastError();
  }

  static cudaError_t import_B(Sim* s, const double* src) {
    const int nc = s->g.nx * s->g.ny;
    k_import_B<T><<<grid_for(nc), kBlock, 0, s->stream>>>(P(s).B, src, nc);
    return cudaGetLastError();
  }

  static cudaError_t export_particles(Sim* s, int buf, double* dst, int* cell,
                                      uint32_t* id, int* count) {
    if (s->g.dim == 1)
      k_export_particles<T, 1><<<s->g.ntiles, kBlock, 0, s->stream>>>(P(s), s->g, buf, dst, cell, id, count);
    else
      k_export_particles<T, 2><<<s->g.ntiles, kBlock, 0, s->stream>>>(P(s), s->g, buf, dst, cell, id, count);
    return cudaGetLastError();
  }

  static Ops make() {
    Ops o;
    o.init_particles = init_particles;
    o.deposit_all = deposit_all;
    o.moments = moments;
    o.ohm_final = ohm_final;
    o.step = step;
    o.fields = fields;
    o.insert_staged = insert_staged;
    o.diag = diag;
    o.hist = hist;
    o.profiles = profiles;
    o.export_grid = export_grid;
    o.import_B = import_B;
    o.step_rest = step_rest;
    o.batch_run_bytes = batch_run_bytes;
    o.fill_batch_run = fill_batch_run;
    o.batch_smem = batch_smem;
    o.batch_setup = batch_setup;
    o.push_batch = push_batch;
    o.batch_rest = batch_rest;
    o.profile_B = profile_B;
    o.spectrum_bperp = spectrum_bperp;
    o.spectrum_p = spectrum_p;
    o.export_particles = export_particles;
    return o;
  }
};

template <typename T>
size_t push_smem_bytes(int dim, int tx, int ty, int chunk) {
  using S = PushShape<T>;
  const int ns = (chunk == S::kChunkSmall) ? S::kStagesSmall : S::kStagesLarge;
  return dim == 1 ? PushLayout<T, 1>(tx, ty, chunk, ns).bytes
                  : PushLayout<T, 2>(tx, ty, chunk, ns).bytes;
}

}  // namespace fsx
