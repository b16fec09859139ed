// fs_push.cuh -- the fused particle step (gather, Boris, move, open wall,
// faux shock, in-tile counting sort, CIC deposit), one persistent CTA per
// group of tiles with the next chunk of particles prefetched into shared
// memory by the TMA bulk-copy engine while the current one is processed.
//
// Per chunk (at most CH particles of one tile):
//   1. wait for the chunk's bulk copies (its particle columns and the tile's
//      packed E / Bbar nodes) on an mbarrier;
//   2. push every particle in shared memory in place and give it a sort key:
//      its new cell in the tile (interior cells first), a halo cell, FAR
//      (moved more than one cell out of the tile) or REMOVED;
//   3. deposit in push order, warp-cooperatively: the particles of a warp
//      mostly share one cell, and for each distinct cell a transpose
//      reduction of the lanes' corner contributions leaves one sum per value
//      to add to the tile's node accumulator;
//   4. counting sort: per-key counts and in-key ranks -> offsets by a warp
//      scan;
//   5. every thread writes its own particles at offset + rank: stayers to the
//      tile's bucket of the output buffer in cell order, leavers to the
//      tile's range of the mover list.
// When a tile's last chunk is done its node accumulator is written out as
// the tile's deposit partial (summed per node in a fixed order later).
#pragma once
#include "fs_engine.cuh"

namespace fsx {

// ---------------------------------------------------------------- PTX glue
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// one bulk copy global -> shared, completion counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], "
      "%2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 4-byte asynchronous global -> shared copy (no register holds the value)
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// bounded wait: false if the phase did not complete within the limit
constexpr int kWaitLimit = 1 << 20;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

struct StepArgs {
  Geo g;
  Phys ph;
  int in, out;
  long long step;
};

// ---------------------------------------------------------------- layout
constexpr int kMaxStages = 4;

template <typename T, int DIM>
struct PushLayout {
  int TX, TY, NFX, NFY, AX, AY, NA, EX, EY, NE, NINT, NK, CH, NS;
  // stage 0's regions; stage b sits b * bstride bytes further
  size_t F[1], cell[1], ox[1], oy[1], vx[1], vy[1], vz[1], id[1];
  size_t acc, kc, ko, e2k, k2e, desc, bar, pf, bytes;
  size_t bstride;  // distance between the two chunk buffers
  __host__ __device__ static size_t take(size_t& o, size_t n) {
    o = (o + 15) / 16 * 16;
    const size_t r = o;
    o += n;
    return r;
  }
  __host__ __device__ PushLayout(int tx_, int ty_, int ch, int ns) {
    TX = tx_;
    TY = (DIM == 2) ? ty_ : 1;
    NFX = TX + 1;
    NFY = (DIM == 2) ? TY + 1 : 1;
    AX = TX + 3;
    AY = (DIM == 2) ? TY + 3 : 1;
    NA = AX * AY;
    EX = TX + 2;
    EY = (DIM == 2) ? TY + 2 : 1;
    NE = EX * EY;
    NINT = TX * TY;
    NK = NE + 2;
    CH = ch;
    NS = ns;
    size_t o = 0;
    bar = take(o, kMaxStages * sizeof(unsigned long long));
    desc = take(o, (kMaxStages + 1) * sizeof(int4));
    F[0] = take(o, sizeof(T) * 8 * NFX * NFY);
    cell[0] = take(o, sizeof(int) * CH);
    ox[0] = take(o, sizeof(T) * CH);
    oy[0] = take(o, DIM == 2 ? sizeof(T) * CH : 0);
    vx[0] = take(o, sizeof(T) * CH);
    vy[0] = take(o, sizeof(T) * CH);
    vz[0] = take(o, sizeof(T) * CH);
    id[0] = take(o, sizeof(uint32_t) * CH);
    o = (o + 15) / 16 * 16;
    bstride = o - F[0];
    o += (size_t)(NS - 1) * bstride;
    pf = take(o, 16);
    acc = take(o, sizeof(typename Num<T>::acc) * 4 * NA);
    kc = take(o, sizeof(int) * NK);
    ko = take(o, sizeof(int) * (NK + 1));
    e2k = take(o, sizeof(uint16_t) * NE);
    k2e = take(o, sizeof(int) * NE);
    bytes = (o + 127) / 128 * 128;
  }
  // bytes one chunk of m particles brings in
  __host__ __device__ uint32_t chunk_bytes(int m) const {
    const uint32_t m4 = (uint32_t)((m + 3) & ~3);
    const uint32_t per = 4u + (uint32_t)sizeof(T) * (DIM == 2 ? 5u : 4u) + 4u;
    return (uint32_t)(sizeof(T) * 8 * NFX) * NFY + m4 * per;
  }
};

// exclusive scan of n ints by one warp (lanes of warp w); out[n] = total
__device__ __forceinline__ void warp_scan_excl(const int* in, int* out, int n,
                                               int lane) {
  const int per = (n + 31) / 32;
  const int b = lane * per, e = min(b + per, n);
  int s = 0;
  for (int k = b; k < e; ++k) s += in[k];
  int inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  int run = inc - s;
  for (int k = b; k < e; ++k) {
    out[k] = run;
    run += in[k];
  }
  if (lane == 31) out[n] = inc;
}

// The chunk after c = {tile, first particle, count, tile count} for a CTA
// that owns tiles blockIdx.x, blockIdx.x + G, ...; tile >= ntiles: done.
// pf[0] holds the count of tile c.x + G, copied asynchronously into shared
// memory one tile transition earlier; the count of the tile after it is
// requested now.
__device__ __forceinline__ int4 next_chunk(int4 c, int G, int ntiles, int CH,
                                           const int* cnt_in, int cap, int* pf) {
  if (c.x >= ntiles) return c;
  if (c.y + CH < c.w) return make_int4(c.x, c.y + CH, min(CH, c.w - c.y - CH), c.w);
  const int t = c.x + G;
  if (t >= ntiles) return make_int4(ntiles, 0, 0, 0);
  cp_async_wait_all();
  const int n = min(pf[0], cap);
  if (t + G < ntiles) cp_async4(pf, cnt_in + t + G);
  return make_int4(t, 0, min(CH, n), n);
}

// ---------------------------------------------------------------- push
// One particle: CIC gather from the tile's node block F (local cell lx, ly),
// Boris, move, x walls / faux shock. Returns the sort key. Counters and
// energies are accumulated in the caller's registers.
struct PushTally {
  long long inc, tr, ref, esc;
  double fse, rem;
  int status;
};

template <typename T, int DIM>
__device__ __forceinline__ int push_one(const T* __restrict__ F, int NFX, int& cell,
                                        T& fx, T& fy, T& vx, T& vy, T& vz,
                                        uint32_t& id, int i0, int j0, int TX, int TY,
                                        int EX, int EY, int NE, const uint16_t* e2k,
                                        const Geo& g, const Phys& ph, T dtdx, T dtdy,
                                        T hdt, long long step, PushTally& tl) {
  const int i = cell & 0xFFFF, j = cell >> 16;
  const int lx = i - i0, ly = j - j0;
  if (lx < 0 || lx >= TX || ly < 0 || ly >= TY) {
    tl.status |= kStatusBadCell;
    return NE + 1;
  }
  T Ep[3], Bp[3];
  if (DIM == 1) {
    const T g0 = (T)1 - fx;
    const T* n0 = F + lx * 8;
    const T* n1 = n0 + 8;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      Ep[q] = fmaT(fx, n1[q], g0 * n0[q]);
      Bp[q] = fmaT(fx, n1[3 + q], g0 * n0[3 + q]);
    }
  } else {
    const T gx0 = (T)1 - fx, gy0 = (T)1 - fy;
    const T w00 = gx0 * gy0, w10 = fx * gy0, w01 = gx0 * fy, w11 = fx * fy;
    const T* n00 = F + (ly * NFX + lx) * 8;
    const T* n10 = n00 + 8;
    const T* n01 = n00 + NFX * 8;
    const T* n11 = n01 + 8;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      Ep[q] = fmaT(w11, n11[q], fmaT(w01, n01[q], fmaT(w10, n10[q], w00 * n00[q])));
      Bp[q] = fmaT(w11, n11[3 + q],
                   fmaT(w01, n01[3 + q], fmaT(w10, n10[3 + q], w00 * n00[3 + q])));
    }
  }
  boris<T>(vx, vy, vz, Ep, Bp, hdt);
  const T fxr = fmaT(vx, dtdx, fx);
  T fyr = fy;
  if (DIM == 2) fyr = fmaT(vy, dtdy, fy);
  // whole-cell shift floor(f): by comparison for |shift| <= 1 (the common
  // case), by floor otherwise; the same value either way
  T kx, ky = (T)0;
  bool far_shift = false;
  if (fxr >= (T)0 && fxr < (T)1) kx = (T)0;
  else if (fxr >= (T)1 && fxr < (T)2) kx = (T)1;
  else if (fxr < (T)0 && fxr >= (T)-1) kx = (T)-1;
  else { kx = Num<T>::fl(fxr); far_shift = true; }
  if (DIM == 2) {
    if (fyr >= (T)0 && fyr < (T)1) ky = (T)0;
    else if (fyr >= (T)1 && fyr < (T)2) ky = (T)1;
    else if (fyr < (T)0 && fyr >= (T)-1) ky = (T)-1;
    else { ky = Num<T>::fl(fyr); far_shift = true; }
  }
  // a shift of more than one cell: reject non-finite or absurd motion
  if (far_shift && (!(Num<T>::ab(kx) < (T)1.0e9) || !(Num<T>::ab(ky) < (T)1.0e9))) {
    tl.status |= kStatusNaN;
    return NE + 1;
  }
  const T offmax = Num<T>::offmax;
  const int ikx = (kx == (T)0) ? 0 : (kx == (T)1) ? 1 : (kx == (T)-1) ? -1 : (int)kx;
  int inew = i + ikx;
  T fxn = fxr - kx;
  if (fxn >= (T)1) fxn = offmax;
  int jraw = j, jnew = j;
  T fyn = fy;
  if (DIM == 2) {
    const int iky = (ky == (T)0) ? 0 : (ky == (T)1) ? 1 : (ky == (T)-1) ? -1 : (int)ky;
    jraw = j + iky;
    jnew = jraw;
    if (jnew < 0 || jnew >= g.ny) {
      jnew = (jnew < 0 && jnew >= -g.ny) ? jnew + g.ny
             : (jnew >= g.ny && jnew < 2 * g.ny) ? jnew - g.ny
                                                 : wrap(jnew, g.ny);
    }
    fyn = fyr - ky;
    if (fyn >= (T)1) fyn = offmax;
  }
  const bool cr = (id & kIdCR) != 0;
  int iunw = inew;
  if (g.bc_x == FS_BC_PERIODIC) {
    if (inew < 0 || inew >= g.nx) inew = wrap(inew, g.nx);
  } else if (inew >= g.nx) {
    ++tl.esc;
    tl.rem += kinetic(cr ? ph.w_cr : ph.w_th, (double)vx, (double)vy, (double)vz,
                      ph.cellvol);
    return NE + 1;
  } else if (inew < 0) {
    const int mode = cr ? FS_SHOCK : ph.fs_mode_thermal;
    const double wpd = cr ? ph.w_cr : ph.w_th;
    ++tl.inc;
    double dvx = vx, dvy = vy, dvz = vz;
    const double e0 = kinetic(wpd, dvx, dvy, dvz, ph.cellvol);
    if (mode == FS_SHOCK &&
        fs_return(dvx, dvy, dvz, ph.u2, ph.fs_frame, ph.seed, id & kIdMask, step)) {
      ++tl.ref;
      tl.fse = __dadd_rn(tl.fse, __dsub_rn(kinetic(wpd, dvx, dvy, dvz, ph.cellvol), e0));
      const double Xo = __dadd_rn((double)i, (double)fx);
      const double Xn = __dadd_rn((double)i, (double)fxr);
      const double gfr = __ddiv_rn(Xn, __dsub_rn(Xn, Xo));
      double f = __dmul_rn(gfr, __dmul_rn(dvx, ph.dtdx));
      if (f < 0.0) f = 0.0;
      if (f >= 1.0) f = (double)Num<double>::offmax;
      T ft = (T)f;
      if (ft >= (T)1) ft = offmax;
      fxn = ft;
      inew = 0;
      iunw = 0;
      vx = (T)dvx;
      vy = (T)dvy;
      vz = (T)dvz;
      id |= kIdReturned;
    } else {
      ++tl.tr;
      tl.rem = __dadd_rn(tl.rem, e0);
      return NE + 1;
    }
  }
  cell = (jnew << 16) | inew;
  fx = fxn;
  fy = fyn;
  const int lxn = iunw - i0 + 1;
  const int lyn = (DIM == 2) ? jraw - j0 + 1 : 0;
  if (lxn < 0 || lxn >= EX || lyn < 0 || lyn >= EY) return NE;  // FAR
  if (lxn >= 1 && lxn <= TX && (DIM == 1 || (lyn >= 1 && lyn <= TY)))
    return (lxn - 1) + (DIM == 2 ? (lyn - 1) * TX : 0);
  return e2k[lxn + lyn * EX];
}

// Thread 0 only: record chunk c as buffer b's descriptor and start the bulk
// copies of its tile's node block and particle columns.
template <typename T, int DIM>
__device__ __forceinline__ void issue_chunk(unsigned char* sm, const PushLayout<T, DIM>& L,
                                            int b, int4 c, const DevPtrs<T>& d,
                                            const Parts<T>& PI, const Geo& g) {
  int4* desc = (int4*)(sm + L.desc);
  uint64_t* bar = (uint64_t*)(sm + L.bar) + b;
  desc[b] = c;
  if (c.x >= g.ntiles || c.z <= 0) return;
  const int tx = c.x % g.ntx, ty = c.x / g.ntx;
  const int i0 = tx * L.TX, j0 = ty * L.TY;
  const size_t bo = (size_t)b * L.bstride;
  mbar_arrive_expect_tx(bar, L.chunk_bytes(c.z));
  const uint32_t row = (uint32_t)(sizeof(T) * 8 * L.NFX);
  for (int ly = 0; ly < L.NFY; ++ly)
    bulk_g2s(sm + L.F[0] + bo + (size_t)ly * row,
             d.G + ((size_t)(j0 + ly) * (g.nx + 1) + i0) * 8, row, bar);
  const size_t first = (size_t)d.tile_base[c.x] + c.y;
  const uint32_t m4 = (uint32_t)((c.z + 3) & ~3);
  bulk_g2s(sm + L.cell[0] + bo, PI.cell + first, 4 * m4, bar);
  bulk_g2s(sm + L.ox[0] + bo, PI.ox + first, sizeof(T) * m4, bar);
  if (DIM == 2) bulk_g2s(sm + L.oy[0] + bo, PI.oy + first, sizeof(T) * m4, bar);
  bulk_g2s(sm + L.vx[0] + bo, PI.vx + first, sizeof(T) * m4, bar);
  bulk_g2s(sm + L.vy[0] + bo, PI.vy + first, sizeof(T) * m4, bar);
  bulk_g2s(sm + L.vz[0] + bo, PI.vz + first, sizeof(T) * m4, bar);
  bulk_g2s(sm + L.id[0] + bo, PI.id + first, 4 * m4, bar);
}

// Warp-cooperative CIC deposit of the lanes' particles (push order): for each
// distinct cell key among the lanes, the lanes of that cell contribute their
// corner values and a transpose reduction leaves value q(L) summed over the
// warp in lane L; the owner lanes add to the tile's node accumulator.
template <typename T, int DIM>
__device__ __forceinline__ void warp_deposit(typename Num<T>::acc* ACC, int NA, int AX,
                                             const int* k2e, int key, bool active, T fx,
                                             T fy, T wp, T vx, T vy, T vz, int lane) {
  using A = typename Num<T>::acc;
  constexpr int NV = 4 * (DIM == 2 ? 4 : 2);
  unsigned todo = __ballot_sync(0xffffffffu, active);
  if (!todo) return;
  A val[NV];
  if (DIM == 1) {
    const T c0 = wp * ((T)1 - fx), c1 = wp * fx;
    val[0] = to_acc(c0); val[1] = to_acc_prod(c0, vx);
    val[2] = to_acc_prod(c0, vy); val[3] = to_acc_prod(c0, vz);
    val[4] = to_acc(c1); val[5] = to_acc_prod(c1, vx);
    val[6] = to_acc_prod(c1, vy); val[7] = to_acc_prod(c1, vz);
  } else {
    const T gx0 = (T)1 - fx, gy0 = (T)1 - fy;
    const T cw[4] = {wp * (gx0 * gy0), wp * (fx * gy0), wp * (gx0 * fy), wp * (fx * fy)};
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      val[4 * cc + 0] = to_acc(cw[cc]);
      val[4 * cc + 1] = to_acc_prod(cw[cc], vx);
      val[4 * cc + 2] = to_acc_prod(cw[cc], vy);
      val[4 * cc + 3] = to_acc_prod(cw[cc], vz);
    }
  }
  int qi = 0;
  {
    int h = NV / 2, off = 16;
    while (h >= 1) {
      if (lane & off) qi += h;
      h >>= 1;
      off >>= 1;
    }
  }
  const bool owner = (NV == 16) ? ((lane & 1) == 0) : ((lane & 3) == 0);
  while (todo) {
    const int lead = __ffs(todo) - 1;
    const int kk = __shfl_sync(0xffffffffu, key, lead);
    const bool mine = active && (key == kk);
    todo &= ~__ballot_sync(0xffffffffu, mine);
    A w[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) w[q] = mine ? val[q] : (A)0;
    int half = NV / 2;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      if (half >= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int q = 0; q < NV / 2; ++q) {
          if (q < half) {
            const A send = up ? w[q] : w[q + half];
            const A keep = up ? w[q + half] : w[q];
            w[q] = keep + shfl_xor(send, off);
          }
        }
        half >>= 1;
      } else {
        w[0] = w[0] + shfl_xor(w[0], off);
      }
    }
    if (owner) {
      const int le = k2e[kk];
      const int a00 = (le & 0xFFFF) + (le >> 16) * AX;
      const int corner = qi >> 2, qty = qi & 3;
      const int an = (DIM == 1) ? a00 + corner : a00 + (corner & 1) + (corner >> 1) * AX;
      atomic_acc(&ACC[qty * NA + an], w[0]);
    }
  }
}

template <typename T, int DIM, int CH, int NS>
__global__ void __launch_bounds__(kBlock, (sizeof(T) == 4 ? 3 : 2)) k_push(DevPtrs<T> d, StepArgs a) {
  using A = typename Num<T>::acc;
  constexpr int PPT = CH / kBlock;
  extern __shared__ __align__(128) unsigned char sm[];
  const Geo g = a.g;
  const Phys ph = a.ph;
  const PushLayout<T, DIM> L(g.TX, g.TY, CH, NS);
  const int TX = L.TX, TY = L.TY, EX = L.EX, EY = L.EY, NE = L.NE, NINT = L.NINT,
            NK = L.NK, NA = L.NA, AX = L.AX;
  uint64_t* bar = (uint64_t*)(sm + L.bar);
  int4* desc = (int4*)(sm + L.desc);
  A* ACC = (A*)(sm + L.acc);
  int* kcount = (int*)(sm + L.kc);
  int* koff = (int*)(sm + L.ko);
  uint16_t* e2k = (uint16_t*)(sm + L.e2k);
  int* k2e = (int*)(sm + L.k2e);
  int* pf = (int*)(sm + L.pf);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  const int* cnt_in = d.cnt[a.in];
  const Parts<T> PI = d.P[a.in];
  const Parts<T> PO = d.P[a.out];
  const T dtdx = (T)ph.dtdx, dtdy = (T)ph.dtdy, hdt = (T)ph.hdt;
  const T wth = (T)(ph.w_th * (double)deposit_weight_scale<T>());
  const T wcr = (T)(ph.w_cr * (double)deposit_weight_scale<T>());
  const long long step = d.ctr->step;  // device step counter (graph-replayable)

  // ---- per-CTA tables: extended cell <-> sort key; zero accumulators
  for (int e = tid; e < NE; e += kBlock) {
    const int lx = e % EX, ly = e / EX;
    const bool inx = (lx >= 1 && lx <= TX);
    const bool iny = (DIM == 1) || (ly >= 1 && ly <= TY);
    int key;
    if (inx && iny) {
      key = (lx - 1) + (DIM == 2 ? (ly - 1) * TX : 0);
    } else {
      const int before = (DIM == 1) ? min(max(lx - 1, 0), TX)
                                    : min(max(ly - 1, 0), TY) * TX +
                                          ((ly >= 1 && ly <= TY) ? min(max(lx - 1, 0), TX) : 0);
      key = NINT + e - before;
    }
    e2k[e] = (uint16_t)key;
    k2e[key] = lx | (ly << 16);
  }
  for (int k = tid; k < 4 * NA; k += kBlock) ACC[k] = (A)0;
  for (int k = tid; k < NK; k += kBlock) kcount[k] = 0;

  if (tid == 0) {
    for (int b = 0; b < NS; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    // prologue: the CTA's first NS chunks, one per stage
    int4 c;
    if ((int)blockIdx.x < g.ntiles) {
      const int n = min(cnt_in[blockIdx.x], g.tile_cap);
      c = make_int4(blockIdx.x, 0, min(CH, n), n);
    } else {
      c = make_int4(g.ntiles, 0, 0, 0);
    }
    if ((int)blockIdx.x + G < g.ntiles) cp_async4(pf, cnt_in + blockIdx.x + G);
    for (int b = 0; b < NS; ++b) {
      issue_chunk<T, DIM>(sm, L, b, c, d, PI, g);
      if (b + 1 < NS) c = next_chunk(c, G, g.ntiles, CH, cnt_in, g.tile_cap, pf);
    }
    *(int4*)(sm + L.desc + NS * sizeof(int4)) = c;  // the last chunk issued
  }
  __syncthreads();

  uint32_t parity = 0;  // bit b: phase parity expected next on stage b
  int outRun = 0, movRun = 0;
  PushTally tl = {0, 0, 0, 0, 0.0, 0.0, 0};

  for (int b = 0;; b = (b + 1 == NS) ? 0 : b + 1) {
    const int4 c = desc[b];
    if (c.x >= g.ntiles) break;
    const int t = c.x, m = c.z;
    if (m > 0) {
      const bool ok = mbar_wait(&bar[b], (parity >> b) & 1u);
      parity ^= 1u << b;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(&d.ctr->status, kStatusTimeout);
          // let the other stages' copies land before the CTA exits (bounded)
          for (int o = 0; o < NS; ++o)
            if (o != b && desc[o].x < g.ntiles && desc[o].z > 0)
              mbar_wait(&bar[o], (parity >> o) & 1u);
        }
        return;
      }
    }
    const int tx = t % g.ntx, ty = t / g.ntx;
    const int i0 = tx * TX, j0 = ty * TY;
    const size_t bo = (size_t)b * L.bstride;
    const T* F = (const T*)(sm + L.F[0] + bo);
    int* sc = (int*)(sm + L.cell[0] + bo);
    T* sx = (T*)(sm + L.ox[0] + bo);
    T* sy = (T*)(sm + L.oy[0] + bo);
    T* svx = (T*)(sm + L.vx[0] + bo);
    T* svy = (T*)(sm + L.vy[0] + bo);
    T* svz = (T*)(sm + L.vz[0] + bo);
    uint32_t* sid = (uint32_t*)(sm + L.id[0] + bo);

    // ---- push in place, deposit (warp-cooperative, push order), key, rank
    int rk[PPT], ky[PPT];
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      const int p = tid + r * kBlock;
      rk[r] = 0;
      ky[r] = NE + 1;
      if (r * kBlock >= m) continue;  // whole block past the chunk: uniform skip
      int key = NE + 1;
      T fx = (T)0, fy = (T)0, vx = (T)0, vy = (T)0, vz = (T)0;
      uint32_t id = 0;
      if (p < m) {
        int cell = sc[p];
        fx = sx[p];
        fy = (DIM == 2) ? sy[p] : (T)0;
        vx = svx[p];
        vy = svy[p];
        vz = svz[p];
        id = sid[p];
        key = push_one<T, DIM>(F, L.NFX, cell, fx, fy, vx, vy, vz, id, i0, j0, TX, TY, EX,
                               EY, NE, e2k, g, ph, dtdx, dtdy, hdt, step, tl);
        sc[p] = cell;
        sx[p] = fx;
        if (DIM == 2) sy[p] = fy;
        svx[p] = vx;
        svy[p] = vy;
        svz[p] = vz;
        sid[p] = id;
        rk[r] = atomicAdd(&kcount[key], 1);
        ky[r] = key;
        if (key == NE) {  // far mover: deposit straight to the global far sums
          deposit_far<T, DIM>(d, g, cell & 0xFFFF, cell >> 16, fx, fy,
                              (id & kIdCR) ? wcr : wth, vx, vy, vz);
        }
      }
      const T wp = (id & kIdCR) ? wcr : wth;
      warp_deposit<T, DIM>(ACC, NA, AX, k2e, key, key < NE, fx, fy, wp, vx, vy, vz, lane);
    }
    __syncthreads();
    if (warp == 0) warp_scan_excl(kcount, koff, NK, lane);
    __syncthreads();

    // ---- write: stayers to the tile's bucket in cell order, leavers to the
    //      tile's range of the mover list
    const int S = koff[NINT];
    const int Lv = koff[NE + 1] - S;
    const int obase = d.tile_base[t] + outRun;
    const int mbase = t * g.mover_per_tile + movRun;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      const int p = tid + r * kBlock;
      const int key = ky[r];
      if (p >= m || key > NE) continue;
      const int pos = koff[key] + rk[r];
      int gi;
      Parts<T> dst;
      if (pos < S) {
        gi = obase + pos;
        dst = PO;
      } else {
        const int slot = movRun + (pos - S);
        if (slot >= g.mover_per_tile) {
          tl.status |= kStatusCapacity;
          continue;
        }
        gi = mbase + (pos - S);
        dst = d.M;
      }
      dst.cell[gi] = sc[p];
      dst.ox[gi] = sx[p];
      if (DIM == 2) dst.oy[gi] = sy[p];
      dst.vx[gi] = svx[p];
      dst.vy[gi] = svy[p];
      dst.vz[gi] = svz[p];
      dst.id[gi] = sid[p];
    }
    outRun += S;
    movRun += Lv;
    for (int q = tid; q < NK; q += kBlock) kcount[q] = 0;
    if (c.y + m >= c.w) {
      // last chunk of tile t: its deposit partial, output and mover counts
      A* part = (A*)d.partial + (size_t)t * 4 * NA;
      for (int q = tid; q < 4 * NA; q += kBlock) {
        part[q] = ACC[q];
        ACC[q] = (A)0;
      }
      if (tid == 0) {
        d.cnt[a.out][t] = outRun;
        d.mcnt[t] = min(movRun, g.mover_per_tile);
      }
      outRun = 0;
      movRun = 0;
    }
    __syncthreads();
    // stage b is free: prefetch the chunk after the most recently issued one
    if (tid == 0) {
      fence_proxy_async_smem();
      int4* lastc = (int4*)(sm + L.desc + NS * sizeof(int4));
      const int4 nc = next_chunk(*lastc, G, g.ntiles, CH, cnt_in, g.tile_cap, pf);
      *lastc = nc;
      issue_chunk<T, DIM>(sm, L, b, nc, d, PI, g);
    }
  }

  if (tl.inc | tl.esc) {
    if (tl.inc) atomicAdd(&d.ctr->incident, (unsigned long long)tl.inc);
    if (tl.tr) atomicAdd(&d.ctr->transmitted, (unsigned long long)tl.tr);
    if (tl.ref) atomicAdd(&d.ctr->reflected, (unsigned long long)tl.ref);
    if (tl.esc) atomicAdd(&d.ctr->escaped, (unsigned long long)tl.esc);
    if (tl.fse != 0.0) atomicAdd(&d.ctr->fs_energy, tl.fse);
    if (tl.rem != 0.0) atomicAdd(&d.ctr->removed_energy, tl.rem);
  }
  if (tl.status) atomicOr(&d.ctr->status, tl.status);
}

}  // namespace fsx
