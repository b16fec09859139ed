// fs_push.cuh -- the fused particle step (gather, Boris, move, open wall,
// faux shock, in-tile counting sort, CIC deposit), one persistent CTA per
// group of tiles with the next chunks of particles prefetched into shared
// memory by the TMA bulk-copy engine while the current one is processed.
//
// Per chunk (at most CH particles of one tile):
//   1. wait for the chunk's bulk copies (its particle columns and the tile's
//      packed E / Bbar nodes) on an mbarrier;
//   2. push every particle (the state written back in place in FP32, kept in
//      registers in FP64) and give it a sort key: its new cell in the tile
//      (interior cells first), a halo cell, FAR (moved more than one cell out
//      of the tile) or REMOVED; lanes with the same key take consecutive
//      ranks after one shared atomic per key; then deposit the PREVIOUS
//      chunk, in pieces (a key's particles, at most kPiece) that the warps
//      claim from a shared counter, each piece a corner x split team
//      reduction, so that warps which finished their push early take more;
//   3. (barrier) each warp scans the key counts; every thread copies its
//      particles into the key-sorted buffer;
//   4. (barrier) the stage is refilled with a later chunk; coalesced writes
//      from the sorted buffer: stayers to the tile's bucket of the output
//      buffer, leavers to the tile's range of the mover list.
// A tile's node accumulator is written out as its deposit partial after the
// first barrier of the chunk that follows the tile's last chunk (whose
// deposit is done by then); two accumulators alternate between tiles. Each
// chunk costs two block-wide barriers; the CTA's last chunk is deposited
// after the loop.
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

// bounded wait: false if the phase did not complete within `limit` tries
constexpr int kWaitLimit = 1 << 20;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          int limit = kWaitLimit) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Failure-detection self-test: one CTA waits, with the push's bounded wait,
// on an mbarrier that nothing arrives on and no bulk copy targets. The wait
// runs out after `limit` tries; the CTA records the timeout bit in *status
// (as the push does in its counters) and returns with nothing in flight.
static __global__ void k_wait_selftest(int* status, int limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0u, limit);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

struct StepArgs {
  Geo g;
  Phys ph;
  int in, out;
  long long step;
};

// ---------------------------------------------------------------- layout
constexpr int kMaxStages = 4;
constexpr int kWarps = kBlock / 32;

template <typename T, int DIM>
struct PushLayout {
  int TX, TY, NFX, NFY, AX, AY, NA, EX, EY, NE, NINT, NK, CH, NS;
  // stage 0's regions; stage b sits b * bstride bytes further
  size_t F[1], cell[1], ox[1], oy[1], vx[1], vy[1], vz[1], id[1];
  size_t sW, sV, sF, scell, sid;  // key-sorted buffer
  size_t acc, kc, wk, e2k, k2e, desc, bar, pf, tally, pst, dq, bytes;
  size_t bstride;  // distance between two chunk buffers
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
    // per stage {tile, first particle, count, tile count} and {i0, j0,
    // inner-tile flag, tile base}; then the last chunk issued
    desc = take(o, (2 * kMaxStages + 1) * sizeof(int4));
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
    // the key-sorted copy of the chunk being finished: the four CIC corner
    // weights, {vx, vy, vz, 1/gamma}, {fx, fy}, cell and id per particle
    // FP32: no weights (the deposit forms them from the offsets)
    sW = take(o, sizeof(T) == 4 ? 0 : sizeof(T) * 4 * CH);
    sV = take(o, sizeof(T) * 4 * CH);
    sF = take(o, sizeof(T) * 2 * CH);
    scell = take(o, sizeof(int) * CH);
    sid = take(o, sizeof(uint32_t) * CH);
    pf = take(o, 16);
    tally = take(o, sizeof(unsigned long long) * 4 + sizeof(double) * 2);
    acc = take(o, sizeof(typename Num<T>::acc) * 2 * 4 * NA);  // two tiles in flight
    kc = take(o, sizeof(int) * 2 * NK);                         // two chunks in flight
    wk = take(o, sizeof(int) * kWarps * (NK + 1));              // key offsets per warp
    pst = take(o, sizeof(int) * (NK + 1));  // first deposit piece of each key
    dq = take(o, sizeof(int) * 2);          // deposit piece counters, two chunks
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
  if (n <= 32) {  // one value per lane
    const int s = lane < n ? in[lane] : 0;
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane < n) out[lane] = inc - s;
    if (lane == 31) out[n] = inc;
    return;
  }
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
// that owns tiles cta, cta + G, ...; tile >= ntiles: done.
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
// One node of the packed field block (Ex Ey Ez Bx By Bz, two pad words) in
// 16-byte loads; node blocks are 16-byte aligned in shared memory.
__device__ __forceinline__ void load_node(const float* n, float (&v)[6]) {
  const float4 a = reinterpret_cast<const float4*>(n)[0];
  const float4 b = reinterpret_cast<const float4*>(n)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}
__device__ __forceinline__ void load_node(const double* n, double (&v)[6]) {
  const double2 a = reinterpret_cast<const double2*>(n)[0];
  const double2 b = reinterpret_cast<const double2*>(n)[1];
  const double2 c = reinterpret_cast<const double2*>(n)[2];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

// 4- and 2-wide shared-memory accesses of T (16-byte aligned)
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st2(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void st2(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
__device__ __forceinline__ void ld2(const float* p, float (&v)[2]) {
  const float2 a = *reinterpret_cast<const float2*>(p);
  v[0] = a.x; v[1] = a.y;
}
__device__ __forceinline__ void ld2(const double* p, double (&v)[2]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  v[0] = a.x; v[1] = a.y;
}

// Ordered integer key of a double: monotone in its value, with -0 and +0
// equal and a NaN beyond every finite key, so that x >= c (c finite) is the
// same test as ordered_key(x) >= ordered_key(c).
__device__ __forceinline__ long long ordered_key(double x) {
  const long long b = __double_as_longlong(x);
  const long long m = b & 0x7FFFFFFFFFFFFFFFLL;
  return b < 0 ? -m : m;
}
constexpr long long kKeyOne = 0x3FF0000000000000LL;  // ordered_key(1.0)
constexpr long long kKeyTwo = 0x4000000000000000LL;  // ordered_key(2.0)
__device__ __forceinline__ bool ge_one(double x) { return ordered_key(x) >= kKeyOne; }
__device__ __forceinline__ bool ge_one(float x) { return x >= 1.0f; }

// Faux-shock and open-wall bookkeeping of one CTA (rare events): shared
// memory, added to the global counters once at the end.
struct PushTally {
  unsigned long long inc, tr, ref, esc;
  double fse, rem;
};

template <typename T, int DIM, bool REL>
__device__ __forceinline__ int push_one(const T* __restrict__ F, int NFX, int& cell,
                                        T& fx, T& fy, T& vx, T& vy, T& vz,
                                        uint32_t& id, int i0, int j0, int TX, int TY,
                                        int EX, int EY, int NE, const uint16_t* e2k,
                                        const Geo& g, const Phys& ph, T dtdx, T dtdy,
                                        T hdt, T c2inv_t, long long step, PushTally* tl,
                                        int& status, bool inner) {
  const int i = cell & 0xFFFF, j = cell >> 16;
  const int lx = i - i0, ly = j - j0;
  if ((unsigned)lx >= (unsigned)TX || (unsigned)ly >= (unsigned)TY) {
    status |= kStatusBadCell;
    return NE + 1;
  }
  T Ep[3], Bp[3];
  if (DIM == 1) {
    const T g0 = (T)1 - fx;
    T a[6], b[6];
    load_node(F + lx * 8, a);
    load_node(F + lx * 8 + 8, b);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      Ep[q] = fmaT(fx, b[q], g0 * a[q]);
      Bp[q] = fmaT(fx, b[3 + q], g0 * a[3 + q]);
    }
  } else if constexpr (sizeof(T) == 4) {
    // FP32: the same products and fused multiply-adds, two components per
    // paired instruction (Ex Ey | Ez Bx | By Bz, the node's 16-byte halves)
    const T gx0 = (T)1 - fx, gy0 = (T)1 - fy;
    const T w00 = gx0 * gy0, w10 = fx * gy0, w01 = gx0 * fy, w11 = fx * fy;
    const float* n00 = reinterpret_cast<const float*>(F) + (ly * NFX + lx) * 8;
    const float4 a0 = reinterpret_cast<const float4*>(n00)[0];
    const float2 b0 = reinterpret_cast<const float2*>(n00)[2];
    const float4 a1 = reinterpret_cast<const float4*>(n00 + 8)[0];
    const float2 b1 = reinterpret_cast<const float2*>(n00 + 8)[2];
    const float4 a2 = reinterpret_cast<const float4*>(n00 + NFX * 8)[0];
    const float2 b2 = reinterpret_cast<const float2*>(n00 + NFX * 8)[2];
    const float4 a3 = reinterpret_cast<const float4*>(n00 + NFX * 8 + 8)[0];
    const float2 b3 = reinterpret_cast<const float2*>(n00 + NFX * 8 + 8)[2];
    const float2 W00 = make_float2(w00, w00), W10 = make_float2(w10, w10);
    const float2 W01 = make_float2(w01, w01), W11 = make_float2(w11, w11);
    float2 p0 = __fmul2_rn(W00, make_float2(a0.x, a0.y));
    float2 p1 = __fmul2_rn(W00, make_float2(a0.z, a0.w));
    float2 p2 = __fmul2_rn(W00, b0);
    p0 = __ffma2_rn(W10, make_float2(a1.x, a1.y), p0);
    p1 = __ffma2_rn(W10, make_float2(a1.z, a1.w), p1);
    p2 = __ffma2_rn(W10, b1, p2);
    p0 = __ffma2_rn(W01, make_float2(a2.x, a2.y), p0);
    p1 = __ffma2_rn(W01, make_float2(a2.z, a2.w), p1);
    p2 = __ffma2_rn(W01, b2, p2);
    p0 = __ffma2_rn(W11, make_float2(a3.x, a3.y), p0);
    p1 = __ffma2_rn(W11, make_float2(a3.z, a3.w), p1);
    p2 = __ffma2_rn(W11, b3, p2);
    Ep[0] = p0.x;
    Ep[1] = p0.y;
    Ep[2] = p1.x;
    Bp[0] = p1.y;
    Bp[1] = p2.x;
    Bp[2] = p2.y;
  } else {
    const T gx0 = (T)1 - fx, gy0 = (T)1 - fy;
    const T w00 = gx0 * gy0, w10 = fx * gy0, w01 = gx0 * fy, w11 = fx * fy;
    // node by node, in the order w00, w10, w01, w11 of the nested fma
    const T* n00 = F + (ly * NFX + lx) * 8;
    T v[6];
    load_node(n00, v);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      Ep[q] = w00 * v[q];
      Bp[q] = w00 * v[3 + q];
    }
    load_node(n00 + 8, v);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      Ep[q] = fmaT(w10, v[q], Ep[q]);
      Bp[q] = fmaT(w10, v[3 + q], Bp[q]);
    }
    load_node(n00 + NFX * 8, v);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      Ep[q] = fmaT(w01, v[q], Ep[q]);
      Bp[q] = fmaT(w01, v[3 + q], Bp[q]);
    }
    load_node(n00 + NFX * 8 + 8, v);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      Ep[q] = fmaT(w11, v[q], Ep[q]);
      Bp[q] = fmaT(w11, v[3 + q], Bp[q]);
    }
  }
  // REL = false: the relativistic terms are compiled out (c2inv taken as 0)
  const T c2inv = REL ? c2inv_t : (T)0;
  boris<T>(vx, vy, vz, Ep, Bp, hdt, c2inv);
  // the move uses the velocity (v = u / gamma for relativistic ions)
  T mvx = vx, mvy = vy, ig = (T)1;
  if (c2inv > (T)0) {
    ig = inv_gamma_u(vx, vy, vz, c2inv);
    mvx = vx * ig;
    mvy = vy * ig;
  }
  const T fxr = fmaT(mvx, dtdx, fx);
  T fyr = fy;
  if (DIM == 2) fyr = fmaT(mvy, dtdy, fy);
  // Common case: a tile away from every box edge and a shift of at most one
  // cell: no wall, wrap or far-mover handling can apply. Same values as the
  // general path below (shift in {-1, 0, 1}, subtracted exactly). The
  // comparisons with -1, 0, 1 and 2 are exact either way; in FP64 they run
  // on the ordered integer key of the value, off GB300's narrow FP64 pipe.
  bool inr, xp, xm, yp = false, ym = false;
  if constexpr (sizeof(T) == 8) {
    const long long kx = ordered_key(fxr);
    inr = kx >= -kKeyOne && kx < kKeyTwo;
    xp = kx >= kKeyOne;
    xm = kx < 0;
    if (DIM == 2) {
      const long long ky = ordered_key(fyr);
      inr = inr && ky >= -kKeyOne && ky < kKeyTwo;
      yp = ky >= kKeyOne;
      ym = ky < 0;
    }
  } else {
    inr = fxr >= (T)-1 && fxr < (T)2 && (DIM == 1 || (fyr >= (T)-1 && fyr < (T)2));
    xp = fxr >= (T)1;
    xm = fxr < (T)0;
    if (DIM == 2) {
      yp = fyr >= (T)1;
      ym = fyr < (T)0;
    }
  }
  if (inner && inr) {
    const int ikx = xp ? 1 : (xm ? -1 : 0);
    T fxn = fxr - (xp ? (T)1 : (xm ? (T)-1 : (T)0));
    if (ge_one(fxn)) fxn = Num<T>::offmax;
    int iky = 0;
    if (DIM == 2) {
      iky = yp ? 1 : (ym ? -1 : 0);
      T fyn = fyr - (yp ? (T)1 : (ym ? (T)-1 : (T)0));
      if (ge_one(fyn)) fyn = Num<T>::offmax;
      fy = fyn;
    }
    cell = ((j + iky) << 16) | (i + ikx);
    fx = fxn;
    const int lxn = lx + ikx, lyn = ly + iky;  // interior-relative
    if ((unsigned)lxn < (unsigned)TX && (unsigned)lyn < (unsigned)TY) return lxn + lyn * TX;
    return e2k[(lxn + 1) + (DIM == 2 ? (lyn + 1) * EX : 0)];
  }
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
    status |= kStatusNaN;
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
    atomicAdd(&tl->esc, 1ull);
    atomicAdd(&tl->rem, kinetic(cr ? ph.w_cr : ph.w_th, (double)vx, (double)vy, (double)vz,
                                ph.cellvol, ph.c2inv));
    return NE + 1;
  } else if (inew < 0) {
    const int mode = cr ? FS_SHOCK : ph.fs_mode_thermal;
    const double wpd = cr ? ph.w_cr : ph.w_th;
    atomicAdd(&tl->inc, 1ull);
    const double e0 = kinetic(wpd, (double)vx, (double)vy, (double)vz, ph.cellvol, ph.c2inv);
    // the rule acts on the velocity: a relativistic ion's u -> v -> u
    double dvx = mvx, dvy = (c2inv > (T)0) ? vy * ig : vy, dvz = (c2inv > (T)0) ? vz * ig : vz;
    if (mode == FS_SHOCK &&
        fs_return(dvx, dvy, dvz, ph.u2, ph.fs_frame, ph.seed, id & kIdMask, step)) {
      double ux = dvx, uy = dvy, uz = dvz;
      if (REL && ph.c2inv > 0.0) {
        const double gv = gamma_v(dvx, dvy, dvz, ph.c2inv);
        ux = __dmul_rn(dvx, gv); uy = __dmul_rn(dvy, gv); uz = __dmul_rn(dvz, gv);
      }
      atomicAdd(&tl->ref, 1ull);
      atomicAdd(&tl->fse, __dsub_rn(kinetic(wpd, ux, uy, uz, ph.cellvol, ph.c2inv), e0));
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
      vx = (T)ux;
      vy = (T)uy;
      vz = (T)uz;
      id |= kIdReturned;
    } else {
      atomicAdd(&tl->tr, 1ull);
      atomicAdd(&tl->rem, e0);
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
  desc[2 * b] = c;
  if (c.x >= g.ntiles) return;
  const int tx = c.x % g.ntx, ty = c.x / g.ntx;
  const int i0 = tx * L.TX, j0 = ty * L.TY;
  // no particle of the tile can reach a box edge by a one-cell shift
  const int inner =
      i0 >= 1 && i0 + L.TX < g.nx && (DIM == 1 || (j0 >= 1 && j0 + L.TY < g.ny));
  // a tile's bucket starts at tile x capacity (fixed at set-up)
  const int tbase = c.x * g.tile_cap;
  desc[2 * b + 1] = make_int4(i0, j0, inner, tbase);
  if (c.z <= 0) return;
  const size_t bo = (size_t)b * L.bstride;
  mbar_arrive_expect_tx(bar, L.chunk_bytes(c.z));
  const uint32_t row = (uint32_t)(sizeof(T) * 8 * L.NFX);
  for (int ly = 0; ly < L.NFY; ++ly)
    bulk_g2s(sm + L.F[0] + bo + (size_t)ly * row,
             d.G + ((size_t)(j0 + ly) * (g.nx + 1) + i0) * 8, row, bar);
  const size_t first = (size_t)tbase + c.y;
  const uint32_t m4 = (uint32_t)((c.z + 3) & ~3);
  bulk_g2s(sm + L.cell[0] + bo, PI.cell + first, 4 * m4, bar);
  bulk_g2s(sm + L.ox[0] + bo, PI.ox + first, sizeof(T) * m4, bar);
  if (DIM == 2) bulk_g2s(sm + L.oy[0] + bo, PI.oy + first, sizeof(T) * m4, bar);
  bulk_g2s(sm + L.vx[0] + bo, PI.vx + first, sizeof(T) * m4, bar);
  bulk_g2s(sm + L.vy[0] + bo, PI.vy + first, sizeof(T) * m4, bar);
  bulk_g2s(sm + L.vz[0] + bo, PI.vz + first, sizeof(T) * m4, bar);
  bulk_g2s(sm + L.id[0] + bo, PI.id + first, 4 * m4, bar);
}


// CIC deposit of one key's particles, which sit contiguously in [b0, b1) of
// the key-sorted chunk (W: corner weights, V: {vx, vy, vz, 1/gamma}). The warp
// works as NC corners x SPL splits: lane (corner c, split s) sums corner c's
// four quantities (weight, weight * v) over particles b0 + s, b0 + s + SPL,
// ...; a transpose reduction over the splits then leaves each quantity's
// total in one lane, which adds it to the tile's node accumulator. Each
// contribution is formed as in the per-particle scheme, so in fixed point
// the sums do not depend on the order.
template <typename T, int DIM, bool REL>
__device__ __forceinline__ void team_add(typename Num<T>::acc (&acc)[4], const T* W,
                                         const T* V, const T* Fo, const uint32_t* ID,
                                         T wth, T wcr, int i, int c) {
  T cw;
  T v[4];
  ld4(V + 4 * i, v);
  if constexpr (sizeof(T) == 4) {  // corner weight wp * (gx * gy) from the offsets
    T f[2];
    ld2(Fo + 2 * i, f);
    // the particle weight: in V's fourth slot without relativistic terms
    const T wp = REL ? ((ID[i] & kIdCR) ? wcr : wth) : v[3];
    // gx = fx or 1 - fx by one fused multiply-add (the same rounded value)
    const T gx = fmaT((c & 1) ? (T)1 : (T)-1, f[0], (c & 1) ? (T)0 : (T)1);
    if (DIM == 2) {
      const T gy = fmaT((c >> 1) ? (T)1 : (T)-1, f[1], (c >> 1) ? (T)0 : (T)1);
      cw = wp * (gx * gy);
    } else {
      cw = wp * gx;
    }
  } else {
    cw = W[4 * i + c];
  }
  if (REL) {  // relativistic ions: V holds u and 1/gamma
    v[0] = v[0] * v[3];
    v[1] = v[1] * v[3];
    v[2] = v[2] * v[3];
  }
  acc[0] = acc[0] + to_acc(cw);
  acc[1] = acc[1] + to_acc_prod(cw, v[0]);
  acc[2] = acc[2] + to_acc_prod(cw, v[1]);
  acc[3] = acc[3] + to_acc_prod(cw, v[2]);
}

template <typename T, int DIM, bool REL>
__device__ __forceinline__ void team_deposit(typename Num<T>::acc* ACC, int NA, int AX,
                                             int le, int b0, int b1, const T* W, const T* V,
                                             const T* Fo, const uint32_t* ID, T wth, T wcr,
                                             int lane) {
  using A_t = typename Num<T>::acc;
  constexpr int NC = (DIM == 2) ? 4 : 2;
  constexpr int SPL = 32 / NC;
  const int s = lane % SPL, c = lane / SPL;
  A_t acc[4] = {(A_t)0, (A_t)0, (A_t)0, (A_t)0};
  int i = b0 + s;
  for (; i + SPL < b1; i += 2 * SPL) {  // two particles in flight per lane
    team_add<T, DIM, REL>(acc, W, V, Fo, ID, wth, wcr, i, c);
    team_add<T, DIM, REL>(acc, W, V, Fo, ID, wth, wcr, i + SPL, c);
  }
  if (i < b1) team_add<T, DIM, REL>(acc, W, V, Fo, ID, wth, wcr, i, c);
  // two halving levels leave one quantity per lane, the rest add pairs
  {
    const bool up = (s & (SPL / 2)) != 0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const A_t send = up ? acc[q] : acc[q + 2];
      const A_t keep = up ? acc[q + 2] : acc[q];
      acc[q] = keep + shfl_xor(send, SPL / 2);
    }
  }
  {
    const bool up = (s & (SPL / 4)) != 0;
    const A_t send = up ? acc[0] : acc[1];
    const A_t keep = up ? acc[1] : acc[0];
    acc[0] = keep + shfl_xor(send, SPL / 4);
  }
#pragma unroll
  for (int off = SPL / 8; off >= 1; off >>= 1) acc[0] = acc[0] + shfl_xor(acc[0], off);
  if ((s & (SPL / 4 - 1)) == 0) {
    const int q = ((s & (SPL / 2)) ? 2 : 0) + ((s & (SPL / 4)) ? 1 : 0);
    const int a00 = (le & 0xFFFF) + (le >> 16) * AX;
    const int an = a00 + (c & 1) + ((DIM == 2) ? (c >> 1) * AX : 0);
    atomic_acc(&ACC[q * NA + an], acc[0]);
  }
}

// Deposit of a key-sorted chunk in pieces: key k's particles [wk[k], wk[k+1])
// form ceil(n / kPiece) pieces of at most kPiece, numbered from pst[k]. Warp
// w > 0 takes piece w - 1, then (and warp 0 from the start) the next
// unclaimed piece from the counter *q until none is left, so that warps which
// reach the deposit early take more of it. A piece is one team reduction:
// whole keys (cells) where they are not large, since the reduction, not the
// particle count, sets most of a piece's cost. Each particle's contributions
// are formed as in the per-particle scheme, so in fixed point (FP64) the sums
// do not depend on which warp takes which piece.
constexpr int kPiece = 160;
template <typename T, int DIM, bool REL>
__device__ __forceinline__ void deposit_pieces(typename Num<T>::acc* ACC, int NA, int AX, int NE,
                                               const int* wk, const int* pst, const int* k2e,
                                               const T* W, const T* V, const T* Fo,
                                               const uint32_t* ID, T wth, T wcr, int* q,
                                               int warp, int lane) {
  constexpr int PS = kPiece;
  const int np = pst[NE];
  // warp 0 (which issues the bulk copies) claims from the start; warp w > 0
  // takes piece w - 1 first
  int gi;
  if (warp == 0) {
    int nx = 0;
    if (lane == 0) nx = atomicAdd(q, 1);
    gi = kWarps - 1 + __shfl_sync(0xffffffffu, nx, 0);
  } else {
    gi = warp - 1;
  }
  while (gi < np) {
    int k = -1;
    for (int kb = 0; kb < NE; kb += 32) {
      const int kk = kb + lane;
      const unsigned h =
          __ballot_sync(0xffffffffu, kk < NE && pst[kk] <= gi && gi < pst[kk + 1]);
      if (h) {
        k = kb + __ffs(h) - 1;
        break;
      }
    }
    if (k < 0) break;
    const int b0 = wk[k] + (gi - pst[k]) * PS;
    const int b1 = min(b0 + PS, wk[k + 1]);
    team_deposit<T, DIM, REL>(ACC, NA, AX, k2e[k], b0, b1, W, V, Fo, ID, wth, wcr, lane);
    int nx = 0;
    if (lane == 0) nx = atomicAdd(q, 1);
    gi = kWarps - 1 + __shfl_sync(0xffffffffu, nx, 0);
  }
}

// Every stage holds a chunk not yet consumed.
template <typename T, int DIM>
__device__ __forceinline__ void drain_stages(unsigned char* sm, const PushLayout<T, DIM>& L,
                                             uint32_t parity, int ntiles) {
  const int4* desc = (const int4*)(sm + L.desc);
  uint64_t* bar = (uint64_t*)(sm + L.bar);
  for (int o = 0; o < L.NS; ++o)
    if (desc[2 * o].x < ntiles && desc[2 * o].z > 0) mbar_wait(&bar[o], (parity >> o) & 1u);
}

// The push of one run by one CTA of a group of G CTAs (rank cta in the
// group): tiles cta, cta + G, ... of the run; sm is the dynamic shared memory.
// TXC, TYC: the tile shape as compile-time constants (0: the run's g.TX, g.TY)
template <typename T, int DIM, int CH, int NS, bool REL, int TXC = 0, int TYC = 0>
__device__ __forceinline__ void push_run(const DevPtrs<T>& d, const Geo& g, const Phys& ph,
                                         const PushConst<T>& pc, int in, int out, int cta,
                                         int G, unsigned char* sm) {
  using A = typename Num<T>::acc;
  constexpr int PPT = (CH + kBlock - 1) / kBlock;
  const PushLayout<T, DIM> L(TXC ? TXC : g.TX, TXC ? TYC : g.TY, CH, NS);
  const int TX = L.TX, TY = L.TY, EX = L.EX, EY = L.EY, NE = L.NE, NINT = L.NINT,
            NK = L.NK, NA = L.NA, AX = L.AX;
  uint64_t* bar = (uint64_t*)(sm + L.bar);
  int4* desc = (int4*)(sm + L.desc);
  A* ACC0 = (A*)(sm + L.acc);
  int* kc0 = (int*)(sm + L.kc);
  uint16_t* e2k = (uint16_t*)(sm + L.e2k);
  int* k2e = (int*)(sm + L.k2e);
  int* pf = (int*)(sm + L.pf);
  PushTally* tl = (PushTally*)(sm + L.tally);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int* wk = (int*)(sm + L.wk) + warp * (NK + 1);
  const int* cnt_in = d.cnt[in];
  const Parts<T> PI = d.P[in];
  const Parts<T> PO = d.P[out];
  const T dtdx = pc.dtdx, dtdy = pc.dtdy, hdt = pc.hdt;
  const T wth = pc.wth, wcr = pc.wcr;
  const long long step = d.ctr->step;  // device step counter (graph-replayable)
  // relativistic ions (REL and c2inv > 0): states hold u = gamma v
  const bool rel = REL && ph.c2inv > 0.0;
  const T c2inv = REL ? pc.c2inv : (T)0;

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
  for (int k = tid; k < 2 * 4 * NA; k += kBlock) ACC0[k] = (A)0;
  for (int k = tid; k < 2 * NK; k += kBlock) kc0[k] = 0;
  int* pst = (int*)(sm + L.pst);
  int* dq = (int*)(sm + L.dq);
  if (tid < 2) dq[tid] = 0;

  if (tid == 0) {
    for (int b = 0; b < NS; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
    *tl = PushTally{0, 0, 0, 0, 0.0, 0.0};
  }
  __syncthreads();
  if (tid == 0) {
    // prologue: the CTA's first NS chunks, one per stage
    int4 c;
    if (cta < g.ntiles) {
      const int n = min(cnt_in[cta], g.tile_cap);
      c = make_int4(cta, 0, min(CH, n), n);
    } else {
      c = make_int4(g.ntiles, 0, 0, 0);
    }
    if (cta + G < g.ntiles) cp_async4(pf, cnt_in + cta + G);
    for (int b = 0; b < NS; ++b) {
      issue_chunk<T, DIM>(sm, L, b, c, d, PI, g);
      if (b + 1 < NS) c = next_chunk(c, G, g.ntiles, CH, cnt_in, g.tile_cap, pf);
    }
    *(int4*)(sm + L.desc + 2 * NS * sizeof(int4)) = c;  // the last chunk issued
  }
  __syncthreads();

  uint32_t parity = 0;  // bit b: phase parity expected next on stage b
  int outRun = 0, movRun = 0;
  int tiles_seen = 0, tpar = 0;  // accumulator buffer of the current tile
  int pend = -1, pend_par = 0;   // tile whose partial is written next chunk
  int status = 0;
  int dpar = -1;  // accumulator buffer of the chunk whose deposit is pending (-1: none)
  int* oc = (int*)(sm + L.scell);
  uint32_t* oid = (uint32_t*)(sm + L.sid);
  T* oW = (T*)(sm + L.sW);
  T* oV = (T*)(sm + L.sV);
  T* oF = (T*)(sm + L.sF);

  int b = 0;
  for (int ci = 0;; ++ci, b = (b + 1 == NS) ? 0 : b + 1) {
    const int4 c = desc[2 * b];
    if (c.x >= g.ntiles) {
      // the last chunk's deposit
      if (dpar >= 0)
        deposit_pieces<T, DIM, REL>(ACC0 + dpar * 4 * NA, NA, AX, NE, wk, pst, k2e, oW, oV,
                                    oF, oid, wth, wcr, dq + ((ci - 1) & 1), warp, lane);
      break;
    }
    const int i0 = desc[2 * b + 1].x, j0 = desc[2 * b + 1].y;
    const bool inner = desc[2 * b + 1].z != 0;
    const int t = c.x, m = c.z;
    if (c.y == 0) tpar = (tiles_seen++) & 1;
    bool ok = true;
    if (m > 0) {
      ok = mbar_wait(&bar[b], (parity >> b) & 1u);
      parity ^= 1u << b;
    }
    const int mloc = ok ? m : 0;  // a thread whose wait gave up touches nothing
    const size_t bo = (size_t)b * L.bstride;
    const T* F = (const T*)(sm + L.F[0] + bo);
    int* sc = (int*)(sm + L.cell[0] + bo);
    T* sx = (T*)(sm + L.ox[0] + bo);
    T* sy = (T*)(sm + L.oy[0] + bo);
    T* svx = (T*)(sm + L.vx[0] + bo);
    T* svy = (T*)(sm + L.vy[0] + bo);
    T* svz = (T*)(sm + L.vz[0] + bo);
    uint32_t* sid = (uint32_t*)(sm + L.id[0] + bo);
    int* kc = kc0 + (ci & 1) * NK;
    A* ACC = ACC0 + tpar * 4 * NA;

    // ---- push, key, rank within the key. FP32: the pushed state written back
    //      in place; FP64 (128 registers at two CTAs per SM): kept in
    //      registers until the key-order copy
    int ky[PPT], rk[PPT];
    int rc_[PPT];
    uint32_t rid_[PPT];
    T rfx_[PPT], rfy_[PPT], rvx_[PPT], rvy_[PPT], rvz_[PPT];
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      const int p = tid + r * kBlock;
      ky[r] = NE + 1;
      rk[r] = 0;
      if (r * kBlock >= m) continue;  // whole block past the chunk: uniform skip
      int key = -1;
      if (p < mloc) {
        int cell = sc[p];
        T fx = sx[p];
        T fy = (DIM == 2) ? sy[p] : (T)0;
        T vx = svx[p], vy = svy[p], vz = svz[p];
        uint32_t id = sid[p];
        key = push_one<T, DIM, REL>(F, L.NFX, cell, fx, fy, vx, vy, vz, id, i0, j0, TX, TY, EX,
                               EY, NE, e2k, g, ph, dtdx, dtdy, hdt, c2inv, step, tl,
                               status, inner);
        if (key == NE) {  // far mover: straight to the global far sums
          T dvx, dvy, dvz;  // the current uses the velocity
          velocity_of<T>(vx, vy, vz, c2inv, dvx, dvy, dvz);
          deposit_far<T, DIM>(d, g, cell & 0xFFFF, cell >> 16, fx, fy,
                              (id & kIdCR) ? wcr : wth, dvx, dvy, dvz);
        }
        if constexpr (sizeof(T) == 8) {
          rc_[r] = cell;
          rfx_[r] = fx;
          rfy_[r] = fy;
          rvx_[r] = vx;
          rvy_[r] = vy;
          rvz_[r] = vz;
          rid_[r] = id;
        } else {
          sc[p] = cell;
          sx[p] = fx;
          if (DIM == 2) sy[p] = fy;
          svx[p] = vx;
          svy[p] = vy;
          svz[p] = vz;
          sid[p] = id;
        }
        ky[r] = key;
      }
      // lanes with equal keys take consecutive ranks after one atomic
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      int base = 0;
      if (lane == leader && key >= 0) base = atomicAdd(&kc[key], __popc(peers));
      base = __shfl_sync(0xffffffffu, base, leader);
      rk[r] = base + __popc(peers & ((1u << lane) - 1u));
    }
    // ---- the previous chunk's deposit, after this chunk's push: warps that
    //      finished their push early take more of it
    if (dpar >= 0)
      deposit_pieces<T, DIM, REL>(ACC0 + dpar * 4 * NA, NA, AX, NE, wk, pst, k2e, oW, oV, oF,
                                  oid, wth, wcr, dq + ((ci - 1) & 1), warp, lane);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(&d.ctr->status, kStatusTimeout);
        drain_stages<T, DIM>(sm, L, parity ^ (1u << b), g.ntiles);
      }
      return;
    }

    // ---- the previous tile's deposit partial is complete: write it out
    if (pend >= 0) {
      A* part = (A*)d.partial + (size_t)pend * 4 * NA;
      A* Q = ACC0 + pend_par * 4 * NA;
      for (int q = tid; q < 4 * NA; q += kBlock) {
        part[q] = Q[q];
        Q[q] = (A)0;
      }
      pend = -1;
    }
    for (int q = tid; q < NK; q += kBlock) kc0[((ci + 1) & 1) * NK + q] = 0;
    if (tid == 0) dq[ci & 1] = 0;
    const int tbase = desc[2 * b + 1].w;  // read before the stage is refilled
    // ---- key offsets (each warp its own copy); copy into key order
    warp_scan_excl(kc, wk, NK, lane);
    __syncwarp();
    if (warp == kWarps - 1) {  // the deposit's pieces per key
      constexpr int PS = kPiece;
      int carry = 0;
      for (int kb = 0; kb < NE; kb += 32) {
        const int kk = kb + lane;
        const int n = kk < NE ? wk[kk + 1] - wk[kk] : 0;
        const int pc = (n + PS - 1) / PS;
        int inc = pc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += v;
        }
        if (kk < NE) pst[kk] = carry + inc - pc;
        carry += __shfl_sync(0xffffffffu, inc, 31);
      }
      if (lane == 0) pst[NE] = carry;
    }
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      const int key = ky[r];
      if (key > NE) continue;
      const int p = tid + r * kBlock;
      const int pos = wk[key] + rk[r];
      constexpr bool inreg = sizeof(T) == 8;
      const uint32_t id = inreg ? rid_[r] : sid[p];
      const T fx = inreg ? rfx_[r] : sx[p];
      const T fy = (DIM == 2) ? (inreg ? rfy_[r] : sy[p]) : (T)0;
      const T ux = inreg ? rvx_[r] : svx[p];
      const T uy = inreg ? rvy_[r] : svy[p];
      const T uz = inreg ? rvz_[r] : svz[p];
      const T wp = (id & kIdCR) ? wcr : wth;
      oc[pos] = inreg ? rc_[r] : sc[p];
      oid[pos] = id;
      st2(oF + 2 * pos, fx, fy);
      // {u} of the state, and 1/gamma (the current uses v = u / gamma)
      // (FP32 without relativistic terms: the particle weight, which the
      // deposit lanes use to form their corner weights)
      st4(oV + 4 * pos, ux, uy, uz,
          (sizeof(T) == 4 && !REL) ? wp : (rel ? inv_gamma_u(ux, uy, uz, c2inv) : (T)1));
      // corner weights: wp * (gx * gy), corners (0,0) (1,0) (0,1) (1,1)
      // (FP32: formed in the deposit)
      if constexpr (sizeof(T) == 8) {
        const T gx0 = (T)1 - fx;
        if (DIM == 2) {
          const T gy0 = (T)1 - fy;
          st4(oW + 4 * pos, wp * (gx0 * gy0), wp * (fx * gy0), wp * (gx0 * fy), wp * (fx * fy));
        } else {
          st4(oW + 4 * pos, wp * gx0, wp * fx, (T)0, (T)0);
        }
      }
    }
    __syncthreads();
    // ---- stage b is free: prefetch the chunk after the most recently issued one
    if (tid == 0) {
      fence_proxy_async_smem();
      int4* lastc = (int4*)(sm + L.desc + 2 * NS * sizeof(int4));
      const int4 nc = next_chunk(*lastc, G, g.ntiles, CH, cnt_in, g.tile_cap, pf);
      *lastc = nc;
      issue_chunk<T, DIM>(sm, L, b, nc, d, PI, g);
    }

    // ---- write: stayers to the tile's bucket in cell order, leavers to the
    //      tile's range of the mover list
    const int S = wk[NINT];
    const int Lv = wk[NE + 1] - S;
    {
      const int obase = tbase + outRun;
      for (int i = tid; i < S; i += kBlock) {
        const int gi = obase + i;
        T vf[2], vv[4];
        ld2(oF + 2 * i, vf);
        ld4(oV + 4 * i, vv);
        PO.cell[gi] = oc[i];
        PO.ox[gi] = vf[0];
        if (DIM == 2) PO.oy[gi] = vf[1];
        PO.vx[gi] = vv[0];
        PO.vy[gi] = vv[1];
        PO.vz[gi] = vv[2];
        PO.id[gi] = oid[i];
      }
      const int room = g.mover_per_tile - movRun;
      const int nm = Lv < room ? Lv : (room > 0 ? room : 0);
      if (nm < Lv) status |= kStatusCapacity;
      const int mb = t * g.mover_per_tile + movRun;
      for (int i = tid; i < nm; i += kBlock) {
        const int gi = mb + i, si = S + i;
        T vf[2], vv[4];
        ld2(oF + 2 * si, vf);
        ld4(oV + 4 * si, vv);
        d.M.cell[gi] = oc[si];
        d.M.ox[gi] = vf[0];
        if (DIM == 2) d.M.oy[gi] = vf[1];
        d.M.vx[gi] = vv[0];
        d.M.vy[gi] = vv[1];
        d.M.vz[gi] = vv[2];
        d.M.id[gi] = oid[si];
      }
    }
    dpar = tpar;  // deposited after the next chunk's push
    outRun += S;
    movRun += Lv;
    if (c.y + m >= c.w) {
      // last chunk of tile t: output and mover counts now, partial next chunk
      if (tid == 0) {
        d.cnt[out][t] = outRun;
        d.mcnt[t] = min(movRun, g.mover_per_tile);
      }
      pend = t;
      pend_par = tpar;
      outRun = 0;
      movRun = 0;
    }
  }
  __syncthreads();
  if (pend >= 0) {
    A* part = (A*)d.partial + (size_t)pend * 4 * NA;
    const A* Q = ACC0 + pend_par * 4 * NA;
    for (int q = tid; q < 4 * NA; q += kBlock) part[q] = Q[q];
  }

  if (status) atomicOr(&d.ctr->status, status);
  if (tid == 0 && (tl->inc | tl->esc)) {
    if (tl->inc) atomicAdd(&d.ctr->incident, tl->inc);
    if (tl->tr) atomicAdd(&d.ctr->transmitted, tl->tr);
    if (tl->ref) atomicAdd(&d.ctr->reflected, tl->ref);
    if (tl->esc) atomicAdd(&d.ctr->escaped, tl->esc);
    if (tl->fse != 0.0) atomicAdd(&d.ctr->fs_energy, tl->fse);
    if (tl->rem != 0.0) atomicAdd(&d.ctr->removed_energy, tl->rem);
  }
}


// REL: compiled with the relativistic terms (used when c2inv > 0). TXC, TYC:
// a tile shape compiled in (0: any shape, read from the geometry).
template <typename T, int DIM, int CH, int NS, bool REL, int TXC = 0, int TYC = 0>
__global__ void __launch_bounds__(kBlock, (sizeof(T) == 4 ? 4 : 2))
    k_push(DevPtrs<T> d, StepArgs a, PushConst<T> pc) {
  extern __shared__ __align__(128) unsigned char sm[];
  push_run<T, DIM, CH, NS, REL, TXC, TYC>(d, a.g, a.ph, pc, a.in, a.out, blockIdx.x, gridDim.x,
                                          sm);
}

// Batched push of an ensemble of independent runs in one persistent launch:
// CTA b works on run cta_map[b].x as rank cta_map[b].y of that run's group of
// runs[run].ncta CTAs; the run's pointers, geometry and physics come from the
// device table, copied once into shared memory.
// TXC: the tile width of every run the launch serves, compiled in (0: any)
// Three CTAs per SM in FP32 (at the four of k_push, its register cap spills).
template <typename T, int DIM, int CH, int NS, bool REL, int TXC = 0>
__global__ void __launch_bounds__(kBlock, (sizeof(T) == 4 ? 3 : 2))
    k_push_batch(const BatchRun<T>* __restrict__ runs, const int2* __restrict__ cta_map) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(16) BatchRun<T> R;
  const int2 cm = cta_map[blockIdx.x];
  static_assert(sizeof(BatchRun<T>) % 4 == 0, "run record copied as words");
  const int* src = reinterpret_cast<const int*>(runs + cm.x);
  int* dst = reinterpret_cast<int*>(&R);
  for (int k = threadIdx.x; k < (int)(sizeof(BatchRun<T>) / 4); k += kBlock) dst[k] = src[k];
  __syncthreads();
  push_run<T, DIM, CH, NS, REL, TXC, (TXC ? 1 : 0)>(R.d, R.g, R.ph, R.pc, R.in, R.out, cm.y,
                                                      R.ncta, sm);
}

// ---------------------------------------------------------------- batched step tail
// The rest of a batched step (movers, injection, moments, the 1D tiled field
// advance, the step counter) as one launch per kernel over every run of the
// batch: block b belongs to the run r with pre[r] <= b < pre[r + 1] and works
// as block b - pre[r] of that run's own launch; the run's record is copied
// into shared memory first. Same bodies, so the same results, as the per-run
// kernels.
__device__ __forceinline__ int batch_run_of(const int* pre, int nruns, int b) {
  int lo = 0, hi = nruns;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <typename T>
__device__ __forceinline__ int load_batch_run(const BatchRun<T>* runs, const int* pre, int nruns,
                                              BatchRun<T>& R) {
  __shared__ int s_run;
  if (threadIdx.x == 0) s_run = pre ? batch_run_of(pre, nruns, blockIdx.x) : (int)blockIdx.x;
  __syncthreads();
  const int r = s_run;
  const int* src = reinterpret_cast<const int*>(runs + r);
  int* dst = reinterpret_cast<int*>(&R);
  for (int k = threadIdx.x; k < (int)(sizeof(BatchRun<T>) / 4); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  return r;
}

template <typename T, int DIM>
__global__ void k_movers_batch(const BatchRun<T>* __restrict__ runs, const int* __restrict__ pre,
                               int nruns) {
  __shared__ __align__(16) BatchRun<T> R;
  const int r = load_batch_run<T>(runs, pre, nruns, R);
  movers_body<T, DIM>(R.d, R.g, R.out, blockIdx.x - pre[r], pre[r + 1] - pre[r]);
}

// one block per run
template <typename T, int DIM>
__global__ void k_inject_batch(const BatchRun<T>* __restrict__ runs, int nruns) {
  __shared__ __align__(16) BatchRun<T> R;
  load_batch_run<T>(runs, nullptr, nruns, R);
  if (R.g.bc_x == FS_BC_FAUXSHOCK && (R.ph.inject_thermal || R.ph.cr_enable))
    inject_run_block<T, DIM>(R.d, R.g, R.ph, R.out);
}

template <typename T, int DIM>
__global__ void k_moments_batch(const BatchRun<T>* __restrict__ runs,
                                const int* __restrict__ pre, int nruns) {
  __shared__ __align__(16) BatchRun<T> R;
  const int r = load_batch_run<T>(runs, pre, nruns, R);
  moments_body<T, DIM>(R.d, R.g, R.ph, blockIdx.x - pre[r], pre[r + 1] - pre[r]);
}

template <typename T>
__global__ void __launch_bounds__(kF1Threads)
    k_field1_batch(const BatchRun<T>* __restrict__ runs, const int* __restrict__ pre,
                   int nruns) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) BatchRun<T> R;
  const int r = load_batch_run<T>(runs, pre, nruns, R);
  const FieldConst<T> fc = field_const_dev<T>(R.ph);
  field_step1_body<T>(R.d.B, R.d.Bs, R.d.n, R.d.u, R.d.E, R.d.Bb, R.d.G, R.g, fc, R.n_sub,
                      blockIdx.x - pre[r], smem);
}

// the new B back from the stage buffer: tile b's cells, as the per-run copy
template <typename T>
__global__ void __launch_bounds__(kF1Threads)
    k_copyB_batch(const BatchRun<T>* __restrict__ runs, const int* __restrict__ pre,
                  int nruns) {
  __shared__ __align__(16) BatchRun<T> R;
  const int r = load_batch_run<T>(runs, pre, nruns, R);
  const int nx = R.g.nx, c0 = (blockIdx.x - pre[r]) * kF1, c1 = min(nx, c0 + kF1);
  for (int k = threadIdx.x; k < 3 * kF1; k += blockDim.x) {
    const int c = k / kF1, i = c0 + k % kF1;
    if (i < c1) R.d.B[c * nx + i] = R.d.Bs[c * nx + i];
  }
}

template <typename T>
__global__ void k_step_end_batch(const BatchRun<T>* __restrict__ runs, int nruns) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nruns; r += gridDim.x * blockDim.x)
    runs[r].d.ctr->step += 1;
}

}  // namespace fsx
