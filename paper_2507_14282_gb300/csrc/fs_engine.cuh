// fs_engine.cuh -- the hot-path kernels of one hybrid step, templated on the
// arithmetic type T (float or double) and the dimension DIM (1 or 2).
//
// Step n -> n+1 (Sec. 2 boundary inside a textbook hybrid PIC step):
//   k_push     persistent CTAs, each over a group of tiles of cells
//              (fs_push.cuh): CIC gather of E^n and Bbar^n from a
//              shared-memory field tile, Boris push, move, open far wall,
//              faux-shock pass/return (Eq. 1), in-tile counting sort by new
//              cell, CIC deposit of n and J by runs of sorted particles with a
//              warp team reduction into a shared-memory node tile, then
//              stayers written back to the tile's bucket and leavers to the
//              mover list. Deposit partials per tile, no global atomics
//              (except rare far movers).
//   k_movers   leavers appended to their destination tile's bucket (in the
//              captured step, beside the next three, which read no bucket).
//   k_inject_* thermal inflow at x = L and the cosmic-ray source at x = 0.
//   k_moments  sum of the per-tile partials in a fixed order, wall
//              half-volume correction, density floor, u = J / n
//              (k_moments_ct: the same with the 2D tile shape compiled in).
//   k_ohm / k_faraday  RK4 substeps of dB/dt = -curl E(B), E from Ohm's law.
//   k_ohm (final) also packs E and Bbar per node for the next gather.
//
// The FP64 instantiation is compiled without FMA contraction and evaluates
// every expression in the same order as the written scheme, so that it agrees
// bit for bit with an implementation of the same scheme on the CPU. Node sums
// of the FP64 deposit are int64 fixed point (2^-40), independent of order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fs_device.cuh"
#include "fs_internal.h"

namespace fsx {

constexpr int kBlock = 256;

template <typename T>
struct Num;
template <>
struct Num<float> {
  using acc = float;
  static constexpr float offmax = 0x1.fffffep-1f;
  __device__ static float fl(float x) { return floorf(x); }
  __device__ static float ab(float x) { return fabsf(x); }
};
template <>
struct Num<double> {
  using acc = unsigned long long;  // int64 fixed point, two's complement
  static constexpr double offmax = 0x1.fffffffffffffp-1;
  __device__ static double fl(double x) { return floor(x); }
  __device__ static double ab(double x) { return fabs(x); }
};

// A deposit contribution c (already scaled by 2^40 for FP64) in accumulator
// form. FP64: c rounded to the nearest integer, ties to even (llrint(c)),
// worked out on the bit pattern with integer shifts: the value is
// mant * 2^(e - 1075); the bits shifted out decide the rounding. Exact for
// every double; it keeps the addition off GB300's narrow FP64 pipe.
__device__ __forceinline__ float to_acc(float c) { return c; }
__device__ __forceinline__ unsigned long long to_acc(double c) {
  const long long b = __double_as_longlong(c);
  const int e = (int)((b >> 52) & 0x7FF);
  const long long mant = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const int sh = 1075 - e;  // right shift of the 53-bit significand
  long long r;
  if (e == 0 || sh > 53) {
    r = 0;  // zero, subnormal, or |c| < 1/2
  } else if (sh <= 0) {
    r = mant << (-sh);  // already an integer (|c| >= 2^52; a shift of at most 10 here)
  } else {
    const long long q = mant >> sh;
    const long long rem = mant - (q << sh);
    const long long half = 1LL << (sh - 1);
    r = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
  }
  return (unsigned long long)(b < 0 ? -r : r);
}
// a * b in accumulator form. FP64: rounded once from the exact product to
// the nearest integer (fma with 1.5 * 2^52), as the written scheme states.
// (An all-integer version with the 106-bit product measured 3 % slower in the
// push: the fused multiply-add is worth its FP64 pipe slot here.)
__device__ __forceinline__ float to_acc_prod(float a, float b) { return a * b; }
__device__ __forceinline__ unsigned long long to_acc_prod(double a, double b) {
  const double m = __fma_rn(a, b, 0x1.8p52);
  return (unsigned long long)(__double_as_longlong(m) -
                              __double_as_longlong(0x1.8p52));
}
__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rcpT(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double rcpT(double a) { return __drcp_rn(a); }
__device__ __forceinline__ float sqrtT(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrtT(double a) { return __dsqrt_rn(a); }
// an accumulator's value in the run's precision: FP32 sums as they are (no
// round trip through FP64, whose conversions use GB300's narrow FP64 pipe),
// FP64 fixed point scaled back by 2^-40
__device__ __forceinline__ float acc_value(float a) { return a; }
__device__ __forceinline__ double acc_value(unsigned long long a) {
  return (double)(long long)a * 0x1p-40;
}

template <typename T>
__device__ __forceinline__ T deposit_weight_scale() {
  return (T)1;
}
template <>
__device__ __forceinline__ double deposit_weight_scale<double>() {
  return 0x1p40;
}

__device__ __forceinline__ void atomic_acc(float* a, float v) { atomicAdd(a, v); }
__device__ __forceinline__ void atomic_acc(unsigned long long* a,
                                           unsigned long long v) {
  atomicAdd(a, v);
}

__device__ __forceinline__ float shfl_up(float v, int o) {
  return __shfl_up_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ unsigned long long shfl_up(unsigned long long v,
                                                      int o) {
  return __shfl_up_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ float shfl_xor(float v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ unsigned long long shfl_xor(unsigned long long v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}

__device__ __forceinline__ int wrap(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// Kinetic energy of a macroparticle of weight wp: wp v^2 / 2 (v stored), or
// for relativistic ions (u = gamma v stored, c2inv = 1/c^2 > 0)
// wp (gamma - 1) c^2 = wp u.u / (gamma + 1).
__device__ __forceinline__ double kinetic(double wp, double vx, double vy,
                                          double vz, double vol, double c2inv = 0.0) {
  if (c2inv > 0.0) {
    const double uu = __fma_rn(vz, vz, __fma_rn(vy, vy, __dmul_rn(vx, vx)));
    const double gamma = __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(uu, c2inv)));
    return __dmul_rn(__dmul_rn(wp, __ddiv_rn(uu, __dadd_rn(gamma, 1.0))), vol);
  }
  return __dmul_rn(
      __dmul_rn(__dmul_rn(wp, 0.5),
                __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)),
                          __dmul_rn(vz, vz))),
      vol);
}

// 1/gamma of a stored u = gamma v: 1 / sqrt(1 + u.u / c^2)
template <typename T>
__device__ __forceinline__ T inv_gamma_u(T ux, T uy, T uz, T c2inv) {
  const T uu = fmaT(uz, uz, fmaT(uy, uy, ux * ux));
  return (T)1 / sqrtT((T)1 + uu * c2inv);
}
// gamma of a velocity: 1 / sqrt(1 - v.v / c^2)
__device__ __forceinline__ double gamma_v(double vx, double vy, double vz, double c2inv) {
  const double vv = __fma_rn(vz, vz, __fma_rn(vy, vy, __dmul_rn(vx, vx)));
  return __ddiv_rn(1.0, __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(vv, c2inv))));
}
// the velocity of a stored state (u for relativistic ions, v otherwise)
template <typename T>
__device__ __forceinline__ void velocity_of(T ux, T uy, T uz, T c2inv, T& vx, T& vy, T& vz) {
  if (c2inv > (T)0) {
    const T ig = inv_gamma_u(ux, uy, uz, c2inv);
    vx = ux * ig;
    vy = uy * ig;
    vz = uz * ig;
  } else {
    vx = ux;
    vy = uy;
    vz = uz;
  }
}

// ------------------------------------------------------------------------
// Boris rotation, the written order: half kick, t = B dt/2,
// s = 2 t / (1 + t.t), v' = v- + v- x t, v+ = v- + v' x s (each component as
// two fused multiply-adds), half kick.
// ------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void boris(T& vx, T& vy, T& vz, const T E[3],
                                      const T B[3], T hdt, T c2inv = (T)0) {
  const T emx = hdt * E[0], emy = hdt * E[1], emz = hdt * E[2];
  const T vmx = vx + emx, vmy = vy + emy, vmz = vz + emz;
  // relativistic ions (u = gamma v stored): t = B dt / (2 gamma-), gamma-
  // from the half-kicked u
  T hg = hdt;
  if (c2inv > (T)0) {
    const T uu = fmaT(vmz, vmz, fmaT(vmy, vmy, vmx * vmx));
    hg = hdt / sqrtT((T)1 + uu * c2inv);
  }
  const T tx = hg * B[0], ty = hg * B[1], tz = hg * B[2];
  const T tt = fmaT(tz, tz, fmaT(ty, ty, tx * tx));
  // 2 / (1 + t.t) as 2 * (correctly rounded reciprocal): doubling is exact,
  // so this is the same number as the rounded quotient
  const T f = (T)2 * rcpT((T)1 + tt);
  const T sx = f * tx, sy = f * ty, sz = f * tz;
  const T px = fmaT(vmy, tz, fmaT(-vmz, ty, vmx));
  const T py = fmaT(vmz, tx, fmaT(-vmx, tz, vmy));
  const T pz = fmaT(vmx, ty, fmaT(-vmy, tx, vmz));
  const T qx = fmaT(py, sz, fmaT(-pz, sy, vmx));
  const T qy = fmaT(pz, sx, fmaT(-px, sz, vmy));
  const T qz = fmaT(px, sy, fmaT(-py, sx, vmz));
  vx = qx + emx;
  vy = qy + emy;
  vz = qz + emz;
}

// ------------------------------------------------------------------------
// Faux-shock decision (Sec. 2, Eq. 1) in FP64. Returns true and overwrites v
// when the particle is returned: P = ((1 - u2/v)/(1 + u2/v))^2 with v the
// speed in the chosen frame (0 when v <= u2); returned iff U0 < P and the
// downstream-frame speed |v'| = |v + u2 x| exceeds u2; the new direction has
// mu' = a + (1 - a) sqrt(U1), a = u2/|v'| (flux-weighted, isotropic in the
// downstream), azimuth 2 pi U2; |v'| is kept.
// ------------------------------------------------------------------------
__device__ __forceinline__ bool fs_return(double& vx, double& vy, double& vz,
                                          double u2, int frame,
                                          unsigned long long seed,
                                          uint32_t pid, long long step) {
  const double sp = __dsqrt_rn(__dadd_rn(
      __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
  const double wx = __dadd_rn(vx, u2);
  const double w = __dsqrt_rn(__dadd_rn(
      __dadd_rn(__dmul_rn(wx, wx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
  const double vp = (frame == FS_FRAME_SHOCK) ? sp : w;
  double prob = 0.0;
  if (vp > u2) {
    const double a = __ddiv_rn(u2, vp);
    const double q = __ddiv_rn(__dsub_rn(1.0, a), __dadd_rn(1.0, a));
    prob = __dmul_rn(q, q);
  }
  const Philox4 r = draw4(seed, pid, step, kPurposeFS);
  const double U0 = u01(r.x[0]), U1 = u01(r.x[1]), U2 = u01(r.x[2]);
  if (!(U0 < prob && w > u2)) return false;
  const double a = __ddiv_rn(u2, w);
  const double mu = __dadd_rn(a, __dmul_rn(__dsub_rn(1.0, a), __dsqrt_rn(U1)));
  const double sn = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(mu, mu)));
  double c, s;
  fs_sincos2pi(U2, &c, &s);
  const double ws = __dmul_rn(w, sn);
  vx = __dsub_rn(__dmul_rn(w, mu), u2);
  vy = __dmul_rn(ws, c);
  vz = __dmul_rn(ws, s);
  return true;
}

// ------------------------------------------------------------------------
// k_movers: append each leaver to its destination tile's bucket.
// ------------------------------------------------------------------------
// Block blk of nblk: one warp per source tile, its leavers go to their
// destination tiles.
// One leaver record of the mover list.
template <typename T>
struct MoverRec {
  int cell;
  T ox, oy, vx, vy, vz;
  uint32_t id;
};
template <typename T, int DIM>
__device__ __forceinline__ MoverRec<T> mover_load(const DevPtrs<T>& d, bool act, int src) {
  MoverRec<T> r;
  r.cell = act ? d.M.cell[src] : 0;
  r.ox = act ? d.M.ox[src] : (T)0;
  r.oy = (DIM == 2 && act) ? d.M.oy[src] : (T)0;
  r.vx = act ? d.M.vx[src] : (T)0;
  r.vy = act ? d.M.vy[src] : (T)0;
  r.vz = act ? d.M.vz[src] : (T)0;
  r.id = act ? d.M.id[src] : 0u;
  return r;
}
// destination tile of an active record (-1: none)
template <typename T>
__device__ __forceinline__ int mover_dest(const Geo& g, bool act, const MoverRec<T>& r) {
  const int i = r.cell & 0xFFFF, j = r.cell >> 16;
  return act ? (j / g.TY) * g.ntx + i / g.TX : -1;
}
template <typename T, int DIM>
__device__ __forceinline__ void mover_store(const DevPtrs<T>& d, const Geo& g, int out, bool act,
                                            int dt, int slot, const MoverRec<T>& r) {
  if (!act) return;
  if (slot >= g.tile_cap) {
    atomicSub(&d.cnt[out][dt], 1);
    atomicOr(&d.ctr->status, kStatusCapacity);
    return;
  }
  const Parts<T> PO = d.P[out];
  const int gi = dt * g.tile_cap + slot;  // a tile's bucket starts at tile x capacity
  PO.cell[gi] = r.cell;
  PO.ox[gi] = r.ox;
  if (DIM == 2) PO.oy[gi] = r.oy;
  PO.vx[gi] = r.vx;
  PO.vy[gi] = r.vy;
  PO.vz[gi] = r.vz;
  PO.id[gi] = r.id;
}

// Block blk of nblk: one warp per source tile, its leavers go to their
// destination tiles; each warp works on two source tiles at a time (their
// loads and slot atomics in flight together). Lanes bound for the same tile
// take consecutive slots after one atomic by the lowest of them.
template <typename T, int DIM>
__device__ __forceinline__ void movers_body(const DevPtrs<T>& d, const Geo& g, int out, int blk,
                                            int nblk) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int stride = nblk * wpb;
  const unsigned below = (1u << lane) - 1u;
  for (int t = blk * wpb + (threadIdx.x >> 5); t < g.ntiles; t += 2 * stride) {
    const int t2 = t + stride;
    const int nm1 = d.mcnt[t];
    const int nm2 = t2 < g.ntiles ? d.mcnt[t2] : 0;
    const int mb1 = t * g.mover_per_tile, mb2 = t2 * g.mover_per_tile;
    for (int k0 = 0; k0 < nm1 || k0 < nm2; k0 += 32) {  // counts are warp-uniform
      const int k = k0 + lane;
      const bool a1 = k < nm1, a2 = k < nm2;
      const MoverRec<T> r1 = mover_load<T, DIM>(d, a1, mb1 + k);
      const MoverRec<T> r2 = mover_load<T, DIM>(d, a2, mb2 + k);
      const int dt1 = mover_dest(g, a1, r1), dt2 = mover_dest(g, a2, r2);
      const unsigned p1 = __match_any_sync(0xffffffffu, dt1);
      const unsigned p2 = __match_any_sync(0xffffffffu, dt2);
      const int l1 = __ffs(p1) - 1, l2 = __ffs(p2) - 1;
      int b1 = 0, b2 = 0;
      if (a1 && lane == l1) b1 = atomicAdd(&d.cnt[out][dt1], __popc(p1));
      if (a2 && lane == l2) b2 = atomicAdd(&d.cnt[out][dt2], __popc(p2));
      b1 = __shfl_sync(0xffffffffu, b1, l1);
      b2 = __shfl_sync(0xffffffffu, b2, l2);
      mover_store<T, DIM>(d, g, out, a1, dt1, b1 + __popc(p1 & below), r1);
      mover_store<T, DIM>(d, g, out, a2, dt2, b2 + __popc(p2 & below), r2);
    }
  }
}

template <typename T, int DIM>
__global__ void k_movers(DevPtrs<T> d, Geo g, int out) {
  movers_body<T, DIM>(d, g, out, blockIdx.x, gridDim.x);
}

// Deposit of one particle into the far accumulators (global atomics).
template <typename T, int DIM>
__device__ __forceinline__ void deposit_far(const DevPtrs<T>& d, const Geo& g,
                                            int i, int j, T fx, T fy, T wp,
                                            T vx, T vy, T vz) {
  using A = typename Num<T>::acc;
  A* far = (A*)d.far;
  const size_t nn = (size_t)g.nxn * g.ny;
  const int i1 = (g.bc_x == FS_BC_PERIODIC && i + 1 == g.nx) ? 0 : i + 1;
  if (DIM == 1) {
    const T c0 = wp * ((T)1 - fx), c1 = wp * fx;
    atomic_acc(&far[0 * nn + i], to_acc(c0));
    atomic_acc(&far[1 * nn + i], to_acc_prod(c0, vx));
    atomic_acc(&far[2 * nn + i], to_acc_prod(c0, vy));
    atomic_acc(&far[3 * nn + i], to_acc_prod(c0, vz));
    atomic_acc(&far[0 * nn + i1], to_acc(c1));
    atomic_acc(&far[1 * nn + i1], to_acc_prod(c1, vx));
    atomic_acc(&far[2 * nn + i1], to_acc_prod(c1, vy));
    atomic_acc(&far[3 * nn + i1], to_acc_prod(c1, vz));
  } else {
    const int j1 = (j + 1 == g.ny) ? 0 : j + 1;
    const T gx0 = (T)1 - fx, gy0 = (T)1 - fy;
    const int nd[4] = {j * g.nxn + i, j * g.nxn + i1, j1 * g.nxn + i,
                       j1 * g.nxn + i1};
    const T cw[4] = {wp * (gx0 * gy0), wp * (fx * gy0), wp * (gx0 * fy),
                     wp * (fx * fy)};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      atomic_acc(&far[0 * nn + nd[c]], to_acc(cw[c]));
      atomic_acc(&far[1 * nn + nd[c]], to_acc_prod(cw[c], vx));
      atomic_acc(&far[2 * nn + nd[c]], to_acc_prod(cw[c], vy));
      atomic_acc(&far[3 * nn + nd[c]], to_acc_prod(cw[c], vz));
    }
  }
}

// Place one new particle into the bucket of its tile; deposit it.
template <typename T, int DIM>
__device__ __forceinline__ void place_new(const DevPtrs<T>& d, const Geo& g,
                                          const Phys& ph, int buf, int i, int j,
                                          T fx, T fy, T vx, T vy, T vz,
                                          uint32_t id) {
  const int t = (j / g.TY) * g.ntx + i / g.TX;
  const int slot = atomicAdd(&d.cnt[buf][t], 1);
  if (slot >= g.tile_cap) {
    atomicSub(&d.cnt[buf][t], 1);
    atomicOr(&d.ctr->status, kStatusCapacity);
    return;
  }
  const int gi = t * g.tile_cap + slot;  // a tile's bucket starts at tile x capacity
  const Parts<T> P = d.P[buf];
  P.cell[gi] = (j << 16) | i;
  P.ox[gi] = fx;
  if (DIM == 2) P.oy[gi] = fy;
  P.vx[gi] = vx;
  P.vy[gi] = vy;
  P.vz[gi] = vz;
  P.id[gi] = id;
  const double ws = deposit_weight_scale<T>();
  const T wp = (T)(((id & kIdCR) ? ph.w_cr : ph.w_th) * ws);
  T dvx, dvy, dvz;  // the current uses the velocity
  velocity_of<T>(vx, vy, vz, (T)ph.c2inv, dvx, dvy, dvz);
  deposit_far<T, DIM>(d, g, i, j, fx, fy, wp, dvx, dvy, dvz);
}

// ------------------------------------------------------------------------
// Injection (Sec. 2). k_inject_count (one CTA): per transverse row the
// accumulator advances by ppc u_sh dt/dx, its integer part is this step's
// count; a scan over rows gives each row's first id. k_inject_gen: one thread
// per (row, slot) draws the particle.
// ------------------------------------------------------------------------
// The whole block (any multiple of 32 threads up to 1024) counts every row.
__device__ __forceinline__ void inject_count_body(double* acc, int* rowcnt, int* rowoff, int ny,
                                                  double rate, int per_row_mult) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b = 0; b < ny; b += blockDim.x) {
    const int j = b + threadIdx.x;
    int n = 0;
    if (j < ny) {
      double v = __dadd_rn(acc[j], rate);
      const double fl = floor(v);
      n = (int)fl;
      acc[j] = __dsub_rn(v, fl);
      rowcnt[j] = n;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = n * per_row_mult;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
      int s = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
      int si = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, si, o);
        if (lane >= o) si += v;
      }
      if (lane < (int)(blockDim.x >> 5)) wsum[lane] = si - s;
    }
    __syncthreads();
    if (j < ny) rowoff[j] = carry + wsum[w] + inc - n * per_row_mult;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += wsum[w] + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) rowoff[ny] = carry;
}

static __global__ void k_inject_count(double* acc, int* rowcnt, int* rowoff, int ny,
                                      double rate, int per_row_mult) {
  inject_count_body(acc, rowcnt, rowoff, ny, rate, per_row_mult);
}

// New particle k of row j (thermal at x = L, then the cosmic rays at x = 0),
// ids from `first` (next_id before this step's injection) in (row, slot)
// order; counts and energy added to the caller's l_inj, l_e.
template <typename T, int DIM>
__device__ __forceinline__ void inject_one(const DevPtrs<T>& d, const Geo& g, const Phys& ph,
                                           int buf, const int* rowcnt, const int* rowoff, int j,
                                           int k, unsigned long long first, long long step,
                                           long long& l_inj, double& l_e) {
  if (j < g.ny) {
    const int n = rowcnt[j];
    if (k < n) {
      const int nx = g.nx;
      if (ph.inject_thermal) {
        const unsigned long long num = first + rowoff[j] + k;
        if (num > kIdMask) {
          atomicOr(&d.ctr->status, kStatusIdOverflow);
        } else {
          const uint32_t pid = (uint32_t)num;
          const Philox4 ra = draw4(ph.seed, pid, step, kPurposeInjA);
          const Philox4 rb = draw4(ph.seed, pid, step, kPurposeInjB);
          double g0, g1, g2, g3;
          gauss2(u01(ra.x[0]), u01(ra.x[1]), &g0, &g1);
          gauss2(u01(ra.x[2]), u01(ra.x[3]), &g2, &g3);
          const double vx = __dsub_rn(__dmul_rn(ph.vth, g0), ph.mach_a);
          const double vy = __dmul_rn(ph.vth, g1);
          const double vz = __dmul_rn(ph.vth, g2);
          const double X = __dsub_rn(
              (double)nx, __dmul_rn(__dmul_rn(u01(rb.x[0]), fabs(vx)), ph.dtdx));
          const double ix = floor(X);
          int i = (int)ix;
          double fx = __dsub_rn(X, ix);
          if (i >= nx) { i = nx - 1; fx = Num<double>::offmax; }
          if (i < 0) { i = 0; fx = 0.0; }
          if (fx >= 1.0) fx = Num<double>::offmax;
          const double fy = (DIM == 2) ? u01(rb.x[1]) : 0.0;
          T ft = (T)fx;
          if (ft >= (T)1) ft = Num<T>::offmax;
          T fyt = (T)fy;
          if (fyt >= (T)1) fyt = Num<T>::offmax;
          double ux = vx, uy = vy, uz = vz;  // stored as u = gamma v
          if (ph.c2inv > 0.0) {
            const double gv = gamma_v(vx, vy, vz, ph.c2inv);
            ux = __dmul_rn(vx, gv); uy = __dmul_rn(vy, gv); uz = __dmul_rn(vz, gv);
          }
          place_new<T, DIM>(d, g, ph, buf, i, j, ft, fyt, (T)ux, (T)uy, (T)uz, pid);
          ++l_inj;
          l_e = __dadd_rn(l_e, kinetic(ph.w_th, ux, uy, uz, ph.cellvol, ph.c2inv));
        }
      }
      if (ph.cr_enable) {
        const int thermal_n = ph.inject_thermal ? n : 0;
        const unsigned long long num = first + rowoff[j] + thermal_n + k;
        if (num > kIdMask) {
          atomicOr(&d.ctr->status, kStatusIdOverflow);
        } else {
          const uint32_t pid = (uint32_t)num;
          const Philox4 rc = draw4(ph.seed, pid, step, kPurposeInjCR);
          // speed p_iso / gamma(p_iso) in the downstream frame (p_iso without c)
          const double a = __ddiv_rn(ph.u_cr, ph.p_iso_v);
          const double mu =
              __dadd_rn(a, __dmul_rn(__dsub_rn(1.0, a), __dsqrt_rn(u01(rc.x[0]))));
          const double sn = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(mu, mu)));
          double c, s;
          fs_sincos2pi(u01(rc.x[1]), &c, &s);
          const double ws = __dmul_rn(ph.p_iso_v, sn);
          const double vx = __dsub_rn(__dmul_rn(ph.p_iso_v, mu), ph.u_cr);
          const double vy = __dmul_rn(ws, c);
          const double vz = __dmul_rn(ws, s);
          const double X = __dmul_rn(__dmul_rn(u01(rc.x[2]), vx), ph.dtdx);
          const double ix = floor(X);
          int i = (int)ix;
          double fx = __dsub_rn(X, ix);
          if (i >= nx) { i = nx - 1; fx = Num<double>::offmax; }
          if (i < 0) { i = 0; fx = 0.0; }
          if (fx >= 1.0) fx = Num<double>::offmax;
          const double fy = (DIM == 2) ? u01(rc.x[3]) : 0.0;
          T ft = (T)fx;
          if (ft >= (T)1) ft = Num<T>::offmax;
          T fyt = (T)fy;
          if (fyt >= (T)1) fyt = Num<T>::offmax;
          double ux = vx, uy = vy, uz = vz;  // stored as u = gamma v
          if (ph.c2inv > 0.0) {
            const double gv = gamma_v(vx, vy, vz, ph.c2inv);
            ux = __dmul_rn(vx, gv); uy = __dmul_rn(vy, gv); uz = __dmul_rn(vz, gv);
          }
          place_new<T, DIM>(d, g, ph, buf, i, j, ft, fyt, (T)ux, (T)uy, (T)uz,
                            pid | kIdCR);
          ++l_inj;
          l_e = __dadd_rn(l_e, kinetic(ph.w_cr, ux, uy, uz, ph.cellvol, ph.c2inv));
        }
      }
    }
  }
}

template <typename T, int DIM>
__global__ void k_inject_gen(DevPtrs<T> d, Geo g, Phys ph, int buf,
                             const int* rowcnt, const int* rowoff, int maxk) {
  const long long step = d.ctr->step;
  const int gidx = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = gidx / maxk, k = gidx % maxk;
  __shared__ unsigned long long s_first;
  if (threadIdx.x == 0) s_first = d.ctr->next_id;
  __syncthreads();
  const unsigned long long first = s_first;
  long long l_inj = 0;
  double l_e = 0.0;
  inject_one<T, DIM>(d, g, ph, buf, rowcnt, rowoff, j, k, first, step, l_inj, l_e);
  if (l_inj) {
    atomicAdd(&d.ctr->injected, (unsigned long long)l_inj);
    atomicAdd(&d.ctr->injected_energy, l_e);
  }
}

// The injection of one run by one whole block: the row counts (as
// k_inject_count), every (row, slot) draw (as k_inject_gen) and the id
// commit (as k_inject_commit), with block barriers between them.
template <typename T, int DIM>
__device__ __forceinline__ void inject_run_block(const DevPtrs<T>& d, const Geo& g,
                                                 const Phys& ph, int buf) {
  const int mult = (ph.inject_thermal ? 1 : 0) + (ph.cr_enable ? 1 : 0);
  int* rowcnt = d.inj;
  int* rowoff = rowcnt + g.ny;
  inject_count_body(d.acc, rowcnt, rowoff, g.ny, ph.rate, mult);
  __shared__ unsigned long long s_first;
  __shared__ long long s_step;
  if (threadIdx.x == 0) {
    s_first = d.ctr->next_id;
    s_step = d.ctr->step;
  }
  __syncthreads();
  const int maxk = (int)ph.rate + 2;
  long long l_inj = 0;
  double l_e = 0.0;
  for (int gidx = threadIdx.x; gidx < g.ny * maxk; gidx += blockDim.x)
    inject_one<T, DIM>(d, g, ph, buf, rowcnt, rowoff, gidx / maxk, gidx % maxk, s_first,
                       s_step, l_inj, l_e);
  if (l_inj) {
    atomicAdd(&d.ctr->injected, (unsigned long long)l_inj);
    atomicAdd(&d.ctr->injected_energy, l_e);
  }
  __syncthreads();
  if (threadIdx.x == 0) d.ctr->next_id += rowoff[g.ny];
}

// end of a step: advance the device step counter
static __global__ void k_step_end(Counters* ctr) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctr->step += 1;
}

// advance next_id by this step's total (after k_inject_gen has read it)
static __global__ void k_inject_commit(Counters* ctr, const int* rowoff, int ny) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctr->next_id += rowoff[ny];
}

// ------------------------------------------------------------------------
// k_moments: per node, the deposit partials of every tile whose accumulator
// covers it (tiles in increasing row, then column order; within a tile every
// accumulator slot that maps to the node), plus the far accumulator; then the
// wall half-volume correction (x2 at i = 0 and i = nx in the faux-shock box),
// the density floor and u = J / n.
// ------------------------------------------------------------------------
// The node's moments from its sums s (n, Jx, Jy, Jz); clears its far sums.
template <typename T, int DIM>
__device__ __forceinline__ void moments_finish(const DevPtrs<T>& d, const Geo& g, const Phys& ph,
                                               int q, int i, const typename Num<T>::acc (&s)[4]) {
  using A = typename Num<T>::acc;
  const int nn = g.nxn * g.ny;
  T nt = acc_value(s[0]), jxt = acc_value(s[1]), jyt = acc_value(s[2]), jzt = acc_value(s[3]);
  if (g.bc_x == FS_BC_FAUXSHOCK && (i == 0 || i == g.nx)) {
    nt = nt * (T)2; jxt = jxt * (T)2; jyt = jyt * (T)2; jzt = jzt * (T)2;
  }
  d.J[q] = jxt;
  d.J[(size_t)nn + q] = jyt;
  d.J[(size_t)2 * nn + q] = jzt;
  const T nf = (T)ph.n_floor;
  if (nt < nf) nt = nf;
  d.n[q] = nt;
  d.u[q] = jxt / nt;
  d.u[(size_t)nn + q] = jyt / nt;
  d.u[(size_t)2 * nn + q] = jzt / nt;
  A* farw = (A*)d.far;
#pragma unroll
  for (int c = 0; c < 4; ++c) farw[(size_t)c * nn + q] = (A)0;
}

template <typename T, int DIM>
__device__ __forceinline__ void moments_body(const DevPtrs<T>& d, const Geo& g, const Phys& ph,
                                             int blk, int nblk) {
  using A = typename Num<T>::acc;
  const int nn = g.nxn * g.ny;
  const int AX = g.TX + 3, AY = (DIM == 2) ? g.TY + 3 : 1, NA = AX * AY;
  for (int q = blk * blockDim.x + threadIdx.x; q < nn; q += nblk * blockDim.x) {
    const int i = q % g.nxn, j = q / g.nxn;
    // candidate tile columns / rows (distinct): a tile's accumulator spans
    // nodes i0 - 1 .. i0 + TX + 1, so tiles home - 2 .. home + 1 can cover i
    int tcx[4], ncx = 0, tcy[4], ncy = 0;
    {
      const int home = min(i / g.TX, g.ntx - 1);
      for (int dd = -2; dd <= 1; ++dd) {
        int c = home + dd;
        if (g.bc_x == FS_BC_PERIODIC) c = wrap(c, g.ntx);
        else if (c < 0 || c >= g.ntx) continue;
        bool dup = false;
        for (int k = 0; k < ncx; ++k) dup |= (tcx[k] == c);
        if (!dup) tcx[ncx++] = c;
      }
    }
    if (DIM == 2) {
      const int home = j / g.TY;
      for (int dd = -2; dd <= 1; ++dd) {
        const int c = wrap(home + dd, g.nty);
        bool dup = false;
        for (int k = 0; k < ncy; ++k) dup |= (tcy[k] == c);
        if (!dup) tcy[ncy++] = c;
      }
    } else {
      tcy[0] = 0;
      ncy = 1;
    }
    // sort candidates ascending (fixed summation order)
    for (int a = 0; a < ncx; ++a)
      for (int b = a + 1; b < ncx; ++b)
        if (tcx[b] < tcx[a]) { int t = tcx[a]; tcx[a] = tcx[b]; tcx[b] = t; }
    for (int a = 0; a < ncy; ++a)
      for (int b = a + 1; b < ncy; ++b)
        if (tcy[b] < tcy[a]) { int t = tcy[a]; tcy[a] = tcy[b]; tcy[b] = t; }
    A s[4];
    const A* far = (const A*)d.far;
#pragma unroll
    for (int c = 0; c < 4; ++c) s[c] = far[(size_t)c * nn + q];
    for (int yy = 0; yy < ncy; ++yy) {
      const int ty = tcy[yy];
      // accumulator rows of node row j (more than one only when the box is
      // narrower than a tile's accumulator)
      int ay0 = 0;
      if (DIM == 2) ay0 = wrap(j - (ty * g.TY - 1), g.ny);
      for (int ay = ay0; ay < AY; ay += (DIM == 2 ? g.ny : AY)) {
        for (int xx = 0; xx < ncx; ++xx) {
          const int tx = tcx[xx];
          const int t = ty * g.ntx + tx;
          const A* part = (const A*)d.partial + (size_t)t * 4 * NA;
          int ax0 = i - (tx * g.TX - 1);
          int step = AX;
          if (g.bc_x == FS_BC_PERIODIC) {
            ax0 = wrap(ax0, g.nx);
            step = g.nx;
          }
          for (int ax = ax0; ax >= 0 && ax < AX; ax += step) {
            const int k = ax + ay * AX;
#pragma unroll
            for (int c = 0; c < 4; ++c) s[c] += part[c * NA + k];
          }
        }
      }
    }
    moments_finish<T, DIM>(d, g, ph, q, i, s);
  }
}

template <typename T, int DIM>
__global__ void k_moments(DevPtrs<T> d, Geo g, Phys ph) {
  moments_body<T, DIM>(d, g, ph, blockIdx.x, gridDim.x);
}

// The same sums for a 2D box with x walls whose tile shape TXC x TYC is
// compiled in (and whose rows hold more than one tile's accumulator rows and
// more tile rows than cover a node): the candidate tiles of a node are a
// fixed, small set (MX columns by MY rows), so every load is issued without a
// data-dependent loop; rows are taken in increasing wrapped order, columns
// in increasing order, as in moments_body.
template <typename T, int TXC, int TYC>
__global__ void k_moments_ct(DevPtrs<T> d, Geo g, Phys ph) {
  using A = typename Num<T>::acc;
  constexpr int AX = TXC + 3, AY = TYC + 3, NA = AX * AY;
  constexpr int MX = (AX + TXC - 1) / TXC, MY = (AY + TYC - 1) / TYC;
  const int nn = g.nxn * g.ny;
  const A* far = (const A*)d.far;
  const A* partial = (const A*)d.partial;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nn; q += gridDim.x * blockDim.x) {
    const int i = q % g.nxn, j = q / g.nxn;
    // candidate rows: ty with 0 <= j - (ty TYC - 1) < AY, wrapped, ascending
    int tyw[MY], ayv[MY];
    const int tyh = (j + 1) / TYC;
#pragma unroll
    for (int u = 0; u < MY; ++u) {
      const int ty = tyh - (MY - 1) + u;
      const int ay = j - (ty * TYC - 1);
      const bool ok = ay >= 0 && ay < AY;
      tyw[u] = ok ? (ty < 0 ? ty + g.nty : (ty >= g.nty ? ty - g.nty : ty)) : 0x7fffffff;
      ayv[u] = ay;
    }
#pragma unroll
    for (int a = 0; a < MY; ++a)
#pragma unroll
      for (int b = a + 1; b < MY; ++b)
        if (tyw[b] < tyw[a]) {
          const int t0 = tyw[a], t1 = ayv[a];
          tyw[a] = tyw[b]; ayv[a] = ayv[b];
          tyw[b] = t0; ayv[b] = t1;
        }
    A s[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) s[c] = far[(size_t)c * nn + q];
    const int txh = (i + 1) / TXC;
#pragma unroll
    for (int u = 0; u < MY; ++u) {
      if (tyw[u] == 0x7fffffff) continue;
#pragma unroll
      for (int x = 0; x < MX; ++x) {
        const int tx = txh - (MX - 1) + x;
        const int ax = i - (tx * TXC - 1);
        if (tx < 0 || tx >= g.ntx || ax < 0 || ax >= AX) continue;
        const A* part = partial + (size_t)(tyw[u] * g.ntx + tx) * 4 * NA + ax + ayv[u] * AX;
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] += part[c * NA];
      }
    }
    moments_finish<T, 2>(d, g, ph, q, i, s);
  }
}

// ------------------------------------------------------------------------
// Ohm's law at the nodes (massless isothermal electrons, J = curl B), the
// cross products and the 1/n scaling written as fused multiply-adds:
//   E = ((curl B - j_ext x) x Bbar)/n - u x Bbar - T_e grad n / n (+ eta curl B)
// Bbar is B averaged onto the nodes; derivatives are two-point differences
// averaged across the transverse direction; x walls use zero-gradient ghost
// cells (and a mirrored density gradient), periodic boxes wrap.
// With G != nullptr also packs (E, Bbar) per node, plus a ghost row ny
// (copy of row 0) and, in a periodic box, a ghost column nx (copy of 0).
// With pre != nullptr the density terms come from k_ohm_pre (same values).
// ------------------------------------------------------------------------
// The density terms of Ohm's law at node (i, j), fixed while n is: 1/n and
// the pressure terms -(T_e dn/dx), -(T_e dn/dy) (two-point differences, a
// mirrored density gradient at the x walls, periodic wrap).
template <typename T, int DIM>
__device__ __forceinline__ void density_terms(const T* __restrict__ nN, int i, int j,
                                              const Geo& g, const Phys& ph, T& inv_n,
                                              T& pgx, T& pgy) {
  const int nx = g.nx, ny = g.ny, nxn = g.nxn;
  const bool per = (g.bc_x == FS_BC_PERIODIC);
  const T te = (T)ph.te;
  auto nxo = [&](int c) {
    if (per) return wrap(c, nx);
    if (c < 0) return -c;
    if (c > nx) return 2 * nx - c;
    return c;
  };
  T dnx, dny;
  if (DIM == 1) {
    dnx = (nN[nxo(i + 1)] - nN[nxo(i - 1)]) * (T)ph.hdx;
    dny = (T)0;
  } else {
    dnx = (nN[j * nxn + nxo(i + 1)] - nN[j * nxn + nxo(i - 1)]) * (T)ph.hdx;
    dny = (nN[wrap(j + 1, ny) * nxn + i] - nN[wrap(j - 1, ny) * nxn + i]) * (T)ph.hdy;
  }
  inv_n = (T)1 / nN[j * nxn + i];
  pgx = -(te * dnx);
  pgy = -(te * dny);
}

// Writes density_terms for every node once per step (n is fixed during the
// field substeps): pre = [1/n][-(T_e dn/dx)][-(T_e dn/dy)] planes.
template <typename T, int DIM>
__global__ void k_ohm_pre(const T* __restrict__ nN, T* __restrict__ pre, Geo g, Phys ph) {
  const int nxn = g.nxn;
  const int nn = nxn * g.ny;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nn; q += gridDim.x * blockDim.x) {
    const int i = q % nxn, j = q / nxn;
    T inv_n, pgx, pgy;
    density_terms<T, DIM>(nN, i, j, g, ph, inv_n, pgx, pgy);
    pre[q] = inv_n;
    pre[nn + q] = pgx;
    pre[2 * nn + q] = pgy;
  }
}

// The node value of Ohm's law from curl B (cxv, cyv, czv), Bbar, 1/n, the
// pressure terms and u.
template <typename T>
__device__ __forceinline__ void ohm_e(T cxv, T cyv, T czv, T bbx, T bby, T bbz, T inv_n, T pgx,
                                      T pgy, T ux, T uy, T uz, T jcr, T eta, bool resist,
                                      T& ex, T& ey, T& ez) {
  const T ax = cxv - jcr, ay = cyv, az = czv;
  const T cax = fmaT(ay, bbz, -(az * bby));
  const T cay = fmaT(az, bbx, -(ax * bbz));
  const T caz = fmaT(ax, bby, -(ay * bbx));
  const T cux = fmaT(uy, bbz, -(uz * bby));
  const T cuy = fmaT(uz, bbx, -(ux * bbz));
  const T cuz = fmaT(ux, bby, -(uy * bbx));
  ex = fmaT(pgx, inv_n, fmaT(cax, inv_n, -cux));
  ey = fmaT(pgy, inv_n, fmaT(cay, inv_n, -cuy));
  ez = fmaT(caz, inv_n, -cuz);
  if (resist) {
    ex = ex + eta * cxv;
    ey = ey + eta * cyv;
    ez = ez + eta * czv;
  }
}

// The RK4 stage update of one B component from K = -curl E:
//   stage 1: Bsum = K;            Bs = B + (h/2) K
//   stage 2: Bsum = Bsum + 2 K;   Bs = B + (h/2) K
//   stage 3: Bsum = Bsum + 2 K;   Bs = B + h K
//   stage 4: Bsum = Bsum + K;     B  = B + (h/6) Bsum
template <typename T>
__device__ __forceinline__ void rk4_stage(int stage, T K, T& bsum, T& bs, T& b, T h, T hh,
                                          T h6) {
  if (stage == 1) {
    bsum = K;
    bs = fmaT(hh, K, b);
  } else if (stage == 2) {
    bsum = fmaT((T)2, K, bsum);
    bs = fmaT(hh, K, b);
  } else if (stage == 3) {
    bsum = fmaT((T)2, K, bsum);
    bs = fmaT(h, K, b);
  } else {
    const T sum = bsum + K;
    b = fmaT(h6, sum, b);
  }
}

// Ohm's law at node q = j * nxn + i (the body of k_ohm).
template <typename T, int DIM>
__device__ __forceinline__ void ohm_node(int q, const T* Bc, const T* nN, const T* uN,
                                         const T* pre, T* Eo, T* Bbo, T* G, const Geo& g,
                                         const Phys& ph) {
  const int nx = g.nx, ny = g.ny, nxn = g.nxn;
  const int nc = nx * ny, nn = nxn * ny;
  const T hdx = (T)ph.hdx, hdy = (T)ph.hdy, idx = (T)ph.idx;
  const T jcr = (T)ph.jcr, eta = (T)ph.eta;
  const bool per = (g.bc_x == FS_BC_PERIODIC);
  {
    const int i = q % nxn, j = q / nxn;
    auto cxo = [&](int c) { return per ? wrap(c, nx) : min(max(c, 0), nx - 1); };
    T bbx, bby, bbz, cxv, cyv, czv;
    if (DIM == 1) {
      const int im = cxo(i - 1), ip = cxo(i);
      const T bmx = Bc[im], bpx = Bc[ip];
      const T bmy = Bc[nc + im], bpy = Bc[nc + ip];
      const T bmz = Bc[2 * nc + im], bpz = Bc[2 * nc + ip];
      bbx = (T)0.5 * (bmx + bpx);
      bby = (T)0.5 * (bmy + bpy);
      bbz = (T)0.5 * (bmz + bpz);
      const T dby = (bpy - bmy) * idx;
      const T dbz = (bpz - bmz) * idx;
      cxv = (T)0;
      cyv = -dbz;
      czv = dby;
    } else {
      const int im = cxo(i - 1), ip = cxo(i);
      const int jm = wrap(j - 1, ny), jp = j;
      const int cmm = jm * nx + im, cpm = jm * nx + ip;
      const int cmp = jp * nx + im, cpp = jp * nx + ip;
      T b[3][4];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        b[c][0] = Bc[c * nc + cmm];
        b[c][1] = Bc[c * nc + cpm];
        b[c][2] = Bc[c * nc + cmp];
        b[c][3] = Bc[c * nc + cpp];
      }
      bbx = (T)0.25 * ((b[0][0] + b[0][1]) + (b[0][2] + b[0][3]));
      bby = (T)0.25 * ((b[1][0] + b[1][1]) + (b[1][2] + b[1][3]));
      bbz = (T)0.25 * ((b[2][0] + b[2][1]) + (b[2][2] + b[2][3]));
      const T dxby = ((b[1][3] + b[1][1]) - (b[1][2] + b[1][0])) * hdx;
      const T dxbz = ((b[2][3] + b[2][1]) - (b[2][2] + b[2][0])) * hdx;
      const T dybx = ((b[0][3] + b[0][2]) - (b[0][1] + b[0][0])) * hdy;
      const T dybz = ((b[2][3] + b[2][2]) - (b[2][1] + b[2][0])) * hdy;
      cxv = dybz;
      cyv = -dxbz;
      czv = dxby - dybx;
    }
    T inv_n, pgx, pgy;
    if (pre) {
      inv_n = pre[q];
      pgx = pre[nn + q];
      pgy = pre[2 * nn + q];
    } else {
      density_terms<T, DIM>(nN, i, j, g, ph, inv_n, pgx, pgy);
    }
    T ex, ey, ez;
    ohm_e<T>(cxv, cyv, czv, bbx, bby, bbz, inv_n, pgx, pgy, uN[q], uN[nn + q], uN[2 * nn + q],
             jcr, eta, ph.eta != 0.0, ex, ey, ez);
    Eo[q] = ex;
    Eo[nn + q] = ey;
    Eo[2 * nn + q] = ez;
    if (Bbo) {
      Bbo[q] = bbx;
      Bbo[nn + q] = bby;
      Bbo[2 * nn + q] = bbz;
    }
    if (G) {
      const T v[8] = {ex, ey, ez, bbx, bby, bbz, (T)0, (T)0};
      const int gx = nx + 1;
      auto put = [&](int gi, int gj) {
        T* dst = G + ((size_t)gj * gx + gi) * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) dst[c] = v[c];
      };
      put(i, j);
      if (j == 0) put(i, ny);
      if (per && i == 0) {
        put(nx, j);
        if (j == 0) put(nx, ny);
      }
    }
  }
}

template <typename T, int DIM>
__global__ void k_ohm(const T* __restrict__ Bc, const T* __restrict__ nN,
                      const T* __restrict__ uN, const T* __restrict__ pre,
                      T* __restrict__ Eo, T* __restrict__ Bbo, T* __restrict__ G, Geo g,
                      Phys ph) {
  const int nn = g.nxn * g.ny;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nn; q += gridDim.x * blockDim.x)
    ohm_node<T, DIM>(q, Bc, nN, uN, pre, Eo, Bbo, G, g, ph);
}

// Faraday at centre c = j * nx + i, K = -curl E from the four corner nodes
// (two in 1D), and the RK4 stage update (rk4_stage): the body of k_faraday.
template <typename T, int DIM>
__device__ __forceinline__ void faraday_cell(int c, const T* En, T* B, T* Bs, T* Bsum,
                                             int stage, const Geo& g, const Phys& ph) {
  const int nx = g.nx, ny = g.ny, nxn = g.nxn;
  const int nc = nx * ny, nn = nxn * ny;
  const T hdx = (T)ph.hdx, hdy = (T)ph.hdy, idx = (T)ph.idx;
  const T h = (T)ph.h, hh = (T)ph.hh, h6 = (T)ph.h6;
  const bool per = (g.bc_x == FS_BC_PERIODIC);
  {
    const int i = c % nx, j = c / nx;
    const int i1 = (per && i + 1 == nx) ? 0 : i + 1;
    T K[3];
    if (DIM == 1) {
      const T dxey = (En[nn + i1] - En[nn + i]) * idx;
      const T dxez = (En[2 * nn + i1] - En[2 * nn + i]) * idx;
      K[0] = (T)0;
      K[1] = dxez;
      K[2] = -dxey;
    } else {
      const int j1 = (j + 1 == ny) ? 0 : j + 1;
      const int q00 = j * nxn + i, q10 = j * nxn + i1;
      const int q01 = j1 * nxn + i, q11 = j1 * nxn + i1;
      const T dxey = ((En[nn + q10] + En[nn + q11]) - (En[nn + q00] + En[nn + q01])) * hdx;
      const T dxez = ((En[2 * nn + q10] + En[2 * nn + q11]) -
                      (En[2 * nn + q00] + En[2 * nn + q01])) * hdx;
      const T dyex = ((En[q01] + En[q11]) - (En[q00] + En[q10])) * hdy;
      const T dyez = ((En[2 * nn + q01] + En[2 * nn + q11]) -
                      (En[2 * nn + q00] + En[2 * nn + q10])) * hdy;
      K[0] = -dyez;
      K[1] = dxez;
      K[2] = dyex - dxey;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const size_t k = (size_t)q * nc + c;
      rk4_stage<T>(stage, K[q], Bsum[k], Bs[k], B[k], h, hh, h6);
    }
  }
}

template <typename T, int DIM>
__global__ void k_faraday(const T* __restrict__ En, T* __restrict__ B,
                          T* __restrict__ Bs, T* __restrict__ Bsum, int stage,
                          Geo g, Phys ph) {
  const int nc = g.nx * g.ny;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
    faraday_cell<T, DIM>(c, En, B, Bs, Bsum, stage, g, ph);
}

// The field kernels' constants in the run's precision, formed on the host
// (kernel parameters of that type need no FP64 conversion on the device).
template <typename T>
struct FieldConst {
  T idx, hdx, hdy, te, jcr, eta;  // 1/dx, 1/(2dx), 1/(2dy), T_e, j_cr, eta
  T h, hh, h6;                    // RK4 substep h, h/2, h/6
  int resist;                     // eta != 0
};
template <typename T>
inline FieldConst<T> field_const(const Phys& ph) {
  return FieldConst<T>{(T)ph.idx, (T)ph.hdx, (T)ph.hdy, (T)ph.te, (T)ph.jcr,
                       (T)ph.eta, (T)ph.h,   (T)ph.hh,  (T)ph.h6, ph.eta != 0.0 ? 1 : 0};
}
// the same on the device (IEEE conversions round alike on host and device)
template <typename T>
__device__ __forceinline__ FieldConst<T> field_const_dev(const Phys& ph) {
  return FieldConst<T>{(T)ph.idx, (T)ph.hdx, (T)ph.hdy, (T)ph.te, (T)ph.jcr,
                       (T)ph.eta, (T)ph.h,   (T)ph.hh,  (T)ph.h6, ph.eta != 0.0 ? 1 : 0};
}

// ------------------------------------------------------------------------
// The whole field advance of a 1D step with x walls (n_sub RK4 substeps,
// then Ohm's E and Bbar for the next gather) in one launch: on a 1D grid
// the separate passes are tens of tiny launches per step. A CTA owns kF1
// cells (and their left nodes; the last tile also node nx) and runs every
// pass in shared memory over its cells plus field1_halo(n_sub) cells around
// them, which it recomputes: each pass's stencil reaches one cell, so
// values made wrong at a tile's inner edges (read with indices clamped to
// the tile) move in by one cell per pass and stay outside the owned cells;
// at a wall the clamped indices are the wall's ghost cells and the density
// is mirrored as in density_terms. Reads B from Bin, writes the new B to
// Bout (neighbouring tiles read Bin's cells), E, Bbar and the packed gather
// block G at the owned nodes. Same per-element arithmetic as ohm_node /
// faraday_cell (1D), so FP64 results are those of the separate passes.
constexpr int kF1 = 64, kF1Threads = 128;
__host__ __device__ inline int field1_halo(int n_sub) { return 4 * n_sub + 2; }
template <typename T>
inline size_t field1_smem(int n_sub) {
  const size_t L = kF1 + 2 * (size_t)field1_halo(n_sub);
  return sizeof(T) * (9 * L + 7 * (L + 1));
}

// Tile blk of the 1D field advance (the body of k_field_step1); smem is the
// block's dynamic shared memory (field1_smem(n_sub) bytes).
template <typename T>
__device__ __forceinline__ void field_step1_body(const T* __restrict__ Bin, T* __restrict__ Bout,
                                                 const T* __restrict__ nN,
                                                 const T* __restrict__ uN, T* __restrict__ Eo,
                                                 T* __restrict__ Bbo, T* __restrict__ G,
                                                 const Geo& g, const FieldConst<T>& fc,
                                                 int n_sub, int blk, unsigned char* smem) {
  const int nx = g.nx, nxn = g.nxn, t0 = threadIdx.x, nt = blockDim.x;
  const int H = field1_halo(n_sub);
  const int c0 = blk * kF1, c1 = min(nx, c0 + kF1);
  const int lo = max(0, c0 - H), L = min(nx, c1 + H) - lo, Ln = L + 1;
  T* sB = (T*)smem;
  T* sBs = sB + 3 * L;
  T* sK = sBs + 3 * L;
  T* sE = sK + 3 * L;  // [3][Ln]
  T* sn = sE + 3 * Ln;
  T* su = sn + Ln;     // [3][Ln]
#pragma unroll
  for (int c = 0; c < 3; ++c)
    for (int a = t0; a < L; a += nt) sB[c * L + a] = Bin[c * nx + lo + a];
  for (int a = t0; a < Ln; a += nt) {
    sn[a] = nN[lo + a];
#pragma unroll
    for (int c = 0; c < 3; ++c) su[c * Ln + a] = uN[c * nxn + lo + a];
  }
  __syncthreads();
  const T idx = fc.idx, hdx = fc.hdx, te = fc.te, jcr = fc.jcr, eta = fc.eta;
  const T h = fc.h, hh = fc.hh, h6 = fc.h6;
  const bool resist = fc.resist != 0;
  // Ohm at local node a from the centre field Bc (local layout)
  auto ohm = [&](const T* Bc, int a, T E[3], T Bb[3]) {
    const int im = min(max(a - 1, 0), L - 1), ip = min(a, L - 1);
    const T bmy = Bc[L + im], bpy = Bc[L + ip], bmz = Bc[2 * L + im], bpz = Bc[2 * L + ip];
    Bb[0] = (T)0.5 * (Bc[im] + Bc[ip]);
    Bb[1] = (T)0.5 * (bmy + bpy);
    Bb[2] = (T)0.5 * (bmz + bpz);
    const T dby = (bpy - bmy) * idx;
    const T dbz = (bpz - bmz) * idx;
    const int gi = lo + a;
    const int xp = ((gi + 1 > nx) ? 2 * nx - (gi + 1) : gi + 1) - lo;
    const int xm = ((gi - 1 < 0) ? -(gi - 1) : gi - 1) - lo;
    const T dnx = (sn[min(max(xp, 0), L)] - sn[min(max(xm, 0), L)]) * hdx;
    const T inv_n = (T)1 / sn[a];
    ohm_e<T>((T)0, -dbz, dby, Bb[0], Bb[1], Bb[2], inv_n, -(te * dnx), -(te * (T)0), su[a],
             su[Ln + a], su[2 * Ln + a], jcr, eta, resist, E[0], E[1], E[2]);
  };
  for (int sub = 0; sub < n_sub; ++sub) {
    for (int stage = 1; stage <= 4; ++stage) {
      const T* Bc = (stage == 1) ? sB : sBs;
      for (int a = t0; a < Ln; a += nt) {
        T E[3], Bb[3];
        ohm(Bc, a, E, Bb);
        sE[a] = E[0];
        sE[Ln + a] = E[1];
        sE[2 * Ln + a] = E[2];
      }
      __syncthreads();
      for (int a = t0; a < L; a += nt) {
        const T dxey = (sE[Ln + a + 1] - sE[Ln + a]) * idx;
        const T dxez = (sE[2 * Ln + a + 1] - sE[2 * Ln + a]) * idx;
        const T K[3] = {(T)0, dxez, -dxey};
#pragma unroll
        for (int c = 0; c < 3; ++c)
          rk4_stage<T>(stage, K[c], sK[c * L + a], sBs[c * L + a], sB[c * L + a], h, hh, h6);
      }
      __syncthreads();
    }
  }
  for (int a = t0; a < Ln; a += nt) {
    const int gi = lo + a;
    if (gi < c0 || (gi >= c1 && !(gi == nx && c1 == nx))) continue;
    T E[3], Bb[3];
    ohm(sB, a, E, Bb);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Eo[c * nxn + gi] = E[c];
      Bbo[c * nxn + gi] = Bb[c];
    }
    const T v[8] = {E[0], E[1], E[2], Bb[0], Bb[1], Bb[2], (T)0, (T)0};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      G[(size_t)gi * 8 + c] = v[c];                  // row 0
      G[((size_t)(nx + 1) + gi) * 8 + c] = v[c];     // its ghost copy (row ny = 1)
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
    for (int a = t0; a < L; a += nt) {
      const int gi = lo + a;
      if (gi >= c0 && gi < c1) Bout[c * nx + gi] = sB[c * L + a];
    }
}

template <typename T>
__global__ void __launch_bounds__(kF1Threads)
    k_field_step1(const T* __restrict__ Bin, T* __restrict__ Bout, const T* __restrict__ nN,
                  const T* __restrict__ uN, T* __restrict__ Eo, T* __restrict__ Bbo,
                  T* __restrict__ G, Geo g, Phys ph, FieldConst<T> fc, int n_sub) {
  extern __shared__ __align__(16) unsigned char smem[];
  field_step1_body<T>(Bin, Bout, nN, uN, Eo, Bbo, G, g, fc, n_sub, blockIdx.x, smem);
}

// ------------------------------------------------------------------------
// One RK4 substep of the 2D field advance by tiles, for boxes with x walls
// (as separate passes it is memory-bound in FP32: each stage's Ohm and
// Faraday re-read and re-write the grid). A CTA owns kFTX x kFTY cells (and
// their lower-left nodes; the last tile in x also the wall nodes nx) and
// runs the four stages in shared memory over its cells plus a halo of 4
// cells (5 when it also forms E), which it recomputes: a stage's stencils reach one cell (node (i, j) reads
// cells i-1..i, j-1..j and n at i±1, j±1; cell (i, j) reads nodes i..i+1,
// j..j+1), so values made wrong at a tile's inner edges (read there with
// indices clamped to the tile) move in by one cell per pass and stay outside
// the owned cells. At an x wall the tile ends at the wall, where the clamped
// indices are the wall's zero-gradient ghost cells and the density is
// mirrored as in density_terms; y is periodic (rows wrap when loaded).
// Reads B from Bin and writes the new B to Bout (neighbouring tiles read
// Bin's cells). With `fin`, also Ohm's E and Bbar at the owned nodes from
// the new B (Eo, Bbo, and the packed gather block G with its ghost row), as
// the step's final k_ohm does. Same per-element arithmetic as ohm_node /
// faraday_cell (2D). Boxes that are a whole number of tiles (x and y) run
// the interior tile columns 1 .. gx - 2 (full tiles whose halo lies inside
// the box) as one launch with the tile's local sizes compiled in, and the
// two wall columns as a second launch of the general form.
constexpr int kFTX = 32, kFTY = 16, kFH = 5;  // owned cells; halo of the last substep
constexpr int kFLX = kFTX + 2 * kFH, kFLY = kFTY + 2 * kFH;
constexpr int kFNPT = ((kFLX + 1) * (kFLY + 1) + kBlock - 1) / kBlock;  // nodes per thread
// (the density, needed only for the density terms at the start, shares the
// first E plane)
template <typename T>
constexpr size_t field_tile_smem() {
  return sizeof(T) * (9 * (size_t)kFLX * kFLY + 3 * (size_t)(kFLX + 1) * (kFLY + 1));
}

// Walks the elements k = t0, t0 + kBlock, ... of an nx-by-ny local array,
// keeping (a, b) = (k mod nx, k div nx) by increments.
struct TileWalk {
  int k, a, b, da, db, n, w;
  __device__ __forceinline__ TileWalk(int t0, int w_, int h_) : k(t0), n(w_ * h_), w(w_) {
    b = t0 / w_;
    a = t0 - b * w_;
    db = kBlock / w_;
    da = kBlock - db * w_;
  }
  __device__ __forceinline__ void next() {
    k += kBlock;
    a += da;
    b += db;
    if (a >= w) {
      a -= w;
      ++b;
    }
  }
};

// FINC: -1 / -2 (fin from the argument) or the compile-time fin of an interior
// tile launch (a full tile whose halo lies inside the box: its local sizes
// are constants); bx0: the first tile column of the launch (blockIdx.x + bx0)
template <typename T, int FINC>
__global__ void __launch_bounds__(kBlock, (FINC >= 0 ? 4 : 1))
    k_field_substep2(const T* __restrict__ Bin, T* __restrict__ Bout, const T* __restrict__ nN,
                     const T* __restrict__ uN, T* __restrict__ Eo, T* __restrict__ Bbo,
                     T* __restrict__ G, Geo g, Phys ph, FieldConst<T> fc, int fin_arg, int bx0,
                     int bx_last) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int fin = FINC >= 0 ? FINC : fin_arg;
  const int nx = g.nx, ny = g.ny, nxn = g.nxn;
  const int nc = nx * ny, nn = nxn * ny;
  const int H = fin ? kFH : kFH - 1;  // four stages need 4 cells, the final Ohm one more
  // interior launch: columns bx0 ..; edge launch (FINC -1): columns 0 and
  // bx_last; FINC -2: every column, general sizes
  const int bx = (FINC >= 0) ? (int)blockIdx.x + bx0
                 : (FINC == -1 ? (blockIdx.x == 0 ? 0 : bx_last) : (int)blockIdx.x);
  const int cx0 = bx * kFTX, cx1 = (FINC >= 0) ? cx0 + kFTX : min(nx, cx0 + kFTX);
  const int cy0 = blockIdx.y * kFTY, cy1 = (FINC >= 0) ? cy0 + kFTY : min(ny, cy0 + kFTY);
  const int lx0 = (FINC >= 0) ? cx0 - H : max(0, cx0 - H);
  const int LX = (FINC >= 0) ? kFTX + 2 * H : min(nx, cx1 + H) - lx0;  // local cell columns
  const int ly0 = cy0 - H, LY = (cy1 - cy0) + 2 * H;             // local rows (unwrapped)
  const int NX = LX + 1, NC = LX * LY, NN = NX * (LY + 1);        // nodes: NX x (LY + 1)
  T* sB = (T*)smem;
  T* sBs = sB + 3 * NC;
  T* sK = sBs + 3 * NC;
  T* sE = sK + 3 * NC;  // [3][NN]
  T* sn = sE;           // [NN], read only before the first stage writes sE
  const int t0 = threadIdx.x;
  auto row = [&](int b) { return wrap(ly0 + b, ny); };
  // (unrolled so that a thread's loads are in flight together)
#pragma unroll 8
  for (TileWalk w(t0, LX, 3 * LY); w.k < 3 * NC; w.next()) {
    const int c = w.b / LY, b = w.b - c * LY;
    sB[w.k] = Bin[(size_t)c * nc + (size_t)row(b) * nx + lx0 + w.a];
  }
  // this thread's nodes: u and (after the barrier) the density terms, fixed
  // for the substep, stay in registers
  T u[kFNPT][3], inv_n[kFNPT], pgx[kFNPT], pgy[kFNPT];
  {
    TileWalk w(t0, NX, LY + 1);
#pragma unroll
    for (int r = 0; r < kFNPT; ++r, w.next()) {
      if (w.k < NN) {
        const size_t q = (size_t)row(w.b) * nxn + lx0 + w.a;
        sn[w.k] = nN[q];
        u[r][0] = uN[q];
        u[r][1] = uN[nn + q];
        u[r][2] = uN[2 * nn + q];
      }
    }
  }
  __syncthreads();
  const T hdx = fc.hdx, hdy = fc.hdy, te = fc.te, jcr = fc.jcr, eta = fc.eta;
  const T h = fc.h, hh = fc.hh, h6 = fc.h6;
  const bool resist = fc.resist != 0;
  {
    TileWalk w(t0, NX, LY + 1);
#pragma unroll
    for (int r = 0; r < kFNPT; ++r, w.next()) {
      if (w.k < NN) {
        // x neighbours mirrored at the walls, y neighbours in the tile
        const int gx = lx0 + w.a;
        const int xp = ((gx + 1 > nx) ? 2 * nx - (gx + 1) : gx + 1) - lx0;
        const int xm = ((gx - 1 < 0) ? -(gx - 1) : gx - 1) - lx0;
        const int rb = w.b * NX;
        const T dnx = (sn[rb + min(max(xp, 0), LX)] - sn[rb + min(max(xm, 0), LX)]) * hdx;
        const T dny = (sn[min(w.b + 1, LY) * NX + w.a] - sn[max(w.b - 1, 0) * NX + w.a]) * hdy;
        inv_n[r] = (T)1 / sn[w.k];
        pgx[r] = -(te * dnx);
        pgy[r] = -(te * dny);
      }
    }
  }
  __syncthreads();  // the density terms are read before sE (which holds sn) is written
  // Ohm at local node (a, b), the r-th of this thread, from the centre field Bc
  auto ohm = [&](const T* Bc, int a, int b, int r, T E[3], T Bb[3]) {
    const int im = min(max(a - 1, 0), LX - 1), ip = min(a, LX - 1);
    const int jm = min(max(b - 1, 0), LY - 1), jp = min(b, LY - 1);
    const int cmm = jm * LX + im, cpm = jm * LX + ip, cmp = jp * LX + im, cpp = jp * LX + ip;
    T v[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[c][0] = Bc[c * NC + cmm];
      v[c][1] = Bc[c * NC + cpm];
      v[c][2] = Bc[c * NC + cmp];
      v[c][3] = Bc[c * NC + cpp];
    }
    Bb[0] = (T)0.25 * ((v[0][0] + v[0][1]) + (v[0][2] + v[0][3]));
    Bb[1] = (T)0.25 * ((v[1][0] + v[1][1]) + (v[1][2] + v[1][3]));
    Bb[2] = (T)0.25 * ((v[2][0] + v[2][1]) + (v[2][2] + v[2][3]));
    const T dxby = ((v[1][3] + v[1][1]) - (v[1][2] + v[1][0])) * hdx;
    const T dxbz = ((v[2][3] + v[2][1]) - (v[2][2] + v[2][0])) * hdx;
    const T dybx = ((v[0][3] + v[0][2]) - (v[0][1] + v[0][0])) * hdy;
    const T dybz = ((v[2][3] + v[2][2]) - (v[2][1] + v[2][0])) * hdy;
    ohm_e<T>(dybz, -dxbz, dxby - dybx, Bb[0], Bb[1], Bb[2], inv_n[r], pgx[r], pgy[r], u[r][0],
             u[r][1], u[r][2], jcr, eta, resist, E[0], E[1], E[2]);
  };
  for (int stage = 1; stage <= 4; ++stage) {
    const T* Bc = (stage == 1) ? sB : sBs;
    {
      TileWalk w(t0, NX, LY + 1);
#pragma unroll
      for (int r = 0; r < kFNPT; ++r, w.next()) {
        if (w.k < NN) {
          T E[3], Bb[3];
          ohm(Bc, w.a, w.b, r, E, Bb);
          sE[w.k] = E[0];
          sE[NN + w.k] = E[1];
          sE[2 * NN + w.k] = E[2];
        }
      }
    }
    __syncthreads();
    for (TileWalk w(t0, LX, LY); w.k < NC; w.next()) {
      const int k = w.k;
      const int q00 = w.b * NX + w.a, q10 = q00 + 1, q01 = q00 + NX, q11 = q01 + 1;
      const T dxey = ((sE[NN + q10] + sE[NN + q11]) - (sE[NN + q00] + sE[NN + q01])) * hdx;
      const T dxez =
          ((sE[2 * NN + q10] + sE[2 * NN + q11]) - (sE[2 * NN + q00] + sE[2 * NN + q01])) * hdx;
      const T dyex = ((sE[q01] + sE[q11]) - (sE[q00] + sE[q10])) * hdy;
      const T dyez =
          ((sE[2 * NN + q01] + sE[2 * NN + q11]) - (sE[2 * NN + q00] + sE[2 * NN + q10])) * hdy;
      const T K[3] = {-dyez, dxez, dyex - dxey};
#pragma unroll
      for (int c = 0; c < 3; ++c)
        rk4_stage<T>(stage, K[c], sK[c * NC + k], sBs[c * NC + k], sB[c * NC + k], h, hh, h6);
    }
    __syncthreads();
  }
  // owned cells: the new B
  const int oa0 = cx0 - lx0, ob0 = H;
  const int ow = cx1 - cx0, oh = cy1 - cy0;
  for (TileWalk w(t0, ow, 3 * oh); w.k < 3 * ow * oh; w.next()) {
    const int c = w.b / oh, y = w.b - c * oh;
    Bout[(size_t)c * nc + (size_t)(cy0 + y) * nx + cx0 + w.a] =
        sB[c * NC + (ob0 + y) * LX + oa0 + w.a];
  }
  if (!fin) return;
  // owned nodes (and the wall nodes nx in the last tile): E, Bbar, G; each
  // thread takes the owned nodes among its own (their density terms and u
  // are in its registers)
  const int ox1 = cx1 + (cx1 == nx ? 1 : 0);
  TileWalk w(t0, NX, LY + 1);
#pragma unroll
  for (int r = 0; r < kFNPT; ++r, w.next()) {
    if (w.k >= NN) continue;
    const int i = lx0 + w.a, y = w.b - ob0;
    if (i < cx0 || i >= ox1 || y < 0 || y >= oh) continue;
    const int j = cy0 + y;
    T E[3], Bb[3];
    ohm(sB, w.a, w.b, r, E, Bb);
    const size_t q = (size_t)j * nxn + i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Eo[(size_t)c * nn + q] = E[c];
      Bbo[(size_t)c * nn + q] = Bb[c];
    }
    const T v[8] = {E[0], E[1], E[2], Bb[0], Bb[1], Bb[2], (T)0, (T)0};
    T* dst = G + ((size_t)j * (nx + 1) + i) * 8;
#pragma unroll
    for (int c = 0; c < 8; ++c) dst[c] = v[c];
    if (j == 0) {
      T* gh = G + ((size_t)ny * (nx + 1) + i) * 8;
#pragma unroll
      for (int c = 0; c < 8; ++c) gh[c] = v[c];
    }
  }
}

// ------------------------------------------------------------------------
// Initial load (Sec. 2 set-up): ppc particles per cell, ids in cell-major
// order, position uniform in the cell, velocity a Maxwellian of thermal speed
// sqrt(beta_i/2) drifting at -u_sh x.
// ------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void k_init_particles(DevPtrs<T> d, Geo g, Phys ph, int buf, int ppc) {
  const long long total = (long long)g.nx * g.ny * ppc;
  const Parts<T> P = d.P[buf];
  for (long long pidl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       pidl < total; pidl += (long long)gridDim.x * blockDim.x) {
    const uint32_t pid = (uint32_t)pidl;
    const long long cidx = pidl / ppc;
    const int k = (int)(pidl % ppc);
    const int i = (int)(cidx % g.nx), j = (int)(cidx / g.nx);
    const int tx = i / g.TX, ty = j / g.TY;
    const int t = ty * g.ntx + tx;
    const int lc = (i - tx * g.TX) + (j - ty * g.TY) * g.TX;
    const int gi = d.tile_base[t] + lc * ppc + k;
    const Philox4 ra = draw4(ph.seed, pid, 0, kPurposeInitA);
    const Philox4 rb = draw4(ph.seed, pid, 0, kPurposeInitB);
    const double fx = u01(ra.x[0]);
    const double fy = (DIM == 2) ? u01(ra.x[1]) : 0.0;
    double g0, g1, g2, g3;
    gauss2(u01(ra.x[2]), u01(ra.x[3]), &g0, &g1);
    gauss2(u01(rb.x[0]), u01(rb.x[1]), &g2, &g3);
    double vx = __dsub_rn(__dmul_rn(ph.vth, g0), ph.mach_a);
    double vy = __dmul_rn(ph.vth, g1);
    double vz = __dmul_rn(ph.vth, g2);
    if (ph.c2inv > 0.0) {  // stored as u = gamma v
      const double gv = gamma_v(vx, vy, vz, ph.c2inv);
      vx = __dmul_rn(vx, gv); vy = __dmul_rn(vy, gv); vz = __dmul_rn(vz, gv);
    }
    T ft = (T)fx, fyt = (T)fy;
    if (ft >= (T)1) ft = Num<T>::offmax;
    if (fyt >= (T)1) fyt = Num<T>::offmax;
    P.cell[gi] = (j << 16) | i;
    P.ox[gi] = ft;
    if (DIM == 2) P.oy[gi] = fyt;
    P.vx[gi] = (T)vx;
    P.vy[gi] = (T)vy;
    P.vz[gi] = (T)vz;
    P.id[gi] = pid;
  }
}

// Deposit every particle of buffer buf into the far accumulators (set-up and
// after a host injection; the per-tile partials are zero then).
template <typename T, int DIM>
__global__ void k_deposit_all(DevPtrs<T> d, Geo g, Phys ph, int buf) {
  const int t = blockIdx.x;
  const int cnt = min(d.cnt[buf][t], g.tile_cap);
  const int base = d.tile_base[t];
  const Parts<T> P = d.P[buf];
  const double ws = deposit_weight_scale<T>();
  const T wth = (T)(ph.w_th * ws), wcr = (T)(ph.w_cr * ws);
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
    const int gi = base + p;
    const int cell = P.cell[gi];
    const uint32_t id = P.id[gi];
    T vx, vy, vz;  // the current uses the velocity
    velocity_of<T>(P.vx[gi], P.vy[gi], P.vz[gi], (T)ph.c2inv, vx, vy, vz);
    deposit_far<T, DIM>(d, g, cell & 0xFFFF, cell >> 16, P.ox[gi],
                        DIM == 2 ? P.oy[gi] : (T)0, (id & kIdCR) ? wcr : wth, vx, vy, vz);
  }
}

// Insert n staged particles (validated on the host) into buffer buf.
template <typename T, int DIM>
__global__ void k_insert_staged(DevPtrs<T> d, Parts<T> src, Geo g, int buf, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += gridDim.x * blockDim.x) {
    const int cell = src.cell[k];
    const int i = cell & 0xFFFF, j = cell >> 16;
    const int t = (j / g.TY) * g.ntx + i / g.TX;
    const int slot = atomicAdd(&d.cnt[buf][t], 1);
    if (slot >= g.tile_cap) {
      atomicSub(&d.cnt[buf][t], 1);
      atomicOr(&d.ctr->status, kStatusCapacity);
      continue;
    }
    const int gi = d.tile_base[t] + slot;
    const Parts<T> P = d.P[buf];
    P.cell[gi] = cell;
    P.ox[gi] = src.ox[k];
    if (DIM == 2) P.oy[gi] = src.oy[k];
    P.vx[gi] = src.vx[k];
    P.vy[gi] = src.vy[k];
    P.vz[gi] = src.vz[k];
    P.id[gi] = src.id[k];
  }
}

// ------------------------------------------------------------------------
// Diagnostics (FP64 sums; order of the block partial sums is not fixed).
// ------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, int DIM>
__global__ void k_diag_particles(DevPtrs<T> d, Geo g, Phys ph, int buf) {
  const int t = blockIdx.x;
  const int cnt = min(d.cnt[buf][t], g.tile_cap), base = d.tile_base[t];
  const Parts<T> P = d.P[buf];
  double s[4] = {0, 0, 0, 0};
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
    const int gi = base + p;
    const double wp = (P.id[gi] & kIdCR) ? ph.w_cr : ph.w_th;
    const double vx = P.vx[gi], vy = P.vy[gi], vz = P.vz[gi];
    s[0] += kinetic(wp, vx, vy, vz, ph.cellvol, ph.c2inv);
    s[1] += (wp * vx) * ph.cellvol;
    s[2] += (wp * vy) * ph.cellvol;
    s[3] += (wp * vz) * ph.cellvol;
  }
  __shared__ double red[4][kBlock / 32];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double v = warp_sum(s[q]);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    atomicAdd(&d.ctr->sums[threadIdx.x], v);
  }
}

template <typename T>
__global__ void k_diag_field(DevPtrs<T> d, Geo g, Phys ph) {
  const int nc = g.nx * g.ny;
  double s = 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc;
       c += gridDim.x * blockDim.x) {
    const double bx = d.B[c], by = d.B[nc + c], bz = d.B[2 * nc + c];
    s += (0.5 * ((bx * bx + by * by) + bz * bz)) * ph.cellvol;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(&d.ctr->sums[4], s);
  // Stability number of the field integrator, z = h omega_max with h the
  // RK4 substep: the fastest discrete mode is bounded by the grid-scale
  // whistler, k^2 |Bbar| / n with k^2 <= 4/dx^2 + 4/dy^2 for the staggered
  // differences, plus advection, k |u| with k <= 2/dx + 2/dy. Kept as the
  // maximum over nodes in sums[5] (non-negative doubles order like their
  // bit patterns).
  const double kk = 16.0 * (ph.hdx * ph.hdx + ph.hdy * ph.hdy);
  const double ka = 4.0 * (ph.hdx + ph.hdy);
  const int nn = g.nxn * g.ny;
  double zmax = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nn;
       c += gridDim.x * blockDim.x) {
    const double bx = d.Bb[c], by = d.Bb[nn + c], bz = d.Bb[2 * nn + c];
    const double ux = d.u[c], uy = d.u[nn + c], uz = d.u[2 * nn + c];
    const double b = sqrt(bx * bx + by * by + bz * bz);
    const double um = sqrt(ux * ux + uy * uy + uz * uz);
    const double z = ph.h * (kk * b / (double)d.n[c] + ka * um);
    zmax = z > zmax ? z : zmax;  // a NaN z leaves zmax; NaN is caught elsewhere
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, zmax, o);
    zmax = w > zmax ? w : zmax;
  }
  if ((threadIdx.x & 31) == 0 && zmax > 0.0)
    atomicMax((unsigned long long*)&d.ctr->sums[5], (unsigned long long)__double_as_longlong(zmax));
}

template <typename T, int DIM>
__global__ void k_hist(DevPtrs<T> d, Geo g, Phys ph, int buf, int species) {
  const int t = blockIdx.x;
  const int cnt = min(d.cnt[buf][t], g.tile_cap), base = d.tile_base[t];
  const Parts<T> P = d.P[buf];
  const double hsx = (double)ph.hist_nx / (double)g.nx;
  const double hsp = (double)ph.hist_np / (ph.hist_pmax - ph.hist_pmin);
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
    const int gi = base + p;
    const int cr = (P.id[gi] & kIdCR) ? 1 : 0;
    if (species >= 0 && cr != species) continue;
    const int cell = P.cell[gi];
    int bx = (int)floor(((double)(cell & 0xFFFF) + (double)P.ox[gi]) * hsx);
    bx = min(max(bx, 0), ph.hist_nx - 1);
    const double bpd = floor(((double)P.vx[gi] - ph.hist_pmin) * hsp);
    if (!(bpd >= 0.0 && bpd < (double)ph.hist_np)) continue;
    atomicAdd(&d.hist[(size_t)bx * ph.hist_np + (int)bpd], 1ull);
  }
}

// y-averaged n at nodes and |B - B0|^2 at centres (rows summed in order)
template <typename T>
__global__ void k_profiles(DevPtrs<T> d, Geo g, Phys ph) {
  const int nc = g.nx * g.ny, nn = g.nxn * g.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.nxn;
       i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < g.ny; ++j) acc = acc + (double)d.n[j * g.nxn + i];
    d.prof[i] = acc / (double)g.ny;
    if (i < g.nx) {
      double a2 = 0.0;
      for (int j = 0; j < g.ny; ++j) {
        const int c = j * g.nx + i;
        const double dbx = (double)d.B[c] - ph.b0x;
        const double dby = (double)d.B[nc + c] - ph.b0y;
        const double dbz = (double)d.B[2 * nc + c] - ph.b0z;
        a2 = a2 + ((dbx * dbx + dby * dby) + dbz * dbz);
      }
      d.prof[g.nxn + i] = a2 / (double)g.ny;
    }
  }
  (void)nn;
}

// Grid export / import in FP64 host layout ([row][col][component]).
template <typename T>
__global__ void k_export_grid(const T* src, int planes, int cols, int rows,
                              double* dst) {
  const int n = cols * rows;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += gridDim.x * blockDim.x)
    for (int c = 0; c < planes; ++c)
      dst[(size_t)q * planes + c] = (double)src[(size_t)c * n + q];
}

template <typename T>
__global__ void k_import_B(T* B, const double* src, int nc) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc;
       q += gridDim.x * blockDim.x)
    for (int c = 0; c < 3; ++c) B[(size_t)c * nc + q] = (T)src[(size_t)q * 3 + c];
}

// Compact every live particle of buffer buf: dst rows (fx, fy, vx, vy, vz).
template <typename T, int DIM>
__global__ void k_export_particles(DevPtrs<T> d, Geo g, int buf, double* dst,
                                   int* cell_out, uint32_t* id_out,
                                   int* count) {
  const int t = blockIdx.x;
  const int cnt = min(d.cnt[buf][t], g.tile_cap), base = d.tile_base[t];
  __shared__ int sb;
  if (threadIdx.x == 0) sb = atomicAdd(count, cnt);
  __syncthreads();
  const Parts<T> P = d.P[buf];
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
    const int gi = base + p, o = sb + p;
    cell_out[o] = P.cell[gi];
    id_out[o] = P.id[gi];
    dst[(size_t)o * 5 + 0] = (double)P.ox[gi];
    dst[(size_t)o * 5 + 1] = DIM == 2 ? (double)P.oy[gi] : 0.0;
    dst[(size_t)o * 5 + 2] = (double)P.vx[gi];
    dst[(size_t)o * 5 + 3] = (double)P.vy[gi];
    dst[(size_t)o * 5 + 4] = (double)P.vz[gi];
  }
}

}  // namespace fsx
