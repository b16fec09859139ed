// fs_window.cu -- the differentiable window of the 1D faux-shock box: a
// forward pass of `steps` hybrid steps that keeps checkpoints, and the
// reverse (adjoint) sweep that gives the gradient of a loss at the window's
// end with respect to theta = (a_1..a_M, u_cr, u2): the amplitudes of seeded
// transverse-B modes, the cosmic-ray drift speed and the faux-shock kick.
//
// The step is the engine's (Sec. 2): CIC gather, Boris push, move, open far
// wall, faux-shock return (Eq. 1) at x = 0, thermal inflow at x = L and the
// cosmic-ray source at x = 0, CIC deposit, RK4 Ohm's law + Faraday with the
// moments frozen. The window keeps its particles in fixed slots (birth
// order; removed particles keep a dead slot), so that each particle's tape
// and adjoint stay in place across steps. Branches (crossings, returns,
// escapes, the density floor) and random draws are frozen: the backward
// differentiates the discrete map along the forward's branches. Every
// segment of `ckpt` steps is recomputed from its checkpoint during the
// backward; the deposit sums are int64 fixed point, so a recomputed segment
// reproduces the forward exactly in either precision.
#include <algorithm>
#include <vector>

#include "fs_engine.cuh"

namespace fsx {
namespace win {

constexpr double kUnfix = 1.0 / 1099511627776.0;
enum : uint8_t { kEvNone = 0, kEvReturned = 1, kEvRemoved = 2 };

template <typename T>
struct Slots {  // particle slots: cell (-1: removed), offset, velocity, id
  int* ci;
  T* f;
  T* v;  // [3][cap]
  uint32_t* id;
};

template <typename T>
struct Win {
  int cap;  // particle slots
  Slots<T> s;
  // fields: B at centres [3][nx] (and the buffer the next B is written to);
  // E, Bbar at nodes [3][nxn]
  T *B, *Bx, *E, *Bb;
  T *n, *u, *nraw;             // moments in use [nxn], [3][nxn], [nxn]
  unsigned long long* q;       // fixed-point deposit sums [4][nxn]
  unsigned long long* ctr;     // incident, returned, transmitted, escaped, injected
  // adjoint
  T *lf, *lv;                  // particle adjoints: offset, velocity [3][cap]
  double *lB, *lBx;            // of B [3][nx] (and the buffer the next one goes to)
  double *lE, *lBb;            // of E, Bbar [3][nxn]
  double *lNm, *lUm;           // of the moments that E^n used [nxn], [3][nxn]
  T *lNr, *lJ;                 // of the deposit sums (raw density, current), run precision
  double* grad;                // d loss / d theta [M + 2]
};

// ---------------------------------------------------------------- forward
// Gather, Boris push, move, far wall and faux-shock crossing of slot p.
template <typename T>
__device__ __forceinline__ void push_slot(int p, const Win<T>& w, const Slots<T>& tape,
                                          uint8_t* ev, const Geo& g, const Phys& ph,
                                          const PushConst<T>& pc, long long step) {
  const int nxn = g.nxn;
  {
    int ci = w.s.ci[p];
    T f = w.s.f[p];
    T vx = w.s.v[p], vy = w.s.v[w.cap + p], vz = w.s.v[2 * w.cap + p];
    uint32_t id = w.s.id[p];
    if (tape.ci) {
      tape.ci[p] = ci;
      tape.f[p] = f;
      tape.v[p] = vx;
      tape.v[w.cap + p] = vy;
      tape.v[2 * w.cap + p] = vz;
    }
    if (ci < 0) {
      if (ev) ev[p] = kEvRemoved;
      return;
    }
    uint8_t e = kEvNone;
    const T g0 = (T)1 - f;
    T Ep[3], Bp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Ep[c] = fmaT(f, w.E[c * nxn + ci + 1], g0 * w.E[c * nxn + ci]);
      Bp[c] = fmaT(f, w.Bb[c * nxn + ci + 1], g0 * w.Bb[c * nxn + ci]);
    }
    boris<T>(vx, vy, vz, Ep, Bp, pc.hdt);
    const T fr = fmaT(vx, pc.dtdx, f);
    const T k = Num<T>::fl(fr);
    int inew = ci + (int)k;
    T fn = fr - k;
    if (fn >= (T)1) fn = Num<T>::offmax;
    if (inew >= g.nx) {
      atomicAdd(&w.ctr[3], 1ull);
      e = kEvRemoved;
    } else if (inew < 0) {
      atomicAdd(&w.ctr[0], 1ull);
      const int mode = (id & kIdCR) ? FS_SHOCK : ph.fs_mode_thermal;
      double dvx = vx, dvy = vy, dvz = vz;
      if (mode == FS_SHOCK &&
          fs_return(dvx, dvy, dvz, ph.u2, ph.fs_frame, ph.seed, id & kIdMask, step)) {
        atomicAdd(&w.ctr[1], 1ull);
        const double Xo = __dadd_rn((double)ci, (double)f);
        const double Xn = __dadd_rn((double)ci, (double)fr);
        const double gfr = __ddiv_rn(Xn, __dsub_rn(Xn, Xo));
        double ff = __dmul_rn(gfr, __dmul_rn(dvx, ph.dtdx));
        if (ff < 0.0) ff = 0.0;
        if (ff >= 1.0) ff = (double)Num<double>::offmax;
        T ft = (T)ff;
        if (ft >= (T)1) ft = Num<T>::offmax;
        fn = ft;
        inew = 0;
        vx = (T)dvx;
        vy = (T)dvy;
        vz = (T)dvz;
        id |= kIdReturned;
        e = kEvReturned;
      } else {
        atomicAdd(&w.ctr[2], 1ull);
        e = kEvRemoved;
      }
    }
    if (ev) ev[p] = e;
    if (e == kEvRemoved) {
      w.s.ci[p] = -1;
      return;
    }
    w.s.ci[p] = inew;
    w.s.f[p] = fn;
    w.s.v[p] = vx;
    w.s.v[w.cap + p] = vy;
    w.s.v[2 * w.cap + p] = vz;
    w.s.id[p] = id;
  }
}

// The velocity and placement of a new cosmic ray (speed p_iso, direction
// flux-weighted in the frame drifting at u_cr), drawn as the engine draws
// it. Returns X in cells; U (optional) = {sqrt(U1), cos, sin, U_place}.
__device__ __forceinline__ double cr_draw(const Phys& ph, uint32_t pid, long long step,
                                          double* v, double* U) {
  const Philox4 rc = draw4(ph.seed, pid, step, kPurposeInjCR);
  const double s1 = __dsqrt_rn(u01(rc.x[0]));
  const double a = __ddiv_rn(ph.u_cr, ph.p_iso_v);
  const double mu = __dadd_rn(a, __dmul_rn(__dsub_rn(1.0, a), s1));
  const double sn = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(mu, mu)));
  double c, s;
  fs_sincos2pi(u01(rc.x[1]), &c, &s);
  const double ws = __dmul_rn(ph.p_iso_v, sn);
  v[0] = __dsub_rn(__dmul_rn(ph.p_iso_v, mu), ph.u_cr);
  v[1] = __dmul_rn(ws, c);
  v[2] = __dmul_rn(ws, s);
  if (U) {
    U[0] = s1;
    U[1] = c;
    U[2] = s;
    U[3] = u01(rc.x[2]);
  }
  return __dmul_rn(__dmul_rn(u01(rc.x[2]), v[0]), ph.dtdx);
}

// n_new thermal ions at x = L, then n_new cosmic rays at x = 0, into slots
// np .. np + 2 n_new (ids first, first + 1, ...), as the engine draws them.
template <typename T>
__device__ __forceinline__ void inject_one(int k, const Win<T>& w, const Geo& g,
                                           const Phys& ph, long long step, int np, int n_new,
                                           unsigned long long first) {
  const int nth = ph.inject_thermal ? n_new : 0;
  const int ncr = ph.cr_enable ? n_new : 0;
  if (k >= nth + ncr) return;
  const uint32_t pid = (uint32_t)(first + k);
  const int nx = g.nx;
  double vx, vy, vz, X;
  uint32_t id = pid;
  if (k < nth) {
    const Philox4 ra = draw4(ph.seed, pid, step, kPurposeInjA);
    const Philox4 rb = draw4(ph.seed, pid, step, kPurposeInjB);
    double g0, g1, g2, g3;
    gauss2(u01(ra.x[0]), u01(ra.x[1]), &g0, &g1);
    gauss2(u01(ra.x[2]), u01(ra.x[3]), &g2, &g3);
    vx = __dsub_rn(__dmul_rn(ph.vth, g0), ph.mach_a);
    vy = __dmul_rn(ph.vth, g1);
    vz = __dmul_rn(ph.vth, g2);
    X = __dsub_rn((double)nx, __dmul_rn(__dmul_rn(u01(rb.x[0]), fabs(vx)), ph.dtdx));
  } else {
    double v[3];
    X = cr_draw(ph, pid, step, v, nullptr);
    vx = v[0];
    vy = v[1];
    vz = v[2];
    id |= kIdCR;
  }
  const double ix = floor(X);
  int i = (int)ix;
  double fx = __dsub_rn(X, ix);
  if (i >= nx) { i = nx - 1; fx = Num<double>::offmax; }
  if (i < 0) { i = 0; fx = 0.0; }
  if (fx >= 1.0) fx = Num<double>::offmax;
  T ft = (T)fx;
  if (ft >= (T)1) ft = Num<T>::offmax;
  const int p = np + k;
  w.s.ci[p] = i;
  w.s.f[p] = ft;
  w.s.v[p] = (T)vx;
  w.s.v[w.cap + p] = (T)vy;
  w.s.v[2 * w.cap + p] = (T)vz;
  w.s.id[p] = id;
  if (k == 0) atomicAdd(&w.ctr[4], (unsigned long long)(nth + ncr));
}

// One launch for the push of slots 0 .. np - 1 and the injection into
// slots np .. (the two touch disjoint slots): the first `ib` blocks inject,
// so that their long FP64 draw chains start first, the rest push. Also
// clears the fixed-point sums for the step's deposit.
template <typename T>
__global__ void k_win_push_inject(Win<T> w, Slots<T> tape, uint8_t* ev, Geo g, Phys ph,
                                  PushConst<T> pc, long long step, int np, int n_new,
                                  unsigned long long first, int ib) {
  // the deposit sums, read by the previous step's field kernel, start over
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 4 * g.nxn; k += gridDim.x * blockDim.x)
    w.q[k] = 0ull;
  if ((int)blockIdx.x < ib) {
    inject_one<T>(blockIdx.x * blockDim.x + threadIdx.x, w, g, ph, step, np, n_new, first);
    return;
  }
  const int stride = (gridDim.x - ib) * blockDim.x;
  for (int p = (blockIdx.x - ib) * blockDim.x + threadIdx.x; p < np; p += stride)
    push_slot<T>(p, w, tape, ev, g, ph, pc, step);
}

// c * 2^40 rounded to the nearest integer, ties to even (the value of
// __double2ll_rn(c * 2^40) for |c| < 2^23), on the bit pattern with integer
// operations: the significand shifted right by 1035 - e with the rounding
// of the bits shifted out, kept off the FP64 pipe.
__device__ __forceinline__ unsigned long long fix(double c) {
  const long long b = __double_as_longlong(c);
  const int e = (int)((b >> 52) & 0x7FF);
  const long long mant = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const int sh = 1035 - e;
  long long r;
  if (e == 0 || sh > 53) {
    r = 0;  // zero, subnormal, or |c| 2^40 < 1/2
  } else if (sh <= 0) {
    r = mant << (-sh);
  } else {
    const long long q = mant >> sh;
    const long long rem = mant - (q << sh);
    const long long half = 1LL << (sh - 1);
    r = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
  }
  return (unsigned long long)(b < 0 ? -r : r);
}

// c * 2^40 rounded to the nearest integer for an FP32 value c (|c| < 2^23):
// the scaling is exact; below 2^30 the int32 conversion rounds to nearest
// (ties to even), at or above it the value is an integer already (its ulp is
// at least 2^7) and its significand is shifted into place.
__device__ __forceinline__ long long fix32(float c) {
  const float y = c * 0x1p40f;
  if (fabsf(y) < 0x1p30f) return (long long)__float2int_rn(y);
  const int b = __float_as_int(y);
  const int e = (b >> 23) & 0xFF;
  const long long r = (long long)((b & 0x7FFFFF) | 0x800000) << (e - 150);
  return b < 0 ? -r : r;
}

// Sum of v over the lanes of `mask` (all of which call it with that mask),
// exact for |v| < 2^57: the 16-bit low parts and the 32-bit high part are
// added as 32-bit integers and recombined.
__device__ __forceinline__ long long group_sum(unsigned mask, long long v) {
  const unsigned l0 = __reduce_add_sync(mask, (unsigned)(v & 0xFFFF));
  const unsigned l1 = __reduce_add_sync(mask, (unsigned)((v >> 16) & 0xFFFF));
  const int hi = __reduce_add_sync(mask, (int)(v >> 32));
  return ((long long)hi << 32) + ((long long)l1 << 16) + (long long)l0;
}

// CIC deposit of every live slot into the fixed-point sums. The slots of a
// warp sit mostly in a few cells (birth order), so the lanes of each cell
// first add their contributions (integer sums: the result does not depend on
// the grouping) and one lane per cell issues the atomics. The contributions
// are formed in the run's precision (FP32 runs: no FP64 conversions).
template <typename T>
__global__ void k_win_deposit(Win<T> w, Geo g, Phys ph, PushConst<T> pc, int np) {
  const int nxn = g.nxn;
  const int lane = threadIdx.x & 31;
  constexpr long long kBig = 1LL << 57;
  for (int base = blockIdx.x * blockDim.x + threadIdx.x - lane; base < np;
       base += gridDim.x * blockDim.x) {
    const int p = base + lane;
    const int ci = (p < np) ? w.s.ci[p] : -1;
    long long a[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // n at ci, ci + 1; J_c at ci, ci + 1
    if (ci >= 0) {
      if constexpr (sizeof(T) == 4) {
        const float wp = (w.s.id[p] & kIdCR) ? pc.wcr : pc.wth;
        const float f = w.s.f[p];
        const float c0 = wp * (1.0f - f), c1 = wp * f;
        const float v[3] = {w.s.v[p], w.s.v[w.cap + p], w.s.v[2 * w.cap + p]};
        a[0] = fix32(c0);
        a[1] = fix32(c1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          a[2 + 2 * c] = fix32(c0 * v[c]);
          a[3 + 2 * c] = fix32(c1 * v[c]);
        }
      } else {
        const double wp = (w.s.id[p] & kIdCR) ? ph.w_cr : ph.w_th;
        const double f = (double)w.s.f[p];
        const double c0 = wp * (1.0 - f), c1 = wp * f;
        const double v[3] = {(double)w.s.v[p], (double)w.s.v[w.cap + p],
                             (double)w.s.v[2 * w.cap + p]};
        a[0] = (long long)fix(c0);
        a[1] = (long long)fix(c1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          a[2 + 2 * c] = (long long)fix(c0 * v[c]);
          a[3 + 2 * c] = (long long)fix(c1 * v[c]);
        }
      }
    }
    bool big = false;
#pragma unroll
    for (int k = 0; k < 8; ++k) big |= (a[k] >= kBig || a[k] <= -kBig);
    const unsigned grp = __match_any_sync(0xffffffffu, ci);
    const bool lead = !__any_sync(0xffffffffu, big);
    if (lead) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = group_sum(grp, a[k]);
    }
    if (ci < 0 || (lead && lane != __ffs(grp) - 1)) continue;
    atomicAdd(&w.q[ci], (unsigned long long)a[0]);
    atomicAdd(&w.q[ci + 1], (unsigned long long)a[1]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicAdd(&w.q[(c + 1) * nxn + ci], (unsigned long long)a[2 + 2 * c]);
      atomicAdd(&w.q[(c + 1) * nxn + ci + 1], (unsigned long long)a[3 + 2 * c]);
    }
  }
}

// Moments at node i from the fixed-point sums: wall nodes x2, the density
// floor, u = J / n; nraw is the density before the floor.
template <typename T>
__device__ __forceinline__ void moment_values(int i, const unsigned long long* q, const Geo& g,
                                              const Phys& ph, T& n, T& nraw, T u[3]) {
  const int nxn = g.nxn;
  const double sc = (i == 0 || i == g.nx) ? 2.0 : 1.0;
  const double nr = (double)(long long)q[i] * kUnfix * sc;
  n = (T)nr;
  nraw = (T)nr;
  const T nf = (T)ph.n_floor;
  if (n < nf) n = nf;
#pragma unroll
  for (int c = 0; c < 3; ++c) u[c] = (T)((double)(long long)q[(c + 1) * nxn + i] * kUnfix * sc) / n;
}

// The moments at the start of the window; clears the sums.
template <typename T>
__global__ void k_win_moments(Win<T> w, Geo g, Phys ph) {
  const int nxn = g.nxn;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nxn) return;
  T n, nr, u[3];
  moment_values<T>(i, w.q, g, ph, n, nr, u);
#pragma unroll
  for (int k = 0; k < 4; ++k) w.q[k * nxn + i] = 0ull;
  w.nraw[i] = nr;
  w.n[i] = n;
#pragma unroll
  for (int c = 0; c < 3; ++c) w.u[c * nxn + i] = u[c];
}

// B = B0 + sum_m a_m (cos, sin)(2 pi m x / L + phi_m) at the centres
template <typename T>
__global__ void k_win_seed_B(T* B, Geo g, Phys ph, double dx, const double* amps,
                             const double* phases, int M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nx) return;
  const double x = ((double)i + 0.5) * dx;
  const double L = (double)g.nx * dx;
  double by = ph.b0y, bz = ph.b0z;
  for (int m = 0; m < M; ++m) {
    const double arg = 2.0 * 3.14159265358979323846 * (double)(m + 1) * x / L + phases[m];
    double s, c;
    sincos(arg, &s, &c);
    by += amps[m] * c;
    bz += amps[m] * s;
  }
  B[i] = (T)ph.b0x;
  B[g.nx + i] = (T)by;
  B[2 * g.nx + i] = (T)bz;
}

// loss = sum_{i >= i0} |B_perp - B0_perp|^2 dx (into *out), and its
// gradient with respect to B times `scale` (into lB) when lB is given. One
// CTA: the sum is taken in a fixed order, so the loss is reproducible.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_win_loss(const T* B, Geo g, Phys ph, int i0, double dx,
                                                     double* out, double* lB, double scale) {
  __shared__ double red[kBlock / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
    double dy = 0.0, dz = 0.0;
    if (i >= i0) {
      dy = (double)B[g.nx + i] - ph.b0y;
      dz = (double)B[2 * g.nx + i] - ph.b0z;
      s += (dy * dy + dz * dz) * dx;
    }
    if (lB) {
      lB[i] = 0.0;
      lB[g.nx + i] = scale * (2.0 * dy * dx);
      lB[2 * g.nx + i] = scale * (2.0 * dz * dx);
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0 && out) {
    double tot = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += red[k];
    *out = tot;
  }
}

// ---------------------------------------------------------------- adjoint
// Adjoint of Ohm's law at one node of the 1D grid with n, u frozen. In: the
// centre fields Bm, Bp of the node's two cells (clamped at the walls), 1/n
// at the node (in) and the pressure term pgx = -T_e (n(i+1) - n(i-1))/(2 dx)
// (neighbours mirrored at the walls; both fixed while n is), u at the node
// and the adjoint (lex, ley, lez) of E there. Out: the
// adjoints of Bbar_y, Bbar_z, dB_y/dx, dB_z/dx at the node (P), that of n at
// the node (ln), the weight lp of n at the right neighbour (its negative at
// the left one: the pressure term's two-point difference) and the adjoint
// of u (lu).
//   E = ((curl B - jcr x) x Bbar - T_e grad n)/n - u x Bbar + eta curl B,
//   curl B = (0, -dB_z/dx, dB_y/dx)
struct OhmAdj {
  double P[4], ln, lp, lu[3];
};
__device__ __forceinline__ OhmAdj ohm_adj_point(const double Bm[3], const double Bp[3],
                                                double in, double pgx, const double u[3],
                                                double lex, double ley, double lez,
                                                const Phys& ph) {
  const double idx = ph.idx, te = ph.te, jcr = ph.jcr, eta = ph.eta;
  const double bbx = 0.5 * (Bm[0] + Bp[0]);
  const double bby = 0.5 * (Bm[1] + Bp[1]);
  const double bbz = 0.5 * (Bm[2] + Bp[2]);
  const double dby = (Bp[1] - Bm[1]) * idx;
  const double dbz = (Bp[2] - Bm[2]) * idx;
  const double ux = u[0], uy = u[1], uz = u[2];
  OhmAdj r;
  r.P[0] = lex * (-dby * in + uz) + lez * (-jcr * in - ux);
  r.P[1] = lex * (-dbz * in - uy) + ley * (jcr * in + ux);
  r.P[2] = lex * (-bby * in) + ley * (bbx * in) + lez * eta;
  r.P[3] = lex * (-bbz * in) + lez * (bbx * in) - ley * eta;
  const double cax = -dbz * bbz - dby * bby;
  const double cay = dby * bbx + jcr * bbz;
  const double caz = -jcr * bby + dbz * bbx;
  r.ln = -(lex * (pgx + cax) + ley * cay + lez * caz) * in * in;
  r.lp = -lex * in * te * ph.hdx;
  r.lu[0] = ley * bbz - lez * bby;
  r.lu[1] = -lex * bbz + lez * bbx;
  r.lu[2] = lex * bby - ley * bbx;
  return r;
}

// Centre part: the adjoint (ly, lz) of B_y, B_z at cell c from the node
// partials of its two nodes c (Pc) and c + 1 (Pc1) (Bbar = (Bm + Bp)/2,
// dB = (Bp - Bm)/dx); the wall nodes 0 and nx read cell 0 or nx - 1 twice.
__device__ __forceinline__ void curl_adj_point(const double Pc[4], const double Pc1[4],
                                               bool left_wall, bool right_wall, double idx,
                                               double& ly, double& lz) {
  ly = 0.0;
  lz = 0.0;
  ly += 0.5 * Pc[0] + Pc[2] * idx;  // node c sees cell c as its p side
  lz += 0.5 * Pc[1] + Pc[3] * idx;
  ly += 0.5 * Pc1[0] - Pc1[2] * idx;  // node c + 1 sees it as its m side
  lz += 0.5 * Pc1[1] - Pc1[3] * idx;
  if (left_wall) {  // node 0: m side clamped to cell 0
    ly += 0.5 * Pc[0] - Pc[2] * idx;
    lz += 0.5 * Pc[1] - Pc[3] * idx;
  }
  if (right_wall) {  // node nx: p side clamped to cell nx - 1
    ly += 0.5 * Pc1[0] + Pc1[2] * idx;
    lz += 0.5 * Pc1[1] + Pc1[3] * idx;
  }
}

// Adjoint of the moments at node i: from the adjoints ln, lu of n (floored)
// and u = J / n to those of the raw sums (wall nodes x2, no gradient through
// a floored density).
template <typename T>
__device__ __forceinline__ void moments_adj_node(int i, const T* nN, const T* uN,
                                                 const T* nraw, double ln, const double lu[3],
                                                 T* lNr, T* lJ, const Geo& g,
                                                 const Phys& ph) {
  const int nxn = g.nxn;
  const double sc = (i == 0 || i == g.nx) ? 2.0 : 1.0;
  const double n = (double)nN[i];
  for (int c = 0; c < 3; ++c) {
    lJ[c * nxn + i] = (T)(lu[c] / n * sc);
    ln -= lu[c] * (double)uN[c * nxn + i] / n;
  }
  lNr[i] = (T)(((double)nraw[i] < ph.n_floor) ? 0.0 : ln * sc);
}

// ------------------------------------------------ blocked field kernels
// A step's field work is tens of dependent phases over a small 1D grid. Each
// CTA owns kTbCells cells (and their left nodes; the last CTA also node nx)
// and runs all phases of the step in shared memory over its cells plus a
// halo, recomputing the halo: the stencils reach one cell per phase, so
// wrong values enter from a tile's inner edges (read there with clamped
// indices) at one cell per phase and never reach the owned cells while the
// halo is at least the number of phases. At the domain walls the tile edge is
// the wall and the clamped and mirrored indices are the walls' own. No
// synchronisation between CTAs, and the FP64 work spreads over the SMs.
constexpr int kTbCells = 16;
constexpr int kTbThreads = 64;

// halos: the forward's 4 n_sub stages and final Ohm; the adjoint's stage
// recompute, its 4 n_sub reverse stages and the moment adjoints
__host__ __device__ inline int halo_fields(int n_sub) { return 4 * n_sub + 2; }
__host__ __device__ inline int halo_rk4_adj(int n_sub) { return 8 * n_sub + 3; }

struct Tile {
  int c0, c1;  // owned cells [c0, c1)
  int lo, L;   // local cells lo .. lo + L - 1, local nodes lo .. lo + L
  int nx;
  __device__ __forceinline__ Tile(int b, int nx_, int halo) : nx(nx_) {
    c0 = b * kTbCells;
    c1 = min(nx, c0 + kTbCells);
    lo = max(0, c0 - halo);
    L = min(nx, c1 + halo) - lo;
  }
  // global cell (clamped at the walls) -> local cell (clamped to the tile)
  __device__ __forceinline__ int cell(int c) const {
    c = min(max(c, 0), nx - 1);
    return min(max(c - lo, 0), L - 1);
  }
  // global node (mirrored at the walls) -> local node (clamped to the tile)
  __device__ __forceinline__ int node(int i) const {
    i = (i < 0) ? -i : ((i > nx) ? 2 * nx - i : i);
    return min(max(i - lo, 0), L);
  }
  __device__ __forceinline__ bool owns_cell(int c) const { return c >= c0 && c < c1; }
  __device__ __forceinline__ bool owns_node(int i) const {
    return (i >= c0 && i < c1) || (i == nx && c1 == nx);
  }
};

// Ohm's law at global node gi of a tile, from the tile's centre field B
// [3][L], density n [L + 1] and velocity u [3][L + 1] (the 1D form of
// ohm_node).
template <typename T>
__device__ __forceinline__ void tile_ohm(const Tile& t, int gi, const T* B, const T* n,
                                         const T* u, const Phys& ph, const FieldConst<T>& fc,
                                         T E[3], T Bb[3]) {
  const int L = t.L, Ln = L + 1, i = gi - t.lo;
  const int im = t.cell(gi - 1), ip = t.cell(gi);
  const T idx = fc.idx;
  const T bmy = B[L + im], bpy = B[L + ip], bmz = B[2 * L + im], bpz = B[2 * L + ip];
  Bb[0] = (T)0.5 * (B[im] + B[ip]);
  Bb[1] = (T)0.5 * (bmy + bpy);
  Bb[2] = (T)0.5 * (bmz + bpz);
  const T dby = (bpy - bmy) * idx;
  const T dbz = (bpz - bmz) * idx;
  const T te = fc.te;
  const T dnx = (n[t.node(gi + 1)] - n[t.node(gi - 1)]) * fc.hdx;
  const T inv_n = (T)1 / n[i];
  ohm_e<T>((T)0, -dbz, dby, Bb[0], Bb[1], Bb[2], inv_n, -(te * dnx), -(te * (T)0), u[i],
           u[Ln + i], u[2 * Ln + i], fc.jcr, fc.eta, fc.resist != 0, E[0], E[1], E[2]);
}

// Faraday + RK4 stage update at local cell c of a tile (1D: K = (0, dEz/dx,
// -dEy/dx) from the nodes c, c + 1).
template <typename T>
__device__ __forceinline__ void tile_faraday(const Tile& t, int c, const T* E, T* B, T* Bs,
                                             T* K, int stage, const FieldConst<T>& fc) {
  const int L = t.L, Ln = L + 1;
  const T idx = fc.idx;
  const T dxey = (E[Ln + c + 1] - E[Ln + c]) * idx;
  const T dxez = (E[2 * Ln + c + 1] - E[2 * Ln + c]) * idx;
  const T Kc[3] = {(T)0, dxez, -dxey};
#pragma unroll
  for (int q = 0; q < 3; ++q)
    rk4_stage<T>(stage, Kc[q], K[q * L + c], Bs[q * L + c], B[q * L + c], fc.h, fc.hh, fc.h6);
}

constexpr size_t kMaxSmem = 227 * 1024;  // shared memory a CTA may opt in to

inline size_t fields_smem(int n_sub, size_t tsz) {
  const size_t L = kTbCells + 2 * halo_fields(n_sub);
  return tsz * (9 * L + 7 * (L + 1));
}
inline size_t rk4_adj_smem(int n_sub, size_t tsz) {
  const size_t L = kTbCells + 2 * halo_rk4_adj(n_sub), Ln = L + 1;
  return tsz * (9 * L + 7 * Ln) + 8 * ((12 * (size_t)n_sub + 12) * L + 12 * Ln);
}

// One step's moments (and their tape) from the deposit sums, B's tape, the
// n_sub RK4 substeps of Ohm + Faraday with n, u frozen, then E, Bbar for the
// next gather and the new B (into Bout; B is read by neighbouring tiles).
template <typename T>
__global__ void __launch_bounds__(kTbThreads)
    k_win_fields(Win<T> w, Geo g, Phys ph, FieldConst<T> fc, int n_sub, T* Bout, T* tn, T* tu,
                 T* tr, T* tapeB) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nx = g.nx, nxn = g.nxn, t0 = threadIdx.x, nt = blockDim.x;
  const Tile t(blockIdx.x, nx, halo_fields(n_sub));
  const int L = t.L, Ln = L + 1;
  T* sB = (T*)smem;
  T* sBs = sB + 3 * L;
  T* sK = sBs + 3 * L;
  T* sE = sK + 3 * L;
  T* sn = sE + 3 * Ln;
  T* su = sn + Ln;
  for (int k = t0; k < 3 * L; k += nt) {
    const int q = k / L, gc = t.lo + k - q * L;
    const T v = w.B[q * nx + gc];
    sB[k] = v;
    if (tapeB && t.owns_cell(gc)) tapeB[q * nx + gc] = v;
  }
  for (int i = t0; i < Ln; i += nt) {
    const int gi = t.lo + i;
    T n, nr, u[3];
    moment_values<T>(gi, w.q, g, ph, n, nr, u);
    sn[i] = n;
#pragma unroll
    for (int c = 0; c < 3; ++c) su[c * Ln + i] = u[c];
    if (t.owns_node(gi)) {
      w.n[gi] = n;
      w.nraw[gi] = nr;
#pragma unroll
      for (int c = 0; c < 3; ++c) w.u[c * nxn + gi] = u[c];
      if (tn) {
        tn[gi] = n;
        tr[gi] = nr;
#pragma unroll
        for (int c = 0; c < 3; ++c) tu[c * nxn + gi] = u[c];
      }
    }
  }
  __syncthreads();
  for (int sub = 0; sub < n_sub; ++sub) {
    for (int stage = 1; stage <= 4; ++stage) {
      const T* Bin = (stage == 1) ? sB : sBs;
      for (int i = t0; i < Ln; i += nt) {
        T E[3], Bb[3];
        tile_ohm<T>(t, t.lo + i, Bin, sn, su, ph, fc, E, Bb);
#pragma unroll
        for (int c = 0; c < 3; ++c) sE[c * Ln + i] = E[c];
      }
      __syncthreads();
      for (int c = t0; c < L; c += nt) tile_faraday<T>(t, c, sE, sB, sBs, sK, stage, fc);
      __syncthreads();
    }
  }
  for (int i = t0; i < Ln; i += nt) {
    const int gi = t.lo + i;
    if (!t.owns_node(gi)) continue;
    T E[3], Bb[3];
    tile_ohm<T>(t, gi, sB, sn, su, ph, fc, E, Bb);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      w.E[c * nxn + gi] = E[c];
      w.Bb[c * nxn + gi] = Bb[c];
    }
  }
  for (int k = t0; k < 3 * L; k += nt) {
    const int q = k / L, gc = t.lo + k - q * L;
    if (t.owns_cell(gc)) Bout[q * nx + gc] = sB[k];
  }
}

// Reverse of one step's field update and moments. In: B^n (Bn, tape),
// M^{n+1} (n1, u1, nr1), M^n (n0, u0), lBin = adjoint of B^{n+1}, lNm, lUm
// = what E^{n+1}'s Ohm added to the adjoint of M^{n+1}. Per tile:
//   1. the RK4 stage inputs from B^n with n, u frozen at M^{n+1}, recomputed
//      with the forward's arithmetic (Y);
//   2. the stages in reverse: per stage the node part of Ohm's adjoint
//      (partials P, the n and u adjoints), then the centre part (the running
//      sum, the next stage's adjoint gk), to the adjoint of B^n (lBout);
//   3. the adjoints of the raw deposit sums (lNr, lJ) from those of M^{n+1};
//   4. E^n, Bbar^n from B^n and M^n for the particle adjoint; lE = lBb = 0;
//      lNm = lUm = 0 for the next Ohm adjoint.
template <typename T>
__global__ void __launch_bounds__(kTbThreads)
    k_win_rk4_adj(Win<T> w, Geo g, Phys ph, FieldConst<T> fc, int ns, const T* Bn, const T* n1,
                  const T* u1, const T* nr1, const T* n0, const T* u0, const double* lBin,
                  double* lBout) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nx = g.nx, nxn = g.nxn, t0 = threadIdx.x, nt = blockDim.x;
  const Tile t(blockIdx.x, nx, halo_rk4_adj(ns));
  const int L = t.L, Ln = L + 1;
  double* Y = (double*)smem;        // [4 ns][3][L]
  double* lB = Y + 12 * ns * L;     // [3][L]
  double* lend = lB + 3 * L;        // [3][L]
  double* lsum = lend + 3 * L;      // [3][L]
  double* gk = lsum + 3 * L;        // [3][L]
  double* P = gk + 3 * L;           // [4][Ln]
  double* lN = P + 4 * Ln;          // [Ln]
  double* lU = lN + Ln;             // [3][Ln]
  double* lnS = lU + 3 * Ln;        // [Ln]
  double* lpS = lnS + Ln;           // [Ln]
  double* sIn = lpS + Ln;           // [Ln] 1/n at M^{n+1}
  double* sPg = sIn + Ln;           // [Ln] its pressure term
  T* sB = (T*)(sPg + Ln);           // [3][L]
  T* sBs = sB + 3 * L;
  T* sK = sBs + 3 * L;
  T* sE = sK + 3 * L;               // [3][Ln]
  T* sn = sE + 3 * Ln;              // [Ln]
  T* su = sn + Ln;                  // [3][Ln]
  const double h = ph.h, hh = ph.hh, h6 = ph.h6, idx = ph.idx;
  for (int k = t0; k < 3 * L; k += nt) {
    const int q = k / L, gc = t.lo + k - q * L;
    sB[k] = Bn[q * nx + gc];
    lB[k] = lBin[q * nx + gc];
  }
  for (int i = t0; i < Ln; i += nt) {
    const int gi = t.lo + i;
    const bool own = t.owns_node(gi);
    sn[i] = n1[gi];
    lN[i] = own ? w.lNm[gi] : 0.0;
    if (own) w.lNm[gi] = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      su[c * Ln + i] = u1[c * nxn + gi];
      lU[c * Ln + i] = own ? w.lUm[c * nxn + gi] : 0.0;
      if (own) w.lUm[c * nxn + gi] = 0.0;
    }
  }
  __syncthreads();
  // n is frozen at M^{n+1}: 1/n and the pressure term once per node (first
  // read in 2., many barriers later)
  for (int i = t0; i < Ln; i += nt) {
    const int gi = t.lo + i;
    sIn[i] = 1.0 / (double)sn[i];
    sPg[i] = -(ph.te * (((double)sn[t.node(gi + 1)] - (double)sn[t.node(gi - 1)]) * ph.hdx));
  }
  // 1.
  for (int sub = 0; sub < ns; ++sub) {
    for (int stage = 1; stage <= 4; ++stage) {
      const T* Bin = (stage == 1) ? sB : sBs;
      double* y = Y + (size_t)(4 * sub + stage - 1) * 3 * L;
      for (int k = t0; k < 3 * L; k += nt) y[k] = (double)Bin[k];
      for (int i = t0; i < Ln; i += nt) {
        T E[3], Bb[3];
        tile_ohm<T>(t, t.lo + i, Bin, sn, su, ph, fc, E, Bb);
#pragma unroll
        for (int c = 0; c < 3; ++c) sE[c * Ln + i] = E[c];
      }
      __syncthreads();
      for (int c = t0; c < L; c += nt) tile_faraday<T>(t, c, sE, sB, sBs, sK, stage, fc);
      __syncthreads();
    }
  }
  // 2. lambda_start = lambda_end + sum over the stages of lambda_Y; the stage
  //    adjoints g4 = h6 lend, g3 = 2 h6 lend + h lY4, g2 = 2 h6 lend + hh lY3,
  //    g1 = h6 lend + hh lY2
  const double an[3] = {2 * h6, 2 * h6, h6};
  const double bn[3] = {h, hh, hh};
  for (int sub = ns - 1; sub >= 0; --sub) {
    for (int k = t0; k < 3 * L; k += nt) {
      const double l = lB[k];
      lend[k] = l;
      lsum[k] = l;
      gk[k] = h6 * l;
    }
    __syncthreads();
    for (int s = 3; s >= 0; --s) {
      const double* y = Y + (size_t)(4 * sub + s) * 3 * L;
      for (int i = t0; i < Ln; i += nt) {
        const int gi = t.lo + i;
        const int cm = t.cell(gi - 1), cp = t.cell(gi);
        // E adjoint at the node from K's: K_y(c) = (E_z(c+1) - E_z(c))/dx,
        // K_z(c) = -(E_y(c+1) - E_y(c))/dx
        const double gym = (gi >= 1) ? gk[L + cm] : 0.0, gy = (gi < nx) ? gk[L + cp] : 0.0;
        const double gzm = (gi >= 1) ? gk[2 * L + cm] : 0.0, gz = (gi < nx) ? gk[2 * L + cp] : 0.0;
        const double Bm[3] = {y[cm], y[L + cm], y[2 * L + cm]};
        const double Bp[3] = {y[cp], y[L + cp], y[2 * L + cp]};
        const double u[3] = {(double)su[i], (double)su[Ln + i], (double)su[2 * Ln + i]};
        const OhmAdj r = ohm_adj_point(Bm, Bp, sIn[i], sPg[i], u, 0.0, (gz - gzm) * idx,
                                       (gym - gy) * idx, ph);
#pragma unroll
        for (int q = 0; q < 4; ++q) P[q * Ln + i] = r.P[q];
        lnS[i] = r.ln;
        lpS[i] = r.lp;
#pragma unroll
        for (int c = 0; c < 3; ++c) lU[c * Ln + i] += r.lu[c];
      }
      __syncthreads();
      const int q = 3 - s;
      for (int c = t0; c < L; c += nt) {
        const int gc = t.lo + c;
        const double Pc[4] = {P[c], P[Ln + c], P[2 * Ln + c], P[3 * Ln + c]};
        const double Pc1[4] = {P[c + 1], P[Ln + c + 1], P[2 * Ln + c + 1], P[3 * Ln + c + 1]};
        double ly, lz;
        curl_adj_point(Pc, Pc1, gc == 0, gc == nx - 1, idx, ly, lz);
        lsum[L + c] += ly;
        lsum[2 * L + c] += lz;
        if (s > 0) {
          gk[c] = 0.0;
          gk[L + c] = an[q] * lend[L + c] + bn[q] * ly;
          gk[2 * L + c] = an[q] * lend[2 * L + c] + bn[q] * lz;
        }
      }
      // n adjoint: the node's own term and its neighbours' pressure weights
      // (node j - 1 adds lp at j, node j + 1 adds -lp at j; the mirrored
      // wall nodes 0 and nx add their other term at 1 and nx - 1)
      for (int j = t0; j < Ln; j += nt) {
        const int gj = t.lo + j;
        double a = lnS[j];
        if (gj >= 1) a += lpS[t.node(gj - 1)];
        if (gj + 1 <= nx) a -= lpS[t.node(gj + 1)];
        if (gj == nx - 1) a += lpS[t.node(nx)];
        if (gj == 1) a -= lpS[t.node(0)];
        lN[j] += a;
      }
      __syncthreads();
    }
    for (int k = t0; k < 3 * L; k += nt) lB[k] = lsum[k];
    __syncthreads();
  }
  // 3., 4.
  for (int i = t0; i < Ln; i += nt) {
    const int gi = t.lo + i;
    if (!t.owns_node(gi)) continue;
    const double lu[3] = {lU[i], lU[Ln + i], lU[2 * Ln + i]};
    moments_adj_node<T>(gi, n1, u1, nr1, lN[i], lu, w.lNr, w.lJ, g, ph);
    ohm_node<T, 1>(gi, Bn, n0, u0, nullptr, w.E, w.Bb, nullptr, g, ph);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      w.lE[c * nxn + gi] = 0.0;
      w.lBb[c * nxn + gi] = 0.0;
    }
  }
  for (int k = t0; k < 3 * L; k += nt) {
    const int q = k / L, gc = t.lo + k - q * L;
    if (t.owns_cell(gc)) lBout[q * nx + gc] = lB[k];
  }
}

// The adjoint of Ohm's law at the start of step n (B^n in Bn, M^n in n0,
// u0), after the particle adjoint (lE, lBb): lB += its share at the owned
// cells; the owned nodes add their n, u adjoints to lNm (atomics: the
// pressure term reaches the neighbours) and lUm.
template <typename T>
__global__ void __launch_bounds__(kTbThreads)
    k_win_ohm_adj_step(Win<T> w, Geo g, Phys ph, const T* Bn, const T* n0, const T* u0) {
  __shared__ double P[4][kTbCells + 1];
  const int nx = g.nx, nxn = g.nxn, t0 = threadIdx.x, nt = blockDim.x;
  const int c0 = blockIdx.x * kTbCells, c1 = min(nx, c0 + kTbCells);
  for (int k = t0; k <= c1 - c0; k += nt) {  // nodes c0 .. c1
    const int gi = c0 + k;
    const int im = min(max(gi - 1, 0), nx - 1), ip = min(gi, nx - 1);
    const double Bm[3] = {(double)Bn[im], (double)Bn[nx + im], (double)Bn[2 * nx + im]};
    const double Bp[3] = {(double)Bn[ip], (double)Bn[nx + ip], (double)Bn[2 * nx + ip]};
    const int ipn = (gi + 1 > nx) ? 2 * nx - (gi + 1) : gi + 1;
    const int imn = (gi - 1 < 0) ? -(gi - 1) : gi - 1;
    const double u[3] = {(double)u0[gi], (double)u0[nxn + gi], (double)u0[2 * nxn + gi]};
    const double pg = -(ph.te * (((double)n0[ipn] - (double)n0[imn]) * ph.hdx));
    const OhmAdj r = ohm_adj_point(Bm, Bp, 1.0 / (double)n0[gi], pg, u, w.lE[gi],
                                   w.lE[nxn + gi], w.lE[2 * nxn + gi], ph);
    P[0][k] = r.P[0] + w.lBb[nxn + gi];
    P[1][k] = r.P[1] + w.lBb[2 * nxn + gi];
    P[2][k] = r.P[2];
    P[3][k] = r.P[3];
    if (gi < c1 || gi == nx) {  // owned node
      atomicAdd(&w.lNm[gi], r.ln);
      if (r.lp != 0.0) {
        atomicAdd(&w.lNm[ipn], r.lp);
        atomicAdd(&w.lNm[imn], -r.lp);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) w.lUm[c * nxn + gi] += r.lu[c];
    }
  }
  __syncthreads();
  for (int k = t0; k < c1 - c0; k += nt) {
    const int gc = c0 + k;
    const double Pc[4] = {P[0][k], P[1][k], P[2][k], P[3][k]};
    const double Pc1[4] = {P[0][k + 1], P[1][k + 1], P[2][k + 1], P[3][k + 1]};
    double ly, lz;
    curl_adj_point(Pc, Pc1, gc == 0, gc == nx - 1, ph.idx, ly, lz);
    w.lB[nx + gc] += ly;
    w.lB[2 * nx + gc] += lz;
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Adjoint of one step for slot p < np1 (alive at the end of the step or born
// in it). In: lf, lv = adjoints of the state after the step;
// lNr, lJ = adjoints of the step's deposit; E, Bb = the node fields the
// step's gather used. Out: lf, lv = adjoints of the state before the step
// (zero for slots born or removed in it); the slot's shares of lE, lBb at
// the nodes c0, c0 + 1 (out; returns c0, or -1 when it has none); its terms
// of grad[M] (u_cr, into gucr) and grad[M + 1] (u2, into gu2). The
// deposit's adjoint, the injection's and the faux-shock
// return's are taken in FP64; the push's (Boris, gather) in the run's
// precision, that of the per-slot adjoints lf, lv; the sums into lE, lBb and
// the gradient are FP64.
template <typename T>
__device__ __forceinline__ int particle_adj_slot(int p, const Win<T>& w, const Slots<T>& t0,
                                                 const Slots<T>& t1, const uint8_t* ev,
                                                 const Geo& g, const Phys& ph,
                                                 const PushConst<T>& pc, long long step,
                                                 int np0, double& gu2, double& gucr, T out[12]) {
  using A = T;  // arithmetic of the push's adjoint
  const int nxn = g.nxn;
  const int cap = w.cap;
  {
    const bool born = p >= np0;
    const uint8_t e = born ? (uint8_t)kEvNone : ev[p];
    const int c1 = t1.ci[p];
    if (c1 < 0 || (!born && t0.ci[p] < 0) || e == kEvRemoved) {
      w.lf[p] = (T)0;
      w.lv[p] = w.lv[cap + p] = w.lv[2 * cap + p] = (T)0;
      return -1;
    }
    // ---- deposit at the state after the step (in the run's precision)
    const uint32_t id = w.s.id[p];
    A wp;
    if constexpr (sizeof(T) == 4) wp = (id & kIdCR) ? pc.wcr : pc.wth;
    else wp = (id & kIdCR) ? ph.w_cr : ph.w_th;
    const A f1 = t1.f[p];
    const A v1[3] = {t1.v[p], t1.v[cap + p], t1.v[2 * cap + p]};
    A lf1 = w.lf[p];
    A lv[3] = {w.lv[p], w.lv[cap + p], w.lv[2 * cap + p]};
    {
      A dj = w.lNr[c1 + 1] - w.lNr[c1];
      for (int c = 0; c < 3; ++c) {
        const A ja = w.lJ[c * nxn + c1], jb = w.lJ[c * nxn + c1 + 1];
        dj += (jb - ja) * v1[c];
        lv[c] += wp * (((A)1 - f1) * ja + f1 * jb);
      }
      lf1 += wp * dj;
    }
    if (born) {
      if (id & kIdCR) {  // v = p (mu, sn c, sn s) - u_cr x, mu = a + (1 - a) s1, a = u_cr / p
        double v[3], U[4];
        const double X = cr_draw(ph, id & kIdMask, step, v, U);
        const double pv = ph.p_iso_v, s1 = U[0], mu = (v[0] + ph.u_cr) / pv;
        const double sn = sqrt(fmax(1.0 - mu * mu, 0.0));
        const double dmu = (1.0 - s1) / pv;
        const double dsn = (sn > 0.0) ? -mu * dmu / sn : 0.0;
        const double dvx = pv * dmu - 1.0, dvy = pv * dsn * U[1], dvz = pv * dsn * U[2];
        gucr += (double)lv[0] * dvx + (double)lv[1] * dvy + (double)lv[2] * dvz;
        const double ix = floor(X);
        if (ix >= 0.0 && ix < (double)g.nx)  // placement not clamped
          gucr += (double)lf1 * U[3] * dvx * ph.dtdx;
      }
      w.lf[p] = (T)0;
      w.lv[p] = w.lv[cap + p] = w.lv[2 * cap + p] = (T)0;
      return -1;
    }
    // ---- recompute the push from the state before the step
    const int c0 = t0.ci[p];
    const A f0 = (A)t0.f[p];
    const T ft0 = t0.f[p];
    const T g0t = (T)1 - ft0;
    T Ep[3], Bp[3];
    A Ed[3], Bd[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Ep[c] = fmaT(ft0, w.E[c * nxn + c0 + 1], g0t * w.E[c * nxn + c0]);
      Bp[c] = fmaT(ft0, w.Bb[c * nxn + c0 + 1], g0t * w.Bb[c * nxn + c0]);
      Ed[c] = (A)w.E[c * nxn + c0 + 1] - (A)w.E[c * nxn + c0];
      Bd[c] = (A)w.Bb[c * nxn + c0 + 1] - (A)w.Bb[c * nxn + c0];
    }
    const A v0[3] = {(A)t0.v[p], (A)t0.v[cap + p], (A)t0.v[2 * cap + p]};
    T vxt = t0.v[p], vyt = t0.v[cap + p], vzt = t0.v[2 * cap + p];
    boris<T>(vxt, vyt, vzt, Ep, Bp, pc.hdt);
    const A vp[3] = {(A)vxt, (A)vyt, (A)vzt};  // before the return
    A lvp[3];  // adjoint of vp
    A lf0;
    if (e == kEvReturned) {
      // vnew = R(vp; u2), f1 = clamp(gf * vnew_x * dtdx), gf = Xn/(Xn - Xo)
      const Philox4 r = draw4(ph.seed, id & kIdMask, step, kPurposeFS);
      const double s1 = sqrt(u01(r.x[1]));
      double cs, sn2;
      fs_sincos2pi(u01(r.x[2]), &cs, &sn2);
      const double u2 = ph.u2;
      const double wx = (double)vp[0] + u2;
      const double wv = sqrt(wx * wx + (double)vp[1] * vp[1] + (double)vp[2] * vp[2]);
      const double a = u2 / wv;
      const double mu = a + (1.0 - a) * s1;
      const double snm = sqrt(fmax(1.0 - mu * mu, 0.0));
      const double vnx = wv * mu - u2;
      const double av = (double)vp[0] * ph.dtdx;  // Xn - Xo
      const double Xo = (double)c0 + (double)f0;
      const double gf = (Xo + av) / av;
      const double fraw = gf * vnx * ph.dtdx;
      double Lx = lv[0], Ly = lv[1], Lz = lv[2];
      const double lf1d = lf1;
      double lXo = 0.0, lav = 0.0;
      if (fraw >= 0.0 && fraw < 1.0) {
        Lx += lf1d * gf * ph.dtdx;
        const double lgf = lf1d * vnx * ph.dtdx;
        lXo = lgf / av;
        lav = -lgf * Xo / (av * av);
      }
      // through the return map R
      const double Lsn = (Ly * cs + Lz * sn2) * wv;
      double Lw = Lx * mu + (Ly * cs + Lz * sn2) * snm;
      const double Lmu = Lx * wv - ((snm > 0.0) ? Lsn * mu / snm : 0.0);
      const double La = Lmu * (1.0 - s1);
      Lw -= La * u2 / (wv * wv);
      double Lu2 = -Lx + La / wv;
      Lu2 += Lw * wx / wv;
      gu2 += Lu2;
      lvp[0] = (A)(Lw * wx / wv + lav * ph.dtdx);
      lvp[1] = (A)(Lw * vp[1] / wv);
      lvp[2] = (A)(Lw * vp[2] / wv);
      lf0 = (A)lXo;
    } else {
      lvp[0] = lv[0] + lf1 * pc.dtdx;
      lvp[1] = lv[1];
      lvp[2] = lv[2];
      lf0 = lf1;
    }
    // ---- Boris adjoint: v+ = q + em, q = vm + p x s, p = vm + vm x t,
    //      s = (2 / (1 + t.t)) t, t = hdt B, vm = v + em, em = hdt E
    const A hdt = pc.hdt;
    A em[3], vm[3], t[3], sv[3], pp[3];
    for (int c = 0; c < 3; ++c) {
      em[c] = hdt * (A)Ep[c];
      vm[c] = v0[c] + em[c];
      t[c] = hdt * (A)Bp[c];
    }
    const A tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const A fct = (A)2 / ((A)1 + tt);
    for (int c = 0; c < 3; ++c) sv[c] = fct * t[c];
    pp[0] = vm[0] + (vm[1] * t[2] - vm[2] * t[1]);
    pp[1] = vm[1] + (vm[2] * t[0] - vm[0] * t[2]);
    pp[2] = vm[2] + (vm[0] * t[1] - vm[1] * t[0]);
    const A* Lq = lvp;
    A Lem[3] = {lvp[0], lvp[1], lvp[2]};
    A Lvm[3] = {Lq[0], Lq[1], Lq[2]};
    // q = vm + p x s: L_p = s x L_q, L_s = L_q x p
    const A Lp[3] = {sv[1] * Lq[2] - sv[2] * Lq[1], sv[2] * Lq[0] - sv[0] * Lq[2],
                          sv[0] * Lq[1] - sv[1] * Lq[0]};
    const A Ls[3] = {Lq[1] * pp[2] - Lq[2] * pp[1], Lq[2] * pp[0] - Lq[0] * pp[2],
                          Lq[0] * pp[1] - Lq[1] * pp[0]};
    // p = vm + vm x t: L_vm += L_p + t x L_p, L_t = L_p x vm
    Lvm[0] += Lp[0] + (t[1] * Lp[2] - t[2] * Lp[1]);
    Lvm[1] += Lp[1] + (t[2] * Lp[0] - t[0] * Lp[2]);
    Lvm[2] += Lp[2] + (t[0] * Lp[1] - t[1] * Lp[0]);
    A Lt[3] = {Lp[1] * vm[2] - Lp[2] * vm[1], Lp[2] * vm[0] - Lp[0] * vm[2],
                    Lp[0] * vm[1] - Lp[1] * vm[0]};
    // s = fct t, fct = 2 / (1 + tt)
    const A Lf = Ls[0] * t[0] + Ls[1] * t[1] + Ls[2] * t[2];
    const A Ltt = -Lf * fct * fct * (A)0.5;
    for (int c = 0; c < 3; ++c) {
      Lt[c] += fct * Ls[c] + (A)2 * Ltt * t[c];
      Lem[c] += Lvm[c];
    }
    const A LE[3] = {hdt * Lem[0], hdt * Lem[1], hdt * Lem[2]};
    const A LB[3] = {hdt * Lt[0], hdt * Lt[1], hdt * Lt[2]};
    // ---- gather adjoint at the state before the step: the shares of the
    //      nodes c0, c0 + 1 in lE, lBb go to the caller
    for (int c = 0; c < 3; ++c) {
      out[4 * c] = ((A)1 - f0) * LE[c];
      out[4 * c + 1] = f0 * LE[c];
      out[4 * c + 2] = ((A)1 - f0) * LB[c];
      out[4 * c + 3] = f0 * LB[c];
      lf0 += LE[c] * Ed[c] + LB[c] * Bd[c];
    }
    w.lf[p] = (T)lf0;
    w.lv[p] = (T)Lvm[0];
    w.lv[cap + p] = (T)Lvm[1];
    w.lv[2 * cap + p] = (T)Lvm[2];
    return c0;
  }
}

// An FP32 value as an FP64 one (exact) by integer operations on its bit
// pattern (the conversion instruction runs on GB300's narrow FP64 pipe):
// sign kept, exponent rebiased, significand shifted into place; zero and
// subnormals (below 2^-126) give zero, infinities and NaN stay so.
__device__ __forceinline__ double widen(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned long long s = (unsigned long long)(b >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)s);
  const unsigned long long ed = (e == 0xFFu) ? 0x7FFull : (unsigned long long)(e + 896u);
  const unsigned long long m = (unsigned long long)(b & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(s | (ed << 52) | m));
}
__device__ __forceinline__ double widen(double x) { return x; }

// Adds one slot's shares (out of particle_adj_slot) to lE, lBb at c0, c0 + 1.
template <typename T>
__device__ __forceinline__ void add_node_shares(const Win<T>& w, int nxn, int c0, const T a[12]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    atomicAdd(&w.lE[c * nxn + c0], widen(a[4 * c]));
    atomicAdd(&w.lE[c * nxn + c0 + 1], widen(a[4 * c + 1]));
    atomicAdd(&w.lBb[c * nxn + c0], widen(a[4 * c + 2]));
    atomicAdd(&w.lBb[c * nxn + c0 + 1], widen(a[4 * c + 3]));
  }
}
// Adjoint of one step for every slot p < np1 (slots alive at the end of the
// step or born in it): particle_adj_slot per slot. In the FP32 run the lanes
// of a warp whose slots sit in at most 4 cells first add the shares of each
// cell (slots in birth order share cells), so that one lane per cell issues
// its atomics; otherwise every lane issues its own.
template <typename T>
__global__ void __launch_bounds__(kBlock, 4)
    k_win_particle_adj(Win<T> w, Slots<T> t0, Slots<T> t1, const uint8_t* ev, Geo g, Phys ph,
                       PushConst<T> pc, long long step, int np0, int np1, int M) {
  const int nxn = g.nxn;
  const int lane = threadIdx.x & 31;
  double gu2 = 0.0, gucr = 0.0;
  for (int base = blockIdx.x * blockDim.x + threadIdx.x - lane; base < np1;
       base += gridDim.x * blockDim.x) {
    const int p = base + lane;
    T a[12];
    const int c0 =
        (p < np1) ? particle_adj_slot<T>(p, w, t0, t1, ev, g, ph, pc, step, np0, gu2, gucr, a)
                   : -1;
    if (sizeof(T) == 4) {
      const unsigned grp = __match_any_sync(0xffffffffu, c0);
      const bool lead = c0 >= 0 && lane == __ffs(grp) - 1;
      unsigned leads = __ballot_sync(0xffffffffu, lead);
      if (__popc(leads) <= 4) {
        while (leads) {
          const int l = __ffs(leads) - 1;
          leads &= leads - 1;
          const int key = __shfl_sync(0xffffffffu, c0, l);
          T s[12];
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            s[k] = (c0 == key) ? a[k] : (T)0;
            for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
          }
          if (lane == l) add_node_shares<T>(w, nxn, key, s);
        }
        continue;
      }
    }
    if (c0 >= 0) add_node_shares<T>(w, nxn, c0, a);
  }
  // only slots that were returned or injected add to these: most warps have
  // none (tested on the bit patterns, off the FP64 pipe)
  const bool any = __double_as_longlong(gu2) != 0 || __double_as_longlong(gucr) != 0;
  if (__any_sync(0xffffffffu, any)) {
    gu2 = warp_sum_d(gu2);
    gucr = warp_sum_d(gucr);
    if ((threadIdx.x & 31) == 0) {
      if (gucr != 0.0) atomicAdd(&w.grad[M], gucr);
      if (gu2 != 0.0) atomicAdd(&w.grad[M + 1], gu2);
    }
  }
}

// d loss / d a_m = sum_c lB_y(c) cos(arg) + lB_z(c) sin(arg), one CTA per mode
__global__ void k_win_mode_grad(const double* lB, double* grad, const double* phases, Geo g,
                                double dx) {
  const int m = blockIdx.x;
  const double L = (double)g.nx * dx;
  double s = 0.0;
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
    const double x = ((double)i + 0.5) * dx;
    const double arg = 2.0 * 3.14159265358979323846 * (double)(m + 1) * x / L + phases[m];
    double sn, cs;
    sincos(arg, &sn, &cs);
    s += lB[g.nx + i] * cs + lB[2 * g.nx + i] * sn;
  }
  __shared__ double red[32];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    r = warp_sum_d(r);
    if (threadIdx.x == 0) grad[m] = r;
  }
}

}  // namespace win
}  // namespace fsx

// =====================================================================
// Host side and C ABI
// =====================================================================
using namespace fsx;
using namespace fsx::win;

namespace {
constexpr size_t kAl = 256;
inline size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }
inline int blocks(long long n) { return (int)std::max<long long>(1, (n + kBlock - 1) / kBlock); }
inline int tiles(int nx) { return (nx + kTbCells - 1) / kTbCells; }
}  // namespace

struct fs_window {
  fs_params p;
  Geo g;
  Phys ph;
  int steps, ckpt, nseg, M, loss_i0;
  long long n_init;
  int cap;
  size_t tsz;  // sizeof(T)
  char* base;
  cudaStream_t st;
  // regions (byte offsets)
  size_t o_state, o_ckpt, o_tape, o_ev, o_tapeB, o_tapeM, o_fields, o_q, o_ctr, o_adj,
      o_params;
  // slot schedule: slots at the start of step n (n = 0..steps), new
  // particles of each kind in step n, first new id of step n
  std::vector<int> np_at;
  std::vector<int> ninj;
  std::vector<unsigned long long> first_id;
  bool have_forward = false;
  int bsel = 0;  // which of the two B buffers holds the current field
  long long counts[5] = {0, 0, 0, 0, 0};  // of the last forward
};

namespace {

// bytes of one copy of the per-slot state (ci, f, v[3], id)
size_t slot_bytes(int cap, size_t tsz) {
  return al(4 * (size_t)cap) + al(tsz * cap) + al(3 * tsz * cap) + al(4 * (size_t)cap);
}
size_t tape_slot_bytes(int cap, size_t tsz) {  // ci, f, v
  return al(4 * (size_t)cap) + al(tsz * cap) + al(3 * tsz * cap);
}
size_t mom_bytes(int nxn, size_t tsz) { return 5 * al(tsz * nxn); }  // n, u[3], nraw

// per step the integer part of an accumulator advanced by ppc u_sh dt/dx
// (the engine's inflow count, one transverse row)
void injection_schedule(const Phys& ph, int steps, std::vector<int>* ninj) {
  double acc = 0.0;
  ninj->assign(steps, 0);
  for (int n = 0; n < steps; ++n) {
    acc = acc + ph.rate;
    const double fl = std::floor(acc);
    (*ninj)[n] = (int)fl;
    acc = acc - fl;
  }
}

int window_sizes(const fs_params* p, int steps, int ckpt, long long n_init, int M, Geo* g,
                 Phys* ph, int* cap, size_t* total, size_t off[11]) {
  if (!p || steps < 1 || ckpt < 1 || n_init < 0 || M < 0 || M > 4096) return FS_EINVAL;
  if (p->dim != 1 || p->bc_x != FS_BC_FAUXSHOCK || p->c_light != 0.0) return FS_EINVAL;
  // the blocked field kernels keep a tile's RK4 stage inputs in shared memory
  const size_t tb = (p->precision == FS_FP64) ? 8 : 4;
  if (p->n_sub < 1 || p->n_sub > 64 || rk4_adj_smem(p->n_sub, tb) > kMaxSmem) return FS_EINVAL;
  int rc = derive_geometry(p, g, ph);
  if (rc) return rc;
  std::vector<int> ninj;
  injection_schedule(*ph, steps, &ninj);
  long long c = n_init;
  const int kinds = (p->inject_thermal ? 1 : 0) + (p->cr_enable ? 1 : 0);
  for (int v : ninj) c += (long long)v * kinds;
  if (c > (1LL << 30)) return FS_EINVAL;
  *cap = (int)std::max<long long>(c, 1);
  const size_t tsz = (p->precision == FS_FP64) ? 8 : 4;
  const int nx = g->nx, nxn = g->nxn;
  const int nseg = (steps + ckpt - 1) / ckpt;
  const int K = std::min(ckpt, steps);
  size_t o = 0;
  off[0] = o; o += slot_bytes(*cap, tsz);                                  // state
  off[1] = o;                                                               // checkpoints
  o += (size_t)nseg * (slot_bytes(*cap, tsz) + al(3 * tsz * nx) + mom_bytes(nxn, tsz));
  off[2] = o; o += (size_t)(K + 1) * tape_slot_bytes(*cap, tsz);           // particle tape
  off[3] = o; o += (size_t)K * al((size_t)*cap);                           // events
  off[4] = o; o += (size_t)(K + 1) * al(3 * tsz * nx);                     // B^n tape
  off[5] = o; o += (size_t)(K + 1) * mom_bytes(nxn, tsz);                  // moments tape
  off[6] = o; o += 2 * al(3 * tsz * nxn) + 2 * al(3 * tsz * nx) + mom_bytes(nxn, tsz);
  off[7] = o; o += al(8 * 4 * (size_t)nxn);                                // fixed-point sums
  off[8] = o; o += al(8 * 8);                                              // counters
  off[9] = o;
  o += al(tsz * *cap) + al(3 * tsz * *cap);                                // lf, lv
  o += 8 * al(8 * 3 * (size_t)(nx + nxn));                                 // field adjoints
  off[10] = o; o += al(8 * (size_t)(3 * M + 2));                           // amps, phases, grad
  *total = o;
  return FS_OK;
}

template <typename T>
Slots<T> slots_at(char* b, int cap, bool with_id) {
  Slots<T> s;
  size_t o = 0;
  s.ci = (int*)(b + o); o += al(4 * (size_t)cap);
  s.f = (T*)(b + o); o += al(sizeof(T) * cap);
  s.v = (T*)(b + o); o += al(3 * sizeof(T) * cap);
  s.id = with_id ? (uint32_t*)(b + o) : nullptr;
  return s;
}

template <typename T>
Win<T> win_ptrs(fs_window* w) {
  Win<T> r;
  const int nx = w->g.nx, nxn = w->g.nxn;
  r.cap = w->cap;
  r.s = slots_at<T>(w->base + w->o_state, w->cap, true);
  char* f = w->base + w->o_fields;
  size_t o = 0;
  auto take = [&](size_t bytes) { char* q = f + o; o += al(bytes); return q; };
  r.E = (T*)take(3 * sizeof(T) * nxn);
  r.Bb = (T*)take(3 * sizeof(T) * nxn);
  T* B0 = (T*)take(3 * sizeof(T) * nx);
  T* B1 = (T*)take(3 * sizeof(T) * nx);
  r.B = w->bsel ? B1 : B0;  // the current B
  r.Bx = w->bsel ? B0 : B1;
  r.n = (T*)take(sizeof(T) * nxn);
  r.u = (T*)take(3 * sizeof(T) * nxn);
  r.nraw = (T*)take(sizeof(T) * nxn);
  r.q = (unsigned long long*)(w->base + w->o_q);
  r.ctr = (unsigned long long*)(w->base + w->o_ctr);
  char* a = w->base + w->o_adj;
  o = 0;
  auto tka = [&](size_t bytes) { char* q = a + o; o += al(bytes); return q; };
  r.lf = (T*)tka(sizeof(T) * w->cap);
  r.lv = (T*)tka(3 * sizeof(T) * w->cap);
  const size_t fb = 8 * 3 * (size_t)(nx + nxn);
  r.lB = (double*)tka(fb);
  r.lBx = (double*)tka(fb);
  r.lE = (double*)tka(fb);
  r.lBb = (double*)tka(fb);
  r.lNm = (double*)tka(fb);
  r.lUm = (double*)tka(fb);
  r.lNr = (T*)tka(fb);
  r.lJ = (T*)tka(fb);
  r.grad = (double*)(w->base + w->o_params) + 2 * w->M;
  return r;
}

// dynamic shared memory of the blocked field kernels beyond the default 48 KB
template <typename T>
bool smem_opt_in(int n_sub) {
  const int f = (int)fields_smem(n_sub, sizeof(T)), a = (int)rk4_adj_smem(n_sub, sizeof(T));
  return cudaFuncSetAttribute(k_win_fields<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, f) ==
             cudaSuccess &&
         cudaFuncSetAttribute(k_win_rk4_adj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, a) ==
             cudaSuccess;
}

// checkpoint c: slots, B, moments
struct Ck {
  char* slots;
  char* B;
  char* mom;
};
Ck ckpt_at(fs_window* w, int c) {
  const size_t sb = slot_bytes(w->cap, w->tsz), bb = al(3 * w->tsz * w->g.nx);
  const size_t one = sb + bb + mom_bytes(w->g.nxn, w->tsz);
  char* b = w->base + w->o_ckpt + (size_t)c * one;
  return Ck{b, b + sb, b + sb + bb};
}
template <typename T>
void mom_ptrs(char* b, int nxn, T** n, T** u, T** r) {
  *n = (T*)b;
  *u = (T*)(b + al(sizeof(T) * nxn));
  *r = (T*)(b + 4 * al(sizeof(T) * nxn));
}
template <typename T>
Slots<T> tape_at(fs_window* w, int k) {
  return slots_at<T>(w->base + w->o_tape + (size_t)k * tape_slot_bytes(w->cap, w->tsz), w->cap,
                     false);
}
uint8_t* ev_at(fs_window* w, int k) {
  return (uint8_t*)(w->base + w->o_ev) + (size_t)k * al(w->cap);
}
template <typename T>
T* tapeB_at(fs_window* w, int k) {
  return (T*)(w->base + w->o_tapeB + (size_t)k * al(3 * sizeof(T) * w->g.nx));
}
char* tapeM_at(fs_window* w, int k) {
  return w->base + w->o_tapeM + (size_t)k * mom_bytes(w->g.nxn, w->tsz);
}

void cpy(void* d, const void* s, size_t n, cudaStream_t st) {
  cudaMemcpyAsync(d, s, n, cudaMemcpyDeviceToDevice, st);
}

// one forward step n; with tape index k >= 0 the step's inputs are taped
template <typename T>
void forward_step(fs_window* w, Win<T>& r, int n, int k) {
  const int np = w->np_at[n];
  Slots<T> tp{};
  uint8_t* ev = nullptr;
  T *tn = nullptr, *tu = nullptr, *tr = nullptr, *tB = nullptr;
  if (k >= 0) {
    tp = tape_at<T>(w, k);
    ev = ev_at(w, k);
    tB = tapeB_at<T>(w, k);
    mom_ptrs<T>(tapeM_at(w, k + 1), w->g.nxn, &tn, &tu, &tr);
  }
  const int kinds = (w->ph.inject_thermal ? 1 : 0) + (w->ph.cr_enable ? 1 : 0);
  const int nadd = w->ninj[n] * kinds;
  const int ib = (nadd > 0) ? blocks(nadd) : 0;
  const int pb = (np > 0) ? blocks(np) : 1;  // one block at least: it clears the sums
  k_win_push_inject<T><<<ib + pb, kBlock, 0, w->st>>>(r, tp, ev, w->g, w->ph,
                                                      push_const<T>(w->ph), n, np, w->ninj[n],
                                                      w->first_id[n], ib);
  const int np1 = w->np_at[n + 1];
  if (np1 > 0) k_win_deposit<T><<<blocks(np1), kBlock, 0, w->st>>>(r, w->g, w->ph, push_const<T>(w->ph),
                                                        np1);
  k_win_fields<T><<<tiles(w->g.nx), kTbThreads, fields_smem(w->p.n_sub, sizeof(T)), w->st>>>(
      r, w->g, w->ph, field_const<T>(w->ph), w->p.n_sub, r.Bx, tn, tu, tr, tB);
  std::swap(r.B, r.Bx);  // the step's B went to the other buffer
  w->bsel ^= 1;
}

template <typename T>
void save_ckpt(fs_window* w, Win<T>& r, int c) {
  Ck ck = ckpt_at(w, c);
  cpy(ck.slots, w->base + w->o_state, slot_bytes(w->cap, w->tsz), w->st);
  cpy(ck.B, r.B, 3 * sizeof(T) * w->g.nx, w->st);
  T *n, *u, *q;
  mom_ptrs<T>(ck.mom, w->g.nxn, &n, &u, &q);
  cpy(n, r.n, sizeof(T) * w->g.nxn, w->st);
  cpy(u, r.u, 3 * sizeof(T) * w->g.nxn, w->st);
  cpy(q, r.nraw, sizeof(T) * w->g.nxn, w->st);
}
template <typename T>
void load_ckpt(fs_window* w, Win<T>& r, int c) {
  Ck ck = ckpt_at(w, c);
  cpy(w->base + w->o_state, ck.slots, slot_bytes(w->cap, w->tsz), w->st);
  cpy(r.B, ck.B, 3 * sizeof(T) * w->g.nx, w->st);
  T *n, *u, *q;
  mom_ptrs<T>(ck.mom, w->g.nxn, &n, &u, &q);
  cpy(r.n, n, sizeof(T) * w->g.nxn, w->st);
  cpy(r.u, u, 3 * sizeof(T) * w->g.nxn, w->st);
  cpy(r.nraw, q, sizeof(T) * w->g.nxn, w->st);
  k_ohm<T, 1><<<blocks(w->g.nxn), kBlock, 0, w->st>>>(r.B, r.n, r.u, nullptr, r.E, r.Bb,
                                                       nullptr, w->g, w->ph);
}

template <typename T>
int do_forward(fs_window* w, const double* theta, double* loss) {
  Win<T> r = win_ptrs<T>(w);
  const int M = w->M;
  if (!(theta[M + 1] > 0.0) || !(theta[M] >= 0.0) || !(theta[M] < w->ph.p_iso_v))
    return FS_EINVAL;
  w->ph.u_cr = theta[M];
  w->ph.u2 = theta[M + 1];
  double* amps = (double*)(w->base + w->o_params);
  if (M > 0 && cudaMemcpyAsync(amps, theta, sizeof(double) * M, cudaMemcpyHostToDevice,
                               w->st) != cudaSuccess)
    return FS_ECUDA;
  cudaMemsetAsync(r.ctr, 0, 8 * 8, w->st);
  // initial state: the caller's particles (kept in checkpoint 0's slots
  // since fs_window_init), B0 + modes, moments, E
  Ck c0 = ckpt_at(w, 0);
  cpy(w->base + w->o_state, c0.slots, slot_bytes(w->cap, w->tsz), w->st);
  k_win_seed_B<T><<<blocks(w->g.nx), kBlock, 0, w->st>>>(r.B, w->g, w->ph, w->p.dx, amps,
                                                          amps + M, M);
  cudaMemsetAsync(r.q, 0, 8 * 4 * (size_t)w->g.nxn, w->st);
  const int np0 = w->np_at[0];
  if (np0 > 0) k_win_deposit<T><<<blocks(np0), kBlock, 0, w->st>>>(r, w->g, w->ph, push_const<T>(w->ph),
                                                        np0);
  k_win_moments<T><<<blocks(w->g.nxn), kBlock, 0, w->st>>>(r, w->g, w->ph);
  k_ohm<T, 1><<<blocks(w->g.nxn), kBlock, 0, w->st>>>(r.B, r.n, r.u, nullptr, r.E, r.Bb,
                                                       nullptr, w->g, w->ph);
  for (int n = 0; n < w->steps; ++n) {
    if (n % w->ckpt == 0) save_ckpt<T>(w, r, n / w->ckpt);
    forward_step<T>(w, r, n, -1);
  }
  double* dl = r.lBx;  // scratch for the loss (free outside the backward)
  k_win_loss<T><<<1, kBlock, 0, w->st>>>(r.B, w->g, w->ph, w->loss_i0, w->p.dx,
                                                       dl, nullptr, 1.0);
  unsigned long long c[5];
  if (cudaMemcpyAsync(loss, dl, 8, cudaMemcpyDeviceToHost, w->st) != cudaSuccess ||
      cudaMemcpyAsync(c, r.ctr, sizeof(c), cudaMemcpyDeviceToHost, w->st) != cudaSuccess ||
      cudaStreamSynchronize(w->st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return FS_ECUDA;
  for (int k = 0; k < 5; ++k) w->counts[k] = (long long)c[k];
  w->have_forward = true;
  return FS_OK;
}

template <typename T>
int do_backward(fs_window* w, double dloss, double* grad) {
  if (!w->have_forward) return FS_EINVAL;
  Win<T> r = win_ptrs<T>(w);
  const int nx = w->g.nx, nxn = w->g.nxn, M = w->M;
  const size_t fb = 8 * 3 * (size_t)(nx + nxn);
  cudaMemsetAsync(r.grad, 0, 8 * (M + 2), w->st);
  cudaMemsetAsync(r.lf, 0, sizeof(T) * w->cap, w->st);
  cudaMemsetAsync(r.lv, 0, 3 * sizeof(T) * w->cap, w->st);
  cudaMemsetAsync(r.lNm, 0, fb, w->st);
  cudaMemsetAsync(r.lUm, 0, fb, w->st);
  // d loss / d B at the end (r.B holds the final field after the forward)
  k_win_loss<T><<<1, kBlock, 0, w->st>>>(r.B, w->g, w->ph, w->loss_i0, w->p.dx,
                                                  nullptr, r.lB, dloss);
  for (int seg = w->nseg - 1; seg >= 0; --seg) {
    const int n0 = seg * w->ckpt;
    const int n1 = std::min(w->steps, n0 + w->ckpt);
    // recompute the segment with its tape
    load_ckpt<T>(w, r, seg);
    {
      T *tn, *tu, *tr;
      mom_ptrs<T>(tapeM_at(w, 0), nxn, &tn, &tu, &tr);
      cpy(tn, r.n, sizeof(T) * nxn, w->st);
      cpy(tu, r.u, 3 * sizeof(T) * nxn, w->st);
      cpy(tr, r.nraw, sizeof(T) * nxn, w->st);
    }
    for (int n = n0; n < n1; ++n) forward_step<T>(w, r, n, n - n0);
    {
      Slots<T> tk = tape_at<T>(w, n1 - n0);  // the state after the segment
      cpy(tk.ci, r.s.ci, 4 * (size_t)w->cap, w->st);
      cpy(tk.f, r.s.f, sizeof(T) * w->cap, w->st);
      cpy(tk.v, r.s.v, 3 * sizeof(T) * w->cap, w->st);
    }
    for (int n = n1 - 1; n >= n0; --n) {
      const int k = n - n0;
      T *mn1, *mu1, *mr1, *mn0, *mu0, *mr0;
      mom_ptrs<T>(tapeM_at(w, k + 1), nxn, &mn1, &mu1, &mr1);
      mom_ptrs<T>(tapeM_at(w, k), nxn, &mn0, &mu0, &mr0);
      const T* Bn = tapeB_at<T>(w, k);
      // the step's field update and moments in reverse; E^n, Bbar^n as the
      // forward had them
      k_win_rk4_adj<T><<<tiles(w->g.nx), kTbThreads, rk4_adj_smem(w->p.n_sub, sizeof(T)), w->st>>>(
          r, w->g, w->ph, field_const<T>(w->ph), w->p.n_sub, Bn, mn1, mu1, mr1, mn0, mu0, r.lB,
          r.lBx);
      std::swap(r.lB, r.lBx);
      const int npa = w->np_at[n], npb = w->np_at[n + 1];
      if (npb > 0)
        k_win_particle_adj<T><<<blocks(npb), kBlock, 0, w->st>>>(
            r, tape_at<T>(w, k), tape_at<T>(w, k + 1), ev_at(w, k), w->g, w->ph,
            push_const<T>(w->ph), n, npa, npb, M);
      // Ohm at the start of the step: lB += ..., lNm, lUm = adjoint of M^n
      k_win_ohm_adj_step<T><<<tiles(w->g.nx), kTbThreads, 0, w->st>>>(r, w->g, w->ph, Bn, mn0, mu0);
    }
  }
  double* phases = (double*)(w->base + w->o_params) + M;
  if (M > 0) k_win_mode_grad<<<M, kBlock, 0, w->st>>>(r.lB, r.grad, phases, w->g, w->p.dx);
  if (cudaMemcpyAsync(grad, r.grad, 8 * (M + 2), cudaMemcpyDeviceToHost, w->st) != cudaSuccess ||
      cudaStreamSynchronize(w->st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return FS_ECUDA;
  // the recompute overwrote the forward's final state: a new forward is due
  w->have_forward = false;
  return FS_OK;
}

}  // namespace

extern "C" {

int fs_window_query(const fs_params* p, int steps, int ckpt_every, long long n_init,
                    int n_modes, size_t* bytes) {
  FS_GUARD_BEGIN
  if (!bytes) return FS_EINVAL;
  Geo g;
  Phys ph;
  int cap;
  size_t off[11];
  return window_sizes(p, steps, ckpt_every, n_init, n_modes, &g, &ph, &cap, bytes, off);
  FS_GUARD_END
}

int fs_window_init(const fs_params* p, int steps, int ckpt_every, long long n_init,
                   const double* x_init, const double* v_init, int n_modes,
                   const double* mode_phase, int loss_i0, void* dev_buf, size_t bytes,
                   void* cuda_stream, fs_window** out) {
  FS_GUARD_BEGIN
  if (!out || (n_init > 0 && (!x_init || !v_init)) || (n_modes > 0 && !mode_phase) || !dev_buf)
    return FS_EINVAL;
  *out = nullptr;
  Geo g;
  Phys ph;
  int cap;
  size_t need, off[11];
  int rc = window_sizes(p, steps, ckpt_every, n_init, n_modes, &g, &ph, &cap, &need, off);
  if (rc) return rc;
  if (bytes < need || ((uintptr_t)dev_buf % kAl) != 0) return FS_EINVAL;
  if (loss_i0 < 0 || loss_i0 > g.nx) return FS_EINVAL;
  for (long long k = 0; k < n_init; ++k)
    if (!(x_init[k] >= 0.0 && x_init[k] < (double)g.nx)) return FS_EINVAL;
  fs_window* w = new fs_window();
  w->p = *p;
  w->g = g;
  w->ph = ph;
  w->steps = steps;
  w->ckpt = ckpt_every;
  w->nseg = (steps + ckpt_every - 1) / ckpt_every;
  w->M = n_modes;
  w->loss_i0 = loss_i0;
  w->n_init = n_init;
  w->cap = cap;
  w->tsz = (p->precision == FS_FP64) ? 8 : 4;
  w->base = (char*)dev_buf;
  w->st = (cudaStream_t)cuda_stream;
  w->o_state = off[0]; w->o_ckpt = off[1]; w->o_tape = off[2]; w->o_ev = off[3];
  w->o_tapeB = off[4]; w->o_tapeM = off[5]; w->o_fields = off[6]; w->o_q = off[7];
  w->o_ctr = off[8]; w->o_adj = off[9]; w->o_params = off[10];
  // slot schedule: initial particles, then per step the thermal and
  // cosmic-ray injections (ids continue from n_init)
  injection_schedule(ph, steps, &w->ninj);
  const int kinds = (p->inject_thermal ? 1 : 0) + (p->cr_enable ? 1 : 0);
  w->np_at.assign(steps + 1, 0);
  w->first_id.assign(steps, 0);
  long long np = n_init;
  for (int n = 0; n < steps; ++n) {
    w->np_at[n] = (int)np;
    w->first_id[n] = (unsigned long long)np;
    np += (long long)w->ninj[n] * kinds;
  }
  w->np_at[steps] = (int)np;
  // initial particles into checkpoint 0's slots (cell + offset)
  const size_t tsz = w->tsz;
  std::vector<char> host(slot_bytes(cap, tsz), 0);
  int* hci = (int*)host.data();
  char* hf = host.data() + al(4 * (size_t)cap);
  char* hv = hf + al(tsz * cap);
  uint32_t* hid = (uint32_t*)(hv + al(3 * tsz * cap));
  for (int k = 0; k < cap; ++k) hci[k] = -1;
  for (long long k = 0; k < n_init; ++k) {
    const double X = x_init[k];
    const double ix = std::floor(X);
    hci[k] = (int)ix;
    const double fx = X - ix;
    hid[k] = (uint32_t)k;
    if (tsz == 8) {
      ((double*)hf)[k] = fx;
      for (int c = 0; c < 3; ++c) ((double*)hv)[(size_t)c * cap + k] = v_init[3 * k + c];
    } else {
      float ft = (float)fx;
      if (ft >= 1.0f) ft = 0x1.fffffep-1f;
      ((float*)hf)[k] = ft;
      for (int c = 0; c < 3; ++c) ((float*)hv)[(size_t)c * cap + k] = (float)v_init[3 * k + c];
    }
  }
  Ck c0 = ckpt_at(w, 0);
  bool ok = (tsz == 8 ? smem_opt_in<double>(p->n_sub) : smem_opt_in<float>(p->n_sub)) &&
            cudaMemcpyAsync(c0.slots, host.data(), host.size(), cudaMemcpyHostToDevice, w->st) ==
                cudaSuccess &&
            (n_modes == 0 ||
             cudaMemcpyAsync(w->base + w->o_params + 8 * (size_t)n_modes, mode_phase,
                             8 * (size_t)n_modes, cudaMemcpyHostToDevice, w->st) == cudaSuccess) &&
            cudaStreamSynchronize(w->st) == cudaSuccess;
  if (!ok) {
    delete w;
    return FS_ECUDA;
  }
  *out = w;
  return FS_OK;
  FS_GUARD_END
}

int fs_window_forward(fs_window* w, const double* theta, double* loss) {
  FS_GUARD_BEGIN
  if (!w || !theta || !loss) return FS_EINVAL;
  return w->tsz == 8 ? do_forward<double>(w, theta, loss) : do_forward<float>(w, theta, loss);
  FS_GUARD_END
}

int fs_window_backward(fs_window* w, double dloss, double* grad) {
  FS_GUARD_BEGIN
  if (!w || !grad) return FS_EINVAL;
  return w->tsz == 8 ? do_backward<double>(w, dloss, grad) : do_backward<float>(w, dloss, grad);
  FS_GUARD_END
}

int fs_window_counts(fs_window* w, long long* out5) {
  FS_GUARD_BEGIN
  if (!w || !out5) return FS_EINVAL;
  for (int k = 0; k < 5; ++k) out5[k] = w->counts[k];
  return FS_OK;
  FS_GUARD_END
}

int fs_window_destroy(fs_window* w) {
  FS_GUARD_BEGIN
  delete w;
  return FS_OK;
  FS_GUARD_END
}

}  // extern "C"
