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
#include <mutex>
#include <vector>

#include "fs_engine.cuh"

namespace fsx {
namespace win {

constexpr double kFix = 1099511627776.0;  // 2^40
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
  // fields: B at centres [3][nx]; E, Bbar at nodes [3][nxn]; RK4 stages
  T *B, *Bs, *Bsum, *E, *Es, *Bb;
  T *n, *u, *nraw;             // moments in use [nxn], [3][nxn], [nxn]
  unsigned long long* q;       // fixed-point deposit sums [4][nxn]
  unsigned long long* ctr;     // incident, returned, transmitted, escaped, injected
  // adjoint
  T *lf, *lv;                  // particle adjoints: offset, velocity [3][cap]
  double *lB, *lE, *lBb;       // [3][nx], [3][nxn], [3][nxn]
  double *lN, *lU;             // adjoint of the moments of the step being reversed
  double *lNm, *lUm;           // adjoint of the moments that E^n used
  double *lNr, *lJ;            // deposit adjoints (raw density, current)
  double *P;                   // node partials [4][nxn]
  double *Y;                   // RK4 stage inputs [n_sub][4][3][nx]
  double *g, *lY, *lsum, *lend;  // RK4 adjoint work [3][nx]
  double* grad;                // d loss / d theta [M + 2]
};

// ---------------------------------------------------------------- forward
template <typename T>
__global__ void k_win_push(Win<T> w, Slots<T> tape, uint8_t* ev, Geo g, Phys ph,
                           long long step, int np) {
  const int nxn = g.nxn;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
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
      continue;
    }
    uint8_t e = kEvNone;
    const T g0 = (T)1 - f;
    T Ep[3], Bp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Ep[c] = fmaT(f, w.E[c * nxn + ci + 1], g0 * w.E[c * nxn + ci]);
      Bp[c] = fmaT(f, w.Bb[c * nxn + ci + 1], g0 * w.Bb[c * nxn + ci]);
    }
    boris<T>(vx, vy, vz, Ep, Bp, (T)ph.hdt);
    const T fr = fmaT(vx, (T)ph.dtdx, f);
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
      continue;
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
__global__ void k_win_inject(Win<T> w, Geo g, Phys ph, long long step, int np, int n_new,
                             unsigned long long first) {
  const int nth = ph.inject_thermal ? n_new : 0;
  const int ncr = ph.cr_enable ? n_new : 0;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
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

__device__ __forceinline__ unsigned long long fix(double c) {
  return (unsigned long long)__double2ll_rn(c * kFix);
}

// CIC deposit of every live slot into the fixed-point sums (order free).
template <typename T>
__global__ void k_win_deposit(Win<T> w, Geo g, Phys ph, int np) {
  const int nxn = g.nxn;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    const int ci = w.s.ci[p];
    if (ci < 0) continue;
    const double wp = (w.s.id[p] & kIdCR) ? ph.w_cr : ph.w_th;
    const double f = (double)w.s.f[p];
    const double c0 = wp * (1.0 - f), c1 = wp * f;
    const double v[3] = {(double)w.s.v[p], (double)w.s.v[w.cap + p],
                         (double)w.s.v[2 * w.cap + p]};
    atomicAdd(&w.q[ci], fix(c0));
    atomicAdd(&w.q[ci + 1], fix(c1));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicAdd(&w.q[(c + 1) * nxn + ci], fix(c0 * v[c]));
      atomicAdd(&w.q[(c + 1) * nxn + ci + 1], fix(c1 * v[c]));
    }
  }
}

// Moments from the sums: wall nodes x2, density floor, u = J / n; clears the
// sums. Also writes a copy (the tape of these moments) when given.
template <typename T>
__global__ void k_win_moments(Win<T> w, Geo g, Phys ph, T* tn, T* tu, T* tr) {
  const int nxn = g.nxn;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nxn) return;
  const double sc = (i == 0 || i == g.nx) ? 2.0 : 1.0;
  const double nr = (double)(long long)w.q[i] * kUnfix * sc;
  double J[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    J[c] = (double)(long long)w.q[(c + 1) * nxn + i] * kUnfix * sc;
    w.q[(c + 1) * nxn + i] = 0ull;
  }
  w.q[i] = 0ull;
  T n = (T)nr;
  const T nf = (T)ph.n_floor;
  if (n < nf) n = nf;
  w.nraw[i] = (T)nr;
  w.n[i] = n;
#pragma unroll
  for (int c = 0; c < 3; ++c) w.u[c * nxn + i] = (T)J[c] / n;
  if (tn) {
    tn[i] = n;
    tr[i] = (T)nr;
#pragma unroll
    for (int c = 0; c < 3; ++c) tu[c * nxn + i] = w.u[c * nxn + i];
  }
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
// gradient with respect to B (into lB) when lB is given
template <typename T>
__global__ void k_win_loss(const T* B, Geo g, Phys ph, int i0, double dx, double* out,
                           double* lB) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.nx; i += gridDim.x * blockDim.x) {
    double dy = 0.0, dz = 0.0;
    if (i >= i0) {
      dy = (double)B[g.nx + i] - ph.b0y;
      dz = (double)B[2 * g.nx + i] - ph.b0z;
      s += (dy * dy + dz * dz) * dx;
    }
    if (lB) {
      lB[i] = 0.0;
      lB[g.nx + i] = 2.0 * dy * dx;
      lB[2 * g.nx + i] = 2.0 * dz * dx;
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && out) atomicAdd(out, s);
}

// ---------------------------------------------------------------- adjoint
// Node-local part of the adjoint of Ohm's law (1D, nodes i = 0..nx), for a
// centre field Bc with n, u frozen. The adjoint of E at the node comes from
// lE, or, with gK != nullptr, from the adjoint gK of K = -curl E at the
// centres (Faraday: K_y(c) = (E_z(c+1) - E_z(c))/dx, K_z(c) = -(E_y(c+1) -
// E_y(c))/dx). lBbar (optional) adds the adjoint of Bbar. Writes the
// adjoints of the node's Bbar_y, Bbar_z, dB_y/dx, dB_z/dx into P and adds the
// adjoints of n and u.
template <typename T>
__global__ void k_win_ohm_adj(const double* Bc, const T* nN, const T* uN, const double* gK,
                              const double* lE, const double* lBbar, double* P, double* lN,
                              double* lU, Geo g, Phys ph) {
  const int nx = g.nx, nxn = g.nxn;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nxn) return;
  const double idx = ph.idx, te = ph.te, jcr = ph.jcr, eta = ph.eta;
  double lex, ley, lez;
  if (gK) {
    const double gym = (i >= 1) ? gK[nx + i - 1] : 0.0, gy = (i < nx) ? gK[nx + i] : 0.0;
    const double gzm = (i >= 1) ? gK[2 * nx + i - 1] : 0.0, gz = (i < nx) ? gK[2 * nx + i] : 0.0;
    lex = 0.0;
    lez = (gym - gy) * idx;
    ley = (gz - gzm) * idx;
  } else {
    lex = lE[i];
    ley = lE[nxn + i];
    lez = lE[2 * nxn + i];
  }
  const int im = min(max(i - 1, 0), nx - 1), ip = min(max(i, 0), nx - 1);
  const double bbx = 0.5 * (Bc[im] + Bc[ip]);
  const double bby = 0.5 * (Bc[nx + im] + Bc[nx + ip]);
  const double bbz = 0.5 * (Bc[2 * nx + im] + Bc[2 * nx + ip]);
  const double dby = (Bc[nx + ip] - Bc[nx + im]) * idx;
  const double dbz = (Bc[2 * nx + ip] - Bc[2 * nx + im]) * idx;
  const double n = (double)nN[i];
  const double ux = (double)uN[i], uy = (double)uN[nxn + i], uz = (double)uN[2 * nxn + i];
  const double in = 1.0 / n;
  // E = ((curl B - jcr x) x Bbar - T_e grad n)/n - u x Bbar + eta curl B,
  // curl B = (0, -dbz, dby)
  double lbby = lex * (-dby * in + uz) + lez * (-jcr * in - ux);
  double lbbz = lex * (-dbz * in - uy) + ley * (jcr * in + ux);
  const double ldby = lex * (-bby * in) + ley * (bbx * in) + lez * eta;
  const double ldbz = lex * (-bbz * in) + lez * (bbx * in) - ley * eta;
  if (lBbar) {
    lbby += lBbar[nxn + i];
    lbbz += lBbar[2 * nxn + i];
  }
  P[i] = lbby;
  P[nxn + i] = lbbz;
  P[2 * nxn + i] = ldby;
  P[3 * nxn + i] = ldbz;
  // moments: 1/n and the pressure term -T_e (n(i+1) - n(i-1)) / (2 dx)
  // (mirrored density at the walls); neighbours add too, so atomics
  const double cax = -dbz * bbz - dby * bby;
  const double cay = dby * bbx + jcr * bbz;
  const double caz = -jcr * bby + dbz * bbx;
  const int ipn = (i + 1 > nx) ? 2 * nx - (i + 1) : i + 1;
  const int imn = (i - 1 < 0) ? -(i - 1) : i - 1;
  const double pgx = -(te * (((double)nN[ipn] - (double)nN[imn]) * ph.hdx));
  atomicAdd(&lN[i], -(lex * (pgx + cax) + ley * cay + lez * caz) * in * in);
  const double lp = -lex * in * te * ph.hdx;  // d ex / d n(i+1); the negative for n(i-1)
  if (lp != 0.0) {
    atomicAdd(&lN[ipn], lp);
    atomicAdd(&lN[imn], -lp);
  }
  // u x Bbar: ex = .. - (uy bbz - uz bby), ey = .. - (uz bbx - ux bbz),
  // ez = .. - (ux bby - uy bbx); only node i touches lU(i)
  lU[i] += ley * bbz - lez * bby;
  lU[nxn + i] += -lex * bbz + lez * bbx;
  lU[2 * nxn + i] += lex * bby - ley * bbx;
}

// Centre part: the adjoint of B(c) from its two nodes (Bbar = (Bm + Bp)/2,
// dB = (Bp - Bm)/dx, with the wall nodes reading cell 0 or nx - 1 twice).
// out = adjoint of B; then acc += out (if acc) and gn = a * lend + b * out
// (if gn: the next RK4 stage's adjoint).
__global__ void k_win_curl_adj(const double* P, double* out, double* acc, double* gn,
                               const double* lend, double a, double b, Geo g, Phys ph) {
  const int nx = g.nx, nxn = g.nxn;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nx) return;
  const double idx = ph.idx;
  double ly = 0.0, lz = 0.0;
  // node c sees cell c as its p side, node c + 1 sees it as its m side
  ly += 0.5 * P[c] + P[2 * nxn + c] * idx;
  lz += 0.5 * P[nxn + c] + P[3 * nxn + c] * idx;
  ly += 0.5 * P[c + 1] - P[2 * nxn + c + 1] * idx;
  lz += 0.5 * P[nxn + c + 1] - P[3 * nxn + c + 1] * idx;
  if (c == 0) {  // node 0: m side clamped to cell 0
    ly += 0.5 * P[0] - P[2 * nxn] * idx;
    lz += 0.5 * P[nxn] - P[3 * nxn] * idx;
  }
  if (c == nx - 1) {  // node nx: p side clamped to cell nx - 1
    ly += 0.5 * P[nx] + P[2 * nxn + nx] * idx;
    lz += 0.5 * P[nxn + nx] + P[3 * nxn + nx] * idx;
  }
  out[c] = 0.0;
  out[nx + c] = ly;
  out[2 * nx + c] = lz;
  if (acc) {
    acc[nx + c] += ly;
    acc[2 * nx + c] += lz;
  }
  if (gn) {
    gn[c] = 0.0;
    gn[nx + c] = a * lend[nx + c] + b * ly;
    gn[2 * nx + c] = a * lend[2 * nx + c] + b * lz;
  }
}

// dst = a * x (+ b * y)
__global__ void k_win_axpy(double* dst, const double* x, double a, const double* y, double b,
                           int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

template <typename T>
__global__ void k_win_to_double(double* dst, const T* src, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i];
}

// Adjoint of the moments of one step: from the adjoints of n (floored) and
// u = J / n to those of the raw sums (wall nodes x2, no gradient through a
// floored density).
template <typename T>
__global__ void k_win_moments_adj(const T* nN, const T* uN, const T* nraw, const double* lN,
                                  const double* lU, double* lNr, double* lJ, Geo g, Phys ph) {
  const int nxn = g.nxn;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nxn) return;
  const double sc = (i == 0 || i == g.nx) ? 2.0 : 1.0;
  const double n = (double)nN[i];
  double ln = lN[i];
  for (int c = 0; c < 3; ++c) {
    lJ[c * nxn + i] = lU[c * nxn + i] / n * sc;
    ln -= lU[c * nxn + i] * (double)uN[c * nxn + i] / n;
  }
  lNr[i] = ((double)nraw[i] < ph.n_floor) ? 0.0 : ln * sc;
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Adjoint of one step for every slot p < np1 (slots alive at the end of the
// step or born in it). In: lf, lv = adjoints of the state after the step;
// lNr, lJ = adjoints of the step's deposit; E, Bb = the node fields the
// step's gather used. Out: lf, lv = adjoints of the state before the step
// (zero for slots born or removed in it); lE, lBb (atomics); grad[M] (u_cr),
// grad[M + 1] (u2).
template <typename T>
__global__ void k_win_particle_adj(Win<T> w, Slots<T> t0, Slots<T> t1, const uint8_t* ev,
                                   Geo g, Phys ph, long long step, int np0, int np1, int M) {
  const int nxn = g.nxn;
  const int cap = w.cap;
  double gu2 = 0.0, gucr = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np1; p += gridDim.x * blockDim.x) {
    const bool born = p >= np0;
    const uint8_t e = born ? (uint8_t)kEvNone : ev[p];
    const int c1 = t1.ci[p];
    if (c1 < 0 || (!born && t0.ci[p] < 0) || e == kEvRemoved) {
      w.lf[p] = (T)0;
      w.lv[p] = w.lv[cap + p] = w.lv[2 * cap + p] = (T)0;
      continue;
    }
    // ---- deposit at the state after the step
    const uint32_t id = w.s.id[p];
    const double wp = (id & kIdCR) ? ph.w_cr : ph.w_th;
    const double f1 = (double)t1.f[p];
    const double v1[3] = {(double)t1.v[p], (double)t1.v[cap + p], (double)t1.v[2 * cap + p]};
    double lf1 = (double)w.lf[p];
    double lv[3] = {(double)w.lv[p], (double)w.lv[cap + p], (double)w.lv[2 * cap + p]};
    {
      double dj = w.lNr[c1 + 1] - w.lNr[c1];
      for (int c = 0; c < 3; ++c) {
        const double ja = w.lJ[c * nxn + c1], jb = w.lJ[c * nxn + c1 + 1];
        dj += (jb - ja) * v1[c];
        lv[c] += wp * ((1.0 - f1) * ja + f1 * jb);
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
        gucr += lv[0] * dvx + lv[1] * dvy + lv[2] * dvz;
        const double ix = floor(X);
        if (ix >= 0.0 && ix < (double)g.nx)  // placement not clamped
          gucr += lf1 * U[3] * dvx * ph.dtdx;
      }
      w.lf[p] = (T)0;
      w.lv[p] = w.lv[cap + p] = w.lv[2 * cap + p] = (T)0;
      continue;
    }
    // ---- recompute the push from the state before the step
    const int c0 = t0.ci[p];
    const double f0 = (double)t0.f[p];
    const T ft0 = t0.f[p];
    const T g0t = (T)1 - ft0;
    T Ep[3], Bp[3];
    double Ed[3], Bd[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Ep[c] = fmaT(ft0, w.E[c * nxn + c0 + 1], g0t * w.E[c * nxn + c0]);
      Bp[c] = fmaT(ft0, w.Bb[c * nxn + c0 + 1], g0t * w.Bb[c * nxn + c0]);
      Ed[c] = (double)w.E[c * nxn + c0 + 1] - (double)w.E[c * nxn + c0];
      Bd[c] = (double)w.Bb[c * nxn + c0 + 1] - (double)w.Bb[c * nxn + c0];
    }
    const double v0[3] = {(double)t0.v[p], (double)t0.v[cap + p], (double)t0.v[2 * cap + p]};
    T vxt = t0.v[p], vyt = t0.v[cap + p], vzt = t0.v[2 * cap + p];
    boris<T>(vxt, vyt, vzt, Ep, Bp, (T)ph.hdt);
    const double vp[3] = {(double)vxt, (double)vyt, (double)vzt};  // before the return
    double lvp[3];  // adjoint of vp
    double lf0;
    if (e == kEvReturned) {
      // vnew = R(vp; u2), f1 = clamp(gf * vnew_x * dtdx), gf = Xn/(Xn - Xo)
      const Philox4 r = draw4(ph.seed, id & kIdMask, step, kPurposeFS);
      const double s1 = sqrt(u01(r.x[1]));
      double cs, sn2;
      fs_sincos2pi(u01(r.x[2]), &cs, &sn2);
      const double u2 = ph.u2;
      const double wx = vp[0] + u2;
      const double wv = sqrt(wx * wx + vp[1] * vp[1] + vp[2] * vp[2]);
      const double a = u2 / wv;
      const double mu = a + (1.0 - a) * s1;
      const double snm = sqrt(fmax(1.0 - mu * mu, 0.0));
      const double vnx = wv * mu - u2;
      const double av = vp[0] * ph.dtdx;  // Xn - Xo
      const double Xo = (double)c0 + f0;
      const double gf = (Xo + av) / av;
      const double fraw = gf * vnx * ph.dtdx;
      double Lx = lv[0], Ly = lv[1], Lz = lv[2];
      double lXo = 0.0, lav = 0.0;
      if (fraw >= 0.0 && fraw < 1.0) {
        Lx += lf1 * gf * ph.dtdx;
        const double lgf = lf1 * vnx * ph.dtdx;
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
      lvp[0] = Lw * wx / wv + lav * ph.dtdx;
      lvp[1] = Lw * vp[1] / wv;
      lvp[2] = Lw * vp[2] / wv;
      lf0 = lXo;
    } else {
      lvp[0] = lv[0] + lf1 * ph.dtdx;
      lvp[1] = lv[1];
      lvp[2] = lv[2];
      lf0 = lf1;
    }
    // ---- Boris adjoint: v+ = q + em, q = vm + p x s, p = vm + vm x t,
    //      s = (2 / (1 + t.t)) t, t = hdt B, vm = v + em, em = hdt E
    const double hdt = ph.hdt;
    double em[3], vm[3], t[3], sv[3], pp[3];
    for (int c = 0; c < 3; ++c) {
      em[c] = hdt * (double)Ep[c];
      vm[c] = v0[c] + em[c];
      t[c] = hdt * (double)Bp[c];
    }
    const double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const double fct = 2.0 / (1.0 + tt);
    for (int c = 0; c < 3; ++c) sv[c] = fct * t[c];
    pp[0] = vm[0] + (vm[1] * t[2] - vm[2] * t[1]);
    pp[1] = vm[1] + (vm[2] * t[0] - vm[0] * t[2]);
    pp[2] = vm[2] + (vm[0] * t[1] - vm[1] * t[0]);
    const double* Lq = lvp;
    double Lem[3] = {lvp[0], lvp[1], lvp[2]};
    double Lvm[3] = {Lq[0], Lq[1], Lq[2]};
    // q = vm + p x s: L_p = s x L_q, L_s = L_q x p
    const double Lp[3] = {sv[1] * Lq[2] - sv[2] * Lq[1], sv[2] * Lq[0] - sv[0] * Lq[2],
                          sv[0] * Lq[1] - sv[1] * Lq[0]};
    const double Ls[3] = {Lq[1] * pp[2] - Lq[2] * pp[1], Lq[2] * pp[0] - Lq[0] * pp[2],
                          Lq[0] * pp[1] - Lq[1] * pp[0]};
    // p = vm + vm x t: L_vm += L_p + t x L_p, L_t = L_p x vm
    Lvm[0] += Lp[0] + (t[1] * Lp[2] - t[2] * Lp[1]);
    Lvm[1] += Lp[1] + (t[2] * Lp[0] - t[0] * Lp[2]);
    Lvm[2] += Lp[2] + (t[0] * Lp[1] - t[1] * Lp[0]);
    double Lt[3] = {Lp[1] * vm[2] - Lp[2] * vm[1], Lp[2] * vm[0] - Lp[0] * vm[2],
                    Lp[0] * vm[1] - Lp[1] * vm[0]};
    // s = fct t, fct = 2 / (1 + tt)
    const double Lf = Ls[0] * t[0] + Ls[1] * t[1] + Ls[2] * t[2];
    const double Ltt = -Lf * fct * fct * 0.5;
    for (int c = 0; c < 3; ++c) {
      Lt[c] += fct * Ls[c] + 2.0 * Ltt * t[c];
      Lem[c] += Lvm[c];
    }
    const double LE[3] = {hdt * Lem[0], hdt * Lem[1], hdt * Lem[2]};
    const double LB[3] = {hdt * Lt[0], hdt * Lt[1], hdt * Lt[2]};
    // ---- gather adjoint at the state before the step
    for (int c = 0; c < 3; ++c) {
      atomicAdd(&w.lE[c * nxn + c0], (1.0 - f0) * LE[c]);
      atomicAdd(&w.lE[c * nxn + c0 + 1], f0 * LE[c]);
      atomicAdd(&w.lBb[c * nxn + c0], (1.0 - f0) * LB[c]);
      atomicAdd(&w.lBb[c * nxn + c0 + 1], f0 * LB[c]);
      lf0 += LE[c] * Ed[c] + LB[c] * Bd[c];
    }
    w.lf[p] = (T)lf0;
    w.lv[p] = (T)Lvm[0];
    w.lv[cap + p] = (T)Lvm[1];
    w.lv[2 * cap + p] = (T)Lvm[2];
  }
  gu2 = warp_sum_d(gu2);
  gucr = warp_sum_d(gucr);
  if ((threadIdx.x & 31) == 0) {
    if (gucr != 0.0) atomicAdd(&w.grad[M], gucr);
    if (gu2 != 0.0) atomicAdd(&w.grad[M + 1], gu2);
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
  off[6] = o; o += 3 * al(3 * tsz * nxn) + 3 * al(3 * tsz * nx) + mom_bytes(nxn, tsz);
  off[7] = o; o += al(8 * 4 * (size_t)nxn);                                // fixed-point sums
  off[8] = o; o += al(8 * 8);                                              // counters
  off[9] = o;
  o += al(tsz * *cap) + al(3 * tsz * *cap);                                // lf, lv
  o += 14 * al(8 * 3 * (size_t)(nx + nxn));                                // field adjoints
  o += al(8 * (size_t)p->n_sub * 4 * 3 * nx);                              // stage inputs
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
  r.Es = (T*)take(3 * sizeof(T) * nxn);
  r.Bb = (T*)take(3 * sizeof(T) * nxn);
  r.B = (T*)take(3 * sizeof(T) * nx);
  r.Bs = (T*)take(3 * sizeof(T) * nx);
  r.Bsum = (T*)take(3 * sizeof(T) * nx);
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
  r.lE = (double*)tka(fb);
  r.lBb = (double*)tka(fb);
  r.lN = (double*)tka(fb);
  r.lU = (double*)tka(fb);
  r.lNm = (double*)tka(fb);
  r.lUm = (double*)tka(fb);
  r.lNr = (double*)tka(fb);
  r.lJ = (double*)tka(fb);
  r.P = (double*)tka(fb);
  r.g = (double*)tka(fb);
  r.lY = (double*)tka(fb);
  r.lsum = (double*)tka(fb);
  r.lend = (double*)tka(fb);
  r.Y = (double*)tka(8 * (size_t)w->p.n_sub * 4 * 3 * nx);
  r.grad = (double*)(w->base + w->o_params) + 2 * w->M;
  return r;
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

// RK4 substeps and the final Ohm of one step (the engine's kernels).
template <typename T>
void fields_step(fs_window* w, Win<T>& r) {
  const int nx = w->g.nx, nxn = w->g.nxn;
  const int gn = blocks(nxn), gc = blocks(nx);
  for (int sub = 0; sub < w->p.n_sub; ++sub) {
    for (int stage = 1; stage <= 4; ++stage) {
      const T* Bin = (stage == 1) ? r.B : r.Bs;
      k_ohm<T, 1><<<gn, kBlock, 0, w->st>>>(Bin, r.n, r.u, nullptr, r.Es, nullptr, nullptr, w->g,
                                             w->ph);
      k_faraday<T, 1><<<gc, kBlock, 0, w->st>>>(r.Es, r.B, r.Bs, r.Bsum, stage, w->g, w->ph);
    }
  }
  k_ohm<T, 1><<<gn, kBlock, 0, w->st>>>(r.B, r.n, r.u, nullptr, r.E, r.Bb, nullptr, w->g, w->ph);
}

// one forward step n; with tape index k >= 0 the step's inputs are taped
template <typename T>
void forward_step(fs_window* w, Win<T>& r, int n, int k) {
  const int np = w->np_at[n];
  Slots<T> tp{};
  uint8_t* ev = nullptr;
  if (k >= 0) {
    tp = tape_at<T>(w, k);
    ev = ev_at(w, k);
    cpy(tapeB_at<T>(w, k), r.B, 3 * sizeof(T) * w->g.nx, w->st);
  }
  if (np > 0)
    k_win_push<T><<<blocks(np), kBlock, 0, w->st>>>(r, tp, ev, w->g, w->ph, n, np);
  const int kinds = (w->ph.inject_thermal ? 1 : 0) + (w->ph.cr_enable ? 1 : 0);
  const int nadd = w->ninj[n] * kinds;
  if (nadd > 0)
    k_win_inject<T><<<blocks(nadd), kBlock, 0, w->st>>>(r, w->g, w->ph, n, np, w->ninj[n],
                                                        w->first_id[n]);
  const int np1 = w->np_at[n + 1];
  if (np1 > 0) k_win_deposit<T><<<blocks(np1), kBlock, 0, w->st>>>(r, w->g, w->ph, np1);
  T *tn = nullptr, *tu = nullptr, *tr = nullptr;
  if (k >= 0) mom_ptrs<T>(tapeM_at(w, k + 1), w->g.nxn, &tn, &tu, &tr);
  k_win_moments<T><<<blocks(w->g.nxn), kBlock, 0, w->st>>>(r, w->g, w->ph, tn, tu, tr);
  fields_step<T>(w, r);
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
  if (np0 > 0) k_win_deposit<T><<<blocks(np0), kBlock, 0, w->st>>>(r, w->g, w->ph, np0);
  k_win_moments<T><<<blocks(w->g.nxn), kBlock, 0, w->st>>>(r, w->g, w->ph, nullptr, nullptr,
                                                            nullptr);
  k_ohm<T, 1><<<blocks(w->g.nxn), kBlock, 0, w->st>>>(r.B, r.n, r.u, nullptr, r.E, r.Bb,
                                                       nullptr, w->g, w->ph);
  for (int n = 0; n < w->steps; ++n) {
    if (n % w->ckpt == 0) save_ckpt<T>(w, r, n / w->ckpt);
    forward_step<T>(w, r, n, -1);
  }
  double* dl = r.lsum;  // scratch for the loss
  cudaMemsetAsync(dl, 0, 8, w->st);
  k_win_loss<T><<<blocks(w->g.nx), kBlock, 0, w->st>>>(r.B, w->g, w->ph, w->loss_i0, w->p.dx,
                                                       dl, nullptr);
  unsigned long long c[5];
  if (cudaMemcpyAsync(loss, dl, 8, cudaMemcpyDeviceToHost, w->st) != cudaSuccess ||
      cudaMemcpyAsync(c, r.ctr, sizeof(c), cudaMemcpyDeviceToHost, w->st) != cudaSuccess ||
      cudaStreamSynchronize(w->st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return FS_ECUDA;
  for (int k = 0; k < 5; ++k) w->counts[k] = (long long)c[k];
  w->have_forward = true;
  return FS_OK;
}

// Adjoint of one step's RK4 substeps (n, u frozen at the tape moments n1,
// u1), from B^n: the stage inputs are recomputed with the engine's kernels;
// on entry r.lB is the adjoint of B^{n+1}, on exit that of B^n; the moment
// adjoints accumulate into r.lN, r.lU.
template <typename T>
void rk4_adjoint(fs_window* w, Win<T>& r, const T* Bn, const T* n1, const T* u1) {
  const int nx = w->g.nx, nxn = w->g.nxn;
  const int gn = blocks(nxn), gc = blocks(nx);
  const double h = w->ph.h, hh = w->ph.hh, h6 = w->ph.h6;
  const int ns = w->p.n_sub;
  auto Yp = [&](int sub, int s) { return r.Y + ((size_t)sub * 4 + s) * 3 * nx; };
  cpy(r.Bs, Bn, 3 * sizeof(T) * nx, w->st);
  T* Bsub = r.Bs;    // start of the substep (advanced in place by stage 4)
  T* Bst = r.Es;     // stage input (a node-sized buffer holds a centre field)
  T* Ksum = r.Bsum;
  T* Etmp = r.E;     // overwritten; E^n is recomputed after this
  for (int sub = 0; sub < ns; ++sub) {
    for (int stage = 1; stage <= 4; ++stage) {
      const T* Bin = (stage == 1) ? Bsub : Bst;
      k_win_to_double<T><<<blocks(3 * nx), kBlock, 0, w->st>>>(Yp(sub, stage - 1), Bin, 3 * nx);
      k_ohm<T, 1><<<gn, kBlock, 0, w->st>>>(Bin, n1, u1, nullptr, Etmp, nullptr, nullptr, w->g,
                                             w->ph);
      k_faraday<T, 1><<<gc, kBlock, 0, w->st>>>(Etmp, Bsub, Bst, Ksum, stage, w->g, w->ph);
    }
  }
  for (int sub = ns - 1; sub >= 0; --sub) {
    cpy(r.lend, r.lB, 8 * 3 * nx, w->st);
    cpy(r.lsum, r.lB, 8 * 3 * nx, w->st);  // lambda_start = lambda_end + sum lambda_Y
    // g4 = h6 lend; then g3 = 2 h6 lend + h lY4, g2 = 2 h6 lend + hh lY3,
    // g1 = h6 lend + hh lY2
    k_win_axpy<<<blocks(3 * nx), kBlock, 0, w->st>>>(r.g, r.lend, h6, nullptr, 0.0, 3 * nx);
    const double an[3] = {2 * h6, 2 * h6, h6};
    const double bn[3] = {h, hh, hh};
    for (int s = 3; s >= 0; --s) {
      k_win_ohm_adj<T><<<gn, kBlock, 0, w->st>>>(Yp(sub, s), n1, u1, r.g, nullptr, nullptr, r.P,
                                                  r.lN, r.lU, w->g, w->ph);
      const int q = 3 - s;
      k_win_curl_adj<<<gc, kBlock, 0, w->st>>>(r.P, r.lY, r.lsum, s > 0 ? r.g : nullptr, r.lend,
                                               s > 0 ? an[q] : 0.0, s > 0 ? bn[q] : 0.0, w->g,
                                               w->ph);
    }
    cpy(r.lB, r.lsum, 8 * 3 * nx, w->st);
  }
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
  k_win_loss<T><<<blocks(nx), kBlock, 0, w->st>>>(r.B, w->g, w->ph, w->loss_i0, w->p.dx,
                                                  nullptr, r.lB);
  k_win_axpy<<<blocks(3 * nx), kBlock, 0, w->st>>>(r.lB, r.lB, dloss, nullptr, 0.0, 3 * nx);
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
      // lN, lU: adjoint of the moments M^{n+1}, starting from what E^{n+1} added
      cpy(r.lN, r.lNm, fb, w->st);
      cpy(r.lU, r.lUm, fb, w->st);
      rk4_adjoint<T>(w, r, tapeB_at<T>(w, k), mn1, mu1);
      k_win_moments_adj<T><<<blocks(nxn), kBlock, 0, w->st>>>(mn1, mu1, mr1, r.lN, r.lU, r.lNr,
                                                              r.lJ, w->g, w->ph);
      // E^n, Bbar^n from B^n and M^n, as the forward had them
      k_ohm<T, 1><<<blocks(nxn), kBlock, 0, w->st>>>(tapeB_at<T>(w, k), mn0, mu0, nullptr, r.E,
                                                     r.Bb, nullptr, w->g, w->ph);
      cudaMemsetAsync(r.lE, 0, fb, w->st);
      cudaMemsetAsync(r.lBb, 0, fb, w->st);
      const int npa = w->np_at[n], npb = w->np_at[n + 1];
      if (npb > 0)
        k_win_particle_adj<T><<<blocks(npb), kBlock, 0, w->st>>>(
            r, tape_at<T>(w, k), tape_at<T>(w, k + 1), ev_at(w, k), w->g, w->ph, n, npa, npb, M);
      // Ohm at the start of the step: lB += ..., lNm, lUm = adjoint of M^n
      cudaMemsetAsync(r.lNm, 0, fb, w->st);
      cudaMemsetAsync(r.lUm, 0, fb, w->st);
      k_win_to_double<T><<<blocks(3 * nx), kBlock, 0, w->st>>>(r.Y, tapeB_at<T>(w, k), 3 * nx);
      k_win_ohm_adj<T><<<blocks(nxn), kBlock, 0, w->st>>>(r.Y, mn0, mu0, nullptr, r.lE, r.lBb,
                                                          r.P, r.lNm, r.lUm, w->g, w->ph);
      k_win_curl_adj<<<blocks(nx), kBlock, 0, w->st>>>(r.P, r.lY, r.lB, nullptr, nullptr, 0.0,
                                                       0.0, w->g, w->ph);
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
  if (!bytes) return FS_EINVAL;
  Geo g;
  Phys ph;
  int cap;
  size_t off[11];
  return window_sizes(p, steps, ckpt_every, n_init, n_modes, &g, &ph, &cap, bytes, off);
}

int fs_window_init(const fs_params* p, int steps, int ckpt_every, long long n_init,
                   const double* x_init, const double* v_init, int n_modes,
                   const double* mode_phase, int loss_i0, void* dev_buf, size_t bytes,
                   void* cuda_stream, fs_window** out) {
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
  bool ok = cudaMemcpyAsync(c0.slots, host.data(), host.size(), cudaMemcpyHostToDevice, w->st) ==
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
}

int fs_window_forward(fs_window* w, const double* theta, double* loss) {
  if (!w || !theta || !loss) return FS_EINVAL;
  return w->tsz == 8 ? do_forward<double>(w, theta, loss) : do_forward<float>(w, theta, loss);
}

int fs_window_backward(fs_window* w, double dloss, double* grad) {
  if (!w || !grad) return FS_EINVAL;
  return w->tsz == 8 ? do_backward<double>(w, dloss, grad) : do_backward<float>(w, dloss, grad);
}

int fs_window_counts(fs_window* w, long long* out5) {
  if (!w || !out5) return FS_EINVAL;
  for (int k = 0; k < 5; ++k) out5[k] = w->counts[k];
  return FS_OK;
}

int fs_window_destroy(fs_window* w) {
  delete w;
  return FS_OK;
}

}  // extern "C"
