/*
 * fs_oracle.c -- TEST INFRASTRUCTURE ONLY (see fs_oracle.h).
 *
 * A plain, slow, single-threaded FP64 hybrid particle-in-cell simulation of
 * the faux-shock box of Simon et al. (Sec. 2). Kinetic ions, massless
 * isothermal electron fluid (Sec. 2: "fully kinetic ions and a
 * charge-neutralizing electron fluid"), a faux-shock wall at x = 0 that lets
 * particles pass or returns them with the probability of Eq. 1, an open far
 * wall with continuous plasma inflow (Sec. 2), periodic transverse direction.
 *
 * The paper states no numerics for the host hybrid code; the step below is
 * the textbook scheme this project adopts (CIC gather, non-relativistic Boris
 * push, cell sort, CIC deposit, RK4 Ohm + Faraday). Every arithmetic
 * expression is written in one fixed order, with fused multiply-adds (C99
 * fma(), one IEEE-754 rounding) where the scheme says so and no other
 * contraction (-ffp-contract=off), so that a GPU implementation that writes
 * the same expressions in the same order reproduces every FP64 bit.
 *
 * Particle state per macroparticle: integer cell (i, j), in-cell offset
 * (fx, fy) in [0, 1), velocity (vx, vy, vz) at the half step, and a 32-bit
 * id word: bits 0..29 particle number, bit 30 cosmic-ray species, bit 31 set
 * once the faux shock has returned the particle.
 */
#include "fs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ID_MASK 0x3FFFFFFFu
#define ID_CR 0x40000000u
#define ID_RETURNED 0x80000000u

/* Philox counter "purpose" words: which random draw of a particle-step */
#define PURPOSE_INIT_A 1u
#define PURPOSE_INIT_B 2u
#define PURPOSE_FS 3u
#define PURPOSE_INJ_A 4u
#define PURPOSE_INJ_B 5u
#define PURPOSE_INJ_CR 6u

/* largest double below 1: offsets stay in [0, 1) */
#define OFFMAX 0x1.fffffffffffffp-1
/* deposit fixed point: each contribution is rounded to a multiple of 2^-40 */
#define FP_SCALE 0x1p40
#define FP_UNSCALE 0x1p-40
/* adding 1.5 * 2^52 rounds a double of magnitude below 2^51 to an integer */
#define ROUND_MAGIC 0x1.8p52
#define PI_DEC 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of the     */
/* two-multiplier S-box with a Weyl-sequence key schedule.                   */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                      uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform on (0, 1): midpoint of the k-th of 2^32 equal bins (exact) */
double or_u01(uint32_t k) { return ((double)k + 0.5) * 0x1p-32; }

static void draw4(uint64_t seed, uint32_t pid, long long step,
                  uint32_t purpose, uint32_t out[4]) {
  uint32_t ctr[4] = {pid, (uint32_t)step, purpose, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm by argument reduction to [sqrt(1/2), sqrt(2)) and the   */
/* series log m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), s=(m-1)/(m+1).   */
/* Coefficients are 1/(2k+1) rounded to nearest; ln 2 is split hi + lo with */
/* a 32-bit hi part so that e * hi is exact.                                 */
/* ------------------------------------------------------------------------ */
double or_log(double x) {
  int e;
  double m = frexp(x, &e); /* x = m 2^e, m in [0.5, 1) */
  m = m * 2.0;
  e = e - 1;
  if (m > 0x1.6a09e667f3bcdp+0) { /* sqrt(2) */
    m = m * 0.5;
    e = e + 1;
  }
  double s = (m - 1.0) / (m + 1.0);
  double z = s * s;
  double p = 0x1.642c8590b2164p-5; /* 1/23 */
  p = p * z + 0x1.8618618618618p-5; /* 1/21 */
  p = p * z + 0x1.af286bca1af28p-5; /* 1/19 */
  p = p * z + 0x1.e1e1e1e1e1e1ep-5; /* 1/17 */
  p = p * z + 0x1.1111111111111p-4; /* 1/15 */
  p = p * z + 0x1.3b13b13b13b14p-4; /* 1/13 */
  p = p * z + 0x1.745d1745d1746p-4; /* 1/11 */
  p = p * z + 0x1.c71c71c71c71cp-4; /* 1/9 */
  p = p * z + 0x1.2492492492492p-3; /* 1/7 */
  p = p * z + 0x1.999999999999ap-3; /* 1/5 */
  p = p * z + 0x1.5555555555555p-2; /* 1/3 */
  p = p * z + 1.0;
  double lm = (2.0 * s) * p;
  double de = (double)e;
  return de * 0x1.62e42fee00000p-1 + (lm + de * 0x1.a39ef35793c76p-33);
}

/* ------------------------------------------------------------------------ */
/* (cos 2 pi u, sin 2 pi u): quadrant from t = 4u, remainder angle           */
/* r = (t - q) pi/2 in [-pi/4, pi/4], Taylor series of sin and cos to r^19.  */
/* ------------------------------------------------------------------------ */
void or_sincos2pi(double u, double* cout, double* sout) {
  double t = 4.0 * u;
  double q = floor(t + 0.5);
  double d = t - q;
  double r = d * 0x1.921fb54442d18p+0; /* pi/2 */
  double z = r * r;
  double ps = -0x1.2f49b46814157p-57; /* -1/19! */
  ps = ps * z + 0x1.952c77030ad4ap-49; /* 1/17! */
  ps = ps * z - 0x1.ae7f3e733b81fp-41; /* 1/15! */
  ps = ps * z + 0x1.6124613a86d09p-33; /* 1/13! */
  ps = ps * z - 0x1.ae64567f544e4p-26; /* 1/11! */
  ps = ps * z + 0x1.71de3a556c734p-19; /* 1/9! */
  ps = ps * z - 0x1.a01a01a01a01ap-13; /* 1/7! */
  ps = ps * z + 0x1.1111111111111p-7;  /* 1/5! */
  ps = ps * z - 0x1.5555555555555p-3;  /* 1/3! */
  double sr = r + (r * z) * ps;
  double pc = -0x1.6827863b97d97p-53; /* -1/18! */
  pc = pc * z + 0x1.ae7f3e733b81fp-45; /* 1/16! */
  pc = pc * z - 0x1.93974a8c07c9dp-37; /* 1/14! */
  pc = pc * z + 0x1.1eed8eff8d898p-29; /* 1/12! */
  pc = pc * z - 0x1.27e4fb7789f5cp-22; /* 1/10! */
  pc = pc * z + 0x1.a01a01a01a01ap-16; /* 1/8! */
  pc = pc * z - 0x1.6c16c16c16c17p-10; /* 1/6! */
  pc = pc * z + 0x1.5555555555555p-5;  /* 1/4! */
  pc = pc * z - 0.5;                   /* 1/2! */
  double cr = 1.0 + z * pc;
  int iq = ((int)q) & 3;
  double c, s;
  if (iq == 0) { c = cr; s = sr; }
  else if (iq == 1) { c = -sr; s = cr; }
  else if (iq == 2) { c = -cr; s = -sr; }
  else { c = sr; s = -cr; }
  *cout = c;
  *sout = s;
}

/* Box-Muller: two independent standard normals from two uniforms */
static void gauss2(double u1, double u2, double* g0, double* g1) {
  double rad = sqrt(-2.0 * or_log(u1));
  double c, s;
  or_sincos2pi(u2, &c, &s);
  *g0 = rad * c;
  *g1 = rad * s;
}

/* ------------------------------------------------------------------------ */
/* Non-relativistic Boris rotation (dv/dt = E + v x B, q/m = 1):            */
/* half electric kick, magnetic rotation with t = B dt/2, s = 2t/(1+t.t),   */
/* second half kick.                                                         */
/* ------------------------------------------------------------------------ */
static void boris(double* v, const double* E, const double* B, double hdt,
                  double c2inv) {
  double emx = hdt * E[0], emy = hdt * E[1], emz = hdt * E[2];
  double vmx = v[0] + emx, vmy = v[1] + emy, vmz = v[2] + emz;
  /* relativistic ions (v holds u = gamma v): the rotation uses
     t = B dt / (2 gamma-), gamma- from the half-kicked u */
  double hg = hdt;
  if (c2inv > 0.0) {
    double uu = fma(vmz, vmz, fma(vmy, vmy, vmx * vmx));
    hg = hdt / sqrt(1.0 + uu * c2inv);
  }
  double tx = hg * B[0], ty = hg * B[1], tz = hg * B[2];
  double tt = fma(tz, tz, fma(ty, ty, tx * tx));
  double f = 2.0 / (1.0 + tt);
  double sx = f * tx, sy = f * ty, sz = f * tz;
  /* v' = v- + v- x t, v+ = v- + v' x s, each component as two fused steps */
  double px = fma(vmy, tz, fma(-vmz, ty, vmx));
  double py = fma(vmz, tx, fma(-vmx, tz, vmy));
  double pz = fma(vmx, ty, fma(-vmy, tx, vmz));
  double qx = fma(py, sz, fma(-pz, sy, vmx));
  double qy = fma(pz, sx, fma(-px, sz, vmy));
  double qz = fma(px, sy, fma(-py, sx, vmz));
  v[0] = qx + emx;
  v[1] = qy + emy;
  v[2] = qz + emz;
}

void or_boris(double* v, const double* E, const double* B, double dt) {
  boris(v, E, B, 0.5 * dt, 0.0);
}

void or_boris_rel(double* u, const double* E, const double* B, double dt,
                  double c_light) {
  boris(u, E, B, 0.5 * dt, c_light > 0.0 ? 1.0 / (c_light * c_light) : 0.0);
}

/* ------------------------------------------------------------------------ */
/* Faux-shock pass/return decision and returned velocity (Sec. 2, Eq. 1).   */
/* Returns 1 and overwrites v when the particle is returned, 0 when it     */
/* passes. The return probability is Eq. 1 with the particle speed in the   */
/* frame chosen by fs_speed_frame (the shock frame as the paper states it). */
/* A returned particle keeps its downstream-frame speed |v'| (v' = v + u2 x,*/
/* the downstream flows at -u2 x in the shock frame); its new direction is */
/* drawn isotropic in the downstream frame, weighted by the flux of such    */
/* particles through the shock (pdf of mu' proportional to mu' - u2/|v'|).  */
/* ------------------------------------------------------------------------ */
static int fs_rule_impl(double u2, int frame, uint64_t seed, double* v,
                        uint32_t pid, long long step, double* mu_out) {
  double vx = v[0], vy = v[1], vz = v[2];
  double sp = sqrt((vx * vx + vy * vy) + vz * vz);
  double wx = vx + u2;
  double w = sqrt((wx * wx + vy * vy) + vz * vz);
  double vp = (frame == OR_FRAME_SHOCK) ? sp : w;
  double prob = 0.0;
  if (vp > u2) {
    double a = u2 / vp;
    double q = (1.0 - a) / (1.0 + a);
    prob = q * q;
  }
  uint32_t r[4];
  draw4(seed, pid, step, PURPOSE_FS, r);
  double U0 = or_u01(r[0]), U1 = or_u01(r[1]), U2 = or_u01(r[2]);
  if (!(U0 < prob && w > u2)) return 0;
  double a = u2 / w;
  double mu = a + (1.0 - a) * sqrt(U1);
  double sn = sqrt(1.0 - mu * mu);
  double c, s;
  or_sincos2pi(U2, &c, &s);
  double ws = w * sn;
  v[0] = w * mu - u2;
  v[1] = ws * c;
  v[2] = ws * s;
  if (mu_out) *mu_out = mu;
  return 1;
}

static double param_u2(const or_params* p) {
  return p->u2 > 0.0 ? p->u2 : p->mach_a / p->r_comp;
}

int or_fs_rule(const or_params* p, double* v, uint32_t pid, long long step,
               double* mu_out) {
  return fs_rule_impl(param_u2(p), p->fs_speed_frame, p->seed, v, pid, step,
                      mu_out);
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                          */
/* ------------------------------------------------------------------------ */
struct or_sim {
  or_params p;
  int nxn;            /* node columns: nx + 1 (faux-shock box) or nx */
  double dtdx, dtdy, hdt, hdx, hdy, idx, h, hh, h6, te, vth, w_th, w_cr;
  double u2, u_cr, b0x, b0y, b0z, cellvol, rate;
  double c2inv;      /* 1 / c^2, 0 for non-relativistic ions */
  double p_iso_v;    /* CR injection speed: p_iso / gamma(p_iso) */
  double* spec_e;    /* momentum-spectrum bin edges [spec_np + 1] */
  /* particles (SoA) */
  long long np, cap;
  int32_t *ci, *cj;
  double *fx, *fy, *vx, *vy, *vz;
  uint32_t* id;
  /* grid */
  double* B;      /* centres [ny][nx][3] */
  double *E, *Bb; /* nodes [ny][nxn][3] */
  double *n, *J, *u; /* nodes: n [ny][nxn]; J, u [ny][nxn][3] */
  int64_t *qn, *qj; /* fixed-point accumulators */
  double* acc;        /* injection accumulators [ny] */
  /* stage buffers */
  double *Bs, *Bsum, *K, *Es;
  /* counters */
  long long step, next_id;
  long long incident, transmitted, reflected, escaped, injected;
  double fs_energy, injected_energy, removed_energy;
  double push_work;  /* cumulative work of E on the ions in the pushes */
  int err;
};

static void reserve(or_sim* s, long long need) {
  if (need <= s->cap) return;
  long long nc = s->cap ? s->cap : 1024;
  while (nc < need) nc *= 2;
  s->ci = (int32_t*)realloc(s->ci, nc * sizeof(int32_t));
  s->cj = (int32_t*)realloc(s->cj, nc * sizeof(int32_t));
  s->fx = (double*)realloc(s->fx, nc * sizeof(double));
  s->fy = (double*)realloc(s->fy, nc * sizeof(double));
  s->vx = (double*)realloc(s->vx, nc * sizeof(double));
  s->vy = (double*)realloc(s->vy, nc * sizeof(double));
  s->vz = (double*)realloc(s->vz, nc * sizeof(double));
  s->id = (uint32_t*)realloc(s->id, nc * sizeof(uint32_t));
  s->cap = nc;
}

static void push_particle(or_sim* s, int32_t i, int32_t j, double fx,
                          double fy, double vx, double vy, double vz,
                          uint32_t id) {
  reserve(s, s->np + 1);
  long long k = s->np++;
  s->ci[k] = i; s->cj[k] = j; s->fx[k] = fx; s->fy[k] = fy;
  s->vx[k] = vx; s->vy[k] = vy; s->vz[k] = vz; s->id[k] = id;
}

static double weight_of(const or_sim* s, uint32_t id) {
  return (id & ID_CR) ? s->w_cr : s->w_th;
}

/* 1/gamma of a stored u (momentum per mass): 1/sqrt(1 + u.u/c^2); 1 for
   non-relativistic ions */
static double inv_gamma_u(const or_sim* s, double ux, double uy, double uz) {
  if (s->c2inv == 0.0) return 1.0;
  double uu = fma(uz, uz, fma(uy, uy, ux * ux));
  return 1.0 / sqrt(1.0 + uu * s->c2inv);
}
/* gamma of a velocity: 1/sqrt(1 - v.v/c^2) */
static double gamma_v(const or_sim* s, double vx, double vy, double vz) {
  if (s->c2inv == 0.0) return 1.0;
  double vv = fma(vz, vz, fma(vy, vy, vx * vx));
  return 1.0 / sqrt(1.0 - vv * s->c2inv);
}

static int wrapj(const or_sim* s, int j) {
  int ny = s->p.ny;
  j %= ny;
  if (j < 0) j += ny;
  return j;
}

/* centre column index with the x boundary rule: zero-gradient ghosts at the
   walls of the faux-shock box, wrap-around in a periodic box */
static int cx_of(const or_sim* s, int i) {
  int nx = s->p.nx;
  if (s->p.bc_x == OR_BC_PERIODIC) {
    i %= nx;
    if (i < 0) i += nx;
    return i;
  }
  if (i < 0) return 0;
  if (i >= nx) return nx - 1;
  return i;
}

/* node column index for the density gradient: mirror about the wall nodes
   (n(-1) = n(1), n(nx+1) = n(nx-1)) in the faux-shock box, wrap otherwise */
static int nx_of(const or_sim* s, int i) {
  int nx = s->p.nx;
  if (s->p.bc_x == OR_BC_PERIODIC) {
    i %= nx;
    if (i < 0) i += nx;
    return i;
  }
  if (i < 0) return -i;
  if (i > nx) return 2 * nx - i;
  return i;
}

/* node column reached from a cell: i or i + 1 (wraps in a periodic box) */
static int node_col(const or_sim* s, int i) {
  if (s->p.bc_x == OR_BC_PERIODIC && i >= s->p.nx) return i - s->p.nx;
  return i;
}

static long long cidx(const or_sim* s, int i, int j) {
  return (long long)j * s->p.nx + i;
}
static long long nidx(const or_sim* s, int i, int j) {
  return (long long)j * s->nxn + i;
}

/* ------------------------------------------------------------------------ */
/* CIC gather of E and B-bar at a particle position (weights (1-f, f) per  */
/* dimension, summed in the order 00, 10, 01, 11).                          */
/* ------------------------------------------------------------------------ */
static void gather(const or_sim* s, int i, int j, double fx, double fy,
                   double* Ep, double* Bp) {
  int i1 = node_col(s, i + 1);
  if (s->p.dim == 1) {
    double g0 = 1.0 - fx;
    const double* E0 = s->E + 3 * nidx(s, i, 0);
    const double* E1 = s->E + 3 * nidx(s, i1, 0);
    const double* B0 = s->Bb + 3 * nidx(s, i, 0);
    const double* B1 = s->Bb + 3 * nidx(s, i1, 0);
    for (int c = 0; c < 3; ++c) {
      Ep[c] = fma(fx, E1[c], g0 * E0[c]);
      Bp[c] = fma(fx, B1[c], g0 * B0[c]);
    }
    return;
  }
  int j1 = wrapj(s, j + 1);
  double gx0 = 1.0 - fx, gy0 = 1.0 - fy;
  double w00 = gx0 * gy0, w10 = fx * gy0, w01 = gx0 * fy, w11 = fx * fy;
  long long n00 = 3 * nidx(s, i, j), n10 = 3 * nidx(s, i1, j);
  long long n01 = 3 * nidx(s, i, j1), n11 = 3 * nidx(s, i1, j1);
  for (int c = 0; c < 3; ++c) {
    Ep[c] = fma(w11, s->E[n11 + c],
                fma(w01, s->E[n01 + c], fma(w10, s->E[n10 + c], w00 * s->E[n00 + c])));
    Bp[c] = fma(w11, s->Bb[n11 + c],
                fma(w01, s->Bb[n01 + c], fma(w10, s->Bb[n10 + c], w00 * s->Bb[n00 + c])));
  }
}

void or_gather(const or_sim* s, int i, int j, double fx, double fy,
               double* out6) {
  gather(s, i, j, fx, fy, out6, out6 + 3);
}

/* ------------------------------------------------------------------------ */
/* Moments: CIC deposit of n and J = n u_i at the new positions with the    */
/* half-step velocities, each contribution rounded to the nearest multiple  */
/* of 2^-40 and summed in int64, so that the node sums do not depend on the */
/* order of the particles. The weight is carried scaled by 2^40 (exact), the*/
/* current terms are rounded from the exact product (one fused rounding).   */
/* Then the wall half-volume correction, the density floor and u_i = J / n. */
/* ------------------------------------------------------------------------ */
static int64_t to_fixed(double scaled) {
  return (int64_t)((scaled + ROUND_MAGIC) - ROUND_MAGIC);
}
static int64_t to_fixed_prod(double a, double b) {
  return (int64_t)(fma(a, b, ROUND_MAGIC) - ROUND_MAGIC);
}

/* cns: the particle weight times the corner weight, scaled by 2^40 */
static void dep1(or_sim* s, long long node, double cns, double vx, double vy,
                 double vz) {
  s->qn[node] += to_fixed(cns);
  s->qj[3 * node + 0] += to_fixed_prod(cns, vx);
  s->qj[3 * node + 1] += to_fixed_prod(cns, vy);
  s->qj[3 * node + 2] += to_fixed_prod(cns, vz);
}

static void deposit_and_finish(or_sim* s) {
  long long nn = (long long)s->nxn * s->p.ny;
  memset(s->qn, 0, nn * sizeof(int64_t));
  memset(s->qj, 0, 3 * nn * sizeof(int64_t));
  for (long long k = 0; k < s->np; ++k) {
    double wp = weight_of(s, s->id[k]) * FP_SCALE;
    int i = s->ci[k], j = s->cj[k];
    int i1 = node_col(s, i + 1);
    double fx = s->fx[k];
    double vx = s->vx[k], vy = s->vy[k], vz = s->vz[k];
    if (s->c2inv > 0.0) {  /* the current of relativistic ions uses v = u / gamma */
      double ig = inv_gamma_u(s, vx, vy, vz);
      vx = vx * ig; vy = vy * ig; vz = vz * ig;
    }
    if (s->p.dim == 1) {
      double g0 = 1.0 - fx;
      dep1(s, nidx(s, i, 0), wp * g0, vx, vy, vz);
      dep1(s, nidx(s, i1, 0), wp * fx, vx, vy, vz);
    } else {
      double fy = s->fy[k];
      int j1 = wrapj(s, j + 1);
      double gx0 = 1.0 - fx, gy0 = 1.0 - fy;
      double w00 = gx0 * gy0, w10 = fx * gy0, w01 = gx0 * fy, w11 = fx * fy;
      dep1(s, nidx(s, i, j), wp * w00, vx, vy, vz);
      dep1(s, nidx(s, i1, j), wp * w10, vx, vy, vz);
      dep1(s, nidx(s, i, j1), wp * w01, vx, vy, vz);
      dep1(s, nidx(s, i1, j1), wp * w11, vx, vy, vz);
    }
  }
  for (int j = 0; j < s->p.ny; ++j) {
    for (int i = 0; i < s->nxn; ++i) {
      long long q = nidx(s, i, j);
      double n = (double)s->qn[q] * FP_UNSCALE;
      double jx = (double)s->qj[3 * q + 0] * FP_UNSCALE;
      double jy = (double)s->qj[3 * q + 1] * FP_UNSCALE;
      double jz = (double)s->qj[3 * q + 2] * FP_UNSCALE;
      if (s->p.bc_x == OR_BC_FAUXSHOCK && (i == 0 || i == s->p.nx)) {
        /* a wall node owns half a cell of plasma volume */
        n = n * 2.0; jx = jx * 2.0; jy = jy * 2.0; jz = jz * 2.0;
      }
      s->J[3 * q + 0] = jx; s->J[3 * q + 1] = jy; s->J[3 * q + 2] = jz;
      if (n < s->p.n_floor) n = s->p.n_floor;
      s->n[q] = n;
      s->u[3 * q + 0] = jx / n;
      s->u[3 * q + 1] = jy / n;
      s->u[3 * q + 2] = jz / n;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Ohm's law at the nodes for a given centre field Bc (massless isothermal  */
/* electrons, quasi-neutral, J = curl B):                                    */
/*   E = -u_i x Bbar + ((curl B - j_ext x) x Bbar)/n - T_e grad n / n        */
/*       (+ eta curl B)                                                      */
/* Also returns Bbar (B averaged onto the nodes).                            */
/* ------------------------------------------------------------------------ */
static void ohm(const or_sim* s, const double* Bc, double* Eo, double* Bbo) {
  const int nx = s->p.nx, ny = s->p.ny;
  const double te = s->te, jcr = s->p.j_cr_ext, eta = s->p.eta;
  const int nlast = (s->p.bc_x == OR_BC_PERIODIC) ? nx - 1 : nx;
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i <= nlast; ++i) {
      double bbx, bby, bbz, cxv, cyv, czv, dnx, dny;
      if (s->p.dim == 1) {
        const double* Bm = Bc + 3 * cidx(s, cx_of(s, i - 1), 0);
        const double* Bp = Bc + 3 * cidx(s, cx_of(s, i), 0);
        bbx = 0.5 * (Bm[0] + Bp[0]);
        bby = 0.5 * (Bm[1] + Bp[1]);
        bbz = 0.5 * (Bm[2] + Bp[2]);
        double dby = (Bp[1] - Bm[1]) * s->idx;
        double dbz = (Bp[2] - Bm[2]) * s->idx;
        cxv = 0.0;
        cyv = -dbz;
        czv = dby;
        dnx = (s->n[nidx(s, nx_of(s, i + 1), 0)] -
               s->n[nidx(s, nx_of(s, i - 1), 0)]) * s->hdx;
        dny = 0.0;
      } else {
        int im = cx_of(s, i - 1), ip = cx_of(s, i);
        int jm = wrapj(s, j - 1), jp = j;
        const double* Bmm = Bc + 3 * cidx(s, im, jm);
        const double* Bpm = Bc + 3 * cidx(s, ip, jm);
        const double* Bmp = Bc + 3 * cidx(s, im, jp);
        const double* Bpp = Bc + 3 * cidx(s, ip, jp);
        bbx = 0.25 * ((Bmm[0] + Bpm[0]) + (Bmp[0] + Bpp[0]));
        bby = 0.25 * ((Bmm[1] + Bpm[1]) + (Bmp[1] + Bpp[1]));
        bbz = 0.25 * ((Bmm[2] + Bpm[2]) + (Bmp[2] + Bpp[2]));
        double dxby = ((Bpp[1] + Bpm[1]) - (Bmp[1] + Bmm[1])) * s->hdx;
        double dxbz = ((Bpp[2] + Bpm[2]) - (Bmp[2] + Bmm[2])) * s->hdx;
        double dybx = ((Bpp[0] + Bmp[0]) - (Bpm[0] + Bmm[0])) * s->hdy;
        double dybz = ((Bpp[2] + Bmp[2]) - (Bpm[2] + Bmm[2])) * s->hdy;
        cxv = dybz;
        cyv = -dxbz;
        czv = dxby - dybx;
        dnx = (s->n[nidx(s, nx_of(s, i + 1), j)] -
               s->n[nidx(s, nx_of(s, i - 1), j)]) * s->hdx;
        dny = (s->n[nidx(s, i, wrapj(s, j + 1))] -
               s->n[nidx(s, i, wrapj(s, j - 1))]) * s->hdy;
      }
      long long q = nidx(s, i, j);
      double n = s->n[q];
      double ux = s->u[3 * q + 0], uy = s->u[3 * q + 1], uz = s->u[3 * q + 2];
      double ax = cxv - jcr, ay = cyv, az = czv;
      double inv_n = 1.0 / n;
      /* (a x Bbar) and (u x Bbar), each component as one fused step */
      double cax = fma(ay, bbz, -(az * bby));
      double cay = fma(az, bbx, -(ax * bbz));
      double caz = fma(ax, bby, -(ay * bbx));
      double cux = fma(uy, bbz, -(uz * bby));
      double cuy = fma(uz, bbx, -(ux * bbz));
      double cuz = fma(ux, bby, -(uy * bbx));
      double ex = fma(-(te * dnx), inv_n, fma(cax, inv_n, -cux));
      double ey = fma(-(te * dny), inv_n, fma(cay, inv_n, -cuy));
      double ez = fma(caz, inv_n, -cuz);
      if (eta != 0.0) {
        ex = ex + eta * cxv;
        ey = ey + eta * cyv;
        ez = ez + eta * czv;
      }
      Eo[3 * q + 0] = ex; Eo[3 * q + 1] = ey; Eo[3 * q + 2] = ez;
      if (Bbo) {
        Bbo[3 * q + 0] = bbx; Bbo[3 * q + 1] = bby; Bbo[3 * q + 2] = bbz;
      }
    }
    if (s->p.bc_x == OR_BC_PERIODIC) {
      /* no separate node nx in a periodic box */
    }
  }
}

/* Faraday at the centres: dB/dt = -curl E, curl from the four corner nodes */
static void faraday(const or_sim* s, const double* En, double* K) {
  const int nx = s->p.nx, ny = s->p.ny;
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      long long c = cidx(s, i, j);
      int i1 = node_col(s, i + 1);
      if (s->p.dim == 1) {
        const double* E0 = En + 3 * nidx(s, i, 0);
        const double* E1 = En + 3 * nidx(s, i1, 0);
        double dxey = (E1[1] - E0[1]) * s->idx;
        double dxez = (E1[2] - E0[2]) * s->idx;
        K[3 * c + 0] = 0.0;
        K[3 * c + 1] = dxez;
        K[3 * c + 2] = -dxey;
      } else {
        int j1 = wrapj(s, j + 1);
        const double* E00 = En + 3 * nidx(s, i, j);
        const double* E10 = En + 3 * nidx(s, i1, j);
        const double* E01 = En + 3 * nidx(s, i, j1);
        const double* E11 = En + 3 * nidx(s, i1, j1);
        double dxey = ((E10[1] + E11[1]) - (E00[1] + E01[1])) * s->hdx;
        double dxez = ((E10[2] + E11[2]) - (E00[2] + E01[2])) * s->hdx;
        double dyex = ((E01[0] + E11[0]) - (E00[0] + E10[0])) * s->hdy;
        double dyez = ((E01[2] + E11[2]) - (E00[2] + E10[2])) * s->hdy;
        K[3 * c + 0] = -dyez;
        K[3 * c + 1] = dxez;
        K[3 * c + 2] = dyex - dxey;
      }
    }
  }
}

/* Classical RK4 for dB/dt = -curl E(B), moments frozen, n_sub substeps;
   then E and Bbar at the nodes for the next gather. */
static void advance_fields(or_sim* s) {
  const long long nc3 = 3LL * s->p.nx * s->p.ny;
  for (int sub = 0; sub < s->p.n_sub; ++sub) {
    /* stage 1 */
    ohm(s, s->B, s->Es, NULL);
    faraday(s, s->Es, s->K);
    for (long long k = 0; k < nc3; ++k) {
      s->Bsum[k] = s->K[k];
      s->Bs[k] = fma(s->hh, s->K[k], s->B[k]);
    }
    /* stage 2 */
    ohm(s, s->Bs, s->Es, NULL);
    faraday(s, s->Es, s->K);
    for (long long k = 0; k < nc3; ++k) {
      s->Bsum[k] = fma(2.0, s->K[k], s->Bsum[k]);
      s->Bs[k] = fma(s->hh, s->K[k], s->B[k]);
    }
    /* stage 3 */
    ohm(s, s->Bs, s->Es, NULL);
    faraday(s, s->Es, s->K);
    for (long long k = 0; k < nc3; ++k) {
      s->Bsum[k] = fma(2.0, s->K[k], s->Bsum[k]);
      s->Bs[k] = fma(s->h, s->K[k], s->B[k]);
    }
    /* stage 4 */
    ohm(s, s->Bs, s->Es, NULL);
    faraday(s, s->Es, s->K);
    for (long long k = 0; k < nc3; ++k) {
      s->Bsum[k] = s->Bsum[k] + s->K[k];
      s->B[k] = fma(s->h6, s->Bsum[k], s->B[k]);
    }
  }
  ohm(s, s->B, s->E, s->Bb);
}

/* ------------------------------------------------------------------------ */
/* Stable counting sort of the particles by linear cell j * nx + i.         */
/* ------------------------------------------------------------------------ */
static void sort_by_cell(or_sim* s) {
  long long ncell = (long long)s->p.nx * s->p.ny;
  long long* start = (long long*)calloc(ncell + 1, sizeof(long long));
  for (long long k = 0; k < s->np; ++k)
    start[cidx(s, s->ci[k], s->cj[k]) + 1]++;
  for (long long c = 0; c < ncell; ++c) start[c + 1] += start[c];
  long long np = s->np;
  int32_t* ci = (int32_t*)malloc(np * sizeof(int32_t) + 1);
  int32_t* cj = (int32_t*)malloc(np * sizeof(int32_t) + 1);
  double* fx = (double*)malloc(np * sizeof(double) + 1);
  double* fy = (double*)malloc(np * sizeof(double) + 1);
  double* vx = (double*)malloc(np * sizeof(double) + 1);
  double* vy = (double*)malloc(np * sizeof(double) + 1);
  double* vz = (double*)malloc(np * sizeof(double) + 1);
  uint32_t* id = (uint32_t*)malloc(np * sizeof(uint32_t) + 1);
  for (long long k = 0; k < np; ++k) {
    long long d = start[cidx(s, s->ci[k], s->cj[k])]++;
    ci[d] = s->ci[k]; cj[d] = s->cj[k]; fx[d] = s->fx[k]; fy[d] = s->fy[k];
    vx[d] = s->vx[k]; vy[d] = s->vy[k]; vz[d] = s->vz[k]; id[d] = s->id[k];
  }
  memcpy(s->ci, ci, np * sizeof(int32_t));
  memcpy(s->cj, cj, np * sizeof(int32_t));
  memcpy(s->fx, fx, np * sizeof(double));
  memcpy(s->fy, fy, np * sizeof(double));
  memcpy(s->vx, vx, np * sizeof(double));
  memcpy(s->vy, vy, np * sizeof(double));
  memcpy(s->vz, vz, np * sizeof(double));
  memcpy(s->id, id, np * sizeof(uint32_t));
  free(ci); free(cj); free(fx); free(fy); free(vx); free(vy); free(vz);
  free(id); free(start);
}

/* kinetic energy of a macroparticle: w v^2 / 2, or w (gamma - 1) c^2 =
   w u.u / (gamma + 1) for relativistic ions (u stored) */
static double kin(const or_sim* s, double wp, double vx, double vy,
                  double vz) {
  if (s->c2inv > 0.0) {
    double uu = fma(vz, vz, fma(vy, vy, vx * vx));
    double gamma = sqrt(1.0 + uu * s->c2inv);
    return (wp * (uu / (gamma + 1.0))) * s->cellvol;
  }
  return ((wp * 0.5) * ((vx * vx + vy * vy) + vz * vz)) * s->cellvol;
}

/* Work done by E on one macroparticle in a Boris step. The magnetic
   rotation keeps |u-| (u = v, or gamma v for relativistic ions), so
   |u_new|^2 - |u_old|^2 = dt E.(u_new + u_old) exactly, and the kinetic
   energy w (gamma - 1) c^2 (w u^2 / 2 without c) changes by
   w dt E.(u_new + u_old) / (gamma_new + gamma_old), gamma = 1 without c. */
static double push_work_of(const or_sim* s, double wp, const double* E,
                           const double* uo, const double* un) {
  double es = E[0] * (uo[0] + un[0]) + E[1] * (uo[1] + un[1]) +
              E[2] * (uo[2] + un[2]);
  double gsum = 2.0;
  if (s->c2inv > 0.0) {
    double uuo = uo[0] * uo[0] + uo[1] * uo[1] + uo[2] * uo[2];
    double uun = un[0] * un[0] + un[1] * un[1] + un[2] * un[2];
    gsum = sqrt(1.0 + uuo * s->c2inv) + sqrt(1.0 + uun * s->c2inv);
  }
  return ((wp * s->p.dt) * es / gsum) * s->cellvol;
}

/* ------------------------------------------------------------------------ */
/* Injection (Sec. 2): thermal plasma enters through x = L drifting at -u_sh*/
/* (a drifting Maxwellian); optionally cosmic rays enter at the faux shock  */
/* with speed p_iso, isotropic in the frame of the downstream flow, which   */
/* drifts at u_cr. Per transverse cell the number per step is the integer  */
/* part of an accumulator advanced by ppc u_sh dt / dx.                     */
/* ------------------------------------------------------------------------ */
static void inject(or_sim* s, long long step) {
  const int nx = s->p.nx;
  const double dtdx = s->dtdx;
  for (int j = 0; j < s->p.ny; ++j) {
    s->acc[j] = s->acc[j] + s->rate;
    double fl = floor(s->acc[j]);
    long long nnew = (long long)fl;
    s->acc[j] = s->acc[j] - fl;
    if (s->p.inject_thermal) {
      for (long long k = 0; k < nnew; ++k) {
        uint32_t pid = (uint32_t)s->next_id++;
        uint32_t ra[4], rb[4];
        draw4(s->p.seed, pid, step, PURPOSE_INJ_A, ra);
        draw4(s->p.seed, pid, step, PURPOSE_INJ_B, rb);
        double g0, g1, g2, g3;
        gauss2(or_u01(ra[0]), or_u01(ra[1]), &g0, &g1);
        gauss2(or_u01(ra[2]), or_u01(ra[3]), &g2, &g3);
        double vx = s->vth * g0 - s->p.mach_a;
        double vy = s->vth * g1;
        double vz = s->vth * g2;
        double X = (double)nx - (or_u01(rb[0]) * fabs(vx)) * dtdx;
        double ix = floor(X);
        int i = (int)ix;
        double fx = X - ix;
        if (i >= nx) { i = nx - 1; fx = OFFMAX; }
        if (i < 0) { i = 0; fx = 0.0; }
        if (fx >= 1.0) fx = OFFMAX;
        double fy = (s->p.dim == 2) ? or_u01(rb[1]) : 0.0;
        double gv = gamma_v(s, vx, vy, vz);
        vx = vx * gv; vy = vy * gv; vz = vz * gv;  /* stored as u */
        push_particle(s, i, j, fx, fy, vx, vy, vz, pid);
        s->injected++;
        s->injected_energy += kin(s, s->w_th, vx, vy, vz);
      }
    }
    if (s->p.cr_enable) {
      for (long long k = 0; k < nnew; ++k) {
        uint32_t pid = (uint32_t)s->next_id++;
        uint32_t rc[4];
        draw4(s->p.seed, pid, step, PURPOSE_INJ_CR, rc);
        /* speed p_iso / gamma(p_iso) in the downstream frame (p_iso without c) */
        double a = s->u_cr / s->p_iso_v;
        double mu = a + (1.0 - a) * sqrt(or_u01(rc[0]));
        double sn = sqrt(1.0 - mu * mu);
        double c, sv;
        or_sincos2pi(or_u01(rc[1]), &c, &sv);
        double ws = s->p_iso_v * sn;
        double vx = s->p_iso_v * mu - s->u_cr;
        double vy = ws * c;
        double vz = ws * sv;
        double X = (or_u01(rc[2]) * vx) * dtdx;
        double ix = floor(X);
        int i = (int)ix;
        double fx = X - ix;
        if (i >= nx) { i = nx - 1; fx = OFFMAX; }
        if (i < 0) { i = 0; fx = 0.0; }
        if (fx >= 1.0) fx = OFFMAX;
        double fy = (s->p.dim == 2) ? or_u01(rc[3]) : 0.0;
        double gv = gamma_v(s, vx, vy, vz);
        vx = vx * gv; vy = vy * gv; vz = vz * gv;  /* stored as u */
        push_particle(s, i, j, fx, fy, vx, vy, vz, pid | ID_CR);
        s->injected++;
        s->injected_energy += kin(s, s->w_cr, vx, vy, vz);
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* One particle step for every particle: gather, Boris, move, boundaries.   */
/* Removed particles are compacted out, survivors keep their order.         */
/* ------------------------------------------------------------------------ */
static void push_all(or_sim* s, long long step) {
  const int nx = s->p.nx, ny = s->p.ny;
  long long out = 0;
  for (long long k = 0; k < s->np; ++k) {
    int i = s->ci[k], j = s->cj[k];
    double fx = s->fx[k], fy = s->fy[k];
    double v[3] = {s->vx[k], s->vy[k], s->vz[k]};
    uint32_t id = s->id[k];
    double Ep[3], Bp[3];
    gather(s, i, j, fx, fy, Ep, Bp);
    const double vo[3] = {v[0], v[1], v[2]};
    boris(v, Ep, Bp, s->hdt, s->c2inv);
    s->push_work += push_work_of(s, weight_of(s, id), Ep, vo, v);
    /* the move uses the velocity (v = u / gamma for relativistic ions) */
    double ig = inv_gamma_u(s, v[0], v[1], v[2]);
    double vxm = (s->c2inv > 0.0) ? v[0] * ig : v[0];
    double vym = (s->c2inv > 0.0) ? v[1] * ig : v[1];
    /* move in x */
    double fxr = fma(vxm, s->dtdx, fx);
    double kx = floor(fxr);
    if (!(fabs(kx) < 1.0e9)) { s->err = 1; continue; }
    int inew = i + (int)kx;
    double fxn = fxr - kx;
    if (fxn >= 1.0) fxn = OFFMAX;
    /* move in y (periodic) */
    int jnew = j;
    double fyn = fy;
    if (s->p.dim == 2) {
      double fyr = fma(vym, s->dtdy, fy);
      double ky = floor(fyr);
      if (!(fabs(ky) < 1.0e9)) { s->err = 1; continue; }
      jnew = wrapj(s, j + (int)ky);
      fyn = fyr - ky;
      if (fyn >= 1.0) fyn = OFFMAX;
    }
    double wp = weight_of(s, id);
    if (s->p.bc_x == OR_BC_PERIODIC) {
      inew %= nx;
      if (inew < 0) inew += nx;
    } else if (inew >= nx) {
      /* open far wall: the particle escapes to upstream infinity */
      s->escaped++;
      s->removed_energy += kin(s, wp, v[0], v[1], v[2]);
      continue;
    } else if (inew < 0) {
      /* crossed the faux shock at x = 0 */
      int mode = (id & ID_CR) ? OR_FS_SHOCK : s->p.fs_mode_thermal;
      s->incident++;
      double e0 = kin(s, wp, v[0], v[1], v[2]);
      /* the rule acts on the velocity; a relativistic ion's u is
         converted to v and back */
      double vel[3] = {v[0], v[1], v[2]};
      if (s->c2inv > 0.0) { vel[0] = v[0] * ig; vel[1] = v[1] * ig; vel[2] = v[2] * ig; }
      if (mode == OR_FS_SHOCK &&
          fs_rule_impl(s->u2, s->p.fs_speed_frame, s->p.seed, vel,
                       id & ID_MASK, step, NULL)) {
        if (s->c2inv > 0.0) {
          double gv = gamma_v(s, vel[0], vel[1], vel[2]);
          v[0] = vel[0] * gv; v[1] = vel[1] * gv; v[2] = vel[2] * gv;
        } else {
          v[0] = vel[0]; v[1] = vel[1]; v[2] = vel[2];
        }
        s->reflected++;
        s->fs_energy += kin(s, wp, v[0], v[1], v[2]) - e0;
        /* re-place: the fraction g of the step spent beyond x = 0 is
           travelled again with the returned velocity */
        double Xo = (double)i + fx;
        double Xn = (double)i + fxr;
        double g = Xn / (Xn - Xo);
        double f = g * (vel[0] * s->dtdx);
        if (f < 0.0) f = 0.0;
        if (f >= 1.0) f = OFFMAX;
        inew = 0;
        fxn = f;
        id |= ID_RETURNED;
      } else {
        s->transmitted++;
        s->removed_energy += e0;
        continue;
      }
    }
    s->ci[out] = inew; s->cj[out] = jnew; s->fx[out] = fxn; s->fy[out] = fyn;
    s->vx[out] = v[0]; s->vy[out] = v[1]; s->vz[out] = v[2]; s->id[out] = id;
    (void)ny;
    ++out;
  }
  s->np = out;
}

int or_step(or_sim* s, int nsteps) {
  for (int it = 0; it < nsteps; ++it) {
    long long step = s->step;
    push_all(s, step);
    if (s->p.bc_x == OR_BC_FAUXSHOCK) inject(s, step);
    sort_by_cell(s);
    deposit_and_finish(s);
    advance_fields(s);
    s->step++;
  }
  return s->err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Set-up: derived constants, B0, the uniform drifting Maxwellian plasma    */
/* (ppc per cell, positions uniform in the cell), first deposit and E^0.    */
/* ------------------------------------------------------------------------ */
or_sim* or_create(const or_params* p) {
  if (p->dim != 1 && p->dim != 2) return NULL;
  if (p->nx < 2 || p->ny < 1 || (p->dim == 1 && p->ny != 1)) return NULL;
  if (p->ppc < 1 || p->n_sub < 1 || !(p->dt > 0) || !(p->dx > 0)) return NULL;
  or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
  s->p = *p;
  const int nx = p->nx, ny = p->ny;
  s->nxn = (p->bc_x == OR_BC_PERIODIC) ? nx : nx + 1;
  s->dtdx = p->dt / p->dx;
  s->dtdy = (p->dim == 2) ? p->dt / p->dy : 0.0;
  s->hdt = 0.5 * p->dt;
  s->hdx = 0.5 / p->dx;
  s->hdy = (p->dim == 2) ? 0.5 / p->dy : 0.0;
  s->idx = 1.0 / p->dx;
  s->h = p->dt / (double)p->n_sub;
  s->hh = 0.5 * s->h;
  s->h6 = s->h / 6.0;
  s->te = 0.5 * p->beta_e;
  s->vth = sqrt(0.5 * p->beta_i);
  s->w_th = 1.0 / (double)p->ppc;
  s->w_cr = p->n_cr_ratio / (double)p->ppc;
  s->u2 = param_u2(p);
  s->u_cr = p->u_cr > 0.0 ? p->u_cr : s->u2;
  double th = p->theta_bn_deg * (PI_DEC / 180.0);
  s->b0x = cos(th);
  s->b0y = sin(th);
  s->b0z = 0.0;
  s->cellvol = (p->dim == 2) ? p->dx * p->dy : p->dx;
  s->c2inv = (p->c_light > 0.0) ? 1.0 / (p->c_light * p->c_light) : 0.0;
  s->p_iso_v = (s->c2inv > 0.0) ? p->p_iso / sqrt(1.0 + (p->p_iso * p->p_iso) * s->c2inv)
                                : p->p_iso;
  if (p->spec_np > 0 && p->spec_pmin > 0.0 && p->spec_pmax > p->spec_pmin) {
    s->spec_e = (double*)malloc((size_t)(p->spec_np + 1) * sizeof(double));
    double lr = log(p->spec_pmax / p->spec_pmin);
    for (int k = 0; k <= p->spec_np; ++k)
      s->spec_e[k] = p->spec_pmin * exp(((double)k / (double)p->spec_np) * lr);
  }
  s->rate = (((double)p->ppc * p->mach_a) * p->dt) / p->dx;
  long long nc = (long long)nx * ny, nn = (long long)s->nxn * ny;
  s->B = (double*)calloc(3 * nc, sizeof(double));
  s->Bs = (double*)calloc(3 * nc, sizeof(double));
  s->Bsum = (double*)calloc(3 * nc, sizeof(double));
  s->K = (double*)calloc(3 * nc, sizeof(double));
  s->E = (double*)calloc(3 * nn, sizeof(double));
  s->Es = (double*)calloc(3 * nn, sizeof(double));
  s->Bb = (double*)calloc(3 * nn, sizeof(double));
  s->n = (double*)calloc(nn, sizeof(double));
  s->J = (double*)calloc(3 * nn, sizeof(double));
  s->u = (double*)calloc(3 * nn, sizeof(double));
  s->qn = (int64_t*)calloc(nn, sizeof(int64_t));
  s->qj = (int64_t*)calloc(3 * nn, sizeof(int64_t));
  s->acc = (double*)calloc(ny, sizeof(double));
  for (long long c = 0; c < nc; ++c) {
    s->B[3 * c + 0] = s->b0x;
    s->B[3 * c + 1] = s->b0y;
    s->B[3 * c + 2] = s->b0z;
  }
  if (p->init_plasma) {
    reserve(s, nc * p->ppc);
    for (int j = 0; j < ny; ++j) {
      for (int i = 0; i < nx; ++i) {
        for (int k = 0; k < p->ppc; ++k) {
          uint32_t pid = (uint32_t)s->next_id++;
          uint32_t ra[4], rb[4];
          draw4(p->seed, pid, 0, PURPOSE_INIT_A, ra);
          draw4(p->seed, pid, 0, PURPOSE_INIT_B, rb);
          double fx = or_u01(ra[0]);
          double fy = (p->dim == 2) ? or_u01(ra[1]) : 0.0;
          double g0, g1, g2, g3;
          gauss2(or_u01(ra[2]), or_u01(ra[3]), &g0, &g1);
          gauss2(or_u01(rb[0]), or_u01(rb[1]), &g2, &g3);
          double vx = s->vth * g0 - p->mach_a;
          double vy = s->vth * g1;
          double vz = s->vth * g2;
          double gv = gamma_v(s, vx, vy, vz);
          vx = vx * gv; vy = vy * gv; vz = vz * gv;  /* stored as u */
          push_particle(s, i, j, fx, fy, vx, vy, vz, pid);
        }
      }
    }
  }
  deposit_and_finish(s);
  ohm(s, s->B, s->E, s->Bb);
  return s;
}

void or_destroy(or_sim* s) {
  if (!s) return;
  free(s->ci); free(s->cj); free(s->fx); free(s->fy);
  free(s->vx); free(s->vy); free(s->vz); free(s->id);
  free(s->B); free(s->Bs); free(s->Bsum); free(s->K);
  free(s->E); free(s->Es); free(s->Bb); free(s->n); free(s->J); free(s->u);
  free(s->qn); free(s->qj); free(s->acc); free(s->spec_e);
  free(s);
}

int or_nxn(const or_sim* s) { return s->nxn; }
long long or_num_particles(const or_sim* s) { return s->np; }

int or_get_particles(const or_sim* s, int32_t* ci, int32_t* cj, double* fx,
                     double* fy, double* vx, double* vy, double* vz,
                     uint32_t* id) {
  long long np = s->np;
  memcpy(ci, s->ci, np * sizeof(int32_t));
  memcpy(cj, s->cj, np * sizeof(int32_t));
  memcpy(fx, s->fx, np * sizeof(double));
  memcpy(fy, s->fy, np * sizeof(double));
  memcpy(vx, s->vx, np * sizeof(double));
  memcpy(vy, s->vy, np * sizeof(double));
  memcpy(vz, s->vz, np * sizeof(double));
  memcpy(id, s->id, np * sizeof(uint32_t));
  return 0;
}

int or_get_grid(const or_sim* s, int what, double* out) {
  long long nc = (long long)s->p.nx * s->p.ny;
  long long nn = (long long)s->nxn * s->p.ny;
  switch (what) {
    case OR_GRID_B: memcpy(out, s->B, 3 * nc * sizeof(double)); return 0;
    case OR_GRID_E: memcpy(out, s->E, 3 * nn * sizeof(double)); return 0;
    case OR_GRID_BBAR: memcpy(out, s->Bb, 3 * nn * sizeof(double)); return 0;
    case OR_GRID_N: memcpy(out, s->n, nn * sizeof(double)); return 0;
    case OR_GRID_J: memcpy(out, s->J, 3 * nn * sizeof(double)); return 0;
    case OR_GRID_U: memcpy(out, s->u, 3 * nn * sizeof(double)); return 0;
    case OR_GRID_PROFILE_N:
      for (int i = 0; i < s->nxn; ++i) {
        double acc = 0.0;
        for (int j = 0; j < s->p.ny; ++j) acc = acc + s->n[nidx(s, i, j)];
        out[i] = acc / (double)s->p.ny;
      }
      return 0;
    case OR_GRID_PROFILE_DB2:
      for (int i = 0; i < s->p.nx; ++i) {
        double acc = 0.0;
        for (int j = 0; j < s->p.ny; ++j) {
          const double* b = s->B + 3 * cidx(s, i, j);
          double dbx = b[0] - s->b0x, dby = b[1] - s->b0y, dbz = b[2] - s->b0z;
          acc = acc + ((dbx * dbx + dby * dby) + dbz * dbz);
        }
        out[i] = acc / (double)s->p.ny;
      }
      return 0;
  }
  return -1;
}

int or_set_B(or_sim* s, const double* B) {
  memcpy(s->B, B, 3LL * s->p.nx * s->p.ny * sizeof(double));
  ohm(s, s->B, s->E, s->Bb);
  return 0;
}

int or_set_node_fields(or_sim* s, const double* E, const double* Bbar) {
  long long nn = (long long)s->nxn * s->p.ny;
  memcpy(s->E, E, 3 * nn * sizeof(double));
  memcpy(s->Bb, Bbar, 3 * nn * sizeof(double));
  return 0;
}

/* Appends particles (cell, offset, velocity, id word; ids NULL -> fresh
   thermal ids), re-sorts, re-deposits the moments and recomputes E and
   Bbar from the current B. */
int or_inject(or_sim* s, long long n, const int32_t* ci, const int32_t* cj,
              const double* fx, const double* fy, const double* vx,
              const double* vy, const double* vz, const uint32_t* ids) {
  for (long long k = 0; k < n; ++k) {
    if (ci[k] < 0 || ci[k] >= s->p.nx || cj[k] < 0 || cj[k] >= s->p.ny)
      return -1;
    if (!(fx[k] >= 0.0 && fx[k] < 1.0)) return -1;
    if (s->p.dim == 2 && !(fy[k] >= 0.0 && fy[k] < 1.0)) return -1;
  }
  for (long long k = 0; k < n; ++k) {
    uint32_t id;
    if (ids) {
      id = ids[k];
      long long num = (long long)(id & ID_MASK);
      if (num >= s->next_id) s->next_id = num + 1;
    } else {
      id = (uint32_t)s->next_id++;
    }
    push_particle(s, ci[k], cj[k], fx[k], s->p.dim == 2 ? fy[k] : 0.0, vx[k],
                  vy[k], vz[k], id);
  }
  sort_by_cell(s);
  deposit_and_finish(s);
  ohm(s, s->B, s->E, s->Bb);
  return 0;
}

int or_diag(const or_sim* s, or_diag_t* o) {
  memset(o, 0, sizeof(*o));
  o->step = s->step;
  o->n_particles = s->np;
  o->next_id = s->next_id;
  o->incident = s->incident;
  o->transmitted = s->transmitted;
  o->reflected = s->reflected;
  o->escaped = s->escaped;
  o->injected = s->injected;
  o->fs_energy = s->fs_energy;
  o->injected_energy = s->injected_energy;
  o->removed_energy = s->removed_energy;
  o->push_work = s->push_work;
  double ke = 0.0, px = 0.0, py = 0.0, pz = 0.0, ub = 0.0;
  for (long long k = 0; k < s->np; ++k) {
    double wp = weight_of(s, s->id[k]);
    ke += kin(s, wp, s->vx[k], s->vy[k], s->vz[k]);
    px += (wp * s->vx[k]) * s->cellvol;
    py += (wp * s->vy[k]) * s->cellvol;
    pz += (wp * s->vz[k]) * s->cellvol;
  }
  long long nc = (long long)s->p.nx * s->p.ny;
  for (long long c = 0; c < nc; ++c) {
    const double* b = s->B + 3 * c;
    ub += (0.5 * ((b[0] * b[0] + b[1] * b[1]) + b[2] * b[2])) * s->cellvol;
  }
  o->kinetic = ke;
  o->magnetic = ub;
  o->px = px; o->py = py; o->pz = pz;
  return 0;
}

/* x - p_x histogram of macroparticle counts; species 0 thermal, 1 cosmic
   rays, -1 all. Bin index bx = floor(X nbx / nx) with X = i + fx in cells,
   bp = floor((vx - pmin) nbp / (pmax - pmin)); out-of-range p_x not counted */
int or_spectrum_p(const or_sim* s, int species, long long* out) {
  int nb = s->p.spec_np;
  if (nb < 1 || !s->spec_e) return -1;
  memset(out, 0, (size_t)nb * sizeof(long long));
  for (long long k = 0; k < s->np; ++k) {
    int cr = (s->id[k] & ID_CR) ? 1 : 0;
    if (species >= 0 && cr != species) continue;
    double ux = s->vx[k], uy = s->vy[k], uz = s->vz[k];
    double p = sqrt(fma(uz, uz, fma(uy, uy, ux * ux)));
    if (!(p >= s->spec_e[0]) || !(p < s->spec_e[nb])) continue;
    int lo = 0, hi = nb;  /* e[lo] <= p < e[hi] */
    while (hi - lo > 1) {
      int mid = (lo + hi) / 2;
      if (p >= s->spec_e[mid]) lo = mid; else hi = mid;
    }
    out[lo]++;
  }
  return 0;
}

int or_histogram(const or_sim* s, int species, long long* out) {
  int nbx = s->p.hist_nx, nbp = s->p.hist_np;
  if (nbx < 1 || nbp < 1) return -1;
  memset(out, 0, (size_t)nbx * nbp * sizeof(long long));
  double hsx = (double)nbx / (double)s->p.nx;
  double hsp = (double)nbp / (s->p.hist_pmax - s->p.hist_pmin);
  for (long long k = 0; k < s->np; ++k) {
    int cr = (s->id[k] & ID_CR) ? 1 : 0;
    if (species >= 0 && cr != species) continue;
    int bx = (int)floor(((double)s->ci[k] + s->fx[k]) * hsx);
    if (bx < 0) bx = 0;
    if (bx >= nbx) bx = nbx - 1;
    double bpd = floor((s->vx[k] - s->p.hist_pmin) * hsp);
    if (!(bpd >= 0.0 && bpd < (double)nbp)) continue;
    out[(long long)bx * nbp + (int)bpd]++;
  }
  return 0;
}
