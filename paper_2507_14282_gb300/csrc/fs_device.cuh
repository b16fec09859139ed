// fs_device.cuh -- device building blocks: counter-based random numbers and
// the elementary functions the particle draws need.
//
// Every random draw is keyed on (particle number, step, purpose) through
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), so a draw does not
// depend on thread or launch order. The Gaussian and angle draws use this
// file's own log and sincos (argument reduction plus series, written out
// below with correctly rounded coefficients) so that FP64 draws are the same
// bits on any IEEE-754 machine that evaluates the same expressions without
// contraction; the FP64 translation unit is compiled with -fmad=false.
#pragma once
#include <stdint.h>

#include "fs_internal.h"

namespace fsx {

// Philox purposes: which draw of a particle-step a counter belongs to.
enum : uint32_t {
  kPurposeInitA = 1u,
  kPurposeInitB = 2u,
  kPurposeFS = 3u,
  kPurposeInjA = 4u,
  kPurposeInjB = 5u,
  kPurposeInjCR = 6u
};


// Philox4x32-10: ten rounds of the two-multiplier S-box
//   (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0))
// with the Weyl key schedule k += (W0, W1) between rounds.
struct Philox4 {
  uint32_t x[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1,
                                                 uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  Philox4 r;
  r.x[0] = c0; r.x[1] = c1; r.x[2] = c2; r.x[3] = c3;
  return r;
}

__device__ __forceinline__ Philox4 draw4(unsigned long long seed, uint32_t pid,
                                         long long step, uint32_t purpose) {
  return philox4x32_10(pid, (uint32_t)step, purpose, 0u, (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

// uniform on (0,1): the midpoint of bin k of 2^32 (exact in FP64)
__device__ __forceinline__ double u01(uint32_t k) {
  return __dmul_rn(__dadd_rn((double)k, 0.5), 0x1p-32);
}

// log x: x = m 2^e with m in [sqrt(1/2), sqrt(2)); log m = 2 atanh(s),
// s = (m-1)/(m+1), as the odd series 2 s (1 + s^2/3 + s^4/5 + ... + s^22/23)
// by Horner in z = s^2; e ln2 with ln2 split into a 32-bit head and a tail.
__device__ __forceinline__ double fs_log(double x) {
  int e;
  double m = frexp(x, &e);
  m = __dmul_rn(m, 2.0);
  e = e - 1;
  if (m > 0x1.6a09e667f3bcdp+0) {
    m = __dmul_rn(m, 0.5);
    e = e + 1;
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double z = __dmul_rn(s, s);
  double p = 0x1.642c8590b2164p-5;
  p = __dadd_rn(__dmul_rn(p, z), 0x1.8618618618618p-5);
  p = __dadd_rn(__dmul_rn(p, z), 0x1.af286bca1af28p-5);
  p = __dadd_rn(__dmul_rn(p, z), 0x1.e1e1e1e1e1e1ep-5);
  p = __dadd_rn(__dmul_rn(p, z), 0x1.1111111111111p-4);
  p = __dadd_rn(__dmul_rn(p, z), 0x1.3b13b13b13b14p-4);
  p = __dadd_rn(__dmul_rn(p, z), 0x1.745d1745d1746p-4);
  p = __dadd_rn(__dmul_rn(p, z), 0x1.c71c71c71c71cp-4);
  p = __dadd_rn(__dmul_rn(p, z), 0x1.2492492492492p-3);
  p = __dadd_rn(__dmul_rn(p, z), 0x1.999999999999ap-3);
  p = __dadd_rn(__dmul_rn(p, z), 0x1.5555555555555p-2);
  p = __dadd_rn(__dmul_rn(p, z), 1.0);
  const double lm = __dmul_rn(__dmul_rn(2.0, s), p);
  const double de = (double)e;
  return __dadd_rn(__dmul_rn(de, 0x1.62e42fee00000p-1),
                   __dadd_rn(lm, __dmul_rn(de, 0x1.a39ef35793c76p-33)));
}

// (cos 2 pi u, sin 2 pi u): quadrant q = round(4u), remainder angle
// r = (4u - q) pi/2 in [-pi/4, pi/4], Taylor series to r^19 / r^18.
__device__ __forceinline__ void fs_sincos2pi(double u, double* co, double* si) {
  const double t = __dmul_rn(4.0, u);
  const double q = floor(__dadd_rn(t, 0.5));
  const double d = __dsub_rn(t, q);
  const double r = __dmul_rn(d, 0x1.921fb54442d18p+0);
  const double z = __dmul_rn(r, r);
  double ps = -0x1.2f49b46814157p-57;
  ps = __dadd_rn(__dmul_rn(ps, z), 0x1.952c77030ad4ap-49);
  ps = __dsub_rn(__dmul_rn(ps, z), 0x1.ae7f3e733b81fp-41);
  ps = __dadd_rn(__dmul_rn(ps, z), 0x1.6124613a86d09p-33);
  ps = __dsub_rn(__dmul_rn(ps, z), 0x1.ae64567f544e4p-26);
  ps = __dadd_rn(__dmul_rn(ps, z), 0x1.71de3a556c734p-19);
  ps = __dsub_rn(__dmul_rn(ps, z), 0x1.a01a01a01a01ap-13);
  ps = __dadd_rn(__dmul_rn(ps, z), 0x1.1111111111111p-7);
  ps = __dsub_rn(__dmul_rn(ps, z), 0x1.5555555555555p-3);
  const double sr = __dadd_rn(r, __dmul_rn(__dmul_rn(r, z), ps));
  double pc = -0x1.6827863b97d97p-53;
  pc = __dadd_rn(__dmul_rn(pc, z), 0x1.ae7f3e733b81fp-45);
  pc = __dsub_rn(__dmul_rn(pc, z), 0x1.93974a8c07c9dp-37);
  pc = __dadd_rn(__dmul_rn(pc, z), 0x1.1eed8eff8d898p-29);
  pc = __dsub_rn(__dmul_rn(pc, z), 0x1.27e4fb7789f5cp-22);
  pc = __dadd_rn(__dmul_rn(pc, z), 0x1.a01a01a01a01ap-16);
  pc = __dsub_rn(__dmul_rn(pc, z), 0x1.6c16c16c16c17p-10);
  pc = __dadd_rn(__dmul_rn(pc, z), 0x1.5555555555555p-5);
  pc = __dsub_rn(__dmul_rn(pc, z), 0.5);
  const double cr = __dadd_rn(1.0, __dmul_rn(z, pc));
  const int iq = ((int)q) & 3;
  double c, s;
  if (iq == 0) { c = cr; s = sr; }
  else if (iq == 1) { c = -sr; s = cr; }
  else if (iq == 2) { c = -cr; s = -sr; }
  else { c = sr; s = -cr; }
  *co = c;
  *si = s;
}

// Box-Muller: two independent standard normals from two uniforms
__device__ __forceinline__ void gauss2(double u1, double u2, double* g0,
                                       double* g1) {
  const double rad = __dsqrt_rn(__dmul_rn(-2.0, fs_log(u1)));
  double c, s;
  fs_sincos2pi(u2, &c, &s);
  *g0 = __dmul_rn(rad, c);
  *g1 = __dmul_rn(rad, s);
}

}  // namespace fsx
