// fs_spectra.cuh -- diagnostics of the paper's Sec. 3: transversely averaged
// lineouts of Bx, By, Bz and the perpendicular power spectrum
// < |F_perp(k_x, y)|^2 > = |F[By]|^2 + |F[Bz]|^2 averaged over y (Sec. 3.1,
// Fig. 3 caption), F the DFT along x normalised by 1/nx; and the momentum
// spectrum n(p) of the particles (the CR spectra of Sec. 3). FP64 in every
// precision; not on the per-step path.
//
// The spectrum packs each row into one complex sequence z = By + i Bz: for
// real By, Bz, F[By](k) = (Z(k) + conj Z(-k)) / 2 and F[Bz](k) =
// (Z(k) - conj Z(-k)) / 2i, so |F[By]|^2 + |F[Bz]|^2 = (|Z(k)|^2 +
// |Z(-k)|^2) / 2 with Z = F[z]. Rows of power-of-two length up to
// kFftMax are transformed in shared memory by an iterative radix-2
// Cooley-Tukey FFT (one CTA per row); other lengths by a direct DFT.
#pragma once
#include "fs_engine.cuh"

namespace fsx {

constexpr int kFftMax = 8192;     // complex doubles in shared memory: 128 KB
constexpr int kFftThreads = 512;

// y-averaged B: out[i * 3 + c] = (1/ny) sum_j B_c(i, j)
template <typename T>
__global__ void k_profile_B(const T* __restrict__ B, int nx, int ny, double* __restrict__ out) {
  const size_t nc = (size_t)nx * ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
    double a[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < ny; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) a[c] += (double)B[c * nc + (size_t)j * nx + i];
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * i + c] = a[c] / (double)ny;
  }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// the row's contribution to P[k] from Z(k) and Z(nx - k); P is pre-zeroed
__device__ __forceinline__ void add_power(double* P, int k, double2 zk, double2 zm, int nx,
                                          int ny) {
  const double s = 0.5 * ((zk.x * zk.x + zk.y * zk.y) + (zm.x * zm.x + zm.y * zm.y));
  atomicAdd(&P[k], s / ((double)nx * (double)nx) / (double)ny);
}

// One CTA per row j; nx = 2^logn <= kFftMax; dynamic shared memory nx double2.
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_bperp_fft(const T* __restrict__ B, int nx,
                                                           int ny, int logn,
                                                           double* __restrict__ P) {
  extern __shared__ double2 z[];
  const int j = blockIdx.x;
  const size_t nc = (size_t)nx * ny;
  const T* by = B + nc + (size_t)j * nx;
  const T* bz = B + 2 * nc + (size_t)j * nx;
  // load in bit-reversed order
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    const int r = (int)(__brev((unsigned)x) >> (32 - logn));
    z[r] = make_double2((double)by[x], (double)bz[x]);
  }
  __syncthreads();
  for (int len = 2; len <= nx; len <<= 1) {
    const int half = len >> 1;
    for (int t = threadIdx.x; t < nx / 2; t += blockDim.x) {
      const int pos = t & (half - 1);
      const int i0 = (t - pos) * 2 + pos, i1 = i0 + half;
      double sn, cs;
      sincospi(-2.0 * (double)pos / (double)len, &sn, &cs);  // exp(-2 pi i pos / len)
      const double2 v = cmul(z[i1], make_double2(cs, sn));
      const double2 u = z[i0];
      z[i0] = make_double2(u.x + v.x, u.y + v.y);
      z[i1] = make_double2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k <= nx / 2; k += blockDim.x)
    add_power(P, k, z[k], z[(nx - k) & (nx - 1)], nx, ny);
}

// Direct DFT, one thread per (k, row): Z(k) and Z(nx - k) as sums over x
// with the phase step multiplied in and re-anchored every 64 terms.
template <typename T>
__global__ void k_bperp_dft(const T* __restrict__ B, int nx, int ny, double* __restrict__ P) {
  const int nk = nx / 2 + 1;
  const size_t nc = (size_t)nx * ny;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)nk * ny;
       q += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(q % nk), j = (int)(q / nk);
    const T* by = B + nc + (size_t)j * nx;
    const T* bz = B + 2 * nc + (size_t)j * nx;
    double2 zk = make_double2(0.0, 0.0), zm = make_double2(0.0, 0.0);
    double2 w = make_double2(1.0, 0.0), step;
    sincospi(-2.0 * (double)k / (double)nx, &step.y, &step.x);
    for (int x = 0; x < nx; ++x) {
      if ((x & 63) == 0) {  // exact phase exp(-2 pi i k x / nx) from the integer k x mod nx
        const long long kx = ((long long)k * x) % nx;
        sincospi(-2.0 * (double)kx / (double)nx, &w.y, &w.x);
      }
      const double2 v = make_double2((double)by[x], (double)bz[x]);
      const double2 a = cmul(v, w);                              // v exp(-i theta)
      const double2 b = cmul(v, make_double2(w.x, -w.y));        // v exp(+i theta): Z(-k)
      zk.x += a.x; zk.y += a.y;
      zm.x += b.x; zm.y += b.y;
      w = cmul(w, step);
    }
    add_power(P, k, zk, zm, nx, ny);
  }
}

// Momentum spectrum n(p): counts of |u| between the log-spaced edges
// e[0..np] (e[k] <= |u| < e[k+1]); species -1 all, 1 cosmic rays only.
// Integer counts, bins chosen by exact comparisons with |u| = sqrt(u.u).
template <typename T>
__global__ void k_spectrum_p(DevPtrs<T> d, Geo g, int buf, int species, int np,
                             const double* __restrict__ e,
                             unsigned long long* __restrict__ out) {
  const int t = blockIdx.x;
  const int cnt = min(d.cnt[buf][t], g.tile_cap), base = d.tile_base[t];
  const Parts<T> P = d.P[buf];
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int gi = base + q;
    if (species == 1 && !(P.id[gi] & kIdCR)) continue;
    const double ux = P.vx[gi], uy = P.vy[gi], uz = P.vz[gi];
    const double p = __dsqrt_rn(__fma_rn(uz, uz, __fma_rn(uy, uy, __dmul_rn(ux, ux))));
    if (!(p >= e[0]) || !(p < e[np])) continue;
    int lo = 0, hi = np;  // e[lo] <= p < e[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (p >= e[mid]) lo = mid; else hi = mid;
    }
    atomicAdd(&out[lo], 1ull);
  }
}

}  // namespace fsx
