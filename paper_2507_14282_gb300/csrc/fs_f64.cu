// FP64 instantiation of the hybrid-step kernels. Compiled with -fmad=false:
// every expression rounds exactly as written, without fused multiply-add,
// so the results match the same scheme evaluated on any IEEE-754 CPU.
#include "fs_ops.cuh"

namespace fsx {
const Ops& ops_f64() {
  static const Ops o = OpsImpl<double>::make();
  return o;
}
size_t push_smem_bytes_f64(int dim, int tx, int ty, int chunk) {
  return push_smem_bytes<double>(dim, tx, ty, chunk);
}
}  // namespace fsx

// ---------------------------------------------------------------------------
// fs_field_advance_noalloc: the FP64 field advance of one particle step with
// its RK4 stage buffers in a fixed, file-scope device array instead of
// caller-provided or allocated memory.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

// Stage buffers for the allocation-free field advance: 2^20 doubles (8 MiB)
// held by every GPU that loads the library until the process exits.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;
static __device__ __align__(256) double fs_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device. The host-side
// symbol is only a stand-in, not a device address. Outside stream capture
// the address is looked up on every call (cheap, host-side), so a module
// loaded again into a new context (after cudaDeviceReset, say) is found at
// its new address; the last address seen on the device is kept for calls
// made while `st` is being captured, where the lookup is not made.
int noalloc_scratch(cudaStream_t st, double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FS_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return FS_EINVAL;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FS_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, fs_noalloc_scratch) != cudaSuccess || !ptr)
      return FS_ECUDA;
    g_scratch_addr[dev] = (double*)ptr;
  }
  if (!g_scratch_addr[dev]) return FS_EINVAL;  // first call on the device made under capture
  *out = g_scratch_addr[dev];
  return FS_OK;
}

// [a, a + na) and [b, b + nb) share a byte
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

template <int DIM>
void noalloc_launch(const fsx::Geo& g, const fsx::Phys& ph, int n_sub, double* B,
                    const double* n, const double* u, double* E, double* scr,
                    cudaStream_t st) {
  using namespace fsx;
  const long long nc = (long long)g.nx * g.ny, nn = (long long)g.nxn * g.ny;
  double* Bs = scr;
  double* Bsum = scr + 3 * nc;
  double* Es = scr + 6 * nc;
  const int gn = grid_for(nn), gc = grid_for(nc);
  for (int sub = 0; sub < n_sub; ++sub) {
    k_ohm<double, DIM><<<gn, kBlock, 0, st>>>(B, n, u, nullptr, Es, nullptr, nullptr, g, ph);
    k_faraday<double, DIM><<<gc, kBlock, 0, st>>>(Es, B, Bs, Bsum, 1, g, ph);
    k_ohm<double, DIM><<<gn, kBlock, 0, st>>>(Bs, n, u, nullptr, Es, nullptr, nullptr, g, ph);
    k_faraday<double, DIM><<<gc, kBlock, 0, st>>>(Es, B, Bs, Bsum, 2, g, ph);
    k_ohm<double, DIM><<<gn, kBlock, 0, st>>>(Bs, n, u, nullptr, Es, nullptr, nullptr, g, ph);
    k_faraday<double, DIM><<<gc, kBlock, 0, st>>>(Es, B, Bs, Bsum, 3, g, ph);
    k_ohm<double, DIM><<<gn, kBlock, 0, st>>>(Bs, n, u, nullptr, Es, nullptr, nullptr, g, ph);
    k_faraday<double, DIM><<<gc, kBlock, 0, st>>>(Es, B, Bs, Bsum, 4, g, ph);
  }
  k_ohm<double, DIM><<<gn, kBlock, 0, st>>>(B, n, u, nullptr, E, nullptr, nullptr, g, ph);
}

}  // namespace

extern "C" int fs_field_advance_noalloc(const fs_params* p, const double* B_in,
                                        const double* n, const double* u,
                                        double* B_out, double* E_out,
                                        void* cuda_stream) {
  FS_GUARD_BEGIN
  if (!p || !B_in || !n || !u || !B_out || !E_out) return FS_EINVAL;
  if (p->precision != FS_FP64) return FS_EINVAL;
  fsx::Geo g;
  fsx::Phys ph;
  int r = fsx::derive_geometry(p, &g, &ph);
  if (r) return r;
  const size_t nc = (size_t)g.nx * g.ny, nn = (size_t)g.nxn * g.ny;
  if (6 * nc + 3 * nn > kNoAllocScratchDoubles) return FS_EINVAL;
  // the outputs share no byte with each other or with the inputs, except
  // B_out == B_in exactly (the field advanced in place)
  const size_t bB = 3 * nc * sizeof(double), bE = 3 * nn * sizeof(double);
  const size_t bn = nn * sizeof(double), bu = 3 * nn * sizeof(double);
  if (B_out != B_in && overlaps(B_out, bB, B_in, bB)) return FS_EINVAL;
  if (overlaps(B_out, bB, n, bn) || overlaps(B_out, bB, u, bu) ||
      overlaps(B_out, bB, E_out, bE))
    return FS_EINVAL;
  if (overlaps(E_out, bE, n, bn) || overlaps(E_out, bE, u, bu) ||
      overlaps(E_out, bE, B_in, bB))
    return FS_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // a launch error left by an earlier, unrelated call is cleared here, so the
  // check after this call's launches reports only its own
  (void)cudaGetLastError();
  double* scr = nullptr;
  r = noalloc_scratch(st, &scr);
  if (r) return r;
  if (B_out != B_in &&
      cudaMemcpyAsync(B_out, B_in, 3 * nc * sizeof(double), cudaMemcpyDeviceToDevice,
                      st) != cudaSuccess)
    return FS_ECUDA;
  if (g.dim == 1)
    noalloc_launch<1>(g, ph, p->n_sub, B_out, n, u, E_out, scr, st);
  else
    noalloc_launch<2>(g, ph, p->n_sub, B_out, n, u, E_out, scr, st);
  return cudaGetLastError() == cudaSuccess ? FS_OK : FS_ECUDA;
  FS_GUARD_END
}
