// FP32 instantiation of the hybrid-step kernels (FMA contraction allowed).
#include "fs_ops.cuh"

namespace fsx {
const Ops& ops_f32() {
  static const Ops o = OpsImpl<float>::make();
  return o;
}
size_t push_smem_bytes_f32(int dim, int tx, int ty, int chunk) {
  return push_smem_bytes<float>(dim, tx, ty, chunk);
}
cudaError_t launch_wait_selftest(int* status, int limit, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(status, limit);
  return cudaGetLastError();
}
}  // namespace fsx
