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
}  // namespace fsx
