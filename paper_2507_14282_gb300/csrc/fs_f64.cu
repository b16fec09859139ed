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
