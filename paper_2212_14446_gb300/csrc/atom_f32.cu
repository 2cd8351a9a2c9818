// FP32 (mixed-precision) instantiations of the fused atom kernel.
#include "atom_impl.cuh"

namespace fastpod {
int atom_warps(int N, int K, int wpb) { return atom_warps_t(N, K, wpb > 0 ? wpb : WPB_ATOM); }
cudaError_t launch_atom_f32(int mode, const AtomArgs<float>& p, int PA, bool has4, cudaStream_t st) {
  return launch_atom_t<float>(mode, p, PA, has4, st);
}
}  // namespace fastpod
