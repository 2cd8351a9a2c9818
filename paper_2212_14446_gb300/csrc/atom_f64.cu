// FP64 (reference-path) instantiations of the fused atom kernel.
#include "atom_impl.cuh"

namespace fastpod {
cudaError_t launch_atom_f64(int mode, const AtomArgs<double>& p, int PA, bool has4, cudaStream_t st) {
  return launch_atom_t<double>(mode, p, PA, has4, st);
}
}  // namespace fastpod
