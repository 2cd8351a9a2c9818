// FP32 (mixed-precision) instantiations of the fused atom kernel for the embedding model.
#include "atom_impl.cuh"

namespace fastpod {
cudaError_t launch_atom_emb_f32(const AtomArgs<float>& p, int PA, bool has4, cudaStream_t st) {
  return launch_atom_emb_t<float>(p, PA, has4, st);
}
}  // namespace fastpod
