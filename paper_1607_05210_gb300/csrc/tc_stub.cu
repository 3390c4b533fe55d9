// Placeholder for the tensor-core (mixed form) kernels until they are built.
#include "hapod_internal.cuh"
namespace hapod {
cudaError_t launch_gram_tc(const GramJob*, const int4*, int, const int4*, int, double*, int*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_modes_tc(const ModesJob*, int, int64_t, int*, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace hapod
