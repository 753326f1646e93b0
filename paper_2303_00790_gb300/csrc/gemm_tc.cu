// Tensor-core (tcgen05) GEMMs of the subspace steps -- placeholder until the
// split-bf16 kernels land; the tensor mode reports "not supported" meanwhile.
#include <cuda_runtime.h>

#include "kscf_internal.h"

namespace kscf {

bool tc_available() { return false; }
size_t gram_tc_work_bytes(int64_t, int, int) { return 0; }
size_t rotate_tc_work_bytes(int64_t, int, int) { return 0; }

cudaError_t launch_gram_tc(const float*, int64_t, const float*, int64_t, int64_t, int, int, double, double*, int64_t,
                           bool, void*, size_t, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_rotate_tc(const float*, int64_t, const double*, int64_t, int64_t, int, int, bool, float*, int64_t,
                             void*, size_t, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace kscf
