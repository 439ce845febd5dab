// Persistent decode kernels for N = 4096 (instantiations of bp_decode.cuh).
#include "bp_decode.cuh"

namespace polarbp {
cudaError_t launch_persistent_m12(const SegLaunch& q) { return launch_persistent<12>(q); }
}  // namespace polarbp
