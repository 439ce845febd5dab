// Persistent decode kernels for N = 2048 (instantiations of bp_decode.cuh).
#include "bp_decode.cuh"

namespace polarbp {
cudaError_t launch_persistent_m11(const SegLaunch& q) { return launch_persistent<11>(q); }
}  // namespace polarbp
