// Persistent decode kernels for N = 1024 (instantiations of bp_decode.cuh).
#include "bp_decode.cuh"

namespace polarbp {
cudaError_t launch_persistent_m10(const SegLaunch& q) { return launch_persistent<10>(q); }
}  // namespace polarbp
