// Persistent decode kernels for N = 256 (instantiations of bp_decode.cuh).
#include "bp_decode.cuh"

namespace polarbp {
cudaError_t launch_persistent_m8(const SegLaunch& q) { return launch_persistent<8>(q); }
}  // namespace polarbp
