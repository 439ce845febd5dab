// Persistent decode kernels for N = 512 (instantiations of bp_decode.cuh).
#include "bp_decode.cuh"

namespace polarbp {
cudaError_t launch_persistent_m9(const SegLaunch& q) { return launch_persistent<9>(q); }
}  // namespace polarbp
