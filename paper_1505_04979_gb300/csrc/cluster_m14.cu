// Decode kernels for N = 16384: clusters of 4 thread blocks (instantiations of bp_cluster.cuh).
#include "bp_cluster.cuh"

namespace polarbp {
cudaError_t launch_m14(const LaunchReq& q) { return launch_cluster<2>(q); }
}  // namespace polarbp
