// Decode kernels for N = 2 .. 256 (instantiations of bp_decode.cuh).
#include "bp_pipe.cuh"

namespace polarbp {
cudaError_t launch_m1(const LaunchReq& q) { return launch_decode<1>(q); }
cudaError_t launch_m2(const LaunchReq& q) { return launch_decode<2>(q); }
cudaError_t launch_m3(const LaunchReq& q) { return launch_decode<3>(q); }
cudaError_t launch_m4(const LaunchReq& q) { return launch_decode<4>(q); }
cudaError_t launch_m5(const LaunchReq& q) { return launch_decode<5>(q); }
cudaError_t launch_m6(const LaunchReq& q) { return launch_decode<6>(q); }
cudaError_t launch_m7(const LaunchReq& q) { return launch_decode<7>(q); }
cudaError_t launch_m8(const LaunchReq& q) { return launch_decode_pipe<8>(q); }
}  // namespace polarbp
