// One-launch mixed-stream decoder whose longest code length is 2^11 (bp_mixed.cuh).
#include "bp_mixed.cuh"

namespace polarbp {
cudaError_t launch_mixed_m11(const MixedArgs& a, int stop_mode, int freeze_mode, int sms, cudaStream_t s)
{
    return launch_mixed<11>(a, stop_mode, freeze_mode, sms, s);
}
}  // namespace polarbp
