// BF16 tcgen05 grouped network (pass 1): placeholder until the tensor-core kernel lands.
#include "coral_internal.cuh"

namespace coral {
int pass1_bf16_grid(int) { return 0; }
size_t pass1_bf16_smem() { return 0; }
cudaError_t launch_pass1_bf16(const StepArgs&, cudaStream_t, int) { return cudaErrorNotSupported; }
}  // namespace coral
