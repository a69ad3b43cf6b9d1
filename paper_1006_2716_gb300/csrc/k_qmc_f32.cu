// k_qmc_f32.cu -- single-precision sweeps with FP64 Dyson refresh (placeholder until built).
#include "hf_internal.cuh"

namespace hfk {

bool qmc_f32_supported(int) { return false; }
int qmc_f32_chains_per_block(int) { return 1; }
size_t qmc_f32_smem_bytes(int) { return 0; }
cudaError_t launch_qmc_f32(const QmcBatch&, size_t, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace hfk
