// Reach kernels for the u8 one-byte table mode (see reach_impl.cuh).
#include "reach_impl.cuh"

namespace slpf {
bool launch_reach_smem8(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                        int sm_count) {
    return reach::launch_ms<TM_SMEM8>(p, map, smaps, s, ms, sm_count);
}
bool launch_reach_batch_smem8(const BatchGroup &b, cudaStream_t s, uint32_t ms, int sm_count) {
    return reach::launch_ms_batch<TM_SMEM8>(b, s, ms, sm_count);
}
}  // namespace slpf
