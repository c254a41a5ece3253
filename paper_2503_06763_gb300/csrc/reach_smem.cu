// Reach kernels for the smem table mode (see reach_impl.cuh).
#include "reach_impl.cuh"

namespace slpf {
bool launch_reach_smem(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                        int sm_count) {
    return reach::launch_ms<TM_SMEM>(p, map, smaps, s, ms, sm_count);
}
bool launch_reach_batch_smem(const BatchGroup &b, cudaStream_t s, uint32_t ms, int sm_count) {
    return reach::launch_ms_batch<TM_SMEM>(b, s, ms, sm_count);
}
}  // namespace slpf
