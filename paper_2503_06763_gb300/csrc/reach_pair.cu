// Reach kernels for the pair table mode (see reach_impl.cuh).
#include "reach_impl.cuh"

namespace slpf {
bool launch_reach_pair(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                        int sm_count) {
    return reach::launch_ms<TM_PAIR>(p, map, smaps, s, ms, sm_count);
}
bool launch_reach_batch_pair(const BatchGroup &b, cudaStream_t s, uint32_t ms, int sm_count) {
    return reach::launch_ms_batch<TM_PAIR>(b, s, ms, sm_count);
}
}  // namespace slpf
