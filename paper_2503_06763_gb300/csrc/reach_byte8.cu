// Reach kernels for the byte-indexed table mode (see reach_impl.cuh).
#include "reach_impl.cuh"

namespace slpf {
bool launch_reach_byte8(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                        int sm_count) {
    if (p.mat) return reach::launch_dir_ms<true>(p, map, smaps, s, ms, sm_count);
    return reach::launch_dir_ms<false>(p, map, smaps, s, ms, sm_count);
}
bool launch_reach_batch_byte8(const BatchGroup &b, uint32_t ms, cudaStream_t s, int sm_count) {
    return reach::launch_dir_batch(b, ms, s, sm_count);
}
uint64_t reach_byte8_warps(const Params &p, uint32_t ms, int sm_count) {
    return p.mat ? reach::dir_warps<true>(p, ms, sm_count) : reach::dir_warps<false>(p, ms, sm_count);
}
}  // namespace slpf
