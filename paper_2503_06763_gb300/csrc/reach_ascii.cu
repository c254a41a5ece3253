// Reach kernels for byte-indexed tables with ASCII rows (TM_BYTE7, see
// reach_impl.cuh): the RE's bytes >= 128 fold onto bytes below 128 of their
// class, so a block's table is half the size and the block holds more warps.
#include "reach_impl.cuh"

namespace slpf {
bool launch_reach_ascii(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                        int sm_count) {
    if (p.mat) return reach::launch_dir_ms<true, true>(p, map, smaps, s, ms, sm_count);
    return reach::launch_dir_ms<false, true>(p, map, smaps, s, ms, sm_count);
}
bool launch_reach_batch_ascii(const BatchGroup &b, uint32_t ms, cudaStream_t s, int sm_count) {
    return reach::launch_dir_batch<true>(b, ms, s, sm_count);
}
uint64_t reach_ascii_warps(const Params &p, uint32_t ms, int sm_count) {
    return p.mat ? reach::dir_warps<true, true>(p, ms, sm_count) : reach::dir_warps<false, true>(p, ms, sm_count);
}
}  // namespace slpf
