// Reach kernels for the byte-indexed table mode with full rows (see
// reach_impl.cuh); an RE whose bytes >= 128 fold onto ASCII bytes of their
// class takes the ASCII-row kernels of reach_ascii.cu instead.
#include "reach_impl.cuh"

namespace slpf {
bool launch_reach_ascii(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                        int sm_count);
bool launch_reach_batch_ascii(const BatchGroup &b, uint32_t ms, cudaStream_t s, int sm_count);
uint64_t reach_ascii_warps(const Params &p, uint32_t ms, int sm_count);

bool launch_reach_byte8(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                        int sm_count) {
    if (p.t.hirep) return launch_reach_ascii(p, map, smaps, s, ms, sm_count);
    if (p.mat) return reach::launch_dir_ms<true, false>(p, map, smaps, s, ms, sm_count);
    return reach::launch_dir_ms<false, false>(p, map, smaps, s, ms, sm_count);
}
bool launch_reach_batch_byte8(const BatchGroup &b, uint32_t ms, cudaStream_t s, int sm_count) {
    if (b.t.hirep) return launch_reach_batch_ascii(b, ms, s, sm_count);
    return reach::launch_dir_batch<false>(b, ms, s, sm_count);
}
uint64_t reach_byte8_warps(const Params &p, uint32_t ms, int sm_count) {
    if (p.t.hirep) return reach_ascii_warps(p, ms, sm_count);
    return p.mat ? reach::dir_warps<true, false>(p, ms, sm_count) : reach::dir_warps<false, false>(p, ms, sm_count);
}
}  // namespace slpf
