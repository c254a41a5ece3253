// Reach kernels for the global table mode (see reach_impl.cuh).
#include "reach_impl.cuh"

namespace slpf {
bool launch_reach_global(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                         int sm_count) {
    return reach::launch_ms<TM_GLOBAL>(p, map, smaps, s, ms, sm_count);
}

bool launch_reach_batch_global(const BatchGroup &b, cudaStream_t s, uint32_t ms, int sm_count) {
    return reach::launch_ms_batch<TM_GLOBAL>(b, s, ms, sm_count);
}

bool launch_reach_pair(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                       int sm_count);
bool launch_reach_batch_pair(const BatchGroup &b, cudaStream_t s, uint32_t ms, int sm_count);
bool launch_reach_batch_smem(const BatchGroup &b, cudaStream_t s, uint32_t ms, int sm_count);
bool launch_reach_smem(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                       int sm_count);

bool launch_reach_smem8(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                        int sm_count);
bool launch_reach_batch_smem8(const BatchGroup &b, cudaStream_t s, uint32_t ms, int sm_count);

// One-byte tables with at most 256 states per direction: the reach stages
// them as u8 (TM_SMEM8), a quarter of the u32 rows, so more blocks fit an SM.
static bool byte_states(const DevTables &t) { return t.nf <= 256 && t.nb <= 256; }

bool launch_reach_byte8(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                        int sm_count);

bool launch_reach(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                  int sm_count) {
    // shape 1, byte-indexed tables: no class lookup per byte; a block per direction
    if (p.rvar == 1 && p.t.fbyte && p.t.bbyte) return launch_reach_byte8(p, map, smaps, s, ms, sm_count);
    if (p.tmode == TM_PAIR) return launch_reach_pair(p, map, smaps, s, ms, sm_count);
    if (p.tmode == TM_SMEM && byte_states(p.t)) return launch_reach_smem8(p, map, smaps, s, ms, sm_count);
    if (p.tmode == TM_SMEM) return launch_reach_smem(p, map, smaps, s, ms, sm_count);
    return launch_reach_global(p, map, smaps, s, ms, sm_count);
}

bool launch_reach_batch(const BatchGroup &b, uint32_t tmode, uint32_t ms, cudaStream_t s, int sm_count) {
    if (tmode == TM_PAIR) return launch_reach_batch_pair(b, s, ms, sm_count);
    if (tmode == TM_SMEM && byte_states(b.t)) return launch_reach_batch_smem8(b, s, ms, sm_count);
    if (tmode == TM_SMEM) return launch_reach_batch_smem(b, s, ms, sm_count);
    return launch_reach_batch_global(b, s, ms, sm_count);
}
}  // namespace slpf
