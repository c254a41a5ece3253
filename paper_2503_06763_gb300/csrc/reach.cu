// Reach phase (arXiv 2503.06763, Eq. reacher; Sect. 4.1 fuses the forward and
// backward reacher of a chunk into one task, as here).
//
// One thread per chunk y_i runs, in the same loop, the forward ME-DFA from
// every speculation slot of the chunk left to right and the reverse ME-DFA
// from every backward slot right to left: two independent dependency chains.
// Slots are the distinct start sets after the boundary byte (a run from a
// singleton {q} reaches D_end(q) after one byte), restricted by the class of
// the byte before the boundary (the last-character filter of Sect. 6).
// Chunk 0 runs forward from I and chunk c-1 backward from F without
// speculation (J_0 = I, Ĵ_{c+1} = F, Eq. joiner).
//
// Runs are compared at every 64-byte sub-chunk boundary.  Once all live runs
// of a direction hold the same state they stay equal, so from there on the
// common state is the exact state of the text for any live input: the thread
// writes it as a checkpoint (FC / BC), keeps one run and remembers which slots
// were live.  Outputs: end state per slot (R, R̂), checkpoints, and the first
// (forward) / last (backward) boundary where the runs agreed.
#include "kernels.cuh"

namespace slpf {
namespace {

template <bool SMEM, int MS, bool MULTI, bool EDGE>
__device__ __forceinline__ void walk_block(const Params &p, const Tabs &T, uint64_t fpos, uint64_t bpos,
                                           uint32_t (&sf)[MS], uint32_t (&sb)[MS], uint32_t mf, uint32_t mb,
                                           bool bwd, int f_lo, int f_hi, int b_lo, int b_hi) {
    // forward bytes fpos + 16q + u (ascending), backward bytes bpos + 16(3-q) + 15-u (descending)
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        const uint4 fx = load16(p.x, p.n, fpos + 16 * q);
        const uint4 bx = bwd ? load16(p.x, p.n, bpos + 16 * (3 - q)) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int tf = 16 * q + u, tb = 63 - tf;
            if (!EDGE || (tf >= f_lo && tf < f_hi)) {
                const uint32_t c = clsof<SMEM>(T, byte_of(fx, u));
                if (MULTI) {
#pragma unroll
                    for (int j = 0; j < MS; ++j)
                        if (j < (int)mf) sf[j] = fnext<SMEM>(T, sf[j], c);
                } else {
                    sf[0] = fnext<SMEM>(T, sf[0], c);
                }
            }
            if (bwd && (!EDGE || (tb >= b_lo && tb <= b_hi))) {
                const uint32_t c = clsof<SMEM>(T, byte_of(bx, 15 - u));
                if (MULTI) {
#pragma unroll
                    for (int j = 0; j < MS; ++j)
                        if (j < (int)mb) sb[j] = bnext<SMEM>(T, sb[j], c);
                } else {
                    sb[0] = bnext<SMEM>(T, sb[0], c);
                }
            }
        }
    }
}

// If all live runs agree, keep one run and record the live slots.
template <int MS>
__device__ __forceinline__ bool try_converge(uint32_t (&s)[MS], uint32_t &m, uint32_t (&live)[(MS + 31) / 32]) {
    uint32_t rep = 0;
    bool same = true;
#pragma unroll
    for (int j = 0; j < MS; ++j)
        if (j < (int)m && s[j]) {
            if (!rep) rep = s[j];
            else if (s[j] != rep) same = false;
        }
    if (!same) return false;
#pragma unroll
    for (int w = 0; w < (MS + 31) / 32; ++w) live[w] = 0;
#pragma unroll
    for (int j = 0; j < MS; ++j)
        if (j < (int)m && s[j]) live[j >> 5] |= 1u << (j & 31);
    s[0] = rep;
    m = 1;
    return true;
}

template <bool SMEM, int MS>
__device__ void reach_chunk(const Params &p, const Tabs &T, uint32_t i) {
    const DevTables &t = p.t;
    const uint64_t base = (uint64_t)i * p.k;
    const uint32_t len = chunk_len(p, i);
    const uint32_t nsub = (len + 63) / 64;
    const bool bwd = !p.recognize;
    uint32_t sf[MS], sb[MS];
    uint32_t livef[(MS + 31) / 32], liveb[(MS + 31) / 32];
#pragma unroll
    for (int j = 0; j < MS; ++j) { sf[j] = 0u; sb[j] = 0u; }
    uint32_t mf, mf0, mb = 0, mb0 = 0;
    int tstart, tlast = -1;
    if (i == 0) {
        mf = 1; sf[0] = t.fI; tstart = 0;                  // J_0 = I
    } else {
        const uint32_t pr = clsof<SMEM>(T, __ldg(p.x + base - 1)) * t.ncls + clsof<SMEM>(T, __ldg(p.x + base));
        mf = __ldg(t.fSlotCount + pr);
#pragma unroll
        for (int j = 0; j < MS; ++j)
            if (j < (int)mf) sf[j] = __ldg(t.fSlotStart + pr * t.msf + j);
        tstart = 1;                                        // slot states follow byte 0
    }
    mf0 = mf;
    if (bwd) {
        if (i == p.c - 1) {
            mb = 1; sb[0] = t.bF; tlast = (int)len - 1;    // Ĵ_{c+1} = F
        } else {
            const uint32_t pr = clsof<SMEM>(T, __ldg(p.x + base + len - 1)) * t.ncls +
                                clsof<SMEM>(T, __ldg(p.x + base + len));
            mb = __ldg(t.bSlotCount + pr);
#pragma unroll
            for (int j = 0; j < MS; ++j)
                if (j < (int)mb) sb[j] = __ldg(t.bSlotStart + pr * t.msb + j);
            tlast = (int)len - 2;                          // slot states precede the last byte
        }
        mb0 = mb;
    }
#pragma unroll
    for (int w = 0; w < (MS + 31) / 32; ++w) { livef[w] = ~0u; liveb[w] = ~0u; }
    bool fconv = false, bconv = false;
    uint32_t fconv_sub = nsub, bconv_sub = 0;
    if (mf <= 1) { fconv = true; fconv_sub = 1; }
    if (mb <= 1) { bconv = true; bconv_sub = nsub - 1; }

    for (uint32_t blk = 0; blk < nsub; ++blk) {
        const uint32_t fb = blk, bb = nsub - 1 - blk;
        if (fb >= 1) {                                      // boundary before forward block fb
            if (!fconv && try_converge<MS>(sf, mf, livef)) { fconv = true; fconv_sub = fb; }
            p.w.FC[(uint64_t)i * p.S + fb] = fconv ? sf[0] : kUnknown;
        }
        const uint64_t fpos = base + 64ull * fb, bpos = base + 64ull * bb;
        const int f_lo = fb == 0 ? tstart : 0;
        const int f_hi = (int)min(64u, len - 64 * fb);
        const int b_hi = min(63, tlast - (int)(64 * bb));
        const bool edge = f_lo != 0 || f_hi != 64 || (bwd && b_hi != 63);
        const bool multi = mf > 1 || mb > 1;
        if (edge) {
            if (multi) walk_block<SMEM, MS, true, true>(p, T, fpos, bpos, sf, sb, mf, mb, bwd, f_lo, f_hi, 0, b_hi);
            else walk_block<SMEM, MS, false, true>(p, T, fpos, bpos, sf, sb, mf, mb, bwd, f_lo, f_hi, 0, b_hi);
        } else {
            if (multi) walk_block<SMEM, MS, true, false>(p, T, fpos, bpos, sf, sb, mf, mb, bwd, 0, 64, 0, 63);
            else walk_block<SMEM, MS, false, false>(p, T, fpos, bpos, sf, sb, mf, mb, bwd, 0, 64, 0, 63);
        }
        if (bwd && bb >= 1) {                               // boundary at the start of backward block bb
            if (!bconv && try_converge<MS>(sb, mb, liveb)) { bconv = true; bconv_sub = bb; }
            p.w.BC[(uint64_t)i * p.S + bb - 1] = bconv ? sb[0] : kUnknown;
        }
    }
    // end state of every original slot (a slot dead at convergence stays dead)
    const uint32_t msf = t.msf;
    for (uint32_t j = 0; j < msf; ++j) {
        uint32_t v = 0;
        if (j < mf0) {
            if (mf == 1 && mf0 > 1) v = ((livef[j >> 5] >> (j & 31)) & 1) ? sf[0] : 0u;
            else {
#pragma unroll
                for (int jj = 0; jj < MS; ++jj) if (jj == (int)j) v = sf[jj];
            }
        }
        p.w.Rf[(size_t)i * msf + j] = v;
    }
    p.w.fconv[i] = fconv_sub;
    if (bwd) {
        const uint32_t msb = t.msb;
        for (uint32_t j = 0; j < msb; ++j) {
            uint32_t v = 0;
            if (j < mb0) {
                if (mb == 1 && mb0 > 1) v = ((liveb[j >> 5] >> (j & 31)) & 1) ? sb[0] : 0u;
                else {
#pragma unroll
                    for (int jj = 0; jj < MS; ++jj) if (jj == (int)j) v = sb[jj];
                }
            }
            p.w.Rb[(size_t)i * msb + j] = v;
        }
        p.w.bconv[i] = bconv_sub;
    }
}

template <bool SMEM, int MS>
__global__ void __launch_bounds__(kBlockThreads) reach_kernel(Params p) {
    extern __shared__ __align__(16) uint8_t sm[];
    Tabs T;
    stage_tables<SMEM>(p, sm, T);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < p.c; i += stride) reach_chunk<SMEM, MS>(p, T, i);
}

template <bool SMEM, int MS>
void launch_one(const Params &p, cudaStream_t s, int sm_count) {
    const size_t smem = SMEM ? tables_smem_bytes(p.t) : 0;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(reach_kernel<SMEM, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reach_kernel<SMEM, MS>, kBlockThreads, smem);
    uint64_t want = (p.c + kBlockThreads - 1) / kBlockThreads;
    uint64_t blocks = std::min<uint64_t>(want, (uint64_t)std::max(per_sm, 1) * sm_count);
    reach_kernel<SMEM, MS><<<(uint32_t)std::max<uint64_t>(blocks, 1), kBlockThreads, smem, s>>>(p);
}

template <bool SMEM>
bool launch_ms(const Params &p, cudaStream_t s, uint32_t ms, int sm_count) {
    if (SMEM && ms <= 2) launch_one<SMEM, 2>(p, s, sm_count);
    else if (SMEM && ms <= 4) launch_one<SMEM, 4>(p, s, sm_count);
    else if (ms <= 8) launch_one<SMEM, 8>(p, s, sm_count);
    else if (SMEM && ms <= 16) launch_one<SMEM, 16>(p, s, sm_count);
    else if (ms <= 32) launch_one<SMEM, 32>(p, s, sm_count);
    else return false;
    return true;
}

}  // namespace

bool launch_reach(const Params &p, cudaStream_t s, uint32_t ms, int sm_count) {
    return p.smem_tables ? launch_ms<true>(p, s, ms, sm_count) : launch_ms<false>(p, s, ms, sm_count);
}

}  // namespace slpf
