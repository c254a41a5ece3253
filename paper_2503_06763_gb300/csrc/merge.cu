// Checkpoint fix-up and build & merge (arXiv 2503.06763, Eqs. builder and
// merger, Fig. builders&merger, compose of Sect. 3.2).
//
// fix-up: for the sub-chunk boundaries a chunk's reach runs reached before
//   they agreed, walk the DFA from J_{i-1} (forward) and the reverse DFA from
//   Ĵ_{i+1} (backward) and write the exact checkpoints.
// build & merge: one thread per column group g (64 columns).  Forward
//   B_{64g+u} from FC[g] over bytes 64g.., backward B̂ from BC[g] over the same
//   bytes right to left, and the clean column C_r = B_r ∩ B̂_r written in the
//   requested encoding (DENSE bitset, or DICT index through the pair table
//   built at compile time).  The forward states of a group stay in registers
//   (the fused builder & merger of Fig. builders&merger keeps B in M and
//   intersects during the backward scan; here M is the register file).
#include "kernels.cuh"

namespace slpf {
namespace {

// ------------------------------------------------------------------ fix-up
template <bool SMEM>
__global__ void __launch_bounds__(kBlockThreads) fixup_kernel(Params p) {
    extern __shared__ __align__(16) uint8_t sm[];
    Tabs T;
    stage_tables<SMEM>(p, sm, T);
    if (*p.status != RE_OK) return;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < p.c; i += stride) {
        const uint64_t base = (uint64_t)i * p.k;
        const uint32_t len = chunk_len(p, i);
        const uint32_t nsub = (len + 63) / 64;
        const uint32_t fcs = p.w.fconv[i], bcs = p.w.bconv[i];
        const uint32_t fsteps = fcs > 1 ? (fcs - 1) * 64 : 0;            // bytes [0, fsteps)
        const uint32_t bstop = (bcs + 1) * 64;                            // bytes [bstop, len) backwards
        const uint32_t bsteps = (nsub >= 2 && bcs + 1 <= nsub - 1) ? len - bstop : 0;
        uint32_t sF = p.w.FJ[i], sB = p.w.BJ[i + 1];
        const uint32_t steps = max(fsteps, bsteps);
        for (uint32_t s = 0; s < steps; ++s) {
            if (s < fsteps) {
                const uint32_t t = s;
                sF = fnext<SMEM>(T, sF, clsof<SMEM>(T, __ldg(p.x + base + t)));
                if (((t + 1) & 63) == 0) p.w.FC[(uint64_t)i * p.S + (t + 1) / 64] = sF;
            }
            if (s < bsteps) {
                const uint32_t t = len - 1 - s;
                sB = bnext<SMEM>(T, sB, clsof<SMEM>(T, __ldg(p.x + base + t)));
                if ((t & 63) == 0) p.w.BC[(uint64_t)i * p.S + t / 64 - 1] = sB;
            }
        }
    }
}

// ------------------------------------------------------------------ encodings
enum { ENC_D1 = 1, ENC_D2 = 2, ENC_D4 = 4, ENC_D8 = 8, ENC_X2 = 0x12, ENC_X4 = 0x14 };

struct Enc {
    const uint64_t *fbits, *bbits;   // DENSE: segment set of each state (W == 1)
    const uint16_t *pt16;            // DICT: pair table in shared memory (u16)
    const uint32_t *pt32;            // DICT: pair table (u32; shared or global)
    uint32_t nbd1, nfd, nbd;
};

template <int E>
__device__ __forceinline__ uint32_t enc_lo(const Enc &e, uint32_t f, uint32_t b, bool &bad) {
    if (E == ENC_X2 || E == ENC_X4) {
        bad |= (f > e.nfd) | (b > e.nbd);
        f = min(f, e.nfd);
        b = min(b, e.nbd);
        const uint32_t at = f * e.nbd1 + b;
        return e.pt16 ? (uint32_t)e.pt16[at] : (e.pt32 == nullptr ? 0u : e.pt32[at]);
    }
    return (uint32_t)(e.fbits[f] & e.bbits[b]);
}
__device__ __forceinline__ uint64_t enc_d8(const Enc &e, uint32_t f, uint32_t b) { return e.fbits[f] & e.bbits[b]; }

template <int E>
__device__ __forceinline__ void store_col(void *out, uint64_t r, uint64_t v) {
    if (E == ENC_D1) reinterpret_cast<uint8_t *>(out)[r] = (uint8_t)v;
    else if (E == ENC_D2 || E == ENC_X2) reinterpret_cast<uint16_t *>(out)[r] = (uint16_t)v;
    else if (E == ENC_D4 || E == ENC_X4) reinterpret_cast<uint32_t *>(out)[r] = (uint32_t)v;
    else reinterpret_cast<uint64_t *>(out)[r] = v;
}

constexpr int bytes_of(int E) { return (E == ENC_X2) ? 2 : (E == ENC_X4) ? 4 : E; }

// Full group: 64 columns, forward 63 steps, backward 64 steps, all unrolled.
template <bool SMEM, int E>
__device__ __forceinline__ void group_full(const Params &p, const Tabs &T, const Enc &e, uint64_t g, bool &bad) {
    const uint64_t pos = g * 64;
    uint4 xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) xv[q] = __ldg(reinterpret_cast<const uint4 *>(p.x + pos) + q);
    uint32_t f = p.w.FC[g];
    uint32_t b = p.w.BC[g];
    if (f == kUnknown || b == kUnknown) { bad = true; f = 0; b = 0; }   // never index with the sentinel
    // forward states B_{pos+u}, two 16-bit states per register when the tables allow
    constexpr bool PACK = SMEM;                      // shared-memory tables: state ids < 65536
    uint32_t F[PACK ? 32 : 64];
    {
        uint32_t cur = f;
#pragma unroll
        for (int u = 0; u < 64; ++u) {
            if (u > 0) cur = fnext<SMEM>(T, cur, clsof<SMEM>(T, byte_of(xv[(u - 1) >> 4], (u - 1) & 15)));
            if (PACK) {
                if (u & 1) F[u >> 1] |= cur << 16;
                else F[u >> 1] = cur;
            } else {
                F[u] = cur;
            }
        }
    }
    auto fwd_at = [&](int u) -> uint32_t { return PACK ? ((F[u >> 1] >> (16 * (u & 1))) & 0xFFFFu) : F[u]; };
    constexpr int CB = bytes_of(E);
    // backward walk from the right end; columns are packed and stored in 16-byte
    // vectors as soon as a vector is complete (stores run from the group's end)
    uint8_t *gout = reinterpret_cast<uint8_t *>(p.out) + pos * CB;
    if constexpr (CB == 8) {
        uint64_t hi = 0;
#pragma unroll
        for (int u = 63; u >= 0; --u) {
            b = bnext<SMEM>(T, b, clsof<SMEM>(T, byte_of(xv[u >> 4], u & 15)));
            const uint64_t v = enc_d8(e, fwd_at(u), b);
            if (u & 1) hi = v;
            else reinterpret_cast<uint4 *>(gout)[u >> 1] =
                make_uint4((uint32_t)v, (uint32_t)(v >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
        }
    } else {
        constexpr int PER = 4 / CB;                  // columns per 32-bit word
        uint32_t word = 0, w4[4];
#pragma unroll
        for (int u = 63; u >= 0; --u) {
            b = bnext<SMEM>(T, b, clsof<SMEM>(T, byte_of(xv[u >> 4], u & 15)));
            uint32_t v = enc_lo<E>(e, fwd_at(u), b, bad);
            if (CB < 4) v &= (1u << (8 * CB)) - 1;
            word |= v << (8 * CB * (u % PER));
            if (u % PER == 0) {
                const int w = u / PER;               // word index within the group
                w4[w & 3] = word;
                word = 0;
                if ((w & 3) == 0) reinterpret_cast<uint4 *>(gout)[w >> 2] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
        }
    }
}

// Last group (fewer than 64 columns or no byte after it): plain loops.
template <bool SMEM, int E>
__device__ void group_tail(const Params &p, const Tabs &T, const Enc &e, uint64_t g, bool &bad) {
    const uint64_t pos = g * 64;
    const uint64_t nleft = p.n + 1 - pos;
    const uint32_t ncol = nleft < 64 ? (uint32_t)nleft : 64u;
    uint32_t F[64], B[64];
    uint32_t f = p.w.FC[g], b = p.w.BC[g];
    if (f == kUnknown || b == kUnknown) { bad = true; f = 0; b = 0; }
    F[0] = f;
    for (uint32_t u = 1; u < ncol; ++u) F[u] = fnext<SMEM>(T, F[u - 1], clsof<SMEM>(T, __ldg(p.x + pos + u - 1)));
    if (pos + 64 <= p.n) b = bnext<SMEM>(T, b, clsof<SMEM>(T, __ldg(p.x + pos + 63)));
    B[ncol - 1] = b;
    for (int u = (int)ncol - 2; u >= 0; --u) B[u] = bnext<SMEM>(T, B[u + 1], clsof<SMEM>(T, __ldg(p.x + pos + u)));
    for (uint32_t u = 0; u < ncol; ++u) {
        uint64_t v = bytes_of(E) == 8 ? enc_d8(e, F[u], B[u]) : (uint64_t)enc_lo<E>(e, F[u], B[u], bad);
        store_col<E>(p.out, pos + u, v);
    }
}

template <bool SMEM, int E>
__global__ void __launch_bounds__(kBlockThreads, 2) merge_kernel(Params p) {
    extern __shared__ __align__(16) uint8_t sm[];
    Tabs T;
    uint8_t *rest = stage_tables<SMEM>(p, sm, T);
    Enc e{};
    const DevTables &t = p.t;
    e.nbd1 = t.nbd + 1; e.nfd = t.nfd; e.nbd = t.nbd;
    if (E == ENC_X2 || E == ENC_X4) {
        if (p.pt_in_smem) {
            const size_t cnt = (size_t)(t.nfd + 1) * (t.nbd + 1);
            if (E == ENC_X2) {
                uint16_t *pt = reinterpret_cast<uint16_t *>(rest);
                for (size_t i = threadIdx.x; i < cnt; i += blockDim.x) pt[i] = (uint16_t)__ldg(t.pt + i);
                e.pt16 = pt;
            } else {
                uint32_t *pt = reinterpret_cast<uint32_t *>(rest);
                for (size_t i = threadIdx.x; i < cnt; i += blockDim.x) pt[i] = __ldg(t.pt + i);
                e.pt32 = pt;
            }
        } else {
            e.pt32 = t.pt;
        }
    } else {
        uint64_t *fb = reinterpret_cast<uint64_t *>(rest);
        uint64_t *bb = fb + t.nf;
        for (uint32_t i = threadIdx.x; i < t.nf; i += blockDim.x) fb[i] = __ldg(t.fBits + i);
        for (uint32_t i = threadIdx.x; i < t.nb; i += blockDim.x) bb[i] = __ldg(t.bBits + i);
        e.fbits = fb; e.bbits = bb;
    }
    __syncthreads();
    const bool ok = *p.status == RE_OK;
    bool bad = false;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < p.Gc; g += stride) {
        if (!ok) {                                           // rejected text: every column is empty
            const uint64_t pos = g * 64;
            const uint64_t nleft = p.n + 1 - pos;
    const uint32_t ncol = nleft < 64 ? (uint32_t)nleft : 64u;
            for (uint32_t u = 0; u < ncol; ++u) store_col<E>(p.out, pos + u, 0);
            continue;
        }
        if (g * 64 + 64 <= p.n) group_full<SMEM, E>(p, T, e, g, bad);
        else group_tail<SMEM, E>(p, T, e, g, bad);
    }
    if (bad) atomicExch(p.status, RE_E_INTERNAL);
}

// Empty text: one column C_0 = I ∩ F.
__global__ void empty_text_kernel(Params p) {
    const DevTables &t = p.t;
    const uint64_t v = t.fBits[(size_t)t.fI * t.W] & t.bBits[(size_t)t.bF * t.W];
    bool meet = false;
    for (uint32_t w = 0; w < t.W; ++w) meet |= (t.fBits[(size_t)t.fI * t.W + w] & t.bBits[(size_t)t.bF * t.W + w]) != 0;
    *p.status = meet ? RE_OK : RE_REJECTED;
    if (!p.out) return;
    if (p.kind == RE_SLPF_DICT) {
        const uint32_t d = meet ? t.pt[(size_t)t.fI * (t.nbd + 1) + t.bF] : 0u;
        if (p.col_bytes == 2) reinterpret_cast<uint16_t *>(p.out)[0] = (uint16_t)d;
        else reinterpret_cast<uint32_t *>(p.out)[0] = d;
    } else {
        switch (p.col_bytes) {
            case 1: reinterpret_cast<uint8_t *>(p.out)[0] = (uint8_t)v; break;
            case 2: reinterpret_cast<uint16_t *>(p.out)[0] = (uint16_t)v; break;
            case 4: reinterpret_cast<uint32_t *>(p.out)[0] = (uint32_t)v; break;
            default: reinterpret_cast<uint64_t *>(p.out)[0] = v; break;
        }
    }
}

template <typename K>
int grid_for(K kernel, size_t smem, uint64_t items, int sm_count) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlockThreads, smem);
    const uint64_t want = (items + kBlockThreads - 1) / kBlockThreads;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(per_sm, 1) * sm_count));
}

template <bool SMEM, int E>
void merge_one(const Params &p, cudaStream_t s, int sm_count) {
    const size_t smem = (SMEM ? tables_smem_bytes(p.t) : 0) + merge_extra_smem(p);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(merge_kernel<SMEM, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    merge_kernel<SMEM, E><<<grid_for(merge_kernel<SMEM, E>, smem, p.Gc, sm_count), kBlockThreads, smem, s>>>(p);
}

template <bool SMEM>
void merge_enc(const Params &p, cudaStream_t s, int sm_count) {
    if (p.kind == RE_SLPF_DICT) {
        if (p.col_bytes == 2) merge_one<SMEM, ENC_X2>(p, s, sm_count);
        else merge_one<SMEM, ENC_X4>(p, s, sm_count);
    } else {
        switch (p.col_bytes) {
            case 1: merge_one<SMEM, ENC_D1>(p, s, sm_count); break;
            case 2: merge_one<SMEM, ENC_D2>(p, s, sm_count); break;
            case 4: merge_one<SMEM, ENC_D4>(p, s, sm_count); break;
            default: merge_one<SMEM, ENC_D8>(p, s, sm_count); break;
        }
    }
}

template <bool SMEM>
void fixup_one(const Params &p, cudaStream_t s, int sm_count) {
    const size_t smem = SMEM ? tables_smem_bytes(p.t) : 0;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(fixup_kernel<SMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    fixup_kernel<SMEM><<<grid_for(fixup_kernel<SMEM>, smem, p.c, sm_count), kBlockThreads, smem, s>>>(p);
}

}  // namespace

size_t merge_extra_smem(const Params &p) {
    const DevTables &t = p.t;
    if (p.kind == RE_SLPF_DICT)
        return p.pt_in_smem ? (size_t)(t.nfd + 1) * (t.nbd + 1) * p.col_bytes : 0;
    return (size_t)(t.nf + t.nb) * 8;
}

void launch_fixup(const Params &p, cudaStream_t s, int sm_count) {
    if (p.smem_tables) fixup_one<true>(p, s, sm_count);
    else fixup_one<false>(p, s, sm_count);
}

void launch_merge(const Params &p, cudaStream_t s, int sm_count) {
    if (p.smem_tables) merge_enc<true>(p, s, sm_count);
    else merge_enc<false>(p, s, sm_count);
}

void launch_empty(const Params &p, cudaStream_t s) { empty_text_kernel<<<1, 1, 0, s>>>(p); }

}  // namespace slpf
