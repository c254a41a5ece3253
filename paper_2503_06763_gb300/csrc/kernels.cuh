// Device-side definitions shared by the parse kernels (reach_*.cu, join.cu,
// merge.cu) and the host launchers (api.cu, batch.cu).
//
// Geometry of one parse (arXiv 2503.06763, Sect. 3.2, split phase):
//   text x[0..n), n >= 1; chunks y_i = x[i*k, min((i+1)*k, n)), k a multiple of
//   L = 64, c = ceil(n/k) chunks of S = k/L sub-chunks; SLPF columns r = 0..n
//   (column r lies between bytes r-1 and r).
//   Column groups g = 0 .. Gc-1, Gc = floor(n/L) + 1: group g holds columns
//   64g .. min(64g+63, n), so each group's output starts on a 64-column
//   boundary of the output array.
//   Checkpoints: FC[g] = forward state B at position 64g,
//                BC[g] = backward state B̂ at position min(64g+64, n).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <utility>

#include "re_internal.h"

namespace slpf {

constexpr int kMaxW = 64;           // segments per column <= 4096
constexpr uint32_t kBlockThreads = 256;     // build & merge
constexpr uint32_t kChunkThreads = 128;     // batch reach and recognizer reach blocks
constexpr uint32_t kFixupThreads = 256;     // fix-up blocks: one thread per chunk and direction
constexpr uint32_t kRecBounds = 32;   // boundaries recorded per chunk and direction before runs meet
constexpr uint32_t kRecEntries = 96;  // (state, slot set) entries recorded per chunk and direction

enum Flag { FLAG_FFAIL = 0, FLAG_BFAIL = 1, FLAG_INTERNAL = 2, FLAG_DONE = 3, FLAG_TIMEOUT = 4, FLAG_COUNT = 5 };

enum { SHARD_PREV = 1, SHARD_NEXT = 2 };

// Join as a scan over chunk maps (join.cu): used when both classic DFAs have
// at most kScanStates states (ids fit a byte), so a chunk's map over them is
// a byte table.
constexpr uint32_t kScanStates = 256;
constexpr uint32_t kScanRounds = 40;        // pointer-jumping rounds (chains up to 2^40 chunks)
constexpr uint32_t kScanWords = 64;         // barrier words + per-round counters
constexpr uint32_t kScanGeneral = 2 + kScanRounds;   // scan word: chunks whose output depends on their input

struct Work {                       // device workspace, carved from the caller's buffer
    uint32_t *Rf, *Rb;              // [c][msf], [c][msb] end state of each speculation slot
    uint32_t *FJ, *BJ;              // [c+1]: state at the boundary before chunk i
    uint32_t *FC, *BC;              // [Gc] checkpoints
    uint32_t *fconv, *bconv;        // [c] first / last sub-chunk boundary the reach runs agree on
    uint32_t *fkind, *bkind;        // [c] 0: every live slot ends in one state, 1: several
    uint32_t *fnrec, *bnrec;        // [c] boundaries recorded (from the chunk's start / end)
    uint32_t *fhit, *bhit;          // [c] slots the exact input state J_{i-1} / Ĵ_{i+1} enters
    uint32_t *recFc, *recBc;        // [c][kRecBounds] runs recorded at each boundary
    uint2 *recFe, *recBe;           // [c][kRecEntries] (state, slot set) of those runs
    int32_t *flags;                 // [FLAG_COUNT]
    uint8_t *FS, *BS;               // [n+1+pad] per-position forward / backward states (mat), one byte each
    uint8_t *fTab, *bTab;           // [2][c][nfd+1], [2][c][nbd+1]: maps of chunk ranges (scan join)
    uint32_t *fLink, *bLink;        // [2][c]: chunk whose output feeds the range's map (scan join)
    uint32_t *scan;                 // [kScanWords]: grid barrier and per-round counters (scan join)
};

struct Params {
    DevTables t;
    const uint8_t *x;
    uint64_t n;
    uint32_t k, c, S;               // chunk length, chunks, sub-chunks per chunk
    uint64_t Gc;                    // column groups
    Work w;
    void *out;
    uint32_t col_bytes, kind;       // output encoding (re_slpf_kind)
    int32_t *status;
    uint32_t recognize;             // forward reach + join only
    uint32_t scan;                  // join by the pointer-jumping scan (else chains, one thread each)
    uint32_t scan_stall;            // test hook: one block of the scan never reaches its first barrier
    uint32_t mat;                   // reach writes every position's state once its runs have met; the
                                    // fix-up fills the positions before; build & merge is a gather
    uint32_t state_tma;             // reach stores its state rows through TMA (mat)
    uint32_t rvar;                  // reach shape (RE_PARSE_REACH): 1 byte tables, one direction per
                                    // block; 2 / 3 warp pairs, 3 / 2 stages; 4 one lane per chunk
    uint32_t rstages;               // TMA ring stages of the warp-pair and one-lane shapes
    uint32_t shard;                 // a slice of a longer text: SHARD_PREV, its first chunk speculates from
                                    // the byte before it (x[-1]); SHARD_NEXT, its last chunk from the
                                    // byte after it (x[len])
    uint32_t tmode;                 // TM_GLOBAL / TM_SMEM / TM_PAIR (see Tabs)
    uint32_t enc_in_smem;           // encoder table (DICT pair table, DENSE bitsets) in shared memory
    uint32_t merge_reg;             // one-byte tables: build & merge stages the classic-DFA rows and the
                                    // encoder over classic-DFA state pairs only, and keeps the first
                                    // half of each builder's states in registers
    uint32_t out_tma;               // full column groups leave through TMA tensor stores
    uint32_t text_tma;              // reach reads full chunks through TMA tiles
    const CUtensorMap *tmaps;       // batch texts: device copies of the text, FS and BS tensor maps
    uint32_t c_full;                // chunks of exactly k bytes (rows of the text tensor map)
    uint64_t Gfast;                 // groups g with 64g + 64 <= n (computed on the fast path)
};

// TMA maps of the per-position state arrays FS and BS (mat): rows of k
// positions (one chunk), boxes of 32 rows x 64 positions, SWIZZLE_64B.
struct StateMaps {
    CUtensorMap f, b;
};

// Texts of one batch that share one compiled RE (re_parse_batch).  Every
// phase kernel of the group takes its units of work -- 32-chunk reach tiles,
// chunks, 32-group merge tiles -- in one flat index space per kind: the
// prefix sums below give each text's first unit, and a unit finds its text
// by binary search.  Reach and merge tiles are handed out by atomic work
// counters; texts come longest chunks first, so the longest reach tiles
// start first.  A text's parameters (geometry, text, workspace and output
// pointers) are a Params in device memory.  The group shares tables, table
// mode and output encoding, so each block stages the tables once.
struct BatchGroup {
    DevTables t;
    const Params *texts;            // [nt]
    const uint64_t *chunk_base;     // [nt+1] chunks before each text
    const uint64_t *rtile_base;     // [nt+1] reach tiles (32 chunks) before each text
    const uint64_t *mtile_base;     // [nt+1] merge tiles (32 column groups) before each text
    uint32_t *queue;                // [kQueues] work counters, zeroed before the group runs
    uint64_t chunks, n_reach, n_merge;
    uint32_t nt, recognize;
};
enum Queue { Q_REACH = 0, Q_MERGE = 1, kQueues = 4 };

// The text owning flat unit j: the last text whose first unit is <= j.
__device__ __forceinline__ uint32_t text_of(const uint64_t *base, uint32_t nt, uint64_t j) {
    uint32_t lo = 0, hi = nt;                    // base[lo] <= j < base[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (__ldg(base + mid) <= j) lo = mid; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint32_t chunk_len(const Params &p, uint32_t i) {
    uint64_t rest = p.n - (uint64_t)i * p.k;
    return rest < p.k ? (uint32_t)rest : p.k;
}

__device__ __forceinline__ bool any_and(const uint64_t *a, const uint64_t *b, uint32_t W) {
    for (uint32_t w = 0; w < W; ++w)
        if (__ldg(a + w) & __ldg(b + w)) return true;
    return false;
}

// Slots of the class pair pr that input state S enters (bit j: slot j).
__device__ __forceinline__ uint32_t slot_hits(const DevTables &t, bool fwd, uint32_t pr, uint32_t S) {
    const uint8_t *of = fwd ? t.fSlotOf : t.bSlotOf;
    if (of) {                                    // starts from every DFA state: S enters its own slot only
        const uint32_t n = fwd ? t.nf : t.nb;
        const uint32_t j = S < n ? __ldg(of + (size_t)pr * n + S) : 0xFFu;
        return j == 0xFFu ? 0u : 1u << j;
    }
    const uint32_t W = t.W;
    const uint32_t m = __ldg((fwd ? t.fSlotCount : t.bSlotCount) + pr);
    const uint32_t ms = fwd ? t.msf : t.msb;
    const uint64_t *mask = (fwd ? t.fSlotMask : t.bSlotMask) + (size_t)pr * ms * W;
    const uint64_t *sb = (fwd ? t.fBits : t.bBits) + (size_t)S * W;
    uint32_t H = 0;
    for (uint32_t j = 0; j < m; ++j)
        if (any_and(sb, mask + (size_t)j * W, W)) H |= 1u << j;
    return H;
}

// 16 text bytes from x[at..at+16); bytes at or past n read as 0.
__device__ __forceinline__ uint4 load16(const uint8_t *x, uint64_t n, uint64_t at) {
    if (at + 16 <= n) return __ldg(reinterpret_cast<const uint4 *>(x + at));
    uint32_t w[4] = {0, 0, 0, 0};
    for (int j = 0; j < 16; ++j)
        if (at + j < n) w[j >> 2] |= (uint32_t)__ldg(x + at + j) << (8 * (j & 3));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ uint32_t byte_of(const uint4 &v, int u) {   // u in 0..15, unrolled
    uint32_t w = (u < 4) ? v.x : (u < 8) ? v.y : (u < 12) ? v.z : v.w;
    return (w >> (8 * (u & 3))) & 0xFFu;
}

// Empty text: one column C_0 = I ∩ F, and the status.
__device__ inline void empty_text(const Params &p) {
    const DevTables &t = p.t;
    const uint64_t v = t.fBits[(size_t)t.fI * t.W] & t.bBits[(size_t)t.bF * t.W];
    bool meet = false;
    for (uint32_t w = 0; w < t.W; ++w) meet |= (t.fBits[(size_t)t.fI * t.W + w] & t.bBits[(size_t)t.bF * t.W + w]) != 0;
    *p.status = meet ? RE_OK : RE_REJECTED;
    if (!p.out) return;
    if (p.kind == RE_SLPF_PAIRS) {                              // (I, F), or (0, 0) when they do not meet
        if (p.col_bytes == 4) reinterpret_cast<uint32_t *>(p.out)[0] = meet ? (t.fI | (t.bF << 16)) : 0u;
        else reinterpret_cast<uint64_t *>(p.out)[0] = meet ? ((uint64_t)t.fI | ((uint64_t)t.bF << 32)) : 0ull;
    } else if (p.kind == RE_SLPF_DICT) {
        const uint32_t d = meet ? t.pt[(size_t)t.fI * t.nb + t.bF] : 0u;
        if (p.col_bytes == 1) reinterpret_cast<uint8_t *>(p.out)[0] = (uint8_t)d;
        else if (p.col_bytes == 2) reinterpret_cast<uint16_t *>(p.out)[0] = (uint16_t)d;
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

// ---------------------------------------------------------------- tables
// Transition tables in one of three modes (template parameter TM):
//   TM_GLOBAL: one-byte tables read from global memory (u32 states);
//   TM_SMEM:   one-byte tables staged in shared memory as u16;
//   TM_PAIR:   two-byte tables in shared memory, one 32-bit entry per
//              (state, class pair): low half the state after the first byte
//              consumed, high half after both (used when ncls^2 is small);
//   TM_SMEM8:  one-byte tables in shared memory as u8 (at most 256 states per
//              direction; the reach's choice for larger class alphabets, a
//              quarter of the u32 footprint, so more blocks fit an SM);
//   TM_BYTE8:  tables indexed by the text byte itself (not its class), u8,
//              rows of kByteRow bytes (256 entries and 4 of padding, which
//              puts equal bytes of different states in different banks); a
//              reach block stages one direction's table (about 65 KB).
//   TM_BYTE7:  the same with rows of the bytes below 128 only (kAsciiRow
//              bytes: 128 entries and 4 of padding, so entry (s, b) sits in
//              bank (s + b / 4) mod 32 as in TM_BYTE8); the walk first
//              replaces every byte >= 128 by a byte below 128 of its class
//              (DevTables::hirep), which every class holding one has.
// Row s, column = byte class (or class pair c1*ncls + c2 for the left and
// right byte of the pair).  A forward pair consumes c1 then c2, a backward
// pair c2 then c1.
enum { TM_GLOBAL = 0, TM_SMEM = 1, TM_PAIR = 2, TM_SMEM8 = 3, TM_BYTE8 = 4, TM_BYTE7 = 5 };
constexpr uint32_t kByteRow = 260;
constexpr uint32_t kAsciiRow = 132;

struct Tabs {
    const uint8_t *cls;
    const uint16_t *f16, *b16;
    const uint8_t *f8, *b8;
    const uint32_t *f32, *b32;
    const uint32_t *f2, *b2;
    uint32_t ncls, nc2;
    uint32_t rowb, nf, magic;       // reach in pair mode: run-state encoding (see reach_impl.cuh)
    const uint8_t *rep;             // TM_BYTE7: [128] representative of byte b + 128 (shared memory)
};

template <int TM>
__device__ __forceinline__ uint32_t fnext(const Tabs &T, uint32_t s, uint32_t c) {
    if (TM == TM_SMEM) return T.f16[s * T.ncls + c];
    if (TM == TM_SMEM8) return T.f8[s * T.ncls + c];
    if (TM == TM_BYTE8) return T.f8[s * kByteRow + c];          // c is the byte itself
    if (TM == TM_BYTE7) return T.f8[s * kAsciiRow + c];         // c is the byte, folded below 128
    if (TM == TM_PAIR) return T.f2[s * T.nc2 + c * T.ncls] & 0xFFFFu;
    return __ldg(T.f32 + (size_t)s * T.ncls + c);
}
template <int TM>
__device__ __forceinline__ uint32_t bnext(const Tabs &T, uint32_t s, uint32_t c) {
    if (TM == TM_SMEM) return T.b16[s * T.ncls + c];
    if (TM == TM_SMEM8) return T.b8[s * T.ncls + c];
    if (TM == TM_BYTE8) return T.b8[s * kByteRow + c];
    if (TM == TM_BYTE7) return T.b8[s * kAsciiRow + c];
    if (TM == TM_PAIR) return T.b2[s * T.nc2 + c] & 0xFFFFu;
    return __ldg(T.b32 + (size_t)s * T.ncls + c);
}
__device__ __forceinline__ uint32_t fpair(const Tabs &T, uint32_t s, uint32_t cp) { return T.f2[s * T.nc2 + cp]; }
__device__ __forceinline__ uint32_t bpair(const Tabs &T, uint32_t s, uint32_t cp) { return T.b2[s * T.nc2 + cp]; }

template <int TM>
__device__ __forceinline__ uint32_t clsof(const Tabs &T, uint32_t b) {
    if (TM == TM_BYTE8 || TM == TM_BYTE7) return b;             // the tables are indexed by the byte
    if (TM != TM_GLOBAL) return T.cls[b];
    return __ldg(T.cls + b);
}
// The byte class itself (slot selection), in every table mode.
template <int TM>
__device__ __forceinline__ uint32_t class_of(const Tabs &T, const DevTables &t, uint32_t b) {
    if (TM == TM_BYTE8 || TM == TM_BYTE7) return __ldg(t.cls + b);
    return clsof<TM>(T, b);
}

// TM_BYTE7: bytes >= 128 of a word replaced by their representatives below
// 128 (one shared-memory lookup per such byte; none for ASCII text).
__device__ __forceinline__ uint32_t fold_word(const uint8_t *rep, uint32_t w) {
    for (uint32_t hi = w & 0x80808080u; hi; hi &= hi - 1) {
        const uint32_t sh = (uint32_t)__ffs(hi) - 8;             // the byte's lowest bit
        w = (w & ~(0xFFu << sh)) | ((uint32_t)rep[(w >> sh) & 0x7Fu] << sh);
    }
    return w;
}
__device__ __forceinline__ uint4 fold_high_bytes(const uint8_t *rep, uint4 x) {
    if (((x.x | x.y | x.z | x.w) & 0x80808080u) == 0) return x;
    return make_uint4(fold_word(rep, x.x), fold_word(rep, x.y), fold_word(rep, x.z), fold_word(rep, x.w));
}

// Stage the byte-indexed tables of the directions asked for (block-wide;
// ends with __syncthreads).  Returns the end of the used area.
__device__ inline uint8_t *stage_byte8(const DevTables &t, uint8_t *sm, Tabs &T, bool fwd, bool bwd,
                                       bool ascii = false) {
    T.ncls = t.ncls;
    T.nc2 = t.ncls * t.ncls;
    T.cls = t.cls;
    T.f32 = t.fT;
    T.b32 = t.bT;
    T.f16 = T.b16 = nullptr;
    T.f2 = T.b2 = nullptr;
    T.f8 = T.b8 = nullptr;
    uint8_t *at = sm;
    for (int d = 0; d < 2; ++d) {
        if (!(d == 0 ? fwd : bwd)) continue;
        const uint8_t *src = d == 0 ? t.fbyte : t.bbyte;
        const uint32_t n = d == 0 ? t.nf : t.nb;
        uint32_t *dst = reinterpret_cast<uint32_t *>(at);
        const uint32_t *src32 = reinterpret_cast<const uint32_t *>(src);
        if (ascii) {   // row s: the 32 words of bytes 0..127, then one word of padding
            for (uint32_t q = threadIdx.x; q < n * 32; q += blockDim.x)
                dst[(q >> 5) * (kAsciiRow / 4) + (q & 31)] = __ldg(src32 + (q >> 5) * 64 + (q & 31));
        } else {       // row s: 64 words of entries, then one word of padding
            for (uint32_t q = threadIdx.x; q < n * 64; q += blockDim.x)
                dst[(q >> 6) * (kByteRow / 4) + (q & 63)] = __ldg(src32 + q);
        }
        (d == 0 ? T.f8 : T.b8) = at;
        at += (((size_t)n * (ascii ? kAsciiRow : kByteRow)) + 15) & ~(size_t)15;
    }
    T.rep = nullptr;
    if (ascii) {
        for (uint32_t q = threadIdx.x; q < 32; q += blockDim.x)
            reinterpret_cast<uint32_t *>(at)[q] = __ldg(reinterpret_cast<const uint32_t *>(t.hirep) + q);
        T.rep = at;
        at += 128;
    }
    __syncthreads();
    return at;
}
__host__ __device__ inline size_t byte8_smem_bytes(const DevTables &t, bool fwd, bool bwd, bool ascii = false) {
    const size_t row = ascii ? kAsciiRow : kByteRow;
    return (fwd ? (((size_t)t.nf * row) + 15) & ~(size_t)15 : 0) +
           (bwd ? (((size_t)t.nb * row) + 15) & ~(size_t)15 : 0) + (ascii ? 128 : 0);
}

// Bytes of shared memory used by stage_tables.
__host__ __device__ inline size_t tables_smem_bytes(const DevTables &t, int tm) {
    if (tm == TM_GLOBAL) return 0;
    size_t a = 256;
    if (tm == TM_SMEM || tm == TM_SMEM8) {
        const size_t eb = tm == TM_SMEM ? 2 : 1;
        a += ((size_t)t.nf * t.ncls * eb + 15) & ~(size_t)15;
        a += ((size_t)t.nb * t.ncls * eb + 15) & ~(size_t)15;
    } else {
        a += (size_t)(t.nf + t.nb) * t.ncls * t.ncls * 4;
        a = (a + 15) & ~(size_t)15;                  // keep the next area 16-byte aligned
    }
    return a;
}

// Stage the byte-class map and the transition tables in shared memory
// (block-wide; ends with __syncthreads).  Returns the end of the used area.
template <int TM>
__device__ uint8_t *stage_tables(const DevTables &t, uint8_t *sm, Tabs &T) {
    T.ncls = t.ncls;
    T.nc2 = t.ncls * t.ncls;
    T.f32 = t.fT;
    T.b32 = t.bT;
    T.f16 = T.b16 = nullptr;
    T.f8 = T.b8 = nullptr;
    T.f2 = T.b2 = nullptr;
    if (TM == TM_GLOBAL) {
        T.cls = t.cls;
        return sm;
    }
    uint8_t *cls = sm;
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) cls[i] = __ldg(t.cls + i);
    T.cls = cls;
    if (TM == TM_SMEM) {
        uint16_t *f16 = reinterpret_cast<uint16_t *>(sm + 256);
        const size_t fsz = (size_t)t.nf * t.ncls;
        uint16_t *b16 = reinterpret_cast<uint16_t *>(sm + 256 + ((fsz * 2 + 15) & ~(size_t)15));
        const size_t bsz = (size_t)t.nb * t.ncls;
        for (size_t i = threadIdx.x; i < fsz; i += blockDim.x) f16[i] = (uint16_t)__ldg(t.fT + i);
        for (size_t i = threadIdx.x; i < bsz; i += blockDim.x) b16[i] = (uint16_t)__ldg(t.bT + i);
        T.f16 = f16;
        T.b16 = b16;
        __syncthreads();
        return reinterpret_cast<uint8_t *>(b16) + ((bsz * 2 + 15) & ~(size_t)15);
    }
    if (TM == TM_SMEM8) {
        uint8_t *f8 = sm + 256;
        const size_t fsz = (size_t)t.nf * t.ncls;
        uint8_t *b8 = f8 + ((fsz + 15) & ~(size_t)15);
        const size_t bsz = (size_t)t.nb * t.ncls;
        for (size_t i = threadIdx.x; i < fsz; i += blockDim.x) f8[i] = (uint8_t)__ldg(t.fT + i);
        for (size_t i = threadIdx.x; i < bsz; i += blockDim.x) b8[i] = (uint8_t)__ldg(t.bT + i);
        T.f8 = f8;
        T.b8 = b8;
        __syncthreads();
        return b8 + ((bsz + 15) & ~(size_t)15);
    }
    const uint32_t nc2 = t.ncls * t.ncls;
    uint32_t *f2 = reinterpret_cast<uint32_t *>(sm + 256);
    uint32_t *b2 = f2 + (size_t)t.nf * nc2;
    // copy the two-byte tables built at compile time (16-byte vectors where possible)
    const size_t nwords = (size_t)(t.nf + t.nb) * nc2;
    const bool contiguous = t.b2 == t.f2 + (size_t)t.nf * nc2;
    if (contiguous && ((reinterpret_cast<uintptr_t>(t.f2) & 15) == 0)) {
        const uint4 *src = reinterpret_cast<const uint4 *>(t.f2);
        uint4 *dst = reinterpret_cast<uint4 *>(f2);
        for (size_t i = threadIdx.x; i < nwords / 4; i += blockDim.x) dst[i] = __ldg(src + i);
        for (size_t i = (nwords / 4) * 4 + threadIdx.x; i < nwords; i += blockDim.x) f2[i] = __ldg(t.f2 + i);
    } else {
        for (size_t i = threadIdx.x; i < (size_t)t.nf * nc2; i += blockDim.x) f2[i] = __ldg(t.f2 + i);
        for (size_t i = threadIdx.x; i < (size_t)t.nb * nc2; i += blockDim.x) b2[i] = __ldg(t.b2 + i);
    }
    T.f2 = f2;
    T.b2 = b2;
    __syncthreads();
    // end of the used area, rounded up to 16 bytes exactly as in tables_smem_bytes
    const size_t used = (256 + (size_t)(t.nf + t.nb) * nc2 * 4 + 15) & ~(size_t)15;
    return sm + used;
}

// ---------------------------------------------------------------- TMA (bulk async copies)
__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}
// Bring the 128-byte line holding addr into L2 (no register result).
__device__ __forceinline__ void prefetch_l2(const void *addr) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(addr));
}

// Make this thread's generic-proxy shared-memory writes visible to the async proxy.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 2D tiled store shared -> global (box from the tensor map), coordinates {x, y}.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int32_t x, int32_t y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                 :: "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(src) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// A tensor map read from global memory (a batch text's): acquire it for the
// tensor-map proxy before the first copy that uses it.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" :: "l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}
// 2D tiled load global -> shared, completion counted on an mbarrier (bytes).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int32_t x, int32_t y, uint32_t bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}
// One bounded wait on phase parity `ph`: true once that phase has completed.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t ph) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(bar), "r"(ph) : "memory");
    return ok != 0;
}
constexpr uint32_t kWaitLimit = 1u << 22;   // try_wait rounds before a wait is declared lost
// The bulk groups of this thread have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// At most one bulk group of this thread still reads shared memory.
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// The bulk groups of this thread have completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---------------------------------------------------------------- dependent launches
// The kernels of one parse after the first are launched as programmatic
// dependents of the kernel before them (sm_90 and later).  A dependent grid
// may become resident while its predecessor drains and run its prologue
// (staging immutable tables into shared memory); before it touches anything
// an earlier kernel of the parse reads or writes it executes pdl_wait(),
// which returns once the predecessor grid has completed and its memory is
// visible.  Every block of such a kernel waits before it can exit, so a
// completed grid implies that every grid before it has completed too.  In a
// kernel launched the ordinary way the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the dependent grid launch once every block of this grid has issued it
// (or exited).  Issued after pdl_wait, so at most two grids overlap.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch kernel as a programmatic dependent of the previous work on stream s.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                    Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------- launchers
// Raise a kernel's dynamic shared-memory limit once per device (the setting
// belongs to the device; *done holds one bit per device already set).  Host
// threads may race here: the bit is read and set atomically, and a thread
// that finds it clear sets the attribute again, which is harmless.
template <typename K>
inline void allow_smem(K kernel, uint64_t *done, int bytes = 200 * 1024) {
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (__atomic_load_n(done, __ATOMIC_ACQUIRE) & bit)) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    __atomic_fetch_or(done, bit, __ATOMIC_RELEASE);
}

size_t merge_extra_smem(const Params &p);
size_t merge_smem_bytes(const Params &p);
size_t mat_gather_smem(const Params &p);
// The classic-DFA part of the tables: forward states 0 .. nfd (the DFA states
// reachable from I get the first ids, and transitions from them stay among
// them), reverse states 0 .. nbd.  Build & merge only meets these states: its
// checkpoints are exact forward / backward states of the text.
__host__ __device__ inline DevTables dfa_tables(const DevTables &t) {
    DevTables c = t;
    c.nf = t.nfd + 1;
    c.nb = t.nbd + 1;
    return c;
}
bool launch_reach(const Params &p, const CUtensorMap &text_map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                  int sm_count);
// Batch group with per-position states: the byte-table reach over its tiles,
// the fix-up of the chunk heads and the gather of the columns.
bool launch_reach_batch_byte8(const BatchGroup &b, uint32_t ms, cudaStream_t s, int sm_count);
void launch_fixup_mat_batch(const BatchGroup &b, cudaStream_t s, int sm_count);
void launch_gather_batch(const BatchGroup &b, const Params &like, cudaStream_t s, int sm_count);
// Warps per direction of the byte-table reach (shape 1) on this device.
uint64_t reach_byte8_warps(const Params &p, uint32_t ms, int sm_count);
bool launch_join(const Params &p, cudaStream_t s, int sm_count);
bool launch_shard_map(const Params &p, uint8_t *d_maps, cudaStream_t s, int sm_count);
void launch_fixup(const Params &p, cudaStream_t s, int sm_count);
void launch_merge(const Params &p, const CUtensorMap &out_map, cudaStream_t s, int sm_count);
void launch_empty(const Params &p, cudaStream_t s);

// Match extraction (matches.cu).
constexpr int kMatchW = 8;                    // segment words supported (ell <= 512)

struct MatchArgs {
    const void *cols;                         // SLPF columns C_0 .. C_n
    uint32_t col_bytes, kind, W;
    uint64_t n;                               // text length (columns n + 1)
    const uint64_t *folseg;                   // [ell][W]
    const uint64_t *dict;                     // [dict_size][W] (DICT)
    const uint64_t *fbits, *bbits;            // [states][W] segment sets of the states (PAIRS)
    uint64_t open[kMatchW], close_first[kMatchW], whole[kMatchW], none[kMatchW];
    const int32_t *status;                    // parse status: anything but RE_OK gives no matches
    uint64_t *cnt;                            // [G] pairs per warp range, then their exclusive offsets
    uint64_t *bsum;                           // [ceil(G / kScanBlock)] block totals, then offsets
    uint64_t G;
    uint64_t *pairs;                          // [cap][2]
    uint64_t cap;
    uint64_t *count;
};

size_t match_workspace_bytes(uint64_t n);
void launch_matches(MatchArgs a, void *ws, cudaStream_t s);

// Batch launchers: one launch per phase for every text of the group.
void launch_batch_init(const Params *texts, uint32_t nt, uint32_t *queues, uint32_t nq, cudaStream_t s);
bool launch_reach_batch(const BatchGroup &b, uint32_t tmode, uint32_t ms, cudaStream_t s, int sm_count);
void launch_join_batch(const BatchGroup &b, cudaStream_t s);
void launch_fixup_batch(const BatchGroup &b, uint32_t tmode, cudaStream_t s, int sm_count);
void launch_merge_batch(const BatchGroup &b, const Params &like, cudaStream_t s, int sm_count);

}  // namespace slpf
