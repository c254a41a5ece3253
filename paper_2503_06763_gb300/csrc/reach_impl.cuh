// Reach phase, shared implementation included by reach_pair.cu, reach_smem.cu
// and reach_global.cu (one translation unit per table mode).
//
// Reach phase (arXiv 2503.06763, Eq. reacher).
//
// One lane per chunk y_i and direction runs the forward ME-DFA from every
// speculation slot of the chunk left to right, or the reverse ME-DFA from
// every backward slot right to left.  A parse gives the two directions of a
// 32-chunk tile to two warps (Sect. 4.1 fuses them into one task; on the GPU
// separate warps double the chains in flight); batches and the recognizer
// walk the needed directions in one warp.
// Slots are the distinct start sets after the boundary byte (a run from a
// singleton {q} reaches D_end(q) after one byte), restricted by the class of
// the byte before the boundary (the last-character filter of Sect. 6).
// Chunk 0 runs forward from I and chunk c-1 backward from F without
// speculation (J_0 = I, Ĵ_{c+1} = F, Eq. joiner).
//
// Runs are kept distinct: at every 64-byte sub-chunk boundary dead runs are
// dropped and runs in equal states are merged (equal states stay equal), each
// run carrying the set of slots it stands for.  While several runs are live
// the lane records, per boundary, the (state, slot set) of each run; the
// fix-up later turns a record into the exact state by the union of Eq. joiner
// over the slots its input enters.  Once one run is left its state is exact
// for any input that enters a live slot, and the lane writes it as a
// checkpoint (FC / BC).  At the end it writes the end state of every slot
// (R, R̂) and the first (forward) / last (backward) boundary where a single
// run was left.  Active runs drop fast after a few bytes (Sect. 4.3), so
// most of every chunk runs with one run per direction.
#pragma once

#include "kernels.cuh"

namespace slpf {
namespace reach {

// ------------------------------------------------------------------ pair-mode layout
// In pair mode (at most 16 byte classes) the reach keeps every run state as
// the byte offset of its row in one shared-memory array of two-byte
// transition rows, forward rows first:
//     forward state s  -> s * rowb,        backward state s -> (nf + s) * rowb,
// rowb = ncls^2 * 2.  An entry of row s, column (c1, c2), is the offset (a
// u16: pair-mode tables are at most 48 KB as u32, so offsets stay below 2^16)
// of the state after the byte pair, so one step is an add and a load:
//     run = *(u16 *)(sm + kRows + run + cp2),  cp2 = 2 * (c1 * ncls + c2),
// and cp2 comes from two byte-indexed class tables, H[b] = c(b) * ncls and
// L[b] = 2 * c(b), as (H[b1] << 1) + L[b2].  Two-byte entries halve the
// rows' footprint in the banks, so fewer lanes of a warp meet in one bank.  The run's state id is needed only
// at 64-byte boundaries (records, checkpoints, end states) and is the offset
// divided by rowb (a multiply-high by a reciprocal: offsets are exact
// multiples of rowb and small).  Blocks that start or end inside a chunk's
// edge step one byte at a time on state ids with the one-byte tables.
//   [0, 256) H    [256, 512) L    [512, 768) byte -> class
//   [kRows, kRows + (nf + nb) * rowb) rows, then one-byte tables (u16)
constexpr uint32_t kClsH = 0, kClsL = 256, kCls = 512, kRows = 1024;

__host__ __device__ inline size_t reach_pair_smem(const DevTables &t) {
    const size_t rows = (size_t)(t.nf + t.nb) * t.ncls * t.ncls * 2;
    return kRows + ((rows + 15) & ~(size_t)15) + (((size_t)t.nf * t.ncls * 2 + 15) & ~(size_t)15) +
           (((size_t)t.nb * t.ncls * 2 + 15) & ~(size_t)15);
}

// Stage the pair-mode layout (block-wide; ends with __syncthreads).
__device__ inline uint8_t *stage_reach_pair(const DevTables &t, uint8_t *sm, Tabs &T) {
    const uint32_t ncls = t.ncls, nc2 = ncls * ncls, rowb = nc2 * 2;
    for (uint32_t b = threadIdx.x; b < 256; b += blockDim.x) {
        const uint32_t c = __ldg(t.cls + b);
        sm[kClsH + b] = (uint8_t)(c * ncls);
        sm[kClsL + b] = (uint8_t)(2 * c);
        sm[kCls + b] = (uint8_t)c;
    }
    uint16_t *rows = reinterpret_cast<uint16_t *>(sm + kRows);
    const size_t nfw = (size_t)t.nf * nc2, nbw = (size_t)t.nb * nc2;
    for (size_t i = threadIdx.x; i < nfw; i += blockDim.x) rows[i] = (uint16_t)((__ldg(t.f2 + i) >> 16) * rowb);
    for (size_t i = threadIdx.x; i < nbw; i += blockDim.x)
        rows[nfw + i] = (uint16_t)((t.nf + (__ldg(t.b2 + i) >> 16)) * rowb);
    uint8_t *after = sm + kRows + (((nfw + nbw) * 2 + 15) & ~(size_t)15);
    uint16_t *f16 = reinterpret_cast<uint16_t *>(after);
    const size_t fsz = (size_t)t.nf * ncls, bsz = (size_t)t.nb * ncls;
    uint16_t *b16 = reinterpret_cast<uint16_t *>(after + ((fsz * 2 + 15) & ~(size_t)15));
    for (size_t i = threadIdx.x; i < fsz; i += blockDim.x) f16[i] = (uint16_t)__ldg(t.fT + i);
    for (size_t i = threadIdx.x; i < bsz; i += blockDim.x) b16[i] = (uint16_t)__ldg(t.bT + i);
    T.cls = sm + kCls;
    T.f16 = f16;
    T.b16 = b16;
    T.f8 = T.b8 = nullptr;
    T.f32 = t.fT;
    T.b32 = t.bT;
    T.f2 = T.b2 = nullptr;
    T.ncls = ncls;
    T.nc2 = nc2;
    T.rowb = rowb;
    T.nf = t.nf;
    T.magic = 0xFFFFFFFFu / rowb + 1u;
    __syncthreads();
    return reinterpret_cast<uint8_t *>(b16) + ((bsz * 2 + 15) & ~(size_t)15);
}

// Run state <-> state id (identity outside pair mode).
template <int TM> __device__ __forceinline__ uint32_t enc_f(const Tabs &T, uint32_t id) {
    return TM == TM_PAIR ? id * T.rowb : id;
}
template <int TM> __device__ __forceinline__ uint32_t enc_b(const Tabs &T, uint32_t id) {
    return TM == TM_PAIR ? (T.nf + id) * T.rowb : id;
}
template <int TM> __device__ __forceinline__ uint32_t dec_f(const Tabs &T, uint32_t e) {
    return TM == TM_PAIR ? __umulhi(e, T.magic) : e;
}
template <int TM> __device__ __forceinline__ uint32_t dec_b(const Tabs &T, uint32_t e) {
    return TM == TM_PAIR ? __umulhi(e, T.magic) - T.nf : e;
}

// Byte k (0..3) of w, zero-extended (one byte permute).
__device__ __forceinline__ uint32_t byte_k(uint32_t w, int k) { return __byte_perm(w, 0u, 0x4440u | (uint32_t)k); }

// 2 * class pair of bytes (lo, hi) of w at positions k, k+1 in pair mode.
__device__ __forceinline__ uint32_t cp2_of(const uint8_t *sm, uint32_t w, int k) {
    return ((uint32_t)sm[kClsH + byte_k(w, k)] << 1) + sm[kClsL + byte_k(w, k + 1)];
}

// One 64-byte block of both directions.  Runs j < W are stepped, W a
// compile-time width chosen per block from the warp's largest run count (so
// the loops are fully unrolled without predication); a lane with fewer runs
// steps empty states, which stay empty (row 0 of every table).
// Bytes come from this lane's row of the warp's forward / backward tile
// (64-byte rows, SWIZZLE_64B layout: 16-byte chunk q of row r sits at chunk
// q ^ ((r >> 1) & 3)), filled by TMA or, for warps TMA cannot serve, by the
// lanes themselves.
// With OUT (one-byte modes, a lane walking one direction) the lane also
// writes the state of run 0 at every column of the block into its row of the
// warp's state tile (same row layout as the text tile): forward, column t is
// the state before byte t; backward, the state after consuming byte t (right
// to left).  Columns the lane does not consume keep the state it has there.
template <int TM, int MS, bool EDGE, int W, bool FW = true, bool OUT = false>
__device__ __forceinline__ void walk_block(const Params &p, const Tabs &T, const uint8_t *frow, const uint8_t *brow,
                                           uint32_t (&sf)[MS], uint32_t (&sb)[MS], uint32_t wmf, uint32_t wmb,
                                           bool bwd, int f_lo, int f_hi, int b_lo, int b_hi,
                                           uint8_t *orow = nullptr) {
    static_assert(!OUT || TM != TM_PAIR, "state rows need one-byte steps");
    const uint32_t swz = ((threadIdx.x & 31) >> 1) & 3;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        uint4 fx = FW ? *reinterpret_cast<const uint4 *>(frow + (((uint32_t)q ^ swz) << 4))
                      : make_uint4(0, 0, 0, 0);
        uint4 bx = bwd ? *reinterpret_cast<const uint4 *>(brow + (((uint32_t)(3 - q) ^ swz) << 4))
                       : make_uint4(0, 0, 0, 0);
        if (TM == TM_BYTE7) {                         // rows hold bytes below 128 only
            if (FW) fx = fold_high_bytes(T.rep, fx);
            if (bwd) bx = fold_high_bytes(T.rep, bx);
        }
        if (TM == TM_PAIR && !EDGE) {                 // two bytes per table lookup (run states are row offsets)
            extern __shared__ __align__(16) uint8_t sm[];
            const uint32_t fw[4] = {fx.x, fx.y, fx.z, fx.w}, bw[4] = {bx.x, bx.y, bx.z, bx.w};
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                if (FW) {
                    const uint32_t cpf = cp2_of(sm, fw[v >> 1], 2 * (v & 1));
#pragma unroll
                    for (int j = 0; j < W; ++j) sf[j] = *reinterpret_cast<const uint16_t *>(sm + kRows + sf[j] + cpf);
                }
                if (bwd) {                            // pair (14-2v, 15-2v), consumed right to left
                    const uint32_t cpb = cp2_of(sm, bw[(7 - v) >> 1], 2 * ((7 - v) & 1));
#pragma unroll
                    for (int j = 0; j < W; ++j) sb[j] = *reinterpret_cast<const uint16_t *>(sm + kRows + sb[j] + cpb);
                }
            }
        } else {
            uint32_t ow[4] = {0, 0, 0, 0};                      // OUT: 16 states of this q (forward) or 3-q
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int tf = 16 * q + u, tb = 63 - tf;
                if (OUT && FW) ow[u >> 2] |= (sf[0] & 0xFFu) << (8 * (u & 3));
                if (FW && (!EDGE || (tf >= f_lo && tf < f_hi))) {
                    const uint32_t c = clsof<TM>(T, byte_of(fx, u));
#pragma unroll
                    for (int j = 0; j < W; ++j) sf[j] = fnext<TM>(T, sf[j], c);
                }
                if (bwd && (!EDGE || (tb >= b_lo && tb <= b_hi))) {
                    const uint32_t c = clsof<TM>(T, byte_of(bx, 15 - u));
#pragma unroll
                    for (int j = 0; j < W; ++j) sb[j] = bnext<TM>(T, sb[j], c);
                }
                if (OUT && !FW) ow[(15 - u) >> 2] |= (sb[0] & 0xFFu) << (8 * ((15 - u) & 3));
            }
            if (OUT)
                *reinterpret_cast<uint4 *>(orow + ((((uint32_t)(FW ? q : 3 - q)) ^ swz) << 4)) =
                    make_uint4(ow[0], ow[1], ow[2], ow[3]);
        }
    }
}

// Per-warp ring of TMA tiles: kStages stages of a forward and a backward tile
// (32 chunk rows x 64 bytes each) and one mbarrier per stage.
constexpr int kStages = 3;
constexpr uint32_t kTileBytes = 32 * 64;
struct Ring {
    uint8_t *tiles;       // [nst][2][kTileBytes], 1024-byte aligned
    uint32_t bars;        // shared address of nst mbarriers
    uint32_t phase;       // bit s: parity of the next completion of stage s
    uint32_t nst = kStages;   // stages (kStages; 2 in the one-direction-per-block kernel)
    uint32_t nout = 2;        // MAT: state tiles per warp (2; 1 in the one-direction-per-block kernel)
    uint32_t obuf = 0;        // MAT: the state tile the next block fills; it alternates across the
                              // warp's chunk tiles too, so the wait before a fill (at most one store
                              // group still reading) always concerns the other tile
};

// Directions a warp walks: both (one lane per chunk), or one of them (the
// forward and the backward walk of a chunk in two warps).
enum { DIR_BOTH = 0, DIR_F = 1, DIR_B = 2 };
template <int DIR> __device__ __forceinline__ uint8_t *tile_f(const Ring &r, int s) {
    return r.tiles + (DIR == DIR_BOTH ? 2 * s : s) * kTileBytes;
}
template <int DIR> __device__ __forceinline__ uint8_t *tile_b(const Ring &r, int s) {
    return r.tiles + (DIR == DIR_BOTH ? 2 * s + 1 : s) * kTileBytes;
}

template <int DIR>
__device__ __forceinline__ void ring_issue(const Params &p, const CUtensorMap *map, const Ring &r, int s,
                                           uint32_t i0, uint32_t fb, uint32_t bb, bool fwd, bool bwd) {
    const uint32_t bar = r.bars + 8 * s;
    mbar_expect_tx(bar, ((fwd ? 1u : 0u) + (bwd ? 1u : 0u)) * kTileBytes);
    if (fwd) tma_load_2d(smem_u32(tile_f<DIR>(r, s)), map, 64 * fb, (int32_t)i0, bar);
    if (bwd) tma_load_2d(smem_u32(tile_b<DIR>(r, s)), map, 64 * bb, (int32_t)i0, bar);
}

// Fill this lane's rows of stage s with plain loads (warps TMA cannot serve:
// the text's last, shorter chunk, or no tensor map).  Bytes past n read as 0.
template <int DIR>
__device__ __forceinline__ void ring_fill_plain(const Params &p, const Ring &r, int s, uint64_t fpos, uint64_t bpos,
                                                bool fwd, bool bwd) {
    const uint32_t lane = threadIdx.x & 31, swz = (lane >> 1) & 3;
    uint8_t *frow = tile_f<DIR>(r, s) + lane * 64;
    uint8_t *brow = tile_b<DIR>(r, s) + lane * 64;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (fwd) *reinterpret_cast<uint4 *>(frow + (((uint32_t)q ^ swz) << 4)) = load16(p.x, p.n, fpos + 16 * q);
        if (bwd) *reinterpret_cast<uint4 *>(brow + (((uint32_t)q ^ swz) << 4)) = load16(p.x, p.n, bpos + 16 * q);
    }
}

// Wait for stage s (every lane waits, so every lane acquires the tile data).
__device__ __forceinline__ bool ring_wait(Ring &r, int s) {
    const uint32_t bar = r.bars + 8 * s, ph = (r.phase >> s) & 1u;
    bool ok = false;
    for (uint32_t it = 0; it < kWaitLimit && !ok; ++it) ok = mbar_try_wait(bar, ph);
    r.phase ^= 1u << s;
    return __all_sync(0xFFFFFFFFu, ok);
}

// Drop dead runs and merge runs in equal states (their slot sets are joined).
// All indexing is static so the run arrays stay in registers.
template <int MS>
__device__ __forceinline__ void compact(uint32_t (&s)[MS], uint32_t (&mk)[MS], uint32_t &m, uint32_t dead) {
    uint32_t ns[MS], nk[MS];
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < MS; ++j) { ns[j] = dead; nk[j] = 0; }   // unused runs hold the empty state
#pragma unroll
    for (int j = 0; j < MS; ++j) {
        if (j < (int)m && s[j] != dead) {
            bool merged = false;
#pragma unroll
            for (int k = 0; k < j; ++k)
                if (k < (int)cnt && ns[k] == s[j]) { nk[k] |= mk[j]; merged = true; }
            if (!merged) {
#pragma unroll
                for (int k = 0; k <= j; ++k)
                    if (k == (int)cnt) { ns[k] = s[j]; nk[k] = mk[j]; }
                ++cnt;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < MS; ++j) { s[j] = ns[j]; mk[j] = nk[j]; }
    m = cnt;
}

// Wide lanes: a chunk whose speculation starts with more runs than the
// register arrays hold keeps its runs in per-lane local arrays (they spill to
// local memory, cached in L1) and walks them one byte at a time, merging runs
// after every byte; once at most MS runs are left at a sub-chunk boundary they
// move into the registers.  Runs drop fast after the first bytes of a chunk
// (Sect. 4.3), so the register arrays, and the kernel's register budget, can be
// sized for the common case instead of for the largest slot count.
constexpr int kWide = 32;                    // local run capacity (= slot capacity)

// Drop dead runs and merge equal ones (slot sets joined), in place.
__device__ __forceinline__ void compact_local(uint32_t *s, uint32_t *mk, uint32_t &m) {
    uint32_t cnt = 0;
    for (uint32_t j = 0; j < m; ++j) {
        const uint32_t v = s[j];
        if (v == 0) continue;
        uint32_t k = 0;
        while (k < cnt && s[k] != v) ++k;
        if (k < cnt) { mk[k] |= mk[j]; continue; }
        s[cnt] = v;
        mk[cnt] = mk[j];
        ++cnt;
    }
    m = cnt;
}

// Walk bytes [lo, hi) of this lane's 64-byte tile row (forward: ascending;
// backward: descending from hi - 1) for the m runs of the local arrays (state
// ids), with the one-byte tables; runs are merged after every byte.
template <int TM, bool FWD>
__device__ __forceinline__ void walk_local(const Tabs &T, const uint8_t *row, uint32_t *s, uint32_t *mk, uint32_t &m,
                                          int lo, int hi) {
    constexpr int T1 = TM == TM_PAIR ? TM_SMEM : TM;     // pair layouts stage the one-byte tables too
    const uint32_t swz = ((threadIdx.x & 31) >> 1) & 3;
    for (int u = 0; u < hi - lo; ++u) {
        const int t = FWD ? lo + u : hi - 1 - u;
        uint32_t b = row[((((uint32_t)t >> 4) ^ swz) << 4) | ((uint32_t)t & 15)];
        if (TM == TM_BYTE7 && b >= 128) b = T.rep[b - 128];
        const uint32_t c = clsof<T1>(T, b);
        for (uint32_t j = 0; j < m; ++j) s[j] = FWD ? fnext<T1>(T, s[j], c) : bnext<T1>(T, s[j], c);
        compact_local(s, mk, m);
    }
}

// Record the runs at one boundary (while more than one run is live).
template <int TM, int MS, bool FWD>
__device__ __forceinline__ void record(const Params &p, const Tabs &T, uint32_t *cnt_row, uint2 *ent_row,
                                       uint32_t &used, uint32_t &nrec, bool &open, uint32_t slot,
                                       const uint32_t (&s)[MS], const uint32_t (&mk)[MS], uint32_t m) {
    if (!open) return;
    if (slot >= kRecBounds || used + m > kRecEntries) { open = false; return; }
#pragma unroll
    for (int j = 0; j < MS; ++j)
        if (j < (int)m) ent_row[used + j] = make_uint2(FWD ? dec_f<TM>(T, s[j]) : dec_b<TM>(T, s[j]), mk[j]);
    used += m;
    cnt_row[slot] = m;
    nrec = slot + 1;
}

// record() for the runs of a wide lane (state ids in local arrays).
template <bool FWD>
__device__ __forceinline__ void record_local(uint32_t *cnt_row, uint2 *ent_row, uint32_t &used, uint32_t &nrec,
                                             bool &open, uint32_t slot, const uint32_t *s, const uint32_t *mk,
                                             uint32_t m) {
    if (!open) return;
    if (slot >= kRecBounds || used + m > kRecEntries) { open = false; return; }
    for (uint32_t j = 0; j < m; ++j) ent_row[used + j] = make_uint2(s[j], mk[j]);
    used += m;
    cnt_row[slot] = m;
    nrec = slot + 1;
}

// Lanes of this warp that process block blk: chunk i = i0 + lane with
// i0 = i - lane (chunks are consecutive across a warp).  Full chunks have
// the same number of blocks; only the last chunk of the text may be shorter.
__device__ __forceinline__ unsigned block_lanes(const Params &p, uint32_t i, uint32_t blk) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t i0 = i - lane;
    const uint32_t last = p.c - 1;
    unsigned mask = 0;
    if (last > i0) {
        const uint32_t full = last - i0;                  // lanes holding chunks i0 .. c-2
        mask = full >= 32 ? 0xFFFFFFFFu : ((1u << full) - 1);
    }
    if (last - i0 < 32) {                                  // this warp holds the last chunk
        const uint32_t nsub_last = (uint32_t)((p.n - (uint64_t)last * p.k + 63) / 64);
        if (blk < nsub_last) mask |= 1u << (last - i0);
    }
    return mask;
}

// MAT: the lane also writes the state of every column of its chunk into FS
// (forward) or BS (backward), block by block, through the warp's two state
// tiles (TMA tensor stores, or plain stores where TMA does not serve); rows
// of blocks walked with more than one live run are written too and are
// overwritten by the fix-up, which gets here the first (forward) / last
// (backward) block the lane walked with one run.  No records or checkpoints.
template <int TM, int MS, int DIR = DIR_BOTH, bool WIDE = false, bool MAT = false>
__device__ bool reach_chunk(const Params &p, const Tabs &T, uint32_t i, const CUtensorMap *map, Ring &ring,
                            bool tma, const CUtensorMap *smap = nullptr, uint8_t *otile = nullptr) {
    static_assert(!WIDE || DIR != DIR_BOTH, "wide lanes walk one direction");
    static_assert(!MAT || (DIR != DIR_BOTH && TM != TM_PAIR), "state rows: one direction, one-byte steps");
    constexpr bool FW = DIR != DIR_B;
    const DevTables &t = p.t;
    const uint64_t base = (uint64_t)i * p.k;
    const uint32_t len = chunk_len(p, i);
    const uint32_t nsub = (len + 63) / 64;
    const bool bwd = DIR != DIR_F && !p.recognize;
    uint32_t sf[MS], sb[MS], kf[MS], kb[MS];
    const uint32_t dead_f = enc_f<TM>(T, 0), dead_b = enc_b<TM>(T, 0);
#pragma unroll
    for (int j = 0; j < MS; ++j) { sf[j] = dead_f; sb[j] = dead_b; kf[j] = 0u; kb[j] = 0u; }
    uint32_t mf = 0, mb = 0;
    int tstart = 0, tlast = -1;
    // wide lanes: the runs of the one direction this warp walks, as state ids
    uint32_t xs[WIDE ? kWide : 1], xk[WIDE ? kWide : 1], mx = 0;
    bool big = false;
    if (!FW) {
    } else if (i == 0 && !(p.shard & SHARD_PREV)) {
        mf = 1; sf[0] = enc_f<TM>(T, t.fI); kf[0] = 1; tstart = 0;      // J_0 = I (a slice: its entry state)
    } else {
        const uint32_t pr = class_of<TM>(T, t, __ldg(p.x + base - 1)) * t.ncls + class_of<TM>(T, t, __ldg(p.x + base));
        mf = __ldg(t.fSlotCount + pr);
        if (WIDE && mf > (uint32_t)MS) {
            big = true;
            mx = mf;
            mf = 0;
            for (uint32_t j = 0; j < mx; ++j) { xs[j] = __ldg(t.fSlotStart + pr * t.msf + j); xk[j] = 1u << j; }
        }
#pragma unroll
        for (int j = 0; j < MS; ++j)
            if (j < (int)mf) { sf[j] = enc_f<TM>(T, __ldg(t.fSlotStart + pr * t.msf + j)); kf[j] = 1u << j; }
        tstart = 1;                                        // slot states follow byte 0
    }
    if (bwd) {
        if (i == p.c - 1 && !(p.shard & SHARD_NEXT)) {
            mb = 1; sb[0] = enc_b<TM>(T, t.bF); kb[0] = 1; tlast = (int)len - 1;   // Ĵ_{c+1} = F (or the slice's)
        } else {
            const uint32_t pr = class_of<TM>(T, t, __ldg(p.x + base + len - 1)) * t.ncls +
                                class_of<TM>(T, t, __ldg(p.x + base + len));
            mb = __ldg(t.bSlotCount + pr);
            if (WIDE && mb > (uint32_t)MS) {
                big = true;
                mx = mb;
                mb = 0;
                for (uint32_t j = 0; j < mx; ++j) { xs[j] = __ldg(t.bSlotStart + pr * t.msb + j); xk[j] = 1u << j; }
            }
#pragma unroll
            for (int j = 0; j < MS; ++j)
                if (j < (int)mb) { sb[j] = enc_b<TM>(T, __ldg(t.bSlotStart + pr * t.msb + j)); kb[j] = 1u << j; }
            tlast = (int)len - 2;                          // slot states precede the last byte
        }
    }
    bool fconv = mf <= 1 && !(FW && big), bconv = mb <= 1 && !(!FW && big);
    const bool single0 = FW ? fconv : bconv;                  // one run from the chunk's edge on
    uint32_t fconv_sub = fconv ? 1 : nsub, bconv_sub = bconv ? nsub - 1 : 0;
    uint32_t *fcnt = p.w.recFc + (size_t)i * kRecBounds, *bcnt = p.w.recBc + (size_t)i * kRecBounds;
    uint2 *fent = p.w.recFe + (size_t)i * kRecEntries, *bent = p.w.recBe + (size_t)i * kRecEntries;
    uint32_t fused = 0, bused = 0, fnrec = 0, bnrec = 0;
    bool fopen = true, bopen = true;

    const uint32_t lane = threadIdx.x & 31, i0 = i - lane;
    if (MAT) {   // a new tile: earlier tiles' state stores have read their tiles (the plain path never waits)
        const unsigned present = p.c - i0 >= 32 ? 0xFFFFFFFFu : ((1u << (p.c - i0)) - 1u);   // lanes with a chunk
        if (lane == 0) bulk_wait_read_all();
        __syncwarp(present);
    }
    if (tma && lane == 0)                                     // prologue: first stages in flight
        for (uint32_t b = 0; b < ring.nst && b < nsub; ++b)
            ring_issue<DIR>(p, map, ring, b, i0, b, nsub - 1 - b, FW, bwd);
    for (uint32_t blk = 0; blk < nsub; ++blk) {
        const uint32_t fb = blk, bb = nsub - 1 - blk;
        const int stage = (int)(blk % ring.nst);
        if (FW && fb >= 1) {                                // boundary before forward block fb
            if (WIDE && big) {
                compact_local(xs, xk, mx);
                if (!MAT && mx > 1) record_local<true>(fcnt, fent, fused, fnrec, fopen, fb - 1, xs, xk, mx);
                if (mx <= (uint32_t)MS) {                     // into the registers
                    big = false;
                    mf = mx;
#pragma unroll
                    for (int j = 0; j < MS; ++j)
                        if (j < (int)mx) { sf[j] = enc_f<TM>(T, xs[j]); kf[j] = xk[j]; }
                    if (mf <= 1) { fconv = true; fconv_sub = fb; }
                }
            } else if (!fconv) {
                compact<MS>(sf, kf, mf, dead_f);
                if (mf <= 1) { fconv = true; fconv_sub = fb; }
                else if (!MAT) record<TM, MS, true>(p, T, fcnt, fent, fused, fnrec, fopen, fb - 1, sf, kf, mf);
            }
            if (!MAT) p.w.FC[(uint64_t)i * p.S + fb] = fconv ? dec_f<TM>(T, sf[0]) : kUnknown;
        }
        const uint64_t fpos = base + 64ull * fb, bpos = base + 64ull * bb;
        const int f_lo = fb == 0 ? tstart : 0;
        const int f_hi = (int)min(64u, len - 64 * fb);
        const int b_hi = min(63, tlast - (int)(64 * bb));
        const bool edge = (FW && (f_lo != 0 || f_hi != 64)) || (bwd && b_hi != 63);
        const unsigned act = block_lanes(p, i, blk);
        const uint32_t wmf = __reduce_max_sync(act, mf), wmb = __reduce_max_sync(act, mb);
        if (tma) {
            if (!ring_wait(ring, stage)) return false;        // lost TMA completion: give up this chunk tile
        } else {
            ring_fill_plain<DIR>(p, ring, stage, fpos, bpos, FW, bwd);
            __syncwarp(act);
        }
        const uint8_t *frow = tile_f<DIR>(ring, stage) + lane * 64;
        const uint8_t *brow = tile_b<DIR>(ring, stage) + lane * 64;
        const uint32_t wm = max(wmf, wmb);
        uint8_t *orow = MAT ? otile + ring.obuf * kTileBytes + lane * 64 : nullptr;
        if (MAT && tma) {                                     // the store that last used this tile has read it
            if (lane == 0) {
                if (ring.nout == 1) bulk_wait_read_all();
                else bulk_wait_read_1();
            }
            __syncwarp();
        }
        if (edge) {
            if constexpr (TM == TM_PAIR) {              // one byte at a time on state ids
#pragma unroll
                for (int j = 0; j < MS; ++j) { sf[j] = dec_f<TM>(T, sf[j]); sb[j] = dec_b<TM>(T, sb[j]); }
                walk_block<TM_SMEM, MS, true, MS, FW>(p, T, frow, brow, sf, sb, wmf, wmb, bwd, f_lo, f_hi, 0, b_hi);
#pragma unroll
                for (int j = 0; j < MS; ++j) { sf[j] = enc_f<TM>(T, sf[j]); sb[j] = enc_b<TM>(T, sb[j]); }
            } else {
                walk_block<TM, MS, true, MS, FW, MAT>(p, T, frow, brow, sf, sb, wmf, wmb, bwd, f_lo, f_hi, 0, b_hi, orow);
            }
        }
        else if (wm <= 1) walk_block<TM, MS, false, 1, FW, MAT>(p, T, frow, brow, sf, sb, wmf, wmb, bwd, 0, 64, 0, 63, orow);
        else if (MS > 2 && wm <= 2) walk_block<TM, MS, false, (MS > 2 ? 2 : MS), FW, MAT>(p, T, frow, brow, sf, sb, wmf, wmb, bwd, 0, 64, 0, 63, orow);
        else if (MS > 4 && wm <= 4) walk_block<TM, MS, false, (MS > 4 ? 4 : MS), FW, MAT>(p, T, frow, brow, sf, sb, wmf, wmb, bwd, 0, 64, 0, 63, orow);
        else walk_block<TM, MS, false, MS, FW, MAT>(p, T, frow, brow, sf, sb, wmf, wmb, bwd, 0, 64, 0, 63, orow);
        if (MAT) {                                            // this block's state row
            const uint32_t ob = FW ? fb : bb;
            uint8_t *dst = (FW ? p.w.FS : p.w.BS) + base + 64ull * ob;
            if (tma) {
                fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    tma_store_2d(smap, smem_u32(otile + ring.obuf * kTileBytes), 64 * ob, (int32_t)i0);
                    bulk_commit();
                }
            } else {                                          // plain stores, clipped to the chunk
                const uint32_t swz = (lane >> 1) & 3;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t col = 64 * ob + 16 * q;
                    if (col >= len) break;
                    const uint4 v = *reinterpret_cast<const uint4 *>(orow + (((uint32_t)q ^ swz) << 4));
                    if (col + 16 <= len) {
                        *reinterpret_cast<uint4 *>(dst + 16 * q) = v;
                    } else {
                        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
                        for (uint32_t u = 0; u < len - col; ++u) dst[16 * q + u] = (uint8_t)(w[u >> 2] >> (8 * (u & 3)));
                    }
                }
            }
            if (ring.nout == 2) ring.obuf ^= 1u;
        }
        if (WIDE && big) {                                    // this lane's runs past the register arrays
            if (FW) walk_local<TM, true>(T, frow, xs, xk, mx, f_lo, f_hi);
            else walk_local<TM, false>(T, brow, xs, xk, mx, 0, b_hi + 1);
        }
        if (tma) {
            __syncwarp();                                     // every lane has read this stage
            if (lane == 0 && blk + ring.nst < nsub)
                ring_issue<DIR>(p, map, ring, stage, i0, blk + ring.nst, nsub - 1 - (blk + ring.nst), FW, bwd);
        } else {
            __syncwarp(act);                                  // stage read before the next fill
        }
        if (bwd && bb >= 1) {                               // boundary at the start of backward block bb
            if (WIDE && big) {
                compact_local(xs, xk, mx);
                if (!MAT && mx > 1) record_local<false>(bcnt, bent, bused, bnrec, bopen, nsub - 1 - bb, xs, xk, mx);
                if (mx <= (uint32_t)MS) {                     // into the registers
                    big = false;
                    mb = mx;
#pragma unroll
                    for (int j = 0; j < MS; ++j)
                        if (j < (int)mx) { sb[j] = enc_b<TM>(T, xs[j]); kb[j] = xk[j]; }
                    if (mb <= 1) { bconv = true; bconv_sub = bb; }
                }
            } else if (!bconv) {
                compact<MS>(sb, kb, mb, dead_b);
                if (mb <= 1) { bconv = true; bconv_sub = bb; }
                else if (!MAT) record<TM, MS, false>(p, T, bcnt, bent, bused, bnrec, bopen, nsub - 1 - bb, sb, kb, mb);
            }
            if (!MAT) p.w.BC[(uint64_t)i * p.S + bb - 1] = bconv ? dec_b<TM>(T, sb[0]) : kUnknown;
        }
    }
    // end state of every slot: the state of the run standing for it (0 if none)
    if (WIDE && big) compact_local(xs, xk, mx);         // runs still past the registers at the end
    if (FW) {
        const uint32_t msf = t.msf;
        for (uint32_t j = 0; j < msf; ++j) {
            uint32_t v = 0;
            if (WIDE && big) {
                for (uint32_t r = 0; r < mx; ++r)
                    if ((xk[r] >> j) & 1) v = xs[r];
            } else {
#pragma unroll
                for (int r = 0; r < MS; ++r)
                    if (r < (int)mf && ((kf[r] >> j) & 1)) v = dec_f<TM>(T, sf[r]);
            }
            p.w.Rf[(size_t)i * msf + j] = v;
        }
        // MAT: the first block walked with one run (every block from there on is exact)
        p.w.fconv[i] = MAT ? (single0 ? 0u : fconv_sub) : fconv_sub;
        p.w.fnrec[i] = fnrec;
    }
    if (bwd) {
        const uint32_t msb = t.msb;
        for (uint32_t j = 0; j < msb; ++j) {
            uint32_t v = 0;
            if (WIDE && big) {
                for (uint32_t r = 0; r < mx; ++r)
                    if ((xk[r] >> j) & 1) v = xs[r];
            } else {
#pragma unroll
                for (int r = 0; r < MS; ++r)
                    if (r < (int)mb && ((kb[r] >> j) & 1)) v = dec_b<TM>(T, sb[r]);
            }
            p.w.Rb[(size_t)i * msb + j] = v;
        }
        // MAT: blocks below this one were walked with one run (exact)
        p.w.bconv[i] = MAT ? (single0 ? nsub : (bconv ? bconv_sub : 0u)) : bconv_sub;
        p.w.bnrec[i] = bnrec;
    }
    return true;
}

// Warps per block of the split parse kernel: four 32-chunk tiles, each walked
// forward by one warp and backward by another, sharing one copy of the tables.
constexpr uint32_t kSplitThreads = 256;

// One parse.  SPLIT: warp pairs take 32-chunk tiles, the even warp walking
// the chunks forward and the odd one backward (each with a one-direction TMA
// ring), which doubles the warps in flight for the same shared memory; in
// recognizer mode every warp takes a tile of its own, forward.  Without SPLIT
// every warp walks its tile in both directions (two tiles per ring stage).
template <int TM, int MS, bool SPLIT, bool WIDE = false, bool MAT = false>
__global__ void __launch_bounds__(kSplitThreads, (SPLIT && MS <= 8) ? 3 : 1)
    reach_kernel(const __grid_constant__ Params p, const __grid_constant__ CUtensorMap map,
                 const __grid_constant__ StateMaps smaps) {
    extern __shared__ __align__(16) uint8_t sm[];
    constexpr int TILES = SPLIT ? 1 : 2;                      // tiles per ring stage
    Tabs T;
    uint8_t *rest = TM == TM_PAIR ? stage_reach_pair(p.t, sm, T) : stage_tables<TM>(p.t, sm, T);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x / 32;
    uint8_t *otile = nullptr;
    Ring ring{};
    const uint32_t nst = p.rstages ? p.rstages : (uint32_t)kStages;   // ring stages (2 or 3)
    {
        const uint32_t a = smem_u32(rest);
        uint8_t *aligned = rest + ((1024 - (a & 1023)) & 1023);
        ring.nst = nst;
        ring.tiles = aligned + warp * (nst * TILES * kTileBytes);
        ring.bars = smem_u32(aligned + wpb * (nst * TILES * kTileBytes)) + warp * nst * 8;
        ring.phase = 0;
        if (MAT) {                                            // two state tiles per warp, 1024-byte aligned
            uint8_t *after = aligned + wpb * (nst * TILES * kTileBytes + nst * 8);
            after += (1024 - (smem_u32(after) & 1023)) & 1023;
            otile = after + warp * 2 * kTileBytes;
        }
        if (p.text_tma && lane == 0) {
            for (uint32_t st = 0; st < nst; ++st) mbar_init(ring.bars + 8 * st, 1);
            mbar_init_fence();
        }
        __syncwarp();
    }
    pdl_wait();                                               // the join flags are set by the kernel before
    pdl_trigger();
    const uint64_t gw = (uint64_t)blockIdx.x * wpb + warp, nw = (uint64_t)gridDim.x * wpb;
    const bool pairs = SPLIT && !p.recognize;                // recognizer: every warp walks its own tile forward
    const uint64_t t0 = pairs ? gw >> 1 : gw, tstep = pairs ? nw >> 1 : nw;
    const bool backward_warp = pairs && (gw & 1);
    for (uint64_t t = t0; t * 32 < p.c; t += tstep) {
        const uint32_t i = (uint32_t)(t * 32) + lane;
        const bool tma = p.text_tma && t * 32 + 32 <= p.c_full;
        if (i >= p.c) continue;                               // lanes past the text (plain path only)
        bool ok;
        if constexpr (!SPLIT) ok = reach_chunk<TM, MS, DIR_BOTH>(p, T, i, &map, ring, tma);
        else if (backward_warp) ok = reach_chunk<TM, MS, DIR_B, WIDE, MAT>(p, T, i, &map, ring, tma, &smaps.b, otile);
        else ok = reach_chunk<TM, MS, DIR_F, WIDE, MAT>(p, T, i, &map, ring, tma, &smaps.f, otile);
        if (!ok) {
            atomicExch(p.status, RE_E_INTERNAL);
            atomicExch(&p.w.flags[FLAG_INTERNAL], 1);
            for (uint32_t st = 0; st < nst; ++st) {           // drain: bounded wait on every stage
                bool done = false;
                for (uint32_t it = 0; it < kWaitLimit && !done; ++it)
                    done = mbar_try_wait(ring.bars + 8 * st, (ring.phase >> st) & 1u);
            }
            if (MAT && lane == 0) bulk_wait_all();
            return;
        }
    }
    if (MAT && lane == 0) bulk_wait_all();                    // state rows written before the grid ends
}

// One parse with byte-indexed tables (TM_BYTE8, or TM_BYTE7 when the bytes
// >= 128 fold onto ASCII bytes of their class): every warp of a block walks
// the same direction, so a block stages one direction's table (about 65 KB
// for 251 states; half that with ASCII rows) instead of both.  Even blocks
// walk 32-chunk tiles forward, odd blocks backward (every block forward in
// recognizer mode); 2-stage TMA rings, and (MAT) one state tile per warp,
// whose store has read it before the next block's states go in.  A warp's
// lookups wait on shared-memory latency, so the block takes as many warps as
// the shared memory left by its table holds (24 with full rows; up to 32
// with ASCII rows, whose kernel is compiled for 1024 threads).  Tiles are
// dealt round-robin over the blocks of a direction (tile t to block t mod
// B), so a text of few tiles still spreads over every SM.
constexpr uint32_t kDirThreads = 768;
constexpr uint32_t kDirThreadsAscii = 1024;
constexpr uint32_t kDirStages = 2;
constexpr uint32_t kDirOut = 1;             // MAT state tiles per warp
// Shared memory after the table: [1024-byte pad][text tiles, kDirStages per
// warp][state tiles, kDirOut per warp][mbarriers, kDirStages per warp]; the
// tiles are 1024-byte multiples, so one pad aligns them all.
template <bool ASC> constexpr uint32_t dir_threads_max() { return ASC ? kDirThreadsAscii : kDirThreads; }

inline size_t dir_table_smem(const DevTables &t, bool asc) {
    return std::max(byte8_smem_bytes(t, true, false, asc), byte8_smem_bytes(t, false, true, asc));
}
inline size_t dir_warp_smem(bool mat) { return (kDirStages + (mat ? kDirOut : 0)) * kTileBytes + kDirStages * 8; }
// Warps per block: as many as the shared memory holds, at most the kernel's bound.
inline uint32_t dir_wpb(const DevTables &t, bool mat, bool asc) {
    const size_t cap = asc ? kDirThreadsAscii / 32 : kDirThreads / 32;
    const size_t avail = 227 * 1024 - dir_table_smem(t, asc) - 1024;
    return (uint32_t)std::max<size_t>(1, std::min(cap, avail / dir_warp_smem(mat)));
}
inline size_t reach_dir_smem(const DevTables &t, bool mat, bool asc) {
    return dir_table_smem(t, asc) + 1024 + dir_wpb(t, mat, asc) * dir_warp_smem(mat);
}

template <int MS, bool WIDE, bool MAT, bool ASC>
__global__ void __launch_bounds__(dir_threads_max<ASC>(), 1)
    reach_dir_kernel(const __grid_constant__ Params p, const __grid_constant__ CUtensorMap map,
                     const __grid_constant__ StateMaps smaps) {
    constexpr int TM = ASC ? TM_BYTE7 : TM_BYTE8;
    extern __shared__ __align__(16) uint8_t sm[];
    const bool pairs = !p.recognize;
    const bool backward_block = pairs && (blockIdx.x & 1);
    Tabs T;
    uint8_t *rest = stage_byte8(p.t, sm, T, !backward_block, backward_block, ASC);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x / 32;
    uint8_t *otile = nullptr;
    Ring ring{};
    ring.nst = kDirStages;
    ring.nout = kDirOut;
    {
        const uint32_t a = smem_u32(rest);
        uint8_t *aligned = rest + ((1024 - (a & 1023)) & 1023);
        const uint32_t outs = MAT ? kDirOut : 0;
        ring.tiles = aligned + warp * (kDirStages * kTileBytes);
        ring.bars = smem_u32(aligned + wpb * (kDirStages + outs) * kTileBytes) + warp * kDirStages * 8;
        ring.phase = 0;
        if (MAT) otile = aligned + wpb * kDirStages * kTileBytes + warp * kDirOut * kTileBytes;
        if (p.text_tma && lane == 0) {
            for (uint32_t st = 0; st < kDirStages; ++st) mbar_init(ring.bars + 8 * st, 1);
            mbar_init_fence();
        }
        __syncwarp();
    }
    pdl_wait();
    pdl_trigger();
    const uint64_t gblk = pairs ? blockIdx.x >> 1 : blockIdx.x, nblk = pairs ? gridDim.x >> 1 : gridDim.x;
    for (uint64_t t = (uint64_t)warp * nblk + gblk; t * 32 < p.c; t += nblk * wpb) {
        const uint32_t i = (uint32_t)(t * 32) + lane;
        const bool tma = p.text_tma && t * 32 + 32 <= p.c_full;
        if (i >= p.c) continue;                               // lanes past the text (plain path only)
        const bool ok = backward_block
                            ? reach_chunk<TM, MS, DIR_B, WIDE, MAT>(p, T, i, &map, ring, tma, &smaps.b, otile)
                            : reach_chunk<TM, MS, DIR_F, WIDE, MAT>(p, T, i, &map, ring, tma, &smaps.f, otile);
        if (!ok) {
            atomicExch(p.status, RE_E_INTERNAL);
            atomicExch(&p.w.flags[FLAG_INTERNAL], 1);
            for (uint32_t st = 0; st < kDirStages; ++st) {   // drain: bounded wait on every stage
                bool done = false;
                for (uint32_t it = 0; it < kWaitLimit && !done; ++it)
                    done = mbar_try_wait(ring.bars + 8 * st, (ring.phase >> st) & 1u);
            }
            if (MAT && lane == 0) bulk_wait_all();
            return;
        }
    }
    if (MAT && lane == 0) bulk_wait_all();
}

// Blocks per direction: every resident block slot, split between the
// directions, but no more blocks per direction than tiles (tiles go
// round-robin over blocks).
template <int MS, bool WIDE, bool MAT, bool ASC>
uint64_t dir_blocks(const Params &p, int sm_count) {
    const size_t smem = reach_dir_smem(p.t, MAT, ASC);
    static uint64_t attr_done = 0;
    allow_smem(reach_dir_kernel<MS, WIDE, MAT, ASC>, &attr_done, 227 * 1024);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reach_dir_kernel<MS, WIDE, MAT, ASC>,
                                                  dir_wpb(p.t, MAT, ASC) * 32, smem);
    const uint64_t tiles = ((uint64_t)p.c + 31) / 32;
    const uint64_t dirs = p.recognize ? 1 : 2;
    const uint64_t slots = (uint64_t)std::max(per_sm, 1) * sm_count;
    return std::max<uint64_t>(1, std::min<uint64_t>(tiles, slots / dirs));
}

template <int MS, bool WIDE, bool MAT, bool ASC>
void launch_dir(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, int sm_count) {
    const size_t smem = reach_dir_smem(p.t, MAT, ASC);
    const uint64_t dirs = p.recognize ? 1 : 2;
    const uint64_t per_dir = dir_blocks<MS, WIDE, MAT, ASC>(p, sm_count);
    const uint64_t blocks = per_dir * dirs;                    // even: one block of each pair per direction
    launch_dependent(reach_dir_kernel<MS, WIDE, MAT, ASC>, (uint32_t)std::max<uint64_t>(blocks, 1),
                     dir_wpb(p.t, MAT, ASC) * 32, smem, s, p, map, smaps);
}

// A batch group (one RE) with byte-indexed tables and per-position states:
// the single-text kernel's shape (blocks alternate directions, one table per
// block) over the 32-chunk tiles of every text of the group, dealt
// round-robin over the blocks; full tiles of texts with tensor maps move by
// TMA, the rest by plain loads and stores.
template <int MS, bool WIDE, bool ASC>
__global__ void __launch_bounds__(dir_threads_max<ASC>(), 1) reach_dir_batch_kernel(const __grid_constant__ BatchGroup b) {
    constexpr int TM = ASC ? TM_BYTE7 : TM_BYTE8;
    extern __shared__ __align__(16) uint8_t sm[];
    const bool backward_block = blockIdx.x & 1;
    Tabs T;
    uint8_t *rest = stage_byte8(b.t, sm, T, !backward_block, backward_block, ASC);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x / 32;
    Ring ring{};
    ring.nst = kDirStages;
    ring.nout = kDirOut;
    const uint32_t a = smem_u32(rest);
    uint8_t *aligned = rest + ((1024 - (a & 1023)) & 1023);
    ring.tiles = aligned + warp * (kDirStages * kTileBytes);
    ring.bars = smem_u32(aligned + wpb * (kDirStages + kDirOut) * kTileBytes) + warp * kDirStages * 8;
    ring.phase = 0;
    uint8_t *otile = aligned + wpb * kDirStages * kTileBytes + warp * kDirOut * kTileBytes;
    if (lane == 0) {
        for (uint32_t st = 0; st < kDirStages; ++st) mbar_init(ring.bars + 8 * st, 1);
        mbar_init_fence();
    }
    __syncwarp();
    const uint64_t gblk = blockIdx.x >> 1, nblk = gridDim.x >> 1;
    for (uint64_t t = (uint64_t)warp * nblk + gblk; t < b.n_reach; t += nblk * wpb) {
        const uint32_t ti = text_of(b.rtile_base, b.nt, t);
        const Params &p = b.texts[ti];
        const uint64_t tile = t - __ldg(b.rtile_base + ti);
        const uint32_t i = (uint32_t)(tile * 32) + lane;
        // full tiles of a text with tensor maps go through TMA (text in, state rows out)
        const bool tma = p.text_tma && p.state_tma && tile * 32 + 32 <= p.c_full;
        if (tma && lane == 0) {
            tensormap_acquire(p.tmaps);
            tensormap_acquire(p.tmaps + (backward_block ? 2 : 1));
        }
        if (tma) __syncwarp();
        if (i >= p.c) continue;                               // lanes past the text's last chunk (plain tiles only)
        const bool ok = backward_block
                            ? reach_chunk<TM, MS, DIR_B, WIDE, true>(p, T, i, p.tmaps, ring, tma, p.tmaps + 2, otile)
                            : reach_chunk<TM, MS, DIR_F, WIDE, true>(p, T, i, p.tmaps, ring, tma, p.tmaps + 1, otile);
        if (!ok) {
            atomicExch(p.status, RE_E_INTERNAL);
            for (uint32_t st = 0; st < kDirStages; ++st) {   // drain: bounded wait on every stage
                bool done = false;
                for (uint32_t it = 0; it < kWaitLimit && !done; ++it)
                    done = mbar_try_wait(ring.bars + 8 * st, (ring.phase >> st) & 1u);
            }
            if (lane == 0) bulk_wait_all();
            return;
        }
    }
    if (lane == 0) bulk_wait_all();
}

template <int MS, bool WIDE, bool ASC>
void launch_dir_batch_one(const BatchGroup &b, cudaStream_t s, int sm_count) {
    const size_t smem = reach_dir_smem(b.t, true, ASC);
    const uint32_t threads = dir_wpb(b.t, true, ASC) * 32;
    static uint64_t attr_done = 0;
    allow_smem(reach_dir_batch_kernel<MS, WIDE, ASC>, &attr_done, 227 * 1024);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reach_dir_batch_kernel<MS, WIDE, ASC>, threads, smem);
    const uint64_t slots = (uint64_t)std::max(per_sm, 1) * sm_count;
    const uint64_t per_dir = std::max<uint64_t>(1, std::min<uint64_t>(b.n_reach, slots / 2));
    reach_dir_batch_kernel<MS, WIDE, ASC><<<(uint32_t)(per_dir * 2), threads, smem, s>>>(b);
}

template <bool ASC>
bool launch_dir_batch(const BatchGroup &b, uint32_t ms, cudaStream_t s, int sm_count) {
    if (ms <= 2) launch_dir_batch_one<2, false, ASC>(b, s, sm_count);
    else if (ms <= 4) launch_dir_batch_one<4, false, ASC>(b, s, sm_count);
    else if (ms <= 8) launch_dir_batch_one<8, false, ASC>(b, s, sm_count);
    else if (ms <= 32) launch_dir_batch_one<4, true, ASC>(b, s, sm_count);
    else return false;
    return true;
}

// Warps per direction the one-direction-per-block reach runs at most (every
// resident block of a direction, dir_wpb warps each).
template <bool MAT, bool ASC>
uint64_t dir_warps(const Params &p, uint32_t ms, int sm_count) {
    Params q = p;
    q.c = 0xFFFFFFFFu;                                         // as many tiles as block slots
    const uint64_t b = ms <= 2 ? dir_blocks<2, false, MAT, ASC>(q, sm_count)
                     : ms <= 4 ? dir_blocks<4, false, MAT, ASC>(q, sm_count)
                     : ms <= 8 ? dir_blocks<8, false, MAT, ASC>(q, sm_count)
                               : dir_blocks<4, true, MAT, ASC>(q, sm_count);
    return b * dir_wpb(p.t, MAT, ASC);
}

template <bool MAT, bool ASC>
bool launch_dir_ms(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
                   int sm_count) {
    if (ms <= 2) launch_dir<2, false, MAT, ASC>(p, map, smaps, s, sm_count);
    else if (ms <= 4) launch_dir<4, false, MAT, ASC>(p, map, smaps, s, sm_count);
    else if (ms <= 8) launch_dir<8, false, MAT, ASC>(p, map, smaps, s, sm_count);
    else if (ms <= 32) launch_dir<4, true, MAT, ASC>(p, map, smaps, s, sm_count);
    else return false;
    return true;
}

// Batch: warps take work items from the group's list (an atomic counter).  An
// item is a 32-chunk tile of any text of the group and, in SPLIT mode, one of
// its two directions (the forward and backward walks of a tile go to two
// warps, as in a single parse).  Text bytes come in by plain loads.  Lanes
// past their text's last chunk skip the tile and meet the others at the
// closing __syncwarp, so no lane waits in a collective the others do not run.
template <int TM, int MS, bool SPLIT, bool WIDE = false>
__global__ void __launch_bounds__(kSplitThreads, (SPLIT && MS <= 8) ? 3 : 1)
    reach_batch_kernel(const __grid_constant__ BatchGroup b) {
    extern __shared__ __align__(16) uint8_t sm[];
    constexpr int TILES = SPLIT ? 1 : 2;
    Tabs T;
    uint8_t *rest = TM == TM_PAIR ? stage_reach_pair(b.t, sm, T) : stage_tables<TM>(b.t, sm, T);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Ring ring{};
    {
        const uint32_t a = smem_u32(rest);
        uint8_t *aligned = rest + ((1024 - (a & 1023)) & 1023);
        ring.tiles = aligned + warp * (kStages * TILES * kTileBytes);
    }
    const uint64_t items = SPLIT ? 2 * b.n_reach : b.n_reach;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(b.queue + Q_REACH, 1u);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item >= items) break;
        const uint32_t tile = SPLIT ? item >> 1 : item;
        const uint32_t ti = text_of(b.rtile_base, b.nt, tile);
        const Params &p = b.texts[ti];
        const uint32_t i = (uint32_t)(tile - b.rtile_base[ti]) * 32 + lane;
        if (i < p.c) {
            bool ok;
            if constexpr (!SPLIT) ok = reach_chunk<TM, MS, DIR_BOTH>(p, T, i, nullptr, ring, false);
            else if (item & 1) ok = reach_chunk<TM, MS, DIR_B, WIDE>(p, T, i, nullptr, ring, false);
            else ok = reach_chunk<TM, MS, DIR_F, WIDE>(p, T, i, nullptr, ring, false);
            if (!ok) atomicExch(&p.w.flags[FLAG_INTERNAL], 1);
        }
        __syncwarp();
    }
}

inline size_t reach_smem(const DevTables &t, int tm, uint32_t threads = kChunkThreads, int tiles = 2,
                         bool mat = false, uint32_t stages = kStages) {
    const size_t tab = tm == TM_PAIR ? reach_pair_smem(t) : tables_smem_bytes(t, tm);
    const size_t out = mat ? 1024 + (threads / 32) * 2 * kTileBytes : 0;   // two state tiles per warp
    return tab + 1024 + (threads / 32) * (stages * tiles * kTileBytes + stages * 8) + out;
}

template <int TM, int MS, bool SPLIT, bool WIDE = false>
void launch_batch_split(const BatchGroup &b, cudaStream_t s, int sm_count) {
    const uint32_t threads = SPLIT ? kSplitThreads : kChunkThreads;
    const size_t smem = reach_smem(b.t, TM, threads, SPLIT ? 1 : 2);
    static uint64_t attr_done = 0;
    allow_smem(reach_batch_kernel<TM, MS, SPLIT, WIDE>, &attr_done);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reach_batch_kernel<TM, MS, SPLIT, WIDE>, threads, smem);
    const uint64_t warps = (uint64_t)b.n_reach * (SPLIT ? 2 : 1);
    const uint64_t want = (warps + threads / 32 - 1) / (threads / 32);
    const uint64_t blocks = std::min<uint64_t>(want, (uint64_t)std::max(per_sm, 1) * sm_count);
    reach_batch_kernel<TM, MS, SPLIT, WIDE><<<(uint32_t)std::max<uint64_t>(blocks, 1), threads, smem, s>>>(b);
}

template <int TM, int MS>
void launch_batch_one(const BatchGroup &b, cudaStream_t s, int sm_count) {
    if (b.recognize) launch_batch_split<TM, MS, false>(b, s, sm_count);
    else launch_batch_split<TM, MS, true>(b, s, sm_count);
}

// More than 8 slots: a parse batch uses wide lanes (4 runs in registers, the
// rest in local memory until they merge); the recognizer batch, which walks
// one chunk in both directions per lane, keeps every run in registers.
template <int TM>
bool launch_ms_batch(const BatchGroup &b, cudaStream_t s, uint32_t ms, int sm_count) {
    constexpr bool FULL = TM != TM_GLOBAL;
    if (FULL && ms <= 2) launch_batch_one<TM, 2>(b, s, sm_count);
    else if (FULL && ms <= 4) launch_batch_one<TM, 4>(b, s, sm_count);
    else if (ms <= 8) launch_batch_one<TM, 8>(b, s, sm_count);
    else if (ms > 32) return false;
    else if (!b.recognize) launch_batch_split<TM, 4, true, true>(b, s, sm_count);
    else if (FULL && ms <= 16) launch_batch_split<TM, 16, false>(b, s, sm_count);
    else launch_batch_split<TM, 32, false>(b, s, sm_count);
    return true;
}

template <int TM, int MS, bool SPLIT, bool WIDE = false, bool MAT = false>
void launch_split(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, int sm_count) {
    const uint32_t threads = SPLIT ? kSplitThreads : kChunkThreads;
    const size_t smem = reach_smem(p.t, TM, threads, SPLIT ? 1 : 2, MAT, p.rstages ? p.rstages : kStages);
    static uint64_t attr_done = 0;
    allow_smem(reach_kernel<TM, MS, SPLIT, WIDE, MAT>, &attr_done);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reach_kernel<TM, MS, SPLIT, WIDE, MAT>, threads, smem);
    const uint64_t warps = ((uint64_t)p.c + 31) / 32 * (SPLIT && !p.recognize ? 2 : 1);
    const uint64_t want = (warps + threads / 32 - 1) / (threads / 32);
    const uint64_t blocks = std::min<uint64_t>(want, (uint64_t)std::max(per_sm, 1) * sm_count);
    launch_dependent(reach_kernel<TM, MS, SPLIT, WIDE, MAT>, (uint32_t)std::max<uint64_t>(blocks, 1), threads, smem,
                     s, p, map, smaps);
}

// A parse: warp pairs per 32-chunk tile; the recognizer: one forward warp per
// tile (the same kernel, so the same register budget and ring depth).  More
// than 8 slots: wide lanes (4 runs in registers, the rest in local memory
// until they merge, which they do within the first bytes of most chunks).
template <int TM>
bool launch_ms(const Params &p, const CUtensorMap &map, const StateMaps &smaps, cudaStream_t s, uint32_t ms,
               int sm_count) {
    constexpr bool FULL = TM != TM_GLOBAL;          // fewer instantiations for the rare global mode
    if (p.rvar == 4) {                              // one lane per chunk, both directions: every run in registers
        if (FULL && ms <= 2) launch_split<TM, 2, false>(p, map, smaps, s, sm_count);
        else if (FULL && ms <= 4) launch_split<TM, 4, false>(p, map, smaps, s, sm_count);
        else if (ms <= 8) launch_split<TM, 8, false>(p, map, smaps, s, sm_count);
        else if (FULL && ms <= 16) launch_split<TM, 16, false>(p, map, smaps, s, sm_count);
        else if (ms <= 32) launch_split<TM, 32, false>(p, map, smaps, s, sm_count);
        else return false;
        return true;
    }
    if constexpr (TM == TM_SMEM8) {                 // per-position states (mat) only here
        if (p.mat) {
            if (ms <= 2) launch_split<TM, 2, true, false, true>(p, map, smaps, s, sm_count);
            else if (ms <= 4) launch_split<TM, 4, true, false, true>(p, map, smaps, s, sm_count);
            else if (ms <= 8) launch_split<TM, 8, true, false, true>(p, map, smaps, s, sm_count);
            else if (ms <= 32) launch_split<TM, 4, true, true, true>(p, map, smaps, s, sm_count);
            else return false;
            return true;
        }
    }
    if (FULL && ms <= 2) launch_split<TM, 2, true>(p, map, smaps, s, sm_count);
    else if (FULL && ms <= 4) launch_split<TM, 4, true>(p, map, smaps, s, sm_count);
    else if (ms <= 8) launch_split<TM, 8, true>(p, map, smaps, s, sm_count);
    else if (ms <= 32) launch_split<TM, 4, true, true>(p, map, smaps, s, sm_count);
    else return false;
    return true;
}

}  // namespace reach
}  // namespace slpf
