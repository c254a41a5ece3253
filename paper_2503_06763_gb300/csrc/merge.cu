// Checkpoint fix-up and build & merge (arXiv 2503.06763, Eqs. builder and
// merger, Fig. builders&merger, compose of Sect. 3.2).
//
// fix-up: the exact checkpoints a chunk's reach runs could not give before
//   they met.  At every recorded boundary the exact state is the union, over
//   the runs whose slot set the chunk's input J_{i-1} (or Ĵ_{i+1}) enters, of
//   the run states: Eq. joiner applied at sub-chunk granularity.  Boundaries
//   beyond the record are walked with the DFA from the last exact state,
//   with the tables staged in shared memory.
// build & merge: one thread per column group g (64 columns).  The forward
//   builder (B from FC[g]) and the backward builder (B̂ from BC[g]) run at the
//   same time from the two ends of the group, keep their first 32 states
//   (in registers with two-byte tables, in shared memory otherwise), meet in
//   the middle and then merge while they proceed to the
//   opposite ends: each new state is intersected with the stored state of the
//   other direction, C_r = B_r ∩ B̂_r (Eq. merger), and written in the
//   requested encoding (DENSE bitset, or DICT index through the pair table
//   built at compile time).  This is the fused builder & merger schedule of
//   Sect. 3.3 (Fig. builders&merger, merging from the midpoint outwards).
#include <type_traits>

#include "kernels.cuh"

namespace slpf {
namespace {

// ------------------------------------------------------------------ fix-up
__device__ uint32_t probe_state(const uint32_t *hash, uint32_t mask, const uint64_t *bits, uint32_t W,
                                const uint64_t *key) {
    uint64_t h = bits_hash(key, W) & mask;
    for (uint32_t step = 0; step <= mask; ++step) {
        const uint32_t id = __ldg(hash + h);
        if (id == 0) return 0;
        bool eq = true;
        for (uint32_t w = 0; w < W; ++w)
            if (__ldg(bits + (size_t)id * W + w) != key[w]) { eq = false; break; }
        if (eq) return id;
        h = (h + 1) & mask;
    }
    return 0;
}

// Exact state at a recorded boundary: union of the runs whose slots H enters.
// The entries are loaded up front (independent loads); the union of W <= 2
// words stays in registers.
__device__ uint32_t record_union(const Params &p, bool fwd, const uint2 *ent, uint32_t cnt, uint32_t H, bool &bad) {
    const DevTables &t = p.t;
    const uint32_t W = t.W;
    const uint64_t *bits = fwd ? t.fBits : t.bBits;
    uint2 r[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) r[e] = (e < (int)cnt) ? ent[e] : make_uint2(0u, 0u);
    uint32_t single = 0;
    bool multi = false;
    if (W <= 2 && cnt <= 8) {
        uint64_t a0 = 0, a1 = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if (!(r[e].y & H)) continue;                         // empty entries have no slots
            const uint32_t st = r[e].x;
            if (!single) single = st;
            else if (st != single) multi = true;
            a0 |= __ldg(bits + (size_t)st * W);
            if (W == 2) a1 |= __ldg(bits + (size_t)st * W + 1);
        }
        if (!multi) return single;
        const uint64_t key[2] = {a0, a1};
        const uint32_t id = fwd ? probe_state(t.fHash, t.fHashMask, t.fBits, W, key)
                                : probe_state(t.bHash, t.bHashMask, t.bBits, W, key);
        if (!id) bad = true;
        return id;
    }
    uint64_t acc[kMaxW];
    for (uint32_t w = 0; w < W; ++w) acc[w] = 0;
    for (uint32_t e = 0; e < cnt; ++e) {
        const uint2 q = e < 8 ? r[e] : ent[e];
        if (!(q.y & H)) continue;
        if (!single) single = q.x;
        else if (q.x != single) multi = true;
        for (uint32_t w = 0; w < W; ++w) acc[w] |= __ldg(bits + (size_t)q.x * W + w);
    }
    if (!multi) return single;
    const uint32_t id = fwd ? probe_state(t.fHash, t.fHashMask, t.fBits, W, acc)
                            : probe_state(t.bHash, t.bHashMask, t.bBits, W, acc);
    if (!id) bad = true;
    return id;
}

// Fast walk of bytes [t0, t1) of a chunk (forward) with the staged tables:
// two bytes per lookup where pair tables exist.  Calls at(tt+1, state) after
// every byte tt whose successor boundary (tt+1) is a multiple of 64.
template <int TM, typename F>
__device__ __forceinline__ uint32_t walk_fwd(const Params &p, const Tabs &T, uint64_t base, uint32_t t0, uint32_t t1,
                                             uint32_t st, F at) {
    uint32_t tt = t0;
    for (; tt < t1 && (tt & 15); ++tt) {                          // to a 16-byte boundary
        st = fnext<TM>(T, st, clsof<TM>(T, __ldg(p.x + base + tt)));
        if (((tt + 1) & 63) == 0) at(tt + 1, st);
    }
    for (; tt + 16 <= t1; tt += 16) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p.x + base + tt));
        if (TM == TM_PAIR) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                st = fpair(T, st, clsof<TM>(T, byte_of(v, 2 * j)) * T.ncls + clsof<TM>(T, byte_of(v, 2 * j + 1))) >> 16;
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) st = fnext<TM>(T, st, clsof<TM>(T, byte_of(v, j)));
        }
        if (((tt + 16) & 63) == 0) at(tt + 16, st);
    }
    for (; tt < t1; ++tt) {
        st = fnext<TM>(T, st, clsof<TM>(T, __ldg(p.x + base + tt)));
        if (((tt + 1) & 63) == 0) at(tt + 1, st);
    }
    return st;
}

// Backward walk of bytes t1-1 down to t0 (t0, t1 multiples of 64 or t1 = len);
// calls at(tt, state) after every byte tt that is a multiple of 64.
template <int TM, typename F>
__device__ __forceinline__ uint32_t walk_bwd(const Params &p, const Tabs &T, uint64_t base, uint32_t t0, uint32_t t1,
                                             uint32_t st, F at) {
    int64_t tt = (int64_t)t1 - 1;
    for (; tt >= (int64_t)t0 && ((tt + 1) & 15); --tt) {          // down to a 16-byte boundary
        st = bnext<TM>(T, st, clsof<TM>(T, __ldg(p.x + base + tt)));
        if ((tt & 63) == 0) at((uint32_t)tt, st);
    }
    for (; tt - 15 >= (int64_t)t0; tt -= 16) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p.x + base + tt - 15));
        if (TM == TM_PAIR) {
#pragma unroll
            for (int j = 7; j >= 0; --j)
                st = bpair(T, st, clsof<TM>(T, byte_of(v, 2 * j)) * T.ncls + clsof<TM>(T, byte_of(v, 2 * j + 1))) >> 16;
        } else {
#pragma unroll
            for (int j = 15; j >= 0; --j) st = bnext<TM>(T, st, clsof<TM>(T, byte_of(v, j)));
        }
        if (((tt - 15) & 63) == 0) at((uint32_t)(tt - 15), st);
    }
    for (; tt >= (int64_t)t0; --tt) {
        st = bnext<TM>(T, st, clsof<TM>(T, __ldg(p.x + base + tt)));
        if ((tt & 63) == 0) at((uint32_t)tt, st);
    }
    return st;
}

// Boundaries of chunk i past its record (nrec records; `from` the state at
// the last recorded boundary): walked with the DFA from the last exact state.
template <int TM>
__device__ void fixup_walk(const Params &p, const Tabs &T, uint64_t i, bool fwd, uint32_t nrec, uint32_t conv,
                           uint32_t from) {
    const uint64_t base = i * p.k;
    const uint32_t len = chunk_len(p, (uint32_t)i);
    const uint32_t nsub = (len + 63) / 64;
    const uint64_t g0 = i * p.S;
    if (fwd) {
        if (nrec + 1 <= conv - 1) {                             // walk boundaries nrec+1 .. conv-1
            const uint32_t start = nrec == 0 ? p.w.FJ[i] : from;
            walk_fwd<TM>(p, T, base, 64 * nrec, 64 * (conv - 1), start,
                         [&](uint32_t b, uint32_t s2) { p.w.FC[g0 + b / 64] = s2; });
        }
    } else {
        const uint32_t bb_first = nsub - 1 - nrec;              // first boundary not recorded
        if (bb_first > conv) {                                  // walk boundaries bb_first .. conv+1
            const uint32_t start = nrec == 0 ? p.w.BJ[i + 1] : from;
            const uint32_t t1 = nrec == 0 ? len : 64 * (bb_first + 1);
            walk_bwd<TM>(p, T, base, 64 * (conv + 1), t1, start,
                         [&](uint32_t b, uint32_t s2) { p.w.BC[g0 + b / 64 - 1] = s2; });
        }
    }
}

// A fix-up block takes kFixItems (chunk, direction) items at a time and
// spreads all their records over its threads, one record per thread: the
// number of records per item varies widely (most chunks' runs meet after a
// few boundaries, a run inside a long match may stay apart for the whole
// record), so a thread per item would leave each warp waiting for its
// longest record chain.
constexpr uint32_t kFixItems = 32;

struct FixShared {
    uint32_t chunk[kFixItems], text[kFixItems], nrec[kFixItems], H[kFixItems], conv[kFixItems];
    uint32_t walk[kFixItems];                 // 1: boundaries past the record remain (after record nrec-1)
    uint32_t first[kFixItems + 1];            // flat index of each item's first record
    uint32_t off[kFixItems][kRecBounds];      // entry offset of each record in its item's row
    uint32_t cnt[kFixItems][kRecBounds];      // entries of each record
    uint32_t ok;
};

// Item slot q of a block iteration: its text, chunk and direction; live =
// an item of a text still being parsed.
struct FixRef {
    uint32_t ti;
    uint64_t i;
    bool fwd, live;
};

// Sets the item's entries in S (warp 0, lane = slot); an inactive item gets
// no records and no walk.  Its three words are loaded together.
__device__ __forceinline__ void fix_item(const Params &p, FixShared &S, uint32_t slot, const FixRef &r) {
    uint32_t conv = 0, nrec = 0, H = 0, walk = 0;
    if (r.live) {
        const uint64_t i = r.i;
        const uint32_t c0 = r.fwd ? p.w.fconv[i] : p.w.bconv[i];
        const uint32_t n0 = r.fwd ? p.w.fnrec[i] : p.w.bnrec[i];
        const uint32_t h0 = r.fwd ? p.w.fhit[i] : p.w.bhit[i];
        const uint32_t nsub = (chunk_len(p, (uint32_t)i) + 63) / 64;
        if (r.fwd) {
            if (c0 > 1) { conv = c0; nrec = n0; H = h0; walk = nrec + 1 <= conv - 1; }   // boundaries 1 .. conv-1
        } else if (!p.recognize && nsub >= 2 && c0 + 1 <= nsub - 1) {                  // boundaries nsub-1 .. conv+1
            conv = c0; nrec = n0; H = h0; walk = nsub - 1 - nrec > conv;
        }
    }
    S.chunk[slot] = (uint32_t)r.i;
    S.text[slot] = r.ti;
    S.nrec[slot] = nrec;
    S.H[slot] = H;
    S.conv[slot] = conv;
    S.walk[slot] = (r.fwd ? 2u : 0u) | walk;                  // bit 1: forward
}

// One block iteration over kFixItems items: R(q) gives item slot q, P(ti)
// the Params of text ti.  Item words and record counts are loaded in one
// round (a count row depends only on the chunk), then scanned; then one
// record per thread; then the walks.  A record whose union is no DFA state
// marks its text's status RE_E_INTERNAL.  Called by the whole block.
template <int TM, typename RF, typename PF>
__device__ void fix_block(const Tabs &T, FixShared &S, RF R, PF P) {
    constexpr uint32_t kWarps = kFixupThreads / 32, kPer = kFixItems / kWarps;
    static_assert(kFixItems % kWarps == 0, "items per warp");
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        const FixRef r = R(lane);
        fix_item(P(r.ti), S, lane, r);
    }
    uint32_t raw[kPer];                                        // count of record `lane` of this warp's items
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
        const FixRef r = R(warp + kWarps * k);
        raw[k] = 0;
        if (r.live) {
            const Params &p = P(r.ti);
            raw[k] = ((r.fwd ? p.w.recFc : p.w.recBc) + r.i * kRecBounds)[lane];
        }
    }
    __syncthreads();
    if (warp == 0) {                                            // first[]: exclusive scan of nrec
        const uint32_t v = S.nrec[lane];
        uint32_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if ((int)lane >= d) x += y;
        }
        S.first[lane] = x - v;
        if (lane == 31) S.first[kFixItems] = x;
    }
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {                      // entry offsets of each item's records
        const uint32_t q = warp + kWarps * k;
        const uint32_t c = lane < S.nrec[q] ? raw[k] : 0u;
        uint32_t x = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if ((int)lane >= d) x += y;
        }
        S.off[q][lane] = x - c;
        S.cnt[q][lane] = c;
    }
    __syncthreads();
    const uint32_t total = S.first[kFixItems];
    for (uint32_t f = threadIdx.x; f < total; f += blockDim.x) {
        uint32_t lo = 0, hi = kFixItems;                        // item q: first[q] <= f < first[q+1]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (S.first[mid] <= f) lo = mid; else hi = mid;
        }
        const uint32_t q = lo, r = f - S.first[q];
        const Params &p = P(S.text[q]);
        const bool fwd = S.walk[q] & 2u;
        const uint64_t i = S.chunk[q];
        const uint2 *ent = (fwd ? p.w.recFe : p.w.recBe) + i * kRecEntries + S.off[q][r];
        bool bad = false;
        const uint32_t st = record_union(p, fwd, ent, S.cnt[q][r], S.H[q], bad);
        if (bad) atomicExch(p.status, RE_E_INTERNAL);
        const uint64_t g0 = i * p.S;
        if (fwd) {
            p.w.FC[g0 + r + 1] = st;                            // record r: boundary r+1
        } else {
            const uint32_t nsub = (chunk_len(p, (uint32_t)i) + 63) / 64;
            p.w.BC[g0 + (nsub - 1 - r) - 1] = st;               // record r: boundary nsub-1-r
        }
        if (r + 1 == S.nrec[q] && (S.walk[q] & 1u)) fixup_walk<TM>(p, T, i, fwd, S.nrec[q], S.conv[q], st);
    }
    if (threadIdx.x < kFixItems && S.nrec[threadIdx.x] == 0 && (S.walk[threadIdx.x] & 1u)) {   // walks with no record
        const uint32_t q = threadIdx.x;
        fixup_walk<TM>(P(S.text[q]), T, S.chunk[q], S.walk[q] & 2u, 0u, S.conv[q], 0u);
    }
    __syncthreads();                                            // S is refilled next
}

// Items 0 .. c-1 are the chunks' forward directions, c .. 2c-1 their
// backward ones.
template <int TM>
__global__ void __launch_bounds__(kFixupThreads, 4) fixup_kernel(const __grid_constant__ Params p) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ FixShared S;
    Tabs T;
    stage_tables<TM>(p.t, sm, T);
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) S.ok = *p.status == RE_OK;
    __syncthreads();
    if (!S.ok) return;                                          // block-uniform
    const uint64_t items = 2 * (uint64_t)p.c;
    for (uint64_t q0 = (uint64_t)blockIdx.x * kFixItems; q0 < items; q0 += (uint64_t)gridDim.x * kFixItems) {
        auto ref = [&](uint32_t q) -> FixRef {
            const uint64_t j = q0 + q;
            const bool fwd = j < p.c;
            return FixRef{0u, fwd ? j : j - p.c, fwd, j < items};
        };
        fix_block<TM>(T, S, ref, [&](uint32_t) -> const Params & { return p; });
    }
}

// Batch: the same items over the flat chunks of every text of the group.
template <int TM>
__global__ void __launch_bounds__(kFixupThreads, 4) fixup_batch_kernel(const __grid_constant__ BatchGroup b) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ FixShared S;
    Tabs T;
    stage_tables<TM>(b.t, sm, T);
    const uint64_t items = 2 * b.chunks;
    for (uint64_t q0 = (uint64_t)blockIdx.x * kFixItems; q0 < items; q0 += (uint64_t)gridDim.x * kFixItems) {
        auto ref = [&](uint32_t q) -> FixRef {
            const uint64_t j = q0 + q;
            if (j >= items) return FixRef{0u, 0u, true, false};
            const bool fwd = j < b.chunks;
            const uint64_t f = fwd ? j : j - b.chunks;
            const uint32_t ti = text_of(b.chunk_base, b.nt, f);
            const bool live = *b.texts[ti].status == RE_OK;
            return FixRef{ti, live ? f - b.chunk_base[ti] : 0u, fwd, live};
        };
        fix_block<TM>(T, S, ref, [&](uint32_t ti) -> const Params & { return b.texts[ti]; });
    }
}

// ------------------------------------------------------------------ encodings
// DENSE bitsets (D), DICT indices (X), PAIRS of state ids (P: forward id in
// the low half, backward id in the high half).
enum { ENC_D1 = 1, ENC_D2 = 2, ENC_D4 = 4, ENC_D8 = 8, ENC_X1 = 0x11, ENC_X2 = 0x12, ENC_X4 = 0x14,
       ENC_P4 = 0x24, ENC_P8 = 0x28 };
constexpr bool is_dict(int E) { return E == ENC_X1 || E == ENC_X2 || E == ENC_X4; }
constexpr bool is_pair(int E) { return E == ENC_P4 || E == ENC_P8; }

struct Enc {
    const uint64_t *fbits, *bbits;   // DENSE: segment set of each state (W == 1)
    const uint8_t *pt8;              // DICT, fewer than 255 columns: pair table in shared memory (u8)
    const uint16_t *pt16;            // DICT: pair table in shared memory (u16)
    const uint32_t *pt32;            // DICT: pair table (u32; shared or global)
    uint32_t nb;
};

template <int E>
__device__ __forceinline__ uint32_t enc_lo(const Enc &e, uint32_t f, uint32_t b, bool &bad) {
    if (is_dict(E)) {
        const uint32_t at = f * e.nb + b;                 // the pair table spans every state pair
        if (E == ENC_X1 && e.pt8) return e.pt8[at];
        return e.pt16 ? (uint32_t)e.pt16[at] : e.pt32[at];
    }
    if (E == ENC_P4) return f | (b << 16);
    return (uint32_t)(e.fbits[f] & e.bbits[b]);
}
__device__ __forceinline__ uint64_t enc_d8(const Enc &e, uint32_t f, uint32_t b) { return e.fbits[f] & e.bbits[b]; }

template <int E>
__device__ __forceinline__ void store_col(void *out, uint64_t r, uint64_t v) {
    if (E == ENC_D1 || E == ENC_X1) reinterpret_cast<uint8_t *>(out)[r] = (uint8_t)v;
    else if (E == ENC_D2 || E == ENC_X2) reinterpret_cast<uint16_t *>(out)[r] = (uint16_t)v;
    else if (E == ENC_D4 || E == ENC_X4 || E == ENC_P4) reinterpret_cast<uint32_t *>(out)[r] = (uint32_t)v;
    else reinterpret_cast<uint64_t *>(out)[r] = v;
}

constexpr int bytes_of(int E) {
    return (E == ENC_X1) ? 1 : (E == ENC_X2) ? 2 : (E == ENC_X4 || E == ENC_P4) ? 4 : (E == ENC_P8) ? 8 : E;
}

// Put one column value into a 16-byte vector being assembled (slot k).
template <int CB>
__device__ __forceinline__ void put_col(uint32_t (&w4)[4], int k, uint64_t v) {
    if constexpr (CB == 8) {
        w4[2 * k] = (uint32_t)v;
        w4[2 * k + 1] = (uint32_t)(v >> 32);
    } else if constexpr (CB == 4) {
        w4[k] = (uint32_t)v;
    } else {
        constexpr uint32_t m = (1u << (8 * CB)) - 1;
        w4[(k * CB) >> 2] |= ((uint32_t)v & m) << (8 * ((k * CB) & 3));
    }
}

template <int TM, int E>
__device__ __forceinline__ uint64_t enc_col(const Enc &e, uint32_t f, uint32_t b, bool &bad) {
    if (E == ENC_P8) return (uint64_t)f | ((uint64_t)b << 32);
    if (bytes_of(E) == 8) return enc_d8(e, f, b);
    return enc_lo<E>(e, f, b, bad);
}

// Where a full group's 16-byte output vectors go: straight to global memory,
// or into this lane's row of the warp's shared-memory tile, swizzled the way
// the TMA tensor store reads it (SWIZZLE_128B for 128-byte rows, 64B for
// 64-byte rows: 16-byte chunk j of row r sits at chunk j ^ f(r)).
template <bool TMA, int CB>
struct Sink {
    uint4 *g;
    uint8_t *row;
    uint32_t lane;
    __device__ __forceinline__ void put(int chunk, uint4 v) const {
        if constexpr (TMA) {
            const uint32_t sw = (CB == 2) ? ((uint32_t)chunk ^ (lane & 7)) : ((uint32_t)chunk ^ ((lane >> 1) & 3));
            *reinterpret_cast<uint4 *>(row + (sw << 4)) = v;
        } else {
            g[chunk] = v;
        }
    }
};

// Full group (one-byte tables): forward states B_0..B_31 and backward states
// B̂_32..B̂_63 go to this thread's column of sF / sB (stride kBlockThreads),
// then the two builders continue past the midpoint and merge.
template <int TM, int E, bool TMA, typename St>
__device__ __forceinline__ void group_full(const Params &p, const Tabs &T, const Enc &e, uint64_t g, bool &bad,
                                           St *sF, St *sB, const Sink<TMA, bytes_of(E)> &out) {
    constexpr uint32_t BD = kBlockThreads;                     // compile-time stride: immediate offsets
    const uint64_t pos = g * 64;
    uint32_t cw[16];                                           // byte classes, four per register
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p.x + pos) + q);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            cw[4 * q + j] = clsof<TM>(T, w[j] & 0xFF) | (clsof<TM>(T, (w[j] >> 8) & 0xFF) << 8) |
                            (clsof<TM>(T, (w[j] >> 16) & 0xFF) << 16) | (clsof<TM>(T, w[j] >> 24) << 24);
    }
    auto cls_at = [&](int u) -> uint32_t { return (cw[u >> 2] >> (8 * (u & 3))) & 0xFFu; };
    uint32_t f = p.w.FC[g];
    uint32_t b = p.w.BC[g];                                    // B̂_64
    if (f == kUnknown || b == kUnknown) { bad = true; f = 0; b = 0; }   // never index with the sentinel
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if (i > 0) f = fnext<TM>(T, f, cls_at(i - 1));        // B_i
        sF[i * BD] = (St)f;
        b = bnext<TM>(T, b, cls_at(63 - i));                  // B̂_{63-i}
        sB[(31 - i) * BD] = (St)b;
        asm volatile("" ::: "memory");                        // keep shared-memory traffic in its step
    }
    constexpr int CB = bytes_of(E);
    constexpr int CPV = 16 / CB;                               // columns per 16-byte vector
    uint32_t wf[4] = {0, 0, 0, 0}, wb[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 32; i < 64; ++i) {
        f = fnext<TM>(T, f, cls_at(i - 1));                   // B_i
        b = bnext<TM>(T, b, cls_at(63 - i));                  // B̂_{63-i}
        const uint64_t vf = enc_col<TM, E>(e, f, sB[(i - 32) * BD], bad);          // column i
        const uint64_t vb = enc_col<TM, E>(e, sF[(63 - i) * BD], b, bad);          // column 63-i
        put_col<CB>(wf, i % CPV, vf);
        if (i % CPV == CPV - 1) {
            out.put(i / CPV, make_uint4(wf[0], wf[1], wf[2], wf[3]));
            wf[0] = wf[1] = wf[2] = wf[3] = 0;
        }
        put_col<CB>(wb, (63 - i) % CPV, vb);
        if ((63 - i) % CPV == 0) {
            out.put((63 - i) / CPV, make_uint4(wb[0], wb[1], wb[2], wb[3]));
            wb[0] = wb[1] = wb[2] = wb[3] = 0;
        }
        asm volatile("" ::: "memory");
    }
}

// Full group with two-byte tables: pair j holds bytes 2j, 2j+1.  Forward:
// B_{2j} -> (B_{2j+1}, B_{2j+2}); backward: B̂_{2j+2} -> (B̂_{2j+1}, B̂_{2j}).
// The first half of each direction stays in registers (two states per word).
template <int E, bool TMA>
__device__ __forceinline__ void group_full_pair(const Params &p, const Tabs &T, const Enc &e, uint64_t g, bool &bad,
                                                const Sink<TMA, bytes_of(E)> &out) {
    const uint64_t pos = g * 64;
    uint32_t cpk[8];                                           // class pair of every byte pair, four per word
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p.x + pos) + q);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t c0 = clsof<TM_PAIR>(T, w[j] & 0xFF) * T.ncls + clsof<TM_PAIR>(T, (w[j] >> 8) & 0xFF);
            const uint32_t c1 = clsof<TM_PAIR>(T, (w[j] >> 16) & 0xFF) * T.ncls + clsof<TM_PAIR>(T, w[j] >> 24);
            const uint32_t two = c0 | (c1 << 8);
            if (j < 2) lo |= two << (16 * j);
            else hi |= two << (16 * (j - 2));
        }
        cpk[2 * q] = lo;
        cpk[2 * q + 1] = hi;
    }
    auto cp_at = [&](int j) -> uint32_t { return (cpk[j >> 2] >> (8 * (j & 3))) & 0xFFu; };
    uint32_t f = p.w.FC[g];                                    // B_0
    uint32_t b = p.w.BC[g];                                    // B̂_64
    if (f == kUnknown || b == kUnknown) { bad = true; f = 0; b = 0; }
    uint32_t sF[16], sB[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t ef = fpair(T, f, cp_at(i));             // pair i: B_{2i+1}, B_{2i+2}
        sF[i] = f | (ef << 16);                                // B_{2i}, B_{2i+1}
        f = ef >> 16;
        const uint32_t eb = bpair(T, b, cp_at(31 - i));        // pair 31-i: B̂_{63-2i}, B̂_{62-2i}
        sB[i] = (eb >> 16) | (eb << 16);                       // B̂_{62-2i}, B̂_{63-2i}
        b = eb >> 16;
    }
    constexpr int CB = bytes_of(E);
    constexpr int CPV = 16 / CB;
    uint32_t wf[4] = {0, 0, 0, 0}, wb[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 16; i < 32; ++i) {
        // forward pair i: columns 2i, 2i+1 (ascending); their B̂ were stored at step 31-i
        const uint32_t ef = fpair(T, f, cp_at(i));
        const uint32_t hb = sB[31 - i];
        const uint64_t v0 = enc_col<TM_PAIR, E>(e, f, hb & 0xFFFF, bad);
        const uint64_t v1 = enc_col<TM_PAIR, E>(e, ef & 0xFFFF, hb >> 16, bad);
        f = ef >> 16;
        // backward pair jb = 31-i: columns 2jb+1, 2jb (descending); their B were stored at step jb
        const int jb = 31 - i;
        const uint32_t eb = bpair(T, b, cp_at(jb));
        const uint32_t hf = sF[jb];
        const uint64_t u1 = enc_col<TM_PAIR, E>(e, hf >> 16, eb & 0xFFFF, bad);
        const uint64_t u0 = enc_col<TM_PAIR, E>(e, hf & 0xFFFF, eb >> 16, bad);
        b = eb >> 16;
        const int c0 = 2 * i, d1 = 2 * jb + 1;
        put_col<CB>(wf, c0 % CPV, v0);
        put_col<CB>(wf, (c0 + 1) % CPV, v1);
        if ((c0 + 1) % CPV == CPV - 1) {
            out.put((c0 + 1) / CPV, make_uint4(wf[0], wf[1], wf[2], wf[3]));
            wf[0] = wf[1] = wf[2] = wf[3] = 0;
        }
        put_col<CB>(wb, d1 % CPV, u1);
        put_col<CB>(wb, (d1 - 1) % CPV, u0);
        if ((d1 - 1) % CPV == 0) {
            out.put((d1 - 1) / CPV, make_uint4(wb[0], wb[1], wb[2], wb[3]));
            wb[0] = wb[1] = wb[2] = wb[3] = 0;
        }
    }
}

// Full group with one-byte tables over the classic-DFA rows: as group_full,
// but the first half of each direction stays in registers, two 16-bit states
// per word (fully unrolled, so every index is static), instead of a staged
// column per thread in shared memory.
template <int E, bool TMA>
__device__ __forceinline__ void group_full_reg(const Params &p, const Tabs &T, const Enc &e, uint64_t g, bool &bad,
                                               const Sink<TMA, bytes_of(E)> &out) {
    const uint64_t pos = g * 64;
    uint32_t cw[16];                                           // byte classes, four per register
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p.x + pos) + q);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            cw[4 * q + j] = clsof<TM_SMEM>(T, w[j] & 0xFF) | (clsof<TM_SMEM>(T, (w[j] >> 8) & 0xFF) << 8) |
                            (clsof<TM_SMEM>(T, (w[j] >> 16) & 0xFF) << 16) | (clsof<TM_SMEM>(T, w[j] >> 24) << 24);
    }
    auto cls_at = [&](int u) -> uint32_t { return (cw[u >> 2] >> (8 * (u & 3))) & 0xFFu; };
    uint32_t f = p.w.FC[g];                                    // B_0
    uint32_t b = p.w.BC[g];                                    // B̂_64
    if (f == kUnknown || b == kUnknown || f > p.t.nfd || b > p.t.nbd) { bad = true; f = 0; b = 0; }
    uint32_t rF[16], rB[16];                                   // B_0..B_31; B̂_32..B̂_63 (two per word)
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if (i > 0) f = fnext<TM_SMEM>(T, f, cls_at(i - 1));   // B_i
        if (i & 1) rF[i >> 1] |= f << 16; else rF[i >> 1] = f;
        b = bnext<TM_SMEM>(T, b, cls_at(63 - i));             // B̂_{63-i}
        const int j = 31 - i;                                  // B̂_{32+j}; j runs down, odd j first
        if (j & 1) rB[j >> 1] = b << 16; else rB[j >> 1] |= b;
    }
    constexpr int CB = bytes_of(E);
    constexpr int CPV = 16 / CB;                               // columns per 16-byte vector
    uint32_t wf[4] = {0, 0, 0, 0}, wb[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 32; i < 64; ++i) {
        f = fnext<TM_SMEM>(T, f, cls_at(i - 1));              // B_i
        b = bnext<TM_SMEM>(T, b, cls_at(63 - i));             // B̂_{63-i}
        const int jb = i - 32, jf = 63 - i;
        const uint32_t hb = (rB[jb >> 1] >> (16 * (jb & 1))) & 0xFFFFu;   // B̂_i
        const uint32_t hf = (rF[jf >> 1] >> (16 * (jf & 1))) & 0xFFFFu;   // B_{63-i}
        const uint64_t vf = enc_col<TM_SMEM, E>(e, f, hb, bad);           // column i
        const uint64_t vb = enc_col<TM_SMEM, E>(e, hf, b, bad);           // column 63-i
        put_col<CB>(wf, i % CPV, vf);
        if (i % CPV == CPV - 1) {
            out.put(i / CPV, make_uint4(wf[0], wf[1], wf[2], wf[3]));
            wf[0] = wf[1] = wf[2] = wf[3] = 0;
        }
        put_col<CB>(wb, (63 - i) % CPV, vb);
        if ((63 - i) % CPV == 0) {
            out.put((63 - i) / CPV, make_uint4(wb[0], wb[1], wb[2], wb[3]));
            wb[0] = wb[1] = wb[2] = wb[3] = 0;
        }
    }
}

// Last group (fewer than 64 columns or no byte after it): plain loops.
template <int TM, int E, bool REG = false>
__device__ void group_tail(const Params &p, const Tabs &T, const Enc &e, uint64_t g, bool &bad) {
    const uint64_t pos = g * 64;
    const uint64_t nleft = p.n + 1 - pos;
    const uint32_t ncol = nleft < 64 ? (uint32_t)nleft : 64u;
    uint32_t F[64], B[64];
    uint32_t f = p.w.FC[g], b = p.w.BC[g];
    if (f == kUnknown || b == kUnknown || (REG && (f > p.t.nfd || b > p.t.nbd))) { bad = true; f = 0; b = 0; }
    F[0] = f;
    for (uint32_t u = 1; u < ncol; ++u) F[u] = fnext<TM>(T, F[u - 1], clsof<TM>(T, __ldg(p.x + pos + u - 1)));
    if (pos + 64 <= p.n) b = bnext<TM>(T, b, clsof<TM>(T, __ldg(p.x + pos + 63)));
    B[ncol - 1] = b;
    for (int u = (int)ncol - 2; u >= 0; --u) B[u] = bnext<TM>(T, B[u + 1], clsof<TM>(T, __ldg(p.x + pos + u)));
    for (uint32_t u = 0; u < ncol; ++u) {
        const uint64_t v = enc_col<TM, E>(e, F[u], B[u], bad);
        store_col<E>(p.out, pos + u, v);
    }
}

// Shared-memory set-up of a merge block: staged tables, the per-thread state
// stage (one-byte tables) and the encoder (pair table or segment bitsets).
// With REG (one-byte tables, merge_reg) only the classic-DFA rows are staged
// and the encoder covers classic-DFA state pairs only (row stride nbd + 1);
// there is no state stage.
template <int TM, int E, bool REG, typename St>
__device__ void merge_setup(const DevTables &t0, uint32_t enc_in_smem, uint8_t *base, Tabs &T, St *&stage, Enc &e) {
    const DevTables t = REG ? dfa_tables(t0) : t0;
    uint8_t *rest = stage_tables<TM>(t, base, T);
    stage = reinterpret_cast<St *>(rest);                     // [2][32][kBlockThreads] (one-byte tables)
    if (TM != TM_PAIR && !REG) rest += (2 * 32 * kBlockThreads * sizeof(St) + 15) & ~(size_t)15;
    e = Enc{};
    e.nb = t.nb;
    if (is_pair(E)) {                                         // the state ids themselves: no encoder
    } else if (is_dict(E)) {
        if (enc_in_smem) {
            const size_t cnt = (size_t)t.nf * t.nb;
            const uint32_t nbs = t0.nb;                       // row stride of the device pair table
            auto src = [&](size_t i) -> uint32_t {
                return REG ? __ldg(t.pt + (i / t.nb) * nbs + i % t.nb) : __ldg(t.pt + i);
            };
            if (E == ENC_X1) {                                // indices below 255 (0xFF: never produced)
                uint8_t *pt = rest;
                for (size_t i = threadIdx.x; i < cnt; i += blockDim.x) pt[i] = (uint8_t)src(i);
                e.pt8 = pt;
            } else if (E == ENC_X2) {
                uint16_t *pt = reinterpret_cast<uint16_t *>(rest);
                for (size_t i = threadIdx.x; i < cnt; i += blockDim.x) pt[i] = (uint16_t)src(i);
                e.pt16 = pt;
            } else {
                uint32_t *pt = reinterpret_cast<uint32_t *>(rest);
                for (size_t i = threadIdx.x; i < cnt; i += blockDim.x) pt[i] = src(i);
                e.pt32 = pt;
            }
        } else {
            e.pt32 = t.pt;
            e.nb = t0.nb;
        }
    } else if (enc_in_smem) {                                 // DENSE: segment bitsets of the states
        uint64_t *fb = reinterpret_cast<uint64_t *>(rest);
        uint64_t *bb = fb + t.nf;
        for (uint32_t i = threadIdx.x; i < t.nf; i += blockDim.x) fb[i] = __ldg(t.fBits + i);
        for (uint32_t i = threadIdx.x; i < t.nb; i += blockDim.x) bb[i] = __ldg(t.bBits + i);
        e.fbits = fb; e.bbits = bb;
    } else {
        e.fbits = t.fBits; e.bbits = t.bBits;                 // too many states to stage
    }
    __syncthreads();
}

// Columns of group g of one text (this lane's group of its warp's tile).
template <int TM, int E, bool TMA, bool REG, typename St>
__device__ __forceinline__ void merge_group(const Params &p, const Tabs &T, const Enc &e, St *stage, uint64_t g,
                                            bool ok, bool &bad, const Sink<TMA, bytes_of(E)> &out) {
    constexpr uint32_t ROWB = 64 * bytes_of(E);
    if (g >= p.Gc) return;
    if (!ok) {                                                // rejected text: every column is empty
        if (TMA && g < p.Gfast) {
#pragma unroll
            for (int v = 0; v < (int)(ROWB / 16); ++v) out.put(v, make_uint4(0, 0, 0, 0));
        } else {
            const uint64_t pos = g * 64;
            const uint64_t nleft = p.n + 1 - pos;
            const uint32_t ncol = nleft < 64 ? (uint32_t)nleft : 64u;
            for (uint32_t u = 0; u < ncol; ++u) store_col<E>(p.out, pos + u, 0);
        }
    } else if (g < p.Gfast) {
        if constexpr (TM == TM_PAIR)
            group_full_pair<E, TMA>(p, T, e, g, bad, out);
        else if constexpr (REG)
            group_full_reg<E, TMA>(p, T, e, g, bad, out);
        else
            group_full<TM, E, TMA, St>(p, T, e, g, bad, stage + threadIdx.x, stage + 32 * kBlockThreads + threadIdx.x,
                                       out);
    } else {
        group_tail<TM, E, REG>(p, T, e, g, bad);
    }
}

template <int TM>
using StOf = typename std::conditional<TM != TM_GLOBAL, uint16_t, uint32_t>::type;

// Persistent grid: each warp takes tiles of 32 consecutive column groups
// (lane = group).  With TMA the warp's tile of outputs is written to shared
// memory and stored with one tensor-store per tile.
template <int TM, int E, bool TMA, bool REG = false>
__global__ void __launch_bounds__(kBlockThreads, (TM == TM_PAIR || REG) ? 2 : 3)
    merge_kernel(const __grid_constant__ Params p, const __grid_constant__ CUtensorMap out_map) {
    using St = StOf<TM>;
    constexpr int CB = bytes_of(E);
    constexpr uint32_t ROWB = 64 * CB;                        // output bytes of one group
    constexpr uint32_t WPB = kBlockThreads / 32;
    extern __shared__ __align__(16) uint8_t sm[];
    uint8_t *base = sm;
    uint8_t *tiles = nullptr;
    if constexpr (TMA) {                                      // warp tiles, 1024-byte aligned for the swizzle
        const uint32_t a = smem_u32(sm);
        tiles = sm + ((1024 - (a & 1023)) & 1023);
        base = tiles + WPB * 32 * ROWB;
    }
    Tabs T;
    St *stage;
    Enc e;
    merge_setup<TM, E, REG, St>(p.t, p.enc_in_smem, base, T, stage, e);
    pdl_wait();
    const bool ok = *p.status == RE_OK;
    bool bad = false;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *tile = TMA ? tiles + warp * 32 * ROWB : nullptr;
    const uint64_t gw = (uint64_t)blockIdx.x * WPB + warp, nw = (uint64_t)gridDim.x * WPB;
    for (uint64_t gb = gw * 32; gb < p.Gc; gb += nw * 32) {
        const uint64_t g = gb + lane;
        {                                                     // next tile's text and checkpoints into L2
            const uint64_t gn = gb + nw * 32;
            if (gn + lane < p.Gfast) prefetch_l2(p.x + (gn + lane) * 64);
            if (lane < 2 && gn < p.Gc) prefetch_l2((lane ? p.w.BC : p.w.FC) + gn);
        }
        if (TMA && gb != gw * 32) {                           // previous tile read by its store?
            if (lane == 0) bulk_wait_read_all();
            __syncwarp();
        }
        Sink<TMA, CB> out{reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(p.out) + g * ROWB),
                          TMA ? tile + lane * ROWB : nullptr, lane};
        merge_group<TM, E, TMA, REG, St>(p, T, e, stage, g, ok, bad, out);
        if constexpr (TMA) {
            fence_async_smem();
            __syncwarp();
            if (lane == 0 && gb < p.Gfast) {                  // rows past Gfast are clipped by the map
                tma_store_2d(&out_map, smem_u32(tile), 0, (int32_t)gb);
                bulk_commit();
            }
        }
    }
    if (TMA && lane == 0) bulk_wait_all();
    if (bad) atomicExch(p.status, RE_E_INTERNAL);
}

// Batch: warps take 32-group tiles of any text of the group from the work
// list; outputs leave through plain 16-byte stores.
template <int TM, int E>
__global__ void __launch_bounds__(kBlockThreads, 3) merge_batch_kernel(const __grid_constant__ BatchGroup b,
                                                                       uint32_t enc_in_smem) {
    using St = StOf<TM>;
    constexpr uint32_t ROWB = 64 * bytes_of(E);
    extern __shared__ __align__(16) uint8_t sm[];
    Tabs T;
    St *stage;
    Enc e;
    merge_setup<TM, E, false, St>(b.t, enc_in_smem, sm, T, stage, e);
    const uint32_t lane = threadIdx.x & 31;
    for (;;) {
        uint32_t tile = 0;
        if (lane == 0) tile = atomicAdd(b.queue + Q_MERGE, 1u);
        tile = __shfl_sync(0xFFFFFFFFu, tile, 0);
        if (tile >= b.n_merge) break;
        const uint32_t ti = text_of(b.mtile_base, b.nt, tile);
        const Params &p = b.texts[ti];
        const bool ok = *p.status == RE_OK;
        const uint64_t g = (tile - b.mtile_base[ti]) * 32 + lane;
        bool bad = false;
        Sink<false, bytes_of(E)> out{reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(p.out) + g * ROWB), nullptr,
                                     lane};
        merge_group<TM, E, false, false, St>(p, T, e, stage, g, ok, bad, out);
        if (bad) atomicExch(p.status, RE_E_INTERNAL);
    }
}

// ------------------------------------------------------------------ per-position states (mat)
// Fix-up: the positions the reach could not give.  Forward, columns 0 ..
// 64 fv - 1 of chunk i (fv: the first block the reach walked with one run),
// walked from the exact J_i; backward, columns len - 1 .. 64 bv, walked from
// the exact Ĵ_{i+1} (bv: the blocks below it were walked with one run).
// Eq. (builder) from the join's exact boundary states, one thread per chunk
// and direction, with the classic-DFA rows of the one-byte tables.
// One item: chunk i of text p in one direction.
template <int TM>
__device__ void fixup_mat_item(const Params &p, const Tabs &T, uint32_t i, bool fwd) {
    {
        const uint64_t base = (uint64_t)i * p.k;
        const uint32_t len = chunk_len(p, i);
        const uint32_t nfs = p.t.nfd + 1, nbs = p.t.nbd + 1;  // the staged rows
        // states go out 16 at a time (16-byte stores; base is a multiple of 64)
        if (fwd) {
            const uint32_t fv = p.w.fconv[i];
            const uint32_t end = max(1u, min(64u * fv, len));  // columns [0, end)
            uint32_t st = p.w.FJ[i];
            if (st >= nfs) st = 0;                              // never for an accepted text
            uint4 nx = load16(p.x, p.n, base);                  // text bytes 16 at a time, one group ahead
            for (uint32_t g = 0; g < end; g += 16) {
                const uint4 x = nx;
                if (g + 16 < end) nx = load16(p.x, p.n, base + g + 16);
                uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
                for (int u = 0; u < 16; ++u) {                  // column g + u: the state before byte g + u
                    w[u >> 2] |= (st & 0xFFu) << (8 * (u & 3));
                    if (g + u + 1 < end) st = fnext<TM>(T, st, clsof<TM>(T, byte_of(x, u)));
                }
                if (g + 16 <= end) {
                    *reinterpret_cast<uint4 *>(p.w.FS + base + g) = make_uint4(w[0], w[1], w[2], w[3]);
                } else {
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        if (g + u < end) p.w.FS[base + g + u] = (uint8_t)(w[u >> 2] >> (8 * (u & 3)));
                }
            }
            if (i == p.c - 1) p.w.FS[p.n] = (uint8_t)p.w.FJ[p.c];
        } else {
            const uint32_t lo = 64u * p.w.bconv[i];            // columns [lo, len)
            uint32_t st = p.w.BJ[i + 1];                        // column len
            if (st >= nbs) st = 0;
            const uint32_t top = (len + 15) & ~15u;             // 16-column groups, from the top
            uint4 nx = load16(p.x, p.n, base + top - 16);
            for (uint32_t g = top; g > lo; g -= 16) {
                const uint32_t g0 = g - 16;                     // columns g0 .. g0 + 15
                const uint4 x = nx;
                if (g0 > lo) nx = load16(p.x, p.n, base + g0 - 16);
                uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
                for (int u = 15; u >= 0; --u) {                 // column g0 + u: after consuming byte g0 + u
                    if (g0 + u < len) st = bnext<TM>(T, st, clsof<TM>(T, byte_of(x, u)));
                    w[u >> 2] |= (st & 0xFFu) << (8 * (u & 3));
                }
                if (g0 + 16 <= len && g0 >= lo) {
                    *reinterpret_cast<uint4 *>(p.w.BS + base + g0) = make_uint4(w[0], w[1], w[2], w[3]);
                } else {
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        if (g0 + u < len && g0 + u >= lo) p.w.BS[base + g0 + u] = (uint8_t)(w[u >> 2] >> (8 * (u & 3)));
                }
            }
            if (i == p.c - 1) p.w.BS[p.n] = (uint8_t)p.w.BJ[p.c];
        }
    }
}

template <int TM>
__global__ void __launch_bounds__(kFixupThreads) fixup_mat_kernel(const __grid_constant__ Params p) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ int ok;
    Tabs T;
    stage_tables<TM>(dfa_tables(p.t), sm, T);
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) ok = *p.status == RE_OK;
    __syncthreads();
    if (!ok) return;                                            // rejected: build & merge writes zeros
    const uint64_t items = 2 * (uint64_t)p.c;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < items;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const bool fwd = j < p.c;
        fixup_mat_item<TM>(p, T, (uint32_t)(fwd ? j : j - p.c), fwd);
    }
}

// Batch: items are (chunk, direction) over every text of the group.
template <int TM>
__global__ void __launch_bounds__(kFixupThreads) fixup_mat_batch_kernel(const __grid_constant__ BatchGroup b) {
    extern __shared__ __align__(16) uint8_t sm[];
    Tabs T;
    stage_tables<TM>(dfa_tables(b.t), sm, T);
    const uint64_t items = 2 * b.chunks;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < items;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const bool fwd = j < b.chunks;
        const uint64_t f = fwd ? j : j - b.chunks;
        const uint32_t ti = text_of(b.chunk_base, b.nt, f);
        const Params &p = b.texts[ti];
        if (*p.status != RE_OK) continue;                       // rejected: the gather writes zeros
        fixup_mat_item<TM>(p, T, (uint32_t)(f - __ldg(b.chunk_base + ti)), fwd);
    }
}

// Build & merge from the stored states: C_r = B_r ∩ B̂_r (Eq. merger) for
// every column, encoded (DENSE bitset, or DICT index through the pair table
// over classic-DFA state pairs).  A thread takes 16 consecutive columns: two
// 16-byte state loads, 16 encoder lookups in shared memory, one vector store.
// The gather's encoder over classic-DFA state pairs, staged in shared memory
// (the caller synchronises): the DICT pair table, or the states' segment sets.
template <int E>
__device__ Enc stage_gather_enc(const DevTables &t, uint8_t *sm) {
    const uint32_t nfs = t.nfd + 1, nbs = t.nbd + 1;
    Enc e{};
    e.nb = nbs;
    if constexpr (is_dict(E)) {
        const size_t cnt = (size_t)nfs * nbs;
        for (size_t q = threadIdx.x; q < cnt; q += blockDim.x) {
            const uint32_t v = __ldg(t.pt + (q / nbs) * t.nb + q % nbs);
            if (E == ENC_X1) sm[q] = (uint8_t)v;
            else if (E == ENC_X2) reinterpret_cast<uint16_t *>(sm)[q] = (uint16_t)v;
            else reinterpret_cast<uint32_t *>(sm)[q] = v;
        }
        if (E == ENC_X1) e.pt8 = sm;
        else if (E == ENC_X2) e.pt16 = reinterpret_cast<uint16_t *>(sm);
        else e.pt32 = reinterpret_cast<uint32_t *>(sm);
    } else if constexpr (!is_pair(E)) {
        uint64_t *fb = reinterpret_cast<uint64_t *>(sm), *bb = fb + nfs;
        for (uint32_t q = threadIdx.x; q < nfs; q += blockDim.x) fb[q] = __ldg(t.fBits + q);
        for (uint32_t q = threadIdx.x; q < nbs; q += blockDim.x) bb[q] = __ldg(t.bBits + q);
        e.fbits = fb;
        e.bbits = bb;
    }
    return e;
}

// 16 columns from r0 on: their forward states a and backward states b (one
// byte each) -> encoded columns, one 16-byte store per CB.
template <int E>
__device__ __forceinline__ void gather_unit(const Params &p, const Enc &e, uint32_t nfs, uint32_t nbs, bool ok,
                                            bool &bad, uint64_t r0, const uint4 &a, const uint4 &b) {
    constexpr int CB = bytes_of(E);
    const uint32_t fw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
    uint32_t ow[CB * 4];                                        // 16 columns of CB bytes
#pragma unroll
    for (int k = 0; k < CB * 4; ++k) ow[k] = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t f = (fw[k >> 2] >> (8 * (k & 3))) & 0xFFu, g = (bw[k >> 2] >> (8 * (k & 3))) & 0xFFu;
        uint64_t v = 0;
        if (ok) {
            if (f >= nfs || g >= nbs) bad = true;
            else v = enc_col<TM_SMEM, E>(e, f, g, bad);
        }
        if constexpr (CB == 8) {
            ow[2 * k] = (uint32_t)v;
            ow[2 * k + 1] = (uint32_t)(v >> 32);
        } else if constexpr (CB == 4) {
            ow[k] = (uint32_t)v;
        } else {
            constexpr uint32_t m = (1u << (8 * CB)) - 1;
            ow[(k * CB) >> 2] |= ((uint32_t)v & m) << (8 * ((k * CB) & 3));
        }
    }
    uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(p.out) + r0 * CB);
#pragma unroll
    for (int q = 0; q < CB; ++q) __stcs(dst + q, make_uint4(ow[4 * q], ow[4 * q + 1], ow[4 * q + 2], ow[4 * q + 3]));
}

// Column r alone (the tail of a text, fewer than 16 columns).
template <int E>
__device__ __forceinline__ void gather_one_column(const Params &p, const Enc &e, uint32_t nfs, uint32_t nbs, bool ok,
                                                  bool &bad, uint64_t r) {
    uint64_t v = 0;
    if (ok) {
        const uint32_t f = p.w.FS[r], b = p.w.BS[r];
        if (f >= nfs || b >= nbs) bad = true;
        else v = enc_col<TM_SMEM, E>(e, f, b, bad);
    }
    store_col<E>(p.out, r, v);
}

// Build & merge from the stored states: C_r = B_r ∩ B̂_r (Eq. merger) for
// every column, encoded (DENSE bitset, DICT index through the pair table over
// classic-DFA state pairs, or the PAIRS of ids).  A thread takes 16
// consecutive columns: two 16-byte state loads, 16 encoder lookups in shared
// memory, one vector store.
template <int E>
__global__ void __launch_bounds__(kBlockThreads) merge_gather_kernel(const __grid_constant__ Params p) {
    extern __shared__ __align__(16) uint8_t sm[];
    const uint32_t nfs = p.t.nfd + 1, nbs = p.t.nbd + 1;
    const Enc e = stage_gather_enc<E>(p.t, sm);
    __syncthreads();
    pdl_wait();
    const bool ok = *p.status == RE_OK;
    bool bad = false;
    const uint64_t ncol = p.n + 1, full = ncol / 16;
    // two units of 16 columns per thread and step (their four 16-byte loads
    // in flight together), and the next step's four loads issued before this
    // step's lookups; every index static, so the values stay in registers
    const uint64_t pairs = full / 2;
    const uint4 zero = make_uint4(0, 0, 0, 0);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint4 a0 = zero, a1 = zero, b0 = zero, b1 = zero;
    if (ok && u < pairs) {
        a0 = __ldcs(reinterpret_cast<const uint4 *>(p.w.FS + 32 * u));
        a1 = __ldcs(reinterpret_cast<const uint4 *>(p.w.FS + 32 * u + 16));
        b0 = __ldcs(reinterpret_cast<const uint4 *>(p.w.BS + 32 * u));
        b1 = __ldcs(reinterpret_cast<const uint4 *>(p.w.BS + 32 * u + 16));
    }
    for (; u < pairs; u += stride) {
        const uint64_t r0 = 32 * u, rn = r0 + 32 * stride;
        uint4 na0 = zero, na1 = zero, nb0 = zero, nb1 = zero;
        if (ok && u + stride < pairs) {
            na0 = __ldcs(reinterpret_cast<const uint4 *>(p.w.FS + rn));
            na1 = __ldcs(reinterpret_cast<const uint4 *>(p.w.FS + rn + 16));
            nb0 = __ldcs(reinterpret_cast<const uint4 *>(p.w.BS + rn));
            nb1 = __ldcs(reinterpret_cast<const uint4 *>(p.w.BS + rn + 16));
        }
        gather_unit<E>(p, e, nfs, nbs, ok, bad, r0, a0, b0);
        gather_unit<E>(p, e, nfs, nbs, ok, bad, r0 + 16, a1, b1);
        a0 = na0; a1 = na1; b0 = nb0; b1 = nb1;
    }
    if (full & 1) {                                             // an odd last full unit
        const uint64_t r0 = 16 * (full - 1);
        if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
            uint4 a = zero, b = zero;
            if (ok) {
                a = __ldcs(reinterpret_cast<const uint4 *>(p.w.FS + r0));
                b = __ldcs(reinterpret_cast<const uint4 *>(p.w.BS + r0));
            }
            gather_unit<E>(p, e, nfs, nbs, ok, bad, r0, a, b);
        }
    }
    // the last columns (fewer than 16), one at a time
    if (blockIdx.x == 0 && threadIdx.x < ncol - 16 * full) gather_one_column<E>(p, e, nfs, nbs, ok, bad, 16 * full + threadIdx.x);
    if (bad) atomicExch(p.status, RE_E_INTERNAL);
}

// Batch: a warp per merge tile (2048 columns of one text of the group).
template <int E>
__global__ void __launch_bounds__(kBlockThreads) gather_batch_kernel(const __grid_constant__ BatchGroup b) {
    extern __shared__ __align__(16) uint8_t sm[];
    const uint32_t nfs = b.t.nfd + 1, nbs = b.t.nbd + 1;
    const Enc e = stage_gather_enc<E>(b.t, sm);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t tile = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; tile < b.n_merge; tile += warps) {
        const uint32_t ti = text_of(b.mtile_base, b.nt, tile);
        const Params &p = b.texts[ti];
        const bool ok = *p.status == RE_OK;
        bool bad = false;
        const uint64_t c0 = (tile - __ldg(b.mtile_base + ti)) * 2048;
        const uint64_t c1 = min(c0 + 2048, p.n + 1);
        const uint4 zero = make_uint4(0, 0, 0, 0);
        for (uint64_t r0 = c0 + 16 * lane; r0 + 16 <= c1; r0 += 512) {
            uint4 a = zero, bb = zero;
            if (ok) {
                a = __ldcs(reinterpret_cast<const uint4 *>(p.w.FS + r0));
                bb = __ldcs(reinterpret_cast<const uint4 *>(p.w.BS + r0));
            }
            gather_unit<E>(p, e, nfs, nbs, ok, bad, r0, a, bb);
        }
        const uint64_t tail = c0 + ((c1 - c0) & ~(uint64_t)15);   // fewer than 16 columns left
        if (tail + lane < c1) gather_one_column<E>(p, e, nfs, nbs, ok, bad, tail + lane);
        if (bad) atomicExch(p.status, RE_E_INTERNAL);
    }
}

__global__ void empty_text_kernel(const __grid_constant__ Params p) { empty_text(p); }

template <typename K>
int grid_for(K kernel, size_t smem, uint64_t items, int sm_count, uint32_t threads) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    const uint64_t want = (items + threads - 1) / threads;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(per_sm, 1) * sm_count));
}

template <int TM, int E, bool TMA, bool REG>
void merge_launch(const Params &p, const CUtensorMap &map, cudaStream_t s, int sm_count) {
    const size_t smem = merge_smem_bytes(p);
    static uint64_t attr_done = 0;
    allow_smem(merge_kernel<TM, E, TMA, REG>, &attr_done);
    const int blocks = grid_for(merge_kernel<TM, E, TMA, REG>, smem, p.Gc, sm_count, kBlockThreads);
    launch_dependent(merge_kernel<TM, E, TMA, REG>, blocks, kBlockThreads, smem, s, p, map);
}

template <int TM, int E, bool TMA>
void merge_one(const Params &p, const CUtensorMap &map, cudaStream_t s, int sm_count) {
    if constexpr (TM == TM_SMEM) {
        if (p.merge_reg) { merge_launch<TM, E, TMA, true>(p, map, s, sm_count); return; }
    }
    merge_launch<TM, E, TMA, false>(p, map, s, sm_count);
}

template <int TM, int E>
void merge_tma(const Params &p, const CUtensorMap &map, cudaStream_t s, int sm_count) {
    constexpr int CB = bytes_of(E);
    if constexpr (CB <= 2) {
        if (p.out_tma) { merge_one<TM, E, true>(p, map, s, sm_count); return; }
    }
    merge_one<TM, E, false>(p, map, s, sm_count);
}

template <int TM>
void merge_enc(const Params &p, const CUtensorMap &map, cudaStream_t s, int sm_count) {
    if (p.kind == RE_SLPF_PAIRS) {
        if (p.col_bytes == 4) merge_tma<TM, ENC_P4>(p, map, s, sm_count);
        else merge_tma<TM, ENC_P8>(p, map, s, sm_count);
    } else if (p.kind == RE_SLPF_DICT) {
        if (p.col_bytes == 1) merge_tma<TM, ENC_X1>(p, map, s, sm_count);
        else if (p.col_bytes == 2) merge_tma<TM, ENC_X2>(p, map, s, sm_count);
        else merge_tma<TM, ENC_X4>(p, map, s, sm_count);
    } else {
        switch (p.col_bytes) {
            case 1: merge_tma<TM, ENC_D1>(p, map, s, sm_count); break;
            case 2: merge_tma<TM, ENC_D2>(p, map, s, sm_count); break;
            case 4: merge_tma<TM, ENC_D4>(p, map, s, sm_count); break;
            default: merge_tma<TM, ENC_D8>(p, map, s, sm_count); break;
        }
    }
}

template <int TM, int E>
void merge_batch_one(const BatchGroup &b, const Params &like, cudaStream_t s, int sm_count) {
    Params q = like;
    q.out_tma = 0;
    const size_t smem = tables_smem_bytes(b.t, TM) + merge_extra_smem(q);
    static uint64_t attr_done = 0;
    allow_smem(merge_batch_kernel<TM, E>, &attr_done);
    const int blocks = grid_for(merge_batch_kernel<TM, E>, smem, (uint64_t)b.n_merge * 32, sm_count, kBlockThreads);
    merge_batch_kernel<TM, E><<<blocks, kBlockThreads, smem, s>>>(b, q.enc_in_smem);
}

template <int TM>
void merge_batch_enc(const BatchGroup &b, const Params &like, cudaStream_t s, int sm_count) {
    if (like.kind == RE_SLPF_PAIRS) {
        if (like.col_bytes == 4) merge_batch_one<TM, ENC_P4>(b, like, s, sm_count);
        else merge_batch_one<TM, ENC_P8>(b, like, s, sm_count);
    } else if (like.kind == RE_SLPF_DICT) {
        if (like.col_bytes == 1) merge_batch_one<TM, ENC_X1>(b, like, s, sm_count);
        else if (like.col_bytes == 2) merge_batch_one<TM, ENC_X2>(b, like, s, sm_count);
        else merge_batch_one<TM, ENC_X4>(b, like, s, sm_count);
    } else {
        switch (like.col_bytes) {
            case 1: merge_batch_one<TM, ENC_D1>(b, like, s, sm_count); break;
            case 2: merge_batch_one<TM, ENC_D2>(b, like, s, sm_count); break;
            case 4: merge_batch_one<TM, ENC_D4>(b, like, s, sm_count); break;
            default: merge_batch_one<TM, ENC_D8>(b, like, s, sm_count); break;
        }
    }
}

template <int TM>
void fixup_batch_one(const BatchGroup &b, cudaStream_t s, int sm_count) {
    const size_t smem = tables_smem_bytes(b.t, TM);
    static uint64_t attr_done = 0;
    allow_smem(fixup_batch_kernel<TM>, &attr_done);
    fixup_batch_kernel<TM><<<grid_for(fixup_batch_kernel<TM>, smem, b.chunks * 2 * (kFixupThreads / kFixItems), sm_count,
                                      kFixupThreads),
                             kFixupThreads, smem, s>>>(b);
}

template <int TM>
void fixup_one(const Params &p, cudaStream_t s, int sm_count) {
    const size_t smem = tables_smem_bytes(p.t, TM);
    static uint64_t attr_done = 0;
    allow_smem(fixup_kernel<TM>, &attr_done);
    // a block per kFixItems items, at most one wave of resident blocks (they loop over the rest)
    const int blocks = grid_for(fixup_kernel<TM>, smem, (uint64_t)p.c * 2 * (kFixupThreads / kFixItems), sm_count,
                                kFixupThreads);
    launch_dependent(fixup_kernel<TM>, blocks, kFixupThreads, smem, s, p);
}

// Shared memory of the gather's encoder (pair table or bitsets over the
// classic-DFA states).
size_t gather_smem(const Params &p) {
    const size_t nfs = p.t.nfd + 1, nbs = p.t.nbd + 1;
    if (p.kind == RE_SLPF_PAIRS) return 0;
    return p.kind == RE_SLPF_DICT ? nfs * nbs * p.col_bytes : (nfs + nbs) * 8;
}

template <int TM>
void fixup_mat_one(const Params &p, cudaStream_t s, int sm_count) {
    const size_t smem = tables_smem_bytes(dfa_tables(p.t), TM);
    static uint64_t attr_done = 0;
    allow_smem(fixup_mat_kernel<TM>, &attr_done);
    const int blocks = grid_for(fixup_mat_kernel<TM>, smem, 2 * (uint64_t)p.c, sm_count, kFixupThreads);
    launch_dependent(fixup_mat_kernel<TM>, blocks, kFixupThreads, smem, s, p);
}

template <int E>
void gather_one(const Params &p, cudaStream_t s, int sm_count) {
    const size_t smem = gather_smem(p);
    static uint64_t attr_done = 0;
    allow_smem(merge_gather_kernel<E>, &attr_done);
    const int blocks = grid_for(merge_gather_kernel<E>, smem, (p.n + 16) / 16, sm_count, kBlockThreads);
    launch_dependent(merge_gather_kernel<E>, blocks, kBlockThreads, smem, s, p);
}

void launch_gather(const Params &p, cudaStream_t s, int sm_count) {
    if (p.kind == RE_SLPF_PAIRS) {
        if (p.col_bytes == 4) gather_one<ENC_P4>(p, s, sm_count);
        else gather_one<ENC_P8>(p, s, sm_count);
    } else if (p.kind == RE_SLPF_DICT) {
        if (p.col_bytes == 1) gather_one<ENC_X1>(p, s, sm_count);
        else if (p.col_bytes == 2) gather_one<ENC_X2>(p, s, sm_count);
        else gather_one<ENC_X4>(p, s, sm_count);
    } else {
        switch (p.col_bytes) {
            case 1: gather_one<ENC_D1>(p, s, sm_count); break;
            case 2: gather_one<ENC_D2>(p, s, sm_count); break;
            case 4: gather_one<ENC_D4>(p, s, sm_count); break;
            default: gather_one<ENC_D8>(p, s, sm_count); break;
        }
    }
}

}  // namespace

size_t mat_gather_smem(const Params &p) { return gather_smem(p); }

size_t merge_extra_smem(const Params &p) {
    const DevTables t = p.merge_reg ? dfa_tables(p.t) : p.t;
    size_t a = 0;
    if (p.out_tma) a += 1024 + (size_t)(kBlockThreads / 32) * 32 * 64 * p.col_bytes;   // warp tiles + alignment
    if (p.tmode != TM_PAIR && !p.merge_reg)
        a += (2 * 32 * kBlockThreads * (p.tmode == TM_GLOBAL ? 4 : 2) + 15) & ~(size_t)15;
    if (!p.enc_in_smem || p.kind == RE_SLPF_PAIRS) return a;
    if (p.kind == RE_SLPF_DICT) return a + (size_t)t.nf * t.nb * p.col_bytes;
    return a + (size_t)(t.nf + t.nb) * 8;
}

// Dynamic shared memory of one build & merge block: staged tables, then the
// areas of merge_extra_smem.
size_t merge_smem_bytes(const Params &p) {
    return tables_smem_bytes(p.merge_reg ? dfa_tables(p.t) : p.t, p.tmode) + merge_extra_smem(p);
}

// The fix-up walks with the parse's staged tables: its duration is that of
// the longest walk past a chunk's record (a run that stays apart for more
// boundaries than the record holds), a serial chain of dependent lookups.
void launch_fixup(const Params &p, cudaStream_t s, int sm_count) {
    if (p.mat) { fixup_mat_one<TM_SMEM8>(p, s, sm_count); return; }
    if (p.tmode == TM_PAIR) fixup_one<TM_PAIR>(p, s, sm_count);
    else if (p.tmode == TM_SMEM) fixup_one<TM_SMEM>(p, s, sm_count);
    else fixup_one<TM_GLOBAL>(p, s, sm_count);
}

void launch_merge(const Params &p, const CUtensorMap &map, cudaStream_t s, int sm_count) {
    if (p.mat) { launch_gather(p, s, sm_count); return; }
    if (p.tmode == TM_PAIR) merge_enc<TM_PAIR>(p, map, s, sm_count);
    else if (p.tmode == TM_SMEM) merge_enc<TM_SMEM>(p, map, s, sm_count);
    else merge_enc<TM_GLOBAL>(p, map, s, sm_count);
}

void launch_empty(const Params &p, cudaStream_t s) { empty_text_kernel<<<1, 1, 0, s>>>(p); }

void launch_fixup_mat_batch(const BatchGroup &b, cudaStream_t s, int sm_count) {
    if (b.recognize || !b.chunks) return;
    const size_t smem = tables_smem_bytes(dfa_tables(b.t), TM_SMEM8);
    static uint64_t attr_done = 0;
    allow_smem(fixup_mat_batch_kernel<TM_SMEM8>, &attr_done);
    const int blocks = grid_for(fixup_mat_batch_kernel<TM_SMEM8>, smem, 2 * b.chunks, sm_count, kFixupThreads);
    fixup_mat_batch_kernel<TM_SMEM8><<<blocks, kFixupThreads, smem, s>>>(b);
}

template <int E>
void gather_batch_one(const BatchGroup &b, const Params &like, cudaStream_t s, int sm_count) {
    const size_t smem = gather_smem(like);
    static uint64_t attr_done = 0;
    allow_smem(gather_batch_kernel<E>, &attr_done);
    const int blocks = grid_for(gather_batch_kernel<E>, smem, b.n_merge * 32, sm_count, kBlockThreads);
    gather_batch_kernel<E><<<blocks, kBlockThreads, smem, s>>>(b);
}

void launch_gather_batch(const BatchGroup &b, const Params &like, cudaStream_t s, int sm_count) {
    if (b.recognize || !b.n_merge) return;
    if (like.kind == RE_SLPF_PAIRS) {
        if (like.col_bytes == 4) gather_batch_one<ENC_P4>(b, like, s, sm_count);
        else gather_batch_one<ENC_P8>(b, like, s, sm_count);
    } else if (like.kind == RE_SLPF_DICT) {
        if (like.col_bytes == 1) gather_batch_one<ENC_X1>(b, like, s, sm_count);
        else if (like.col_bytes == 2) gather_batch_one<ENC_X2>(b, like, s, sm_count);
        else gather_batch_one<ENC_X4>(b, like, s, sm_count);
    } else {
        switch (like.col_bytes) {
            case 1: gather_batch_one<ENC_D1>(b, like, s, sm_count); break;
            case 2: gather_batch_one<ENC_D2>(b, like, s, sm_count); break;
            case 4: gather_batch_one<ENC_D4>(b, like, s, sm_count); break;
            default: gather_batch_one<ENC_D8>(b, like, s, sm_count); break;
        }
    }
}

void launch_fixup_batch(const BatchGroup &b, uint32_t tmode, cudaStream_t s, int sm_count) {
    if (b.recognize || !b.chunks) return;
    if (tmode == TM_PAIR) fixup_batch_one<TM_PAIR>(b, s, sm_count);
    else if (tmode == TM_SMEM) fixup_batch_one<TM_SMEM>(b, s, sm_count);
    else fixup_batch_one<TM_GLOBAL>(b, s, sm_count);
}

void launch_merge_batch(const BatchGroup &b, const Params &like, cudaStream_t s, int sm_count) {
    if (b.recognize || !b.n_merge) return;
    if (like.tmode == TM_PAIR) merge_batch_enc<TM_PAIR>(b, like, s, sm_count);
    else if (like.tmode == TM_SMEM) merge_batch_enc<TM_SMEM>(b, like, s, sm_count);
    else merge_batch_enc<TM_GLOBAL>(b, like, s, sm_count);
}

}  // namespace slpf
