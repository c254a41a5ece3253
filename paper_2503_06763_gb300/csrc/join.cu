// Join phase (arXiv 2503.06763, Eq. joiner): FJ[i] = J_i, the forward state at
// the boundary before chunk i (J_0 = I), and BJ[i] = Ĵ at that boundary
// (BJ[c] = F).
//
// Every chunk maps an input state S to the union, over its slots whose keys
// S contains, of the slot's end state.  When all live slots of a chunk end in
// one state (the common case: speculative runs meet within a few hundred
// bytes, Sect. 4.3) the chunk's output is that state for every input that
// enters a live slot, so it is known without its neighbour.  The remaining
// chunks form chains that are evaluated in order from the nearest known
// neighbour.  A verify pass checks each guessed output against its actual
// input; the first chunk where the text cannot continue makes the whole text
// rejected (no accepting run: every clean column is empty).
#include <algorithm>

#include "kernels.cuh"

namespace slpf {
namespace {

__device__ uint32_t probe(const uint32_t *hash, uint32_t mask, const uint64_t *bits, uint32_t W,
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

__device__ __forceinline__ uint32_t pair_fwd(const Params &p, uint32_t i) {
    const uint64_t base = (uint64_t)i * p.k;
    return __ldg(p.t.cls + __ldg(p.x + base - 1)) * p.t.ncls + __ldg(p.t.cls + __ldg(p.x + base));
}
__device__ __forceinline__ uint32_t pair_bwd(const Params &p, uint32_t i) {
    const uint64_t end = (uint64_t)i * p.k + chunk_len(p, i);
    return __ldg(p.t.cls + __ldg(p.x + end - 1)) * p.t.ncls + __ldg(p.t.cls + __ldg(p.x + end));
}

// State after chunk i for input state S: union over the slots S enters.
__device__ uint32_t eval_chunk(const Params &p, bool fwd, uint32_t i, uint32_t S, bool &bad) {
    const DevTables &t = p.t;
    if (S == 0) return 0;
    const uint32_t W = t.W;
    uint32_t pr, m, ms;
    const uint32_t *R;
    const uint64_t *mask, *bits;
    if (fwd) {
        pr = pair_fwd(p, i); m = __ldg(t.fSlotCount + pr); ms = t.msf; R = p.w.Rf + (size_t)i * ms;
        mask = t.fSlotMask + (size_t)pr * ms * W; bits = t.fBits;
    } else {
        pr = pair_bwd(p, i); m = __ldg(t.bSlotCount + pr); ms = t.msb; R = p.w.Rb + (size_t)i * ms;
        mask = t.bSlotMask + (size_t)pr * ms * W; bits = t.bBits;
    }
    const uint8_t *of = fwd ? t.fSlotOf : t.bSlotOf;
    if (of) {                                    // starts from every DFA state: exact lookup
        const uint32_t n = fwd ? t.nf : t.nb;
        const uint32_t j = S < n ? __ldg(of + (size_t)pr * n + S) : 0xFFu;
        return j == 0xFFu ? 0u : R[j];
    }
    const uint64_t *sb = bits + (size_t)S * W;
    uint32_t single = 0;
    bool multi = false;
    uint64_t acc[kMaxW];
    for (uint32_t w = 0; w < W; ++w) acc[w] = 0;
    for (uint32_t s = 0; s < m; ++s) {
        const uint32_t e = R[s];
        if (!e || !any_and(sb, mask + (size_t)s * W, W)) continue;
        if (!single) single = e;
        else if (e != single) multi = true;
        for (uint32_t w = 0; w < W; ++w) acc[w] |= __ldg(bits + (size_t)e * W + w);
    }
    if (!multi) return single;
    const uint32_t id = fwd ? probe(t.fHash, t.fHashMask, t.fBits, W, acc)
                            : probe(t.bHash, t.bHashMask, t.bBits, W, acc);
    if (!id) bad = true;
    return id;
}

// One live end state (or none) for every chunk?  Record it as the guess.
__device__ void classify(const Params &p, bool fwd, uint32_t i) {
    const DevTables &t = p.t;
    const uint32_t pr = fwd ? pair_fwd(p, i) : pair_bwd(p, i);
    const uint32_t m = __ldg((fwd ? t.fSlotCount : t.bSlotCount) + pr);
    const uint32_t ms = fwd ? t.msf : t.msb;
    const uint32_t *R = (fwd ? p.w.Rf : p.w.Rb) + (size_t)i * ms;
    uint32_t rep = 0;
    bool gen = false;
    for (uint32_t s = 0; s < m; ++s) {
        const uint32_t e = R[s];
        if (e) { if (!rep) rep = e; else if (e != rep) gen = true; }
    }
    if (fwd) {
        p.w.fkind[i] = gen ? 1u : 0u;
        if (!gen) p.w.FJ[i + 1] = rep;
    } else {
        p.w.bkind[i] = gen ? 1u : 0u;
        if (!gen) p.w.BJ[i] = rep;
    }
    if (gen && p.scan) atomicAdd(p.w.scan + kScanGeneral, 1u);   // the scan has work
}

__device__ void classify_at(const Params &p, uint32_t i) {
    if (i == 0 && !(p.shard & SHARD_PREV)) {
        p.w.FJ[0] = p.t.fI;
        p.w.FJ[1] = p.w.Rf[0];
        p.w.fkind[0] = 0;
    } else {
        classify(p, true, i);
    }
    if (p.recognize) return;
    if (i == p.c - 1 && !(p.shard & SHARD_NEXT)) {
        p.w.BJ[p.c] = p.t.bF;
        p.w.BJ[i] = p.w.Rb[(size_t)i * p.t.msb];
        p.w.bkind[i] = 0;
    } else {
        classify(p, false, i);
    }
}

// Chains of general chunks, evaluated in order from their known neighbour
// (started by the chunk just after / before the neighbour).
__device__ void chain_at(const Params &p, uint32_t i) {
    bool bad = false;
    if (p.w.fkind[i] == 1 && p.w.fkind[i - 1] == 0) {     // i >= 1: fkind[0] == 0
        uint32_t cur = p.w.FJ[i];
        for (uint32_t j = i; j < p.c && p.w.fkind[j] == 1; ++j) {
            cur = eval_chunk(p, true, j, cur, bad);
            p.w.FJ[j + 1] = cur;
        }
    }
    if (!p.recognize && p.w.bkind[i] == 1 && p.w.bkind[i + 1] == 0) {   // i <= c-2: bkind[c-1] == 0
        uint32_t cur = p.w.BJ[i + 1];
        for (int64_t j = i; j >= 0 && p.w.bkind[j] == 1; --j) {
            cur = eval_chunk(p, false, (uint32_t)j, cur, bad);
            p.w.BJ[j] = cur;
        }
    }
    if (bad) atomicExch(&p.w.flags[FLAG_INTERNAL], 1);
}

__global__ void join_classify_kernel(const __grid_constant__ Params p) {
    pdl_wait();
    pdl_trigger();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p.c) classify_at(p, i);
}

__global__ void join_chain_kernel(const __grid_constant__ Params p) {
    pdl_wait();
    pdl_trigger();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p.c) chain_at(p, i);
}

__device__ bool grid_barrier(uint32_t *w);

// ------------------------------------------------------------------ slice maps
// A slice of a longer text (sharded parse): its forward map sends the
// forward state S at the slice's start to the state at its end, the
// composition of its chunk maps (Eq. joiner) in order; its backward map sends
// the backward state at the slice's end to the state at its start.  Every
// chunk's map over the classic-DFA states is a byte table (eval_chunk; the
// first chunk of the text's first slice starts from I, so its map is
// constant, and the last chunk of the last slice from F), and the tables are
// composed by a tree reduction: in round r, the table of chunk i (i a
// multiple of 2^{r+1}) absorbs that of chunk i + 2^r.  Cooperative launch,
// the rounds separated by the bounded grid barrier.
template <uint32_t LANES>
__device__ void shard_map(const Params &p, uint8_t *maps) {
    const uint32_t lane = LANES == 1 ? 0u : (threadIdx.x & 31), upb = blockDim.x / LANES;
    const uint64_t gw = (uint64_t)blockIdx.x * upb + threadIdx.x / LANES, nw = (uint64_t)gridDim.x * upb;
    const uint32_t nsf = p.t.nfd + 1, nsb = p.t.nbd + 1, c = p.c;
    bool bad = false;
    for (uint64_t i = gw; i < c; i += nw) {
        uint8_t *T = p.w.fTab + i * nsf;
        const bool first = i == 0 && !(p.shard & SHARD_PREV);           // runs from I: one output
        for (uint32_t S = lane; S < nsf; S += LANES)
            T[S] = (uint8_t)(first ? (S ? p.w.Rf[0] : 0u) : eval_chunk(p, true, (uint32_t)i, S, bad));
        uint8_t *B = p.w.bTab + i * nsb;
        const bool last = i == c - 1 && !(p.shard & SHARD_NEXT);         // runs from F: one output
        for (uint32_t S = lane; S < nsb; S += LANES)
            B[S] = (uint8_t)(last ? (S ? p.w.Rb[(size_t)i * p.t.msb] : 0u) : eval_chunk(p, false, (uint32_t)i, S, bad));
    }
    if (bad) atomicExch(&p.w.flags[FLAG_INTERNAL], 1);
    for (uint32_t r = 0; (1ull << r) < c; ++r) {
        if (!grid_barrier(p.w.scan)) { atomicExch(&p.w.flags[FLAG_TIMEOUT], 1); return; }
        const uint64_t step = 1ull << r, pairs = (c + 2 * step - 1) / (2 * step);
        for (uint64_t q = gw; q < pairs; q += nw) {
            const uint64_t i = q * 2 * step, j = i + step;
            if (j >= c) continue;
            uint8_t *Ti = p.w.fTab + i * nsf;                          // [i, j) then [j, j + step)
            const uint8_t *Tj = p.w.fTab + j * nsf;
            for (uint32_t S = lane; S < nsf; S += LANES) Ti[S] = __ldcg(Tj + __ldcg(Ti + S));
            uint8_t *Bi = p.w.bTab + i * nsb;                          // the later range first
            const uint8_t *Bj = p.w.bTab + j * nsb;
            uint8_t v[kScanStates / (LANES == 1 ? 1 : 32)];
            uint32_t nv = 0;
            for (uint32_t S = lane; S < nsb; S += LANES) v[nv++] = __ldcg(Bi + __ldcg(Bj + S));
            if (LANES == 32) __syncwarp();
            nv = 0;
            for (uint32_t S = lane; S < nsb; S += LANES) Bi[S] = v[nv++];
        }
    }
    if (!grid_barrier(p.w.scan)) { atomicExch(&p.w.flags[FLAG_TIMEOUT], 1); return; }
    if (blockIdx.x == 0) {                                            // the slice's maps
        for (uint32_t S = threadIdx.x; S < nsf; S += blockDim.x) maps[S] = __ldcg(p.w.fTab + S);
        for (uint32_t S = threadIdx.x; S < nsb; S += blockDim.x) maps[nsf + S] = __ldcg(p.w.bTab + S);
        if (threadIdx.x == 0) {
            const int32_t fl = __ldcg(&p.w.flags[FLAG_INTERNAL]), to = __ldcg(&p.w.flags[FLAG_TIMEOUT]);
            *p.status = to ? RE_E_TIMEOUT : fl ? RE_E_INTERNAL : RE_OK;
        }
    }
}

__global__ void __launch_bounds__(kBlockThreads) join_map_kernel(const __grid_constant__ Params p, uint8_t *maps) {
    if (p.t.nfd < 16 && p.t.nbd < 16) shard_map<1>(p, maps);
    else shard_map<32>(p, maps);
}

// Live slots of chunk i (their end state is not the empty set).
__device__ uint32_t live_slots(const Params &p, bool fwd, uint32_t i, uint32_t pr) {
    const DevTables &t = p.t;
    const uint32_t m = __ldg((fwd ? t.fSlotCount : t.bSlotCount) + pr);
    const uint32_t ms = fwd ? t.msf : t.msb;
    const uint32_t *R = (fwd ? p.w.Rf : p.w.Rb) + (size_t)i * ms;
    uint32_t L = 0;
    for (uint32_t s = 0; s < m; ++s)
        if (R[s]) L |= 1u << s;
    return L;
}

// Check each chunk's guessed output against its (now known) input and keep
// the slots that input enters for the fix-up.
__device__ void verify_at(const Params &p, uint32_t i) {
    {   // forward: input FJ[i] -> output FJ[i+1]
        const uint32_t in = p.w.FJ[i], out = p.w.FJ[i + 1];
        bool fail = in == 0 || out == 0;
        uint32_t H = 0;
        if (i > 0 && in != 0) {
            const uint32_t pr = pair_fwd(p, i);
            H = slot_hits(p.t, true, pr, in);
            if (!fail && p.w.fkind[i] == 0) fail = (H & live_slots(p, true, i, pr)) == 0;
        }
        p.w.fhit[i] = H;
        if (fail) atomicMin(&p.w.flags[FLAG_FFAIL], (int32_t)i);
        p.w.FC[(uint64_t)i * p.S] = in;                              // position i*k
        if (i == p.c - 1 && (p.n & 63) == 0) p.w.FC[p.n >> 6] = p.w.FJ[p.c];   // position n
    }
    if (p.recognize) return;
    {   // backward: input BJ[i+1] -> output BJ[i]
        const uint32_t in = p.w.BJ[i + 1], out = p.w.BJ[i];
        bool fail = in == 0 || out == 0;
        uint32_t H = 0;
        if (i < p.c - 1 && in != 0) {
            const uint32_t pr = pair_bwd(p, i);
            H = slot_hits(p.t, false, pr, in);
            if (!fail && p.w.bkind[i] == 0) fail = (H & live_slots(p, false, i, pr)) == 0;
        }
        p.w.bhit[i] = H;
        if (fail) atomicMin(&p.w.flags[FLAG_BFAIL], (int32_t)i);
        if (i + 1 < p.c) {
            p.w.BC[(uint64_t)(i + 1) * p.S - 1] = in;                // position (i+1)*k
        } else {                                                     // groups whose end is clipped to n
            for (uint64_t g = (p.n + 63) / 64 - 1; g < p.Gc; ++g) p.w.BC[g] = in;
        }
    }
}

// verify_at with a warp per chunk: lane j tests slot j (whether the input
// enters it, whether its run is live) and a ballot gathers the masks; lane 0
// does the rest.  Slot counts are at most 32.
__device__ __forceinline__ uint32_t hits_warp(const Params &p, bool fwd, uint32_t i, uint32_t pr, uint32_t S,
                                              uint32_t &live) {
    const DevTables &t = p.t;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t m = __ldg((fwd ? t.fSlotCount : t.bSlotCount) + pr);
    const uint32_t ms = fwd ? t.msf : t.msb;
    const uint32_t *R = (fwd ? p.w.Rf : p.w.Rb) + (size_t)i * ms;
    live = __ballot_sync(0xFFFFFFFFu, lane < m && R[lane] != 0);
    const uint8_t *of = fwd ? t.fSlotOf : t.bSlotOf;
    if (of) {                                    // starts from every DFA state: S enters its own slot only
        const uint32_t n = fwd ? t.nf : t.nb;
        const uint32_t j = S < n ? __ldg(of + (size_t)pr * n + S) : 0xFFu;
        return j == 0xFFu ? 0u : 1u << j;
    }
    const uint32_t W = t.W;
    const uint64_t *mask = (fwd ? t.fSlotMask : t.bSlotMask) + (size_t)pr * ms * W;
    const uint64_t *sb = (fwd ? t.fBits : t.bBits) + (size_t)S * W;
    return __ballot_sync(0xFFFFFFFFu, lane < m && any_and(sb, mask + (size_t)lane * W, W));
}

// Both directions' loads come before any store (a store could alias a later
// load, so the compiler would keep them in order), so the two dependent load
// chains of a chunk overlap.
__device__ void verify_warp(const Params &p, uint32_t i) {
    const uint32_t lane = threadIdx.x & 31;
    const bool both = !p.recognize;
    // forward: input FJ[i] -> output FJ[i+1]; backward: input BJ[i+1] -> output BJ[i]
    const uint32_t fin = p.w.FJ[i], fout = p.w.FJ[i + 1];
    const uint32_t bin = both ? p.w.BJ[i + 1] : 0u, bout = both ? p.w.BJ[i] : 0u;
    const uint32_t fkind = p.w.fkind[i], bkind = both ? p.w.bkind[i] : 1u;
    const uint32_t fend = (i == p.c - 1 && (p.n & 63) == 0) ? p.w.FJ[p.c] : 0u;
    bool ffail = fin == 0 || fout == 0, bfail = both && (bin == 0 || bout == 0);
    uint32_t fH = 0, bH = 0;
    if (i > 0 && fin != 0) {
        uint32_t L;
        fH = hits_warp(p, true, i, pair_fwd(p, i), fin, L);
        if (!ffail && fkind == 0) ffail = (fH & L) == 0;
    }
    if (both && i < p.c - 1 && bin != 0) {
        uint32_t L;
        bH = hits_warp(p, false, i, pair_bwd(p, i), bin, L);
        if (!bfail && bkind == 0) bfail = (bH & L) == 0;
    }
    if (lane != 0) return;
    p.w.fhit[i] = fH;
    if (ffail) atomicMin(&p.w.flags[FLAG_FFAIL], (int32_t)i);
    p.w.FC[(uint64_t)i * p.S] = fin;                                     // position i*k
    if (i == p.c - 1 && (p.n & 63) == 0) p.w.FC[p.n >> 6] = fend;       // position n
    if (!both) return;
    p.w.bhit[i] = bH;
    if (bfail) atomicMin(&p.w.flags[FLAG_BFAIL], (int32_t)i);
    if (i + 1 < p.c) {
        p.w.BC[(uint64_t)(i + 1) * p.S - 1] = bin;                       // position (i+1)*k
    } else {                                                             // groups whose end is clipped to n
        for (uint64_t g = (p.n + 63) / 64 - 1; g < p.Gc; ++g) p.w.BC[g] = bin;
    }
}

// Accept iff both joins ran through and C_0 = I ∩ Ĵ_1 is not empty
// (recognizer: iff the forward join ran through and J_c ∩ F is not empty).
__device__ void status_of(const Params &p) {
    const DevTables &t = p.t;
    int32_t st = RE_OK;
    // flags are updated by atomics of the verify blocks: read them from L2
    const int32_t ffail = __ldcg(&p.w.flags[FLAG_FFAIL]), bfail = __ldcg(&p.w.flags[FLAG_BFAIL]);
    if (ffail < (int32_t)p.c || (!p.recognize && bfail < (int32_t)p.c)) {
        st = RE_REJECTED;
    } else if (p.recognize) {
        const uint32_t jc = p.w.FJ[p.c];
        if (!any_and(t.fBits + (size_t)jc * t.W, t.bBits + (size_t)t.bF * t.W, t.W)) st = RE_REJECTED;
    } else {
        const uint32_t b0 = p.w.BJ[0];
        if (!(b0 && any_and(t.fBits + (size_t)t.fI * t.W, t.bBits + (size_t)b0 * t.W, t.W))) st = RE_REJECTED;
    }
    if (__ldcg(&p.w.flags[FLAG_INTERNAL])) st = RE_E_INTERNAL;
    if (__ldcg(&p.w.flags[FLAG_TIMEOUT])) st = RE_E_TIMEOUT;
    *p.status = st;
}

// Verify every chunk; the last block to finish then sets the status word,
// once every block's writes are visible (each block fences its writes before
// it takes a ticket; the last ticket holder fences again before reading).
__global__ void join_verify_kernel(const __grid_constant__ Params p) {
    pdl_wait();
    pdl_trigger();
    const uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // a warp per chunk
    if (i < p.c) verify_warp(p, (uint32_t)i);
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&p.w.flags[FLAG_DONE], 1) == (int32_t)gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        status_of(p);
    }
}

__global__ void flags_init_kernel(const __grid_constant__ Params p) {
    if (threadIdx.x < FLAG_COUNT) p.w.flags[threadIdx.x] = threadIdx.x < 2 ? (int32_t)p.c : 0;
    if (p.scan)
        for (uint32_t q = threadIdx.x; q < kScanWords; q += blockDim.x) p.w.scan[q] = 0;
}

// ------------------------------------------------------------------ scan join
// Eq. (joiner) as a scan.  Chunk i maps its input state J_i to J_{i+1}; a
// chunk whose live slots all end in one state maps every input that can
// continue to that state (classify resolves it at once).  Every other chunk
// gets its map over the classic-DFA states (a byte table; the union of the
// slot end states the input enters, as eval_chunk computes it), and the
// chunks are resolved by pointer jumping: chunk i holds the map of the
// chunk range (l_i, i] and the link l_i; in each round, if chunk l_i is
// resolved, J_{i+1} = map(J_{l_i + 1}), else the range doubles: map becomes
// map_i o map_{l_i} and l_i becomes l_{l_i}.  A chain of L chunks resolves in
// ceil(log2 L) + 1 rounds instead of L dependent steps.  Backward (Ĵ) the same
// with the chunks taken right to left.  The rounds are separated by a grid
// barrier of this cooperative launch; each barrier wait is bounded, and a
// wait that runs out sets the status RE_E_TIMEOUT.
constexpr uint32_t kResolved = 0xFFFFFFFFu;
static_assert(kScanGeneral < kScanWords, "scan words");

// All blocks of the grid meet here; false when this block's wait ran out.
__device__ bool grid_barrier(uint32_t *w) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile uint32_t *gen = w + 1;
        const uint32_t g = *gen;
        __threadfence();
        if (atomicAdd(w, 1u) == gridDim.x - 1) {
            w[0] = 0;                                   // every other block waits on gen: reset first
            __threadfence();
            atomicAdd(w + 1, 1u);
        } else {
            uint32_t it = 0;
            while (*gen == g)
                if (++it > kWaitLimit) { ok = 0; break; }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// One direction of one chunk in a round.  LANES = 32: a warp, whose lanes
// share the table work; LANES = 1: one thread (small automata, where the
// latency of the link reads, not the table, sets the time of a round).
template <bool FWD, uint32_t LANES>
__device__ uint32_t scan_step(const Params &p, uint32_t i, uint32_t cur) {
    const uint32_t lane = LANES == 1 ? 0u : (threadIdx.x & 31), c = p.c, ns = (FWD ? p.t.nfd : p.t.nbd) + 1;
    uint32_t *link = FWD ? p.w.fLink : p.w.bLink;
    uint8_t *tab = FWD ? p.w.fTab : p.w.bTab;
    uint32_t *J = FWD ? p.w.FJ : p.w.BJ;
    const uint32_t nxt = cur ^ 1u;
    const uint32_t l = __ldcg(link + (size_t)cur * c + i);
    if (l == kResolved) {
        if (lane == 0) link[(size_t)nxt * c + i] = kResolved;
        return 0;
    }
    const uint8_t *Ti = tab + ((size_t)cur * c + i) * ns;
    const uint32_t ll = __ldcg(link + (size_t)cur * c + l);
    if (ll == kResolved) {                             // the range's input is known
        if (lane == 0) {
            const uint32_t v = __ldcg(J + (FWD ? l + 1 : l));   // output of chunk l
            J[FWD ? i + 1 : i] = v < ns ? (uint32_t)__ldcg(Ti + v) : 0u;   // v >= ns: no DFA state, rejected
            link[(size_t)nxt * c + i] = kResolved;
        }
        return 0;
    }
    const uint8_t *Tl = tab + ((size_t)cur * c + l) * ns;
    uint8_t *Tn = tab + ((size_t)nxt * c + i) * ns;
    for (uint32_t S = lane; S < ns; S += LANES) Tn[S] = __ldcg(Ti + __ldcg(Tl + S));
    if (lane == 0) link[(size_t)nxt * c + i] = ll;
    return 1;
}

template <uint32_t LANES>
__device__ void join_scan(const Params &p) {
    const uint32_t lane = LANES == 1 ? 0u : (threadIdx.x & 31), upb = blockDim.x / LANES;
    const uint64_t gw = (uint64_t)blockIdx.x * upb + threadIdx.x / LANES, nw = (uint64_t)gridDim.x * upb;
    const bool bwd = !p.recognize;
    // maps of the chunks whose output depends on their input
    bool bad = false;
    for (uint64_t i = gw; i < p.c; i += nw) {
        if (p.w.fkind[i]) {                           // i >= 1: chunk 0 always has one output
            uint8_t *T = p.w.fTab + i * (p.t.nfd + 1);
            for (uint32_t S = lane; S <= p.t.nfd; S += LANES)
                T[S] = (uint8_t)eval_chunk(p, true, (uint32_t)i, S, bad);
        }
        if (lane == 0) p.w.fLink[i] = p.w.fkind[i] ? (uint32_t)i - 1 : kResolved;
        if (!bwd) continue;
        if (p.w.bkind[i]) {                           // i <= c-2
            uint8_t *T = p.w.bTab + i * (p.t.nbd + 1);
            for (uint32_t S = lane; S <= p.t.nbd; S += LANES)
                T[S] = (uint8_t)eval_chunk(p, false, (uint32_t)i, S, bad);
        }
        if (lane == 0) p.w.bLink[i] = p.w.bkind[i] ? (uint32_t)i + 1 : kResolved;
    }
    if (bad) atomicExch(&p.w.flags[FLAG_INTERNAL], 1);
    if (p.scan_stall && blockIdx.x == 0) return;      // test hook: the other blocks' waits run out
    if (!grid_barrier(p.w.scan)) { atomicExch(&p.w.flags[FLAG_TIMEOUT], 1); return; }
    for (uint32_t r = 0; r < kScanRounds; ++r) {
        uint32_t open = 0;
        for (uint64_t i = gw; i < p.c; i += nw) {
            open += scan_step<true, LANES>(p, (uint32_t)i, r & 1);
            if (bwd) open += scan_step<false, LANES>(p, (uint32_t)i, r & 1);
        }
        if (LANES == 1) open = __reduce_add_sync(0xFFFFFFFFu, open);
        if ((threadIdx.x & 31) == 0 && open) atomicAdd(p.w.scan + 2 + r, open);
        if (!grid_barrier(p.w.scan)) { atomicExch(&p.w.flags[FLAG_TIMEOUT], 1); return; }
        if (__ldcg(p.w.scan + 2 + r) == 0) break;     // every chunk resolved (same value in every block)
    }
}

__global__ void __launch_bounds__(kBlockThreads) join_scan_kernel(const __grid_constant__ Params p) {
    // every chunk has one output for every input (the common case): classify
    // has resolved them all
    if (__ldcg(p.w.scan + kScanGeneral) == 0 && !p.scan_stall) return;
    if (p.t.nfd < 16 && p.t.nbd < 16) join_scan<1>(p);   // tables of at most 16 entries: a thread per chunk
    else join_scan<32>(p);
}

// ------------------------------------------------------------------ batch
// The same steps over every chunk of every text of a group: thread j takes
// flat chunk j (its text by binary search on the chunk prefix sums).
enum BatchStep { B_CLASSIFY = 0, B_CHAIN = 1, B_VERIFY = 2 };

template <int STEP>
__global__ void join_batch_kernel(const __grid_constant__ BatchGroup b) {
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= b.chunks) return;
    const uint32_t ti = text_of(b.chunk_base, b.nt, j);
    const Params &p = b.texts[ti];
    const uint32_t i = (uint32_t)(j - b.chunk_base[ti]);
    if (STEP == B_CLASSIFY) classify_at(p, i);
    else if (STEP == B_CHAIN) chain_at(p, i);
    else verify_at(p, i);
}

// Status of every text; an empty text has the single column C_0 = I ∩ F.
__global__ void status_batch_kernel(const __grid_constant__ BatchGroup b) {
    const uint32_t ti = blockIdx.x * blockDim.x + threadIdx.x;
    if (ti >= b.nt) return;
    const Params &p = b.texts[ti];
    if (p.n == 0) empty_text(p);
    else status_of(p);
}

// Work counters of every group and the join flags of every text.
__global__ void batch_init_kernel(const Params *texts, uint32_t nt, uint32_t *queues, uint32_t nq) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nq) queues[j] = 0;
    if (j < nt && texts[j].n) {
        int32_t *f = texts[j].w.flags;
        for (uint32_t q = 0; q < FLAG_COUNT; ++q) f[q] = q < 2 ? (int32_t)texts[j].c : 0;
    }
}

}  // namespace

// Classify, then the scan (a cooperative launch: its blocks meet at grid
// barriers, so they must all be resident) or the chains, then verify.
bool launch_join(const Params &p, cudaStream_t s, int sm_count) {
    const uint32_t blocks = (p.c + kBlockThreads - 1) / kBlockThreads;
    launch_dependent(join_classify_kernel, blocks, kBlockThreads, 0, s, p);
    if (p.scan) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, join_scan_kernel, kBlockThreads, 0);
        const uint64_t units = p.c;                      // a warp (or a thread) per chunk and round
        const uint64_t want = (units + kBlockThreads / 32 - 1) / (kBlockThreads / 32);
        const uint32_t grid = (uint32_t)std::max<uint64_t>(
            1, std::min<uint64_t>(want, (uint64_t)std::max(per_sm, 1) * sm_count));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = kBlockThreads;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, join_scan_kernel, p) != cudaSuccess) return false;
    } else {
        launch_dependent(join_chain_kernel, blocks, kBlockThreads, 0, s, p);
    }
    const uint32_t vblocks = (uint32_t)(((uint64_t)p.c * 32 + kBlockThreads - 1) / kBlockThreads);
    launch_dependent(join_verify_kernel, vblocks, kBlockThreads, 0, s, p);
    return true;
}

void launch_flags_init(const Params &p, cudaStream_t s) { flags_init_kernel<<<1, 32, 0, s>>>(p); }

void launch_batch_init(const Params *texts, uint32_t nt, uint32_t *queues, uint32_t nq, cudaStream_t s) {
    const uint32_t n = nt > nq ? nt : nq;
    batch_init_kernel<<<(n + kBlockThreads - 1) / kBlockThreads, kBlockThreads, 0, s>>>(texts, nt, queues, nq);
}

// A slice's maps: classify (for the chunks' live slots), then the reduction.
bool launch_shard_map(const Params &p, uint8_t *d_maps, cudaStream_t s, int sm_count) {
    const uint32_t blocks = (p.c + kBlockThreads - 1) / kBlockThreads;
    launch_dependent(join_classify_kernel, blocks, kBlockThreads, 0, s, p);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, join_map_kernel, kBlockThreads, 0);
    const uint64_t want = ((uint64_t)p.c + kBlockThreads / 32 - 1) / (kBlockThreads / 32);
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(per_sm, 1) * sm_count));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = kBlockThreads;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, join_map_kernel, p, d_maps) == cudaSuccess;
}

void launch_join_batch(const BatchGroup &b, cudaStream_t s) {
    if (b.chunks) {
        const uint32_t blocks = (uint32_t)((b.chunks + kBlockThreads - 1) / kBlockThreads);
        join_batch_kernel<B_CLASSIFY><<<blocks, kBlockThreads, 0, s>>>(b);
        join_batch_kernel<B_CHAIN><<<blocks, kBlockThreads, 0, s>>>(b);
        join_batch_kernel<B_VERIFY><<<blocks, kBlockThreads, 0, s>>>(b);
    }
    status_batch_kernel<<<(b.nt + kBlockThreads - 1) / kBlockThreads, kBlockThreads, 0, s>>>(b);
}

}  // namespace slpf
