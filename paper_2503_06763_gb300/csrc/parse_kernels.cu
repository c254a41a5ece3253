// Device parse path of the parallel RE parser (arXiv 2503.06763, Sect. 3.2)
// and the C ABI declared in include/slpf_parser.h.
//
// Text of n bytes, chunks of k bytes (k a multiple of the sub-chunk length
// L = 64; the last chunk may be shorter), sub-chunks g = 0 .. G-1 of L bytes.
// Positions r = 0 .. n are the SLPF column indices (between bytes r-1, r).
//
//   reach   (Eq. reacher)  one thread per chunk and direction runs the DFA /
//           ME-DFA from each speculative start slot of its chunk; it writes the
//           chunk's end states R and, once all live runs of the chunk have met
//           (equal states), the exact state at every later sub-chunk boundary
//           ("checkpoints" FC / BC).
//   join    (Eq. joiner)   FJ[i] / BJ[i] = forward / backward state at the
//           boundary before chunk i.  A chunk whose live runs all end in one
//           state maps every live input to it; the others are chained
//           left-to-right (right-to-left) from their neighbour.  A verify pass
//           checks each guess against its input and finds the first chunk where
//           the text dies: the text is then rejected and the SLPF is empty.
//   fixup   the exact walks from FJ / BJ that fill the checkpoints the reach
//           runs could not give (before they converged).
//   build & merge (Eqs. builder, merger; Fig. builders&merger) one thread per
//           sub-chunk walks forward from FC[g] and backward from BC[g] and
//           writes the clean columns C_r = B_r ∩ B̂_r in the requested encoding
//           (compose, Sect. 3.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "re_internal.h"

namespace slpf {

// ----------------------------------------------------------------------------
// error reporting
static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

static re_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return RE_E_CUDA;
}
#define CUDA_TRY(expr, what)                        \
    do {                                            \
        cudaError_t _e = (expr);                    \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

constexpr int kMaxW = 64;          // segments per column <= 4096
constexpr int kThreads = 128;

enum Flag { FLAG_FFAIL = 0, FLAG_BFAIL = 1, FLAG_INTERNAL = 2, FLAG_COUNT = 4 };

struct Work {                       // device workspace, carved from the caller's buffer
    uint32_t *Rf, *Rb;              // [c][msf], [c][msb] end state of each slot
    uint32_t *FJ, *BJ;              // [c+1]
    uint32_t *FC, *BC;              // [G]
    uint32_t *fconv, *bconv;        // [c]
    uint32_t *fkind, *bkind;        // [c]: 0 = one live end state (or all dead), 1 = several
    int32_t *flags;                 // [FLAG_COUNT]
};

struct Params {
    DevTables t;
    const uint8_t *x;
    uint64_t n;
    uint32_t k, c, S;               // chunk length, chunks, sub-chunks per chunk
    uint64_t G;                     // sub-chunks
    Work w;
    void *out;
    uint32_t col_bytes, kind;       // output encoding
    int32_t *status;
};

__device__ __forceinline__ uint32_t chunk_len(const Params &p, uint32_t i) {
    uint64_t base = (uint64_t)i * p.k;
    uint64_t rest = p.n - base;
    return rest < p.k ? (uint32_t)rest : p.k;
}

__device__ __forceinline__ bool any_and(const uint64_t *a, const uint64_t *b, uint32_t W) {
    for (uint32_t w = 0; w < W; ++w)
        if (__ldg(a + w) & __ldg(b + w)) return true;
    return false;
}

// Text bytes are read 16 at a time when the whole group lies inside [0, n).
__device__ __forceinline__ void load16(const uint8_t *x, uint64_t n, uint64_t at, uint8_t out[16]) {
    if (at + 16 <= n) {
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(x + at));
        memcpy(out, &v, 16);
    } else {
        for (int j = 0; j < 16; ++j) out[j] = (at + j < n) ? __ldg(x + at + j) : 0;
    }
}

// ----------------------------------------------------------------------------
// reach (Eq. reacher): forward direction.
template <int MS>
__global__ void __launch_bounds__(kThreads) reach_fwd_kernel(Params p) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.c) return;
    const DevTables &t = p.t;
    const uint64_t base = (uint64_t)i * p.k;
    const uint32_t len = chunk_len(p, i);
    const uint32_t nsub = (len + kSub - 1) / kSub;
    uint32_t st[MS];
#pragma unroll
    for (int j = 0; j < MS; ++j) st[j] = 0u;               // unused slots stay dead
    uint32_t m, tstart;
    if (i == 0) {
        m = 1; st[0] = t.fI; tstart = 0;                 // J_0 = I: no speculation
    } else {
        uint32_t pr = t.cls[p.x[base - 1]] * t.ncls + t.cls[p.x[base]];
        m = t.fSlotCount[pr];
        for (int j = 0; j < MS; ++j) st[j] = (j < (int)m) ? t.fSlotStart[pr * t.msf + j] : 0u;
        tstart = 1;                                      // start sets are after byte 0
    }
    bool conv = m <= 1;
    uint32_t conv_sub = conv ? 1 : nsub;
    for (uint32_t t0 = 0; t0 < len; t0 += 16) {
        uint8_t b16[16];
        load16(p.x, p.n, base + t0, b16);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            uint32_t tt = t0 + u;
            if (tt >= len) break;
            if (tt > 0 && (tt % kSub) == 0) {            // boundary before byte tt
                uint32_t rep = 0;
                if (!conv) {
                    bool same = true;
#pragma unroll
                    for (int j = 0; j < MS; ++j)
                        if (st[j]) { if (!rep) rep = st[j]; else if (st[j] != rep) same = false; }
                    if (same) { conv = true; conv_sub = tt / kSub; }
                }
                if (conv) {
                    if (!rep) {
#pragma unroll
                        for (int j = 0; j < MS; ++j) if (st[j]) rep = st[j];
                    }
                    p.w.FC[(base + tt) / kSub] = rep;
                } else {
                    p.w.FC[(base + tt) / kSub] = kUnknown;
                }
            }
            if (tt < tstart) continue;
            uint32_t cb = t.cls[b16[u]];
#pragma unroll
            for (int j = 0; j < MS; ++j)
                if (j < (int)m) st[j] = __ldg(t.fT + (size_t)st[j] * t.ncls + cb);
        }
    }
    for (int j = 0; j < MS; ++j)
        if (j < (int)t.msf) p.w.Rf[(size_t)i * t.msf + j] = (j < (int)m) ? st[j] : 0u;
    p.w.fconv[i] = conv_sub;
}

// reach: backward direction (reverse ME-DFA over the reversed chunk).
template <int MS>
__global__ void __launch_bounds__(kThreads) reach_bwd_kernel(Params p) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.c) return;
    const DevTables &t = p.t;
    const uint64_t base = (uint64_t)i * p.k;
    const uint32_t len = chunk_len(p, i);
    const uint32_t nsub = (len + kSub - 1) / kSub;
    uint32_t st[MS];
#pragma unroll
    for (int j = 0; j < MS; ++j) st[j] = 0u;               // unused slots stay dead
    uint32_t m;
    int64_t tlast;                                        // first byte (from the right) to consume
    if (i == p.c - 1) {
        m = 1; st[0] = t.bF; tlast = (int64_t)len - 1;   // Ĵ_{c+1} = F
    } else {
        uint32_t pr = t.cls[p.x[base + len - 1]] * t.ncls + t.cls[p.x[base + len]];
        m = t.bSlotCount[pr];
        for (int j = 0; j < MS; ++j) st[j] = (j < (int)m) ? t.bSlotStart[pr * t.msb + j] : 0u;
        tlast = (int64_t)len - 2;                         // start sets are before the last byte
    }
    bool conv = m <= 1;
    uint32_t conv_sub = conv ? (nsub ? nsub - 1 : 0) : 0;
    // groups of 16 bytes from the right end of the chunk
    int64_t g0 = ((int64_t)len - 1) & ~15ll;
    for (int64_t t0 = g0; t0 >= 0; t0 -= 16) {
        uint8_t b16[16];
        load16(p.x, p.n, base + (uint64_t)t0, b16);
#pragma unroll
        for (int u = 15; u >= 0; --u) {
            int64_t tt = t0 + u;
            if (tt > tlast) continue;
            uint32_t cb = t.cls[b16[u]];
#pragma unroll
            for (int j = 0; j < MS; ++j)
                if (j < (int)m) st[j] = __ldg(t.bT + (size_t)st[j] * t.ncls + cb);
            if (tt > 0 && (tt % kSub) == 0) {             // now at the boundary before byte tt
                uint32_t rep = 0;
                if (!conv) {
                    bool same = true;
#pragma unroll
                    for (int j = 0; j < MS; ++j)
                        if (st[j]) { if (!rep) rep = st[j]; else if (st[j] != rep) same = false; }
                    if (same) { conv = true; conv_sub = (uint32_t)(tt / kSub); }
                }
                if (conv) {
                    if (!rep) {
#pragma unroll
                        for (int j = 0; j < MS; ++j) if (st[j]) rep = st[j];
                    }
                    p.w.BC[(base + (uint64_t)tt) / kSub - 1] = rep;
                } else {
                    p.w.BC[(base + (uint64_t)tt) / kSub - 1] = kUnknown;
                }
            }
        }
    }
    for (int j = 0; j < MS; ++j)
        if (j < (int)t.msb) p.w.Rb[(size_t)i * t.msb + j] = (j < (int)m) ? st[j] : 0u;
    p.w.bconv[i] = conv_sub;
}

// ----------------------------------------------------------------------------
// join (Eq. joiner)
__device__ uint32_t probe(const uint32_t *hash, uint32_t mask, const uint64_t *bits, uint32_t W,
                          const uint64_t *key) {
    uint64_t h = bits_hash(key, W) & mask;
    for (uint32_t step = 0; step <= mask; ++step) {
        uint32_t id = __ldg(hash + h);
        if (id == 0) return 0;
        bool eq = true;
        for (uint32_t w = 0; w < W; ++w)
            if (__ldg(bits + (size_t)id * W + w) != key[w]) { eq = false; break; }
        if (eq) return id;
        h = (h + 1) & mask;
    }
    return 0;
}

// State after chunk i from input state S (union over the slots S can enter).
__device__ uint32_t eval_chunk(const Params &p, bool fwd, uint32_t i, uint32_t S, bool &bad) {
    const DevTables &t = p.t;
    if (S == 0) return 0;
    const uint32_t W = t.W;
    uint32_t pr, m, ms;
    const uint32_t *R;
    const uint64_t *mask, *bits;
    if (fwd) {
        uint64_t base = (uint64_t)i * p.k;
        pr = t.cls[p.x[base - 1]] * t.ncls + t.cls[p.x[base]];
        m = t.fSlotCount[pr]; ms = t.msf; R = p.w.Rf + (size_t)i * ms;
        mask = t.fSlotMask + (size_t)pr * ms * W; bits = t.fBits;
    } else {
        uint64_t end = (uint64_t)i * p.k + chunk_len(p, i);
        pr = t.cls[p.x[end - 1]] * t.ncls + t.cls[p.x[end]];
        m = t.bSlotCount[pr]; ms = t.msb; R = p.w.Rb + (size_t)i * ms;
        mask = t.bSlotMask + (size_t)pr * ms * W; bits = t.bBits;
    }
    const uint64_t *sb = bits + (size_t)S * W;
    uint32_t single = 0;
    bool multi = false;
    uint64_t acc[kMaxW];
    for (uint32_t w = 0; w < W; ++w) acc[w] = 0;
    for (uint32_t s = 0; s < m; ++s) {
        uint32_t e = R[s];
        if (!e || !any_and(sb, mask + (size_t)s * W, W)) continue;
        if (!single) single = e;
        else if (e != single) multi = true;
        for (uint32_t w = 0; w < W; ++w) acc[w] |= __ldg(bits + (size_t)e * W + w);
    }
    if (!multi) return single;
    uint32_t id = fwd ? probe(t.fHash, t.fHashMask, t.fBits, W, acc) : probe(t.bHash, t.bHashMask, t.bBits, W, acc);
    if (!id) bad = true;
    return id;
}

__global__ void join_classify_kernel(Params p) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.c) return;
    const DevTables &t = p.t;
    // forward
    if (i == 0) {
        p.w.FJ[0] = t.fI;
        p.w.FJ[1] = p.w.Rf[0];
        p.w.fkind[0] = 0;
    } else {
        uint64_t base = (uint64_t)i * p.k;
        uint32_t pr = t.cls[p.x[base - 1]] * t.ncls + t.cls[p.x[base]];
        uint32_t m = t.fSlotCount[pr], rep = 0;
        bool gen = false;
        for (uint32_t s = 0; s < m; ++s) {
            uint32_t e = p.w.Rf[(size_t)i * t.msf + s];
            if (e) { if (!rep) rep = e; else if (e != rep) gen = true; }
        }
        p.w.fkind[i] = gen ? 1u : 0u;
        if (!gen) p.w.FJ[i + 1] = rep;
    }
    // backward
    if (i == p.c - 1) {
        p.w.BJ[p.c] = t.bF;
        p.w.BJ[i] = p.w.Rb[(size_t)i * t.msb];
        p.w.bkind[i] = 0;
    } else {
        uint64_t end = (uint64_t)i * p.k + chunk_len(p, i);
        uint32_t pr = t.cls[p.x[end - 1]] * t.ncls + t.cls[p.x[end]];
        uint32_t m = t.bSlotCount[pr], rep = 0;
        bool gen = false;
        for (uint32_t s = 0; s < m; ++s) {
            uint32_t e = p.w.Rb[(size_t)i * t.msb + s];
            if (e) { if (!rep) rep = e; else if (e != rep) gen = true; }
        }
        p.w.bkind[i] = gen ? 1u : 0u;
        if (!gen) p.w.BJ[i] = rep;
    }
}

// Chains of chunks whose runs did not meet: walked from their known neighbour.
__global__ void join_chain_kernel(Params p) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.c) return;
    bool bad = false;
    if (p.w.fkind[i] == 1 && p.w.fkind[i - 1] == 0) {     // i >= 1 since fkind[0] == 0
        uint32_t cur = p.w.FJ[i];
        for (uint32_t j = i; j < p.c && p.w.fkind[j] == 1; ++j) {
            cur = eval_chunk(p, true, j, cur, bad);
            p.w.FJ[j + 1] = cur;
        }
    }
    if (p.w.bkind[i] == 1 && p.w.bkind[i + 1] == 0) {     // i <= c-2 since bkind[c-1] == 0
        uint32_t cur = p.w.BJ[i + 1];
        for (int64_t j = i; j >= 0 && p.w.bkind[j] == 1; --j) {
            cur = eval_chunk(p, false, (uint32_t)j, cur, bad);
            p.w.BJ[j] = cur;
        }
    }
    if (bad) atomicExch(&p.w.flags[FLAG_INTERNAL], 1);
}

// Check each chunk's guessed output against its (now known) input.
__global__ void join_verify_kernel(Params p) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.c) return;
    const DevTables &t = p.t;
    const uint32_t W = t.W;
    // forward: input FJ[i] -> output FJ[i+1]
    {
        uint32_t in = p.w.FJ[i], out = p.w.FJ[i + 1];
        bool fail = (in == 0 || out == 0);
        if (!fail && i > 0 && p.w.fkind[i] == 0) {
            uint64_t base = (uint64_t)i * p.k;
            uint32_t pr = t.cls[p.x[base - 1]] * t.ncls + t.cls[p.x[base]];
            uint32_t m = t.fSlotCount[pr];
            bool hit = false;
            for (uint32_t s = 0; s < m && !hit; ++s)
                hit = p.w.Rf[(size_t)i * t.msf + s] != 0 &&
                      any_and(t.fBits + (size_t)in * W, t.fSlotMask + ((size_t)pr * t.msf + s) * W, W);
            fail = !hit;
        }
        if (fail) atomicMin(&p.w.flags[FLAG_FFAIL], (int32_t)i);
    }
    // backward: input BJ[i+1] -> output BJ[i]
    {
        uint32_t in = p.w.BJ[i + 1], out = p.w.BJ[i];
        bool fail = (in == 0 || out == 0);
        if (!fail && i < p.c - 1 && p.w.bkind[i] == 0) {
            uint64_t end = (uint64_t)i * p.k + chunk_len(p, i);
            uint32_t pr = t.cls[p.x[end - 1]] * t.ncls + t.cls[p.x[end]];
            uint32_t m = t.bSlotCount[pr];
            bool hit = false;
            for (uint32_t s = 0; s < m && !hit; ++s)
                hit = p.w.Rb[(size_t)i * t.msb + s] != 0 &&
                      any_and(t.bBits + (size_t)in * W, t.bSlotMask + ((size_t)pr * t.msb + s) * W, W);
            fail = !hit;
        }
        if (fail) atomicMin(&p.w.flags[FLAG_BFAIL], (int32_t)i);
    }
    // chunk-boundary checkpoints
    p.w.FC[(uint64_t)i * p.S] = p.w.FJ[i];
    if (i + 1 < p.c) p.w.BC[(uint64_t)(i + 1) * p.S - 1] = p.w.BJ[i + 1];
    else p.w.BC[p.G - 1] = p.w.BJ[p.c];
}

// Accept iff both joins ran through and C_0 = I ∩ Ĵ_1 is not empty.
__global__ void status_kernel(Params p) {
    const DevTables &t = p.t;
    int32_t st = RE_OK;
    if (p.w.flags[FLAG_FFAIL] < (int32_t)p.c || p.w.flags[FLAG_BFAIL] < (int32_t)p.c) {
        st = RE_REJECTED;
    } else {
        uint32_t b0 = p.w.BJ[0];
        bool meet = b0 != 0 && any_and(t.fBits + (size_t)t.fI * t.W, t.bBits + (size_t)b0 * t.W, t.W);
        if (!meet) st = RE_REJECTED;
    }
    if (p.w.flags[FLAG_INTERNAL]) st = RE_E_INTERNAL;
    *p.status = st;
}

// ----------------------------------------------------------------------------
// fixup: exact walks for checkpoints before the reach runs met.
__global__ void fixup_kernel(Params p) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.c || *p.status != RE_OK) return;
    const DevTables &t = p.t;
    const uint64_t base = (uint64_t)i * p.k;
    const uint32_t len = chunk_len(p, i);
    const uint32_t nsub = (len + kSub - 1) / kSub;
    // forward: boundaries s = 1 .. fconv-1
    uint32_t fc = p.w.fconv[i];
    if (fc > 1) {
        uint32_t st = p.w.FJ[i];
        uint32_t upto = (fc - 1) * kSub;
        for (uint32_t tt = 0; tt < upto; ++tt) {
            st = __ldg(t.fT + (size_t)st * t.ncls + t.cls[__ldg(p.x + base + tt)]);
            if (((tt + 1) % kSub) == 0) p.w.FC[(base + tt + 1) / kSub] = st;
        }
    }
    // backward: boundaries s = nsub-1 down to bconv+1
    uint32_t bc = p.w.bconv[i];
    if (nsub >= 2 && bc + 1 <= nsub - 1) {
        uint32_t st = p.w.BJ[i + 1];
        int64_t downto = (int64_t)(bc + 1) * kSub;
        for (int64_t tt = (int64_t)len - 1; tt >= downto; --tt) {
            st = __ldg(t.bT + (size_t)st * t.ncls + t.cls[__ldg(p.x + base + tt)]);
            if ((tt % kSub) == 0) p.w.BC[(base + tt) / kSub - 1] = st;
        }
    }
}

// ----------------------------------------------------------------------------
// build & merge (Eqs. builder, merger; Fig. builders&merger) + compose.
template <typename Out>
__device__ __forceinline__ void store_col(const Params &p, uint64_t r, Out v) {
    reinterpret_cast<Out *>(p.out)[r] = v;
}

__device__ __forceinline__ void emit(const Params &p, uint64_t r, uint32_t f, uint32_t b, bool &bad) {
    const DevTables &t = p.t;
    if (p.kind == RE_SLPF_DENSE) {
        uint64_t v = (f && b) ? (__ldg(t.fBits + f) & __ldg(t.bBits + b)) : 0ull;  // W == 1
        switch (p.col_bytes) {
            case 1: store_col<uint8_t>(p, r, (uint8_t)v); break;
            case 2: store_col<uint16_t>(p, r, (uint16_t)v); break;
            case 4: store_col<uint32_t>(p, r, (uint32_t)v); break;
            default: store_col<uint64_t>(p, r, v); break;
        }
    } else {
        uint32_t d = 0;
        if (f && b) {
            if (f > t.nfd || b > t.nbd) bad = true;
            else d = __ldg(t.pt + (size_t)f * (t.nbd + 1) + b);
        }
        if (p.col_bytes == 2) store_col<uint16_t>(p, r, (uint16_t)d);
        else store_col<uint32_t>(p, r, d);
    }
}

__global__ void __launch_bounds__(kThreads) merge_kernel(Params p) {
    uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= p.G) return;
    const DevTables &t = p.t;
    const uint64_t pos0 = g * kSub;
    const uint64_t rest = p.n - pos0;
    const uint32_t len = rest < kSub ? (uint32_t)rest : kSub;
    const bool ok = (*p.status == RE_OK);
    bool bad = false;
    if (!ok) {
        for (uint32_t u = 0; u < len; ++u) emit(p, pos0 + u + 1, 0, 0, bad);
        if (g == 0) emit(p, 0, 0, 0, bad);
        return;
    }
    uint32_t F[kSub], B[kSub];
    uint32_t f = p.w.FC[g];
    uint8_t xb[kSub];
    for (uint32_t u = 0; u < kSub; u += 16) load16(p.x, p.n, pos0 + u, xb + u);
    if (f == kUnknown) { bad = true; f = 0; }           // never index tables with the sentinel
    for (uint32_t u = 0; u < len; ++u) {                  // B at positions pos0+u+1
        f = __ldg(t.fT + (size_t)f * t.ncls + t.cls[xb[u]]);
        F[u] = f;
    }
    uint32_t b = p.w.BC[g];                               // B̂ at position pos0+len
    if (b == kUnknown) { bad = true; b = 0; }
    B[len - 1] = b;
    for (int u = (int)len - 1; u >= 1; --u) {             // B̂ at positions pos0+u
        b = __ldg(t.bT + (size_t)b * t.ncls + t.cls[xb[u]]);
        B[u - 1] = b;
    }
    for (uint32_t u = 0; u < len; ++u) emit(p, pos0 + u + 1, F[u], B[u], bad);
    if (g == 0) {                                         // C_0 = J_0 ∩ Ĵ_1
        uint32_t b0 = __ldg(t.bT + (size_t)B[0] * t.ncls + t.cls[xb[0]]);
        emit(p, 0, p.w.FC[0], b0, bad);
    }
    if (bad) atomicExch(p.status, RE_E_INTERNAL);
}

__global__ void flags_init_kernel(Params p) {
    if (threadIdx.x < FLAG_COUNT)
        p.w.flags[threadIdx.x] = threadIdx.x < 2 ? (int32_t)p.c : 0;   // first failing chunk: none
}

// Empty text: one column C_0 = I ∩ F.
__global__ void empty_text_kernel(Params p) {
    const DevTables &t = p.t;
    bool bad = false;
    bool meet = any_and(t.fBits + (size_t)t.fI * t.W, t.bBits + (size_t)t.bF * t.W, t.W);
    *p.status = meet ? RE_OK : RE_REJECTED;
    emit(p, 0, meet ? t.fI : 0, meet ? t.bF : 0, bad);
    if (bad) *p.status = RE_E_INTERNAL;
}

// ----------------------------------------------------------------------------
// host side
static int g_sm_count = 0;

static uint32_t choose_chunk(uint64_t n, const re_parse_opts *opts) {
    if (opts && opts->chunk_len) return opts->chunk_len;
    uint64_t target = (uint64_t)(g_sm_count ? g_sm_count : 152) * 1024;   // one reach thread per chunk
    uint64_t k = (n + target - 1) / target;
    k = (k + kSub - 1) / kSub * kSub;
    return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(k, kSub), 1u << 20);
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
    uint32_t k, c, S;
    uint64_t G;
    size_t off[11];
    size_t total;
};

static Layout layout_for(const re_handle *h, uint64_t n, uint32_t k) {
    Layout L{};
    L.k = k;
    L.c = (uint32_t)((n + k - 1) / k);
    L.S = k / kSub;
    L.G = (n + kSub - 1) / kSub;
    size_t sizes[11] = {
        (size_t)L.c * h->host.msf * 4, (size_t)L.c * h->host.msb * 4,
        (size_t)(L.c + 1) * 4, (size_t)(L.c + 1) * 4,
        (size_t)L.G * 4, (size_t)L.G * 4,
        (size_t)L.c * 4, (size_t)L.c * 4, (size_t)L.c * 4, (size_t)L.c * 4,
        FLAG_COUNT * 4};
    size_t o = 0;
    for (int j = 0; j < 11; ++j) { L.off[j] = o; o += align256(sizes[j] ? sizes[j] : 4); }
    L.total = o;
    return L;
}

static re_status resolve_kind(const re_handle *h, re_slpf_kind kind, re_slpf_kind &out, uint32_t &cb) {
    const Compiled &C = h->host;
    if (kind == RE_SLPF_AUTO) {
        if (C.ell <= 16) kind = RE_SLPF_DENSE;
        else if (C.has_dict) kind = RE_SLPF_DICT;
        else if (C.ell <= 64) kind = RE_SLPF_DENSE;
        else { set_error("no encoding available: more than 64 segments and no dictionary"); return RE_E_CAPACITY; }
    }
    if (kind == RE_SLPF_DENSE) {
        if (C.ell > 64) { set_error("DENSE needs at most 64 segments"); return RE_E_CAPACITY; }
        cb = C.ell <= 8 ? 1 : C.ell <= 16 ? 2 : C.ell <= 32 ? 4 : 8;
    } else if (kind == RE_SLPF_DICT) {
        if (!C.has_dict) { set_error("this RE has no column dictionary (too many state pairs)"); return RE_E_CAPACITY; }
        cb = C.dict_size < 65535 ? 2 : 4;
    } else {
        set_error("unknown SLPF kind");
        return RE_E_INVALID_ARG;
    }
    out = kind;
    return RE_OK;
}

template <int MS>
static void launch_reach(const Params &p, cudaStream_t s, uint32_t blocks) {
    reach_fwd_kernel<MS><<<blocks, kThreads, 0, s>>>(p);
}
template <int MS>
static void launch_reach_b(const Params &p, cudaStream_t s, uint32_t blocks) {
    reach_bwd_kernel<MS><<<blocks, kThreads, 0, s>>>(p);
}

static bool dispatch_reach_f(const Params &p, cudaStream_t s, uint32_t blocks, uint32_t msf) {
    if (msf <= 2) launch_reach<2>(p, s, blocks);
    else if (msf <= 4) launch_reach<4>(p, s, blocks);
    else if (msf <= 8) launch_reach<8>(p, s, blocks);
    else if (msf <= 16) launch_reach<16>(p, s, blocks);
    else if (msf <= 32) launch_reach<32>(p, s, blocks);
    else if (msf <= 64) launch_reach<64>(p, s, blocks);
    else if (msf <= 128) launch_reach<128>(p, s, blocks);
    else return false;
    return true;
}

static bool dispatch_reach_b(const Params &p, cudaStream_t s, uint32_t blocks, uint32_t msb) {
    if (msb <= 2) launch_reach_b<2>(p, s, blocks);
    else if (msb <= 4) launch_reach_b<4>(p, s, blocks);
    else if (msb <= 8) launch_reach_b<8>(p, s, blocks);
    else if (msb <= 16) launch_reach_b<16>(p, s, blocks);
    else if (msb <= 32) launch_reach_b<32>(p, s, blocks);
    else if (msb <= 64) launch_reach_b<64>(p, s, blocks);
    else if (msb <= 128) launch_reach_b<128>(p, s, blocks);
    else return false;
    return true;
}

}  // namespace slpf

using namespace slpf;

// ============================================================================ C ABI
extern "C" {

const char *re_last_error(void) { return g_last_error.c_str(); }

re_status re_compile(const char *pattern, size_t len, const re_compile_opts *opts, re_handle **out) {
    if (!pattern || !out) { set_error("null argument"); return RE_E_INVALID_ARG; }
    *out = nullptr;
    re_handle *h = new (std::nothrow) re_handle();
    if (!h) { set_error("host allocation failed"); return RE_E_NOMEM; }
    std::string err;
    re_status st;
    try {
        st = compile_pattern(pattern, len, opts, h->host, err);
    } catch (const std::bad_alloc &) {
        st = RE_E_NOMEM; err = "host allocation failed during compile";
    }
    if (st != RE_OK) { set_error(err); delete h; return st; }
    Compiled &C = h->host;
    h->host_only = opts && (opts->flags & RE_COMPILE_HOST_ONLY);
    if (C.W > (uint32_t)kMaxW) { set_error("more than 4096 segments"); delete h; return RE_E_TOO_MANY_STATES; }
    if (C.msf > 128 || C.msb > 128) { set_error("more than 128 speculative runs per chunk"); delete h; return RE_E_TOO_MANY_STATES; }
    // one device allocation for all tables
    struct Piece { const void *src; size_t bytes; size_t off; };
    std::vector<Piece> pc;
    size_t total = 0;
    auto add = [&](const void *src, size_t bytes) {
        pc.push_back({src, bytes, total});
        total += align256(bytes ? bytes : 4);
        return pc.size() - 1;
    };
    size_t i_cls = add(C.cls, 256);
    size_t i_fT = add(C.fT.data(), C.fT.size() * 4), i_bT = add(C.bT.data(), C.bT.size() * 4);
    size_t i_fB = add(C.fBits.data(), C.fBits.size() * 8), i_bB = add(C.bBits.data(), C.bBits.size() * 8);
    size_t i_fH = add(C.fHash.data(), C.fHash.size() * 4), i_bH = add(C.bHash.data(), C.bHash.size() * 4);
    size_t i_fSS = add(C.fSlotStart.data(), C.fSlotStart.size() * 4);
    size_t i_fSM = add(C.fSlotMask.data(), C.fSlotMask.size() * 8);
    size_t i_fSC = add(C.fSlotCount.data(), C.fSlotCount.size() * 4);
    size_t i_bSS = add(C.bSlotStart.data(), C.bSlotStart.size() * 4);
    size_t i_bSM = add(C.bSlotMask.data(), C.bSlotMask.size() * 8);
    size_t i_bSC = add(C.bSlotCount.data(), C.bSlotCount.size() * 4);
    size_t i_pt = add(C.pt.data(), C.pt.size() * 4);
    if (h->host_only) { *out = h; return RE_OK; }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_alloc, total);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "re_compile: device tables"); }
    h->d_bytes = total;
    std::vector<uint8_t> staging(total, 0);
    for (auto &q : pc) if (q.bytes) std::memcpy(staging.data() + q.off, q.src, q.bytes);
    e = cudaMemcpy(h->d_alloc, staging.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(h->d_alloc); delete h; return cuda_fail(e, "re_compile: upload"); }
    if (!g_sm_count) cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, h->device);
    uint8_t *b = (uint8_t *)h->d_alloc;
    DevTables &t = h->dev;
    t.cls = b + pc[i_cls].off;
    t.fT = (const uint32_t *)(b + pc[i_fT].off); t.bT = (const uint32_t *)(b + pc[i_bT].off);
    t.fBits = (const uint64_t *)(b + pc[i_fB].off); t.bBits = (const uint64_t *)(b + pc[i_bB].off);
    t.fHash = (const uint32_t *)(b + pc[i_fH].off); t.bHash = (const uint32_t *)(b + pc[i_bH].off);
    t.fSlotStart = (const uint32_t *)(b + pc[i_fSS].off); t.fSlotMask = (const uint64_t *)(b + pc[i_fSM].off);
    t.fSlotCount = (const uint32_t *)(b + pc[i_fSC].off);
    t.bSlotStart = (const uint32_t *)(b + pc[i_bSS].off); t.bSlotMask = (const uint64_t *)(b + pc[i_bSM].off);
    t.bSlotCount = (const uint32_t *)(b + pc[i_bSC].off);
    t.pt = (const uint32_t *)(b + pc[i_pt].off);
    t.fHashMask = C.fHashMask; t.bHashMask = C.bHashMask;
    t.ncls = C.ncls; t.W = C.W; t.ell = C.ell;
    t.nf = C.nf; t.nb = C.nb; t.nfd = C.nfd; t.nbd = C.nbd;
    t.msf = C.msf; t.msb = C.msb; t.fI = 1; t.bF = 1;
    t.dict_size = C.dict_size;
    *out = h;
    return RE_OK;
}

void re_free(re_handle *h) {
    if (!h) return;
    if (h->d_alloc) cudaFree(h->d_alloc);
    delete h;
}

re_status re_get_info(const re_handle *h, re_info *info) {
    if (!h || !info) { set_error("null argument"); return RE_E_INVALID_ARG; }
    const Compiled &C = h->host;
    info->n_segments = C.ell; info->n_positions = C.npos; info->n_classes = C.ncls;
    info->words_per_col = C.W;
    info->fwd_states = C.nf - 1; info->fwd_dfa_states = C.nfd;
    info->bwd_states = C.nb - 1; info->bwd_dfa_states = C.nbd;
    info->fwd_slots_max = C.msf; info->bwd_slots_max = C.msb;
    info->dict_size = C.has_dict ? C.dict_size : 0;
    return RE_OK;
}

re_status re_segment_name(const re_handle *h, uint32_t id, char *buf, size_t cap) {
    if (!h || !buf || cap == 0) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (id >= h->host.ell) { set_error("segment id out of range"); return RE_E_INVALID_ARG; }
    const std::string &s = h->host.names[id];
    if (s.size() + 1 > cap) { set_error("buffer too small"); return RE_E_CAPACITY; }
    std::memcpy(buf, s.c_str(), s.size() + 1);
    return RE_OK;
}

re_status re_dict_copy(const re_handle *h, uint64_t *host_words, uint64_t cap_words) {
    if (!h || (!host_words && cap_words)) { set_error("null argument"); return RE_E_INVALID_ARG; }
    const Compiled &C = h->host;
    if (!C.has_dict) { set_error("no dictionary"); return RE_E_CAPACITY; }
    if (cap_words < C.dict.size()) { set_error("buffer too small"); return RE_E_CAPACITY; }
    if (!C.dict.empty()) std::memcpy(host_words, C.dict.data(), C.dict.size() * 8);
    return RE_OK;
}

re_status re_slpf_layout(const re_handle *h, uint64_t len, re_slpf_kind kind, re_slpf_kind *kind_out,
                         uint32_t *col_bytes, uint64_t *bytes) {
    if (!h) { set_error("null handle"); return RE_E_INVALID_ARG; }
    re_slpf_kind k;
    uint32_t cb;
    re_status st = resolve_kind(h, kind, k, cb);
    if (st != RE_OK) return st;
    if (kind_out) *kind_out = k;
    if (col_bytes) *col_bytes = cb;
    if (bytes) *bytes = (len + 1) * cb;
    return RE_OK;
}

re_status re_workspace_size(const re_handle *h, uint64_t len, const re_parse_opts *opts, uint64_t *bytes) {
    if (!h || !bytes) { set_error("null argument"); return RE_E_INVALID_ARG; }
    uint32_t k = choose_chunk(len, opts);
    if (k % kSub) { set_error("chunk_len must be a multiple of 64"); return RE_E_INVALID_ARG; }
    *bytes = layout_for(h, len, k).total;
    return RE_OK;
}

re_status re_parse(re_handle *h, const uint8_t *d_text, uint64_t len, re_stream stream, re_slpf *slpf,
                   void *d_workspace, uint64_t workspace_bytes, const re_parse_opts *opts) {
    if (!h || !slpf || !slpf->d_status || (len && !d_text)) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (h->host_only) { set_error("handle was compiled with RE_COMPILE_HOST_ONLY"); return RE_E_INVALID_ARG; }
    if (len && ((uintptr_t)d_text & 15)) { set_error("d_text must be 16-byte aligned"); return RE_E_INVALID_ARG; }
    if (opts && (opts->flags & ~RE_PARSE_RECOGNIZE_ONLY)) { set_error("unknown parse flags"); return RE_E_INVALID_ARG; }
    if (opts && opts->n_events && (opts->n_events != RE_PHASE_EVENTS || !opts->events)) {
        set_error("n_events must be 0 or RE_PHASE_EVENTS"); return RE_E_INVALID_ARG;
    }
    cudaEvent_t *ev = (opts && opts->n_events) ? (cudaEvent_t *)opts->events : nullptr;
    re_slpf_kind kind;
    uint32_t cb;
    re_status st = resolve_kind(h, slpf->kind, kind, cb);
    if (st != RE_OK) return st;
    if (slpf->col_bytes != cb) { set_error("slpf->col_bytes does not match the layout"); return RE_E_INVALID_ARG; }
    if (!slpf->d_cols || slpf->cols_cap_bytes < (len + 1) * cb) { set_error("SLPF buffer too small"); return RE_E_CAPACITY; }
    if (((uintptr_t)slpf->d_cols % cb) != 0) { set_error("d_cols misaligned"); return RE_E_INVALID_ARG; }
    uint32_t k = choose_chunk(len, opts);
    if (k % kSub || k == 0) { set_error("chunk_len must be a positive multiple of 64"); return RE_E_INVALID_ARG; }
    Layout L = layout_for(h, len, k);
    if (len && (!d_workspace || workspace_bytes < L.total || ((uintptr_t)d_workspace & 255))) {
        set_error("workspace missing, too small or not 256-byte aligned");
        return RE_E_CAPACITY;
    }
    slpf->n_cols = len + 1;
    cudaStream_t s = (cudaStream_t)stream;
    Params p{};
    p.t = h->dev;
    p.x = d_text; p.n = len; p.k = k; p.c = L.c; p.S = L.S; p.G = L.G;
    p.out = slpf->d_cols; p.col_bytes = cb; p.kind = kind; p.status = slpf->d_status;
    int dev_now = 0;
    cudaGetDevice(&dev_now);
    if (dev_now != h->device) { set_error("current device differs from the handle's device"); return RE_E_INVALID_ARG; }
    auto mark = [&](int j) -> cudaError_t { return ev ? cudaEventRecord(ev[j], s) : cudaSuccess; };
    if (len == 0) {
        CUDA_TRY(mark(0), "event");
        empty_text_kernel<<<1, 1, 0, s>>>(p);
        for (int j = 1; j < (int)RE_PHASE_EVENTS; ++j) CUDA_TRY(mark(j), "event");
        CUDA_TRY(cudaGetLastError(), "launch");
        return RE_OK;
    }
    uint8_t *w = (uint8_t *)d_workspace;
    p.w.Rf = (uint32_t *)(w + L.off[0]); p.w.Rb = (uint32_t *)(w + L.off[1]);
    p.w.FJ = (uint32_t *)(w + L.off[2]); p.w.BJ = (uint32_t *)(w + L.off[3]);
    p.w.FC = (uint32_t *)(w + L.off[4]); p.w.BC = (uint32_t *)(w + L.off[5]);
    p.w.fconv = (uint32_t *)(w + L.off[6]); p.w.bconv = (uint32_t *)(w + L.off[7]);
    p.w.fkind = (uint32_t *)(w + L.off[8]); p.w.bkind = (uint32_t *)(w + L.off[9]);
    p.w.flags = (int32_t *)(w + L.off[10]);
    CUDA_TRY(mark(0), "event");
    flags_init_kernel<<<1, 32, 0, s>>>(p);
    uint32_t cblocks = (L.c + kThreads - 1) / kThreads;
    if (!dispatch_reach_f(p, s, cblocks, h->host.msf)) { set_error("too many slots"); return RE_E_INTERNAL; }
    CUDA_TRY(mark(1), "event");
    if (!dispatch_reach_b(p, s, cblocks, h->host.msb)) { set_error("too many slots"); return RE_E_INTERNAL; }
    CUDA_TRY(mark(2), "event");
    join_classify_kernel<<<cblocks, kThreads, 0, s>>>(p);
    join_chain_kernel<<<cblocks, kThreads, 0, s>>>(p);
    join_verify_kernel<<<cblocks, kThreads, 0, s>>>(p);
    status_kernel<<<1, 1, 0, s>>>(p);
    CUDA_TRY(mark(3), "event");
    fixup_kernel<<<cblocks, kThreads, 0, s>>>(p);
    CUDA_TRY(mark(4), "event");
    uint64_t gblocks = (L.G + kThreads - 1) / kThreads;
    merge_kernel<<<(uint32_t)gblocks, kThreads, 0, s>>>(p);
    CUDA_TRY(mark(5), "event");
    CUDA_TRY(cudaGetLastError(), "launch");
    return RE_OK;
}

}  // extern "C"
