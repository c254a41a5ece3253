// Internal definitions shared by the host compiler (re_compile.cpp) and the
// device parse path (the .cu files).  Not part of the public ABI.
#pragma once

#include <stdint.h>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/slpf_parser.h"

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace slpf {

constexpr uint32_t kSub = 64;            // sub-chunk length L (bytes) of the checkpoints
constexpr uint32_t kUnknown = 0xFFFFFFFFu;  // checkpoint not produced by a converged reach run

// Hash of a segment bitset; used by the host to build and by the device to
// probe the state tables (bitset -> state id).
__host__ __device__ inline uint64_t bits_hash(const uint64_t *w, uint32_t W) {
    uint64_t h = 0x9E3779B97F4A7C15ull;
    for (uint32_t i = 0; i < W; ++i) {
        h ^= w[i] + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
        h *= 0xFF51AFD7ED558CCDull;
        h ^= h >> 33;
    }
    return h;
}

// Device tables of one compiled RE (all pointers are device pointers into
// one allocation owned by the handle).
struct DevTables {
    const uint8_t *cls;          // [256] byte -> class
    const uint32_t *fT;          // [nf][ncls] forward next state (0 = empty set)
    const uint32_t *bT;          // [nb][ncls] reverse next state
    const uint64_t *fBits;       // [nf][W] segment set of each forward state
    const uint64_t *bBits;       // [nb][W]
    const uint32_t *fHash;       // [fHashMask+1] forward state ids by bits_hash (0 = free)
    const uint32_t *bHash;       // [bHashMask+1]
    const uint32_t *fSlotStart;  // [ncls][ncls][msf] start state after the chunk's first byte
    const uint64_t *fSlotMask;   // [ncls][ncls][msf][W] segments whose end-letter is a key of the slot
    const uint32_t *fSlotCount;  // [ncls][ncls]
    const uint32_t *bSlotStart;  // [ncls][ncls][msb] start state after the chunk's last byte
    const uint64_t *bSlotMask;   // [ncls][ncls][msb][W] segments whose first symbol is a key
    const uint32_t *bSlotCount;  // [ncls][ncls]
    const uint8_t *fSlotOf;      // RE_COMPILE_DFA_STARTS only: [ncls][ncls][nf] forward slot of an
                                 // input state (0xFF: none); null for ME-DFA starts
    const uint8_t *bSlotOf;      // RE_COMPILE_DFA_STARTS_BWD only: [ncls][ncls][nb], the same backwards
    const uint32_t *pt;          // [nf][nb] dictionary index of B ∩ B̂ (DICT); pairs the
                                 // parse never produces hold 0xFFFFFFFF
    const uint32_t *f2, *b2;     // [n][ncls^2] two-byte tables (mid | end << 16), or null
    const uint8_t *fbyte, *bbyte;  // [n][256] next state by byte (not class), u8; null unless n <= 256
    const uint8_t *hirep;        // [128] byte b + 128 -> a byte below 128 of its class; null unless
                                 // every class holding a byte >= 128 holds one below (and fbyte is set)
    uint32_t fHashMask, bHashMask;
    uint32_t ncls, W, ell;
    uint32_t nf, nb, nfd, nbd;   // states incl. empty row 0; nfd/nbd = classic DFA states
    uint32_t msf, msb;           // slot capacity per class pair
    uint32_t fI, bF;             // state ids of I (forward) and F (reverse)
    uint32_t dict_size;
    const uint64_t *folseg;      // [ell][W] FolSeg of each segment (match extraction)
    const uint64_t *dict;        // [dict_size][W] DICT columns, entry d at row d-1 (match extraction)
};

// Host-side compiled RE.
struct Compiled {
    uint32_t ell = 0, W = 0, npos = 0, ncls = 0;
    std::vector<std::string> names;           // canonical segment order
    uint8_t cls[256];
    uint32_t nf = 0, nb = 0, nfd = 0, nbd = 0, msf = 0, msb = 0;
    std::vector<uint32_t> fT, bT;             // [n][ncls]
    std::vector<uint32_t> f2, b2;             // [n][ncls^2] two-byte tables (empty when too large)
    std::vector<uint8_t> fbyte, bbyte;        // [n][256] next state by byte (empty unless n <= 256)
    std::vector<uint8_t> hirep;               // [128] representative below 128 of byte b + 128 (or empty)
    std::vector<uint64_t> fBits, bBits;       // [n][W]
    std::vector<uint32_t> fHash, bHash;
    uint32_t fHashMask = 0, bHashMask = 0;
    std::vector<uint32_t> fSlotStart, fSlotCount, bSlotStart, bSlotCount;
    std::vector<uint64_t> fSlotMask, bSlotMask;
    std::vector<uint8_t> fSlotOf;             // RE_COMPILE_DFA_STARTS: [ncls][ncls][nf] slot of a state
    std::vector<uint8_t> bSlotOf;             // RE_COMPILE_DFA_STARTS_BWD: [ncls][ncls][nb] the same backwards
    std::vector<uint32_t> pt;                 // [nf][nb]
    std::vector<uint64_t> dict;               // [dict_size][W]
    uint32_t dict_size = 0;
    bool has_dict = false;
    std::vector<uint64_t> folseg;             // [ell][W] FolSeg(q) (Eq. folsegdef)
    std::vector<std::vector<int32_t>> parens; // per segment, in order: +k for k(, -k for )k
    uint32_t max_group = 0;                   // largest operator number
    bool inf_amb = false;                     // an iterated sub-RE derives the empty text
    uint32_t sample_limit = 0;                // per-segment symbol limit when sampling (App. A)
};

// Compile; returns RE_OK or an error with a message in err.
re_status compile_pattern(const char *pattern, size_t len, const re_compile_opts *opts,
                          Compiled &out, std::string &err);

void set_error(const std::string &msg);
re_status workspace_rule_bytes(const re_handle *h, uint64_t len, const re_parse_opts *opts, uint64_t *bytes);

}  // namespace slpf

struct re_handle {
    slpf::Compiled host;
    slpf::DevTables dev;
    void *d_alloc = nullptr;
    size_t d_bytes = 0;
    int device = 0;
    bool host_only = false;
    // choices of re_autotune: key = (floor(log2(len)), recognizer), value =
    // (chunk length, reach shape)
    std::mutex tune_lock;
    std::map<std::pair<int, int>, std::pair<uint32_t, uint32_t>> tuned;
};
