// SLPF compression (arXiv 2503.06763, App. C, "SLPF compression").
//
// App. C keeps the SLPF of a text as its initial column and a lookup table
// delta(C_{r-1}, x_r) = C_r over the columns that occur, and rebuilds the
// columns by running the table over the text.  A clean column also depends on
// bytes after r (only segments on a complete LST survive), so the table alone
// does not always give C_r; the archive here adds the positions where it does
// not (exceptions), and a checkpoint column every K positions so that the
// rebuild runs in independent pieces on the device (the evenly spaced
// columns App. C proposes for a parallel rebuild).
//
// Columns are column ids (DICT indices, or DENSE values below 65536).  The
// table row of id v and byte a holds the column that followed the first
// occurrence of (v, a) in the text.
//
// Encoding runs on the host (once per text, for storage); decoding is a
// kernel with one thread per K-column piece.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "re_internal.h"

namespace slpf {
namespace {

constexpr uint32_t kDfaMagic = 0x46504C53u;   // "SLPF"
constexpr uint32_t kDfaVersion = 1;
constexpr uint32_t kNoEntry = 0xFFFFFFFFu;
constexpr uint32_t kMaxIds = 65536;            // table rows (256 words each: at most 64 MiB)

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

struct Sections {
    size_t table, checkpoints, positions, ids, total;
};

Sections sections_of(uint32_t n_ids, uint64_t n_checkpoints, uint64_t n_exceptions) {
    Sections s{};
    s.table = align16(sizeof(re_slpf_dfa_header));
    s.checkpoints = s.table + align16((size_t)n_ids * 256 * 4);
    s.positions = s.checkpoints + align16(n_checkpoints * 4);
    s.ids = s.positions + align16(n_exceptions * 8);
    s.total = s.ids + align16(n_exceptions * 4);
    return s;
}

uint32_t read_id(const void *cols, uint32_t cb, uint64_t r) {
    if (cb == 1) return static_cast<const uint8_t *>(cols)[r];
    if (cb == 2) return static_cast<const uint16_t *>(cols)[r];
    return static_cast<const uint32_t *>(cols)[r];
}

struct DecodeArgs {
    const uint32_t *table;       // [n_ids][256]
    const uint32_t *checkpoints; // [n_checkpoints]
    const uint64_t *positions;   // [n_exceptions], ascending
    const uint32_t *ids;         // [n_exceptions]
    const uint8_t *x;
    uint64_t n, n_checkpoints, n_exceptions;
    uint32_t n_ids, interval, col_bytes, table_in_smem;
    void *out;
    int32_t *status;
};

__device__ __forceinline__ void put(const DecodeArgs &a, uint64_t r, uint32_t v) {
    if (a.col_bytes == 1) static_cast<uint8_t *>(a.out)[r] = (uint8_t)v;
    else if (a.col_bytes == 2) static_cast<uint16_t *>(a.out)[r] = (uint16_t)v;
    else static_cast<uint32_t *>(a.out)[r] = v;
}

// One thread per piece of K columns: the checkpoint, then the table (or the
// exception at that position) column after column.
__global__ void __launch_bounds__(256) slpf_dfa_decode_kernel(const __grid_constant__ DecodeArgs a) {
    extern __shared__ __align__(16) uint32_t stab[];
    const uint32_t *table = a.table;
    if (a.table_in_smem) {
        const size_t words = (size_t)a.n_ids * 256;
        for (size_t q = threadIdx.x; q < words; q += blockDim.x) stab[q] = __ldg(a.table + q);
        __syncthreads();
        table = stab;
    }
    bool bad = false;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_checkpoints;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r0 = s * a.interval;
        const uint64_t r1 = min(r0 + a.interval, a.n + 1);
        uint32_t cur = __ldg(a.checkpoints + s);
        put(a, r0, cur);
        uint64_t lo = 0, hi = a.n_exceptions;                 // first exception past r0
        while (lo < hi) {
            const uint64_t mid = (lo + hi) / 2;
            if (__ldg(a.positions + mid) <= r0) lo = mid + 1; else hi = mid;
        }
        uint64_t e = lo;
        uint64_t next = e < a.n_exceptions ? __ldg(a.positions + e) : ~0ull;
        for (uint64_t r = r0 + 1; r < r1; ++r) {
            if (r == next) {
                cur = __ldg(a.ids + e);
                ++e;
                next = e < a.n_exceptions ? __ldg(a.positions + e) : ~0ull;
            } else {
                const uint32_t v = cur < a.n_ids ? table[(size_t)cur * 256 + __ldg(a.x + r - 1)] : kNoEntry;
                if (v == kNoEntry) { bad = true; cur = 0; }   // not an archive of this text
                else cur = v;
            }
            put(a, r, cur);
        }
    }
    if (bad) atomicExch(a.status, RE_E_INTERNAL);
}

__global__ void slpf_dfa_status_kernel(int32_t *status) { *status = RE_OK; }

}  // namespace
}  // namespace slpf

using namespace slpf;

extern "C" re_status re_slpf_dfa_encode(const void *cols, uint32_t col_bytes, const uint8_t *text, uint64_t len,
                                        uint32_t interval, void *archive, uint64_t cap, uint64_t *size) {
    if (!cols || !size || (len && !text) || (cap && !archive)) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (col_bytes != 1 && col_bytes != 2 && col_bytes != 4) { set_error("col_bytes must be 1, 2 or 4"); return RE_E_INVALID_ARG; }
    if (interval == 0) { set_error("interval must be positive"); return RE_E_INVALID_ARG; }
    uint32_t max_id = 0;
    for (uint64_t r = 0; r <= len; ++r) max_id = std::max(max_id, read_id(cols, col_bytes, r));
    if (max_id >= kMaxIds) { set_error("column ids must be below 65536"); return RE_E_CAPACITY; }
    const uint32_t n_ids = max_id + 1;
    std::vector<uint32_t> table((size_t)n_ids * 256, kNoEntry);
    std::vector<uint64_t> pos;
    std::vector<uint32_t> ids;
    for (uint64_t r = 1; r <= len; ++r) {
        const uint32_t prev = read_id(cols, col_bytes, r - 1), cur = read_id(cols, col_bytes, r);
        uint32_t &slot = table[(size_t)prev * 256 + text[r - 1]];
        if (slot == kNoEntry) slot = cur;
        else if (slot != cur) { pos.push_back(r); ids.push_back(cur); }
    }
    const uint64_t n_cp = len / interval + 1;
    const Sections sec = sections_of(n_ids, n_cp, pos.size());
    *size = sec.total;
    if (cap < sec.total) { set_error("archive buffer too small (size reported)"); return RE_E_CAPACITY; }
    uint8_t *b = static_cast<uint8_t *>(archive);
    std::memset(b, 0, sec.total);
    re_slpf_dfa_header hdr{};
    hdr.magic = kDfaMagic;
    hdr.version = kDfaVersion;
    hdr.n = len;
    hdr.n_ids = n_ids;
    hdr.interval = interval;
    hdr.n_exceptions = pos.size();
    hdr.n_checkpoints = n_cp;
    std::memcpy(b, &hdr, sizeof(hdr));
    std::memcpy(b + sec.table, table.data(), table.size() * 4);
    uint32_t *cp = reinterpret_cast<uint32_t *>(b + sec.checkpoints);
    for (uint64_t s = 0; s < n_cp; ++s) cp[s] = read_id(cols, col_bytes, s * interval);
    if (!pos.empty()) {
        std::memcpy(b + sec.positions, pos.data(), pos.size() * 8);
        std::memcpy(b + sec.ids, ids.data(), ids.size() * 4);
    }
    return RE_OK;
}

extern "C" re_status re_slpf_dfa_decode(const re_slpf_dfa_header *hdr, const void *d_archive, uint64_t archive_bytes,
                                        const uint8_t *d_text, void *d_cols, uint64_t cols_cap_bytes,
                                        uint32_t col_bytes, int32_t *d_status, re_stream stream) {
    if (!hdr || !d_archive || !d_cols || !d_status || (hdr->n && !d_text)) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (hdr->magic != kDfaMagic || hdr->version != kDfaVersion) { set_error("not an SLPF archive of this version"); return RE_E_INVALID_ARG; }
    if (col_bytes != 1 && col_bytes != 2 && col_bytes != 4) { set_error("col_bytes must be 1, 2 or 4"); return RE_E_INVALID_ARG; }
    if (hdr->n_ids == 0 || hdr->n_ids > kMaxIds || hdr->interval == 0 ||
        hdr->n_checkpoints != hdr->n / hdr->interval + 1 || hdr->n_exceptions > hdr->n) {
        set_error("inconsistent archive header");
        return RE_E_INVALID_ARG;
    }
    if (col_bytes < 4 && hdr->n_ids > (1ull << (8 * col_bytes))) { set_error("column ids do not fit col_bytes"); return RE_E_INVALID_ARG; }
    const Sections sec = sections_of(hdr->n_ids, hdr->n_checkpoints, hdr->n_exceptions);
    if (archive_bytes < sec.total) { set_error("archive shorter than its header says"); return RE_E_INVALID_ARG; }
    if (cols_cap_bytes < (hdr->n + 1) * col_bytes) { set_error("column buffer too small"); return RE_E_CAPACITY; }
    if (((uintptr_t)d_archive & 15)) { set_error("archive must be 16-byte aligned"); return RE_E_INVALID_ARG; }
    const uint8_t *b = static_cast<const uint8_t *>(d_archive);
    DecodeArgs a{};
    a.table = reinterpret_cast<const uint32_t *>(b + sec.table);
    a.checkpoints = reinterpret_cast<const uint32_t *>(b + sec.checkpoints);
    a.positions = reinterpret_cast<const uint64_t *>(b + sec.positions);
    a.ids = reinterpret_cast<const uint32_t *>(b + sec.ids);
    a.x = d_text;
    a.n = hdr->n;
    a.n_checkpoints = hdr->n_checkpoints;
    a.n_exceptions = hdr->n_exceptions;
    a.n_ids = hdr->n_ids;
    a.interval = hdr->interval;
    a.col_bytes = col_bytes;
    a.out = d_cols;
    a.status = d_status;
    const size_t tab_bytes = (size_t)hdr->n_ids * 256 * 4;
    a.table_in_smem = tab_bytes <= 200 * 1024 ? 1u : 0u;
    const size_t smem = a.table_in_smem ? tab_bytes : 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(slpf_dfa_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) { set_error(std::string("decode attribute: ") + cudaGetErrorString(e)); return RE_E_CUDA; }
    }
    slpf_dfa_status_kernel<<<1, 1, 0, s>>>(d_status);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (hdr->n_checkpoints + 255) / 256;
    const uint32_t blocks = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 4));
    slpf_dfa_decode_kernel<<<blocks, 256, smem, s>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(std::string("decode launch: ") + cudaGetErrorString(e)); return RE_E_CUDA; }
    return RE_OK;
}
