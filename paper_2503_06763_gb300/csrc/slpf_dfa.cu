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
constexpr uint32_t kDfaVersion = 2;
constexpr uint32_t kNoEntry = 0xFFFFu;          // a table entry no (column, byte) pair filled
constexpr uint32_t kMaxIds = 65535;            // ids fit u16 beside kNoEntry (tables of at most 32 MiB)
constexpr uint32_t kMaxInterval = 65536;       // exception offsets within a piece fit u16

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

struct Sections {
    size_t table, checkpoints, starts, exceptions, total;
};

Sections sections_of(uint32_t n_ids, uint64_t n_checkpoints, uint64_t n_exceptions) {
    Sections s{};
    s.table = align16(sizeof(re_slpf_dfa_header));
    s.checkpoints = s.table + align16((size_t)n_ids * 256 * 2);
    s.starts = s.checkpoints + align16(n_checkpoints * 2);
    s.exceptions = s.starts + align16((n_checkpoints + 1) * 8);
    s.total = s.exceptions + align16(n_exceptions * 4);
    return s;
}

uint32_t read_id(const void *cols, uint32_t cb, uint64_t r) {
    if (cb == 1) return static_cast<const uint8_t *>(cols)[r];
    if (cb == 2) return static_cast<const uint16_t *>(cols)[r];
    return static_cast<const uint32_t *>(cols)[r];
}

struct DecodeArgs {
    const uint16_t *table;       // [n_ids][256]
    const uint16_t *checkpoints; // [n_checkpoints]
    const uint64_t *starts;      // [n_checkpoints + 1]: first exception of each piece
    const uint32_t *exceptions;  // [n_exceptions]: offset in its piece << 16 | id, ascending
    const uint8_t *x;
    uint64_t n, n_checkpoints, n_exceptions;
    uint32_t n_ids, interval, col_bytes, table_in_smem;
    uint32_t vector;             // 16-byte text loads and column stores (aligned buffers, interval % 16 == 0)
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
    extern __shared__ __align__(16) uint16_t stab[];
    const uint16_t *table = a.table;
    if (a.table_in_smem) {
        const size_t entries = (size_t)a.n_ids * 256;
        for (size_t q = threadIdx.x; q < entries; q += blockDim.x) stab[q] = __ldg(a.table + q);
        __syncthreads();
        table = stab;
    }
    bool bad = false;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_checkpoints;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r0 = s * a.interval;
        const uint64_t r1 = min(r0 + a.interval, a.n + 1);
        uint32_t cur = __ldg(a.checkpoints + s);
        uint64_t e = __ldg(a.starts + s);
        const uint64_t e_end = min(__ldg(a.starts + s + 1), a.n_exceptions);
        uint32_t ev = e < e_end ? __ldg(a.exceptions + e) : 0u;
        while (e < e_end && (ev >> 16) == 0) {                 // none at the checkpoint column (a bad archive)
            ++e;
            ev = e < e_end ? __ldg(a.exceptions + e) : 0u;
        }
        uint64_t next = e < e_end ? r0 + (ev >> 16) : ~0ull;
        auto step = [&](uint64_t r, uint32_t byte) {             // column r from column r - 1 and byte x[r-1]
            if (r == next) {
                cur = ev & 0xFFFFu;
                ++e;
                ev = e < e_end ? __ldg(a.exceptions + e) : 0u;
                next = e < e_end ? r0 + (ev >> 16) : ~0ull;
            } else {
                const uint32_t v = cur < a.n_ids ? table[(size_t)cur * 256 + byte] : kNoEntry;
                if (v == kNoEntry) { bad = true; cur = 0; }   // not an archive of this text
                else cur = v;
            }
        };
        if (a.vector) {
            // 16 columns at a time: one 16-byte text load (bytes g .. g+15 serve
            // columns g+1 .. g+16) and the ids packed into 16-byte stores
            uint32_t prev = 0;                                   // x[g - 1]
            for (uint64_t g = r0; g < r1; g += 16) {
                const uint4 xv = load16(a.x, a.n, g);
                const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
                uint32_t ow[16];                                 // up to 16 ids of 4 bytes
#pragma unroll
                for (int q = 0; q < 16; ++q) ow[q] = 0;
                const uint64_t end = min(g + 16, r1);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const uint64_t r = g + u;
                    if (r < end) {
                        if (r > r0) step(r, u == 0 ? prev : (xw[(u - 1) >> 2] >> (8 * ((u - 1) & 3))) & 0xFFu);
                        if (a.col_bytes == 1) ow[u >> 2] |= (cur & 0xFFu) << (8 * (u & 3));
                        else if (a.col_bytes == 2) ow[u >> 1] |= (cur & 0xFFFFu) << (16 * (u & 1));
                        else ow[u] = cur;
                    }
                }
                prev = xw[3] >> 24;
                uint4 *dst = reinterpret_cast<uint4 *>(static_cast<uint8_t *>(a.out) + g * a.col_bytes);
                if (end == g + 16) {                             // a full group: col_bytes stores of 16 bytes
                    dst[0] = make_uint4(ow[0], ow[1], ow[2], ow[3]);
                    if (a.col_bytes >= 2) dst[1] = make_uint4(ow[4], ow[5], ow[6], ow[7]);
                    if (a.col_bytes == 4) {
                        dst[2] = make_uint4(ow[8], ow[9], ow[10], ow[11]);
                        dst[3] = make_uint4(ow[12], ow[13], ow[14], ow[15]);
                    }
                } else {                                         // the piece's last columns, one at a time
                    for (uint64_t q = g; q < end; ++q) {
                        const uint32_t u = (uint32_t)(q - g);
                        const uint32_t v = a.col_bytes == 1 ? (ow[u >> 2] >> (8 * (u & 3))) & 0xFFu
                                         : a.col_bytes == 2 ? (ow[u >> 1] >> (16 * (u & 1))) & 0xFFFFu
                                                            : ow[u];
                        put(a, q, v);
                    }
                }
            }
        } else {
            put(a, r0, cur);
            for (uint64_t r = r0 + 1; r < r1; ++r) {
                step(r, __ldg(a.x + r - 1));
                put(a, r, cur);
            }
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
    if (interval > kMaxInterval) { set_error("interval above 65536"); return RE_E_INVALID_ARG; }
    uint32_t max_id = 0;
    for (uint64_t r = 0; r <= len; ++r) max_id = std::max(max_id, read_id(cols, col_bytes, r));
    if (max_id >= kMaxIds) { set_error("column ids must be below 65535"); return RE_E_CAPACITY; }
    const uint32_t n_ids = max_id + 1;
    std::vector<uint16_t> table((size_t)n_ids * 256, (uint16_t)kNoEntry);
    std::vector<uint32_t> exc;                                  // offset in its piece << 16 | id
    const uint64_t n_cp = len / interval + 1;
    std::vector<uint64_t> starts(n_cp + 1, 0);
    for (uint64_t r = 1; r <= len; ++r) {
        const uint32_t prev = read_id(cols, col_bytes, r - 1), cur = read_id(cols, col_bytes, r);
        uint16_t &slot = table[(size_t)prev * 256 + text[r - 1]];
        if (slot == kNoEntry) slot = (uint16_t)cur;
        else if (slot != cur && r % interval != 0) {           // a checkpoint column needs no exception
            exc.push_back((uint32_t)((r % interval) << 16) | cur);
            ++starts[r / interval + 1];
        }
    }
    for (uint64_t p = 0; p < n_cp; ++p) starts[p + 1] += starts[p];   // exceptions before each piece
    const Sections sec = sections_of(n_ids, n_cp, exc.size());
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
    hdr.n_exceptions = exc.size();
    hdr.n_checkpoints = n_cp;
    std::memcpy(b, &hdr, sizeof(hdr));
    std::memcpy(b + sec.table, table.data(), table.size() * 2);
    uint16_t *cp = reinterpret_cast<uint16_t *>(b + sec.checkpoints);
    for (uint64_t s = 0; s < n_cp; ++s) cp[s] = (uint16_t)read_id(cols, col_bytes, s * interval);
    std::memcpy(b + sec.starts, starts.data(), starts.size() * 8);
    if (!exc.empty()) std::memcpy(b + sec.exceptions, exc.data(), exc.size() * 4);
    return RE_OK;
}

extern "C" re_status re_slpf_dfa_decode(const re_slpf_dfa_header *hdr, const void *d_archive, uint64_t archive_bytes,
                                        const uint8_t *d_text, void *d_cols, uint64_t cols_cap_bytes,
                                        uint32_t col_bytes, int32_t *d_status, re_stream stream) {
    if (!hdr || !d_archive || !d_cols || !d_status || (hdr->n && !d_text)) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (hdr->magic != kDfaMagic || hdr->version != kDfaVersion) { set_error("not an SLPF archive of this version"); return RE_E_INVALID_ARG; }
    if (col_bytes != 1 && col_bytes != 2 && col_bytes != 4) { set_error("col_bytes must be 1, 2 or 4"); return RE_E_INVALID_ARG; }
    if (hdr->n_ids == 0 || hdr->n_ids > kMaxIds || hdr->interval == 0 || hdr->interval > kMaxInterval ||
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
    a.table = reinterpret_cast<const uint16_t *>(b + sec.table);
    a.checkpoints = reinterpret_cast<const uint16_t *>(b + sec.checkpoints);
    a.starts = reinterpret_cast<const uint64_t *>(b + sec.starts);
    a.exceptions = reinterpret_cast<const uint32_t *>(b + sec.exceptions);
    a.x = d_text;
    a.n = hdr->n;
    a.n_checkpoints = hdr->n_checkpoints;
    a.n_exceptions = hdr->n_exceptions;
    a.n_ids = hdr->n_ids;
    a.interval = hdr->interval;
    a.col_bytes = col_bytes;
    a.out = d_cols;
    a.status = d_status;
    const size_t tab_bytes = (size_t)hdr->n_ids * 256 * 2;
    a.table_in_smem = tab_bytes <= 200 * 1024 ? 1u : 0u;
    a.vector = (hdr->interval % 16 == 0 && ((uintptr_t)d_text & 15) == 0 && ((uintptr_t)d_cols & 15) == 0) ? 1u : 0u;
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
