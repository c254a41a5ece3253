// C ABI of include/slpf_parser.h: compile (host tables -> one device
// allocation), layout / workspace sizing, the parse launcher that enqueues
// reach -> join -> fix-up -> build & merge on the caller's stream, and the
// batch planner / launcher (many texts, one launch per phase and RE).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace slpf {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

void launch_flags_init(const Params &p, cudaStream_t s);

namespace {

re_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return RE_E_CUDA;
}
#define CUDA_TRY(expr, what)                               \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

constexpr size_t kSmemTablesMax = 120 * 1024;   // both u16 transition tables + class map
constexpr size_t kSmemPairMax = 48 * 1024;      // both two-byte tables + class map
constexpr size_t kSmemMergeMax = 190 * 1024;    // plus the dictionary pair table

int sm_count_of(int device) {
    static int cached[64] = {0};                        // read and written atomically: host threads share it
    if (device < 0 || device >= 64) return 152;
    int c = __atomic_load_n(&cached[device], __ATOMIC_RELAXED);
    if (!c) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
        c = v > 0 ? v : 152;
        __atomic_store_n(&cached[device], c, __ATOMIC_RELAXED);
    }
    return c;
}

// Chunk length k: one reach thread per chunk, about 2 resident warps per
// scheduler, chunks long enough that speculative runs meet early in them.
uint32_t choose_chunk(uint64_t n, int sms, const re_parse_opts *opts) {
    if (opts && opts->chunk_len) return opts->chunk_len;
    const uint64_t target = (uint64_t)sms * 384;
    uint64_t k = (n + target - 1) / target;
    k = (k + kSub - 1) / kSub * kSub;
    return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(k, 256), 1u << 20);
}

int length_bucket(uint64_t n) {
    int b = 0;
    while (n > 1) { n >>= 1; ++b; }
    return b;
}

// The chunk length re_autotune chose for this length bucket, or 0.
uint32_t tuned_chunk(re_handle *h, uint64_t n, const re_parse_opts *opts) {
    if (opts && opts->chunk_len) return 0;
    const int rec = (opts && (opts->flags & RE_PARSE_RECOGNIZE_ONLY)) ? 1 : 0;
    std::lock_guard<std::mutex> g(h->tune_lock);
    auto it = h->tuned.find({length_bucket(n), rec});
    return it == h->tuned.end() ? 0u : it->second.first;
}

// The reach shape re_autotune chose with that chunk length, or 0.
uint32_t tuned_shape(re_handle *h, uint64_t n, const re_parse_opts *opts) {
    const int rec = (opts && (opts->flags & RE_PARSE_RECOGNIZE_ONLY)) ? 1 : 0;
    std::lock_guard<std::mutex> g(h->tune_lock);
    auto it = h->tuned.find({length_bucket(n), rec});
    return it == h->tuned.end() ? 0u : it->second.second;
}

// Reach shapes this handle can run (bit v: shape v of RE_PARSE_REACH).
uint32_t shapes_of(const re_handle *h) {
    uint32_t m = (1u << 2) | (1u << 3) | (1u << 4);
    if (!h->host.fbyte.empty() && !h->host.bbyte.empty()) m |= 1u << 1;
    return m;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    // A function-local static is initialised once, and other threads wait for it.
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
    }();
    return fn;
}

// Text viewed as rows of full chunks (k bytes), one box = 32 chunks x 64
// bytes, SWIZZLE_64B to match the reach kernel's tile reads.
bool text_tensor_map(CUtensorMap &map, const uint8_t *d_text, uint32_t k, uint64_t rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn || rows < 32 || rows > 0x7FFFFFFFull || (k % 64) != 0) return false;   // int32 row coordinates
    const cuuint64_t dims[2] = {k, rows};
    const cuuint64_t strides[1] = {k};
    const cuuint32_t box[2] = {64u, 32u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = fn(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(d_text), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Output viewed as rows of one 64-column group (64 * cb bytes), one box per
// warp tile of 32 groups, swizzled to match the kernel's shared-memory tile.
bool output_tensor_map(CUtensorMap &map, void *d_cols, uint32_t cb, uint64_t rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn || rows == 0 || rows > 0x7FFFFFFFull || (cb != 1 && cb != 2)) return false;   // int32 row coordinates
    const cuuint64_t dims[2] = {64ull * cb, rows};
    const cuuint64_t strides[1] = {64ull * cb};
    const cuuint32_t box[2] = {64u * cb, 32u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = fn(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, d_cols, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, cb == 2 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

constexpr int kArrays = 26;

struct Layout {
    uint32_t k, c, S;
    uint64_t Gc;
    size_t off[kArrays];
    size_t total;
};

// The join runs as a scan when both classic DFAs fit byte state ids.
bool scan_join(const re_handle *h) { return h->host.nfd + 1 <= kScanStates && h->host.nbd + 1 <= kScanStates; }

uint32_t table_mode(const DevTables &t);

// Per-position states (mat): automata of at most 256 states per direction
// (the byte tables exist, and every classic-DFA state fits a byte).
bool mat_capable(const re_handle *h) {
    const Compiled &C = h->host;
    return !h->host_only && !C.fbyte.empty() && C.nf <= 256 && C.nb <= 256;
}
// Shapes whose reach kernels store the states: byte tables, or warp pairs
// with u8 class tables (not the pair layout of small class alphabets).
bool shape_stores_states(const re_handle *h, uint32_t v) {
    return v == 1 || ((v == 2 || v == 3) && table_mode(h->dev) == TM_SMEM);
}
bool mat_for(const re_handle *h, const re_parse_opts *opts) {
    return mat_capable(h) && !(opts && (opts->flags & RE_PARSE_RECOGNIZE_ONLY));
}

Layout layout_for(const re_handle *h, uint64_t n, uint32_t k, bool mat) {
    Layout L{};
    L.k = k;
    L.c = (uint32_t)((n + k - 1) / k);
    L.S = k / kSub;
    L.Gc = n / kSub + 1;
    const size_t c = L.c;
    const size_t sizes[kArrays] = {
        c * h->host.msf * 4, c * h->host.msb * 4,        // Rf, Rb
        (c + 1) * 4, (c + 1) * 4,                         // FJ, BJ
        (size_t)L.Gc * 4, (size_t)L.Gc * 4,               // FC, BC
        c * 4, c * 4, c * 4, c * 4,                       // fconv, bconv, fkind, bkind
        c * 4, c * 4,                                     // fnrec, bnrec
        c * 4, c * 4,                                     // fhit, bhit
        c * kRecBounds * 4, c * kRecBounds * 4,           // recFc, recBc
        c * kRecEntries * 8, c * kRecEntries * 8,         // recFe, recBe
        FLAG_COUNT * 4,
        scan_join(h) ? 2 * c * (h->host.nfd + 1) : 0,      // fTab
        scan_join(h) ? 2 * c * (h->host.nbd + 1) : 0,      // bTab
        scan_join(h) ? 2 * c * 4 : 0, scan_join(h) ? 2 * c * 4 : 0,   // fLink, bLink
        kScanWords * 4,
        mat ? (size_t)n + 1 + 128 : 0, mat ? (size_t)n + 1 + 128 : 0};   // FS, BS (one byte per column)
    size_t o = 0;
    for (int j = 0; j < kArrays; ++j) {
        L.off[j] = o;
        o += align256(sizes[j] ? sizes[j] : 4);
    }
    L.total = o;
    return L;
}

re_status resolve_kind(const re_handle *h, re_slpf_kind kind, re_slpf_kind &out, uint32_t &cb) {
    const Compiled &C = h->host;
    if (kind == RE_SLPF_AUTO) {
        if (C.ell <= 16) kind = RE_SLPF_DENSE;
        else if (C.has_dict) kind = RE_SLPF_DICT;
        else if (C.ell <= 64) kind = RE_SLPF_DENSE;
        else kind = RE_SLPF_PAIRS;                      // more than 64 segments and no dictionary
    }
    if (kind == RE_SLPF_DENSE) {
        if (C.ell > 64) { set_error("DENSE needs at most 64 segments"); return RE_E_CAPACITY; }
        cb = C.ell <= 8 ? 1 : C.ell <= 16 ? 2 : C.ell <= 32 ? 4 : 8;
    } else if (kind == RE_SLPF_DICT) {
        if (!C.has_dict) { set_error("this RE has no column dictionary (too many state pairs)"); return RE_E_CAPACITY; }
        cb = C.dict_size < 255 ? 1 : C.dict_size < 65535 ? 2 : 4;
    } else if (kind == RE_SLPF_PAIRS) {
        cb = (C.nf <= 65536 && C.nb <= 65536) ? 4 : 8;
    } else {
        set_error("unknown SLPF kind");
        return RE_E_INVALID_ARG;
    }
    out = kind;
    return RE_OK;
}

// True for device (or managed) memory; false for host memory the device
// reaches over the host link (pinned, mapped).
bool in_device_memory(const void *ptr) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Shared memory the merge's encoder table takes when staged.
size_t encoder_bytes(const DevTables &t, re_slpf_kind kind, uint32_t cb) {
    if (kind == RE_SLPF_PAIRS) return 0;
    return kind == RE_SLPF_DICT ? (size_t)t.nf * t.nb * cb : (size_t)(t.nf + t.nb) * 8;
}

uint32_t table_mode(const DevTables &t) {
    const bool fit16 = t.nf < 65536 && t.nb < 65536;
    if (t.f2 && t.b2 && tables_smem_bytes(t, TM_PAIR) <= kSmemPairMax) return TM_PAIR;
    if (fit16 && tables_smem_bytes(t, TM_SMEM) <= kSmemTablesMax) return TM_SMEM;
    return TM_GLOBAL;
}

// Point the workspace arrays of p at their places in w (layout L).
void carve(Params &p, const Layout &L, uint8_t *w) {
    p.w.Rf = (uint32_t *)(w + L.off[0]); p.w.Rb = (uint32_t *)(w + L.off[1]);
    p.w.FJ = (uint32_t *)(w + L.off[2]); p.w.BJ = (uint32_t *)(w + L.off[3]);
    p.w.FC = (uint32_t *)(w + L.off[4]); p.w.BC = (uint32_t *)(w + L.off[5]);
    p.w.fconv = (uint32_t *)(w + L.off[6]); p.w.bconv = (uint32_t *)(w + L.off[7]);
    p.w.fkind = (uint32_t *)(w + L.off[8]); p.w.bkind = (uint32_t *)(w + L.off[9]);
    p.w.fnrec = (uint32_t *)(w + L.off[10]); p.w.bnrec = (uint32_t *)(w + L.off[11]);
    p.w.fhit = (uint32_t *)(w + L.off[12]); p.w.bhit = (uint32_t *)(w + L.off[13]);
    p.w.recFc = (uint32_t *)(w + L.off[14]); p.w.recBc = (uint32_t *)(w + L.off[15]);
    p.w.recFe = (uint2 *)(w + L.off[16]); p.w.recBe = (uint2 *)(w + L.off[17]);
    p.w.flags = (int32_t *)(w + L.off[18]);
    p.w.fTab = w + L.off[19]; p.w.bTab = w + L.off[20];
    p.w.fLink = (uint32_t *)(w + L.off[21]); p.w.bLink = (uint32_t *)(w + L.off[22]);
    p.w.scan = (uint32_t *)(w + L.off[23]);
    p.w.FS = w + L.off[24]; p.w.BS = w + L.off[25];
}

// Check one output descriptor against the resolved encoding.
re_status check_output(const re_slpf *slpf, uint64_t len, uint32_t cb) {
    if (slpf->col_bytes != cb) { set_error("slpf->col_bytes does not match the layout"); return RE_E_INVALID_ARG; }
    if (!slpf->d_cols || slpf->cols_cap_bytes < (len + 1) * cb) { set_error("SLPF buffer too small"); return RE_E_CAPACITY; }
    if ((uintptr_t)slpf->d_cols & 15) { set_error("d_cols must be 16-byte aligned"); return RE_E_INVALID_ARG; }
    return RE_OK;
}

}  // namespace
}  // namespace slpf

using namespace slpf;

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
        st = RE_E_NOMEM;
        err = "host allocation failed during compile";
    }
    if (st != RE_OK) { set_error(err); delete h; return st; }
    Compiled &C = h->host;
    h->host_only = opts && (opts->flags & RE_COMPILE_HOST_ONLY);
    if (C.W > (uint32_t)kMaxW) { set_error("more than 4096 segments"); delete h; return RE_E_TOO_MANY_STATES; }
    if (C.msf > 32 || C.msb > 32) {
        set_error("more than 32 speculative starts for one pair of byte classes");
        delete h;
        return RE_E_TOO_MANY_STATES;
    }
    struct Piece { const void *src; size_t bytes; size_t off; };
    std::vector<Piece> pc;
    size_t total = 0;
    auto add = [&](const void *src, size_t bytes) {
        pc.push_back({src, bytes, total});
        total += align256(bytes ? bytes : 4);
        return pc.size() - 1;
    };
    const size_t i_cls = add(C.cls, 256);
    const size_t i_fT = add(C.fT.data(), C.fT.size() * 4), i_bT = add(C.bT.data(), C.bT.size() * 4);
    const size_t i_fB = add(C.fBits.data(), C.fBits.size() * 8), i_bB = add(C.bBits.data(), C.bBits.size() * 8);
    const size_t i_fH = add(C.fHash.data(), C.fHash.size() * 4), i_bH = add(C.bHash.data(), C.bHash.size() * 4);
    const size_t i_fSS = add(C.fSlotStart.data(), C.fSlotStart.size() * 4);
    const size_t i_fSM = add(C.fSlotMask.data(), C.fSlotMask.size() * 8);
    const size_t i_fSC = add(C.fSlotCount.data(), C.fSlotCount.size() * 4);
    const size_t i_bSS = add(C.bSlotStart.data(), C.bSlotStart.size() * 4);
    const size_t i_bSM = add(C.bSlotMask.data(), C.bSlotMask.size() * 8);
    const size_t i_bSC = add(C.bSlotCount.data(), C.bSlotCount.size() * 4);
    const size_t i_pt = add(C.pt.data(), C.pt.size() * 4);
    const size_t i_f2 = add(C.f2.data(), C.f2.size() * 4), i_b2 = add(C.b2.data(), C.b2.size() * 4);
    const size_t i_fs = add(C.folseg.data(), C.folseg.size() * 8), i_dc = add(C.dict.data(), C.dict.size() * 8);
    const size_t i_fso = add(C.fSlotOf.data(), C.fSlotOf.size());
    const size_t i_bso = add(C.bSlotOf.data(), C.bSlotOf.size());
    const size_t i_fby = add(C.fbyte.data(), C.fbyte.size()), i_bby = add(C.bbyte.data(), C.bbyte.size());
    const size_t i_hr = add(C.hirep.data(), C.hirep.size());
    DevTables &t = h->dev;
    t.fHashMask = C.fHashMask; t.bHashMask = C.bHashMask;
    t.ncls = C.ncls; t.W = C.W; t.ell = C.ell;
    t.nf = C.nf; t.nb = C.nb; t.nfd = C.nfd; t.nbd = C.nbd;
    t.msf = C.msf; t.msb = C.msb; t.fI = 1; t.bF = 1;
    t.dict_size = C.dict_size;
    if (h->host_only) { *out = h; return RE_OK; }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_alloc, total);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "re_compile: device tables"); }
    h->d_bytes = total;
    std::vector<uint8_t> staging(total, 0);
    for (auto &q : pc)
        if (q.bytes) std::memcpy(staging.data() + q.off, q.src, q.bytes);
    e = cudaMemcpy(h->d_alloc, staging.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(h->d_alloc); delete h; return cuda_fail(e, "re_compile: upload"); }
    uint8_t *b = (uint8_t *)h->d_alloc;
    t.cls = b + pc[i_cls].off;
    t.fT = (const uint32_t *)(b + pc[i_fT].off); t.bT = (const uint32_t *)(b + pc[i_bT].off);
    t.fBits = (const uint64_t *)(b + pc[i_fB].off); t.bBits = (const uint64_t *)(b + pc[i_bB].off);
    t.fHash = (const uint32_t *)(b + pc[i_fH].off); t.bHash = (const uint32_t *)(b + pc[i_bH].off);
    t.fSlotStart = (const uint32_t *)(b + pc[i_fSS].off); t.fSlotMask = (const uint64_t *)(b + pc[i_fSM].off);
    t.fSlotCount = (const uint32_t *)(b + pc[i_fSC].off);
    t.bSlotStart = (const uint32_t *)(b + pc[i_bSS].off); t.bSlotMask = (const uint64_t *)(b + pc[i_bSM].off);
    t.bSlotCount = (const uint32_t *)(b + pc[i_bSC].off);
    t.pt = (const uint32_t *)(b + pc[i_pt].off);
    t.fSlotOf = C.fSlotOf.empty() ? nullptr : (const uint8_t *)(b + pc[i_fso].off);
    t.bSlotOf = C.bSlotOf.empty() ? nullptr : (const uint8_t *)(b + pc[i_bso].off);
    t.f2 = C.f2.empty() ? nullptr : (const uint32_t *)(b + pc[i_f2].off);
    t.b2 = C.b2.empty() ? nullptr : (const uint32_t *)(b + pc[i_b2].off);
    t.folseg = (const uint64_t *)(b + pc[i_fs].off);
    t.fbyte = C.fbyte.empty() ? nullptr : b + pc[i_fby].off;
    t.bbyte = C.bbyte.empty() ? nullptr : b + pc[i_bby].off;
    t.hirep = C.hirep.empty() ? nullptr : b + pc[i_hr].off;
    t.dict = C.dict.empty() ? nullptr : (const uint64_t *)(b + pc[i_dc].off);
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
    info->inf_ambiguous = C.inf_amb ? 1u : 0u;
    info->sample_limit = C.sample_limit;
    info->ascii_rows = C.hirep.empty() ? 0u : 1u;
    info->reach_shapes = shapes_of(h);
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
    const re_status st = resolve_kind(h, kind, k, cb);
    if (st != RE_OK) return st;
    if (kind_out) *kind_out = k;
    if (col_bytes) *col_bytes = cb;
    if (bytes) *bytes = (len + 1) * cb;
    return RE_OK;
}

re_status re_workspace_size(const re_handle *h, uint64_t len, const re_parse_opts *opts, uint64_t *bytes) {
    if (!h || !bytes) { set_error("null argument"); return RE_E_INVALID_ARG; }
    const uint32_t kt = tuned_chunk(const_cast<re_handle *>(h), len, opts);
    const uint32_t k = kt ? kt : choose_chunk(len, sm_count_of(h->device), opts);
    if (k % kSub || k == 0) { set_error("chunk_len must be a positive multiple of 64"); return RE_E_INVALID_ARG; }
    *bytes = layout_for(h, len, k, mat_for(h, opts)).total;
    return RE_OK;
}

}  // extern "C"

namespace slpf {
// Workspace for the built-in chunk-length rule, ignoring any autotuned length:
// what re_parse falls back to when the workspace it is given cannot hold the
// tuned layout.
re_status workspace_rule_bytes(const re_handle *h, uint64_t len, const re_parse_opts *opts, uint64_t *bytes) {
    const uint32_t k = choose_chunk(len, sm_count_of(h->device), opts);
    if (k % kSub || k == 0) { set_error("chunk_len must be a positive multiple of 64"); return RE_E_INVALID_ARG; }
    *bytes = layout_for(h, len, k, mat_for(h, opts)).total;
    return RE_OK;
}
}  // namespace slpf

extern "C" {

}  // extern "C"

namespace slpf {
// A slice of a sharded text: its entry states (forward at its start,
// backward at its end; I and F for a whole text), and in map mode the
// device buffer of its maps and its SHARD_* flags.
struct SliceArgs {
    uint32_t fin = 1, bin = 1;
    uint32_t shard = 0;
    uint8_t *maps = nullptr;
};
re_status parse_impl(re_handle *h, const uint8_t *d_text, uint64_t len, re_stream stream, re_slpf *slpf,
                     void *d_workspace, uint64_t workspace_bytes, const re_parse_opts *opts, const SliceArgs &sa);
}  // namespace slpf

extern "C" {

re_status re_parse(re_handle *h, const uint8_t *d_text, uint64_t len, re_stream stream, re_slpf *slpf,
                   void *d_workspace, uint64_t workspace_bytes, const re_parse_opts *opts) {
    return parse_impl(h, d_text, len, stream, slpf, d_workspace, workspace_bytes, opts, SliceArgs{});
}

}  // extern "C"

re_status slpf::parse_impl(re_handle *h, const uint8_t *d_text, uint64_t len, re_stream stream, re_slpf *slpf,
                           void *d_workspace, uint64_t workspace_bytes, const re_parse_opts *opts,
                           const SliceArgs &sa) {
    const bool map_mode = sa.maps != nullptr;
    if (!h || !slpf || !slpf->d_status || (len && !d_text)) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (h->host_only) { set_error("handle was compiled with RE_COMPILE_HOST_ONLY"); return RE_E_INVALID_ARG; }
    if (len && ((uintptr_t)d_text & 15)) { set_error("d_text must be 16-byte aligned"); return RE_E_INVALID_ARG; }
    if (opts && (opts->flags & ~(RE_PARSE_RECOGNIZE_ONLY | RE_PARSE_TEST_STALL_JOIN | RE_PARSE_REACH_MASK))) {
        set_error("unknown parse flags");
        return RE_E_INVALID_ARG;
    }
    uint32_t shape = opts ? (opts->flags & RE_PARSE_REACH_MASK) >> 8 : 0u;
    if (shape > 4 || (shape && !(shapes_of(h) >> shape & 1))) {
        set_error("reach shape not available for this automaton");
        return RE_E_INVALID_ARG;
    }
    if (opts && opts->n_events && (opts->n_events != RE_PHASE_EVENTS || !opts->events)) {
        set_error("n_events must be 0 or RE_PHASE_EVENTS");
        return RE_E_INVALID_ARG;
    }
    const bool recognize = (opts && (opts->flags & RE_PARSE_RECOGNIZE_ONLY)) || map_mode;
    cudaEvent_t *ev = (opts && opts->n_events) ? (cudaEvent_t *)opts->events : nullptr;
    re_slpf_kind kind = RE_SLPF_DENSE;
    uint32_t cb = 1;
    if (map_mode && (!scan_join(h) || !len)) {
        set_error("slice maps need both classic DFAs below 256 states and a non-empty slice");
        return RE_E_INVALID_ARG;
    }
    if (!map_mode && (!recognize || slpf->d_cols)) {
        const re_status st = resolve_kind(h, slpf->kind, kind, cb);
        if (st != RE_OK) return st;
        const re_status so = check_output(slpf, len, cb);
        if (so != RE_OK) return so;
    }
    int dev_now = 0;
    cudaGetDevice(&dev_now);
    if (dev_now != h->device) { set_error("current device differs from the handle's device"); return RE_E_INVALID_ARG; }
    const int sms = sm_count_of(h->device);
    uint32_t k = choose_chunk(len, sms, opts);
    if (const uint32_t kt = tuned_chunk(h, len, opts)) {      // tuned length, if the workspace holds it
        if (!len || layout_for(h, len, kt, mat_for(h, opts)).total <= workspace_bytes) k = kt;
    }
    if (k % kSub || k == 0) { set_error("chunk_len must be a positive multiple of 64"); return RE_E_INVALID_ARG; }
    if (len / k >= 0xFFFFFFF0ull) { set_error("text too long for this chunk length"); return RE_E_INVALID_ARG; }
    const bool mat_ws = !map_mode && mat_for(h, opts);        // the workspace holds FS and BS
    const Layout L = layout_for(h, len, k, mat_ws);
    if (len && (!d_workspace || workspace_bytes < L.total || ((uintptr_t)d_workspace & 255))) {
        set_error("workspace missing, too small or not 256-byte aligned");
        return RE_E_CAPACITY;
    }
    slpf->n_cols = len + 1;
    cudaStream_t s = (cudaStream_t)stream;
    Params p{};
    p.t = h->dev;
    p.t.fI = sa.fin;                                          // a slice starts and ends in its entry states
    p.t.bF = sa.bin;
    p.shard = sa.shard;
    p.x = d_text; p.n = len; p.k = k; p.c = L.c; p.S = L.S; p.Gc = L.Gc;
    p.out = recognize ? nullptr : slpf->d_cols;
    p.col_bytes = cb; p.kind = kind; p.status = slpf->d_status;
    p.recognize = (recognize && !map_mode) ? 1u : 0u;          // map mode walks both directions
    p.scan = scan_join(h) ? 1u : 0u;
    p.scan_stall = (opts && (opts->flags & RE_PARSE_TEST_STALL_JOIN)) ? 1u : 0u;
    const DevTables &t = h->dev;
    p.tmode = table_mode(t);
    if (!shape) shape = tuned_shape(h, len, opts);            // chosen with the tuned chunk length
    if (!shape || !(shapes_of(h) >> shape & 1))
        shape = (shapes_of(h) >> 1 & 1) && p.tmode == TM_SMEM ? 1u : 2u;
    p.rvar = shape;
    p.rstages = shape == 3 ? 2u : 3u;
    const size_t tab = tables_smem_bytes(t, p.tmode);
    p.Gfast = len / kSub;
    alignas(64) CUtensorMap out_map;
    std::memset(&out_map, 0, sizeof(out_map));
    // TMA tensor stores only into device memory; columns may also go straight
    // to pinned host memory (plain stores over the host link).
    p.out_tma = (!recognize && in_device_memory(slpf->d_cols) && output_tensor_map(out_map, slpf->d_cols, cb, p.Gfast))
                    ? 1u : 0u;
    // Stage the encoder table (DICT pair table or DENSE state bitsets) in shared
    // memory when the merge's whole footprint (tables, stage, output tiles and
    // the table) still fits; otherwise it is read from global memory.
    // One-byte tables: build & merge over the classic-DFA rows and pairs, the
    // first half of each builder in registers, when that layout fits.
    if (!recognize && p.tmode == TM_SMEM) {
        Params q = p;
        q.merge_reg = 1;
        q.enc_in_smem = 1;
        if (merge_smem_bytes(q) <= kSmemMergeMax) { p.merge_reg = 1; p.enc_in_smem = 1; }
    }
    if (!recognize && !p.merge_reg && tab + merge_extra_smem(p) + encoder_bytes(t, kind, cb) <= kSmemMergeMax)
        p.enc_in_smem = 1;
    alignas(64) CUtensorMap text_map;
    std::memset(&text_map, 0, sizeof(text_map));
    p.c_full = (uint32_t)(len / k);
    p.text_tma = text_tensor_map(text_map, d_text, k, p.c_full) ? 1u : 0u;
    // Per-position states: the reach writes them, the fix-up fills the heads,
    // build & merge gathers (when the gather's encoder fits shared memory).
    alignas(64) StateMaps smaps;
    std::memset(&smaps, 0, sizeof(smaps));
    if (mat_ws && len && shape_stores_states(h, shape) && mat_gather_smem(p) <= kSmemMergeMax) {
        p.mat = 1;
        uint8_t *w = (uint8_t *)d_workspace;
        const bool maps = p.text_tma && text_tensor_map(smaps.f, w + L.off[24], k, p.c_full) &&
                          text_tensor_map(smaps.b, w + L.off[25], k, p.c_full);
        if (!maps) p.text_tma = 0;                            // state rows and text tiles use the same path
        p.state_tma = p.text_tma;
    }
    auto mark = [&](int j) -> cudaError_t { return ev ? cudaEventRecord(ev[j], s) : cudaSuccess; };
    if (len == 0) {
        CUDA_TRY(mark(0), "event");
        launch_empty(p, s);
        for (int j = 1; j < (int)RE_PHASE_EVENTS; ++j) CUDA_TRY(mark(j), "event");
        CUDA_TRY(cudaGetLastError(), "launch");
        return RE_OK;
    }
    carve(p, L, (uint8_t *)d_workspace);
    CUDA_TRY(mark(0), "event");
    launch_flags_init(p, s);
    if (!launch_reach(p, text_map, smaps, s, std::max(t.msf, p.recognize ? 1u : t.msb), sms)) {
        set_error("too many speculative starts");
        return RE_E_INTERNAL;
    }
    CUDA_TRY(mark(1), "event");
    if (map_mode) {                                           // the slice's maps, no columns
        if (!launch_shard_map(p, sa.maps, s, sms)) return cuda_fail(cudaGetLastError(), "slice map launch");
        for (int j = 2; j < (int)RE_PHASE_EVENTS; ++j) CUDA_TRY(mark(j), "event");
        CUDA_TRY(cudaGetLastError(), "launch");
        return RE_OK;
    }
    if (!launch_join(p, s, sms)) return cuda_fail(cudaGetLastError(), "join launch");
    CUDA_TRY(mark(2), "event");
    if (!recognize) {
        launch_fixup(p, s, sms);
        CUDA_TRY(mark(3), "event");
        launch_merge(p, out_map, s, sms);
    } else {
        CUDA_TRY(mark(3), "event");
    }
    CUDA_TRY(mark(4), "event");
    CUDA_TRY(cudaGetLastError(), "launch");
    return RE_OK;
}

// Time candidate chunk lengths around the rule's choice on the caller's text
// and keep the fastest for this handle and length bucket.
extern "C" re_status re_autotune(re_handle *h, const uint8_t *d_text, uint64_t len, re_slpf *slpf,
                                 void *d_workspace, uint64_t workspace_bytes, re_stream stream,
                                 const re_parse_opts *opts, uint32_t *chunk_len) {
    if (!h || !chunk_len || !len) { set_error("null argument or empty text"); return RE_E_INVALID_ARG; }
    if (opts && opts->chunk_len) { set_error("autotune chooses chunk_len: pass 0"); return RE_E_INVALID_ARG; }
    if (opts && opts->n_events) { set_error("autotune records its own events"); return RE_E_INVALID_ARG; }
    if (opts && (opts->flags & RE_PARSE_REACH_MASK)) { set_error("autotune chooses the reach shape"); return RE_E_INVALID_ARG; }
    const uint32_t k0 = choose_chunk(len, sm_count_of(h->device), nullptr);
    std::vector<uint32_t> cand;
    for (uint32_t num : {2u, 3u, 4u, 5u, 6u, 8u}) {            // k0 * num / 4, multiples of 64, >= 256
        uint64_t k = (uint64_t)k0 * num / 4;
        k = std::max<uint64_t>(256, (k + kSub - 1) / kSub * kSub);
        if (k > (1u << 20) || std::find(cand.begin(), cand.end(), (uint32_t)k) != cand.end()) continue;
        if (layout_for(h, len, (uint32_t)k, mat_for(h, opts)).total > workspace_bytes) continue;
        cand.push_back((uint32_t)k);
    }
    std::vector<uint32_t> shapes;                              // every reach shape this automaton can run
    for (uint32_t v = 1; v <= 4; ++v)
        if (shapes_of(h) >> v & 1) shapes.push_back(v);
    if (!h->host_only && (shapes_of(h) >> 1 & 1)) {
        // Whole rounds of tiles: with m tiles for every warp of the byte-table
        // reach, no warp idles while others walk a last tile.
        Params q{};
        q.t = h->dev;
        q.recognize = (opts && (opts->flags & RE_PARSE_RECOGNIZE_ONLY)) ? 1u : 0u;
        q.mat = mat_for(h, opts) ? 1u : 0u;
        const uint32_t ms = std::max(h->dev.msf, q.recognize ? 1u : h->dev.msb);
        const uint64_t warps = reach_byte8_warps(q, ms, sm_count_of(h->device));
        for (uint64_t m = 1; m <= 4 && warps; ++m) {
            uint64_t k = (len + 32 * warps * m - 1) / (32 * warps * m);
            k = (k + kSub - 1) / kSub * kSub;
            if (k < 256 || k > (1u << 20) || std::find(cand.begin(), cand.end(), (uint32_t)k) != cand.end()) continue;
            if (layout_for(h, len, (uint32_t)k, mat_for(h, opts)).total > workspace_bytes) continue;
            cand.push_back((uint32_t)k);
        }
    }
    if (cand.empty()) { set_error("workspace too small for any candidate chunk length"); return RE_E_CAPACITY; }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0), "event");
    CUDA_TRY(cudaEventCreate(&e1), "event");
    uint32_t best = cand[0], best_shape = shapes[0];
    float best_ms = 1e30f;
    re_status st = RE_OK;
    for (uint32_t v : shapes) {
        for (uint32_t k : cand) {
            re_parse_opts o = opts ? *opts : re_parse_opts{};
            o.chunk_len = k;
            o.flags = (o.flags & ~RE_PARSE_REACH_MASK) | RE_PARSE_REACH(v);
            o.n_events = 0;
            o.events = nullptr;
            float ms = 0.f;
            for (int rep = 0; rep < 3 && st == RE_OK; ++rep) {   // one warm-up, two timed
                cudaEventRecord(e0, s);
                st = re_parse(h, d_text, len, stream, slpf, d_workspace, workspace_bytes, &o);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) { st = cuda_fail(cudaGetLastError(), "autotune"); break; }
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep) ms += t;
            }
            if (st != RE_OK) break;
            if (ms < best_ms) { best_ms = ms; best = k; best_shape = v; }
        }
        if (st != RE_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RE_OK) return st;
    const int rec = (opts && (opts->flags & RE_PARSE_RECOGNIZE_ONLY)) ? 1 : 0;
    {
        std::lock_guard<std::mutex> g(h->tune_lock);
        h->tuned[{length_bucket(len), rec}] = {best, best_shape};
    }
    *chunk_len = best;
    return RE_OK;
}

extern "C" re_status re_tuned(const re_handle *h, uint64_t len, uint32_t flags, uint32_t *chunk_len,
                              uint32_t *shape) {
    if (!h || !chunk_len || !shape) { set_error("null argument"); return RE_E_INVALID_ARG; }
    re_parse_opts o{};
    o.flags = flags & RE_PARSE_RECOGNIZE_ONLY;
    *chunk_len = tuned_chunk(const_cast<re_handle *>(h), len, &o);
    *shape = tuned_shape(const_cast<re_handle *>(h), len, &o);
    return RE_OK;
}

extern "C" re_status re_parse_host(re_handle *h, const uint8_t *text, uint64_t len, void *host_cols,
                                   int32_t *host_status, uint8_t *d_text, re_slpf *slpf, void *d_workspace,
                                   uint64_t workspace_bytes, re_stream stream, const re_parse_opts *opts) {
    const bool recognize = opts && (opts->flags & RE_PARSE_RECOGNIZE_ONLY);
    if (!h || !slpf || !host_status || (len && (!text || !d_text)) || (!recognize && !host_cols)) {
        set_error("null argument");
        return RE_E_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (len) CUDA_TRY(cudaMemcpyAsync(d_text, text, len, cudaMemcpyHostToDevice, s), "text to device");
    // The columns come back by a copy after the parse: on this machine the
    // copy engines move them about 4x faster than the kernels' own stores
    // into pinned host memory would.
    const re_status st = re_parse(h, d_text, len, stream, slpf, d_workspace, workspace_bytes, opts);
    if (st != RE_OK) return st;
    if (!recognize)
        CUDA_TRY(cudaMemcpyAsync(host_cols, slpf->d_cols, (len + 1) * slpf->col_bytes, cudaMemcpyDeviceToHost, s),
                 "columns to host");
    CUDA_TRY(cudaMemcpyAsync(host_status, slpf->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
             "status to host");
    return RE_OK;
}

// ------------------------------------------------------------------ match extraction
extern "C" re_status re_match_workspace_size(const re_handle *h, uint64_t len, uint64_t *bytes) {
    if (!h || !bytes) { set_error("null argument"); return RE_E_INVALID_ARG; }
    *bytes = match_workspace_bytes(len);
    return RE_OK;
}

extern "C" re_status re_matches(re_handle *h, const re_slpf *slpf, uint64_t len, uint32_t group, uint64_t *d_pairs,
                                uint64_t cap_pairs, uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes,
                                re_stream stream) {
    if (!h || !slpf || !d_count || !slpf->d_cols || !slpf->d_status || (cap_pairs && !d_pairs)) {
        set_error("null argument");
        return RE_E_INVALID_ARG;
    }
    if (h->host_only) { set_error("handle was compiled with RE_COMPILE_HOST_ONLY"); return RE_E_INVALID_ARG; }
    const Compiled &C = h->host;
    re_slpf_kind kind;
    uint32_t cb;
    const re_status st = resolve_kind(h, slpf->kind, kind, cb);
    if (st != RE_OK) return st;
    if (slpf->kind == RE_SLPF_AUTO || slpf->col_bytes != cb || slpf->cols_cap_bytes < (len + 1) * cb) {
        set_error("slpf does not describe the columns of a text of this length");
        return RE_E_INVALID_ARG;
    }
    if (C.W > (uint32_t)kMatchW) { set_error("match extraction supports at most 512 segments"); return RE_E_CAPACITY; }
    if (kind == RE_SLPF_DICT && !h->dev.dict) { set_error("no dictionary on the device"); return RE_E_INTERNAL; }
    MatchArgs a{};
    bool is_group = false;
    for (uint32_t q = 0; q < C.ell; ++q) {
        std::vector<int> kp;                                 // +1: k(, -1: )k, in order
        for (int32_t v : C.parens[q])
            if ((uint32_t)(v < 0 ? -v : v) == group) kp.push_back(v > 0 ? 1 : -1);
        const uint64_t bit = 1ull << (q & 63);
        const uint32_t w = q >> 6;
        if (kp.empty()) { a.none[w] |= bit; continue; }
        is_group = true;
        if (kp.back() == 1) a.open[w] |= bit;
        if (kp.front() == -1) a.close_first[w] |= bit;
        for (size_t x = 0; x < kp.size(); ++x)
            if (kp[x] == 1 && std::find(kp.begin() + x + 1, kp.end(), -1) != kp.end()) { a.whole[w] |= bit; break; }
    }
    if (!group || !is_group) { set_error("no group with this number (an operator node of the numbered RE)"); return RE_E_INVALID_ARG; }
    if (!d_workspace || workspace_bytes < match_workspace_bytes(len) || ((uintptr_t)d_workspace & 255)) {
        set_error("workspace missing, too small or not 256-byte aligned");
        return RE_E_CAPACITY;
    }
    int dev_now = 0;
    cudaGetDevice(&dev_now);
    if (dev_now != h->device) { set_error("current device differs from the handle's device"); return RE_E_INVALID_ARG; }
    a.cols = slpf->d_cols;
    a.col_bytes = cb;
    a.kind = kind;
    a.W = C.W;
    a.n = len;
    a.folseg = h->dev.folseg;
    a.dict = h->dev.dict;
    a.fbits = h->dev.fBits;
    a.bbits = h->dev.bBits;
    a.status = slpf->d_status;
    a.pairs = d_pairs;
    a.cap = cap_pairs;
    a.count = d_count;
    launch_matches(a, d_workspace, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError(), "match launch");
    return RE_OK;
}

// ------------------------------------------------------------------ batch
namespace slpf {
// Pinned descriptor buffers of batch plans, kept for reuse: pinning host pages
// costs far more than a small batch's whole parse, and a serving loop plans a
// batch per launch.  Buffers are powers of two of at least 4 KiB; at most 64
// are kept.
struct PinnedPool {
    std::mutex m;
    std::multimap<size_t, void *> free;
    ~PinnedPool() {
        for (auto &kv : free) cudaFreeHost(kv.second);
    }
};
PinnedPool &pinned_pool() {
    static PinnedPool *pool = new PinnedPool();                 // never destroyed: outlives every plan
    return *pool;
}
size_t pinned_size(size_t bytes) {
    size_t s = 4096;
    while (s < bytes) s <<= 1;
    return s;
}
cudaError_t pinned_take(size_t bytes, uint8_t **out) {
    const size_t sz = pinned_size(bytes);
    PinnedPool &pool = pinned_pool();
    {
        std::lock_guard<std::mutex> g(pool.m);
        auto it = pool.free.find(sz);
        if (it != pool.free.end()) {
            *out = static_cast<uint8_t *>(it->second);
            pool.free.erase(it);
            return cudaSuccess;
        }
    }
    return cudaHostAlloc((void **)out, sz, cudaHostAllocDefault);
}
void pinned_give(uint8_t *buf, size_t bytes) {
    if (!buf) return;
    PinnedPool &pool = pinned_pool();
    {
        std::lock_guard<std::mutex> g(pool.m);
        if (pool.free.size() < 64) {
            pool.free.emplace(pinned_size(bytes), buf);
            return;
        }
    }
    cudaFreeHost(buf);
}
}  // namespace slpf

// A planned batch: per text its group (compiled RE), chunk length and
// workspace layout; per group the table mode, encoding and unit counts.  The
// descriptor area at the start of the workspace holds every text's Params,
// the per-group prefix sums and work counters; it is written from a pinned
// host copy by re_parse_batch and only read by the kernels afterwards.
struct re_batch {
    struct Text {
        uint32_t group = 0, slot = 0;   // slot: index of its Params in the descriptor area
        uint64_t len = 0;
        uint32_t k = 0;
        Layout L{};
        size_t ws_off = 0;
    };
    struct Group {
        re_handle *h = nullptr;
        uint32_t tmode = 0, ms = 0, enc_in_smem = 0, cb = 1;
        bool mat = false;               // per-position states (byte-table reach, fix-up of heads, gather)
        re_slpf_kind kind = RE_SLPF_DENSE;
        std::vector<uint32_t> members;  // caller indices, longest chunks first
        size_t params_off = 0, cbase_off = 0, rbase_off = 0, mbase_off = 0;
        uint64_t chunks = 0, n_reach = 0, n_merge = 0;
    };
    int device = 0, sms = 152;
    bool recognize = false;
    std::vector<Text> texts;
    std::vector<Group> groups;
    size_t queue_off = 0, maps_off = 0, desc_bytes = 0, total = 0;
    uint8_t *pinned = nullptr;
    cudaEvent_t uploaded = nullptr;
    bool pending = false;
    uint8_t *d_ws = nullptr;
    // Groups are independent: they run on a few streams of their own, forked
    // from and joined back into the caller's stream by events (also inside a
    // CUDA-graph capture), so one group's small join and fix-up launches
    // overlap another's reach and merge.
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    ~re_batch() {
        for (cudaStream_t st : aux) cudaStreamDestroy(st);
        for (cudaEvent_t ev : done) cudaEventDestroy(ev);
        if (fork) cudaEventDestroy(fork);
        if (uploaded) cudaEventDestroy(uploaded);
        slpf::pinned_give(pinned, desc_bytes);
    }
};

namespace slpf {
namespace {

// Chunk length of one text of a batch: the single-text rule applied to the
// group's total bytes (one reach lane per chunk, about one wave of lanes for
// the whole group), but short enough that the text spans a warp tile of 32
// chunks where it can.
uint32_t batch_chunk(uint64_t len, uint64_t group_bytes, int sms, const re_parse_opts *opts) {
    if (opts && opts->chunk_len) return opts->chunk_len;
    const uint32_t kg = choose_chunk(group_bytes, sms, nullptr);
    uint64_t kt = (len + 31) / 32;
    kt = (kt + kSub - 1) / kSub * kSub;
    return (uint32_t)std::max<uint64_t>(256, std::min<uint64_t>(kg, kt));
}

Params group_like(const re_batch::Group &g, bool recognize) {
    Params q{};
    q.t = g.h->dev;
    q.tmode = g.tmode;
    q.kind = g.kind;
    q.col_bytes = g.cb;
    q.recognize = recognize ? 1u : 0u;
    q.enc_in_smem = g.enc_in_smem;
    q.mat = g.mat ? 1u : 0u;
    return q;
}

re_status batch_run(re_batch *b, cudaStream_t s0) {
    uint8_t *w = b->d_ws;
    launch_batch_init(reinterpret_cast<const Params *>(w), (uint32_t)b->texts.size(),
                      reinterpret_cast<uint32_t *>(w + b->queue_off), (uint32_t)b->groups.size() * kQueues, s0);
    const size_t na = b->aux.size();
    if (na) {
        CUDA_TRY(cudaEventRecord(b->fork, s0), "batch fork");
        for (cudaStream_t a : b->aux) CUDA_TRY(cudaStreamWaitEvent(a, b->fork, 0), "batch fork");
    }
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const re_batch::Group &g = b->groups[gi];
        const cudaStream_t s = na ? b->aux[gi % na] : s0;
        BatchGroup bg{};
        bg.t = g.h->dev;
        bg.texts = reinterpret_cast<const Params *>(w + g.params_off);
        bg.chunk_base = reinterpret_cast<const uint64_t *>(w + g.cbase_off);
        bg.rtile_base = reinterpret_cast<const uint64_t *>(w + g.rbase_off);
        bg.mtile_base = reinterpret_cast<const uint64_t *>(w + g.mbase_off);
        bg.queue = reinterpret_cast<uint32_t *>(w + b->queue_off) + gi * kQueues;
        bg.chunks = g.chunks; bg.n_reach = g.n_reach; bg.n_merge = g.n_merge;
        bg.nt = (uint32_t)g.members.size();
        bg.recognize = b->recognize ? 1u : 0u;
        if (g.mat) {
            if (g.n_reach && !launch_reach_batch_byte8(bg, g.ms, s, b->sms)) {
                set_error("too many speculative starts");
                return RE_E_INTERNAL;
            }
            launch_join_batch(bg, s);
            launch_fixup_mat_batch(bg, s, b->sms);
            launch_gather_batch(bg, group_like(g, b->recognize), s, b->sms);
            continue;
        }
        if (g.n_reach && !launch_reach_batch(bg, g.tmode, g.ms, s, b->sms)) {
            set_error("too many speculative starts");
            return RE_E_INTERNAL;
        }
        launch_join_batch(bg, s);
        launch_fixup_batch(bg, g.tmode, s, b->sms);
        launch_merge_batch(bg, group_like(g, b->recognize), s, b->sms);
    }
    for (size_t a = 0; a < na; ++a) {                         // join: the caller's stream waits for every group
        CUDA_TRY(cudaEventRecord(b->done[a], b->aux[a]), "batch join");
        CUDA_TRY(cudaStreamWaitEvent(s0, b->done[a], 0), "batch join");
    }
    CUDA_TRY(cudaGetLastError(), "batch launch");
    return RE_OK;
}

}  // namespace
}  // namespace slpf

extern "C" {

re_status re_batch_plan(re_handle *const *hs, const uint64_t *lens, uint32_t count, const re_parse_opts *opts,
                        re_batch **out) {
    if (!out || (count && (!hs || !lens))) { set_error("null argument"); return RE_E_INVALID_ARG; }
    *out = nullptr;
    if (opts && (opts->flags & ~RE_PARSE_RECOGNIZE_ONLY)) { set_error("unknown parse flags"); return RE_E_INVALID_ARG; }
    if (opts && opts->n_events) { set_error("batch parses record no phase events"); return RE_E_INVALID_ARG; }
    if (opts && opts->chunk_len && opts->chunk_len % kSub) {
        set_error("chunk_len must be a positive multiple of 64");
        return RE_E_INVALID_ARG;
    }
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    std::unique_ptr<re_batch> b(new (std::nothrow) re_batch());
    if (!b) { set_error("host allocation failed"); return RE_E_NOMEM; }
    b->device = dev;
    b->sms = sm_count_of(dev);
    b->recognize = opts && (opts->flags & RE_PARSE_RECOGNIZE_ONLY);
    b->texts.resize(count);
    std::map<re_handle *, uint32_t> gid;
    std::vector<uint64_t> gbytes;
    for (uint32_t j = 0; j < count; ++j) {
        re_handle *h = hs[j];
        if (!h) { set_error("null handle in batch"); return RE_E_INVALID_ARG; }
        if (h->host_only) { set_error("handle was compiled with RE_COMPILE_HOST_ONLY"); return RE_E_INVALID_ARG; }
        if (h->device != dev) { set_error("current device differs from a handle's device"); return RE_E_INVALID_ARG; }
        auto it = gid.find(h);
        if (it == gid.end()) {
            it = gid.emplace(h, (uint32_t)b->groups.size()).first;
            re_batch::Group g;
            g.h = h;
            g.tmode = table_mode(h->dev);
            g.ms = std::max(h->host.msf, b->recognize ? 1u : h->host.msb);
            // per-position states where the single-text parse would use them (byte
            // tables for both automata) and the slots fit the byte-table reach
            g.mat = !b->recognize && mat_capable(h) && g.ms <= 32;
            if (!b->recognize) {
                const re_status st = resolve_kind(h, opts ? opts->kind : RE_SLPF_AUTO, g.kind, g.cb);
                if (st != RE_OK) return st;
            }
            b->groups.push_back(std::move(g));
            gbytes.push_back(0);
        }
        b->texts[j].group = it->second;
        b->texts[j].len = lens[j];
        b->groups[it->second].members.push_back(j);
        gbytes[it->second] += lens[j];
    }
    // chunk lengths, then members longest chunks first
    for (uint32_t j = 0; j < count; ++j) {
        re_batch::Text &t = b->texts[j];
        t.k = batch_chunk(t.len, gbytes[t.group], b->sms, opts);
        if (t.len / t.k >= 0xFFFFFFF0ull) { set_error("text too long for this chunk length"); return RE_E_INVALID_ARG; }
        if (t.len) t.L = layout_for(b->groups[t.group].h, t.len, t.k, b->groups[t.group].mat);
    }
    uint32_t slot = 0;                                       // every text's Params, group after group
    for (auto &g : b->groups) {
        std::stable_sort(g.members.begin(), g.members.end(), [&](uint32_t a, uint32_t c) {
            return b->texts[a].k > b->texts[c].k;
        });
        g.params_off = (size_t)slot * sizeof(Params);
        for (uint32_t j : g.members) b->texts[j].slot = slot++;
    }
    size_t off = align256((size_t)count * sizeof(Params));
    b->maps_off = off;                                       // per text: text, FS and BS tensor maps
    off = align256(off + (size_t)count * 3 * sizeof(CUtensorMap));
    for (auto &g : b->groups) {
        const size_t arr = (g.members.size() + 1) * sizeof(uint64_t);
        g.cbase_off = off; off = align256(off + arr);
        g.rbase_off = off; off = align256(off + arr);
        g.mbase_off = off; off = align256(off + arr);
        Params q = group_like(g, b->recognize);
        const size_t tab = tables_smem_bytes(g.h->dev, g.tmode);
        if (!b->recognize && tab + merge_extra_smem(q) + encoder_bytes(g.h->dev, g.kind, g.cb) <= kSmemMergeMax)
            g.enc_in_smem = 1;
    }
    b->queue_off = off;
    off = align256(off + b->groups.size() * kQueues * sizeof(uint32_t));
    b->desc_bytes = off;
    for (uint32_t j = 0; j < count; ++j) {
        re_batch::Text &t = b->texts[j];
        if (!t.len) continue;
        t.ws_off = off;
        off += align256(t.L.total);
    }
    b->total = std::max<size_t>(off, 256);
    CUDA_TRY(pinned_take(b->desc_bytes, &b->pinned), "batch descriptor buffer");
    std::memset(b->pinned, 0, b->desc_bytes);
    for (auto &g : b->groups) {                              // prefix sums of the units of each kind
        uint64_t *cb = reinterpret_cast<uint64_t *>(b->pinned + g.cbase_off);
        uint64_t *rb = reinterpret_cast<uint64_t *>(b->pinned + g.rbase_off);
        uint64_t *mb = reinterpret_cast<uint64_t *>(b->pinned + g.mbase_off);
        cb[0] = rb[0] = mb[0] = 0;
        for (size_t m = 0; m < g.members.size(); ++m) {
            const re_batch::Text &t = b->texts[g.members[m]];
            const uint64_t c = t.len ? t.L.c : 0;
            const uint64_t groups = (t.len && !b->recognize) ? t.L.Gc : 0;
            cb[m + 1] = cb[m] + c;
            rb[m + 1] = rb[m] + (c + 31) / 32;
            mb[m + 1] = mb[m] + (groups + 31) / 32;
        }
        g.chunks = cb[g.members.size()];
        g.n_reach = rb[g.members.size()];
        g.n_merge = mb[g.members.size()];
        if (g.n_reach >= 0xFFFFFFFFull || g.n_merge >= 0xFFFFFFFFull) {
            set_error("batch too large for one launch per phase");
            return RE_E_INVALID_ARG;
        }
    }
    CUDA_TRY(cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming), "batch event");
    uint64_t all_bytes = 0;
    for (uint64_t g : gbytes) all_bytes += g;
    if (b->groups.size() > 1 && all_bytes >= (64ull << 20)) {   // small batches: no stream set-up cost
        const size_t na = std::min<size_t>(4, b->groups.size());
        CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "batch event");
        for (size_t a = 0; a < na; ++a) {
            cudaStream_t st;
            cudaEvent_t ev;
            CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "batch stream");
            b->aux.push_back(st);
            CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "batch event");
            b->done.push_back(ev);
        }
    }
    *out = b.release();
    return RE_OK;
}

re_status re_batch_workspace_size(const re_batch *b, uint64_t *bytes) {
    if (!b || !bytes) { set_error("null argument"); return RE_E_INVALID_ARG; }
    *bytes = b->total;
    return RE_OK;
}

re_status re_batch_chunk_len(const re_batch *b, uint32_t j, uint32_t *k) {
    if (!b || !k || j >= b->texts.size()) { set_error("bad argument"); return RE_E_INVALID_ARG; }
    *k = b->texts[j].k;
    return RE_OK;
}

re_status re_parse_batch(re_batch *b, const uint8_t *const *d_texts, re_slpf *outs, void *d_workspace,
                         uint64_t workspace_bytes, re_stream stream) {
    const uint32_t count = b ? (uint32_t)b->texts.size() : 0;
    if (!b || (count && (!d_texts || !outs))) { set_error("null argument"); return RE_E_INVALID_ARG; }
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != b->device) { set_error("current device differs from the batch's device"); return RE_E_INVALID_ARG; }
    if (!d_workspace || workspace_bytes < b->total || ((uintptr_t)d_workspace & 255)) {
        set_error("workspace missing, too small or not 256-byte aligned");
        return RE_E_CAPACITY;
    }
    for (uint32_t j = 0; j < count; ++j) {
        const re_batch::Text &t = b->texts[j];
        const re_batch::Group &g = b->groups[t.group];
        if (!outs[j].d_status || (t.len && !d_texts[j])) { set_error("null text or status in batch"); return RE_E_INVALID_ARG; }
        if (t.len && ((uintptr_t)d_texts[j] & 15)) { set_error("batch text must be 16-byte aligned"); return RE_E_INVALID_ARG; }
        if (!b->recognize) {
            if (outs[j].kind != g.kind) { set_error("slpf->kind differs from the planned encoding"); return RE_E_INVALID_ARG; }
            const re_status so = check_output(&outs[j], t.len, g.cb);
            if (so != RE_OK) return so;
        }
    }
    if (b->pending) CUDA_TRY(cudaEventSynchronize(b->uploaded), "batch descriptor upload");
    uint8_t *w = (uint8_t *)d_workspace;
    for (uint32_t j = 0; j < count; ++j) {
        const re_batch::Text &t = b->texts[j];
        const re_batch::Group &g = b->groups[t.group];
        Params p = group_like(g, b->recognize);
        p.x = d_texts[j];
        p.n = t.len;
        p.k = t.k;
        p.c = t.len ? t.L.c : 0;
        p.S = t.k / kSub;
        p.Gc = t.len / kSub + 1;
        p.out = b->recognize ? nullptr : outs[j].d_cols;
        p.status = outs[j].d_status;
        p.Gfast = t.len / kSub;
        p.c_full = (uint32_t)(t.len / t.k);
        if (t.len) carve(p, t.L, w + t.ws_off);
        if (g.mat && t.len) {                                // TMA for full tiles: maps in the descriptor area
            CUtensorMap *hm = reinterpret_cast<CUtensorMap *>(b->pinned + b->maps_off) + 3 * (size_t)t.slot;
            uint8_t *ws = w + t.ws_off;
            p.text_tma = text_tensor_map(hm[0], d_texts[j], t.k, p.c_full) &&
                         text_tensor_map(hm[1], ws + t.L.off[24], t.k, p.c_full) &&
                         text_tensor_map(hm[2], ws + t.L.off[25], t.k, p.c_full) ? 1u : 0u;
            p.state_tma = p.text_tma;
            p.tmaps = reinterpret_cast<const CUtensorMap *>(w + b->maps_off) + 3 * (size_t)t.slot;
        }
        std::memcpy(b->pinned + (size_t)t.slot * sizeof(Params), &p, sizeof(Params));
        outs[j].n_cols = t.len + 1;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(w, b->pinned, b->desc_bytes, cudaMemcpyHostToDevice, s), "batch descriptor upload");
    CUDA_TRY(cudaEventRecord(b->uploaded, s), "batch event");
    b->pending = true;
    b->d_ws = w;
    return batch_run(b, s);
}

re_status re_batch_run(re_batch *b, re_stream stream) {
    if (!b) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (!b->d_ws) { set_error("batch not bound: call re_parse_batch first"); return RE_E_INVALID_ARG; }
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != b->device) { set_error("current device differs from the batch's device"); return RE_E_INVALID_ARG; }
    return batch_run(b, (cudaStream_t)stream);
}

void re_batch_free(re_batch *b) {
    if (!b) return;
    if (b->pending) cudaEventSynchronize(b->uploaded);
    delete b;                                                   // the destructor releases streams, events, buffers
}

}  // extern "C"

// ------------------------------------------------------------------ sharded parse
extern "C" re_status re_shard_map(re_handle *h, const uint8_t *d_text, uint64_t len, uint32_t flags,
                                  re_stream stream, void *d_workspace, uint64_t workspace_bytes, uint8_t *d_maps,
                                  int32_t *d_status) {
    if (!h || !d_maps || !d_status) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (flags & ~(RE_SHARD_PREV | RE_SHARD_NEXT)) { set_error("unknown shard flags"); return RE_E_INVALID_ARG; }
    re_slpf slot{};
    slot.d_status = d_status;
    SliceArgs sa;
    sa.shard = (flags & RE_SHARD_PREV ? SHARD_PREV : 0u) | (flags & RE_SHARD_NEXT ? SHARD_NEXT : 0u);
    sa.maps = d_maps;
    return parse_impl(h, d_text, len, stream, &slot, d_workspace, workspace_bytes, nullptr, sa);
}

extern "C" re_status re_shard_map_size(const re_handle *h, uint32_t *fwd_entries, uint32_t *bwd_entries) {
    if (!h || !fwd_entries || !bwd_entries) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (!scan_join(h)) { set_error("slice maps need both classic DFAs below 256 states"); return RE_E_CAPACITY; }
    *fwd_entries = h->host.nfd + 1;
    *bwd_entries = h->host.nbd + 1;
    return RE_OK;
}

extern "C" re_status re_shard_entry(const re_handle *h, const uint8_t *maps, uint32_t count, uint32_t *entry,
                                    uint32_t *entry_bwd, int32_t *accepted) {
    if (!h || (count && (!maps || !entry || !entry_bwd)) || !accepted) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (!scan_join(h)) { set_error("slice maps need both classic DFAs below 256 states"); return RE_E_CAPACITY; }
    const Compiled &C = h->host;
    const uint32_t nsf = C.nfd + 1, nsb = C.nbd + 1, per = nsf + nsb;
    if (!count) { *accepted = 0; return RE_OK; }
    // forward: E_0 = I; E_{r+1} = fwd_r(E_r); the text ends in fwd_{N-1}(E_{N-1})
    uint32_t e = 1;
    bool alive = true;
    for (uint32_t r = 0; r < count; ++r) {
        entry[r] = e;
        e = e < nsf ? maps[(size_t)r * per + e] : 0u;
        alive = alive && e != 0;
    }
    // backward: Ê_{N-1} = F; Ê_{r-1} = bwd_r(Ê_r)
    uint32_t b = 1;
    for (uint32_t r = count; r-- > 0;) {
        entry_bwd[r] = b;
        b = b < nsb ? maps[(size_t)r * per + nsf + b] : 0u;
    }
    // accepted iff the forward states survive the whole text and the last one meets F
    bool acc = alive;
    if (acc) {
        acc = false;
        for (uint32_t w = 0; w < C.W; ++w)
            acc = acc || (C.fBits[(size_t)e * C.W + w] & C.bBits[(size_t)1 * C.W + w]) != 0;
    }
    *accepted = acc ? 1 : 0;
    if (!acc)                                                 // every column of a rejected text is empty
        for (uint32_t r = 0; r < count; ++r) entry[r] = 0;
    return RE_OK;
}

extern "C" re_status re_parse_slice(re_handle *h, const uint8_t *d_text, uint64_t len, uint32_t entry,
                                    uint32_t entry_bwd, re_stream stream, re_slpf *slpf, void *d_workspace,
                                    uint64_t workspace_bytes, const re_parse_opts *opts) {
    if (!h) { set_error("null handle"); return RE_E_INVALID_ARG; }
    if (!len) { set_error("a slice is not empty"); return RE_E_INVALID_ARG; }
    if (entry > h->host.nfd || entry_bwd > h->host.nbd) { set_error("entry state out of range"); return RE_E_INVALID_ARG; }
    if (opts && (opts->flags & RE_PARSE_RECOGNIZE_ONLY)) { set_error("slices are parsed, not recognized"); return RE_E_INVALID_ARG; }
    SliceArgs sa;
    sa.fin = entry;
    sa.bin = entry_bwd;
    return parse_impl(h, d_text, len, stream, slpf, d_workspace, workspace_bytes, opts, sa);
}

extern "C" re_status re_state_bits(const re_handle *h, int32_t forward, uint32_t id, uint64_t *bits, uint32_t cap_words) {
    if (!h || !bits) { set_error("null argument"); return RE_E_INVALID_ARG; }
    const Compiled &C = h->host;
    if (cap_words < C.W) { set_error("buffer too small"); return RE_E_CAPACITY; }
    if (id >= (forward ? C.nf : C.nb)) { set_error("state id out of range"); return RE_E_INVALID_ARG; }
    const std::vector<uint64_t> &src = forward ? C.fBits : C.bBits;
    std::memcpy(bits, src.data() + (size_t)id * C.W, C.W * 8);
    return RE_OK;
}
