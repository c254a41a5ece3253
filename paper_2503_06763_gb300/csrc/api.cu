// C ABI of include/slpf_parser.h: compile (host tables -> one device
// allocation), layout / workspace sizing, and the parse launcher that
// enqueues reach -> join -> fix-up -> build & merge on the caller's stream.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <string>

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
    static int cached[64] = {0};
    if (device < 0 || device >= 64) return 152;
    if (!cached[device]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
        cached[device] = v > 0 ? v : 152;
    }
    return cached[device];
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

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// Text viewed as rows of full chunks (k bytes), one box = 32 chunks x 64
// bytes, SWIZZLE_64B to match the reach kernel's tile reads.
bool text_tensor_map(CUtensorMap &map, const uint8_t *d_text, uint32_t k, uint64_t rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn || rows < 32 || rows > 0xFFFFFFFFull || (k % 64) != 0) return false;
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
    if (!fn || rows == 0 || rows > 0xFFFFFFFFull || (cb != 1 && cb != 2)) return false;
    const cuuint64_t dims[2] = {64ull * cb, rows};
    const cuuint64_t strides[1] = {64ull * cb};
    const cuuint32_t box[2] = {64u * cb, 32u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = fn(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, d_cols, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, cb == 2 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

constexpr int kArrays = 19;

struct Layout {
    uint32_t k, c, S;
    uint64_t Gc;
    size_t off[kArrays];
    size_t total;
};

Layout layout_for(const re_handle *h, uint64_t n, uint32_t k) {
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
        FLAG_COUNT * 4};
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
    t.f2 = C.f2.empty() ? nullptr : (const uint32_t *)(b + pc[i_f2].off);
    t.b2 = C.b2.empty() ? nullptr : (const uint32_t *)(b + pc[i_b2].off);
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
    const re_status st = resolve_kind(h, kind, k, cb);
    if (st != RE_OK) return st;
    if (kind_out) *kind_out = k;
    if (col_bytes) *col_bytes = cb;
    if (bytes) *bytes = (len + 1) * cb;
    return RE_OK;
}

re_status re_workspace_size(const re_handle *h, uint64_t len, const re_parse_opts *opts, uint64_t *bytes) {
    if (!h || !bytes) { set_error("null argument"); return RE_E_INVALID_ARG; }
    const uint32_t k = choose_chunk(len, sm_count_of(h->device), opts);
    if (k % kSub || k == 0) { set_error("chunk_len must be a positive multiple of 64"); return RE_E_INVALID_ARG; }
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
        set_error("n_events must be 0 or RE_PHASE_EVENTS");
        return RE_E_INVALID_ARG;
    }
    const bool recognize = opts && (opts->flags & RE_PARSE_RECOGNIZE_ONLY);
    cudaEvent_t *ev = (opts && opts->n_events) ? (cudaEvent_t *)opts->events : nullptr;
    re_slpf_kind kind = RE_SLPF_DENSE;
    uint32_t cb = 1;
    if (!recognize || slpf->d_cols) {
        const re_status st = resolve_kind(h, slpf->kind, kind, cb);
        if (st != RE_OK) return st;
        if (slpf->col_bytes != cb) { set_error("slpf->col_bytes does not match the layout"); return RE_E_INVALID_ARG; }
        if (!slpf->d_cols || slpf->cols_cap_bytes < (len + 1) * cb) { set_error("SLPF buffer too small"); return RE_E_CAPACITY; }
        if ((uintptr_t)slpf->d_cols & 15) { set_error("d_cols must be 16-byte aligned"); return RE_E_INVALID_ARG; }
    }
    int dev_now = 0;
    cudaGetDevice(&dev_now);
    if (dev_now != h->device) { set_error("current device differs from the handle's device"); return RE_E_INVALID_ARG; }
    const int sms = sm_count_of(h->device);
    const uint32_t k = choose_chunk(len, sms, opts);
    if (k % kSub || k == 0) { set_error("chunk_len must be a positive multiple of 64"); return RE_E_INVALID_ARG; }
    if (len / k >= 0xFFFFFFF0ull) { set_error("text too long for this chunk length"); return RE_E_INVALID_ARG; }
    const Layout L = layout_for(h, len, k);
    if (len && (!d_workspace || workspace_bytes < L.total || ((uintptr_t)d_workspace & 255))) {
        set_error("workspace missing, too small or not 256-byte aligned");
        return RE_E_CAPACITY;
    }
    slpf->n_cols = len + 1;
    cudaStream_t s = (cudaStream_t)stream;
    Params p{};
    p.t = h->dev;
    p.x = d_text; p.n = len; p.k = k; p.c = L.c; p.S = L.S; p.Gc = L.Gc;
    p.out = recognize ? nullptr : slpf->d_cols;
    p.col_bytes = cb; p.kind = kind; p.status = slpf->d_status;
    p.recognize = recognize ? 1u : 0u;
    const DevTables &t = h->dev;
    const bool fit16 = t.nf < 65536 && t.nb < 65536;
    if (t.f2 && t.b2 && tables_smem_bytes(t, TM_PAIR) <= kSmemPairMax) p.tmode = TM_PAIR;
    else if (fit16 && tables_smem_bytes(t, TM_SMEM) <= kSmemTablesMax) p.tmode = TM_SMEM;
    else p.tmode = TM_GLOBAL;
    const size_t tab = tables_smem_bytes(t, p.tmode);
    p.Gfast = len / kSub;
    alignas(64) CUtensorMap out_map;
    std::memset(&out_map, 0, sizeof(out_map));
    p.out_tma = (!recognize && output_tensor_map(out_map, slpf->d_cols, cb, p.Gfast)) ? 1u : 0u;
    // Stage the dictionary pair table in shared memory when the merge's whole
    // footprint (tables, stage, output tiles and the table) still fits.
    if (kind == RE_SLPF_DICT && tab + merge_extra_smem(p) + (size_t)t.nf * t.nb * cb <= kSmemMergeMax) p.pt_in_smem = 1;
    alignas(64) CUtensorMap text_map;
    std::memset(&text_map, 0, sizeof(text_map));
    p.c_full = (uint32_t)(len / k);
    p.text_tma = text_tensor_map(text_map, d_text, k, p.c_full) ? 1u : 0u;
    auto mark = [&](int j) -> cudaError_t { return ev ? cudaEventRecord(ev[j], s) : cudaSuccess; };
    if (len == 0) {
        CUDA_TRY(mark(0), "event");
        launch_empty(p, s);
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
    p.w.fnrec = (uint32_t *)(w + L.off[10]); p.w.bnrec = (uint32_t *)(w + L.off[11]);
    p.w.fhit = (uint32_t *)(w + L.off[12]); p.w.bhit = (uint32_t *)(w + L.off[13]);
    p.w.recFc = (uint32_t *)(w + L.off[14]); p.w.recBc = (uint32_t *)(w + L.off[15]);
    p.w.recFe = (uint2 *)(w + L.off[16]); p.w.recBe = (uint2 *)(w + L.off[17]);
    p.w.flags = (int32_t *)(w + L.off[18]);
    CUDA_TRY(mark(0), "event");
    launch_flags_init(p, s);
    if (!launch_reach(p, text_map, s, std::max(t.msf, recognize ? 1u : t.msb), sms)) {
        set_error("too many speculative starts");
        return RE_E_INTERNAL;
    }
    CUDA_TRY(mark(1), "event");
    launch_join(p, s);
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

}  // extern "C"
