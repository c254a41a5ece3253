// re_parse_static: re_parse on a fixed, library-owned device scratch buffer.
//
// For callers that cannot allocate device memory when they parse: a C host
// program with no device allocator of its own, or a request loop that must
// not call cudaMalloc / cudaFree between launches (both may synchronise the
// whole device and stall every other stream).  The scratch is a file-scope
// __device__ array, so it exists once the module is loaded and nothing here
// allocates.
//
// Nothing in the scratch has to start at zero: every parse writes each word of
// its workspace before reading it (the first kernel resets the join's flags).
#include <mutex>

#include "re_internal.h"

namespace {

__device__ __align__(256) unsigned char g_scratch[RE_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" re_status re_parse_static(re_handle *h, const uint8_t *d_text, uint64_t len, re_stream stream,
                                     re_slpf *slpf, const re_parse_opts *opts) {
    if (!h) { slpf::set_error("null handle"); return RE_E_INVALID_ARG; }
    uint64_t need = 0;
    re_status ws = re_workspace_size(h, len, opts, &need);
    if (ws != RE_OK) return ws;
    if (need > RE_STATIC_SCRATCH_BYTES) {
        // an autotuned chunk length can need more than the built-in rule;
        // re_parse then falls back to the rule's length, as with any workspace
        // too small for the tuned layout
        ws = slpf::workspace_rule_bytes(h, len, opts, &need);
        if (ws != RE_OK) return ws;
    }
    if (need > RE_STATIC_SCRATCH_BYTES) {
        slpf::set_error("the text needs " + std::to_string(need) + " bytes of workspace, more than "
                        "RE_STATIC_SCRATCH_BYTES; use re_parse with a caller workspace");
        return RE_E_CAPACITY;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        slpf::set_error("no usable current device");
        return RE_E_CUDA;
    }
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> guard(g_lock);
        if (!g_scratch_ptr[dev]) {                       // once per device, with that device current
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) {
                slpf::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return RE_E_CUDA;
            }
            g_scratch_ptr[dev] = p;
        }
        ptr = g_scratch_ptr[dev];
    }
    return re_parse(h, d_text, len, stream, slpf, ptr, RE_STATIC_SCRATCH_BYTES, opts);
}
