// Match extraction (arXiv 2503.06763, Sect. 4.2, "Match extraction",
// getMatches): the spans (i, j) of a group k -- pairs such that some syntax
// tree has the node k( ... )k over text[i:j] -- read off the clean SLPF.
//
// A segment is the parentheses and leaves before an end letter.  Column r's
// segments that hold a whole "k( ... )k" give (r, r).  Those whose last
// k-parenthesis is k( leave group k open; the visit then follows FolSeg arcs
// (Eq. folsegdef) column by column: segments without a k-parenthesis keep it
// open, and a segment whose first k-parenthesis is )k at column j closes it,
// giving (i, j).  The SLPF is clean, so each such path lies on a whole tree.
//
// One thread per range of 64 start columns.  A count pass, an exclusive scan
// of the counts and a write pass put the pairs in (i, j) order with no
// atomics; the total is reported even when the caller's buffer is smaller.
#include "kernels.cuh"

namespace slpf {

constexpr uint32_t kScanBlock = 1024;

namespace {

__device__ __forceinline__ void load_column(const MatchArgs &a, uint64_t r, uint64_t (&v)[kMatchW]) {
    if (a.kind == RE_SLPF_DICT) {
        const uint32_t id = a.col_bytes == 2 ? __ldg(reinterpret_cast<const uint16_t *>(a.cols) + r)
                                             : __ldg(reinterpret_cast<const uint32_t *>(a.cols) + r);
#pragma unroll
        for (int w = 0; w < kMatchW; ++w)
            v[w] = (w < (int)a.W && id) ? __ldg(a.dict + (size_t)(id - 1) * a.W + w) : 0ull;
    } else {
        uint64_t x;
        switch (a.col_bytes) {
            case 1: x = __ldg(reinterpret_cast<const uint8_t *>(a.cols) + r); break;
            case 2: x = __ldg(reinterpret_cast<const uint16_t *>(a.cols) + r); break;
            case 4: x = __ldg(reinterpret_cast<const uint32_t *>(a.cols) + r); break;
            default: x = __ldg(reinterpret_cast<const unsigned long long *>(a.cols) + r); break;
        }
        v[0] = x;
#pragma unroll
        for (int w = 1; w < kMatchW; ++w) v[w] = 0;
    }
}

// Visit from start column i; emit(j) for every match (i, j), j increasing.
template <typename F>
__device__ void visit(const MatchArgs &a, uint64_t i, F emit) {
    uint64_t C[kMatchW], S[kMatchW];
    load_column(a, i, C);
    bool whole = false, live = false;
#pragma unroll
    for (int w = 0; w < kMatchW; ++w) {
        whole |= (C[w] & a.whole[w]) != 0;
        S[w] = C[w] & a.open[w];
        live |= S[w] != 0;
    }
    if (whole) emit(i);
    uint64_t r = i;
    while (live && r < a.n) {
        uint64_t N[kMatchW];
#pragma unroll
        for (int w = 0; w < kMatchW; ++w) N[w] = 0;
#pragma unroll
        for (int w = 0; w < kMatchW; ++w) {
            uint64_t m = S[w];
            while (m) {
                const uint32_t q = 64 * w + (uint32_t)__ffsll((long long)m) - 1;
                m &= m - 1;
#pragma unroll
                for (int w2 = 0; w2 < kMatchW; ++w2)
                    if (w2 < (int)a.W) N[w2] |= __ldg(a.folseg + (size_t)q * a.W + w2);
            }
        }
        ++r;
        load_column(a, r, C);
        bool close = false;
        live = false;
#pragma unroll
        for (int w = 0; w < kMatchW; ++w) {
            N[w] &= C[w];
            close |= (N[w] & a.close_first[w]) != 0;
            S[w] = N[w] & a.none[w];
            live |= S[w] != 0;
        }
        if (close) emit(r);
    }
}

__global__ void match_count_kernel(MatchArgs a) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.G) return;
    uint64_t c = 0;
    if (*a.status == RE_OK) {
        const uint64_t end = min(64 * g + 64, a.n + 1);
        for (uint64_t i = 64 * g; i < end; ++i) visit(a, i, [&](uint64_t) { ++c; });
    }
    a.cnt[g] = c;
}

// Exclusive scan of kScanBlock values per block (in place); block totals to out.
__global__ void scan_block_kernel(uint64_t *v, uint64_t n, uint64_t *out) {
    __shared__ uint64_t warp_tot[kScanBlock / 32];
    const uint64_t j = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const uint64_t x = j < n ? v[j] : 0;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t s = x;                                          // inclusive within the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, s, d);
        if ((int)lane >= d) s += y;
    }
    if (lane == 31) warp_tot[wid] = s;
    __syncthreads();
    if (wid == 0) {
        uint64_t t = warp_tot[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
            if ((int)lane >= d) t += y;
        }
        warp_tot[lane] = t;                                  // inclusive warp totals
    }
    __syncthreads();
    const uint64_t before = (wid ? warp_tot[wid - 1] : 0) + s - x;
    if (j < n) v[j] = before;
    if (threadIdx.x == kScanBlock - 1) out[blockIdx.x] = warp_tot[31];
}

// Exclusive scan of the block totals by one block, kScanBlock at a time.
__global__ void scan_totals_kernel(uint64_t *v, uint64_t n) {
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < n; base += kScanBlock) {
        const uint64_t j = base + threadIdx.x;
        const uint64_t x = j < n ? v[j] : 0;
        uint64_t s = x;
        for (uint32_t d = 1; d < kScanBlock; d <<= 1) {     // simple Hillis-Steele in shared memory
            __shared__ uint64_t buf[kScanBlock];
            buf[threadIdx.x] = s;
            __syncthreads();
            if (threadIdx.x >= d) s += buf[threadIdx.x - d];
            __syncthreads();
        }
        const uint64_t c0 = carry;
        if (j < n) v[j] = c0 + s - x;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry = c0 + s;
        __syncthreads();
    }
}

__global__ void match_write_kernel(MatchArgs a) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.G) return;
    uint64_t off = a.cnt[g] + a.bsum[g / kScanBlock];
    if (*a.status == RE_OK) {
        const uint64_t end = min(64 * g + 64, a.n + 1);
        for (uint64_t i = 64 * g; i < end; ++i)
            visit(a, i, [&](uint64_t j) {
                if (off < a.cap) { a.pairs[2 * off] = i; a.pairs[2 * off + 1] = j; }
                ++off;
            });
    }
    if (g == a.G - 1) *a.count = off;                       // the last range ends the sequence
}

}  // namespace

size_t match_workspace_bytes(uint64_t n) {
    const uint64_t G = n / 64 + 1;
    const uint64_t nb = (G + kScanBlock - 1) / kScanBlock;
    return ((G * 8 + 255) & ~(size_t)255) + ((nb * 8 + 255) & ~(size_t)255);
}

void launch_matches(MatchArgs a, void *ws, cudaStream_t s) {
    a.G = a.n / 64 + 1;
    const uint64_t nb = (a.G + kScanBlock - 1) / kScanBlock;
    a.cnt = reinterpret_cast<uint64_t *>(ws);
    a.bsum = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(ws) + ((a.G * 8 + 255) & ~(size_t)255));
    const uint32_t threads = 128, blocks = (uint32_t)((a.G + threads - 1) / threads);
    match_count_kernel<<<blocks, threads, 0, s>>>(a);
    scan_block_kernel<<<(uint32_t)nb, kScanBlock, 0, s>>>(a.cnt, a.G, a.bsum);
    scan_totals_kernel<<<1, kScanBlock, 0, s>>>(a.bsum, nb);
    match_write_kernel<<<blocks, threads, 0, s>>>(a);
}

}  // namespace slpf
