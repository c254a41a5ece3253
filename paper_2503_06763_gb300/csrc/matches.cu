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
// One warp per range of 2048 start columns, 32 consecutive ones per step,
// holding 64 columns in registers so that visits read their first 32 columns
// by shuffle.  A count pass, an exclusive scan of the per-warp counts and a
// write pass put the pairs in (i, j) order with no atomics; the total is
// reported even when the caller's buffer is smaller.
#include <type_traits>

#include "kernels.cuh"

namespace slpf {

constexpr uint32_t kScanBlock = 1024;

namespace {

template <int W>
__device__ __forceinline__ void load_column(const MatchArgs &a, uint64_t r, uint64_t (&v)[W]) {
    if (a.kind == RE_SLPF_PAIRS) {                          // C_r = B_r ∩ B̂_r from the two state ids
        uint64_t f, b;
        if (a.col_bytes == 4) {
            const uint32_t x = __ldg(reinterpret_cast<const uint32_t *>(a.cols) + r);
            f = x & 0xFFFFu; b = x >> 16;
        } else {
            const uint64_t x = __ldg(reinterpret_cast<const unsigned long long *>(a.cols) + r);
            f = x & 0xFFFFFFFFull; b = x >> 32;
        }
#pragma unroll
        for (int w = 0; w < W; ++w)
            v[w] = w < (int)a.W ? __ldg(a.fbits + f * a.W + w) & __ldg(a.bbits + b * a.W + w) : 0ull;
    } else if (a.kind == RE_SLPF_DICT) {
        const uint32_t id = a.col_bytes == 1   ? __ldg(reinterpret_cast<const uint8_t *>(a.cols) + r)
                            : a.col_bytes == 2 ? __ldg(reinterpret_cast<const uint16_t *>(a.cols) + r)
                                               : __ldg(reinterpret_cast<const uint32_t *>(a.cols) + r);
#pragma unroll
        for (int w = 0; w < W; ++w)                          // W rounds a.W up: the rows have stride a.W
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
        for (int w = 1; w < W; ++w) v[w] = 0;
    }
}

// Columns per warp: the warp takes 32 consecutive start columns per step, so
// its column loads are coalesced; warp-level scans keep the (i, j) order.
constexpr uint32_t kWarpCols = 2048;

__device__ __forceinline__ uint64_t warp_exclusive(uint64_t c, uint64_t &total) {
    const uint32_t lane = threadIdx.x & 31;
    uint64_t s = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, s, d);
        if ((int)lane >= d) s += y;
    }
    total = __shfl_sync(0xFFFFFFFFu, s, 31);
    return s - c;
}

// One step of a warp: lane l starts the visit at column i = base + l.  The
// warp holds columns base .. base + 63 in registers (c0: base + lane, c1:
// base + 32 + lane), so the first 32 columns of every visit come by shuffle;
// a visit still open after them goes on with loads (visit_from).  Called by
// the whole warp; emit(j) gets the matches (i, j) of this lane in j order.
template <int W, typename F>
__device__ void visit_from(const MatchArgs &a, uint64_t i, uint64_t r, uint64_t (&S)[W], F emit) {
    bool live = true;
    while (live && r < a.n) {
        uint64_t N[W], C[W];
#pragma unroll
        for (int w = 0; w < W; ++w) N[w] = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t m = S[w];
            while (m) {
                const uint32_t q = 64 * w + (uint32_t)__ffsll((long long)m) - 1;
                m &= m - 1;
#pragma unroll
                for (int w2 = 0; w2 < W; ++w2)
                        if (w2 < (int)a.W) N[w2] |= __ldg(a.folseg + (size_t)q * a.W + w2);
            }
        }
        ++r;
        load_column<W>(a, r, C);
        bool close = false;
        live = false;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            N[w] &= C[w];
            close |= (N[w] & a.close_first[w]) != 0;
            S[w] = N[w] & a.none[w];
            live |= S[w] != 0;
        }
        if (close) emit(r);
    }
}

template <int W, typename F>
__device__ __forceinline__ void warp_step(const MatchArgs &a, uint64_t base, const uint64_t (&c0)[W],
                                          const uint64_t (&c1)[W], F emit) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t i = base + lane;
    uint64_t S[W];
    bool whole = false, live = false;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        whole |= (c0[w] & a.whole[w]) != 0;
        S[w] = c0[w] & a.open[w];
        live |= S[w] != 0;
    }
    live = live && i <= a.n;
    if (whole && i <= a.n) emit(i);
    uint32_t d = 1;
    for (; d <= 32 && __any_sync(0xFFFFFFFFu, live); ++d) {
        const uint32_t src = lane + d;                        // column base + src: lane src of c0 or c1
        uint64_t col[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint64_t x0 = __shfl_sync(0xFFFFFFFFu, c0[w], src & 31);
            const uint64_t x1 = __shfl_sync(0xFFFFFFFFu, c1[w], src & 31);
            col[w] = src < 32 ? x0 : x1;
        }
        if (live && i + d - 1 < a.n) {                         // step from column i + d - 1 to i + d
            uint64_t N[W];
#pragma unroll
            for (int w = 0; w < W; ++w) N[w] = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint64_t m = S[w];
                while (m) {
                    const uint32_t q = 64 * w + (uint32_t)__ffsll((long long)m) - 1;
                    m &= m - 1;
#pragma unroll
                    for (int w2 = 0; w2 < W; ++w2)
                        if (w2 < (int)a.W) N[w2] |= __ldg(a.folseg + (size_t)q * a.W + w2);
                }
            }
            bool close = false;
            live = false;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                N[w] &= col[w];
                close |= (N[w] & a.close_first[w]) != 0;
                S[w] = N[w] & a.none[w];
                live |= S[w] != 0;
            }
            if (close) emit(i + d);
        } else {
            live = false;
        }
    }
    if (live) visit_from<W>(a, i, i + 32, S, emit);               // longer than the register window
}

// Columns base .. base + 63 into registers (zero past the last column).
template <int W>
__device__ __forceinline__ void load_window(const MatchArgs &a, uint64_t base, uint64_t (&c0)[W], uint64_t (&c1)[W]) {
    const uint32_t lane = threadIdx.x & 31;
    if (base + lane <= a.n) load_column<W>(a, base + lane, c0);
    else for (int w = 0; w < W; ++w) c0[w] = 0;
    if (base + 32 + lane <= a.n) load_column<W>(a, base + 32 + lane, c1);
    else for (int w = 0; w < W; ++w) c1[w] = 0;
}

template <int W>
__global__ void match_count_kernel(const __grid_constant__ MatchArgs a) {
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= a.G) return;                                   // whole warps: G counts warps
    const uint32_t lane = threadIdx.x & 31;
    uint64_t total = 0;
    if (*a.status == RE_OK) {
        for (uint32_t step = 0; step < kWarpCols / 32; ++step) {
            const uint64_t base = wid * kWarpCols + 32 * step;
            if (base > a.n) break;                            // warp-uniform
            uint64_t c0[W], c1[W];
            load_window<W>(a, base, c0, c1);
            uint64_t c = 0;
            warp_step<W>(a, base, c0, c1, [&](uint64_t) { ++c; });
            uint64_t t;
            warp_exclusive(c, t);
            total += t;
        }
    }
    if (lane == 0) a.cnt[wid] = total;
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

template <int W>
__global__ void match_write_kernel(const __grid_constant__ MatchArgs a) {
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= a.G) return;
    const uint32_t lane = threadIdx.x & 31;
    uint64_t off = a.cnt[wid] + a.bsum[wid / kScanBlock];
    if (*a.status == RE_OK) {
        for (uint32_t step = 0; step < kWarpCols / 32; ++step) {
            const uint64_t base = wid * kWarpCols + 32 * step;
            if (base > a.n) break;                            // warp-uniform
            uint64_t c0[W], c1[W];
            load_window<W>(a, base, c0, c1);
            uint64_t c = 0;
            warp_step<W>(a, base, c0, c1, [&](uint64_t) { ++c; });
            uint64_t t;
            uint64_t o = off + warp_exclusive(c, t);
            if (__any_sync(0xFFFFFFFFu, c != 0)) {
                const uint64_t i = base + lane;
                warp_step<W>(a, base, c0, c1, [&](uint64_t j) {
                    if (o < a.cap) { a.pairs[2 * o] = i; a.pairs[2 * o + 1] = j; }
                    ++o;
                });
            }
            off += t;
        }
    }
    if (wid == a.G - 1 && lane == 0) *a.count = off;          // the last warp ends the sequence
}

}  // namespace

size_t match_workspace_bytes(uint64_t n) {
    const uint64_t G = n / kWarpCols + 1;
    const uint64_t nb = (G + kScanBlock - 1) / kScanBlock;
    return ((G * 8 + 255) & ~(size_t)255) + ((nb * 8 + 255) & ~(size_t)255);
}

void launch_matches(MatchArgs a, void *ws, cudaStream_t s) {
    a.G = a.n / kWarpCols + 1;                                // warps, kWarpCols start columns each
    const uint64_t nb = (a.G + kScanBlock - 1) / kScanBlock;
    a.cnt = reinterpret_cast<uint64_t *>(ws);
    a.bsum = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(ws) + ((a.G * 8 + 255) & ~(size_t)255));
    const uint32_t threads = 128, blocks = (uint32_t)((a.G * 32 + threads - 1) / threads);
    auto run = [&](auto wtag) {
        constexpr int W = decltype(wtag)::value;
        match_count_kernel<W><<<blocks, threads, 0, s>>>(a);
        scan_block_kernel<<<(uint32_t)nb, kScanBlock, 0, s>>>(a.cnt, a.G, a.bsum);
        scan_totals_kernel<<<1, kScanBlock, 0, s>>>(a.bsum, nb);
        match_write_kernel<W><<<blocks, threads, 0, s>>>(a);
    };
    if (a.W <= 1) run(std::integral_constant<int, 1>{});
    else if (a.W <= 2) run(std::integral_constant<int, 2>{});
    else if (a.W <= 4) run(std::integral_constant<int, 4>{});
    else run(std::integral_constant<int, 8>{});
}

}  // namespace slpf
