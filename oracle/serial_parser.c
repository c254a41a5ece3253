/*
 * Oracle: the serial two-way NFA parser of the paper, over bitset columns.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library; the product never does.
 *
 * It computes Eq. (matrixmul) and Eq. (reverseNFAdef) of arXiv 2503.06763,
 * in the order given by Fig. (serialparser):
 *     C_0 = I,   C_r = N_{x_r} x C_{r-1}              r = 1 .. n
 *     Ĉ_n = F,   Ĉ_r = N_{x_{r+1}}^T x Ĉ_{r+1}         r = n-1 .. 0
 *     output C_r ∩ Ĉ_r                                 r = 0 .. n
 * Boolean matrices are stored by column: ncol[(a*ell + j)*W .. +W) is column j
 * of N_a as a bitset of rows.  So
 *     (N_a x V)[row]   = OR over j in V of ncol[a][j][row]
 *     (N_a^T x V)[j]   = (ncol[a][j] AND V) != 0
 * The forward columns are kept in out[], and the backward pass intersects them
 * in place (the memory saving described after Ex. 4).
 */
#include <stdint.h>
#include <string.h>

static int any_and(const uint64_t *a, const uint64_t *b, int W) {
    for (int w = 0; w < W; ++w)
        if (a[w] & b[w]) return 1;
    return 0;
}

/* Returns 0 on success, -1 on bad arguments.
 * ncol : [256][ell][W] column bitsets of N_a
 * I, F : [W] bitsets of the initial and final segments
 * x    : text of n bytes
 * out  : [(n+1)][W] receives the clean SLPF columns C_r ∩ Ĉ_r
 * tmp  : [2][W] scratch                                                    */
int oracle_serial_parse(int ell, int W, const uint64_t *ncol, const uint64_t *I,
                        const uint64_t *F, const uint8_t *x, int64_t n,
                        uint64_t *out, uint64_t *tmp) {
    if (ell <= 0 || W != (ell + 63) / 64 || n < 0) return -1;
    /* forward: C_0 = I, C_r = N_{x_r} x C_{r-1} */
    memcpy(out, I, sizeof(uint64_t) * W);
    for (int64_t r = 1; r <= n; ++r) {
        const uint64_t *prev = out + (r - 1) * W;
        uint64_t *cur = out + r * W;
        memset(cur, 0, sizeof(uint64_t) * W);
        const uint64_t *na = ncol + (int64_t)x[r - 1] * ell * W;
        for (int j = 0; j < ell; ++j) {
            if (prev[j >> 6] >> (j & 63) & 1) {
                const uint64_t *colj = na + (int64_t)j * W;
                for (int w = 0; w < W; ++w) cur[w] |= colj[w];
            }
        }
    }
    /* backward: Ĉ_n = F, Ĉ_r = N_{x_{r+1}}^T x Ĉ_{r+1}; intersect as we go */
    uint64_t *chat = tmp, *chat_next = tmp + W;
    memcpy(chat_next, F, sizeof(uint64_t) * W);
    for (int w = 0; w < W; ++w) out[n * W + w] &= chat_next[w];
    for (int64_t r = n - 1; r >= 0; --r) {
        const uint64_t *na = ncol + (int64_t)x[r] * ell * W;   /* x_{r+1} */
        memset(chat, 0, sizeof(uint64_t) * W);
        for (int j = 0; j < ell; ++j)
            if (any_and(na + (int64_t)j * W, chat_next, W)) chat[j >> 6] |= 1ull << (j & 63);
        for (int w = 0; w < W; ++w) out[r * W + w] &= chat[w];
        uint64_t *t = chat; chat = chat_next; chat_next = t;
    }
    return 0;
}
