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

/* ------------------------------------------------------------------------
 * The same equations with every column interned (hash-consed), for texts of
 * a GiB and more: Fig. (serialparser) keeps one column per position, here one
 * 32-bit id per position instead of W words.  Each distinct column is stored
 * once, and the product N_a x C (forward) or N_a^T x Ĉ (backward) of a stored
 * column with a byte is computed once, by the loops above, and remembered;
 * every later position with the same column and byte reuses it.  Nothing
 * else changes: C_0 = I, C_r = N_{x_r} C_{r-1}; Ĉ_n = F, Ĉ_r =
 * N_{x_{r+1}}^T Ĉ_{r+1}; clean column r = C_r ∩ Ĉ_r.
 */
#include <stdlib.h>

typedef struct {
    int W;
    int64_t n, cap;          /* stored columns, capacity */
    uint64_t *bits;          /* [cap][W] */
    int64_t *slot;           /* [hcap] open addressing, -1 = free */
    int64_t hcap;
    uint32_t *next;          /* [cap][256] product with each byte, 0xFFFFFFFF = not yet */
} Interned;

static uint64_t hash_bits(const uint64_t *v, int W) {
    uint64_t h = 1469598103934665603ull;
    for (int w = 0; w < W; ++w) {
        h ^= v[w];
        h *= 1099511628211ull;
        h ^= h >> 29;
    }
    return h;
}

static int interned_init(Interned *t, int W) {
    t->W = W; t->n = 0; t->cap = 64; t->hcap = 256;
    t->bits = (uint64_t *)malloc(sizeof(uint64_t) * W * t->cap);
    t->next = (uint32_t *)malloc(sizeof(uint32_t) * 256 * t->cap);
    t->slot = (int64_t *)malloc(sizeof(int64_t) * t->hcap);
    if (!t->bits || !t->next || !t->slot) return -1;
    for (int64_t i = 0; i < t->hcap; ++i) t->slot[i] = -1;
    return 0;
}

static void interned_free(Interned *t) { free(t->bits); free(t->next); free(t->slot); }

/* id of column v (stored if new); -1 on allocation failure */
static int64_t intern(Interned *t, const uint64_t *v) {
    const int W = t->W;
    uint64_t h = hash_bits(v, W) & (uint64_t)(t->hcap - 1);
    while (t->slot[h] >= 0) {
        const uint64_t *b = t->bits + t->slot[h] * W;
        int eq = 1;
        for (int w = 0; w < W; ++w) if (b[w] != v[w]) { eq = 0; break; }
        if (eq) return t->slot[h];
        h = (h + 1) & (uint64_t)(t->hcap - 1);
    }
    if (t->n == t->cap) {
        int64_t nc = t->cap * 2;
        uint64_t *nb = (uint64_t *)realloc(t->bits, sizeof(uint64_t) * W * nc);
        if (!nb) return -1;
        t->bits = nb;
        uint32_t *nn = (uint32_t *)realloc(t->next, sizeof(uint32_t) * 256 * nc);
        if (!nn) return -1;
        t->next = nn;
        t->cap = nc;
    }
    const int64_t id = t->n++;
    memcpy(t->bits + id * W, v, sizeof(uint64_t) * W);
    for (int a = 0; a < 256; ++a) t->next[id * 256 + a] = 0xFFFFFFFFu;
    t->slot[h] = id;
    if (t->n * 2 > t->hcap) {                       /* grow the index, rehash */
        int64_t hc = t->hcap * 2;
        int64_t *ns = (int64_t *)malloc(sizeof(int64_t) * hc);
        if (!ns) return -1;
        for (int64_t i = 0; i < hc; ++i) ns[i] = -1;
        for (int64_t k = 0; k < t->n; ++k) {
            uint64_t g = hash_bits(t->bits + k * W, W) & (uint64_t)(hc - 1);
            while (ns[g] >= 0) g = (g + 1) & (uint64_t)(hc - 1);
            ns[g] = k;
        }
        free(t->slot);
        t->slot = ns;
        t->hcap = hc;
    }
    return id;
}

/* Returns 0 on success, -1 on bad arguments or allocation failure, -2 when
 * the text has more than cap distinct clean columns.
 * ids   : [(n+1)] receives, for every r, the index of the clean column C_r ∩ Ĉ_r
 *         in cols
 * cols  : [cap][W] receives the distinct clean columns, in order of first use
 *         from r = n down to 0
 * ncols : receives their number                                             */
int oracle_serial_parse_ids(int ell, int W, const uint64_t *ncol, const uint64_t *I, const uint64_t *F,
                            const uint8_t *x, int64_t n, uint32_t *ids, uint64_t *cols, int64_t cap,
                            int64_t *ncols) {
    if (ell <= 0 || W != (ell + 63) / 64 || n < 0 || cap <= 0) return -1;
    Interned fw, bw;
    if (interned_init(&fw, W) || interned_init(&bw, W)) return -1;
    uint64_t *v = (uint64_t *)malloc(sizeof(uint64_t) * W * 2);
    int rc = v ? 0 : -1;
    /* forward: ids[r] = id of C_r */
    int64_t cur = rc ? -1 : intern(&fw, I);
    if (cur < 0) rc = -1;
    if (!rc) ids[0] = (uint32_t)cur;
    for (int64_t r = 1; r <= n && !rc; ++r) {
        const uint8_t a = x[r - 1];
        uint32_t nx = fw.next[cur * 256 + a];
        if (nx == 0xFFFFFFFFu) {                     /* N_a x C_{r-1}, as in oracle_serial_parse */
            const uint64_t *prev = fw.bits + cur * W;
            memset(v, 0, sizeof(uint64_t) * W);
            const uint64_t *na = ncol + (int64_t)a * ell * W;
            for (int j = 0; j < ell; ++j)
                if (prev[j >> 6] >> (j & 63) & 1)
                    for (int w = 0; w < W; ++w) v[w] |= na[(int64_t)j * W + w];
            const int64_t id = intern(&fw, v);
            if (id < 0) { rc = -1; break; }
            nx = (uint32_t)id;
            fw.next[cur * 256 + a] = nx;
        }
        cur = nx;
        ids[r] = nx;
    }
    /* backward: Ĉ_r, intersected with C_r and interned into cols */
    Interned cl;
    const int cl_made = !rc && interned_init(&cl, W) == 0;
    if (!cl_made) rc = -1;
    int64_t bcur = rc ? -1 : intern(&bw, F);
    if (!rc && bcur < 0) rc = -1;
    for (int64_t r = n; r >= 0 && !rc; --r) {
        if (r < n) {
            const uint8_t a = x[r];                  /* x_{r+1} */
            uint32_t nx = bw.next[bcur * 256 + a];
            if (nx == 0xFFFFFFFFu) {                 /* N_a^T x Ĉ_{r+1} */
                const uint64_t *nxt = bw.bits + bcur * W;
                memset(v, 0, sizeof(uint64_t) * W);
                const uint64_t *na = ncol + (int64_t)a * ell * W;
                for (int j = 0; j < ell; ++j)
                    if (any_and(na + (int64_t)j * W, nxt, W)) v[j >> 6] |= 1ull << (j & 63);
                const int64_t id = intern(&bw, v);
                if (id < 0) { rc = -1; break; }
                nx = (uint32_t)id;
                bw.next[bcur * 256 + a] = nx;
            }
            bcur = nx;
        }
        const uint64_t *fc = fw.bits + (int64_t)ids[r] * W, *bc = bw.bits + bcur * W;
        for (int w = 0; w < W; ++w) v[W + w] = fc[w] & bc[w];
        const int64_t id = intern(&cl, v + W);
        if (id < 0) { rc = -1; break; }
        if (id >= cap) { rc = -2; break; }
        ids[r] = (uint32_t)id;
    }
    if (!rc) {
        memcpy(cols, cl.bits, sizeof(uint64_t) * W * cl.n);
        *ncols = cl.n;
    }
    if (cl_made) interned_free(&cl);
    interned_free(&fw);
    interned_free(&bw);
    free(v);
    return rc;
}
