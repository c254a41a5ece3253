/*
 * slpf_parser.h -- C ABI of the GB300 parallel regular-expression parser.
 *
 * The library computes the clean shared linearized parse forest (SLPF) of a
 * text under a regular expression, following arXiv 2503.06763
 * ("A parallel parser for regular expressions"):
 *   - the SLPF is the series of columns C_0 .. C_n, each a set of segments
 *     (Sect. 2.3.5; definition after Fig. SLPFe3), computed here by the
 *     chunked speculative algorithm of Sect. 3.2 (Eqs. reacher, joiner,
 *     builder, merger) on the device;
 *   - segments, the parser NFA and its DFA / multi-entry DFA are built on the
 *     host by re_compile (Sects. 2.2, 2.3, 3.1, App. A).
 *
 * Conventions for every call:
 *   - Pointers named d_* are device pointers on the device that was current
 *     when the handle was compiled; all other pointers are host pointers.
 *   - Device buffers passed in are owned by the caller and must stay alive
 *     until the stream work that uses them has finished.
 *   - Calls return a re_status synchronously for argument, compile and launch
 *     errors.  Data-dependent results (text accepted / rejected, internal
 *     consistency failure) are written to the device word slpf->status and
 *     are valid once the stream has been synchronised.
 *   - Nothing aborts the process and nothing falls back to the CPU.  When the
 *     CUDA runtime reports an error the call returns RE_E_CUDA and
 *     re_last_error() describes it.
 *   - A handle may be used by several host threads for re_parse concurrently;
 *     re_compile / re_free of the same handle must not race with its use.
 */
#ifndef SLPF_PARSER_H
#define SLPF_PARSER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct re_handle re_handle;     /* opaque: owns host and device tables */
typedef struct CUstream_st *re_stream;  /* a cudaStream_t; NULL = legacy default */

typedef enum {
    RE_OK = 0,
    RE_REJECTED = 1,               /* status word only: text not in L(e); all columns empty */
    RE_E_INVALID_ARG = -1,
    RE_E_SYNTAX = -2,              /* malformed RE */
    RE_E_INFINITE_AMBIGUITY = -3,  /* an iterated sub-RE derives the empty text (Sect. 2.1, App. A)
                                      and re_compile_opts.sample_limit is 0 */
    RE_E_TOO_MANY_STATES = -4,     /* automaton exceeds re_compile_opts.max_states */
    RE_E_NOMEM = -5,               /* host or device allocation failed (re_compile only) */
    RE_E_CUDA = -6,                /* CUDA runtime error; see re_last_error() */
    RE_E_TIMEOUT = -7,             /* status word only: a bounded device wait ran out (the join's grid barrier) */
    RE_E_CAPACITY = -8,            /* an output / workspace buffer is smaller than required */
    RE_E_INTERNAL = -9             /* status word only: a device consistency check failed */
} re_status;

/* SLPF column encodings.
 *   DENSE : column r is the bitset of its segments (bit j = segment id j),
 *           stored little-endian in col_bytes = 1, 2, 4 or 8 bytes.  Needs
 *           ell <= 64.  Segment ids are the canonical order reported by
 *           re_segment_name.
 *   DICT  : column r is an index into the handle's column dictionary
 *           (re_dict_copy); index 0 is the empty column.  col_bytes = 1 when
 *           the dictionary has fewer than 255 entries, 2 when it has fewer
 *           than 65535, else 4.
 *   PAIRS : column r is the pair (f, b) of the forward DFA state B_r and the
 *           reverse DFA state B̂_r at r (Eq. merger: C_r = B_r ∩ B̂_r): f in
 *           the low half, b in the high half of col_bytes = 4 (both automata
 *           of at most 65536 states) or 8 bytes.  re_state_bits gives the
 *           segment sets; a rejected text has every column 0 (state 0 is the
 *           empty set).  Exact for any ell and any automaton size, with no
 *           dictionary; the ids are the handle's, so equal columns may come
 *           from different pairs.
 *   AUTO  : DENSE when ell <= 16, else DICT when the handle has a
 *           dictionary, else DENSE when ell <= 64, else PAIRS.                 */
typedef enum { RE_SLPF_AUTO = 0, RE_SLPF_DENSE = 1, RE_SLPF_DICT = 2, RE_SLPF_PAIRS = 3 } re_slpf_kind;

/* Infinitely ambiguous REs (App. A, "Infinite ambiguity"): an RE whose
 * iterated sub-RE derives the empty text gives some texts infinitely many
 * LSTs.  sample_limit = 0 rejects such an RE with RE_E_INFINITE_AMBIGUITY.
 * sample_limit = L in [1, RE_SAMPLE_LIMIT_MAX] accepts it and keeps a finite
 * sample: the segment computation counts the numbered symbols of each
 * segment and keeps the segments in which every symbol (an operator
 * parenthesis or an ε) occurs at most L times.  The SLPF of a text then
 * holds exactly those LSTs of the text whose every segment obeys the limit;
 * with L = 2 the sample of Fig. (infamb) holds its first three trees, with
 * L = 3 all four shown.  On a finitely ambiguous RE no segment repeats a
 * symbol, so every L gives the exact parser.  The segment count grows about
 * linearly with L on the REs of App. A; re_compile returns
 * RE_E_TOO_MANY_STATES when the enumeration or the automata outgrow their
 * caps.                                                                    */
#define RE_SAMPLE_LIMIT_MAX 16u

typedef struct {
    uint32_t max_states;      /* cap on forward + reverse automaton states; 0 = 1<<20 */
    uint32_t max_dict;        /* cap on dictionary pairs considered; 0 = 1<<24 */
    uint32_t flags;           /* 0 or RE_COMPILE_HOST_ONLY | RE_COMPILE_DFA_STARTS | RE_COMPILE_DFA_STARTS_BWD */
    uint32_t sample_limit;    /* 0 = reject infinitely ambiguous REs; L >= 1 = sample them (above) */
} re_compile_opts;

/* Build the host tables only (no device upload, no CUDA call): the handle
 * answers re_get_info / re_segment_name / re_dict_copy / re_slpf_layout but
 * re_parse rejects it with RE_E_INVALID_ARG.  For inspection on machines
 * without a GPU.                                                            */
#define RE_COMPILE_HOST_ONLY 1u

/* Ablation of the ME-DFA (Sect. 3.1; Sect. 5 compares it with the DFA): the
 * forward speculative runs of a chunk start from every state of the classic
 * forward DFA (those reachable from I), one run per distinct state after the
 * chunk's first byte, with no last-character filter; the join then finds the
 * run of the actual input state by an exact (class pair, state) lookup.
 * Backward runs keep the ME-DFA starts.  Results are identical; only the
 * speculation cost differs.  re_compile returns RE_E_TOO_MANY_STATES when a
 * class pair would need more than 32 runs.                                  */
#define RE_COMPILE_DFA_STARTS 2u

/* The same ablation for the backward runs: a chunk's backward speculative
 * runs start from every state of the classic reverse DFA (those reachable
 * from F), one run per distinct state after the chunk's last byte, and the
 * backward join looks up the run of the actual state at the chunk's right
 * edge.  Combine with RE_COMPILE_DFA_STARTS for both directions.  Results
 * are identical; re_compile returns RE_E_TOO_MANY_STATES when a byte class
 * would need more than 32 runs.                                             */
#define RE_COMPILE_DFA_STARTS_BWD 4u

typedef struct {
    re_slpf_kind kind;        /* requested encoding */
    uint32_t chunk_len;       /* text chunk length k in bytes (multiple of 64); 0 = automatic */
    uint32_t flags;           /* RE_PARSE_RECOGNIZE_ONLY or 0 */
    uint32_t n_events;        /* 0, or RE_PHASE_EVENTS */
    void **events;            /* n_events cudaEvent_t created by the caller; recorded on the
                                 parse stream before the first phase and after each phase
                                 (an event between phases keeps the next kernel from
                                 starting while the previous one drains) */
} re_parse_opts;

/* Phase boundaries recorded into re_parse_opts.events: [0] start,
 * [1] after reach (forward and backward, Eq. reacher), [2] after join
 * (Eq. joiner) and the status word, [3] after checkpoint fix-up, [4] after
 * build & merge (Eqs. builder, merger) and compose.  In recognizer mode
 * [3] and [4] follow [2] immediately.                                      */
#define RE_PHASE_EVENTS 5u

/* Recognizer mode (Sect. 4.2, "Mere recognizer"): run forward reach and join
 * only, write the accept / reject status and no columns.                    */
#define RE_PARSE_RECOGNIZE_ONLY 1u

/* Reach kernel shape (the reach of Sect. 3.2; every shape computes the same
 * end states and the same SLPF).  re_autotune chooses one per handle and
 * length bucket together with the chunk length; RE_PARSE_REACH(v) in
 * re_parse_opts.flags forces one (tests, measurements):
 *   1: tables indexed by the byte itself, one direction per block of 24
 *      warps (32 when every class with a byte >= 128 has one below, so the
 *      rows hold bytes 0..127 only), 2-stage TMA ring (automata of at most
 *      256 states per direction);
 *   2: a warp per direction of each 32-chunk tile (two lanes per chunk),
 *      tables by byte class, 3-stage TMA ring;
 *   3: as 2 with a 2-stage ring;
 *   4: one lane per chunk walking both directions, 3-stage ring.
 * 0 (the default) is the tuned shape, else 1 where it applies, else 2.
 * Shapes 1 (and 2, 3 when the class alphabet is above 16) let the reach
 * store every position's state, so build & merge is a gather.              */
#define RE_PARSE_REACH(v) ((uint32_t)(v) << 8)
#define RE_PARSE_REACH_MASK 0x700u

/* For tests of the join's bounded waits only: one block of the join scan
 * leaves before its first grid barrier, so the others' waits run out (about a
 * second) and the status word becomes RE_E_TIMEOUT.  The device stays usable;
 * the columns of such a parse are unspecified.  No effect when the join runs
 * as chains (automata with more than 255 classic-DFA states).               */
#define RE_PARSE_TEST_STALL_JOIN 0x80000000u

/* Output descriptor.  Filled by the caller: kind, col_bytes, d_cols,
 * cols_cap_bytes and d_status; re_slpf_layout gives the sizes.  n_cols is
 * written by re_parse (len + 1).                                            */
typedef struct {
    re_slpf_kind kind;        /* DENSE or DICT (never AUTO once laid out) */
    uint32_t col_bytes;       /* bytes per column */
    uint64_t n_cols;          /* number of columns, len + 1 */
    void *d_cols;             /* n_cols * col_bytes bytes, written by re_parse: device memory, or
                                 pinned host memory the device addresses (plain stores) */
    uint64_t cols_cap_bytes;  /* capacity of d_cols */
    int32_t *d_status;        /* device: one re_status word (RE_OK / RE_REJECTED / RE_E_INTERNAL /
                                 RE_E_TIMEOUT) */
} re_slpf;

typedef struct {
    uint32_t n_segments;      /* ell = |Q| (Sect. 2.4) */
    uint32_t n_positions;     /* numbered terminals (character-set positions) */
    uint32_t n_classes;       /* byte classes */
    uint32_t words_per_col;   /* ceil(ell / 64) */
    uint32_t fwd_states;      /* forward DFA + ME-DFA states, without the empty set */
    uint32_t fwd_dfa_states;  /* of which reachable from I (the classic DFA, Sect. 3.1) */
    uint32_t bwd_states;      /* reverse DFA + ME-DFA states, without the empty set */
    uint32_t bwd_dfa_states;  /* of which reachable from F */
    uint32_t fwd_slots_max;   /* most forward speculative runs for one chunk */
    uint32_t bwd_slots_max;   /* most backward speculative runs for one chunk */
    uint64_t dict_size;       /* distinct non-empty columns C = B ∩ B̂ (0 = no dictionary) */
    uint32_t inf_ambiguous;   /* 1 when the RE is infinitely ambiguous (its SLPFs are samples) */
    uint32_t sample_limit;    /* the compile option's sample_limit */
    uint32_t ascii_rows;      /* 1 when every byte class holding a byte >= 128 also holds one
                                 below 128: the byte-table reach then stages table rows of the
                                 128 bytes below 128 only and folds the others onto them */
    uint32_t reach_shapes;    /* bit v set: reach shape v (RE_PARSE_REACH) runs for this automaton */
} re_info;

/* Compile a pattern (Sect. 2.1 syntax plus App. A character features:
 * '|' union, juxtaposition, postfix '*', '+', '?', bounded repetition
 * 'e{h}' (1 <= h), 'e{h,k}' (h < k) and 'e{h,}' (bounds up to 4096; every
 * iteration gets its own numbered copy of e), '(' ')' groups,
 * '[...]' / '[^...]' byte sets, '.', '\' escapes incl. \n \t \r \xHH; an empty
 * alternative is ε).  Builds segments (Fig. segmentalgo), FolSeg
 * (Eq. folsegdef), forward / reverse DFA and ME-DFA (Sect. 3.1) and uploads
 * them to the current device.  On success *out owns host and device memory
 * until re_free.                                                            */
re_status re_compile(const char *pattern, size_t len, const re_compile_opts *opts,
                     re_handle **out);
void re_free(re_handle *h);

re_status re_get_info(const re_handle *h, re_info *info);

/* Name of segment id (canonical order): tokens 'k(' ')k' 'tk' 'ek' '$'
 * separated by one space, e.g. "1( 2( t3".  Writes a NUL-terminated string
 * of at most cap bytes.                                                     */
re_status re_segment_name(const re_handle *h, uint32_t id, char *buf, size_t cap);

/* Column dictionary for DICT output: entry d (1-based) occupies words
 * [(d-1)*W, d*W) of host_words; the empty column (index 0) is not stored.   */
re_status re_dict_copy(const re_handle *h, uint64_t *host_words, uint64_t cap_words);

/* Resolve AUTO and report the output size for a text of len bytes.        */
re_status re_slpf_layout(const re_handle *h, uint64_t len, re_slpf_kind kind,
                         re_slpf_kind *kind_out, uint32_t *col_bytes, uint64_t *bytes);

/* Device workspace needed by re_parse for len bytes with these options.    */
re_status re_workspace_size(const re_handle *h, uint64_t len, const re_parse_opts *opts,
                            uint64_t *bytes);

/* Enqueue the parse of d_text[0..len) on stream: reach, join, build&merge and
 * compose (Sect. 3.2).  Asynchronous: returns once the kernels are launched.
 * d_workspace must hold re_workspace_size bytes (256-byte aligned).        */
re_status re_parse(re_handle *h, const uint8_t *d_text, uint64_t len, re_stream stream,
                   re_slpf *slpf, void *d_workspace, uint64_t workspace_bytes,
                   const re_parse_opts *opts);

/* ---------------------------------------------------------------- batches
 * Many texts, each under its own compiled RE, parsed together: the texts
 * that share a handle form a group, and every phase of a group is one kernel
 * launch over all its texts (reach tiles of 32 chunks, chunks, and merge
 * tiles of 32 column groups, handed out by device work counters), instead of
 * one launch per phase and text.  Results are those of re_parse on each text
 * (Sect. 3.2); the chunk length of each text is chosen from its length and
 * its group's total length (re_batch_chunk_len reports it).
 *
 * Use: re_batch_plan (host only; sizes, chunk lengths, a pinned descriptor
 * buffer) -> re_batch_workspace_size -> re_parse_batch (binds text, output
 * and workspace pointers, encodes each text's tensor maps, uploads the
 * descriptors, enqueues the kernels) -> re_batch_run to parse the same bound
 * buffers again (kernels only, nothing copied) -> re_batch_free.
 * A batch of 64 MiB or more under several REs runs its groups on up to four
 * streams of its own, forked from and joined back into the caller's stream
 * by events (a CUDA graph capture of the call captures them too).           */
typedef struct re_batch re_batch;       /* opaque: a planned batch */

/* Plan count texts: text j has lens[j] bytes and is parsed under hs[j] (all
 * handles on the current device).  opts->kind is the encoding for every text
 * (AUTO resolved per handle); opts->chunk_len, if not 0, fixes every chunk
 * length; RE_PARSE_RECOGNIZE_ONLY is honoured; phase events are not.
 * *out owns a pinned host buffer until re_batch_free.                       */
re_status re_batch_plan(re_handle *const *hs, const uint64_t *lens, uint32_t count, const re_parse_opts *opts,
                        re_batch **out);

/* Device workspace the batch needs (descriptors + every text's workspace). */
re_status re_batch_workspace_size(const re_batch *b, uint64_t *bytes);

/* Chunk length chosen for text j.                                          */
re_status re_batch_chunk_len(const re_batch *b, uint32_t j, uint32_t *k);

/* Enqueue the parse of every text: d_texts[j] (16-byte aligned device bytes
 * of lens[j]), outs[j] laid out like re_parse's output (kind = the planned
 * encoding, col_bytes from re_slpf_layout, a status word per text).  The
 * workspace (256-byte aligned, re_batch_workspace_size bytes) is caller
 * owned and bound to the batch until the next re_parse_batch.  Copies the
 * descriptors from the plan's pinned buffer on the stream; a later call on the
 * same plan first waits for that copy.  Asynchronous otherwise.              */
re_status re_parse_batch(re_batch *b, const uint8_t *const *d_texts, re_slpf *outs, void *d_workspace,
                         uint64_t workspace_bytes, re_stream stream);

/* Enqueue the kernels of the last re_parse_batch again, over the same bound
 * text, output and workspace buffers (their contents may have changed).
 * Only kernel launches: no copy, no allocation, no host synchronisation.    */
re_status re_batch_run(re_batch *b, re_stream stream);

/* Free the plan (waits for its last descriptor copy).                      */
void re_batch_free(re_batch *b);

/* Size of the library-owned device scratch used by re_parse_static: 64 MiB,
 * enough for texts up to about 8 MiB with automatic chunking (about 0.54
 * byte of workspace per text byte for texts of 256 MiB, more for short ones,
 * whose chunks are shorter; re_workspace_size gives the exact figure).      */
#define RE_STATIC_SCRATCH_BYTES (64u << 20)

/* re_parse without a caller workspace and without any allocation.  The paper
 * has no counterpart: this is a deployment variant of re_parse, for callers
 * that cannot allocate device memory when they parse -- a C host program with
 * no device allocator of its own, or a request loop that must not call
 * cudaMalloc / cudaFree between launches, since those may synchronise the
 * whole device and stall every other stream.
 *
 * The workspace is one fixed device array of RE_STATIC_SCRATCH_BYTES per
 * device, owned by the library.  Arguments, results and errors are those of
 * re_parse, plus:
 *   - RE_E_CAPACITY (nothing enqueued) when re_workspace_size(h, len, opts)
 *     exceeds RE_STATIC_SCRATCH_BYTES; re_last_error() gives both sizes;
 *   - RE_E_CUDA when the scratch address cannot be resolved.
 * The first call on each device resolves that address (cudaGetSymbolAddress)
 * with the device current; make that first call before any stream capture.
 * The address is kept for the life of the process and belongs to the device's
 * primary context (the one the CUDA runtime uses): it is not valid in another
 * context, nor after cudaDeviceReset.  A text that fits only with the
 * built-in chunk-length rule, not with a length re_autotune chose, is parsed
 * with the rule's length (as re_parse does when its workspace is too small
 * for the tuned layout).
 * Every call on a device shares the one scratch: calls whose work can overlap
 * on the device (different streams with no ordering between them, or several
 * host threads) race and corrupt each other's results.  Successive calls on
 * one stream are ordered and safe.  The scratch needs no clearing between
 * calls.                                                                    */
re_status re_parse_static(re_handle *h, const uint8_t *d_text, uint64_t len, re_stream stream,
                          re_slpf *slpf, const re_parse_opts *opts);

/* ---------------------------------------------------------------- matches
 * Match extraction (Sect. 4.2, "Match extraction", getMatches): the spans of
 * a group.  A group is an operator node k of the numbered RE (its pair k( )k
 * in segment names); a match is a pair (i, j), i <= j, such that in some
 * syntax tree of the text the node k spans text[i:j] (bytes i .. j-1).
 * Computed from the clean SLPF by a visit along FolSeg arcs.
 *
 * re_matches reads the columns of a finished re_parse of a text of len
 * bytes (*slpf as given to that parse; its status word decides: a rejected
 * text has no matches) and writes up to cap_pairs pairs to d_pairs as
 * {i, j} uint64 pairs sorted by (i, j), and the total number of matches to
 * *d_count (device; it may exceed cap_pairs: call again with more room).
 * Enqueued on stream, asynchronous.  Supports at most 512 segments.
 * The visit from a start column follows the group until it closes, so a
 * group inside an ambiguous iteration (an ORF whose codon star also matches
 * stop codons) can have a number of matches, and a cost, quadratic in the
 * text length.
 * d_workspace: re_match_workspace_size bytes, 256-byte aligned.            */
re_status re_match_workspace_size(const re_handle *h, uint64_t len, uint64_t *bytes);
re_status re_matches(re_handle *h, const re_slpf *slpf, uint64_t len, uint32_t group, uint64_t *d_pairs,
                     uint64_t cap_pairs, uint64_t *d_count, void *d_workspace, uint64_t workspace_bytes,
                     re_stream stream);

/* Autotuner (no counterpart in the paper, which fixes c to the thread
 * count).  Parses d_text[0..len) with every reach shape the automaton can
 * run (RE_PARSE_REACH: lanes per chunk, table kind, TMA staging depth) and
 * candidate chunk lengths around the built-in rule's choice (1/2x to 2x,
 * multiples of 64, those whose workspace fits workspace_bytes), one warm-up
 * and two timed runs each on stream, and keeps the fastest (shape, length)
 * for this handle (so for its |Q|), the length bucket floor(log2(len)) and
 * recognizer mode: later re_parse / re_workspace_size calls with chunk_len 0
 * and no shape flag use it (re_parse falls back to the rule's length if the
 * workspace given is too small for it).  Blocks until the timing runs
 * finish; *slpf is overwritten.  *chunk_len receives the chosen length.    */
re_status re_autotune(re_handle *h, const uint8_t *d_text, uint64_t len, re_slpf *slpf, void *d_workspace,
                      uint64_t workspace_bytes, re_stream stream, const re_parse_opts *opts, uint32_t *chunk_len);

/* What re_autotune kept for texts of len bytes (flags: 0 or
 * RE_PARSE_RECOGNIZE_ONLY): the chunk length and the reach shape
 * (RE_PARSE_REACH numbering); both 0 when nothing was tuned.               */
re_status re_tuned(const re_handle *h, uint64_t len, uint32_t flags, uint32_t *chunk_len, uint32_t *shape);

/* re_parse for a text in host memory: enqueue on stream the copy of
 * text[0..len) into d_text, the parse (as re_parse, into the device buffers
 * of *slpf and d_workspace), and the copies of the len + 1 columns into
 * host_cols and of the status word into *host_status.  Asynchronous: the
 * host buffers must stay valid until the stream reaches them, and should be
 * pinned (page-locked) for the copies to overlap other work; the host
 * results are valid once the stream has been synchronised.  Calls on
 * different streams with separate buffers overlap one text's copies with
 * another's kernels.  d_text: device, >= len bytes, 16-byte aligned;
 * host_cols: (len + 1) * slpf->col_bytes bytes, NULL in recognizer mode.   */
re_status re_parse_host(re_handle *h, const uint8_t *text, uint64_t len, void *host_cols, int32_t *host_status,
                        uint8_t *d_text, re_slpf *slpf, void *d_workspace, uint64_t workspace_bytes,
                        re_stream stream, const re_parse_opts *opts);

/* ---------------------------------------------------------------- sharded parse
 * One text split into contiguous slices x[a_r, b_r), r = 0 .. N-1, parsed
 * slice by slice, on different GPUs or one (Sect. 3.2: chunks depend on one
 * another only through the join, Eq. joiner).  Needs both classic DFAs below
 * 256 states (re_shard_map_size says whether).
 *  1. re_shard_map on every slice: reach, and the slice's chunk maps
 *     composed into its maps (bytes, on the device): fwd[S] is the forward
 *     state at b_r when it is S at a_r, bwd[S] the backward state at a_r
 *     when it is S at b_r (classic-DFA state ids, 0 the empty set).  The
 *     maps are exact for every state a text can bring to the slice's edges
 *     (the states after the byte before it, resp. after it).  With
 *     RE_SHARD_PREV the slice's first chunk speculates from the byte before
 *     it (d_text[-1] must be readable); without it the slice is the first
 *     and starts from I.  With RE_SHARD_NEXT the last chunk speculates from
 *     the byte after it (d_text[len]); without it the slice is the last and
 *     ends in F.  d_status receives RE_OK, RE_E_INTERNAL or RE_E_TIMEOUT.
 *  2. re_shard_entry (host) composes the maps of every slice, in order, into
 *     each slice's entry states (forward at a_r, backward at b_r) and the
 *     text's verdict; for a rejected text every forward entry state is 0.
 *  3. re_parse_slice on every slice with its entry states: the slice's
 *     len + 1 columns are columns a_r .. b_r of the whole text's SLPF, as
 *     re_parse lays them out (column b_r is also column 0 of slice r+1).
 * The maps are what the slices exchange: fwd_entries + bwd_entries bytes
 * each (an all-gather).  d_maps: device, fwd then bwd.  Workspace: as
 * re_parse (re_workspace_size of the slice's length).                      */
#define RE_SHARD_PREV 1u
#define RE_SHARD_NEXT 2u
re_status re_shard_map_size(const re_handle *h, uint32_t *fwd_entries, uint32_t *bwd_entries);
re_status re_shard_map(re_handle *h, const uint8_t *d_text, uint64_t len, uint32_t flags, re_stream stream,
                       void *d_workspace, uint64_t workspace_bytes, uint8_t *d_maps, int32_t *d_status);
re_status re_shard_entry(const re_handle *h, const uint8_t *maps, uint32_t count, uint32_t *entry,
                         uint32_t *entry_bwd, int32_t *accepted);
re_status re_parse_slice(re_handle *h, const uint8_t *d_text, uint64_t len, uint32_t entry, uint32_t entry_bwd,
                         re_stream stream, re_slpf *slpf, void *d_workspace, uint64_t workspace_bytes,
                         const re_parse_opts *opts);

/* Segment set of a state (host): bit q of words [0, W) is segment q.
 * forward: 1 for the forward automaton, 0 for the reverse one.             */
re_status re_state_bits(const re_handle *h, int32_t forward, uint32_t id, uint64_t *bits, uint32_t cap_words);

/* ---------------------------------------------------------------------------
 * SLPF compression (App. C, "SLPF compression").  App. C stores an SLPF as its
 * initial column and a table delta(C_{r-1}, x_r) = C_r, and rebuilds it by
 * running the table over the text.  A clean column can also depend on bytes
 * after r, so the archive adds an exception (r, C_r) wherever the table's
 * column differs, and a checkpoint column every `interval` positions so that
 * the rebuild runs in independent pieces (App. C's evenly spaced columns).
 * Columns are ids: DICT indices (re_dict_copy gives their segment sets), or
 * DENSE values; ids must be below 65535, the interval at most 65536.
 *
 * Archive layout (little-endian, every section 16-byte aligned): the header;
 * table u16[n_ids][256] (row v, byte a: the column after the first (v, a),
 * 0xFFFF if the pair never occurs); checkpoints u16[n_checkpoints] (C_0, C_K,
 * C_2K, ...); per piece the index of its first exception, u64[n_checkpoints
 * + 1]; exceptions u32[n_exceptions], ascending, each (offset of the column
 * in its piece) << 16 | id, none at a checkpoint column.                    */
typedef struct {
    uint32_t magic;           /* 0x46504C53 */
    uint32_t version;         /* 2 */
    uint64_t n;               /* text length: columns 0 .. n */
    uint32_t n_ids;           /* table rows: ids 0 .. n_ids - 1 */
    uint32_t interval;        /* K: a checkpoint every K columns */
    uint64_t n_exceptions;
    uint64_t n_checkpoints;   /* n / K + 1 */
} re_slpf_dfa_header;

/* Host: build the archive of columns cols[0 .. len] (host memory, col_bytes
 * 1, 2 or 4 per id) of the host text[0 .. len).  *size receives the archive's
 * byte count; with cap below it nothing is written and RE_E_CAPACITY is
 * returned (cap = 0 queries the size).  The archive starts with the header. */
re_status re_slpf_dfa_encode(const void *cols, uint32_t col_bytes, const uint8_t *text, uint64_t len,
                             uint32_t interval, void *archive, uint64_t cap, uint64_t *size);

/* Device: rebuild columns 0 .. hdr->n into d_cols (col_bytes per id) from an
 * archive copied to device memory (16-byte aligned, archive_bytes long; hdr is
 * a host copy of its header) and the device text.  Asynchronous on stream;
 * *d_status becomes RE_OK, or RE_E_INTERNAL when the table has no entry for a
 * (column, byte) pair the text meets (an archive of another text).         */
re_status re_slpf_dfa_decode(const re_slpf_dfa_header *hdr, const void *d_archive, uint64_t archive_bytes,
                             const uint8_t *d_text, void *d_cols, uint64_t cols_cap_bytes, uint32_t col_bytes,
                             int32_t *d_status, re_stream stream);

/* ---------------------------------------------------------------------------
 * Request loop (no counterpart in the paper: a deployment layer over
 * re_parse and re_parse_batch).  A server keeps compiled REs resident and
 * runs a worker thread over `slots`, each with its own stream, device arena
 * and pinned staging buffers, allocated once.  Submitted requests wait in a
 * queue; while no more wait than slots are free each runs alone at once,
 * beyond that a free slot takes as many as fit (batches grow with the load);
 * the worker launches each
 * slot's requests as one re_parse or re_parse_batch with one copy in and one
 * copy out, and completes a request when its slot's event fires.  Results are
 * those of re_parse on each text alone.                                     */
typedef struct re_server re_server;

typedef struct {
    uint32_t slots;           /* concurrent launches (0 = 4) */
    uint64_t arena_bytes;     /* device bytes per slot: texts, columns, workspace (0 = 1 GiB) */
    uint64_t staging_bytes;   /* pinned host bytes per slot, for texts and again for columns (0 = arena / 2) */
    uint32_t max_batch;       /* requests per launch (0 = 4096) */
} re_server_opts;

/* Start a server over count compiled REs (all on the current device; the
 * handles must outlive it).  Columns use each RE's AUTO encoding.           */
re_status re_server_create(re_handle *const *hs, uint32_t count, const re_server_opts *opts, re_server **out);

/* Queue the parse of host text[0 .. len) under RE re_index.  Its columns (the
 * AUTO layout of re_slpf_layout, cols_cap bytes at least) and status word are
 * written to the host buffers cols and *status when it completes; text, cols
 * and status must stay valid until then.  *ticket identifies the request.
 * RE_E_CAPACITY: the request does not fit one slot's arena or staging.
 * Thread-safe.                                                               */
re_status re_server_submit(re_server *s, uint32_t re_index, const uint8_t *text, uint64_t len, void *cols,
                           uint64_t cols_cap, int32_t *status, uint64_t *ticket);

/* Block until request `ticket` is complete (timeout_ms < 0: no limit).
 * RE_E_TIMEOUT when the limit passes first.                                 */
re_status re_server_wait(re_server *s, uint64_t ticket, int32_t timeout_ms);

/* Tickets completed since the last call (at most cap of them; *n set), and
 * when done_ns is not NULL their completion times on the server clock.      */
re_status re_server_poll(re_server *s, uint64_t *tickets, uint64_t *done_ns, uint32_t cap, uint32_t *n);

/* The server clock: nanoseconds since re_server_create (steady).           */
uint64_t re_server_clock_ns(const re_server *s);

/* stats[0..3]: launches, requests, largest batch, most slots in flight.     */
re_status re_server_stats(re_server *s, uint64_t *stats);

/* Finish every queued request, stop the worker and free the server.        */
void re_server_destroy(re_server *s);

/* Thread-local description of the last error returned on this thread.     */
const char *re_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SLPF_PARSER_H */
