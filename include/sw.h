/*
 * sw.h - exact reset threshold and least shortest reset word of a
 * deterministic finite complete automaton, on one GB300 GPU (sm_103a).
 *
 * The method is the bidirectional breadth-first search of Szykula and Zyzik,
 * "An Improved Algorithm for Finding the Shortest Synchronizing Words"
 * (arXiv 2207.05495), Section 2.1 and Alg. 1: a forward search from Q over
 * images delta(S, a), an inverse search from the singletons over preimages
 * delta^{-1}(S, a), every level deduplicated against all sets seen before in
 * its direction, and after every step the meet condition "some forward set
 * X lies inside some backward set Y" (Section 2), which proves a reset word
 * of length (forward depth) + (backward depth).
 *
 * Conventions shared by every entry point:
 *  - An automaton has n states (1 <= n <= SW_MAX_STATES) and k letters
 *    (1 <= k <= SW_MAX_LETTERS).  Its transition table `delta` is int32
 *    [k][n], letter-major: delta[a*n + q] = delta(q, a) (Section 1).
 *  - r is the reset threshold, the length of the shortest reset words
 *    (Section 1).  The word returned is the lexicographically least reset
 *    word of length r, letters as indices 0..k-1 (the paper does not fix a
 *    tie-break; this is the library's reading).  n = 1 gives r = 0.
 *  - Level i of a direction is the list of distinct sets first reached at
 *    depth i: forward, images delta(Q, w) with |w| = i; backward, nonempty
 *    preimages delta^{-1}({q}, w).  Empty preimages are dropped.
 *  - `stream` is a cudaStream_t (for example torch.cuda.current_stream()
 *    .cuda_stream); NULL is the legacy default stream.  Every call is
 *    synchronous: it returns after its work on `stream` has finished.
 *  - `workspace` is caller-owned device memory of `ws_bytes` bytes (for
 *    example a torch uint8 tensor); the library keeps no pointer to it after
 *    the call returns and never frees it.  Its base must be 256-byte
 *    aligned.  Everything the search stores (levels, parent links, the
 *    deduplication hash table, candidates) lives in it; when it is too small
 *    the call fails with SW_ENOMEM and the caller may retry with more.
 *  - Return value: SW_OK (0) or one of the SW_E* codes below; the same code
 *    is kept as the calling thread's sw_last_error().
 *  - Handles are host objects.  One handle must not be used by two calls at
 *    the same time; different handles may.
 */
#ifndef SW_H
#define SW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SW_MAX_STATES 576
#define SW_MAX_LETTERS 255
#define SW_BEAM_MAX_STATES 8192

enum sw_status {
    SW_OK = 0,
    SW_EINVAL = 1,      /* an argument is out of range or a pointer is NULL */
    SW_ENOTSYNC = 2,    /* the automaton is not synchronizing */
    SW_ENOMEM = 3,      /* the workspace (or a table in it) is too small */
    SW_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
    SW_EWORDCAP = 5,    /* r exceeds the word capacity; r is still written */
    SW_ECUDA = 6,       /* a CUDA runtime call failed */
    SW_EBUSY = 7,       /* server: no room for the request right now */
    SW_EAGAIN = 8,      /* server: no finished request to report */
    SW_EINTERNAL = 9,   /* a self-check of a result failed */
    SW_ENOTFOUND = 10   /* sw_beam: no reset word within max_depth levels */
};

typedef struct sw_automaton *sw_handle;

/*
 * Validates and copies an automaton (Section 1) into a new host-side
 * handle.  delta: host int32 [k][n], read during the call only.  Checks
 * 1 <= n <= SW_MAX_STATES, 1 <= k <= SW_MAX_LETTERS, every entry in [0, n),
 * and that the automaton is synchronizing by the pair test of Section 2
 * (every two states can be mapped to one state, O(k n^2) on the host).
 * Returns NULL on failure (sw_last_error(): SW_EINVAL or SW_ENOTSYNC).
 * Release with sw_free.
 */
sw_handle sw_load_automaton(int32_t n, int32_t k, const int32_t *delta);

/* Releases a handle (NULL is ignored). */
void sw_free(sw_handle h);

/* The status of the calling thread's last failing call (SW_OK if none). */
int32_t sw_last_error(void);

/* A static description of a status code. */
const char *sw_error_string(int32_t code);

/*
 * Smallest workspace in bytes with which a search of `count` automata of
 * at most n_max states and k_max letters can start (it may still need more
 * as its levels grow).
 */
size_t sw_workspace_min_bytes(int32_t n_max, int32_t k_max, int32_t count);

/*
 * Reset threshold and least shortest reset word of one automaton by the
 * bidirectional search of Alg. 1 (Section 2.1) restricted to deletion of
 * duplicates and an equality history, with the meet test after every step
 * (Section 2).  r: host int32, written on SW_OK and on SW_EWORDCAP.
 * word: host uint8 [word_cap] or NULL; on SW_OK holds the r letters.
 * Errors: SW_EINVAL, SW_ENOMEM (workspace too small; retry with more),
 * SW_EWORDCAP (r > word_cap), SW_ECUDA, SW_EINTERNAL (the word failed its
 * on-device check |delta(Q, word)| = 1).
 */
int32_t sw_reset_threshold(sw_handle h, void *stream, void *workspace, size_t ws_bytes,
                           int32_t *r, uint8_t *word, int32_t word_cap);

/*
 * Allocation-free variant of sw_reset_threshold (the paper has no
 * counterpart; this is a library convenience).  Some callers cannot
 * allocate device memory when they call in: a process whose own allocator
 * has already reserved the whole GPU, a plugin loaded into a host program
 * that owns all device memory, or a service that forbids allocation after
 * start-up so that its memory use stays fixed.  This entry point needs no
 * workspace and calls no cudaMalloc, cudaMallocHost, cudaFree or other
 * allocating CUDA or PyTorch routine: its device scratch is one fixed array
 * of SW_STATIC_SCRATCH_BYTES (64 MiB) compiled into the library, which every
 * GPU that loads the library holds until the process exits.  Host-side
 * bookkeeping uses the C++ heap.
 *
 * Arguments, results and errors are those of sw_reset_threshold.  A search
 * that needs more than the scratch holds (its forward and backward levels,
 * their hash tables and one level of candidates: a few million sets for
 * W = 1, fewer for wider automata) fails with SW_ENOMEM ("workspace too
 * small"); use sw_reset_threshold with a larger workspace for those.
 *
 * The first call on each device looks up the scratch's device address
 * (cudaGetSymbolAddress) with that device current.  Under CUDA's lazy
 * module loading that lookup (or this library's first kernel launch) is
 * also when the device reserves the 64 MiB array, so a caller whose
 * allocator will later take the whole GPU must make its first call before
 * that allocator reserves memory: one call at start-up with any automaton
 * (a one-state automaton is enough) loads the module and fixes the address.
 * The call copies through pageable host memory and synchronises `stream`,
 * so it must not be called while `stream` is being captured into a CUDA
 * graph (nor, with a NULL stream, while any capture is in progress).  It
 * also gives up the overlap of the host's planning with the meet kernel
 * that sw_reset_threshold has: it is meant for callers that cannot
 * allocate, not for throughput.
 *
 * Every call on a device shares the one scratch array and starts by
 * re-initialising what it reads, so results never depend on an earlier
 * call; but two calls whose GPU work overlaps (different threads or streams
 * at the same time) race on it and must be serialised by the caller.
 * Every valid automaton passes the size check on entry (its starting state
 * is a few MiB at most); SW_ENOMEM comes from the search itself once its
 * levels and tables have filled the array.
 */
#define SW_STATIC_SCRATCH_BYTES (64u << 20)
int32_t sw_reset_threshold_static(sw_handle h, void *stream, int32_t *r, uint8_t *word,
                                  int32_t word_cap);

/*
 * Heuristic upper bound R >= r (Section 2.1.3, the cut-off inverse BFS the
 * paper cites, which it runs with beam size n log n up to n = 5000 in
 * Section 3).  Level 0 is the n singletons; level d + 1 is made of the
 * distinct nonempty preimages delta^{-1}(S, a) of the sets of level d
 * under every letter (candidate c = p*k + a for the set at position p;
 * among equal sets the smallest c stays), of which only the `beam` largest
 * are kept (ties: smaller c first), in candidate order.  No history is
 * kept.  R is the first depth at which Q itself is kept; the word y returned
 * satisfies delta^{-1}({q}, y) = Q, i.e. delta(Q, y) = {q}, and is checked
 * on the device.  Takes the automaton directly (n up to SW_BEAM_MAX_STATES,
 * beyond the exact search's SW_MAX_STATES; delta host int32 [k][n], not
 * checked for synchronizability).  workspace: caller-owned device memory,
 * 256-byte aligned; besides a few levels of candidates it holds one int64
 * per kept set of every level (for the word).  R: host; word: host uint8
 * [word_cap] or NULL.  Errors: SW_EINVAL, SW_ENOMEM (workspace too small),
 * SW_ENOTSYNC (a level became empty), SW_ENOTFOUND (no Q within max_depth
 * levels; a small beam can cycle), SW_EWORDCAP (R > word_cap; R is still
 * written), SW_ECUDA, SW_EINTERNAL (a table overflowed or the word failed
 * its check).
 */
int32_t sw_beam(int32_t n, int32_t k, const int32_t *delta, void *stream, void *workspace,
                size_t ws_bytes, int64_t beam, int32_t max_depth, int32_t *R, uint8_t *word,
                int32_t word_cap);

/*
 * Per-level sizes of the last search that included `h` (single or batched):
 * fwd[i] = size of forward level i for i < *nf, bwd[j] = size of backward
 * level j for j < *nb.  The search computes forward levels 0..i and
 * backward levels 0..j with i + j = r; which split it takes depends on the
 * direction rule, but every computed level's size is a property of the
 * automaton alone.  At most fwd_cap / bwd_cap entries are written; *nf and
 * *nb are the full counts.  Host pointers.  SW_EINVAL if h has not been
 * searched.
 */
int32_t sw_level_sizes(sw_handle h, int64_t *fwd, int32_t fwd_cap, int32_t *nf, int64_t *bwd,
                       int32_t bwd_cap, int32_t *nb);

/*
 * Batched search of `count` automata (Section 2.1, as sw_reset_threshold):
 * all instances advance together, one level per iteration, so that each
 * kernel launch serves every unfinished instance.  hs: host array of
 * handles.  r_out: host int32 [count]; r_out[i] = r of hs[i], or -1 if that
 * instance failed.  words: host uint8 [words_cap] or NULL; instance i's word
 * is written at words + word_off[i] and may use word_off[i+1] - word_off[i]
 * bytes (word_off: host int64 [count + 1], nondecreasing, word_off[count] <=
 * words_cap).  Returns SW_OK when every instance succeeded, else the first
 * failing instance's code (the others' results are still written).  When
 * the workspace cannot hold all instances at once, they are run in waves.
 */
int32_t sw_batch(const sw_handle *hs, int32_t count, void *stream, void *workspace,
                 size_t ws_bytes, int32_t *r_out, uint8_t *words, const int64_t *word_off,
                 int64_t words_cap);

/*
 * As sw_batch, with the automata and the results in device memory: d_delta
 * is device int32, instance i's table [k[i]][n[i]] starting at element
 * delta_off[i]; n, k, delta_off: host arrays [count].  d_r: device int32
 * [count]; d_words: device uint8 [words_cap] laid out by word_off (host
 * int64 [count + 1]) as in sw_batch.  The automata are not checked for
 * synchronizability up front; a non-synchronizing one ends with r = -1 and
 * SW_ENOTSYNC when one of its searches runs out of new sets.
 */
int32_t sw_batch_device(int32_t count, const int32_t *n, const int32_t *k,
                        const int32_t *d_delta, const int64_t *delta_off, void *stream,
                        void *workspace, size_t ws_bytes, int32_t *d_r, uint8_t *d_words,
                        const int64_t *word_off, int64_t words_cap);

/*
 * Counters of the calling thread's last search (sw_reset_threshold,
 * sw_batch or sw_batch_device), for throughput and roofline reporting.
 * Any pointer may be NULL.
 *   pairs:        (X, Y) pairs tested by the meet kernel (Section 2 meet
 *                 condition), excluding tiles skipped after a meet.
 *   candidates:   sets produced by the image/preimage kernel.
 *   iterations:   search iterations (each advances every unfinished
 *                 instance by one level).
 *   meet_ms, expand_ms, compact_ms: summed device time of those kernels,
 *                 from CUDA events on the search's stream (only when timing
 *                 was enabled by sw_set_timing(1)).
 *   meet_launches: launches of the meet kernel.
 *   launches:     launches of all of the library's kernels.
 *   waves:        waves the instances were run in (1 when all fitted).
 *   evictions:    instances set back to a later wave for lack of room.
 *   arena_peak:   most sets stored at once (all instances of a wave).
 *   and_iters:    warp-wide AND steps of the bitmap meet kernel (each ANDs
 *                 one state's bitmap over a backward chunk, 2048, 4096 or
 *                 8192 bits, into the running intersection).
 *   rows_transposed: backward sets transposed into per-state bitmaps by the
 *                 bitmap meet kernel (once per tile).
 *   words_ms:     device time of the word-recovery kernel (with timing on).
 *   run_ms:       host wall time of the whole search.
 *   sync_ms:      part of run_ms spent waiting for the stream; the rest is
 *                 host work between launches.
 *   select_ms, update_ms: host time choosing each iteration's jobs and
 *                 recording the levels they produced.
 *   meet_lane_words: 64-bit words of the running AND each lane holds in the
 *                 bitmap meet kernel of that search (1, 2 or 4; 0 when the
 *                 direct test ran), so that one AND step ANDs 64 *
 *                 meet_lane_words 32-bit words per warp.
 */
int32_t sw_last_stats(int64_t *pairs, int64_t *candidates, int32_t *iterations,
                      double *meet_ms, double *expand_ms, double *compact_ms,
                      int32_t *meet_launches, int64_t *launches, int32_t *waves,
                      int32_t *evictions, int64_t *arena_peak, int64_t *and_iters,
                      int64_t *rows_transposed, double *words_ms, double *run_ms,
                      double *sync_ms, double *select_ms, double *update_ms,
                      int32_t *meet_lane_words);

/*
 * Counters of the calling thread's last search's memory-bounded inverse
 * phase (sw_options.dfs_sets, Section 2.2): instances that ran it, chunks
 * of roots it expanded (each to its full depth), and sets it made (after
 * the duplicates of each chunk and depth).  Any pointer may be NULL.
 * Returns SW_OK.
 */
int32_t sw_last_dfs_stats(int64_t *instances, int64_t *chunks, int64_t *sets);

/*
 * Where the calling thread's last search spent the time between kernels
 * (no counterpart in the paper; the device figures need sw_set_timing(1)).
 *   stage_ms:  host time building and uploading each iteration's jobs, from
 *              the start of the iteration to its upload (the device waits);
 *   plan_ms:   host time planning the next iteration while the meet kernel
 *              runs (hidden behind it when the meet is longer);
 *   post_ms:   host time after each meet's results arrive: recording meets,
 *              recovering their words, retiring finished instances;
 *   table_ms:  device time from each job upload to the expansion kernel
 *              (the upload, the word recovery of the instances the previous
 *              meet found, hash-table fills and rehashing);
 *   gap_ms:    device time from the end of each meet kernel to the next
 *              iteration's job upload (copies and idle time).
 * Any pointer may be NULL.  Returns SW_OK.
 */
int32_t sw_last_host_stats(double *stage_ms, double *plan_ms, double *post_ms, double *table_ms,
                           double *gap_ms);

/*
 * Counters of the calling thread's last search with sw_options.reduce = 1
 * (the inclusion reductions of Alg. 1, Section 2.1).  mark_ms: device time
 * of the marking kernel (with timing on); mark_pairs: (set, set) pairs it
 * covered; mark_steps: its warp-wide AND steps; mark_rows: sets it
 * transposed into state bitmaps.  Any pointer may be NULL.
 */
int32_t sw_last_reduce_stats(double *mark_ms, int64_t *mark_pairs, int64_t *mark_steps,
                             int64_t *mark_rows);

/*
 * Calibration of the integer-logic peak the meet and marking kernels are
 * reported against (no counterpart in the paper).  Runs one CTA of 1024
 * threads per SM of the current device, each thread issuing independent
 * chains of three-input LOP3, and writes the LOP3 results retired per SM
 * clock cycle (timed with the SM's own cycle counter, so independent of
 * the clock rate).  workspace: device memory of at least 256 + 8 * SMs
 * bytes, 256-byte aligned.  Errors: SW_EINVAL, SW_ENOMEM, SW_ECUDA.
 */
int32_t sw_probe_int_peak(void *stream, void *workspace, size_t ws_bytes, double *lop3_per_clk_per_sm);

/*
 * ExpMark(As, Bs, Ad, Bd) of Section 2.1.2: the expected number of subset
 * checks of MarkSupersets over lists of As and Bs sets with densities Ad
 * and Bd (density = summed cardinality / (n * sets)), as the direction rule
 * dir_rule = 1 uses it.  Densities are clamped into (0, 1).  Host only.
 */
double sw_expmark(double a_s, double b_s, double a_d, double b_d);

/* Enables (1) or disables (0) per-kernel CUDA-event timing for later
 * searches on the calling thread. */
void sw_set_timing(int32_t on);

/*
 * Tunable parameters (all have defaults; values out of range are clamped).
 *   meet_algo:            0 = vertical bitmaps (default): the backward
 *                         chunk is transposed to one bitmap per state and a
 *                         forward set X meets set b iff bit b survives the AND
 *                         of the bitmaps of X's states; 1 = direct test
 *                         X & ~Y == 0 on every pair (LOP3).
 *   meet_rows_per_thread: direct test: forward sets each thread keeps in
 *                         registers (1, 2, 4 or 8; 0 = pick by word count).
 *   meet_b_tile:          direct test: backward sets per shared-memory tile
 *                         (even).
 *   meet_f_rows:          bitmap test: forward sets per tile (0 = 4096);
 *                         a launch with fewer than 8 predicted tiles per SM
 *                         halves it, down to 1024.
 *   meet_lane_words:      bitmap test: 0 = default chunk (4096 backward
 *                         sets for up to 192 states, and for up to 438
 *                         states when the bitmaps of the states that occur
 *                         fit in shared memory; else 2048); 4 = chunks of
 *                         8192 sets (up to 192 states only).
 *   dir_theta:            a forward step is taken when its predicted cost is
 *                         at most dir_theta times the backward step's.
 *   set_cost:             cost of producing one set, in pair tests (the
 *                         paper's SetCost, Section 2.1.2).
 *   reduce:               0 = duplicates and an equality history only (the
 *                         default; levels as described at the top of this
 *                         file, and the least reset word); 1 = the inclusion
 *                         reductions of Alg. 1 (Section 2.1) on both sides:
 *                         after the duplicates, every set that is not
 *                         minimal (BFS) / not maximal (IBFS) among its
 *                         level, and every superset (BFS) / subset (IBFS) of
 *                         a set kept at an earlier level of its direction,
 *                         is removed; 2 = the same on the BFS side only; 3 =
 *                         on the IBFS side only (the other side keeps the
 *                         equality history).  r is the same; a reduced
 *                         side's level sizes are those of its reduced lists
 *                         (a property of the automaton alone, as before);
 *                         with the BFS side reduced the word is a reset word
 *                         of length r: the parent chain of the first meeting
 *                         forward set of the reduced level, then the least
 *                         suffix, so it depends on the forward depth at
 *                         which the search met (sw_level_sizes gives it).
 *   table_cap_slots:      0 (default) or a cap on the slots of every hash
 *                         table, for testing: an instance whose table can
 *                         no longer take its sets fails alone with
 *                         SW_ENOMEM (its result r = -1 in a batch) while
 *                         the other instances of the call go on.
 *   dir_rule:             the meet term of the step costs (Section 2.1.2):
 *                         0 (default) the pair tests left after duplicates,
 *                         k (1 - r_dupl) |L| |other|; 1 the paper's ExpMark
 *                         estimate with the lists' densities (eq. 1 and 4).
 *                         The schedule never changes r, the word or the
 *                         level sizes.
 *   dfs_sets:             the memory-bounded inverse phase (Section 2.2,
 *                         built breadth-first per chunk instead of as a
 *                         depth-first recursion): 0 (default) off, an
 *                         instance whose next step does not fit ends with
 *                         SW_ENOMEM; -1 on when no step of the last active
 *                         instance fits; n > 0 also once an instance's
 *                         stored sets plus its next step's candidates would
 *                         exceed n.  The last forward level F_i stays fixed;
 *                         the last backward level B_j is cut into chunks
 *                         that are expanded D = 1, 2, ... inverse steps deep
 *                         (duplicates removed per chunk and depth, no
 *                         history) and checked against F_i; the first D with
 *                         a meet gives r = i + j + D.  r is exact; the word
 *                         is a reset word of length r, not necessarily the
 *                         least one; sw_level_sizes reports the levels of
 *                         the bidirectional phase only.
 * Applies to later searches on the calling thread.
 */
typedef struct sw_options {
    int32_t meet_algo;
    int32_t meet_rows_per_thread;
    int32_t meet_b_tile;
    int32_t meet_f_rows;
    int32_t meet_lane_words;
    double dir_theta;
    double set_cost;
    int32_t reduce;
    int32_t table_cap_slots;
    int32_t dir_rule;
    int64_t dfs_sets;
} sw_options;

void sw_get_options(sw_options *opt);
void sw_set_options(const sw_options *opt);

/*
 * Serving: continuous batching of searches (Section 2.1 per request, as
 * sw_reset_threshold).  A worker thread owns `stream` and the workspace
 * (caller-owned device memory, kept alive until sw_server_destroy).
 * Requests submitted while others are running join the running iterations:
 * between two iterations the worker admits waiting requests while the set
 * and table pools of the workspace are below half full, and every admitted
 * request advances one level per iteration in the same kernel launches as
 * the others.  Each search's levels and tables stay on the device until it
 * finishes; its result then goes to a completion queue.
 *
 * sw_server_create: n_max, k_max bound the automata that may be submitted;
 *   max_requests bounds requests held at once (queued + running + finished
 *   but not yet polled); word_cap is the longest word kept per request.
 * sw_server_submit: copies the automaton of h (h may be freed afterwards);
 *   non-blocking; SW_EBUSY when max_requests submissions are waiting.
 * sw_server_poll: non-blocking; SW_EAGAIN when no request has finished.
 *   On SW_OK: *req_id, *r (-1 if the search failed), *code (the request's
 *   own status: SW_OK, SW_ENOMEM, SW_EWORDCAP, ...), and when word is not
 *   NULL and *code is SW_OK the r letters of the least reset word.
 * sw_server_pending: counts of queued, running and finished-but-unpolled
 *   requests; returns SW_OK or the worker's fatal error (SW_ECUDA ...).
 * sw_server_destroy: stops the worker after its current iteration.
 */
typedef struct sw_server sw_server;

int32_t sw_server_create(void *workspace, size_t ws_bytes, int32_t n_max, int32_t k_max,
                         int32_t max_requests, int32_t word_cap, void *stream, sw_server **srv);
int32_t sw_server_submit(sw_server *srv, sw_handle h, uint64_t req_id);
int32_t sw_server_poll(sw_server *srv, uint64_t *req_id, int32_t *r, uint8_t *word,
                       int32_t word_cap, int32_t *code);
int32_t sw_server_pending(sw_server *srv, int32_t *queued, int32_t *active, int32_t *finished);

/*
 * Counters of a server since its creation (no counterpart in the paper;
 * they show that the batching is continuous).  admitted: requests admitted
 * into the engine; admitted_while_1 / admitted_while_2: those admitted
 * while at least one / at least two earlier searches were mid-run (their
 * levels on the device, between two iterations); max_active: the most
 * searches advanced by one iteration's launches; iterations: iterations
 * run.  Any pointer may be NULL.  SW_EINVAL if srv is NULL.
 */
int32_t sw_server_stats(sw_server *srv, int64_t *admitted, int64_t *admitted_while_1,
                        int64_t *admitted_while_2, int32_t *max_active, int64_t *iterations);
void sw_server_destroy(sw_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* SW_H */
