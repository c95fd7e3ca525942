// Host side of the GPU search: the C-ABI of include/sw.h, the workspace
// layout, and the level loop that drives the kernels of sw_kernels.cuh.
//
// One search runs any number of instances in lockstep: every iteration
// chooses a direction for each unfinished instance, expands that side by
// one level for all of them in one kernel (images forward, preimages
// backward, Alg. 1), deduplicates and compacts, then runs one meet check
// over all of them (Section 2), and recovers the words of the instances that
// met.  A single instance is the same loop with one member.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <set>
#include <new>
#include <vector>

#include "sw.h"
#include "sw_internal.h"
#include "sw_kernels.cuh"

using namespace sw;

struct sw_automaton {
    int32_t n = 0, k = 0;
    std::vector<uint16_t> delta16;  // [k][n]
    std::vector<int64_t> fwd_sizes, bwd_sizes;
    bool searched = false;
};

namespace {

struct Stats {
    int64_t pairs = 0, candidates = 0;
    int32_t iterations = 0;
    double meet_ms = 0, expand_ms = 0, compact_ms = 0, words_ms = 0, run_ms = 0;
    double sync_ms = 0;  // host time spent waiting for the stream inside the search
    double select_ms = 0, update_ms = 0;  // host: choosing jobs, recording new levels
    int32_t meet_launches = 0;
    int64_t and_iters = 0;  // bitmap meet: warp-wide AND steps
    int64_t rows_transposed = 0;  // bitmap meet: backward rows transposed into shared memory
    int64_t launches = 0;  // every kernel launch of the search
    int32_t waves = 0, evictions = 0;
    int64_t arena_peak = 0;  // most sets stored at once
    int32_t meet_lw = 0;     // bitmap meet: 64-bit words of the running AND per lane (0: direct test)
    double stage_ms = 0, plan_ms = 0, post_ms = 0;  // host: job staging, planning during the meet, after the meet
    double table_ms = 0;     // device: job upload, table fills and rehash before each expansion
    double gap_ms = 0;       // device: from a meet's end to the next iteration's job upload
    int64_t dfs_instances = 0, dfs_chunks = 0, dfs_sets = 0;  // inverse phase: instances, chunks, sets made
    double mark_ms = 0;      // inclusion reductions: device time of the marking kernel
    int64_t mark_pairs = 0, mark_steps = 0, mark_rows = 0;  // its pairs, AND steps, rows transposed
};

thread_local int32_t g_last_error = SW_OK;
thread_local sw_options g_opt = {0, 0, 0, 4096, 0, 1.0, 8192.0, 0, 0, 0, 0};
thread_local bool g_timing = false;
thread_local Stats g_stats;
// Set only while sw_reset_threshold_static runs: staging buffers then come
// from the C++ heap instead of cudaMallocHost.
thread_local bool g_pageable = false;

int32_t fail(int32_t code) {
    g_last_error = code;
    return code;
}

int words_for(int n) { return (n + 63) / 64; }

// ---------------------------------------------------------------- host checks

// Section 2: an automaton is synchronizing iff every pair of states can be
// mapped to one state.  Pairs are marked backwards from the diagonal through
// pairs of preimages (pre lists per letter), O(k n^2).
bool host_is_synchronizing(int n, int k, const int32_t *delta) {
    if (n == 1) return true;
    std::vector<int32_t> start((size_t)k * (n + 1), 0), pre((size_t)k * n);
    for (int a = 0; a < k; ++a) {
        int32_t *st = &start[(size_t)a * (n + 1)];
        for (int q = 0; q < n; ++q) st[delta[(size_t)a * n + q] + 1]++;
        for (int s = 0; s < n; ++s) st[s + 1] += st[s];
        std::vector<int32_t> fill(st, st + n);
        for (int q = 0; q < n; ++q) pre[(size_t)a * n + fill[delta[(size_t)a * n + q]]++] = q;
    }
    std::vector<uint8_t> mark((size_t)n * n, 0);
    std::vector<int32_t> queue;
    queue.reserve((size_t)n * n);
    for (int s = 0; s < n; ++s) {
        mark[(size_t)s * n + s] = 1;
        queue.push_back(s * n + s);
    }
    for (size_t h = 0; h < queue.size(); ++h) {
        int s = queue[h] / n, t = queue[h] % n;
        for (int a = 0; a < k; ++a) {
            const int32_t *st = &start[(size_t)a * (n + 1)];
            const int32_t *pa = &pre[(size_t)a * n];
            for (int i = st[s]; i < st[s + 1]; ++i)
                for (int j = st[t]; j < st[t + 1]; ++j) {
                    size_t pq = (size_t)pa[i] * n + pa[j];
                    if (!mark[pq]) {
                        mark[pq] = 1;
                        queue.push_back((int32_t)pq);
                    }
                }
        }
    }
    return queue.size() == (size_t)n * n;
}

// ---------------------------------------------------------------- pinned staging

struct Pinned {
    void *p = nullptr;
    size_t size = 0;
    std::vector<char> heap;  // used instead of pinned memory when g_pageable
    ~Pinned() {
        if (p) cudaFreeHost(p);
    }
    void *get(size_t bytes) {
        if (g_pageable) {
            if (heap.size() < bytes) heap.resize(std::max(bytes, 2 * heap.size()));
            return heap.data();
        }
        if (bytes > size) {
            if (p) cudaFreeHost(p);
            size_t s = std::max(bytes, size * 2);
            if (cudaMallocHost(&p, s) != cudaSuccess) {
                p = nullptr;
                size = 0;
                return nullptr;
            }
            size = s;
        }
        return p;
    }
};
thread_local Pinned g_up, g_down, g_words, g_wstat;

// ---------------------------------------------------------------- pool allocator

// Best-fit allocator over an index range [0, cap) of device slots (sets or
// table slots), kept on the host; freed ranges are coalesced.
struct Pool {
    int64_t cap = 0, used = 0;
    std::map<int64_t, int64_t> by_off;                 // free: offset -> length
    std::set<std::pair<int64_t, int64_t>> by_len;      // free: (length, offset)
    void init(int64_t c) {
        cap = c;
        used = 0;
        by_off.clear();
        by_len.clear();
        if (c > 0) {
            by_off[0] = c;
            by_len.insert({c, 0});
        }
    }
    int64_t alloc(int64_t n) {
        if (n < 1) n = 1;
        auto it = by_len.lower_bound({n, INT64_MIN});
        if (it == by_len.end()) return -1;
        int64_t len = it->first, off = it->second;
        by_len.erase(it);
        by_off.erase(off);
        if (len > n) {
            by_off[off + n] = len - n;
            by_len.insert({len - n, off + n});
        }
        used += n;
        return off;
    }
    void release(int64_t off, int64_t n) {
        if (n < 1 || off < 0) return;
        used -= n;
        auto next = by_off.lower_bound(off);
        if (next != by_off.end() && next->first == off + n) {
            n += next->second;
            by_len.erase({next->second, next->first});
            next = by_off.erase(next);
        }
        if (next != by_off.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                n += prev->second;
                by_len.erase({prev->second, prev->first});
                by_off.erase(prev);
            }
        }
        by_off[off] = n;
        by_len.insert({n, off});
    }
};

// ---------------------------------------------------------------- per-instance state

// kMet: a meet was found and the word is still being recovered; kDfs:
// waiting for the memory-bounded inverse phase
enum InstState { kWaiting = 0, kActive = 1, kDone = 2, kFailed = 3, kMet = 4, kDfs = 5 };

struct Level {
    int64_t off, cnt, cap;  // arena index, sets, slots reserved
    int64_t ge = -1;        // backward: its cardinality table (int32 index into the set pool), or -1
};

// A run of set slots owned by one instance; levels are bump-allocated in it.
struct Chunk {
    int64_t off, cap, used;
};

struct Inst {
    int32_t n = 0, k = 0, orig = 0;
    int64_t delta_off = 0;
    std::vector<Level> lev[2];
    std::vector<Chunk> chunks;
    int64_t tab_off[2] = {-1, -1}, tab_cap[2] = {0, 0}, stored[2] = {0, 0};
    double dupl[2] = {0.0, 0.0};
    double dens[2] = {1.0, 0.0};  // density (Section 2.1.2) of the last level of each side
    int32_t state = kWaiting, code = SW_OK, r = -1;
    int32_t evictions = 0;
    int64_t word_off = 0, word_cap = 0;    // where the word goes
    std::vector<int64_t> sizes[2];         // level sizes of the finished search
    int64_t footprint() const {
        int64_t b = 0;
        for (auto &c : chunks) b += c.cap;
        for (int d = 0; d < 2; ++d) b += tab_cap[d] / 4;  // a table slot is a quarter of a set (W = 1) or less
        return b;
    }
};

// ---------------------------------------------------------------- workspace layout

struct Layout {
    // staging mirror for per-iteration job uploads (one H2D copy per phase)
    char *mirror;
    size_t mirror_bytes;
    uint64_t *counts;    // per-job survivors
    uint64_t *card_sum;  // per-job summed cardinality of the new level
    int64_t *ntiles;   // meet tiles of the current iteration, then the bitmap kernel's tile counter
    unsigned long long *best;
    uint32_t *word_status;
    uint32_t *status;  // [0] flags of the last launches, [1 + i] flags of instance i
    int64_t status_n;
    unsigned long long *pairs;  // meet: [0] pairs tested, [1] bitmap AND steps, [2] rows transposed;
                                // marking: [3] AND steps, [4] rows transposed, [5] pairs
    uint8_t *word_area;
    int64_t word_area_cap;
    uint16_t *delta16;
    int64_t delta_cap;
    uint64_t *pre;            // preimage tables: [delta entry][W] bitsets
    uint32_t *hist, *cursor;  // per job: survivor cardinalities, bucket cursors
    int32_t *meta;            // the set pool as int32: backward levels' cardinality tables
    // pools
    uint64_t *sets, *link;
    uint32_t *perm;  // forward levels: canonical position of the i-th set by cardinality
    uint4 *rec;      // forward sets: first seven states and cardinality
    int64_t cap_sets;
    uint64_t *table;
    int64_t cap_table;
    // candidates of the running expansion
    uint64_t *cand_sets;
    int64_t *cand_slot;
    uint8_t *flag;
    uint32_t *block_cnt;
    uint64_t *block_off;
    int64_t cap_cand;
};

struct Carver {
    char *base;
    size_t size, used = 0;
    bool ok = true;
    Carver(void *b, size_t s) : base((char *)b), size(s) {}
    template <class T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
        if (used + bytes > size) {
            ok = false;
            return nullptr;
        }
        T *p = (T *)(base + used);
        used += bytes;
        return p;
    }
};

size_t mirror_bytes_for(int32_t count) { return (size_t)std::max(count, 1) * 4096 + (1 << 20); }
int64_t word_area_for(int32_t count) { return (int64_t)std::max<size_t>((size_t)std::max(count, 1) * 512, 1 << 20); }


size_t small_area_bytes(int32_t count, int64_t delta_elems, int W = 9) {
    size_t c = (size_t)std::max(count, 1);
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
    add(mirror_bytes_for(count));
    add(c * sizeof(uint64_t));
    add(c * sizeof(uint64_t));
    add(2 * sizeof(int64_t));
    add(c * sizeof(unsigned long long));
    add(c * sizeof(uint32_t));
    add((c + 1) * sizeof(uint32_t));
    add(6 * sizeof(unsigned long long));
    add((size_t)word_area_for(count));
    add((size_t)std::max<int64_t>(delta_elems, 1) * sizeof(uint16_t));
    add((size_t)std::max<int64_t>(delta_elems, 1) * W * sizeof(uint64_t));
    add(2 * c * card_slots(W) * sizeof(uint32_t));
    return b;
}

// Splits the workspace: small areas, then the set pool (set + link), the
// table pool and the candidate buffers, in proportions for W words.
bool carve(void *ws, size_t bytes, int W, int32_t count, int64_t delta_elems, Layout &L) {
    Carver cv(ws, bytes);
    size_t c = (size_t)std::max(count, 1);
    L.mirror_bytes = mirror_bytes_for(count);
    L.mirror = cv.take<char>(L.mirror_bytes);
    L.counts = cv.take<uint64_t>(c);
    L.card_sum = cv.take<uint64_t>(c);
    L.ntiles = cv.take<int64_t>(2);
    L.best = cv.take<unsigned long long>(c);
    L.word_status = cv.take<uint32_t>(c);
    L.status_n = (int64_t)c + 1;
    L.status = cv.take<uint32_t>(c + 1);
    L.pairs = cv.take<unsigned long long>(6);
    L.word_area_cap = word_area_for(count);
    L.word_area = cv.take<uint8_t>((size_t)L.word_area_cap);
    L.delta_cap = std::max<int64_t>(delta_elems, 1);
    L.delta16 = cv.take<uint16_t>((size_t)L.delta_cap);
    L.pre = cv.take<uint64_t>((size_t)L.delta_cap * W);
    L.hist = cv.take<uint32_t>(c * card_slots(W));
    L.cursor = cv.take<uint32_t>(c * card_slots(W));
    if (!cv.ok) return false;
    size_t rest = cv.size - cv.used;
    if (rest < 256 * 1024) return false;
    rest -= 16 * 1024;
    // bytes: sets 55%, table 25%, candidates 20%
    double set_b = 8.0 * W + 28, cand_b = 8.0 * W + 8 + 1 + 12.0 / kScanBlock;
    int64_t S = (int64_t)(0.55 * rest / set_b);
    int64_t T = (int64_t)(0.25 * rest / 8.0);
    int64_t C = (int64_t)(0.20 * rest / cand_b);
    C = std::min<int64_t>(C, (int64_t)0xF0000000) / kScanBlock * kScanBlock;
    if (S < 64 || T < 256 || C < kScanBlock) return false;
    int64_t nblocks = C / kScanBlock;
    L.sets = cv.take<uint64_t>((size_t)S * W);
    L.meta = (int32_t *)L.sets;  // cardinality tables live in set slots
    L.link = cv.take<uint64_t>((size_t)S);
    L.perm = cv.take<uint32_t>((size_t)S);
    L.rec = cv.take<uint4>((size_t)S);
    L.table = cv.take<uint64_t>((size_t)T);
    L.cand_sets = cv.take<uint64_t>((size_t)C * W);
    L.cand_slot = cv.take<int64_t>((size_t)C);
    L.flag = cv.take<uint8_t>((size_t)C);
    L.block_cnt = cv.take<uint32_t>((size_t)nblocks);
    L.block_off = cv.take<uint64_t>((size_t)nblocks + 1);
    if (!cv.ok) return false;
    L.cap_sets = S;
    L.cap_table = T;
    L.cap_cand = C;
    return true;
}

// Packs several job arrays into the pinned staging buffer and the device
// mirror so that one H2D copy moves them all.
struct Staging {
    char *host = nullptr, *dev = nullptr;
    size_t cap = 0, used = 0;
    bool ok = true;
    template <class T>
    T *take(size_t count, T **dev_ptr) {
        size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
        if (used + bytes > cap) {
            ok = false;
            return nullptr;
        }
        T *h = (T *)(host + used);
        *dev_ptr = (T *)(dev + used);
        used += bytes;
        return h;
    }
    bool fits(size_t more) const { return used + more + 256 * 8 <= cap; }
};

// ---------------------------------------------------------------- kernel dispatch

int g_sm_count = 0;
int sm_count() {
    if (!g_sm_count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 1;
    }
    return g_sm_count;
}

// rows per tile of the marking kernel
constexpr int kMarkRows = 4096;

int default_rows(int W) { return W == 1 ? 8 : (W <= 3 ? 4 : 2); }
int default_btile(int W) { return std::max(64, (4096 / W) & ~1); }

struct MeetCfg {
    int algo;     // 0 vertical bitmaps, 1 direct LOP3 test
    int lw;       // bitmap test: 64-bit words of the running AND per lane
    int R, tb, nt;
    int tf_rows;  // forward rows per tile (bitmap kernel)
    int n_cap;    // bitmap test: state bitmaps held (no automaton of the run has more states)
};

// Opt-in shared memory per block, bytes.
int max_smem_optin() {
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (v <= 0) v = 48 * 1024;
    }
    return v;
}

MeetCfg meet_cfg(int W, int n_max) {
    MeetCfg c;
    int R = g_opt.meet_rows_per_thread;
    if (R != 1 && R != 2 && R != 4 && R != 8) R = default_rows(W);
    if (W >= 3 && R == 8) R = 4;
    if (W <= 2 && R == 1) R = 2;
    c.R = R;
    int tb = g_opt.meet_b_tile > 0 ? g_opt.meet_b_tile : default_btile(W);
    tb = std::max(2, tb & ~1);
    int max_tb = (96 * 1024 / (8 * W)) & ~1;
    c.tb = std::min(tb, max_tb);
    c.nt = 256;
    c.algo = g_opt.meet_algo == 1 ? 1 : 0;
    c.n_cap = std::max(1, std::min(64 * W, n_max));
    c.lw = g_opt.meet_lane_words == 4 && W <= 3 ? 4 : bm_lanes_words(W);
    // wider sets: 4096-set chunks (1024 threads, one CTA per SM) whenever the
    // bitmaps of the states that occur fit in shared memory
    if (W >= 4 && W <= 7 && bm_smem_bytes_n(c.n_cap, 2) + 1024 <= max_smem_optin()) c.lw = 2;
    if (c.algo == 0) c.tb = 2048 * c.lw;
    c.tf_rows = g_opt.meet_f_rows > 0 ? g_opt.meet_f_rows : 4096;
    c.tf_rows = std::max(8, std::min(c.tf_rows, 1 << 20));
    return c;
}

template <int W, int R>
cudaError_t launch_meet_r(const MeetJob *jobs, int njobs, const int64_t *ntiles, int tb, const uint64_t *sets,
                          unsigned long long *best, unsigned long long *pairs, cudaStream_t st) {
    constexpr int NT = 256;
    auto kern = k_meet<W, R, NT>;
    size_t smem = (size_t)tb * 8 * W;
    static thread_local int configured_smem = 0;
    if ((int)smem > configured_smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured_smem = (int)smem;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    int64_t grid = (int64_t)sm_count() * std::max(per_sm, 1);
    kern<<<(unsigned)grid, NT, smem, st>>>(jobs, njobs, ntiles, tb, sets, best, pairs);
    return cudaGetLastError();
}

template <int W, int LW, int NT>
cudaError_t launch_meet_bm(const MeetJob *jobs, int njobs, int64_t *ntiles, int tf_rows, int n_cap, const uint64_t *sets,
                           const uint32_t *perm, const uint4 *rec, unsigned long long *best, unsigned long long *pairs, unsigned long long *iters,
                           unsigned long long *rows, const int32_t *meta, cudaStream_t st) {
    auto kern = k_meet_bm<W, LW, NT>;
    size_t smem = (size_t)bm_smem_bytes_n(n_cap, LW);
    static thread_local size_t configured = 0;
    if (configured < smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    int64_t grid = (int64_t)sm_count() * std::max(per_sm, 1);
    kern<<<(unsigned)grid, NT, smem, st>>>(jobs, njobs, ntiles, tf_rows, n_cap, sets, perm, rec, best, pairs, iters,
                                           rows, meta);
    return cudaGetLastError();
}

template <int W, int LW, int NT>
cudaError_t launch_mark_bm(const MarkJob *jobs, int njobs, int64_t *ntiles, int tr_rows, int n_cap, const Layout &L,
                           cudaStream_t st) {
    auto kern = k_mark_bm<W, LW, NT>;
    size_t smem = (size_t)bm_smem_bytes_n(n_cap, LW);
    static thread_local size_t configured = 0;
    if (configured < smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    int64_t grid = (int64_t)sm_count() * std::max(per_sm, 1);
    kern<<<(unsigned)grid, NT, smem, st>>>(jobs, njobs, ntiles, tr_rows, n_cap, L.sets, L.cand_sets, L.flag, L.meta,
                                           L.perm, L.pairs + 3);
    return cudaGetLastError();
}

template <int W>
struct Ops {
    static cudaError_t fill(const FillJob *j, int nj, int64_t maxlen, const Layout &L, cudaStream_t st) {
        for (int b = 0; b < nj; b += 65535) {
            dim3 grid((unsigned)std::min<int64_t>((maxlen + 255) / 256, 256), (unsigned)std::min(65535, nj - b));
            g_stats.launches++;
            k_fill<<<grid, 256, 0, st>>>(j + b, L.table);
        }
        return cudaGetLastError();
    }
    static cudaError_t roots(const RootJob *j, int nj, int nmax, const Layout &L, cudaStream_t st) {
        for (int b = 0; b < nj; b += 65535) {
            dim3 grid((unsigned)((nmax + 1 + 255) / 256), (unsigned)std::min(65535, nj - b));
            g_stats.launches++;
            k_roots<W><<<grid, 256, 0, st>>>(j + b, L.sets, L.link, L.perm, L.rec, L.table, L.status);
        }
        return cudaGetLastError();
    }
    static cudaError_t pre(const PreJob *j, int nj, int64_t maxlen, const Layout &L, cudaStream_t st) {
        for (int b = 0; b < nj; b += 65535) {
            dim3 grid((unsigned)std::min<int64_t>((maxlen * W + 255) / 256, 64), (unsigned)std::min(65535, nj - b));
            g_stats.launches += 2;
            k_pre_clear<W><<<grid, 256, 0, st>>>(j + b, L.pre);
            k_pre_fill<W><<<grid, 256, 0, st>>>(j + b, L.delta16, L.pre);
        }
        return cudaGetLastError();
    }
    static cudaError_t rehash(const RehashSeg *segs, int nseg, int64_t total, const Layout &L, cudaStream_t st) {
        int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 16);
        g_stats.launches++;
        k_rehash<W><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(segs, nseg, total, L.sets, L.table,
                                                                             L.status);
        return cudaGetLastError();
    }
    static cudaError_t expand(const ExpandJob *jobs, int nj, int64_t ncand, const Layout &L, cudaStream_t st) {
        int64_t blocks = std::min<int64_t>((ncand + 255) / 256, (int64_t)sm_count() * 16);
        g_stats.launches++;
        k_expand<W><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(
            jobs, nj, ncand, L.delta16, L.pre, L.sets, L.table, L.cand_sets, L.cand_slot, L.status);
        return cudaGetLastError();
    }
    // phase 0: the plain search; phase 2: after the reductions marked flags
    static cudaError_t compact(const ExpandJob *jobs, int nj, int64_t ncand, int phase, const Layout &L,
                               cudaStream_t st) {
        int64_t nblocks = ncand / kScanBlock;
        constexpr int HN = card_slots(W);
        g_stats.launches += 5;
        cudaError_t e = cudaMemsetAsync(L.hist, 0, (size_t)nj * HN * sizeof(uint32_t), st);
        if (e != cudaSuccess) return e;
        k_flag_count<W><<<(unsigned)nblocks, kScanThreads, 0, st>>>(jobs, nj, ncand, L.cand_slot, L.table,
                                                                    L.cand_sets, L.flag, L.block_cnt, L.hist, phase);
        k_scan_blocks<<<1, 1024, 0, st>>>(nblocks, L.block_cnt, L.block_off);
        k_ge<<<(unsigned)nj, 32, 0, st>>>(jobs, HN, L.hist, L.cursor, L.meta, L.card_sum);
        k_compact<W><<<(unsigned)nblocks, kScanThreads, 0, st>>>(jobs, nj, ncand, L.flag, L.block_off, L.cand_sets,
                                                                 L.cand_slot, L.table, L.sets, L.link, L.perm,
                                                                 L.rec, L.cursor);
        k_job_counts<<<(unsigned)((nj + 255) / 256), 256, 0, st>>>(jobs, nj, nblocks, L.block_off, L.counts);
        return cudaGetLastError();
    }
    // inclusion reductions: winners (phase 1), then the marking kernel
    // d_nt: device int64[2] = {mark tiles, 0 (the tile counter)}
    static cudaError_t mark(const ExpandJob *jobs, int nj, int64_t ncand, const MarkJob *mj, int nmj, int64_t *d_nt,
                            const MeetCfg &c, const Layout &L, cudaStream_t st) {
        int64_t nblocks = ncand / kScanBlock;
        g_stats.launches += 2;
        k_flag_count<W><<<(unsigned)nblocks, kScanThreads, 0, st>>>(jobs, nj, ncand, L.cand_slot, L.table,
                                                                    L.cand_sets, L.flag, L.block_cnt, L.hist, 1);
        if (nmj == 0) return cudaGetLastError();
        if constexpr (W >= 4 && W <= 7)
            if (c.lw == 2) return launch_mark_bm<W, 2, 1024>(mj, nmj, d_nt, kMarkRows, c.n_cap, L, st);
        return launch_mark_bm<W, bm_lanes_words(W), kBmThreads>(mj, nmj, d_nt, kMarkRows, c.n_cap, L, st);
    }
    // tf_rows: forward rows per tile of the bitmap kernel for this launch
    static cudaError_t meet(MeetJob *jobs, int nj, const MeetCfg &c, int tf_rows, const Layout &L, cudaStream_t st) {
        g_stats.launches += 2;
        const int64_t TF = c.algo == 0 ? (int64_t)tf_rows : (int64_t)c.nt * c.R;
        k_meet_prep<<<1, 1024, 0, st>>>(jobs, nj, L.counts, TF, c.tb, L.ntiles);
        int64_t *ntiles = L.ntiles;
        if (c.algo == 0) {
            // 8192-set chunks: one CTA per SM (200 KB of bitmaps at 192
            // states); 512 threads keep the walk's registers from spilling
            if constexpr (W <= 3)
                if (c.lw == 4)
                    return launch_meet_bm<W, 4, 512>(jobs, nj, ntiles, tf_rows, c.n_cap, L.sets, L.perm, L.rec,
                                                     L.best, L.pairs, L.pairs + 1, L.pairs + 2, L.meta, st);
            if constexpr (W >= 4 && W <= 7)
                if (c.lw == 2)
                    return launch_meet_bm<W, 2, 1024>(jobs, nj, ntiles, tf_rows, c.n_cap, L.sets, L.perm, L.rec,
                                                      L.best, L.pairs, L.pairs + 1, L.pairs + 2, L.meta, st);
            // 2048-set chunks of more than 438 states take more than half of
            // an SM's shared memory: one CTA per SM, so give it 1024 threads
            if constexpr (W >= 4)
                return launch_meet_bm<W, 1, 1024>(jobs, nj, ntiles, tf_rows, c.n_cap, L.sets, L.perm, L.rec,
                                                  L.best, L.pairs, L.pairs + 1, L.pairs + 2, L.meta, st);
            return launch_meet_bm<W, bm_lanes_words(W), kBmThreads>(jobs, nj, ntiles, tf_rows, c.n_cap, L.sets,
                                                                    L.perm, L.rec, L.best, L.pairs, L.pairs + 1,
                                                                    L.pairs + 2, L.meta, st);
        }
        switch (c.R) {
            case 1:
                if constexpr (W >= 3) return launch_meet_r<W, 1>(jobs, nj, ntiles, c.tb, L.sets, L.best, L.pairs, st);
                break;
            case 2: return launch_meet_r<W, 2>(jobs, nj, ntiles, c.tb, L.sets, L.best, L.pairs, st);
            case 4: return launch_meet_r<W, 4>(jobs, nj, ntiles, c.tb, L.sets, L.best, L.pairs, st);
            case 8:
                if constexpr (W <= 2) return launch_meet_r<W, 8>(jobs, nj, ntiles, c.tb, L.sets, L.best, L.pairs, st);
                break;
        }
        return cudaErrorInvalidValue;
    }
    static cudaError_t words(const WordJob *jobs, const int64_t *blevels, int nj, uint8_t *base, const Layout &L,
                             cudaStream_t st) {
        g_stats.launches++;
        k_words<W, 256><<<(unsigned)nj, 256, 0, st>>>(jobs, blevels, L.delta16, L.sets, L.link, L.meta, base,
                                                       L.word_status);
        return cudaGetLastError();
    }
};

struct OpTable {
    cudaError_t (*mark)(const ExpandJob *, int, int64_t, const MarkJob *, int, int64_t *, const MeetCfg &,
                        const Layout &, cudaStream_t);
    cudaError_t (*pre)(const PreJob *, int, int64_t, const Layout &, cudaStream_t);
    cudaError_t (*fill)(const FillJob *, int, int64_t, const Layout &, cudaStream_t);
    cudaError_t (*roots)(const RootJob *, int, int, const Layout &, cudaStream_t);
    cudaError_t (*rehash)(const RehashSeg *, int, int64_t, const Layout &, cudaStream_t);
    cudaError_t (*expand)(const ExpandJob *, int, int64_t, const Layout &, cudaStream_t);
    cudaError_t (*compact)(const ExpandJob *, int, int64_t, int, const Layout &, cudaStream_t);
    cudaError_t (*meet)(MeetJob *, int, const MeetCfg &, int, const Layout &, cudaStream_t);
    cudaError_t (*words)(const WordJob *, const int64_t *, int, uint8_t *, const Layout &, cudaStream_t);
};

template <int W>
OpTable make_ops() {
    return {&Ops<W>::mark, &Ops<W>::pre, &Ops<W>::fill, &Ops<W>::roots, &Ops<W>::rehash, &Ops<W>::expand, &Ops<W>::compact, &Ops<W>::meet,
            &Ops<W>::words};
}

OpTable ops_for(int W) {
    switch (W) {
        case 1: return make_ops<1>();
        case 2: return make_ops<2>();
        case 3: return make_ops<3>();
        case 4: return make_ops<4>();
        case 5: return make_ops<5>();
        case 6: return make_ops<6>();
        case 7: return make_ops<7>();
        case 8: return make_ops<8>();
        default: return make_ops<9>();
    }
}

// ---------------------------------------------------------------- timing

struct EventTimer {
    // 0..7: expansion, marking, compaction and meet bounds of an iteration;
    // 8: its job upload; 9, 10: the end of the meet of alternate iterations
    cudaEvent_t ev[11] = {};
    int64_t meets = 0;  // meets recorded so far (selects ev[9] or ev[10])
    bool made = false;
    void ensure() {
        if (!made) {
            for (auto &e : ev) cudaEventCreate(&e);
            made = true;
        }
    }
    ~EventTimer() {
        if (made)
            for (auto &e : ev) cudaEventDestroy(e);
    }
};
thread_local EventTimer g_ev;

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return SW_ECUDA; \
    } while (0)

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Slots of a hash table of `want` slots under sw_options.table_cap_slots
// (a cap for testing the overflow path; 0 = none).
int64_t capped_slots(int64_t want) {
    const int64_t cap = g_opt.table_cap_slots > 0 ? std::max<int64_t>(64, g_opt.table_cap_slots / 64 * 64) : 0;
    return cap > 0 ? std::min(want, cap) : want;
}

// cudaStreamSynchronize, with the wait added to the search's statistics.
cudaError_t wait_stream(cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaStreamSynchronize(st);
    g_stats.sync_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return e;
}

// ---------------------------------------------------------------- cost estimate

// ExpMark (Section 2.1.2): the expected number of subset checks of
// MarkSupersets(A, B) for lists of As and Bs sets of densities Ad and Bd,
// Bs ((1 + Bd) / Bd + 1 / (Ad - Ad Bd)) As^(log_w (1 + Bd)) with
// w = (1 + Bd) / (1 + Ad Bd - Ad).  Densities are clamped into (0, 1), where
// the formula is defined.
double expmark(double As, double Bs, double Ad, double Bd) {
    if (As <= 0 || Bs <= 0) return 0.0;
    const double lo = 1e-6, hi = 1.0 - 1e-6;
    Ad = std::min(std::max(Ad, lo), hi);
    Bd = std::min(std::max(Bd, lo), hi);
    const double w = (1.0 + Bd) / (1.0 + Ad * Bd - Ad);
    const double e = std::log1p(Bd) / std::log(w);
    return Bs * ((1.0 + Bd) / Bd + 1.0 / (Ad - Ad * Bd)) * std::pow(As, e);
}

// ---------------------------------------------------------------- the search engine

// Runs instances (state kWaiting, in `queue`) to completion.  Memory of an
// instance is released as soon as it finishes; when nothing can advance for
// lack of room, the instance holding the most memory is set back (its
// memory freed) and rerun after the current active set has drained.
struct Engine {
    int W;
    cudaStream_t st;
    Layout L;
    OpTable ops;
    MeetCfg mc;
    Pool set_pool, tab_pool;
    std::vector<Inst> &I;
    bool device_words = false;  // words go straight to the caller's device buffer
    uint8_t *out_words = nullptr;
    Staging stg;
    std::vector<int> active, deferred;
    // Inclusion reductions of Alg. 1 (sw_options.reduce 1: both sides, 2:
    // the BFS side, 3: the IBFS side): an expansion of a reduced side
    // deduplicates in a table of its own (released after the iteration),
    // and the marking kernel removes non-minimal (BFS) / non-maximal (IBFS)
    // sets and supersets / subsets of that side's history.  rdir[d]: side d
    // is reduced.
    bool reduce = false;
    bool rdir[2] = {false, false};

    // n_max: no instance the engine will run has more states
    Engine(int W_, int n_max, cudaStream_t s, std::vector<Inst> &insts, const Layout &lay)
        : W(W_), st(s), L(lay), I(insts) {
        rdir[0] = g_opt.reduce == 1 || g_opt.reduce == 2;
        rdir[1] = g_opt.reduce == 1 || g_opt.reduce == 3;
        reduce = rdir[0] || rdir[1];
        ops = ops_for(W);
        mc = meet_cfg(W, n_max);
        g_stats.meet_lw = mc.algo == 0 ? mc.lw : 0;
        set_pool.init(L.cap_sets);
        tab_pool.init(L.cap_table);
    }

    // Set slots of a cardinality table (int32[card_slots(W)]) kept in the set pool.
    int64_t ge_slots() const { return (card_slots(W) + 2 * W - 1) / (2 * W); }

    // A level of at least this many sets gets a chunk of its own, trimmed to
    // its survivors after compaction, instead of a chunk with room for more.
    static constexpr int64_t kBigLevel = int64_t(1) << 22;

    // n contiguous set slots for instance x: from the end of its last chunk,
    // else from a new chunk (at least four times n and twice the last chunk
    // when the pool allows, or exactly n for a big level); -1 when the pool
    // has no room.
    int64_t inst_alloc(Inst &x, int64_t n) {
        if (n < 1) n = 1;
        if (!x.chunks.empty()) {
            Chunk &c = x.chunks.back();
            if (c.cap - c.used >= n) {
                int64_t off = c.off + c.used;
                c.used += n;
                return off;
            }
        }
        int64_t grow = x.chunks.empty() ? 8 * ((int64_t)x.n + 1) : std::min(x.chunks.back().cap * 2, kBigLevel);
        int64_t want = n >= kBigLevel ? n : std::max<int64_t>(4 * n, grow);
        int64_t off = set_pool.alloc(want);
        if (off < 0) {
            want = n;
            off = set_pool.alloc(n);
        }
        if (off < 0) return -1;
        x.chunks.push_back({off, want, n});
        return off;
    }

    // Returns the unused end of x's most recent allocation [off, off + had);
    // a big level's own chunk gives that end back to the pool.
    void inst_shrink(Inst &x, int64_t off, int64_t had, int64_t keep) {
        Chunk &c = x.chunks.back();
        if (off + had != c.off + c.used) return;
        c.used -= had - keep;
        if (had >= kBigLevel && c.off == off && c.cap > c.used) {
            set_pool.release(c.off + c.used, c.cap - c.used);
            c.cap = c.used;
        }
    }

    bool stage_begin() {
        prestaged = false;
        stg.host = (char *)g_up.get(L.mirror_bytes);
        stg.dev = L.mirror;
        stg.cap = L.mirror_bytes;
        stg.used = 0;
        stg.ok = stg.host != nullptr;
        return stg.ok;
    }
    int stage_flush() {
        if (!stg.ok) return SW_ECUDA;
        if (stg.used) CK(cudaMemcpyAsync(stg.dev, stg.host, stg.used, cudaMemcpyHostToDevice, st));
        return SW_OK;
    }

    // The step-cost comparison of Section 2.1.2 (its one-step greedy rule):
    // the cost of a step is SetCost * k * |L| for making the sets plus the
    // cost of the meet check that follows.  dir_rule 0 counts the meet as
    // the pair tests left after duplicates, k (1 - r_dupl) |L| |other|;
    // dir_rule 1 estimates it with ExpMark (eq. 1 and 4, with the lists'
    // densities).  The side with the smaller cost (up to dir_theta) steps.
    int choose_dir(const Inst &x) const {
        double F = (double)x.lev[0].back().cnt, B = (double)x.lev[1].back().cnt, k = x.k;
        double cF, cB;
        if (g_opt.dir_rule == 1) {
            cF = g_opt.set_cost * k * F + expmark(k * (1.0 - x.dupl[0]) * F, B, x.dens[0], x.dens[1]);
            cB = g_opt.set_cost * k * B + expmark(F, k * (1.0 - x.dupl[1]) * B, x.dens[0], x.dens[1]);
        } else {
            cF = g_opt.set_cost * k * F + k * (1.0 - x.dupl[0]) * F * B;
            cB = g_opt.set_cost * k * B + k * (1.0 - x.dupl[1]) * B * F;
        }
        return cF <= g_opt.dir_theta * cB ? 0 : 1;
    }

    void release(Inst &x) {
        for (auto &c : x.chunks) set_pool.release(c.off, c.cap);
        x.chunks.clear();
        for (int d = 0; d < 2; ++d) {
            x.lev[d].clear();
            if (x.tab_off[d] >= 0) tab_pool.release(x.tab_off[d], x.tab_cap[d]);
            x.tab_off[d] = -1;
            x.tab_cap[d] = 0;
            x.stored[d] = 0;
        }
    }

    void finish(Inst &x, int state, int code) {
        for (int d = 0; d < 2; ++d) {
            x.sizes[d].clear();
            for (auto &l : x.lev[d]) x.sizes[d].push_back(l.cnt);
        }
        x.state = state;
        x.code = code;
        release(x);
    }

    // Stores the roots of as many of `ids` as fit; returns how many.
    int admit(const std::vector<int> &ids, size_t first, size_t *taken) {
        *taken = 0;
        if (!stage_begin()) return SW_ECUDA;
        std::vector<int> ok;
        size_t cap_jobs = (L.mirror_bytes / 2) / (sizeof(RootJob) + 2 * sizeof(FillJob) + sizeof(PreJob));
        for (size_t t = first; t < ids.size() && ok.size() < cap_jobs; ++t) {
            Inst &x = I[ids[t]];
            int64_t tc0 = 64, tc1 = capped_slots(round_up(4 * (int64_t)x.n, 64));
            x.chunks.clear();
            int64_t f = inst_alloc(x, 1);
            int64_t b = f >= 0 ? inst_alloc(x, x.n) : -1;
            int64_t t0 = b >= 0 ? tab_pool.alloc(tc0) : -1;
            int64_t t1 = t0 >= 0 ? tab_pool.alloc(tc1) : -1;
            if (t1 < 0) {
                for (auto &c : x.chunks) set_pool.release(c.off, c.cap);
                x.chunks.clear();
                if (t0 >= 0) tab_pool.release(t0, tc0);
                break;
            }
            for (int d = 0; d < 2; ++d) {
                x.lev[d].clear();
                x.dupl[d] = 0.0;
            }
            x.dens[0] = 1.0;                 // Q
            x.dens[1] = 1.0 / (double)x.n;   // the singletons
            x.lev[0].push_back({f, 1, 1, -1});
            x.lev[1].push_back({b, x.n, x.n, -1});
            x.tab_off[0] = t0;
            x.tab_cap[0] = tc0;
            x.tab_off[1] = t1;
            x.tab_cap[1] = tc1;
            x.stored[0] = 1;
            x.stored[1] = x.n;
            x.state = kActive;
            ok.push_back(ids[t]);
        }
        *taken = ok.size();
        if (ok.empty()) return SW_OK;
        int nj = (int)ok.size();
        RootJob *d_rj = nullptr;
        FillJob *d_fj = nullptr;
        PreJob *d_pj = nullptr;
        RootJob *rj = stg.take<RootJob>(nj, &d_rj);
        FillJob *fj = stg.take<FillJob>(2 * nj, &d_fj);
        PreJob *pj = stg.take<PreJob>(nj, &d_pj);
        if (!stg.ok) return SW_EINTERNAL;
        int64_t maxkn = 1;
        int nmax = 1;
        int64_t maxlen = 1;
        for (int t = 0; t < nj; ++t) {
            Inst &x = I[ok[t]];
            rj[t] = RootJob{x.lev[0][0].off, x.lev[1][0].off, {x.tab_off[0], x.tab_off[1]},
                            {x.tab_cap[0], x.tab_cap[1]}, x.n, ok[t]};
            fj[2 * t] = FillJob{x.tab_off[0], x.tab_cap[0]};
            fj[2 * t + 1] = FillJob{x.tab_off[1], x.tab_cap[1]};
            pj[t] = PreJob{x.delta_off, x.n, x.k};
            maxkn = std::max(maxkn, (int64_t)x.n * x.k);
            nmax = std::max(nmax, x.n);
            maxlen = std::max(maxlen, x.tab_cap[1]);
            active.push_back(ok[t]);
        }
        int rc = stage_flush();
        if (rc) return rc;
        CK(ops.pre(d_pj, nj, maxkn, L, st));
        CK(ops.fill(d_fj, 2 * nj, maxlen, L, st));
        CK(ops.roots(d_rj, nj, nmax, L, st));
        CK(wait_stream(st));  // the staging buffer is reused next
        return SW_OK;
    }

    // A planned step: instance id expands direction d into nc candidates;
    // its new level goes to dest (set pool), ge = its cardinality table
    // (backward) or -1, and new_tab/new_cap = the grown hash table or -1.
    struct Sel {
        int id, d;
        int64_t nc, dest, new_tab, new_cap, ge;
    };
    std::vector<Sel> pending;    // steps planned for the next iteration
    std::vector<char> planned;   // per instance: has a step in `pending`
    cudaEvent_t ev_counts = nullptr;

    ~Engine() {
        if (ev_counts) cudaEventDestroy(ev_counts);
    }

    // Plans the next step of every active instance that has none in `sel`
    // yet: chooses its direction and reserves candidates, table growth and
    // the new level's slots.  An instance whose step does not fit either way
    // is left out (it waits for an iteration).
    void plan(std::vector<Sel> &sel) {
        if (planned.size() < I.size()) planned.resize(I.size(), 0);
        int64_t ncand = 0;
        size_t seg_count = 0, mark_count = 0;
        for (const Sel &s : sel) {
            ncand += round_up(s.nc, kScanBlock);
            if (rdir[s.d]) mark_count += I[s.id].lev[s.d].size() + 1;
            else if (s.new_tab >= 0) seg_count += I[s.id].lev[s.d].size();
        }
        // staging bytes of the job arrays, checked before a table grows
        auto staging_fits = [&](size_t bytes) { return bytes + 256 * 8 <= L.mirror_bytes; };
        auto try_step = [&](int id, int d) -> bool {
            Inst &x = I[id];
            int64_t pc = x.lev[d].back().cnt;
            int64_t nc = pc * x.k;
            int64_t ncp = round_up(nc, kScanBlock);
            if (ncand + ncp > L.cap_cand) return false;
            size_t segs_here = 0;
            int64_t nt = -1, ntc = 0;
            if (rdir[d]) {
                // a table of this expansion's own (load <= 1/2), and room in
                // the staging buffer for its marking jobs
                if (!staging_fits((mark_count + x.lev[d].size() + 1) * sizeof(MarkJob) +
                                  (sel.size() + 2) * (sizeof(ExpandJob) + sizeof(FillJob) + sizeof(MeetJob))))
                    return false;
                ntc = capped_slots(round_up(2 * nc + 64, 64));
                nt = tab_pool.alloc(ntc);
                if (nt < 0) return false;
            } else if (2 * (x.stored[d] + nc) > x.tab_cap[d] && capped_slots(x.tab_cap[d] + 64) > x.tab_cap[d]) {
                // grow the table: load stays <= 1/2 (unless a cap forbids it)
                // to a load of 1/6 while small and the pool has room (fewer
                // rehashes, shorter probes), else to a load of 1/3
                const int64_t need = x.stored[d] + nc;
                segs_here = x.lev[d].size();
                if (!staging_fits((seg_count + segs_here) * sizeof(RehashSeg) + (sel.size() + 2) * sizeof(ExpandJob) +
                                  (sel.size() + 1) * (sizeof(FillJob) + sizeof(MeetJob))))
                    return false;
                if (need < (int64_t(1) << 22)) {
                    ntc = capped_slots(round_up(6 * need, 64));
                    nt = tab_pool.alloc(ntc);
                }
                if (nt < 0) {
                    ntc = capped_slots(round_up(3 * need, 64));
                    nt = tab_pool.alloc(ntc);
                }
                if (nt < 0) return false;
            }
            // the level's cardinality table (backward) and then the level
            // itself, last in the chunk so that its unused end can be returned
            int64_t ge = -1;
            if (d == 1) {
                int64_t gs = inst_alloc(x, ge_slots());
                if (gs >= 0) ge = gs * 2 * W;  // int32 index into the set pool
            }
            int64_t dest = inst_alloc(x, nc);
            if (dest < 0) {
                if (nt >= 0) tab_pool.release(nt, ntc);
                return false;
            }
            if (rdir[d]) {
                mark_count += x.lev[d].size() + 1;
            } else if (nt >= 0) {
                tab_pool.release(x.tab_off[d], x.tab_cap[d]);
                x.tab_off[d] = nt;
                x.tab_cap[d] = ntc;
                seg_count += segs_here;
            }
            sel.push_back({id, d, nc, dest, nt, ntc, ge});
            planned[id] = 1;
            ncand += ncp;
            return true;
        };
        for (int id : active) {
            if (planned[id] || I[id].state != kActive) continue;
            // a step that does not fit in memory counts as infinitely
            // expensive (Section 2.1.2), so the other direction is tried
            const int d = choose_dir(I[id]);
            if (g_opt.dfs_sets > 0) {
                // past the set budget the instance goes on with the inverse phase
                const Inst &x = I[id];
                if (x.stored[0] + x.stored[1] + x.k * x.lev[d].back().cnt > g_opt.dfs_sets) {
                    I[id].state = kDfs;
                    dfs_ids.push_back(id);
                    continue;
                }
            }
            if (!try_step(id, d)) try_step(id, 1 - d);
        }
    }

    // The job arrays of one iteration in the staging buffer (host side, for
    // patching before the upload, and the device addresses they go to).
    struct Staged {
        int nj = 0, n_mark = 0, nfill = 0, nsegs = 0, tf_rows = 0;
        int64_t ncand = 0, rehash_total = 0, maxfill = 1;
        bool marking = false;
        ExpandJob *jobs = nullptr, *d_jobs = nullptr;
        MeetJob *mj = nullptr, *d_mj = nullptr;
        FillJob *d_fill = nullptr;
        RehashSeg *d_segs = nullptr;
        MarkJob *d_mark = nullptr;
        int64_t *d_mark_nt = nullptr;
        FillJob *fills = nullptr;      // host side of the fills and rehash segments
        RehashSeg *segs = nullptr;
        std::vector<int> fill_owner;   // instance of each fill
    };
    // Word jobs staged with an iteration's jobs; their results are read
    // back with that iteration's level sizes.
    struct WordBatch {
        std::vector<WordJob> wj;
        WordJob *d_wj = nullptr;
        int64_t *d_bl = nullptr;
        int64_t area = 0;
        uint32_t *status = nullptr;  // host copy of the word statuses
        uint8_t *hwd = nullptr;      // host copy of the word area (host words)
    };
    // The steps planned while the last meet ran are staged at once (plain
    // searches); prestaged says that the staging buffer holds them.  Any
    // other use of the staging buffer clears it.
    Staged pre;
    bool prestaged = false;
    // Instances whose meet was found (state kMet) and whose words are still
    // to be recovered, with their best (f, b) keys.
    std::vector<int> met_ids;
    std::vector<unsigned long long> met_best;

    // Builds the job arrays of `sel` (steps of active instances) in the
    // staging buffer, without the upload.
    int build_stage(std::vector<Sel> &sel, Staged &S) {
        S = Staged{};
        if (!stage_begin()) return SW_ECUDA;
        // jobs, table fills and rehash segments: one upload
        const int nj = (int)sel.size();
        S.nj = nj;
        S.jobs = stg.take<ExpandJob>(nj, &S.d_jobs);
        if (!stg.ok) return SW_EINTERNAL;
        ExpandJob *jobs = S.jobs;
        std::vector<FillJob> fills;
        std::vector<RehashSeg> segs;
        int64_t cand = 0;
        for (int t = 0; t < nj; ++t) {
            Sel &s = sel[t];
            Inst &x = I[s.id];
            const Level &P = x.lev[s.d].back();
            ExpandJob &J = jobs[t];
            J.cand_off = cand;
            J.parent_off = P.off;
            J.parent_cnt = P.cnt;
            J.delta_off = x.delta_off;
            J.dest_off = s.dest;
            J.tab_off = rdir[s.d] ? s.new_tab : x.tab_off[s.d];
            J.tab_cap = rdir[s.d] ? s.new_cap : x.tab_cap[s.d];
            J.ge_off = s.ge;
            J.dir = s.d;
            J.n = x.n;
            J.k = x.k;
            J.inst = s.id;
            cand += round_up(s.nc, kScanBlock);
            if (rdir[s.d]) {
                fills.push_back({s.new_tab, s.new_cap});
                S.fill_owner.push_back(s.id);
                S.maxfill = std::max(S.maxfill, s.new_cap);
            } else if (s.new_tab >= 0) {
                fills.push_back({s.new_tab, s.new_cap});
                S.fill_owner.push_back(s.id);
                S.maxfill = std::max(S.maxfill, s.new_cap);
                for (auto &l : x.lev[s.d]) {
                    segs.push_back({S.rehash_total, l.off, l.cnt, s.new_tab, s.new_cap, s.d, s.id});
                    S.rehash_total += l.cnt;
                }
            }
        }
        S.ncand = cand;
        S.nfill = (int)fills.size();
        S.nsegs = (int)segs.size();
        if (!fills.empty()) {
            S.fills = stg.take<FillJob>(fills.size(), &S.d_fill);
            S.segs = stg.take<RehashSeg>(std::max<size_t>(segs.size(), 1), &S.d_segs);
            if (!stg.ok) return SW_EINTERNAL;
            std::memcpy(S.fills, fills.data(), fills.size() * sizeof(FillJob));
            if (!segs.empty()) std::memcpy(S.segs, segs.data(), segs.size() * sizeof(RehashSeg));
        }
        // inclusion reductions: per job a self-reduction job over its own
        // candidates and one job per kept level of its direction (the
        // history); the tiles of all of them are numbered in one range
        // the two-phase flags (winners, marks, survivors) are needed when
        // any job of this iteration expands a reduced side; the other jobs
        // get no marks, so phase 2 counts exactly their winners
        for (const Sel &sl : sel) S.marking |= rdir[sl.d];
        if (S.marking) {
            size_t cnt = 0;
            for (const Sel &sl : sel)
                if (rdir[sl.d]) cnt += I[sl.id].lev[sl.d].size() + 1;
            MarkJob *mk = stg.take<MarkJob>(std::max<size_t>(cnt, 1), &S.d_mark);
            int64_t *nt = stg.take<int64_t>(2, &S.d_mark_nt);
            if (!stg.ok) return SW_EINTERNAL;
            const int64_t kr = (int64_t)2048 * (mc.lw == 4 ? bm_lanes_words(W) : mc.lw);  // chunk rows
            int64_t tiles = 0;
            auto add = [&](int64_t r_off, int64_t r_cnt, int r_cand, int64_t c_off, int64_t c_cnt, int c_cand,
                           int64_t ge, int col, int self, int r_perm) {
                if (r_cnt <= 0 || c_cnt <= 0) return;
                MarkJob &M = mk[S.n_mark++];
                M.tile_off = tiles;
                M.ntc = (c_cnt + kr - 1) / kr;
                M.r_off = r_off;
                M.r_cnt = r_cnt;
                M.c_off = c_off;
                M.c_cnt = c_cnt;
                M.ge_off = ge;
                M.r_cand = r_cand;
                M.c_cand = c_cand;
                M.col = col;
                M.self = self;
                M.r_perm = r_perm;
                M.pad = 0;
                tiles += ((r_cnt + kMarkRows - 1) / kMarkRows) * M.ntc;
            };
            for (int t = 0; t < nj; ++t) {
                const Sel &sl = sel[t];
                if (!rdir[sl.d]) continue;
                const Inst &x = I[sl.id];
                const int64_t co = jobs[t].cand_off, cn = sl.nc;
                if (sl.d == 0) {
                    add(co, cn, 1, co, cn, 1, -1, 1, 1, 0);
                    // a forward level's permutation lists its sets by increasing cardinality
                    for (const Level &l : x.lev[0]) add(l.off, l.cnt, 0, co, cn, 1, -1, 1, 0, 1);
                } else {
                    add(co, cn, 1, co, cn, 1, -1, 0, 1, 0);
                    for (const Level &l : x.lev[1]) add(co, cn, 1, l.off, l.cnt, 0, l.ge, 0, 0, 0);
                }
            }
            nt[0] = tiles;
            nt[1] = 0;
        }
        // meet jobs: the size of the level each job produces is filled in on
        // the device (k_meet_prep), so the meet follows without a host sync
        S.mj = stg.take<MeetJob>(nj, &S.d_mj);
        if (!stg.ok) return SW_EINTERNAL;
        // A launch with few tiles gets shorter forward tiles (down to 1024
        // rows): more transposes, fewer idle SMs at its end.  The sizes of
        // the new levels are predicted from their last duplicate ratios.
        S.tf_rows = mc.tf_rows;
        if (mc.algo == 0 && S.tf_rows > 1024) {
            std::vector<std::pair<double, double>> fb((size_t)nj);
            for (int t = 0; t < nj; ++t) {
                const Sel &s = sel[t];
                const Inst &x = I[s.id];
                const double grown = (double)s.nc * (1.0 - x.dupl[s.d]);
                fb[t] = {s.d == 0 ? grown : (double)x.lev[0].back().cnt,
                         s.d == 1 ? grown : (double)x.lev[1].back().cnt};
            }
            auto tiles_for = [&](int tfr) {
                double n = 0;
                for (const auto &v : fb) n += std::ceil(v.first / tfr) * std::ceil(v.second / mc.tb);
                return n;
            };
            const double want = 8.0 * sm_count();
            while (S.tf_rows > 1024 && tiles_for(S.tf_rows) < want) S.tf_rows /= 2;
        }
        for (int t = 0; t < nj; ++t) {
            Sel &s = sel[t];
            Inst &x = I[s.id];
            MeetJob &M = S.mj[t];
            M.f_off = s.d == 0 ? s.dest : x.lev[0].back().off;
            M.f_cnt = s.d == 0 ? 0 : x.lev[0].back().cnt;
            M.b_off = s.d == 1 ? s.dest : x.lev[1].back().off;
            M.b_cnt = s.d == 1 ? 0 : x.lev[1].back().cnt;
            M.tile_off = 0;
            M.ntb = 1;
            M.slot = t;
            M.ge_off = s.d == 1 ? s.ge : x.lev[1].back().ge;
            M.upd = s.d;
            M.count_idx = t;
        }
        return SW_OK;
    }

    // Drops from staged jobs of a plain search, and from `sel`, the steps of
    // instances that are no longer active (they met or failed after the step
    // was planned; the memory planned for it stays with the instance until
    // it ends).  The other jobs keep their order, with candidate ranges,
    // level counts and rehash offsets renumbered.
    void drop_inactive(std::vector<Sel> &sel, Staged &S) {
        int w = 0;
        int64_t cand = 0;
        for (int t = 0; t < S.nj; ++t) {
            const Sel s = sel[t];
            if (I[s.id].state != kActive) {
                planned[s.id] = 0;
                continue;
            }
            ExpandJob J = S.jobs[t];
            J.cand_off = cand;
            cand += round_up(s.nc, kScanBlock);
            MeetJob M = S.mj[t];
            M.slot = w;
            M.count_idx = w;
            S.jobs[w] = J;
            S.mj[w] = M;
            sel[w] = s;
            ++w;
        }
        sel.resize((size_t)w);
        S.nj = w;
        S.ncand = cand;
        int f = 0;
        S.maxfill = 1;
        for (int t = 0; t < S.nfill; ++t) {
            if (I[S.fill_owner[t]].state != kActive) continue;
            S.fills[f] = S.fills[t];
            S.fill_owner[f] = S.fill_owner[t];
            S.maxfill = std::max(S.maxfill, S.fills[f].len);
            ++f;
        }
        S.nfill = f;
        int g = 0;
        int64_t total = 0;
        for (int t = 0; t < S.nsegs; ++t) {
            if (I[S.segs[t].inst].state != kActive) continue;
            RehashSeg r = S.segs[t];
            r.flat_off = total;
            total += r.cnt;
            S.segs[g++] = r;
        }
        S.nsegs = g;
        S.rehash_total = total;
    }

    // Stages word jobs for met[pos ..] (as many as the staging buffer holds;
    // when force_first, at least one) and advances pos.  An instance whose
    // word does not fit in its output ends here with its error.
    int stage_words(const std::vector<int> &met, const std::vector<unsigned long long> &best, size_t &pos,
                    WordBatch &wb, bool force_first) {
        std::vector<int64_t> blev;
        for (; pos < met.size(); ++pos) {
            Inst &x = I[met[pos]];
            int i = (int)x.lev[0].size() - 1, j = (int)x.lev[1].size() - 1;
            int r = i + j;
            x.r = r;
            if (r > x.word_cap) {
                finish(x, kFailed, SW_EWORDCAP);
                continue;
            }
            if (!device_words && r > L.word_area_cap) {
                finish(x, kFailed, SW_ENOMEM);
                continue;
            }
            size_t need = (wb.wj.size() + 1) * sizeof(WordJob) + (blev.size() + 3 * j) * sizeof(int64_t) + 1024;
            const bool room = stg.fits(need) && (device_words || wb.area + r <= L.word_area_cap);
            if (!room && !(force_first && wb.wj.empty())) break;
            WordJob J;
            J.f_arena = x.lev[0].back().off + (int64_t)(best[pos] >> 32);
            J.blev = (int64_t)(blev.size() / 3);
            J.word_off = device_words ? x.word_off : wb.area;
            J.delta_off = x.delta_off;
            J.i = i;
            J.j = j;
            J.n = x.n;
            J.k = x.k;
            J.slot = (int32_t)wb.wj.size();
            J.pad = met[pos];
            for (int m = 0; m < j; ++m) {
                blev.push_back(x.lev[1][m].off);
                blev.push_back(x.lev[1][m].cnt);
                blev.push_back(x.lev[1][m].ge);
            }
            if (!device_words) wb.area += r;
            wb.wj.push_back(J);
        }
        if (wb.wj.empty()) return SW_OK;
        const int nw = (int)wb.wj.size();
        WordJob *hw = stg.take<WordJob>(nw, &wb.d_wj);
        int64_t *hb = stg.take<int64_t>(std::max<size_t>(blev.size(), 3), &wb.d_bl);
        if (!stg.ok) return SW_EINTERNAL;
        std::memcpy(hw, wb.wj.data(), nw * sizeof(WordJob));
        if (!blev.empty()) std::memcpy(hb, blev.data(), blev.size() * sizeof(int64_t));
        return SW_OK;
    }

    // Queues the word kernel of a staged (and uploaded) batch and the copies
    // of its results.
    int launch_words(WordBatch &wb) {
        const int nw = (int)wb.wj.size();
        uint8_t *base = device_words ? out_words : L.word_area;
        if (g_timing) CK(cudaEventRecord(g_ev.ev[5], st));
        CK(ops.words(wb.d_wj, wb.d_bl, nw, base, L, st));
        if (g_timing) CK(cudaEventRecord(g_ev.ev[6], st));
        wb.status = (uint32_t *)g_wstat.get(nw * sizeof(uint32_t));
        if (!wb.status) return SW_ECUDA;
        CK(cudaMemcpyAsync(wb.status, L.word_status, nw * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        wb.hwd = nullptr;
        if (!device_words && wb.area > 0) {
            wb.hwd = (uint8_t *)g_words.get((size_t)wb.area);
            if (!wb.hwd) return SW_ECUDA;
            CK(cudaMemcpyAsync(wb.hwd, L.word_area, (size_t)wb.area, cudaMemcpyDeviceToHost, st));
        }
        return SW_OK;
    }

    // Once the stream has passed a batch's copies: every instance of it ends.
    void collect_words(WordBatch &wb) {
        if (g_timing) g_stats.words_ms += elapsed(g_ev.ev[5], g_ev.ev[6]);
        for (size_t t = 0; t < wb.wj.size(); ++t) {
            Inst &x = I[wb.wj[t].pad];
            if (wb.status[t] != 0) {
                finish(x, kFailed, SW_EINTERNAL);
                continue;
            }
            if (!device_words && out_words)
                std::memcpy(out_words + x.word_off, wb.hwd + wb.wj[t].word_off, (size_t)x.r);
            finish(x, kDone, SW_OK);
        }
        wb.wj.clear();
    }

    // Recovers the words of met instances now (batch by batch, waiting for each).
    int recover_words(const std::vector<int> &met, const std::vector<unsigned long long> &best) {
        size_t pos = 0;
        while (pos < met.size()) {
            if (!stage_begin()) return SW_ECUDA;
            WordBatch wb;
            int rc = stage_words(met, best, pos, wb, true);
            if (rc) return rc;
            if (wb.wj.empty()) continue;
            rc = stage_flush();
            if (rc) return rc;
            rc = launch_words(wb);
            if (rc) return rc;
            CK(wait_stream(st));
            collect_words(wb);
        }
        return SW_OK;
    }

    // ------------------------------------------------------------ DFS phase

    // Instances waiting for the memory-bounded inverse phase (state kDfs).
    std::vector<int> dfs_ids;

    // Runs the inverse phase of every waiting instance, one at a time.
    int run_dfs_pending() {
        std::vector<int> ids;
        ids.swap(dfs_ids);
        for (int id : ids) {
            if (I[id].state != kDfs) continue;  // its last meet found it first
            int rc = dfs_phase(id);
            if (rc) return rc;
        }
        return SW_OK;
    }

    // One chunk of the inverse phase: the roots B_j[c0, c0 + cs) are expanded
    // D inverse steps deep (duplicates removed per depth, in a table of each
    // expansion's own), and the depth-D sets are checked against F_i.
    // Returns SW_OK with *found set when they meet (the word is then
    // recovered and the instance ends), kDfsRetry when the chunk does not
    // fit (the caller halves it), or an error.
    static constexpr int kDfsRetry = -1;
    int dfs_chunk(Inst &x, int id, const Level &F, const Level &B, int64_t c0, int64_t cs, int D, bool *found) {
        *found = false;
        std::vector<Level> T;
        std::vector<std::pair<int64_t, int64_t>> set_allocs, tab_allocs;
        auto release_all = [&]() {
            for (auto &a : set_allocs) set_pool.release(a.first, a.second);
            for (auto &a : tab_allocs) tab_pool.release(a.first, a.second);
        };
        T.push_back({B.off + c0, cs, cs, -1});
        uint64_t *down = (uint64_t *)g_down.get(8 * sizeof(uint64_t));
        if (!down) return SW_ECUDA;
        for (int e = 1; e <= D; ++e) {
            const Level P = T.back();
            const int64_t nc = x.k * P.cnt;
            const int64_t ncp = round_up(nc, kScanBlock);
            if (ncp > L.cap_cand) {
                release_all();
                return kDfsRetry;
            }
            const int64_t tcap = capped_slots(round_up(2 * nc + 64, 64));
            const int64_t gs = set_pool.alloc(ge_slots());
            const int64_t dest = gs >= 0 ? set_pool.alloc(nc) : -1;
            const int64_t tab = dest >= 0 ? tab_pool.alloc(tcap) : -1;
            if (gs >= 0) set_allocs.push_back({gs, ge_slots()});
            if (dest >= 0) set_allocs.push_back({dest, nc});
            if (tab >= 0) tab_allocs.push_back({tab, tcap});
            if (tab < 0) {
                release_all();
                return kDfsRetry;
            }
            if (!stage_begin()) return SW_ECUDA;
            ExpandJob *d_job = nullptr;
            FillJob *d_fill = nullptr;
            ExpandJob *J = stg.take<ExpandJob>(1, &d_job);
            FillJob *fj = stg.take<FillJob>(1, &d_fill);
            if (!stg.ok) return SW_EINTERNAL;
            *J = ExpandJob{};
            J->cand_off = 0;
            J->parent_off = P.off;
            J->parent_cnt = P.cnt;
            J->delta_off = x.delta_off;
            J->dest_off = dest;
            J->tab_off = tab;
            J->tab_cap = tcap;
            J->ge_off = gs * 2 * W;
            J->dir = 1;
            J->n = x.n;
            J->k = x.k;
            J->inst = id;
            *fj = {tab, tcap};
            int rc = stage_flush();
            if (rc) return rc;
            CK(ops.fill(d_fill, 1, tcap, L, st));
            CK(ops.expand(d_job, 1, ncp, L, st));
            CK(ops.compact(d_job, 1, ncp, 0, L, st));
            CK(cudaMemcpyAsync(down, L.counts, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(down + 1, L.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            CK(wait_stream(st));
            g_stats.candidates += ncp;
            g_stats.dfs_sets += (int64_t)down[0];
            if ((uint32_t)(down[1] & 0xFFFFFFFFu) & kStatusTableFull) {
                // probes ran out in this expansion's table: a smaller chunk
                CK(cudaMemsetAsync(L.status, 0, (size_t)L.status_n * sizeof(uint32_t), st));
                CK(wait_stream(st));
                release_all();
                return kDfsRetry;
            }
            const int64_t c = (int64_t)down[0];
            T.push_back({dest, c, c, gs * 2 * W});
            if (c == 0) {  // no preimage of this depth: the chunk cannot meet at depth D
                release_all();
                return SW_OK;
            }
        }
        // the depth-D sets against F_i
        const Level &TD = T.back();
        if (!stage_begin()) return SW_ECUDA;
        MeetJob *d_mj = nullptr;
        MeetJob *M = stg.take<MeetJob>(1, &d_mj);
        if (!stg.ok) return SW_EINTERNAL;
        *M = MeetJob{};
        M->f_off = F.off;
        M->f_cnt = F.cnt;
        M->b_off = TD.off;
        M->b_cnt = TD.cnt;
        M->tile_off = 0;
        M->ntb = 1;
        M->slot = 0;
        M->ge_off = TD.ge;
        M->upd = -1;
        M->count_idx = 0;
        int rc = stage_flush();
        if (rc) return rc;
        CK(cudaMemsetAsync(L.best, 0xFF, sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(L.pairs, 0, 3 * sizeof(unsigned long long), st));
        CK(ops.meet(d_mj, 1, mc, mc.tf_rows, L, st));
        CK(cudaMemcpyAsync(down + 2, L.best, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(down + 3, L.pairs, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        CK(wait_stream(st));
        g_stats.meet_launches++;
        g_stats.pairs += (int64_t)down[3];
        g_stats.and_iters += (int64_t)down[4];
        g_stats.rows_transposed += (int64_t)down[5];
        if (down[2] == ~0ull) {
            release_all();
            return SW_OK;
        }
        // a meet at depth D: the word runs through F_i's parent chain, then
        // the chunk's levels T_{D-1} .. T_1 and the kept levels B_j .. B_0
        *found = true;
        const int i = (int)x.lev[0].size() - 1, j = (int)x.lev[1].size() - 1;
        x.r = i + j + D;
        if (!device_words && x.r > L.word_area_cap) {
            release_all();
            finish(x, kFailed, SW_ENOMEM);
            return SW_OK;
        }
        if (!stage_begin()) return SW_ECUDA;
        WordBatch wb;
        WordJob Jw;
        Jw.f_arena = F.off + (int64_t)(down[2] >> 32);
        Jw.blev = 0;
        Jw.word_off = device_words ? x.word_off : 0;
        Jw.delta_off = x.delta_off;
        Jw.i = i;
        Jw.j = j + D;
        Jw.n = x.n;
        Jw.k = x.k;
        Jw.slot = 0;
        Jw.pad = id;
        wb.wj.push_back(Jw);
        if (!device_words) wb.area = x.r;
        WordJob *hw = stg.take<WordJob>(1, &wb.d_wj);
        int64_t *hb = stg.take<int64_t>(3 * (size_t)(j + D), &wb.d_bl);
        if (!stg.ok) return SW_EINTERNAL;
        *hw = Jw;
        for (int m = 0; m <= j; ++m) {
            hb[3 * m] = x.lev[1][m].off;
            hb[3 * m + 1] = x.lev[1][m].cnt;
            hb[3 * m + 2] = x.lev[1][m].ge;
        }
        for (int e = 1; e < D; ++e) {
            hb[3 * (j + e)] = T[e].off;
            hb[3 * (j + e) + 1] = T[e].cnt;
            hb[3 * (j + e) + 2] = T[e].ge;
        }
        rc = stage_flush();
        if (rc) return rc;
        rc = launch_words(wb);
        if (rc) return rc;
        CK(wait_stream(st));
        release_all();
        collect_words(wb);
        return SW_OK;
    }

    // The memory-bounded inverse phase of Section 2.2 for one instance.  The
    // paper runs it as a depth-first recursion from each set of the last
    // inverse level, checking every set it visits against the last forward
    // level; here the same search runs breadth-first per chunk of roots,
    // depth by depth (D = 1, 2, ...), so that each depth is one expansion
    // launch over the whole chunk.  Correctness: a shortest reset word
    // x y z with |x| = i and |z| = j has delta(Q, x) in F_i and
    // delta^-1({q}, z) in B_j (both first reached at those depths, else a
    // shorter word would exist), and delta^-1(delta^-1({q}, z), y) contains
    // delta(Q, x); no smaller D can meet, for the same reason.
    int dfs_phase(int id) {
        Inst &x = I[id];
        x.state = kActive;
        g_stats.dfs_instances++;
        // no bidirectional step follows: the hash tables go back to the pool
        for (int d = 0; d < 2; ++d) {
            if (x.tab_off[d] >= 0) tab_pool.release(x.tab_off[d], x.tab_cap[d]);
            x.tab_off[d] = -1;
            x.tab_cap[d] = 0;
        }
        const Level F = x.lev[0].back();
        const Level B = x.lev[1].back();
        const int i = (int)x.lev[0].size() - 1, j = (int)x.lev[1].size() - 1;
        // r is at most (n^3 - n) / 6 (the Pin-Frankl bound) and the word cap
        const double pf = ((double)x.n * x.n * x.n - x.n) / 6.0 + 1.0;
        const int64_t rmax = (int64_t)std::min<double>({pf, (double)x.word_cap, 1e6});
        const int64_t dmax = rmax - i - j;
        for (int64_t D = 1; D <= dmax; ++D) {
            // roots per chunk: the chunk's deepest level (at most k^D sets
            // per root) must fit in the candidate buffer and in a quarter of
            // the free set slots (and within dfs_sets when that is set)
            double reach = std::pow((double)x.k, (double)D);
            double room = std::min((double)L.cap_cand, 0.25 * (double)(set_pool.cap - set_pool.used));
            if (g_opt.dfs_sets > 0) room = std::min(room, (double)g_opt.dfs_sets);
            int64_t cs = (int64_t)std::min<double>((double)B.cnt, std::floor(room / reach));
            if (cs < 1) cs = 1;
            for (int64_t c0 = 0; c0 < B.cnt;) {
                const int64_t n_here = std::min(cs, B.cnt - c0);
                bool found = false;
                int rc = dfs_chunk(x, id, F, B, c0, n_here, (int)D, &found);
                if (rc == kDfsRetry) {
                    if (n_here == 1) {  // not even one root fits
                        finish(x, kFailed, SW_ENOMEM);
                        return SW_OK;
                    }
                    cs = std::max<int64_t>(1, n_here / 2);
                    continue;
                }
                if (rc) return rc;
                g_stats.dfs_chunks++;
                if (found) return SW_OK;  // the instance has ended
                c0 += n_here;
            }
        }
        finish(x, kFailed, SW_EWORDCAP);
        return SW_OK;
    }

    // One iteration over the active instances.  The next iteration's steps
    // are planned, and for a plain search staged, on the host while this
    // iteration's meet kernel runs.  The words of the instances that meet
    // finds are recovered at the start of the next iteration, in the same
    // upload and ahead of its expansion (so between one meet and the next
    // expansion the host only drops the met instances' steps and uploads),
    // and end with that iteration's level sizes.  Instances sent to the
    // inverse phase by the planning run it at the start of an iteration (or
    // at once when no other instance is active).
    int iterate() {
        g_stats.iterations++;
        auto t_sel = std::chrono::steady_clock::now();
        // the allocation-free entry point (pageable staging) creates no CUDA
        // objects: it waits for the whole stream instead of a counts event
        const bool counts_event = !g_pageable;
        if (counts_event && !ev_counts) CK(cudaEventCreateWithFlags(&ev_counts, cudaEventDisableTiming));
        if (!dfs_ids.empty()) {
            int rc = run_dfs_pending();
            if (rc) return rc;
        }
        std::vector<Sel> sel;
        sel.swap(pending);
        // the staged jobs serve when every active instance has its step in them
        bool use_pre = prestaged;
        if (use_pre)
            for (int id : active)
                if (!planned[id]) use_pre = false;
        Staged S;
        if (use_pre) {
            S = pre;
            drop_inactive(sel, S);
        } else {
            // steps planned for instances that have since met or failed go,
            // with their memory (kept by the instance until it ends)
            sel.erase(std::remove_if(sel.begin(), sel.end(),
                                     [&](const Sel &s) {
                                         if (I[s.id].state == kActive) return false;
                                         planned[s.id] = 0;
                                         if (rdir[s.d]) tab_pool.release(s.new_tab, s.new_cap);
                                         return true;
                                     }),
                      sel.end());
            plan(sel);  // instances without a planned step: new, or skipped for room
        }
        for (const Sel &s : sel) planned[s.id] = 0;
        if (sel.empty()) {
            prestaged = false;
            int rc = met_ids.empty() ? SW_OK : recover_words(met_ids, met_best);
            met_ids.clear();
            met_best.clear();
            if (rc) return rc;
            // instances just sent to the inverse phase leave the active set and run it now
            active.erase(std::remove_if(active.begin(), active.end(), [&](int a) { return I[a].state != kActive; }),
                         active.end());
            rc = run_dfs_pending();
            if (rc) return rc;
            if (active.empty()) return SW_OK;
            // nothing fits: set back the instance holding the most memory
            auto it = std::max_element(active.begin(), active.end(),
                                       [&](int a, int b) { return I[a].footprint() < I[b].footprint(); });
            int id = *it;
            active.erase(it);
            Inst &x = I[id];
            g_stats.evictions++;
            if (active.empty()) {  // it had all the room there is
                if (g_opt.dfs_sets != 0 && x.state == kActive) {
                    int rc = dfs_phase(id);
                    if (rc) return rc;
                } else {
                    finish(x, kFailed, SW_ENOMEM);
                }
            } else {
                release(x);
                x.state = kWaiting;
                x.evictions++;
                deferred.push_back(id);
            }
            return SW_OK;
        }
        if (!use_pre) {
            int rc = build_stage(sel, S);
            if (rc) return rc;
        }
        prestaged = false;
        const int nj = S.nj;
        const int64_t ncand = S.ncand;
        const bool marking = S.marking;
        // the words of the instances the last meet found, in the same upload
        WordBatch wb;
        if (!met_ids.empty()) {
            size_t pos = 0;
            int rc = stage_words(met_ids, met_best, pos, wb, false);
            if (rc) return rc;
            met_ids.erase(met_ids.begin(), met_ids.begin() + (std::ptrdiff_t)pos);
            met_best.erase(met_best.begin(), met_best.begin() + (std::ptrdiff_t)pos);
        }
        if (g_timing) CK(cudaEventRecord(g_ev.ev[8], st));
        int rc = stage_flush();
        if (rc) return rc;
        if (!wb.wj.empty()) {
            rc = launch_words(wb);
            if (rc) return rc;
        }
        {
            const double ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_sel).count();
            g_stats.select_ms += ms;
            g_stats.stage_ms += ms;
        }
        g_stats.candidates += ncand;
        if (S.nfill) CK(ops.fill(S.d_fill, S.nfill, S.maxfill, L, st));
        if (S.nsegs) CK(ops.rehash(S.d_segs, S.nsegs, S.rehash_total, L, st));
        if (marking) CK(cudaMemsetAsync(L.pairs + 3, 0, 3 * sizeof(unsigned long long), st));
        if (g_timing) CK(cudaEventRecord(g_ev.ev[0], st));
        CK(ops.expand(S.d_jobs, nj, ncand, L, st));
        if (g_timing) CK(cudaEventRecord(g_ev.ev[1], st));
        if (marking) {
            CK(ops.mark(S.d_jobs, nj, ncand, S.d_mark, S.n_mark, S.d_mark_nt, mc, L, st));
            if (g_timing) CK(cudaEventRecord(g_ev.ev[7], st));
        }
        CK(ops.compact(S.d_jobs, nj, ncand, marking ? 2 : 0, L, st));
        if (g_timing) CK(cudaEventRecord(g_ev.ev[2], st));
        // the new levels' sizes and the status come back before the meet
        uint64_t *down = (uint64_t *)g_down.get((3 * nj + 8) * sizeof(uint64_t));
        if (!down) return SW_ECUDA;
        uint64_t *d_status = down + nj, *d_best = down + nj + 1, *d_pairs = down + 2 * nj + 1;
        uint64_t *d_mark_cnt = down + 2 * nj + 4;
        uint64_t *d_card_sum = down + 2 * nj + 8;
        if (marking) d_mark_cnt[0] = d_mark_cnt[1] = d_mark_cnt[2] = 0;
        CK(cudaMemcpyAsync(down, L.counts, nj * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(d_status, L.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(d_card_sum, L.card_sum, nj * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        if (counts_event) CK(cudaEventRecord(ev_counts, st));
        CK(cudaMemsetAsync(L.best, 0xFF, nj * sizeof(unsigned long long), st));
        if (marking) CK(cudaMemcpyAsync(d_mark_cnt, L.pairs + 3, 3 * sizeof(unsigned long long),
                                       cudaMemcpyDeviceToHost, st));
        CK(cudaMemsetAsync(L.pairs, 0, 3 * sizeof(unsigned long long), st));
        if (g_timing) CK(cudaEventRecord(g_ev.ev[3], st));
        CK(ops.meet(S.d_mj, nj, mc, S.tf_rows, L, st));
        if (g_timing) {
            CK(cudaEventRecord(g_ev.ev[4], st));
            CK(cudaEventRecord(g_ev.ev[9 + (g_ev.meets & 1)], st));
        }
        g_stats.meet_launches++;
        CK(cudaMemcpyAsync(d_best, L.best, nj * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(d_pairs, L.pairs, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        if (counts_event) {
            auto t0 = std::chrono::steady_clock::now();
            cudaError_t e = cudaEventSynchronize(ev_counts);
            g_stats.sync_ms +=
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            CK(e);
        } else {
            CK(wait_stream(st));
        }
        // the words queued ahead of this iteration are back: their instances end
        if (!wb.wj.empty()) collect_words(wb);
        if ((uint32_t)(*d_status & 0xFFFFFFFFu) & kStatusTableFull) {
            // a hash table could not take every set of an instance (its
            // probes ran out): that instance fails with SW_ENOMEM, the others
            // go on.  Its level of this iteration is incomplete, so neither
            // the level nor a meet of it is kept.
            CK(wait_stream(st));
            uint32_t *inst_flags = (uint32_t *)g_words.get((size_t)L.status_n * sizeof(uint32_t));
            if (!inst_flags) return SW_ECUDA;
            CK(cudaMemcpyAsync(inst_flags, L.status, (size_t)L.status_n * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                               st));
            CK(wait_stream(st));
            for (int id : active)
                if (I[id].state == kActive && (inst_flags[1 + id] & kStatusTableFull)) finish(I[id], kFailed, SW_ENOMEM);
            CK(cudaMemsetAsync(L.status, 0, (size_t)L.status_n * sizeof(uint32_t), st));
        }
        // new levels; return the unused tail of each destination.  A search
        // with an empty level has run out of new sets: not synchronizing (its
        // meet job has no tiles, so its memory can go at once)
        auto t_upd = std::chrono::steady_clock::now();
        for (int t = 0; t < nj; ++t) {
            Sel &s = sel[t];
            Inst &x = I[s.id];
            if (x.state != kActive) continue;  // met earlier, or failed above: its step was empty or is void
            int64_t c = (int64_t)down[t];
            inst_shrink(x, s.dest, s.nc, c);
            x.lev[s.d].push_back({s.dest, c, c, s.ge});
            x.dupl[s.d] = 1.0 - (double)c / (double)s.nc;
            if (c > 0) x.dens[s.d] = (double)d_card_sum[t] / ((double)x.n * (double)c);
            x.stored[s.d] += c;
            if (c == 0) finish(x, kFailed, SW_ENOTSYNC);
        }
        g_stats.update_ms +=
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_upd).count();
        // plan (and for a plain search stage) the next iteration while the
        // meet kernel runs; a step planned for an instance that meets now is
        // dropped next time
        auto t_plan = std::chrono::steady_clock::now();
        plan(pending);
        if (!pending.empty() && !rdir[0] && !rdir[1]) {
            rc = build_stage(pending, pre);
            if (rc) return rc;
            prestaged = true;
        }
        {
            const double ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_plan).count();
            g_stats.select_ms += ms;
            g_stats.plan_ms += ms;
        }
        CK(wait_stream(st));
        const auto t_post = std::chrono::steady_clock::now();
        if (g_timing) {
            // device time from the previous meet's end to this upload, and
            // from the upload to the expansion (fills, rehash)
            if (g_ev.meets > 0) g_stats.gap_ms += elapsed(g_ev.ev[9 + ((g_ev.meets - 1) & 1)], g_ev.ev[8]);
            g_ev.meets++;
            g_stats.table_ms += elapsed(g_ev.ev[8], g_ev.ev[0]);
            g_stats.expand_ms += elapsed(g_ev.ev[0], g_ev.ev[1]);
            if (marking) {
                g_stats.mark_ms += elapsed(g_ev.ev[1], g_ev.ev[7]);
                g_stats.compact_ms += elapsed(g_ev.ev[7], g_ev.ev[2]);
            } else {
                g_stats.compact_ms += elapsed(g_ev.ev[1], g_ev.ev[2]);
            }
            g_stats.meet_ms += elapsed(g_ev.ev[3], g_ev.ev[4]);
        }
        if (marking) {
            g_stats.mark_steps += (int64_t)d_mark_cnt[0];
            g_stats.mark_rows += (int64_t)d_mark_cnt[1];
            g_stats.mark_pairs += (int64_t)d_mark_cnt[2];
        }
        // this iteration's deduplication tables of reduced sides are done with
        for (const Sel &sl : sel)
            if (rdir[sl.d]) tab_pool.release(sl.new_tab, sl.new_cap);
        g_stats.pairs += (int64_t)d_pairs[0];
        g_stats.and_iters += (int64_t)d_pairs[1];
        g_stats.rows_transposed += (int64_t)d_pairs[2];
        for (int t = 0; t < nj; ++t) {
            Inst &x = I[sel[t].id];
            // an instance sent to the inverse phase while this meet ran keeps its meet
            if ((x.state != kActive && x.state != kDfs) || d_best[t] == ~0ull) continue;
            x.state = kMet;
            met_ids.push_back(sel[t].id);
            met_best.push_back(d_best[t]);
        }
        active.erase(std::remove_if(active.begin(), active.end(), [&](int id) { return I[id].state != kActive; }),
                     active.end());
        if (active.empty()) {
            // no iteration follows to carry the words: recover them now
            prestaged = false;
            rc = met_ids.empty() ? SW_OK : recover_words(met_ids, met_best);
            met_ids.clear();
            met_best.clear();
            if (rc) return rc;
            // finished instances took their memory, planned steps included, with them
            for (const Sel &s : pending) {
                planned[s.id] = 0;
                if (rdir[s.d]) tab_pool.release(s.new_tab, s.new_cap);
            }
            pending.clear();
            rc = run_dfs_pending();
            if (rc) return rc;
        }
        g_stats.arena_peak = std::max(g_stats.arena_peak, set_pool.used);
        g_stats.post_ms +=
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_post).count();
        return SW_OK;
    }

    // Runs every waiting instance to completion.
    int run() {
        std::vector<int> queue;
        for (size_t t = 0; t < I.size(); ++t) {
            Inst &x = I[t];
            if (x.state != kWaiting) continue;
            if (x.n == 1) {  // Q is already a singleton: r = 0
                x.r = 0;
                x.sizes[0] = {1};
                x.sizes[1] = {1};
                x.state = kDone;
                x.code = SW_OK;
                continue;
            }
            queue.push_back((int)t);
        }
        while (!queue.empty()) {
            g_stats.waves++;
            size_t first = 0;
            while (first < queue.size() || !active.empty()) {
                if (first < queue.size()) {
                    size_t taken = 0;
                    int rc = admit(queue, first, &taken);
                    if (rc) return rc;
                    first += taken;
                    if (active.empty() && taken == 0) {  // a single instance's roots do not fit
                        Inst &x = I[queue[first]];
                        x.state = kFailed;
                        x.code = SW_ENOMEM;
                        ++first;
                        continue;
                    }
                }
                if (active.empty()) continue;
                int rc = iterate();
                if (rc) return rc;
            }
            queue.swap(deferred);
            deferred.clear();
        }
        return SW_OK;
    }
};

int32_t common_w(const std::vector<Inst> &I) {
    int W = 1;
    for (auto &x : I) W = std::max(W, words_for(x.n));
    return W;
}

void store_sizes(sw_automaton *h, const Inst &x) {
    h->fwd_sizes = x.sizes[0];
    h->bwd_sizes = x.sizes[1];
    h->searched = true;
}

}  // namespace

// ---------------------------------------------------------------- serving

// Continuous batching: a worker thread owns the stream and one engine.  It
// moves submitted requests into the engine's queue, admits them while the
// set and table pools are below the admission budget, advances every
// admitted request by one level per iteration (all in the same launches),
// and posts finished requests to the completion queue.
struct sw_server {
    int W = 1, n_max = 1, k_max = 1, cap = 0, word_cap = 0;
    double admit_frac = 0.5;
    cudaStream_t st = nullptr;
    Layout L;
    sw_options opt;
    std::vector<Inst> slots;
    std::vector<int> free_slots;
    std::vector<uint64_t> req_of;
    std::vector<uint8_t> words;  // word_cap bytes per slot
    Pool delta_pool;
    std::unique_ptr<Engine> eng;
    // submitted, not yet taken by the worker
    struct Sub {
        uint64_t req;
        int32_t n, k;
        std::vector<uint16_t> delta;
    };
    std::deque<Sub> incoming;
    std::deque<int> queue;  // slots waiting for admission
    std::vector<uint16_t> staged_delta;
    struct Done {
        uint64_t req;
        int32_t r, code;
        std::vector<uint8_t> word;
    };
    std::deque<Done> done;
    std::mutex mu;
    std::condition_variable cv;
    std::atomic<bool> stop{false};
    std::atomic<int32_t> fatal{SW_OK};
    std::atomic<int32_t> n_active{0}, n_queued{0};
    // evidence of continuous batching: requests admitted while other
    // searches were mid-run, and the most searches advanced in one iteration
    std::atomic<int64_t> admitted{0}, admitted_1{0}, admitted_2{0}, iterations{0};
    std::atomic<int32_t> max_active{0};
    std::thread worker;

    void loop();
    int admit_some();
    void collect();
};

int sw_server::admit_some() {
    // take submissions into free slots; their delta tables go to the device
    // together (one staging buffer, one copy per request, no sync between)
    {
        std::lock_guard<std::mutex> lk(mu);
        size_t bytes = 0;
        std::vector<int> taken;
        while (!incoming.empty() && !free_slots.empty()) {
            Sub &sb = incoming.front();
            int64_t doff = delta_pool.alloc((int64_t)sb.n * sb.k);
            if (doff < 0) break;
            int id = free_slots.back();
            free_slots.pop_back();
            Inst x;
            x.n = sb.n;
            x.k = sb.k;
            x.orig = id;
            x.delta_off = doff;
            x.word_off = (int64_t)id * word_cap;
            x.word_cap = word_cap;
            slots[id] = x;
            req_of[id] = sb.req;
            staged_delta.insert(staged_delta.end(), sb.delta.begin(), sb.delta.end());
            bytes += sb.delta.size() * sizeof(uint16_t);
            taken.push_back(id);
            incoming.pop_front();
        }
        if (!taken.empty()) {
            uint16_t *up = (uint16_t *)g_words.get(bytes);
            if (!up) return SW_ECUDA;
            std::memcpy(up, staged_delta.data(), bytes);
            size_t pos = 0;
            for (int id : taken) {
                size_t cnt = (size_t)slots[id].n * slots[id].k;
                if (cudaMemcpyAsync(L.delta16 + slots[id].delta_off, up + pos, cnt * sizeof(uint16_t),
                                    cudaMemcpyHostToDevice, st) != cudaSuccess)
                    return SW_ECUDA;
                pos += cnt;
                queue.push_back(id);
            }
            staged_delta.clear();
            if (cudaStreamSynchronize(st) != cudaSuccess) return SW_ECUDA;  // staging is reused next
        }
    }
    // n = 1 needs no search
    for (auto it = queue.begin(); it != queue.end();) {
        Inst &x = slots[*it];
        if (x.n == 1) {
            x.r = 0;
            x.state = kDone;
            x.code = SW_OK;
            it = queue.erase(it);
        } else {
            ++it;
        }
    }
    // admission by memory budget: every waiting request whose roots and
    // first tables keep both pools under the budget, in one call
    std::vector<int> ids;
    double sets_used = (double)eng->set_pool.used, tab_used = (double)eng->tab_pool.used;
    for (int id : queue) {
        const Inst &x = slots[id];
        double s_need = x.n + 1.0, t_need = 64.0 + 4.0 * x.n + 64.0;
        if (sets_used + s_need > admit_frac * (double)eng->set_pool.cap ||
            tab_used + t_need > admit_frac * (double)eng->tab_pool.cap)
            break;
        sets_used += s_need;
        tab_used += t_need;
        ids.push_back(id);
    }
    if (!ids.empty()) {
        size_t taken = 0;
        const size_t running = eng->active.size();  // searches already mid-run
        int rc = eng->admit(ids, 0, &taken);
        if (rc) return rc;
        queue.erase(queue.begin(), queue.begin() + (std::ptrdiff_t)taken);
        admitted += (int64_t)taken;
        if (running >= 1) admitted_1 += (int64_t)taken;
        if (running >= 2) admitted_2 += (int64_t)taken;
    }
    n_queued = (int32_t)queue.size();
    return SW_OK;
}

void sw_server::collect() {
    std::lock_guard<std::mutex> lk(mu);
    for (size_t id = 0; id < slots.size(); ++id) {
        Inst &x = slots[id];
        if (x.state != kDone && x.state != kFailed) continue;
        Done d;
        d.req = req_of[id];
        d.code = x.code;
        d.r = (x.state == kDone || x.code == SW_EWORDCAP) ? x.r : -1;
        if (x.state == kDone) d.word.assign(words.begin() + x.word_off, words.begin() + x.word_off + x.r);
        done.push_back(std::move(d));
        delta_pool.release(x.delta_off, (int64_t)x.n * x.k);
        x = Inst{};
        x.state = -1;  // free
        free_slots.push_back((int)id);
    }
}

void sw_server::loop() {
    g_opt = opt;
    for (;;) {
        if (stop) break;
        int rc = admit_some();
        if (rc) {
            fatal = rc;
            break;
        }
        // requests set back by an eviction go to the front of the queue
        for (int id : eng->deferred) queue.push_front(id);
        eng->deferred.clear();
        collect();
        cv.notify_all();
        n_active = (int32_t)eng->active.size();
        if (eng->active.empty()) {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return stop || !incoming.empty(); });
            continue;
        }
        max_active = std::max<int32_t>(max_active.load(), (int32_t)eng->active.size());
        iterations++;
        rc = eng->iterate();
        if (rc) {
            fatal = rc;
            break;
        }
        collect();
        cv.notify_all();
    }
}

// ---------------------------------------------------------------- fixed device scratch

// Device scratch for sw_reset_threshold_static, defined in this file so that
// no call ever needs cudaMalloc: every GPU that loads the library holds these
// SW_STATIC_SCRATCH_BYTES until the process exits.  Host code may not use
// the name as an address; it asks the runtime for the address once per
// device (static_scratch_ptr) and passes that on.
static __device__ __align__(256) unsigned char g_static_scratch[SW_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_static_mu;
void *g_static_ptr[128] = {};

// Address of g_static_scratch on the current device, looked up on the first
// call made on that device.
int32_t static_scratch_ptr(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return SW_ECUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return SW_ECUDA;
        g_static_ptr[dev] = ptr;
    }
    *out = g_static_ptr[dev];
    return SW_OK;
}
}  // namespace

// ==================================================================== C-ABI

int32_t sw_internal_fail(int32_t code) { return fail(code); }

int32_t sw_internal_ok() {
    g_last_error = SW_OK;
    return SW_OK;
}

extern "C" {

int32_t sw_last_error(void) { return g_last_error; }

const char *sw_error_string(int32_t code) {
    switch (code) {
        case SW_OK: return "ok";
        case SW_EINVAL: return "invalid argument";
        case SW_ENOTSYNC: return "automaton is not synchronizing";
        case SW_ENOMEM: return "workspace too small";
        case SW_ETIMEOUT: return "bounded device wait gave up";
        case SW_EWORDCAP: return "reset word longer than the word capacity";
        case SW_ECUDA: return "CUDA runtime error";
        case SW_EBUSY: return "no room for the request";
        case SW_EAGAIN: return "no finished request";
        case SW_EINTERNAL: return "internal self-check failed";
        case SW_ENOTFOUND: return "no reset word found within the depth limit";
        default: return "unknown status";
    }
}

sw_handle sw_load_automaton(int32_t n, int32_t k, const int32_t *delta) {
    if (n < 1 || n > SW_MAX_STATES || k < 1 || k > SW_MAX_LETTERS || !delta) {
        fail(SW_EINVAL);
        return nullptr;
    }
    for (int64_t i = 0; i < (int64_t)n * k; ++i)
        if (delta[i] < 0 || delta[i] >= n) {
            fail(SW_EINVAL);
            return nullptr;
        }
    if (!host_is_synchronizing(n, k, delta)) {
        fail(SW_ENOTSYNC);
        return nullptr;
    }
    sw_automaton *h = new (std::nothrow) sw_automaton;
    if (!h) {
        fail(SW_ENOMEM);
        return nullptr;
    }
    h->n = n;
    h->k = k;
    h->delta16.resize((size_t)n * k);
    for (size_t i = 0; i < h->delta16.size(); ++i) h->delta16[i] = (uint16_t)delta[i];
    g_last_error = SW_OK;
    return h;
}

void sw_free(sw_handle h) { delete h; }

size_t sw_workspace_min_bytes(int32_t n_max, int32_t k_max, int32_t count) {
    if (n_max < 1 || k_max < 1 || count < 1) return 0;
    int W = words_for(n_max);
    int64_t delta = (int64_t)n_max * k_max * count;
    double per_set = (8.0 * W + 8) / 0.55;
    return small_area_bytes(count, delta, W) + (size_t)(per_set * ((double)count * (n_max + 1) * 8 + 8192)) + (1 << 20);
}

static int32_t run_instances(std::vector<Inst> &I, const std::vector<uint16_t> *host_delta,
                             const int32_t *d_delta32, const std::vector<int64_t> *src_off, cudaStream_t st,
                             void *ws, size_t ws_bytes, bool device_words, uint8_t *out_words) {
    g_stats = Stats{};
    if (g_timing) {
        g_ev.ensure();
        g_ev.meets = 0;
    }
    int W = common_w(I);
    int64_t delta_elems = 0;
    for (auto &x : I) delta_elems = std::max(delta_elems, x.delta_off + (int64_t)x.n * x.k);
    Layout L;
    if (((uintptr_t)ws & 255) != 0) return SW_EINVAL;
    if (!carve(ws, ws_bytes, W, (int32_t)I.size(), delta_elems, L)) return SW_ENOMEM;
    if (host_delta) {
        void *up = g_up.get(host_delta->size() * sizeof(uint16_t));
        if (!up) return SW_ECUDA;
        std::memcpy(up, host_delta->data(), host_delta->size() * sizeof(uint16_t));
        if (cudaMemcpyAsync(L.delta16, up, host_delta->size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)  // the staging buffer is reused next
            return SW_ECUDA;
    } else {
        // device int32 tables -> uint16, one launch for all instances
        // (grid.y <= 65535 instances per launch); the job rows are staged in
        // the mirror area
        size_t nI = I.size();
        if (nI * sizeof(ConvJob) + 256 > L.mirror_bytes) return SW_EINTERNAL;
        ConvJob *cj = (ConvJob *)g_up.get(nI * sizeof(ConvJob) + 64);
        if (!cj) return SW_ECUDA;
        int64_t maxcnt = 1;
        for (size_t t = 0; t < nI; ++t) {
            cj[t] = ConvJob{(*src_off)[t], I[t].delta_off, (int64_t)I[t].n * I[t].k, I[t].n, 0};
            maxcnt = std::max(maxcnt, cj[t].count);
        }
        ConvJob *d_cj = (ConvJob *)L.mirror;
        if (cudaMemsetAsync(L.status, 0, L.status_n * sizeof(uint32_t), st) != cudaSuccess ||
            cudaMemcpyAsync(d_cj, cj, nI * sizeof(ConvJob), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return SW_ECUDA;
        unsigned gx = (unsigned)std::min<int64_t>((maxcnt + 255) / 256, 64);
        for (size_t b = 0; b < nI; b += 65535) {
            dim3 grid(gx, (unsigned)std::min<size_t>(65535, nI - b));
            g_stats.launches++;
            k_delta_to_u16<<<grid, 256, 0, st>>>(d_cj + b, d_delta32, L.delta16, L.status);
        }
        if (cudaGetLastError() != cudaSuccess) return SW_ECUDA;
        uint32_t *bad = (uint32_t *)g_down.get(sizeof(uint32_t));
        if (!bad) return SW_ECUDA;
        if (cudaMemcpyAsync(bad, L.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SW_ECUDA;
        if (*bad) return SW_EINVAL;
    }
    if (cudaMemsetAsync(L.status, 0, L.status_n * sizeof(uint32_t), st) != cudaSuccess) return SW_ECUDA;
    int n_max = 1;
    for (auto &x : I) n_max = std::max(n_max, (int)x.n);
    Engine E(W, n_max, st, I, L);
    E.device_words = device_words;
    E.out_words = out_words;
    auto t0 = std::chrono::steady_clock::now();
    int rc = E.run();
    g_stats.run_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc == SW_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = SW_ECUDA;
    return rc;
}

int32_t sw_reset_threshold(sw_handle h, void *stream, void *workspace, size_t ws_bytes, int32_t *r,
                           uint8_t *word, int32_t word_cap) {
    if (!h || !r || !workspace || word_cap < 0) return fail(SW_EINVAL);
    std::vector<Inst> I(1);
    I[0].n = h->n;
    I[0].k = h->k;
    I[0].orig = 0;
    I[0].delta_off = 0;
    I[0].word_off = 0;
    I[0].word_cap = word ? word_cap : INT32_MAX;
    int32_t rc = run_instances(I, &h->delta16, nullptr, nullptr, (cudaStream_t)stream, workspace, ws_bytes,
                               false, word);
    if (rc) return fail(rc);
    if (I[0].state == kDone || I[0].code == SW_EWORDCAP) {
        *r = I[0].r;
        store_sizes(h, I[0]);
    }
    if (I[0].state != kDone) return fail(I[0].code ? I[0].code : SW_EINTERNAL);
    g_last_error = SW_OK;
    return SW_OK;
}

int32_t sw_level_sizes(sw_handle h, int64_t *fwd, int32_t fwd_cap, int32_t *nf, int64_t *bwd, int32_t bwd_cap,
                       int32_t *nb) {
    if (!h || !h->searched) return fail(SW_EINVAL);
    if (nf) *nf = (int32_t)h->fwd_sizes.size();
    if (nb) *nb = (int32_t)h->bwd_sizes.size();
    for (int32_t i = 0; fwd && i < fwd_cap && i < (int32_t)h->fwd_sizes.size(); ++i) fwd[i] = h->fwd_sizes[i];
    for (int32_t i = 0; bwd && i < bwd_cap && i < (int32_t)h->bwd_sizes.size(); ++i) bwd[i] = h->bwd_sizes[i];
    g_last_error = SW_OK;
    return SW_OK;
}

int32_t sw_batch(const sw_handle *hs, int32_t count, void *stream, void *workspace, size_t ws_bytes,
                 int32_t *r_out, uint8_t *words, const int64_t *word_off, int64_t words_cap) {
    if (!hs || count < 1 || !r_out || !workspace) return fail(SW_EINVAL);
    if (words && !word_off) return fail(SW_EINVAL);
    std::vector<Inst> I((size_t)count);
    std::vector<uint16_t> delta;
    for (int32_t t = 0; t < count; ++t) {
        if (!hs[t]) return fail(SW_EINVAL);
        Inst &x = I[t];
        x.n = hs[t]->n;
        x.k = hs[t]->k;
        x.orig = t;
        x.delta_off = (int64_t)delta.size();
        delta.insert(delta.end(), hs[t]->delta16.begin(), hs[t]->delta16.end());
        if (words) {
            if (word_off[t] < 0 || word_off[t + 1] < word_off[t] || word_off[t + 1] > words_cap)
                return fail(SW_EINVAL);
            x.word_off = word_off[t];
            x.word_cap = word_off[t + 1] - word_off[t];
        } else {
            x.word_off = 0;
            x.word_cap = INT32_MAX;
        }
    }
    int32_t rc = run_instances(I, &delta, nullptr, nullptr, (cudaStream_t)stream, workspace, ws_bytes, false,
                               words);
    if (rc) return fail(rc);
    int32_t first = SW_OK;
    for (int32_t t = 0; t < count; ++t) {
        Inst &x = I[t];
        r_out[t] = (x.state == kDone || x.code == SW_EWORDCAP) ? x.r : -1;
        if (x.state == kDone) store_sizes(hs[t], x);
        if (x.state != kDone && first == SW_OK) first = x.code ? x.code : SW_EINTERNAL;
    }
    if (first) return fail(first);
    g_last_error = SW_OK;
    return SW_OK;
}

int32_t sw_batch_device(int32_t count, const int32_t *n, const int32_t *k, const int32_t *d_delta,
                        const int64_t *delta_off, void *stream, void *workspace, size_t ws_bytes, int32_t *d_r,
                        uint8_t *d_words, const int64_t *word_off, int64_t words_cap) {
    if (count < 1 || !n || !k || !d_delta || !delta_off || !workspace || !d_r) return fail(SW_EINVAL);
    if (d_words && !word_off) return fail(SW_EINVAL);
    std::vector<Inst> I((size_t)count);
    std::vector<int64_t> src(count);
    int64_t pos = 0;
    for (int32_t t = 0; t < count; ++t) {
        if (n[t] < 1 || n[t] > SW_MAX_STATES || k[t] < 1 || k[t] > SW_MAX_LETTERS || delta_off[t] < 0)
            return fail(SW_EINVAL);
        Inst &x = I[t];
        x.n = n[t];
        x.k = k[t];
        x.orig = t;
        x.delta_off = pos;
        src[t] = delta_off[t];
        pos += (int64_t)n[t] * k[t];
        if (d_words) {
            if (word_off[t] < 0 || word_off[t + 1] < word_off[t] || word_off[t + 1] > words_cap)
                return fail(SW_EINVAL);
            x.word_off = word_off[t];
            x.word_cap = word_off[t + 1] - word_off[t];
        } else {
            x.word_off = 0;
            x.word_cap = 0;  // no word buffer: compute r only
            x.word_cap = INT32_MAX;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    int32_t rc = run_instances(I, nullptr, d_delta, &src, st, workspace, ws_bytes, d_words != nullptr, d_words);
    if (rc) return fail(rc);
    std::vector<int32_t> r(count);
    int32_t first = SW_OK;
    for (int32_t t = 0; t < count; ++t) {
        r[t] = (I[t].state == kDone || I[t].code == SW_EWORDCAP) ? I[t].r : -1;
        if (I[t].state != kDone && first == SW_OK) first = I[t].code ? I[t].code : SW_EINTERNAL;
    }
    int32_t *pr = (int32_t *)g_up.get(count * sizeof(int32_t));
    if (!pr) return fail(SW_ECUDA);
    std::memcpy(pr, r.data(), count * sizeof(int32_t));
    if (cudaMemcpyAsync(d_r, pr, count * sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(SW_ECUDA);
    if (first) return fail(first);
    g_last_error = SW_OK;
    return SW_OK;
}

int32_t sw_last_stats(int64_t *pairs, int64_t *candidates, int32_t *iterations, double *meet_ms,
                      double *expand_ms, double *compact_ms, int32_t *meet_launches, int64_t *launches,
                      int32_t *waves, int32_t *evictions, int64_t *arena_peak, int64_t *and_iters,
                      int64_t *rows_transposed, double *words_ms, double *run_ms, double *sync_ms,
                      double *select_ms, double *update_ms, int32_t *meet_lane_words) {
    if (meet_lane_words) *meet_lane_words = g_stats.meet_lw;
    if (pairs) *pairs = g_stats.pairs;
    if (candidates) *candidates = g_stats.candidates;
    if (iterations) *iterations = g_stats.iterations;
    if (meet_ms) *meet_ms = g_stats.meet_ms;
    if (expand_ms) *expand_ms = g_stats.expand_ms;
    if (compact_ms) *compact_ms = g_stats.compact_ms;
    if (meet_launches) *meet_launches = g_stats.meet_launches;
    if (launches) *launches = g_stats.launches;
    if (waves) *waves = g_stats.waves;
    if (evictions) *evictions = g_stats.evictions;
    if (arena_peak) *arena_peak = g_stats.arena_peak;
    if (and_iters) *and_iters = g_stats.and_iters;
    if (rows_transposed) *rows_transposed = g_stats.rows_transposed;
    if (words_ms) *words_ms = g_stats.words_ms;
    if (run_ms) *run_ms = g_stats.run_ms;
    if (sync_ms) *sync_ms = g_stats.sync_ms;
    if (select_ms) *select_ms = g_stats.select_ms;
    if (update_ms) *update_ms = g_stats.update_ms;
    return SW_OK;
}

void sw_set_timing(int32_t on) { g_timing = on != 0; }

void sw_get_options(sw_options *opt) {
    if (opt) *opt = g_opt;
}

void sw_set_options(const sw_options *opt) {
    if (!opt) return;
    g_opt = *opt;
    if (!(g_opt.dir_theta > 0) || !std::isfinite(g_opt.dir_theta)) g_opt.dir_theta = 1.0;
    if (!(g_opt.set_cost >= 0) || !std::isfinite(g_opt.set_cost)) g_opt.set_cost = 8192.0;
    if (g_opt.meet_b_tile < 0) g_opt.meet_b_tile = 0;
    if (g_opt.meet_algo != 1) g_opt.meet_algo = 0;
    if (g_opt.meet_f_rows < 0) g_opt.meet_f_rows = 0;
    if (g_opt.meet_lane_words != 4) g_opt.meet_lane_words = 0;
    if (g_opt.reduce < 0 || g_opt.reduce > 3) g_opt.reduce = 0;
    if (g_opt.table_cap_slots < 0) g_opt.table_cap_slots = 0;
    if (g_opt.dir_rule != 1) g_opt.dir_rule = 0;
    if (g_opt.dfs_sets < -1) g_opt.dfs_sets = 0;
}

double sw_expmark(double a_s, double b_s, double a_d, double b_d) { return expmark(a_s, b_s, a_d, b_d); }

int32_t sw_last_host_stats(double *stage_ms, double *plan_ms, double *post_ms, double *table_ms, double *gap_ms) {
    if (stage_ms) *stage_ms = g_stats.stage_ms;
    if (plan_ms) *plan_ms = g_stats.plan_ms;
    if (post_ms) *post_ms = g_stats.post_ms;
    if (table_ms) *table_ms = g_stats.table_ms;
    if (gap_ms) *gap_ms = g_stats.gap_ms;
    return SW_OK;
}

int32_t sw_last_dfs_stats(int64_t *instances, int64_t *chunks, int64_t *sets) {
    if (instances) *instances = g_stats.dfs_instances;
    if (chunks) *chunks = g_stats.dfs_chunks;
    if (sets) *sets = g_stats.dfs_sets;
    return SW_OK;
}

int32_t sw_last_reduce_stats(double *mark_ms, int64_t *mark_pairs, int64_t *mark_steps, int64_t *mark_rows) {
    if (mark_rows) *mark_rows = g_stats.mark_rows;
    if (mark_ms) *mark_ms = g_stats.mark_ms;
    if (mark_pairs) *mark_pairs = g_stats.mark_pairs;
    if (mark_steps) *mark_steps = g_stats.mark_steps;
    return SW_OK;
}

int32_t sw_server_create(void *workspace, size_t ws_bytes, int32_t n_max, int32_t k_max, int32_t max_requests,
                         int32_t word_cap, void *stream, sw_server **out) {
    if (!out || !workspace || n_max < 1 || n_max > SW_MAX_STATES || k_max < 1 || k_max > SW_MAX_LETTERS ||
        max_requests < 1 || word_cap < 1)
        return fail(SW_EINVAL);
    if (((uintptr_t)workspace & 255) != 0) return fail(SW_EINVAL);
    std::unique_ptr<sw_server> s(new (std::nothrow) sw_server);
    if (!s) return fail(SW_ENOMEM);
    s->W = words_for(n_max);
    s->n_max = n_max;
    s->k_max = k_max;
    s->cap = max_requests;
    s->word_cap = word_cap;
    s->st = (cudaStream_t)stream;
    s->opt = g_opt;
    if (!carve(workspace, ws_bytes, s->W, max_requests, (int64_t)max_requests * n_max * k_max, s->L))
        return fail(SW_ENOMEM);
    if (cudaMemsetAsync(s->L.status, 0, s->L.status_n * sizeof(uint32_t), s->st) != cudaSuccess ||
        cudaStreamSynchronize(s->st) != cudaSuccess)
        return fail(SW_ECUDA);
    s->slots.assign((size_t)max_requests, Inst{});
    for (auto &x : s->slots) x.state = -1;
    s->req_of.assign((size_t)max_requests, 0);
    s->words.assign((size_t)max_requests * word_cap, 0);
    for (int i = max_requests - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->delta_pool.init(s->L.delta_cap);
    s->eng.reset(new Engine(s->W, s->n_max, s->st, s->slots, s->L));
    s->eng->device_words = false;
    s->eng->out_words = s->words.data();
    sw_server *raw = s.get();
    raw->worker = std::thread([raw] { raw->loop(); });
    *out = s.release();
    g_last_error = SW_OK;
    return SW_OK;
}

int32_t sw_server_submit(sw_server *s, sw_handle h, uint64_t req_id) {
    if (!s || !h) return fail(SW_EINVAL);
    if (h->n > s->n_max || h->k > s->k_max) return fail(SW_EINVAL);
    if (s->fatal != SW_OK) return fail(s->fatal);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if ((int32_t)s->incoming.size() >= s->cap) return fail(SW_EBUSY);
        s->incoming.push_back(sw_server::Sub{req_id, h->n, h->k, h->delta16});
    }
    s->cv.notify_all();
    g_last_error = SW_OK;
    return SW_OK;
}

int32_t sw_server_poll(sw_server *s, uint64_t *req_id, int32_t *r, uint8_t *word, int32_t word_cap,
                       int32_t *code) {
    if (!s || !req_id || !r) return fail(SW_EINVAL);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->done.empty()) {
        if (s->fatal != SW_OK) return fail(s->fatal);
        return SW_EAGAIN;
    }
    sw_server::Done d = std::move(s->done.front());
    s->done.pop_front();
    *req_id = d.req;
    *r = d.r;
    if (code) *code = d.code;
    if (word && d.code == SW_OK) {
        if ((int32_t)d.word.size() > word_cap) return fail(SW_EWORDCAP);
        std::memcpy(word, d.word.data(), d.word.size());
    }
    return SW_OK;
}

int32_t sw_server_pending(sw_server *s, int32_t *queued, int32_t *active, int32_t *finished) {
    if (!s) return fail(SW_EINVAL);
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int32_t)s->incoming.size() + s->n_queued;
    if (active) *active = s->n_active;
    if (finished) *finished = (int32_t)s->done.size();
    return s->fatal;
}

int32_t sw_server_stats(sw_server *s, int64_t *admitted, int64_t *admitted_while_1, int64_t *admitted_while_2,
                        int32_t *max_active, int64_t *iterations) {
    if (!s) return fail(SW_EINVAL);
    if (admitted) *admitted = s->admitted;
    if (admitted_while_1) *admitted_while_1 = s->admitted_1;
    if (admitted_while_2) *admitted_while_2 = s->admitted_2;
    if (max_active) *max_active = s->max_active;
    if (iterations) *iterations = s->iterations;
    return SW_OK;
}

void sw_server_destroy(sw_server *s) {
    if (!s) return;
    s->stop = true;
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->st);
    delete s;
}

int32_t sw_reset_threshold_static(sw_handle h, void *stream, int32_t *r, uint8_t *word, int32_t word_cap) {
    if (!h || !r || word_cap < 0) return fail(SW_EINVAL);
    if (sw_workspace_min_bytes(h->n, h->k, 1) > (size_t)SW_STATIC_SCRATCH_BYTES) return fail(SW_ENOMEM);
    void *scratch = nullptr;
    int32_t rc = static_scratch_ptr(&scratch);
    if (rc) return fail(rc);
    std::vector<Inst> I(1);
    I[0].n = h->n;
    I[0].k = h->k;
    I[0].word_off = 0;
    I[0].word_cap = word ? word_cap : INT32_MAX;
    bool timing = g_timing;
    g_timing = false;  // no events: creating them is not needed here
    g_pageable = true;
    rc = run_instances(I, &h->delta16, nullptr, nullptr, (cudaStream_t)stream, scratch,
                       (size_t)SW_STATIC_SCRATCH_BYTES, false, word);
    g_pageable = false;
    g_timing = timing;
    if (rc) return fail(rc);
    if (I[0].state == kDone || I[0].code == SW_EWORDCAP) {
        *r = I[0].r;
        store_sizes(h, I[0]);
    }
    if (I[0].state != kDone) return fail(I[0].code ? I[0].code : SW_EINTERNAL);
    g_last_error = SW_OK;
    return SW_OK;
}

}  // extern "C"
