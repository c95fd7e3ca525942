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
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "sw.h"
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
    double meet_ms = 0, expand_ms = 0, compact_ms = 0;
    int32_t meet_launches = 0;
    int64_t and_iters = 0;  // bitmap meet: warp-wide AND steps
    int64_t launches = 0;  // every kernel launch of the search
    int32_t waves = 0, evictions = 0;
    int64_t arena_peak = 0;  // most sets stored at once
};

thread_local int32_t g_last_error = SW_OK;
thread_local sw_options g_opt = {0, 0, 0, 0, 1.0, 16384.0};
thread_local bool g_timing = false;
thread_local Stats g_stats;

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
    ~Pinned() {
        if (p) cudaFreeHost(p);
    }
    void *get(size_t bytes) {
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
thread_local Pinned g_up, g_down, g_words;

// ---------------------------------------------------------------- per-instance state

enum InstState { kWaiting = 0, kActive = 1, kDone = 2, kFailed = 3 };

struct Inst {
    int32_t n = 0, k = 0, orig = 0;
    int64_t delta_off = 0;
    std::vector<int64_t> off[2], cnt[2];
    double dupl[2] = {0.0, 0.0};
    int32_t state = kWaiting, code = SW_OK, r = -1;
    int32_t evictions = 0;
    int64_t stored = 0;
    // where the word goes
    int64_t word_off = 0, word_cap = 0;
};

struct Layout {
    // small per-iteration areas
    ExpandJob *jobs;
    MeetJob *mjobs;
    RootJob *rjobs;
    WordJob *wjobs;
    int64_t *blevels;
    int64_t blevels_cap;
    uint64_t *job_rank;     // njobs + 1
    unsigned long long *best;
    uint32_t *word_status;
    uint32_t *status;
    unsigned long long *pairs;  // [0] pairs tested, [1] bitmap AND steps
    uint8_t *word_area;
    int64_t word_area_cap;
    uint16_t *delta16;
    // big areas
    uint64_t *sets, *link;
    uint32_t *owner;
    int64_t cap_sets;
    uint64_t *cand_sets;
    uint32_t *cand_owner;
    int64_t *cand_slot;
    uint8_t *flag;
    uint32_t *block_cnt;
    uint64_t *block_off;
    int64_t cap_cand;
    uint64_t *table;
    uint64_t cap_table;
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

size_t small_area_bytes(int32_t count, int64_t delta_elems) {
    size_t c = (size_t)std::max(count, 1);
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
    add(c * sizeof(ExpandJob));
    add(c * sizeof(MeetJob));
    add(c * sizeof(RootJob));
    add(c * sizeof(WordJob));
    add((c * 256 + 4096) * 2 * sizeof(int64_t));  // blevels
    add((c + 1) * sizeof(uint64_t));
    add(c * sizeof(unsigned long long));
    add(c * sizeof(uint32_t));
    add(sizeof(uint32_t));
    add(2 * sizeof(unsigned long long));
    add(std::max<size_t>(c * 512, 1 << 20));  // word area
    add((size_t)delta_elems * sizeof(uint16_t));
    return b;
}

bool carve(void *ws, size_t bytes, int W, int32_t count, int64_t delta_elems, int kmax, Layout &L) {
    Carver cv(ws, bytes);
    size_t c = (size_t)std::max(count, 1);
    L.jobs = cv.take<ExpandJob>(c);
    L.mjobs = cv.take<MeetJob>(c);
    L.rjobs = cv.take<RootJob>(c);
    L.wjobs = cv.take<WordJob>(c);
    L.blevels_cap = (int64_t)(c * 256 + 4096);
    L.blevels = cv.take<int64_t>((size_t)L.blevels_cap * 2);
    L.job_rank = cv.take<uint64_t>(c + 1);
    L.best = cv.take<unsigned long long>(c);
    L.word_status = cv.take<uint32_t>(c);
    L.status = cv.take<uint32_t>(1);
    L.pairs = cv.take<unsigned long long>(2);
    L.word_area_cap = (int64_t)std::max<size_t>(c * 512, 1 << 20);
    L.word_area = cv.take<uint8_t>((size_t)L.word_area_cap);
    L.delta16 = cv.take<uint16_t>((size_t)std::max<int64_t>(delta_elems, 1));
    if (!cv.ok) return false;
    // The rest: stored sets (set + link + owner), candidates (set + owner +
    // slot + flag + block counts), and the table with two slots per set that
    // can be present at once (stored + candidates), i.e. load <= 1/2.
    double rho = kmax > 2 ? 1.0 : 0.5;  // candidate capacity relative to stored capacity
    double per_set = (8.0 * W + 12) + rho * (8.0 * W + 8 + 4 + 1 + 4.0 / kScanBlock + 8.0 / kScanBlock) +
                     16.0 * (1 + rho);
    size_t rest = cv.size - cv.used;
    if (rest < 64 * 1024) return false;
    int64_t S = (int64_t)((double)(rest - 16 * 1024) / per_set);
    for (;; S = S * 15 / 16) {
        if (S < 64) return false;
        Carver t = cv;
        int64_t C = std::max<int64_t>((int64_t)(S * rho), 64);
        C = std::min<int64_t>(C, (int64_t)0xF0000000);
        int64_t nblocks = (C + kScanBlock - 1) / kScanBlock;
        uint64_t T = (uint64_t)(2 * (S + C));
        L.sets = t.take<uint64_t>((size_t)S * W);
        L.link = t.take<uint64_t>((size_t)S);
        L.owner = t.take<uint32_t>((size_t)S);
        L.cand_sets = t.take<uint64_t>((size_t)C * W);
        L.cand_owner = t.take<uint32_t>((size_t)C);
        L.cand_slot = t.take<int64_t>((size_t)C);
        L.flag = t.take<uint8_t>((size_t)C);
        L.block_cnt = t.take<uint32_t>((size_t)nblocks);
        L.block_off = t.take<uint64_t>((size_t)nblocks + 1);
        L.table = t.take<uint64_t>((size_t)T);
        if (t.ok) {
            L.cap_sets = S;
            L.cap_cand = C;
            L.cap_table = T;
            return true;
        }
    }
}

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

int default_rows(int W) { return W == 1 ? 8 : (W <= 3 ? 4 : 2); }
int default_btile(int W) { return std::max(64, (4096 / W) & ~1); }

struct MeetCfg {
    int algo;  // 0 vertical bitmaps, 1 direct LOP3 test
    int R, tb, nt;
    int tf_rows;  // forward rows per tile (bitmap kernel)
};

MeetCfg meet_cfg(int W) {
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
    if (c.algo == 0) c.tb = kBmRows;
    c.tf_rows = g_opt.meet_f_rows > 0 ? g_opt.meet_f_rows : 2048;
    c.tf_rows = std::max(8, std::min(c.tf_rows, 1 << 20));
    return c;
}

template <int W, int R>
cudaError_t launch_meet_r(const MeetJob *jobs, int njobs, int64_t ntiles, int tb, const uint64_t *sets,
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
    grid = std::min<int64_t>(grid, ntiles);
    kern<<<(unsigned)grid, NT, smem, st>>>(jobs, njobs, ntiles, tb, sets, best, pairs);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_meet_bm(const MeetJob *jobs, int njobs, int64_t ntiles, int tf_rows, const uint64_t *sets,
                           unsigned long long *best, unsigned long long *pairs, unsigned long long *iters,
                           cudaStream_t st) {
    constexpr int NT = 256;
    auto kern = k_meet_bm<W, NT>;
    size_t smem = (size_t)64 * W * kBmStride * sizeof(uint32_t);
    static thread_local bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    int64_t grid = std::min<int64_t>((int64_t)sm_count() * std::max(per_sm, 1), ntiles);
    kern<<<(unsigned)grid, NT, smem, st>>>(jobs, njobs, ntiles, tf_rows, sets, best, pairs, iters);
    return cudaGetLastError();
}

template <int W>
struct Ops {
    static cudaError_t roots(const RootJob *j, int nj, int nmax, const Layout &L, cudaStream_t st) {
        dim3 grid((unsigned)((nmax + 1 + 255) / 256), (unsigned)nj);
        g_stats.launches++;
        k_roots<W><<<grid, 256, 0, st>>>(j, nj, L.sets, L.link, L.owner, L.table, L.cap_table, L.status);
        return cudaGetLastError();
    }
    static cudaError_t expand(int nj, int64_t ncand, const Layout &L, cudaStream_t st) {
        int64_t blocks = std::min<int64_t>((ncand + 255) / 256, (int64_t)sm_count() * 16);
        g_stats.launches++;
        k_expand<W><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(
            L.jobs, nj, ncand, L.delta16, L.sets, L.owner, L.table, L.cap_table, L.cand_sets, L.cand_owner,
            L.cand_slot, L.status);
        return cudaGetLastError();
    }
    static cudaError_t compact(int nj, int64_t ncand, int64_t top, const Layout &L, cudaStream_t st) {
        int64_t nblocks = (ncand + kScanBlock - 1) / kScanBlock;
        g_stats.launches += 3;
        k_flag_count<<<(unsigned)nblocks, kScanThreads, 0, st>>>(ncand, L.cand_slot, L.table, L.flag, L.block_cnt);
        k_scan_blocks<<<1, 1024, 0, st>>>(nblocks, L.block_cnt, L.block_off);
        k_compact<W><<<(unsigned)nblocks, kScanThreads, 0, st>>>(L.jobs, nj, ncand, L.flag, L.block_off, L.cand_sets,
                                                                 L.cand_owner, L.cand_slot, L.table, top, L.sets,
                                                                 L.link, L.owner, L.job_rank);
        return cudaGetLastError();
    }
    static cudaError_t meet(int nj, int64_t ntiles, const MeetCfg &c, const Layout &L, cudaStream_t st) {
        g_stats.launches++;
        if (c.algo == 0)
            return launch_meet_bm<W>(L.mjobs, nj, ntiles, c.tf_rows, L.sets, L.best, L.pairs, L.pairs + 1, st);
        switch (c.R) {
            case 1:
                if constexpr (W >= 3) return launch_meet_r<W, 1>(L.mjobs, nj, ntiles, c.tb, L.sets, L.best, L.pairs, st);
                break;
            case 2: return launch_meet_r<W, 2>(L.mjobs, nj, ntiles, c.tb, L.sets, L.best, L.pairs, st);
            case 4: return launch_meet_r<W, 4>(L.mjobs, nj, ntiles, c.tb, L.sets, L.best, L.pairs, st);
            case 8:
                if constexpr (W <= 2) return launch_meet_r<W, 8>(L.mjobs, nj, ntiles, c.tb, L.sets, L.best, L.pairs, st);
                break;
        }
        return cudaErrorInvalidValue;
    }
    static cudaError_t words(int nj, uint8_t *base, const Layout &L, cudaStream_t st) {
        g_stats.launches++;
        k_words<W, 256><<<(unsigned)nj, 256, 0, st>>>(L.wjobs, L.blevels, L.delta16, L.sets, L.link, base,
                                                       L.word_status);
        return cudaGetLastError();
    }
};

struct OpTable {
    cudaError_t (*roots)(const RootJob *, int, int, const Layout &, cudaStream_t);
    cudaError_t (*expand)(int, int64_t, const Layout &, cudaStream_t);
    cudaError_t (*compact)(int, int64_t, int64_t, const Layout &, cudaStream_t);
    cudaError_t (*meet)(int, int64_t, const MeetCfg &, const Layout &, cudaStream_t);
    cudaError_t (*words)(int, uint8_t *, const Layout &, cudaStream_t);
};

template <int W>
OpTable make_ops() {
    return {&Ops<W>::roots, &Ops<W>::expand, &Ops<W>::compact, &Ops<W>::meet, &Ops<W>::words};
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
    cudaEvent_t ev[8] = {};
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

#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return SW_ECUDA; \
    } while (0)

// ---------------------------------------------------------------- the search

struct Search {
    int W;
    cudaStream_t st;
    Layout L;
    OpTable ops;
    MeetCfg mc;
    std::vector<Inst> &I;
    bool device_words;   // words go straight to the caller's device buffer
    uint8_t *out_words;  // caller's buffer (device when device_words, else host)
    int64_t top = 0, stored_total = 0;

    Search(int W_, cudaStream_t s, std::vector<Inst> &insts) : W(W_), st(s), I(insts) {
        ops = ops_for(W);
        mc = meet_cfg(W);
    }

    int64_t top_peak() const { return top; }

    int choose_dir(const Inst &x) const {
        double F = (double)x.cnt[0].back(), B = (double)x.cnt[1].back(), k = x.k;
        double cF = g_opt.set_cost * k * F + k * (1.0 - x.dupl[0]) * F * B;
        double cB = g_opt.set_cost * k * B + k * (1.0 - x.dupl[1]) * B * F;
        return cF <= g_opt.dir_theta * cB ? 0 : 1;
    }

    // Starts a wave: clears the table and stores the roots of `wave`.
    int start_wave(const std::vector<int> &wave) {
        g_stats.waves++;
        top = 0;
        stored_total = 0;
        CK(cudaMemsetAsync(L.table, 0xFF, L.cap_table * sizeof(uint64_t), st));
        CK(cudaMemsetAsync(L.status, 0, sizeof(uint32_t), st));
        RootJob *rj = (RootJob *)g_up.get(wave.size() * sizeof(RootJob));
        if (!rj) return SW_ECUDA;
        int nmax = 1;
        for (size_t t = 0; t < wave.size(); ++t) {
            Inst &x = I[wave[t]];
            if (top + x.n + 1 > L.cap_sets || 2 * (top + x.n + 1) > (int64_t)L.cap_table) return SW_ENOMEM;
            rj[t] = RootJob{top, (int32_t)wave[t], x.n};
            for (int d = 0; d < 2; ++d) {
                x.off[d].clear();
                x.cnt[d].clear();
                x.dupl[d] = 0.0;
            }
            x.off[0].push_back(top);
            x.cnt[0].push_back(1);
            x.off[1].push_back(top + 1);
            x.cnt[1].push_back(x.n);
            x.stored = x.n + 1;
            x.state = kActive;
            top += x.n + 1;
            nmax = std::max(nmax, x.n);
        }
        stored_total = top;
        // the kernel reads at most 65535 root jobs per launch (grid.y)
        CK(cudaMemcpyAsync(L.rjobs, rj, wave.size() * sizeof(RootJob), cudaMemcpyHostToDevice, st));
        for (size_t b = 0; b < wave.size(); b += 65535)
            CK(ops.roots(L.rjobs + b, (int)std::min<size_t>(65535, wave.size() - b), nmax, L, st));
        CK(cudaStreamSynchronize(st));  // the staging buffer is reused next
        return SW_OK;
    }

    // One iteration over the active instances of the wave.  Returns SW_OK,
    // or a fatal code for the whole wave.
    int iterate(std::vector<int> &active, std::vector<int> &evicted) {
        g_stats.iterations++;
        // 1. directions and expansion jobs that fit
        std::vector<int> who;
        std::vector<int> dirs;
        ExpandJob *jobs = (ExpandJob *)g_up.get(active.size() * sizeof(ExpandJob));
        if (!jobs) return SW_ECUDA;
        int64_t ncand = 0;
        for (int id : active) {
            Inst &x = I[id];
            int d = choose_dir(x);
            int64_t pc = x.cnt[d].back();
            int64_t nc = pc * x.k;
            bool fits = ncand + nc <= L.cap_cand && top + ncand + nc <= L.cap_sets &&
                        2 * (stored_total + ncand + nc) <= (int64_t)L.cap_table;
            if (!fits) continue;
            ExpandJob &J = jobs[who.size()];
            J.cand_off = ncand;
            J.parent_off = x.off[d].back();
            J.parent_cnt = pc;
            J.delta_off = x.delta_off;
            J.owner = (int32_t)(((uint32_t)id << 1) | (uint32_t)d);
            J.n = x.n;
            J.k = x.k;
            J.pad = 0;
            who.push_back(id);
            dirs.push_back(d);
            ncand += nc;
        }
        if (who.empty()) {
            // nothing fits: give up the instance holding the most sets; it
            // is retried in a later wave (the wave loop fails it only if it
            // ran alone)
            auto it = std::max_element(active.begin(), active.end(),
                                       [&](int a, int b) { return I[a].stored < I[b].stored; });
            int id = *it;
            active.erase(it);
            I[id].state = kWaiting;
            I[id].evictions++;
            g_stats.evictions++;
            evicted.push_back(id);
            return SW_OK;
        }
        int nj = (int)who.size();
        g_stats.candidates += ncand;
        CK(cudaMemcpyAsync(L.jobs, jobs, nj * sizeof(ExpandJob), cudaMemcpyHostToDevice, st));
        if (g_timing) CK(cudaEventRecord(g_ev.ev[0], st));
        CK(ops.expand(nj, ncand, L, st));
        if (g_timing) CK(cudaEventRecord(g_ev.ev[1], st));
        CK(ops.compact(nj, ncand, top, L, st));
        if (g_timing) CK(cudaEventRecord(g_ev.ev[2], st));
        int64_t nblocks = (ncand + kScanBlock - 1) / kScanBlock;
        // 2. results of the compaction
        uint64_t *down = (uint64_t *)g_down.get((nj + 2) * sizeof(uint64_t));
        if (!down) return SW_ECUDA;
        CK(cudaMemcpyAsync(down, L.job_rank, nj * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(down + nj, L.block_off + nblocks, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(down + nj + 1, L.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (g_timing) {
            g_stats.expand_ms += elapsed(g_ev.ev[0], g_ev.ev[1]);
            g_stats.compact_ms += elapsed(g_ev.ev[1], g_ev.ev[2]);
        }
        uint32_t status = (uint32_t)(down[nj + 1] & 0xFFFFFFFFu);
        if (status & kStatusTableFull) return SW_ENOMEM;
        uint64_t total = down[nj];
        std::vector<int64_t> rank(down, down + nj);
        rank.push_back((int64_t)total);
        // 3. new levels
        std::vector<int> advanced;
        for (int t = 0; t < nj; ++t) {
            Inst &x = I[who[t]];
            int d = dirs[t];
            int64_t c = rank[t + 1] - rank[t];
            int64_t nc = x.cnt[d].back() * x.k;
            x.off[d].push_back(top + rank[t]);
            x.cnt[d].push_back(c);
            x.dupl[d] = 1.0 - (double)c / (double)nc;
            x.stored += c;
            if (c == 0) {
                x.state = kFailed;
                x.code = SW_ENOTSYNC;
            } else {
                advanced.push_back(who[t]);
            }
        }
        top += (int64_t)total;
        stored_total = top;
        // 4. meet check on the advanced instances
        std::vector<int> met;
        std::vector<unsigned long long> best;
        if (!advanced.empty()) {
            int nm = (int)advanced.size();
            MeetJob *mj = (MeetJob *)g_up.get(nm * sizeof(MeetJob));
            if (!mj) return SW_ECUDA;
            const int64_t TF = mc.algo == 0 ? (int64_t)mc.tf_rows : (int64_t)mc.nt * mc.R;
            int64_t ntiles = 0;
            for (int t = 0; t < nm; ++t) {
                Inst &x = I[advanced[t]];
                MeetJob &M = mj[t];
                M.f_off = x.off[0].back();
                M.f_cnt = x.cnt[0].back();
                M.b_off = x.off[1].back();
                M.b_cnt = x.cnt[1].back();
                M.tile_off = ntiles;
                M.ntb = (M.b_cnt + mc.tb - 1) / mc.tb;
                M.slot = t;
                ntiles += ((M.f_cnt + TF - 1) / TF) * M.ntb;
            }
            CK(cudaMemcpyAsync(L.mjobs, mj, nm * sizeof(MeetJob), cudaMemcpyHostToDevice, st));
            CK(cudaMemsetAsync(L.best, 0xFF, nm * sizeof(unsigned long long), st));
            CK(cudaMemsetAsync(L.pairs, 0, 2 * sizeof(unsigned long long), st));
            if (g_timing) CK(cudaEventRecord(g_ev.ev[3], st));
            CK(ops.meet(nm, ntiles, mc, L, st));
            if (g_timing) CK(cudaEventRecord(g_ev.ev[4], st));
            g_stats.meet_launches++;
            unsigned long long *bd = (unsigned long long *)g_down.get((nm + 2) * sizeof(unsigned long long));
            if (!bd) return SW_ECUDA;
            CK(cudaMemcpyAsync(bd, L.best, nm * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(bd + nm, L.pairs, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (g_timing) g_stats.meet_ms += elapsed(g_ev.ev[3], g_ev.ev[4]);
            g_stats.pairs += (int64_t)bd[nm];
            g_stats.and_iters += (int64_t)bd[nm + 1];
            for (int t = 0; t < nm; ++t)
                if (bd[t] != ~0ull) {
                    met.push_back(advanced[t]);
                    best.push_back(bd[t]);
                }
        }
        // 5. words of the instances that met
        if (!met.empty()) {
            int rc = recover_words(met, best);
            if (rc) return rc;
        }
        // 6. drop finished instances from the active list
        active.erase(std::remove_if(active.begin(), active.end(),
                                    [&](int id) { return I[id].state != kActive; }),
                     active.end());
        return SW_OK;
    }

    int recover_words(const std::vector<int> &met, const std::vector<unsigned long long> &best) {
        size_t pos = 0;
        while (pos < met.size()) {
            // a chunk of word jobs that fits the per-call areas
            std::vector<WordJob> wj;
            std::vector<int64_t> blev;
            int64_t area = 0;
            size_t first = pos;
            for (; pos < met.size(); ++pos) {
                Inst &x = I[met[pos]];
                int i = (int)x.cnt[0].size() - 1, j = (int)x.cnt[1].size() - 1;
                int r = i + j;
                x.r = r;
                if (r > x.word_cap) {
                    x.state = kFailed;
                    x.code = SW_EWORDCAP;
                    continue;
                }
                if (!device_words && area + r > L.word_area_cap && !wj.empty()) break;
                if ((int64_t)(blev.size() / 2) + j > L.blevels_cap && !wj.empty()) break;
                if (!device_words && r > L.word_area_cap) {
                    x.state = kFailed;
                    x.code = SW_ENOMEM;
                    continue;
                }
                WordJob J;
                J.f_arena = x.off[0].back() + (int64_t)(best[pos] >> 32);
                J.blev = (int64_t)(blev.size() / 2);
                J.word_off = device_words ? x.word_off : area;
                J.delta_off = x.delta_off;
                J.i = i;
                J.j = j;
                J.n = x.n;
                J.k = x.k;
                J.slot = (int32_t)(pos - first);
                J.pad = met[pos];
                for (int m = 0; m < j; ++m) {
                    blev.push_back(x.off[1][m]);
                    blev.push_back(x.cnt[1][m]);
                }
                if (!device_words) area += r;
                wj.push_back(J);
            }
            if (wj.empty()) continue;
            int nw = (int)wj.size();
            CK(cudaMemcpyAsync(L.wjobs, wj.data(), nw * sizeof(WordJob), cudaMemcpyHostToDevice, st));
            if (!blev.empty())
                CK(cudaMemcpyAsync(L.blevels, blev.data(), blev.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                   st));
            uint8_t *base = device_words ? out_words : L.word_area;
            CK(ops.words(nw, base, L, st));
            uint32_t *ws = (uint32_t *)g_down.get(nw * sizeof(uint32_t));
            if (!ws) return SW_ECUDA;
            CK(cudaMemcpyAsync(ws, L.word_status, nw * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            uint8_t *hw = nullptr;
            if (!device_words && area > 0) {
                hw = (uint8_t *)g_words.get((size_t)area);
                if (!hw) return SW_ECUDA;
                CK(cudaMemcpyAsync(hw, L.word_area, (size_t)area, cudaMemcpyDeviceToHost, st));
            }
            CK(cudaStreamSynchronize(st));
            for (int t = 0; t < nw; ++t) {
                Inst &x = I[wj[t].pad];
                if (ws[t] != 0) {
                    x.state = kFailed;
                    x.code = SW_EINTERNAL;
                    continue;
                }
                if (!device_words && out_words)
                    std::memcpy(out_words + x.word_off, hw + wj[t].word_off, (size_t)x.r);
                x.state = kDone;
                x.code = SW_OK;
            }
        }
        return SW_OK;
    }

    // Runs every instance (state kWaiting) to completion, in waves.
    int run() {
        std::vector<int> queue;
        for (size_t t = 0; t < I.size(); ++t) {
            Inst &x = I[t];
            if (x.state != kWaiting) continue;
            if (x.n == 1) {  // Q is already a singleton: r = 0
                x.r = 0;
                x.state = kDone;
                x.code = SW_OK;
                x.off[0] = {0};
                x.cnt[0] = {1};
                x.off[1] = {0};
                x.cnt[1] = {1};
                continue;
            }
            queue.push_back((int)t);
        }
        size_t limit = queue.size();
        while (!queue.empty()) {
            // admit as many as the roots allow (and fewer after evictions)
            std::vector<int> wave;
            int64_t need = 0;
            std::vector<int> rest;
            for (int id : queue) {
                int64_t s = I[id].n + 1;
                if (wave.size() < limit && need + s <= L.cap_sets && 2 * (need + s) <= (int64_t)L.cap_table) {
                    wave.push_back(id);
                    need += s;
                } else {
                    rest.push_back(id);
                }
            }
            if (wave.empty()) {
                for (int id : queue) {
                    I[id].state = kFailed;
                    I[id].code = SW_ENOMEM;
                }
                break;
            }
            int rc = start_wave(wave);
            if (rc) return rc;
            std::vector<int> active = wave, evicted;
            while (!active.empty()) {
                rc = iterate(active, evicted);
                if (rc == SW_ENOMEM) {  // table overflow: retry the unfinished ones later
                    for (int id : active) {
                        I[id].state = kWaiting;
                        I[id].evictions++;
                        g_stats.evictions++;
                        evicted.push_back(id);
                    }
                    active.clear();
                    break;
                }
                if (rc) return rc;
            }
            g_stats.arena_peak = std::max(g_stats.arena_peak, top_peak());
            if (wave.size() == 1 && !evicted.empty()) {  // it had the whole workspace
                I[evicted[0]].state = kFailed;
                I[evicted[0]].code = SW_ENOMEM;
                evicted.clear();
            }
            if (!evicted.empty()) limit = std::max<size_t>(1, std::min(limit, wave.size()) / 2);
            queue = evicted;
            queue.insert(queue.end(), rest.begin(), rest.end());
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
    h->fwd_sizes = x.cnt[0];
    h->bwd_sizes = x.cnt[1];
    h->searched = true;
}

}  // namespace

// ==================================================================== C-ABI

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
    double per_set = (8.0 * W + 12) + 1.0 * (8.0 * W + 17) + 32.0;
    return small_area_bytes(count, delta) + (size_t)(per_set * ((double)count * (n_max + 1) * 4 + 4096)) + (1 << 20);
}

static int32_t run_instances(std::vector<Inst> &I, const std::vector<uint16_t> *host_delta,
                             const int32_t *d_delta32, const std::vector<int64_t> *src_off, cudaStream_t st,
                             void *ws, size_t ws_bytes, bool device_words, uint8_t *out_words) {
    g_stats = Stats{};
    if (g_timing) g_ev.ensure();
    int W = common_w(I);
    int kmax = 1;
    int64_t delta_elems = 0;
    for (auto &x : I) {
        kmax = std::max(kmax, x.k);
        delta_elems = std::max(delta_elems, x.delta_off + (int64_t)x.n * x.k);
    }
    Layout L;
    if (((uintptr_t)ws & 255) != 0) return SW_EINVAL;
    if (!carve(ws, ws_bytes, W, (int32_t)I.size(), delta_elems, kmax, L)) return SW_ENOMEM;
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
        // (grid.y <= 65535 instances per launch)
        size_t nI = I.size();
        ConvJob *cj = (ConvJob *)g_up.get(nI * sizeof(ConvJob) + 64);
        if (!cj) return SW_ECUDA;
        int64_t maxcnt = 1;
        for (size_t t = 0; t < nI; ++t) {
            cj[t] = ConvJob{(*src_off)[t], I[t].delta_off, (int64_t)I[t].n * I[t].k, I[t].n, 0};
            maxcnt = std::max(maxcnt, cj[t].count);
        }
        // ConvJob rows go where the expansion jobs will later be staged
        ConvJob *d_cj = (ConvJob *)L.jobs;
        if (nI * sizeof(ConvJob) > (size_t)std::max<int32_t>((int32_t)I.size(), 1) * sizeof(ExpandJob))
            return SW_EINTERNAL;
        if (cudaMemsetAsync(L.status, 0, sizeof(uint32_t), st) != cudaSuccess ||
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
    Search S(W, st, I);
    S.L = L;
    S.device_words = device_words;
    S.out_words = out_words;
    int rc = S.run();
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
                      int32_t *waves, int32_t *evictions, int64_t *arena_peak, int64_t *and_iters) {
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
    if (!(g_opt.set_cost >= 0) || !std::isfinite(g_opt.set_cost)) g_opt.set_cost = 16384.0;
    if (g_opt.meet_b_tile < 0) g_opt.meet_b_tile = 0;
    if (g_opt.meet_algo != 1) g_opt.meet_algo = 0;
    if (g_opt.meet_f_rows < 0) g_opt.meet_f_rows = 0;
}

}  // extern "C"
