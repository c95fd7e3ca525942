// Device kernels of the bidirectional subset search (Section 2.1, Alg. 1).
//
// A subset of Q is stored as W 64-bit words (state q at bit q%64 of word
// q/64; bits >= n are zero).  All levels of all instances and both
// directions live in one arena of sets (each level contiguous, placed by the
// host's pool allocator); a forward set also has a parent link ((parent
// arena index) << 8 | letter).  Every (instance, direction) owns an
// open-addressing hash table in a table pool holding the arena indices of
// every set it has seen: it removes duplicates within a level and sets of
// earlier levels (the equality history).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace sw {

constexpr uint64_t kEmpty = ~0ull;
constexpr uint64_t kCand = 1ull << 62;  // slot value kCand + c: candidate c (this expansion)
constexpr int kScanBlock = 512;         // candidates per block in flag/compact
static_assert(kScanBlock % 32 == 0, "a warp of candidates must lie inside one job");
constexpr int kScanThreads = 256;
constexpr int kMaxProbe = 1 << 14;

enum : uint32_t { kStatusTableFull = 1u, kStatusWordFail = 2u, kStatusVerifyFail = 4u };

struct ExpandJob {
    int64_t cand_off;    // first candidate id (a multiple of kScanBlock)
    int64_t parent_off;  // arena index of the parent level's first set
    int64_t parent_cnt;
    int64_t delta_off;   // instance's uint16 [k][n] table in delta16
    int64_t dest_off;    // arena index where the new level starts
    int64_t tab_off;     // the (instance, direction) hash table
    int64_t tab_cap;
    int64_t ge_off;      // backward: where the new level's cardinality table goes
    int32_t dir, n, k;   // dir 0 forward (images), 1 backward (preimages)
    int32_t inst;        // the instance (its flags in status[1 + inst])
};

struct MeetJob {
    int64_t f_off, f_cnt, b_off, b_cnt;
    int64_t tile_off;    // first tile id of this job
    int64_t ntb;         // tiles along B
    int64_t slot;        // index into best[]
    int64_t ge_off;      // B's cardinality table (ge[c] = rows with |Y| >= c), or -1
    int32_t upd;         // -1: counts known; 0: f_cnt, 1: b_cnt = counts[count_idx]
    int32_t count_idx;
};

// Lays out the meet tiles on the device once the new levels' sizes are
// known: fills the size of the level each job just produced, its tiles
// (tf_rows forward rows x tb backward rows; none if a level is empty) and
// the exclusive scan of tile counts; ntiles[0] = their total, ntiles[1] =
// 0 (the tile counter of the bitmap meet kernel).  One block.
__global__ void __launch_bounds__(1024) k_meet_prep(MeetJob *__restrict__ jobs, int njobs,
                                                    const uint64_t *__restrict__ counts, int64_t tf_rows,
                                                    int64_t tb, int64_t *__restrict__ ntiles) {
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < njobs; base += 1024) {
        int j = base + threadIdx.x;
        int64_t tiles = 0;
        if (j < njobs) {
            MeetJob &M = jobs[j];
            if (M.upd == 0) M.f_cnt = (int64_t)counts[M.count_idx];
            if (M.upd == 1) M.b_cnt = (int64_t)counts[M.count_idx];
            M.ntb = M.b_cnt > 0 ? (M.b_cnt + tb - 1) / tb : 1;
            tiles = (M.f_cnt > 0 && M.b_cnt > 0) ? ((M.f_cnt + tf_rows - 1) / tf_rows) * M.ntb : 0;
        }
        int64_t x = tiles;  // inclusive scan over the block
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) warp_sum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            int64_t v = warp_sum[threadIdx.x];
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (threadIdx.x >= o) v += y;
            }
            warp_sum[threadIdx.x] = v;
        }
        __syncthreads();
        int64_t before = carry + (threadIdx.x >= 32 ? warp_sum[(threadIdx.x >> 5) - 1] : 0) + x - tiles;
        if (j < njobs) jobs[j].tile_off = before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + tiles;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ntiles[0] = carry;
        ntiles[1] = 0;  // tile counter of the bitmap meet kernel
    }
}

// Backward levels are stored in decreasing order of cardinality (the order of
// a backward level never affects r, the word or the level sizes).  A level's
// table ge[c], c = 0 .. 64W + 1, counts its sets with at least c states, so
// a forward set X can only lie in the first ge[|X|] of them.
__host__ __device__ constexpr int card_slots(int W) { return 64 * W + 2; }

struct RootJob {
    int64_t f_off, b_off;         // F_0 = {Q} at f_off; B_0 = the n singletons at b_off
    int64_t tab_off[2], tab_cap[2];
    int32_t n, inst;
};

struct FillJob {
    int64_t off, len;             // table slots to set to kEmpty
};

struct RehashSeg {
    int64_t flat_off;             // first flat index of this segment
    int64_t set_off, cnt;         // stored sets to re-enter
    int64_t tab_off, tab_cap;     // into this table
    int32_t dir, inst;
};

struct WordJob {
    int64_t f_arena;     // arena index of the meeting forward set X
    int64_t blev;        // first (offset, count, table) triple of B_0..B_{j-1} in blevels
    int64_t word_off;    // output position in the word buffer
    int64_t delta_off;
    int32_t i, j, n, k;
    int32_t slot;        // index into word_status[]
    int32_t pad;
};

// ------------------------------------------------------------ small helpers

__device__ __forceinline__ uint64_t fmix64(uint64_t x) {
    // MurmurHash3 finalizer (Appleby), a published 64-bit mixer
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

template <int W>
__device__ __forceinline__ uint64_t hash_set(uint32_t owner, const uint64_t (&s)[W]) {
    uint64_t h = fmix64(0x9E3779B97F4A7C15ull * (owner + 1u));
#pragma unroll
    for (int w = 0; w < W; ++w) h = fmix64(h ^ (s[w] + 0x632BE59BD9B4E019ull * (w + 1)));
    return h;
}

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Slot operations of the deduplication table with the memory ordering the
// table needs and no more: a candidate's set is written, then its id is
// published by a release CAS (or handed over by a release min), and a
// thread that reads an id with acquire semantics sees the set written
// before it was published.
__device__ __forceinline__ uint64_t ld_acquire(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t cas_acq_rel(uint64_t *p, uint64_t cmp, uint64_t val) {
    uint64_t old;
    asm volatile("atom.acq_rel.gpu.global.cas.b64 %0, [%1], %2, %3;" : "=l"(old) : "l"(p), "l"(cmp), "l"(val)
                 : "memory");
    return old;
}

__device__ __forceinline__ void min_release(uint64_t *p, uint64_t val) {
    asm volatile("red.release.gpu.global.min.u64 [%0], %1;" ::"l"(p), "l"(val) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int W>
__device__ __forceinline__ void load_set(const uint64_t *__restrict__ p, uint64_t (&s)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) s[w] = p[w];
}

// bit t of a set held in registers (t < 64 W), without dynamic indexing
template <int W>
__device__ __forceinline__ uint32_t get_bit(const uint64_t (&s)[W], uint32_t t) {
    uint64_t word = s[0];
#pragma unroll
    for (int w = 1; w < W; ++w) word = ((t >> 6) == (uint32_t)w) ? s[w] : word;
    return (uint32_t)(word >> (t & 63)) & 1u;
}

// Image delta(S, a) (Section 2): scatter every set bit of S through delta.
template <int W>
__device__ __forceinline__ void image(const uint64_t (&S)[W], const uint16_t *__restrict__ da,
                                      uint64_t (&T)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) T[w] = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t s = S[w];
        while (s) {
            int b = __ffsll((long long)s) - 1;
            s &= s - 1;
            uint32_t t = __ldg(da + w * 64 + b);
            uint64_t bit = 1ull << (t & 63);
            uint32_t tw = t >> 6;
#pragma unroll
            for (int v = 0; v < W; ++v) T[v] |= (tw == (uint32_t)v) ? bit : 0ull;
        }
    }
}

// Preimage delta^{-1}(S, a) (Section 2): state p is in it iff S holds
// delta(p, a).  pre_a holds, for every state t, the bitset
// delta^{-1}({t}, a) (W words), so the preimage is the union of those rows
// over the states of S.
template <int W>
__device__ __forceinline__ void preimage(const uint64_t (&S)[W], const uint64_t *__restrict__ pre_a,
                                         uint64_t (&T)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) T[w] = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t s = S[w];
        while (s) {
            const int t = w * 64 + __ffsll((long long)s) - 1;
            s &= s - 1;
            const uint64_t *row = pre_a + (int64_t)t * W;
#pragma unroll
            for (int v = 0; v < W; ++v) T[v] |= __ldg(row + v);
        }
    }
}

template <int W>
__device__ __forceinline__ bool set_equal(const uint64_t (&a)[W], const uint64_t *__restrict__ p) {
    bool eq = true;
#pragma unroll
    for (int w = 0; w < W; ++w) eq &= (a[w] == p[w]);
    return eq;
}

template <int W>
__device__ __forceinline__ bool set_equal_cg(const uint64_t (&a)[W], const uint64_t *p) {
    bool eq = true;
#pragma unroll
    for (int w = 0; w < W; ++w) eq &= (a[w] == __ldcg(p + w));
    return eq;
}

__device__ __forceinline__ int find_job_expand(const ExpandJob *__restrict__ jobs, int njobs, int64_t c) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].cand_off <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Linear probing inside one table [tab_off, tab_off + tab_cap): the next slot.
__device__ __forceinline__ uint64_t next_slot(uint64_t pos, int64_t tab_off, int64_t tab_cap) {
    return (pos + 1 == (uint64_t)(tab_off + tab_cap)) ? (uint64_t)tab_off : pos + 1;
}

// A table that could not take a set: status[0] collects the flags of the
// whole launch, status[1 + inst] those of the instance, so that the host
// fails that instance alone.
__device__ __forceinline__ void table_full(uint32_t *status, int inst) {
    atomicOr(status, kStatusTableFull);
    atomicOr(status + 1 + inst, kStatusTableFull);
}

// Enters the stored set g (no equal set is present) into a table.
template <int W>
__device__ __forceinline__ void insert_stored(uint64_t *table, int64_t tab_off, int64_t tab_cap, uint32_t dir,
                                              const uint64_t (&s)[W], int64_t g, uint32_t *status, int inst) {
    uint64_t pos = (uint64_t)tab_off + __umul64hi(hash_set<W>(dir, s), (uint64_t)tab_cap);
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        unsigned long long old = atomicCAS((unsigned long long *)(table + pos), kEmpty, (unsigned long long)g);
        if (old == kEmpty) return;
        pos = next_slot(pos, tab_off, tab_cap);
    }
    table_full(status, inst);
}

// The meet kernel's record of a forward set: its first seven states and its
// cardinality as 16-bit fields (x: s0 | s1 << 16, y: s2 | s3 << 16,
// z: s4 | s5 << 16, w: s6 | card << 16).  A set of fewer than seven states
// repeats its first state in the missing fields: ANDing a state's bitmap a
// second time changes nothing, so the meet kernel walks all seven fields
// without a bound check.  Forward sets are never empty.
template <int W>
__device__ __forceinline__ uint4 row_record(const uint64_t (&s)[W]) {
    uint32_t f[8];
    int card = 0, got = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint64_t b = s[w];
        card += __popcll(b);
        while (b && got < 7) {
            f[got++] = (uint32_t)(w * 64 + __ffsll((long long)b) - 1);
            b &= b - 1;
        }
    }
#pragma unroll
    for (int i = 1; i < 7; ++i)
        if (i >= got) f[i] = f[0];
    f[7] = (uint32_t)card;
    return make_uint4(f[0] | (f[1] << 16), f[2] | (f[3] << 16), f[4] | (f[5] << 16), f[6] | (f[7] << 16));
}

// ------------------------------------------------------------ roots, fill, rehash

// F_0 = {Q} and B_0 = the n singletons of each new instance (Alg. 1,
// initialisation), stored and entered into their tables.  One thread per
// set; blockIdx.y = instance.
template <int W>
__global__ void k_roots(const RootJob *__restrict__ jobs, uint64_t *__restrict__ sets,
                        uint64_t *__restrict__ link, uint32_t *__restrict__ perm, uint4 *__restrict__ rec,
                        uint64_t *table, uint32_t *status) {
    const RootJob J = jobs[blockIdx.y];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= J.n; t += gridDim.x * blockDim.x) {
        uint64_t s[W];
        int64_t g;
        uint32_t dir;
        if (t == 0) {  // Q: the first n bits
#pragma unroll
            for (int w = 0; w < W; ++w) {
                int lo = w * 64;
                s[w] = (J.n >= lo + 64) ? ~0ull : (J.n > lo ? ((1ull << (J.n - lo)) - 1) : 0ull);
            }
            g = J.f_off;
            dir = 0;
            link[g] = ~0ull;
            perm[g] = 0;
            rec[g] = row_record<W>(s);
        } else {
            int q = t - 1;
#pragma unroll
            for (int w = 0; w < W; ++w) s[w] = ((q >> 6) == w) ? (1ull << (q & 63)) : 0ull;
            g = J.b_off + q;
            dir = 1;
        }
#pragma unroll
        for (int w = 0; w < W; ++w) sets[g * W + w] = s[w];
        insert_stored<W>(table, J.tab_off[dir], J.tab_cap[dir], dir, s, g, status, J.inst);
    }
}

// Sets table slots to kEmpty; blockIdx.y = job.
__global__ void k_fill(const FillJob *__restrict__ jobs, uint64_t *__restrict__ table) {
    const FillJob J = jobs[blockIdx.y];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < J.len; i += (int64_t)gridDim.x * blockDim.x)
        table[J.off + i] = kEmpty;
}

// The segment holding flat index t, searched in segs[lo .. hi].
__device__ __forceinline__ int find_seg(const RehashSeg *__restrict__ segs, int lo, int hi, int64_t t) {
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (segs[mid].flat_off <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Re-enters every stored set of a growing (instance, direction) into its
// new, larger table.  Flat over all segments.
template <int W>
__global__ void k_rehash(const RehashSeg *__restrict__ segs, int nseg, int64_t total,
                         const uint64_t *__restrict__ sets, uint64_t *table, uint32_t *status) {
    // a warp takes 32 consecutive indices; lanes 0 and 31 bound the segments
    // they fall in, so every lane searches only that (usually one-entry) range
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < total;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base + lane;
        int a = 0, b = 0;
        if (lane == 0) a = find_seg(segs, 0, nseg - 1, base);
        if (lane == 31) b = find_seg(segs, 0, nseg - 1, min(t, total - 1));
        a = __shfl_sync(0xffffffffu, a, 0);
        b = __shfl_sync(0xffffffffu, b, 31);
        if (t >= total) continue;
        const RehashSeg &S = segs[find_seg(segs, a, b, t)];
        int64_t g = S.set_off + (t - S.flat_off);
        uint64_t s[W];
        load_set<W>(sets + g * W, s);
        insert_stored<W>(table, S.tab_off, S.tab_cap, (uint32_t)S.dir, s, g, status, S.inst);
    }
}

// ------------------------------------------------------------ expand + insert

// CalculateImages / CalculatePreimages (Alg. 1) fused with duplicate
// removal and the equality history: candidate c = p*k + a of a job is the
// image (forward) or preimage (backward) of parent p under letter a.  It is
// written to cand_sets and entered into its (instance, direction) table;
// among equal sets the smallest candidate id keeps the slot (atomicMin), and
// a set already stored (an earlier level) is dropped.  cand_slot[c] = its
// slot, or -1 when dropped (duplicate of history, empty preimage, padding
// between jobs, or table overflow, which also raises kStatusTableFull).
template <int W>
__global__ void __launch_bounds__(256) k_expand(
    const ExpandJob *__restrict__ jobs, int njobs, int64_t ncand, const uint16_t *__restrict__ delta16,
    const uint64_t *__restrict__ pre, const uint64_t *__restrict__ sets, uint64_t *table, uint64_t *cand_sets,
    int64_t *__restrict__ cand_slot, uint32_t *status) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncand;
         c += (int64_t)gridDim.x * blockDim.x) {
        // ncand is a multiple of kScanBlock and jobs start on kScanBlock
        // boundaries, so the 32 candidates of a warp are all in range here
        // and belong to one job: lane 0 finds it for the warp
        int ji = 0;
        if ((threadIdx.x & 31) == 0) ji = find_job_expand(jobs, njobs, c);
        ji = __shfl_sync(0xffffffffu, ji, 0);
        const ExpandJob &J = jobs[ji];
        int64_t local = c - J.cand_off;
        int64_t p = local / J.k;
        if (p >= J.parent_cnt) {  // padding up to the next job's block
            cand_slot[c] = -1;
            continue;
        }
        int a = (int)(local - p * J.k);
        uint64_t S[W], T[W];
        load_set<W>(sets + (J.parent_off + p) * W, S);
        const uint32_t dir = (uint32_t)J.dir;
        if (dir == 0) image<W>(S, delta16 + J.delta_off + (int64_t)a * J.n, T);
        else preimage<W>(S, pre + (J.delta_off + (int64_t)a * J.n) * W, T);
        bool empty = true;
#pragma unroll
        for (int w = 0; w < W; ++w) empty &= (T[w] == 0);
        if (empty) {  // only preimages can be empty; they contain no nonempty set
            cand_slot[c] = -1;
            continue;
        }
#pragma unroll
        for (int w = 0; w < W; ++w) cand_sets[c * W + w] = T[w];
        // the set is published by the release CAS (or release min) below;
        // reads of other candidates' sets follow an acquire of their ids
        const uint64_t me = kCand + (uint64_t)c;
        uint64_t pos = (uint64_t)J.tab_off + __umul64hi(hash_set<W>(dir, T), (uint64_t)J.tab_cap);
        int64_t result = -1;
        int probe = 0;
        for (; probe < kMaxProbe; ++probe) {
            uint64_t *slot = table + pos;
            uint64_t v = ld_acquire(slot);
            if (v == kEmpty) {
                const uint64_t old = cas_acq_rel(slot, kEmpty, me);
                if (old == kEmpty) { result = (int64_t)pos; break; }
                v = old;
            }
            if (v < kCand) {  // a stored set (earlier level)
                if (set_equal<W>(T, sets + v * W)) break;  // seen before: drop
            } else {
                uint64_t c2 = v - kCand;
                if (set_equal_cg<W>(T, cand_sets + c2 * W)) {
                    min_release(slot, me);
                    result = (int64_t)pos;
                    break;
                }
            }
            pos = next_slot(pos, J.tab_off, J.tab_cap);
        }
        if (probe == kMaxProbe) table_full(status, J.inst);
        cand_slot[c] = result;
    }
}

// ------------------------------------------------------------ flag / scan / compact

// A candidate survives when it still owns its slot (it is the first of its
// set in this level and the set was not seen before).  flag[c] = 1 then;
// block_cnt[b] = survivors of block b.  The survivors' cardinalities are
// also counted into hist[job][c] (a block belongs to one job: jobs start on
// block boundaries).
//
// With the inclusion reductions the kernel runs twice.  Phase 1 only sets
// flag[c] (1 = the candidate won its slot, 0 = not).  The marking kernel
// then sets flag[c] = 2 on the winners the reductions remove, and phase 2
// counts and histograms the candidates whose flag is still 1.  Phase 0 is
// the single pass of the plain search.
template <int W>
__global__ void __launch_bounds__(kScanThreads) k_flag_count(
    const ExpandJob *__restrict__ jobs, int njobs, int64_t ncand, const int64_t *__restrict__ cand_slot,
    const uint64_t *__restrict__ table, const uint64_t *__restrict__ cand_sets, uint8_t *__restrict__ flag,
    uint32_t *__restrict__ block_cnt, uint32_t *__restrict__ hist, int phase) {
    constexpr int IPT = kScanBlock / kScanThreads;
    constexpr int HN = card_slots(W);
    __shared__ uint32_t sh[HN];
    int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * IPT;
    if (phase == 1) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            int64_t c = base + i;
            if (c >= ncand) continue;
            int64_t s = cand_slot[c];
            flag[c] = (s >= 0 && table[s] == kCand + (uint64_t)c) ? 1 : 0;
        }
        return;
    }
    const int ji = find_job_expand(jobs, njobs, (int64_t)blockIdx.x * kScanBlock);
    for (int i = threadIdx.x; i < HN; i += kScanThreads) sh[i] = 0;
    __syncthreads();
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        int64_t c = base + i;
        uint8_t f = 0;
        if (c < ncand) {
            if (phase == 0) {
                int64_t s = cand_slot[c];
                f = (s >= 0 && table[s] == kCand + (uint64_t)c) ? 1 : 0;
                flag[c] = f;
            } else {
                f = flag[c] == 1 ? 1 : 0;
            }
            if (f) {
                int pc = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) pc += __popcll(cand_sets[c * W + w]);
                atomicAdd(&sh[pc], 1u);
            }
        }
        cnt += f;
    }
    __shared__ uint32_t red[kScanThreads / 32];
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kScanThreads / 32; ++i) t += red[i];
        block_cnt[blockIdx.x] = t;
    }
    for (int i = threadIdx.x; i < HN; i += kScanThreads)
        if (sh[i]) atomicAdd(&hist[(int64_t)ji * HN + i], sh[i]);
}

// Per job (one block each): the start of every cardinality bucket goes to
// cursor[job][c] - in decreasing order of cardinality for a backward job,
// whose table ge[c] = sets with at least c states also goes to
// meta[ge_off + c] (when the job has a table; ge_off = -1 when the table
// pool was full); in increasing order for a forward job (its permutation).
// card_sum[job] = the summed cardinality of the job's new level (its
// density for the step-cost estimate of Section 2.1.2).
__global__ void k_ge(const ExpandJob *__restrict__ jobs, int hn, const uint32_t *__restrict__ hist,
                     uint32_t *__restrict__ cursor, int32_t *__restrict__ meta, uint64_t *__restrict__ card_sum) {
    const ExpandJob &J = jobs[blockIdx.x];
    if (threadIdx.x != 0) return;
    const uint32_t *h = hist + (int64_t)blockIdx.x * hn;
    uint32_t *cur = cursor + (int64_t)blockIdx.x * hn;
    uint64_t sum = 0;
    for (int c = 0; c < hn; ++c) sum += (uint64_t)c * h[c];
    card_sum[blockIdx.x] = sum;
    if (J.dir == 0) {
        uint32_t below = 0;  // sets with fewer than c states
        for (int c = 0; c < hn; ++c) {
            cur[c] = below;
            below += h[c];
        }
        return;
    }
    uint32_t above = 0;  // sets with more than c states
    for (int c = hn - 1; c >= 0; --c) {
        cur[c] = above;
        above += h[c];
        if (J.ge_off >= 0) meta[J.ge_off + c] = (int32_t)above;
    }
}

// Exclusive scan of the per-block counts in one CTA of 1024 threads;
// block_off[nblocks] = total.
__global__ void __launch_bounds__(1024) k_scan_blocks(int64_t nblocks, const uint32_t *__restrict__ block_cnt,
                                                      uint64_t *__restrict__ block_off) {
    __shared__ uint64_t warp_sum[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nblocks; base += 1024) {
        int64_t i = base + threadIdx.x;
        uint64_t v = (i < nblocks) ? block_cnt[i] : 0;
        uint64_t x = v;  // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) warp_sum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint64_t s = warp_sum[threadIdx.x];
            for (int o = 1; o < 32; o <<= 1) {
                uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (threadIdx.x >= o) s += y;
            }
            warp_sum[threadIdx.x] = s;  // inclusive over warps
        }
        __syncthreads();
        uint64_t before = carry + (threadIdx.x >= 32 ? warp_sum[(threadIdx.x >> 5) - 1] : 0) + x - v;
        if (i < nblocks) block_off[i] = before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) block_off[nblocks] = carry;
}

// Survivors, in candidate order (= the canonical (parent, letter) order),
// are written to their job's new level at dest_off + (rank within the job);
// a job's candidates start on a block boundary, so its first rank is
// block_off of that block.  Forward survivors get their parent link; every
// survivor's table slot is switched from the candidate id to its arena index.
template <int W>
__global__ void __launch_bounds__(kScanThreads) k_compact(
    const ExpandJob *__restrict__ jobs, int njobs, int64_t ncand, const uint8_t *__restrict__ flag,
    const uint64_t *__restrict__ block_off, const uint64_t *__restrict__ cand_sets,
    const int64_t *__restrict__ cand_slot, uint64_t *__restrict__ table, uint64_t *__restrict__ sets,
    uint64_t *__restrict__ link, uint32_t *__restrict__ perm, uint4 *__restrict__ rec,
    uint32_t *__restrict__ cursor) {
    constexpr int IPT = kScanBlock / kScanThreads;
    constexpr int HN = card_slots(W);
    int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * IPT;
    const int ji = find_job_expand(jobs, njobs, (int64_t)blockIdx.x * kScanBlock);
    const ExpandJob &J = jobs[ji];
    uint8_t f[IPT];
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        f[i] = (base + i < ncand && flag[base + i] == 1) ? 1 : 0;  // 2: removed by a reduction
        cnt += f[i];
    }
    // every survivor's place in its cardinality bucket: a block reserves one
    // range per cardinality (the order inside a cardinality is free)
    __shared__ uint32_t sh[HN];
    __shared__ uint32_t sbase[HN];
    for (int i = threadIdx.x; i < HN; i += kScanThreads) sh[i] = 0;
    __syncthreads();
    int pc[IPT];
    uint32_t rk[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        pc[i] = 0;
        rk[i] = 0;
        if (!f[i]) continue;
#pragma unroll
        for (int w = 0; w < W; ++w) pc[i] += __popcll(cand_sets[(base + i) * W + w]);
        rk[i] = atomicAdd(&sh[pc[i]], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < HN; i += kScanThreads)
        sbase[i] = sh[i] ? atomicAdd(&cursor[(int64_t)ji * HN + i], sh[i]) : 0u;
    __syncthreads();
    if (J.dir == 1) {
        // backward: the level itself in decreasing cardinality
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if (!f[i]) continue;
            int64_t c = base + i;
            int64_t g = J.dest_off + (int64_t)(sbase[pc[i]] + rk[i]);
#pragma unroll
            for (int w = 0; w < W; ++w) sets[g * W + w] = cand_sets[c * W + w];
            table[cand_slot[c]] = (uint64_t)g;
        }
        return;
    }
    // forward: the level in canonical (parent, letter) order, plus its
    // permutation perm[dest + i] = canonical position of the i-th set in
    // increasing cardinality
    uint32_t x = cnt;  // inclusive warp scan, then across warps
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    __shared__ uint32_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (cnt == 0) return;
    uint32_t wbefore = 0;
    for (int i = 0; i < (int)(threadIdx.x >> 5); ++i) wbefore += ws[i];
    uint64_t rank = block_off[blockIdx.x] + wbefore + x - cnt;
    const uint64_t first = block_off[J.cand_off / kScanBlock];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        if (!f[i]) continue;
        int64_t c = base + i;
        int64_t g = J.dest_off + (int64_t)(rank - first);
        uint64_t t[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            t[w] = cand_sets[c * W + w];
            sets[g * W + w] = t[w];
        }
        rec[g] = row_record<W>(t);
        int64_t local = c - J.cand_off;
        int64_t p = local / J.k;
        link[g] = ((uint64_t)(J.parent_off + p) << 8) | (uint64_t)(local - p * J.k);
        perm[J.dest_off + sbase[pc[i]] + rk[i]] = (uint32_t)(rank - first);
        table[cand_slot[c]] = (uint64_t)g;
        ++rank;
    }
}

// Survivors per job: block_off at the job's last block minus at its first.
__global__ void k_job_counts(const ExpandJob *__restrict__ jobs, int njobs, int64_t nblocks,
                             const uint64_t *__restrict__ block_off, uint64_t *__restrict__ counts) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= njobs) return;
    int64_t b0 = jobs[j].cand_off / kScanBlock;
    int64_t b1 = (j + 1 < njobs) ? jobs[j + 1].cand_off / kScanBlock : nblocks;
    counts[j] = block_off[b1] - block_off[b0];
}

// ------------------------------------------------------------ meet check

// Meet condition (Section 2): is some forward set X = F[f] inside some
// backward set Y = B[b], i.e. X & ~Y == 0 on every word?  Per job the
// smallest such f is wanted (it gives the least reset word); best[slot]
// = min over found pairs of (f << 32 | b).
//
// The F x B pair space of every job is cut into tiles of TF = NT*R forward
// rows by tb backward rows, numbered F-major so that low f come first.
// Each thread keeps R forward sets in registers as 32-bit halves; the
// backward tile sits in shared memory word-major (word w of set i at
// sB[w*tb + i]) so that one 16-byte broadcast load gives word w of two
// backward sets.  A pair costs 2W three-input LOP3 steps
// acc |= f & ~y and one compare, accumulated into a per-row hit flag; the
// rare hit is located by a second pass.  A tile whose first row is beyond
// the best f already found is skipped.
template <int W, int R, int NT>
__global__ void __launch_bounds__(NT) k_meet(const MeetJob *__restrict__ jobs, int njobs,
                                             const int64_t *__restrict__ ntiles_p, int tb,
                                             const uint64_t *__restrict__ sets, unsigned long long *best,
                                             unsigned long long *pairs_done) {
    const int64_t ntiles = *ntiles_p;
    extern __shared__ __align__(16) uint64_t sB[];  // [W][tb]
    __shared__ int64_t s_job;
    __shared__ int s_skip;
    constexpr int TF = NT * R;
    unsigned long long my_pairs = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = njobs - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (jobs[mid].tile_off <= tile) lo = mid; else hi = mid - 1;
            }
            s_job = lo;
            const MeetJob &J = jobs[lo];
            int64_t local = tile - J.tile_off;
            int64_t tf = local / J.ntb;
            unsigned long long cur = *(volatile unsigned long long *)(best + J.slot);
            s_skip = ((int64_t)(cur >> 32) < tf * TF) ? 1 : 0;
        }
        __syncthreads();
        if (s_skip) { __syncthreads(); continue; }
        const MeetJob &J = jobs[s_job];
        int64_t local = tile - J.tile_off;
        int64_t tf = local / J.ntb;
        int64_t tbi = local - tf * J.ntb;
        int64_t f0 = tf * TF;
        int64_t b0 = tbi * tb;
        int nb = (int)min((int64_t)tb, J.b_cnt - b0);
        // backward tile -> shared memory, word-major; rows nb..(even) are empty sets
        const uint64_t *gB = sets + (J.b_off + b0) * W;
        int nbe = (nb + 1) & ~1;
        for (int e = threadIdx.x; e < nbe * W; e += NT) {
            int i = e / W, w = e - i * W;
            sB[w * tb + i] = (i < nb) ? gB[e] : 0ull;
        }
        // forward rows -> registers
        uint32_t f[R][2 * W];
        bool valid[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t row = f0 + r * NT + threadIdx.x;
            valid[r] = row < J.f_cnt;
            const uint64_t *p = sets + (J.f_off + (valid[r] ? row : 0)) * W;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint64_t v = p[w];
                f[r][2 * w] = (uint32_t)v;
                f[r][2 * w + 1] = (uint32_t)(v >> 32);
            }
        }
        __syncthreads();
        bool hit[R];
#pragma unroll
        for (int r = 0; r < R; ++r) hit[r] = false;
        for (int i = 0; i < nbe; i += 2) {
            uint32_t y0[2 * W], y1[2 * W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint4 v = *reinterpret_cast<const uint4 *>(sB + w * tb + i);
                y0[2 * w] = v.x; y0[2 * w + 1] = v.y;
                y1[2 * w] = v.z; y1[2 * w + 1] = v.w;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                uint32_t a0 = f[r][0] & ~y0[0];
                uint32_t a1 = f[r][0] & ~y1[0];
#pragma unroll
                for (int h = 1; h < 2 * W; ++h) {
                    a0 |= f[r][h] & ~y0[h];
                    a1 |= f[r][h] & ~y1[h];
                }
                hit[r] |= (a0 == 0) | (a1 == 0);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (hit[r] && valid[r]) {  // rare: find the first b of this row
                for (int i = 0; i < nb; ++i) {
                    uint32_t acc = 0;
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        uint64_t y = sB[w * tb + i];
                        acc |= (f[r][2 * w] & ~(uint32_t)y) | (f[r][2 * w + 1] & ~(uint32_t)(y >> 32));
                    }
                    if (acc == 0) {
                        unsigned long long key = ((unsigned long long)(f0 + r * NT + threadIdx.x) << 32) |
                                                 (unsigned long long)(b0 + i);
                        atomicMin(best + J.slot, key);
                        break;
                    }
                }
            }
        }
        if (threadIdx.x == 0) {
            int64_t rows = min((int64_t)TF, J.f_cnt - f0);
            my_pairs += (unsigned long long)rows * (unsigned long long)nb;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && my_pairs) atomicAdd(pairs_done, my_pairs);
}

// Meet check by vertical bitmaps.  A backward chunk of up to kBmRows(LW)
// sets B[b0 ..] is transposed into shared memory as one bitmap per state:
// bit b of M_q is set iff state q lies in B[b0 + b].  Then X is inside
// B[b0 + b] iff bit b survives the AND of M_q over the states q of X.  A
// warp takes one forward set X at a time; lane l holds 64*LW bits of the
// running AND and the warp stops as soon as every lane is zero (after about
// five states of X on random instances, against 2W LOP3 per pair for the
// direct test).  Forward rows are visited in increasing cardinality (the
// level's permutation) and backward sets sit in decreasing cardinality, so
// X needs only the first ge[|X|] backward sets: a row stops at that bound,
// a warp stops at its first row with no candidate in the chunk, and a tile
// whose first (smallest) row has none is skipped before it is transposed.
// The least meeting canonical position f is kept with atomicMin; rows at or
// past the best f found so far are passed over.
//
// Shared layout: M_q occupies kWords = 64*LW 32-bit words, cut into units of
// U words (16 bytes, or 8 when LW = 1); lane l owns units l + 32h, h < UPL.
// Consecutive bitmaps are kStride = kWords + U words apart: in the AND loop a
// warp reads one bitmap as one contiguous run (no bank conflict), and the
// padding of one unit per state spreads the transposing stores (one state
// per lane, same word) over the banks, at most 4-way conflicted.
template <int LW>
struct Bm {
    static constexpr int kRows = 2048 * LW;          // backward sets per chunk
    static constexpr int kWords = 64 * LW;           // 32-bit words per state bitmap
    static constexpr int U = LW >= 2 ? 4 : 2;        // 32-bit words per unit
    static constexpr int UPL = 2 * LW / U;           // units per lane
    static constexpr int kStride = kWords + U;       // words from one bitmap to the next
    __host__ __device__ static constexpr int pos(int q, int g) { return q * kStride + g; }
    // first row of lane l's unit h within the chunk
    __device__ static __forceinline__ int row0(int lane, int h) { return (lane + 32 * h) * 32 * U; }
};

// Words per lane of the running AND by default (4 only on request).
__host__ __device__ constexpr int bm_lanes_words(int W) { return W <= 3 ? 2 : 1; }
__host__ __device__ constexpr int bm_smem_bytes_n(int n_cap, int LW) { return n_cap * (64 * LW + (LW >= 2 ? 4 : 2)) * 4; }
__host__ __device__ constexpr int bm_smem_bytes(int W, int LW) { return bm_smem_bytes_n(64 * W, LW); }
constexpr int kBmThreads = 512;
static_assert(bm_smem_bytes(3, 2) == 64 * 3 * Bm<2>::kStride * 4, "bitmap layout size");

// 32x32 bit transpose across a warp: lane j holds row j on entry (bit i =
// entry (j, i)); on exit lane i holds column i (bit j = entry (j, i)).
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t v, int lane) {
    const uint32_t lo[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int s = 16 >> st;
        uint32_t o = __shfl_xor_sync(0xffffffffu, v, s);
        v = (lane & s) ? ((v & ~lo[st]) | ((o & ~lo[st]) >> s)) : ((v & lo[st]) | ((o & lo[st]) << s));
    }
    return v;
}

template <int W, int LW, int NT>
__global__ void __launch_bounds__(NT) k_meet_bm(const MeetJob *__restrict__ jobs, int njobs,
                                                int64_t *__restrict__ ntiles_p, int tf_rows, int n_cap,
                                                const uint64_t *__restrict__ sets,
                                                const uint32_t *__restrict__ perm,
                                                const uint4 *__restrict__ rec,
                                                unsigned long long *best, unsigned long long *pairs_done,
                                                unsigned long long *and_iters,
                                                unsigned long long *rows_transposed,
                                                const int32_t *__restrict__ meta) {
    constexpr int HN = card_slots(W);
    using G = Bm<LW>;
    constexpr int HW = G::U / 2;  // 64-bit acc words per unit
    const int64_t ntiles = ntiles_p[0];
    // tiles are handed out one at a time from the counter ntiles_p[1]
    // (zeroed by k_meet_prep), in increasing order, so that a CTA that drew
    // cheap or skipped tiles takes more of them
    unsigned long long *next_tile = reinterpret_cast<unsigned long long *>(ntiles_p + 1);
    extern __shared__ __align__(16) uint32_t sT[];  // [n_cap][G::kStride]
    __shared__ int64_t s_job, s_tile;
    __shared__ int s_skip;
    __shared__ unsigned long long s_best;
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long my_rows = 0;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(next_tile, 1ull);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;
        if (threadIdx.x == 0) {
            int lo = 0, hi = njobs - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (jobs[mid].tile_off <= tile) lo = mid; else hi = mid - 1;
            }
            s_job = lo;
            const MeetJob &J = jobs[lo];
            const int64_t local = tile - J.tile_off;
            const int64_t tf = local / J.ntb;
            const int64_t b0 = (local - tf * J.ntb) * G::kRows;
            // forward rows come in increasing cardinality: the tile's first
            // row has the fewest states, and no backward set of this chunk
            // can hold it when the chunk starts past ge[that cardinality]
            int skip = 0;
            if (J.ge_off >= 0) {
                const uint32_t f_first = perm[J.f_off + tf * tf_rows];
                const int card = (int)(rec[J.f_off + f_first].w >> 16);
                skip = b0 >= (int64_t)meta[J.ge_off + min(card, HN - 1)];
            }
            s_best = *(volatile unsigned long long *)(best + J.slot);
            s_skip = skip;
        }
        __syncthreads();
        if (s_skip) { __syncthreads(); continue; }
        const MeetJob &J = jobs[s_job];
        const int64_t local = tile - J.tile_off;
        const int64_t tf = local / J.ntb;
        const int64_t b0 = (local - tf * J.ntb) * G::kRows;
        const int nb = (int)min((int64_t)G::kRows, J.b_cnt - b0);
        const int64_t i0 = tf * tf_rows;
        const int64_t i1 = min(i0 + tf_rows, J.f_cnt);
        // 1. transpose the backward chunk: group g = rows 32g..32g+31
        my_rows += (unsigned long long)nb;
        for (int g = warp; g < G::kRows / 32; g += NW) {
            int row = g * 32 + lane;
            uint64_t y[W];
            if (row < nb) load_set<W>(sets + (J.b_off + b0 + row) * W, y);
            else {
#pragma unroll
                for (int w = 0; w < W; ++w) y[w] = 0;
            }
#pragma unroll
            for (int h = 0; h < 2 * W; ++h) {
                if (32 * h >= n_cap) break;  // no set holds these states: no bitmap is kept
                uint32_t v = (h & 1) ? (uint32_t)(y[h >> 1] >> 32) : (uint32_t)y[h >> 1];
                uint32_t c = warp_transpose32(v, lane);  // column lane: state 32h + lane
                if (32 * h + lane < n_cap) sT[G::pos(32 * h + lane, g)] = c;
            }
        }
        __syncthreads();
        // 2. forward rows (in increasing cardinality), one per warp at a time;
        //    f is the row's canonical position, and only the least meeting f
        //    matters, so rows at or past the best f found are passed over
        const int32_t *ge = J.ge_off >= 0 ? meta + J.ge_off : nullptr;
        // row indices within the tile are 32-bit (a tile has at most
        // tf_rows rows); the tile's rows start at permutation entry i0
        const uint32_t *pt = perm + J.f_off + i0;
        const uint4 *rt = rec + J.f_off;
        const int ni = (int)(i1 - i0);
        int li = warp;
        uint32_t f = 0, fn = 0;
        uint4 r = make_uint4(0, 0, 0, 0);
        if (li < ni) {
            f = __ldg(pt + li);
            r = __ldg(rt + f);
        }
        if (li + NW < ni) fn = __ldg(pt + li + NW);
        int last_card = -1, rows = 0;
        // this warp's counts for the tile (rows tested since the last change
        // of the bound, pairs, AND steps), added to the totals once per tile;
        // 32 bits hold them: a warp tests at most 2^20 / 16 rows of a tile,
        // each against at most 8192 sets and with at most 576 steps
        uint32_t run_rows = 0, t_iters = 0, t_pairs = 0;
        // the least meeting f known to this warp: rows at or past it are
        // passed over.  It is re-read from the block's best every 8 rows and
        // after each meet of this warp; a stale (larger) value only costs
        // work, never a result, since every meet goes through atomicMin.
        uint32_t best_f = 0xFFFFFFFFu;
        uint32_t mask[2 * LW];
        // this lane's units of a state bitmap start at sT + q * kStride + lbase
        const uint32_t *lbase = sT + lane * G::U;
        for (; li < ni; li += NW) {
            // prefetch: the record of the next row, the index of the one after
            uint32_t fnn = 0;
            uint4 rn = make_uint4(0, 0, 0, 0);
            if (li + 2 * NW < ni) fnn = __ldg(pt + li + 2 * NW);
            if (li + NW < ni) rn = __ldg(rt + fn);
            // lane 0 reads the shared best; the whole warp follows its value
            // (the walk's votes need every lane of the warp)
            if (((li / NW) & 7) == 0)
                best_f = __shfl_sync(0xffffffffu,
                                     (uint32_t)(*(volatile unsigned long long *)&s_best >> 32), 0);
            const bool pass = f >= best_f;
            // only the backward sets with at least |X| states can contain X;
            // rows come in increasing cardinality, so the bound changes rarely
            const int card = (int)(r.w >> 16);
            if (card != last_card) {
                t_pairs += run_rows * (uint32_t)rows;
                run_rows = 0;
                int64_t end = ge ? (int64_t)__ldg(ge + min(card, HN - 1)) : J.b_cnt;
                if (end <= b0) break;  // later rows have at least as many states: none fits here
                rows = (int)min((int64_t)nb, end - b0);
#pragma unroll
                for (int j = 0; j < LW; ++j) {
                    int lim = rows - (G::row0(lane, j / HW) + 64 * (j % HW));
                    uint64_t m = lim >= 64 ? ~0ull : (lim > 0 ? ((1ull << lim) - 1) : 0ull);
                    mask[2 * j] = (uint32_t)m;
                    mask[2 * j + 1] = (uint32_t)(m >> 32);
                }
                last_card = card;
            }
            if (!pass) {
                // The running intersection, 2*LW 32-bit words per lane.  The
                // walk ANDs two state bitmaps per step (one three-input LOP3
                // per word) and votes after the 4th, 6th and 7th listed state
                // and after every further state.  The record repeats the
                // first state in the fields of a set with fewer than seven,
                // so every row walks all seven fields.  From the first vote
                // on, a lane whose words are all zero skips its loads (its
                // words stay zero whatever it would have read).
                uint32_t acc[2 * LW];
#pragma unroll
                for (int j = 0; j < 2 * LW; ++j) acc[j] = mask[j];
                struct Frag {
                    uint32_t w[2 * LW];
                };
                // loads the lane's words of state q's bitmap into fr; a lane
                // with `on` false keeps fr's old words (its intersection is
                // already all zero, so they change nothing), which spares
                // the zeroing
                auto load_into = [&](Frag &fr, int q, bool on) {
                    const uint32_t *row = lbase + q * G::kStride;
#pragma unroll
                    for (int h = 0; h < G::UPL; ++h) {
                        const uint32_t *p = row + 32 * h * G::U;
                        if constexpr (G::U == 4) {
                            if (on) {
                                const uint4 v = *reinterpret_cast<const uint4 *>(p);
                                fr.w[4 * h] = v.x;
                                fr.w[4 * h + 1] = v.y;
                                fr.w[4 * h + 2] = v.z;
                                fr.w[4 * h + 3] = v.w;
                            }
                        } else {
                            if (on) {
                                const uint2 v = *reinterpret_cast<const uint2 *>(p);
                                fr.w[2 * h] = v.x;
                                fr.w[2 * h + 1] = v.y;
                            }
                        }
                    }
                };
                auto and2 = [&](const Frag &x, const Frag &y) {
#pragma unroll
                    for (int j = 0; j < 2 * LW; ++j) acc[j] &= x.w[j] & y.w[j];
                };
                auto and1 = [&](const Frag &x) {
#pragma unroll
                    for (int j = 0; j < 2 * LW; ++j) acc[j] &= x.w[j];
                };
                auto lane_alive = [&]() {
                    uint32_t any = 0;
#pragma unroll
                    for (int j = 0; j < 2 * LW; ++j) any |= acc[j];
                    return any != 0;
                };
                const int s0 = (int)(r.x & 0xFFFFu), s1 = (int)(r.x >> 16);
                const int s2 = (int)(r.y & 0xFFFFu), s3 = (int)(r.y >> 16);
                const int s4 = (int)(r.z & 0xFFFFu), s5 = (int)(r.z >> 16);
                const int s6 = (int)(r.w & 0xFFFFu);
                uint32_t steps = 4;
                bool la, alive;
                Frag fa0, fb0, fa1, fb1;
                load_into(fa0, s0, true);
                load_into(fb0, s1, true);
                load_into(fa1, s2, true);
                load_into(fb1, s3, true);
                and2(fa0, fb0);
                and2(fa1, fb1);
                la = lane_alive();
                load_into(fa0, s4, la);
                load_into(fb0, s5, la);
                alive = __any_sync(0xffffffffu, la);
                if (alive) {
                    steps = 6;
                    and2(fa0, fb0);
                    la = lane_alive();
                    load_into(fa1, s6, la);
                    alive = __any_sync(0xffffffffu, la);
                    if (alive) {
                        steps = 7;
                        and1(fa1);
                        la = lane_alive();
                        alive = __any_sync(0xffffffffu, la);
                    }
                }
                if (alive && card > 7) {
                    // the states after the seventh, from the set itself
                    uint64_t x[W];
                    load_set<W>(sets + (J.f_off + f) * W, x);
#pragma unroll
                    for (int h = 0; h < 2 * W; ++h) {
                        uint32_t bits = (h & 1) ? (uint32_t)(x[h >> 1] >> 32) : (uint32_t)x[h >> 1];
                        const int lo = 32 * h;
                        if (s6 >= lo + 31) bits = 0;
                        else if (s6 >= lo) bits &= ~((2u << (s6 - lo)) - 1u);
                        while (bits && alive) {
                            const int q = lo + __ffs(bits) - 1;
                            bits &= bits - 1;
                            load_into(fa0, q, la);
                            and1(fa0);
                            la = lane_alive();
                            alive = __any_sync(0xffffffffu, la);
                            ++steps;
                        }
                    }
                }
                t_iters += steps;
                ++run_rows;
                if (alive) {  // every state of X processed: X lies inside the surviving sets
                    unsigned ball = __ballot_sync(0xffffffffu, la);
                    if (lane == __ffs(ball) - 1) {
                        // first nonzero word of the lane, by selects (no
                        // dynamic index, which would put acc in local memory)
                        int j = 0;
                        uint32_t v = acc[0];
#pragma unroll
                        for (int t = 1; t < 2 * LW; ++t)
                            if (v == 0) {
                                v = acc[t];
                                j = t;
                            }
                        const int j64 = j >> 1;
                        unsigned long long key =
                            ((unsigned long long)f << 32) |
                            (unsigned long long)(b0 + G::row0(lane, j64 / HW) + 64 * (j64 % HW) + 32 * (j & 1) +
                                                 __ffs(v) - 1);
                        atomicMin(&s_best, key);
                        atomicMin(best + J.slot, key);
                    }
                    best_f = min(best_f, f);
                }
            }
            f = fn;
            r = rn;
            fn = fnn;
        }
        t_pairs += run_rows * (uint32_t)rows;
        // per-warp counters: lanes counted the same rows and iterations
        if (lane == 0 && t_iters) {
            atomicAdd(pairs_done, (unsigned long long)t_pairs);
            atomicAdd(and_iters, (unsigned long long)t_iters);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && my_rows) atomicAdd(rows_transposed, my_rows);
}

// ------------------------------------------------------------ inclusion reductions

// One unit of work of the reductions of Alg. 1 (Section 2.1).  rows x chunk
// are tested for inclusion "row inside chunk set":
//   col = 0: the rows are the targets: a row that lies inside some set of
//            the chunk is removed (IBFS: self-reduction to maximal sets,
//            and subsets of the history);
//   col = 1: the chunk sets are the targets: a chunk set that contains some
//            row is removed (BFS: self-reduction to minimal sets, and
//            supersets of the history).
// A side lies either in candidate space (the winners of this expansion,
// flag 1 = kept so far, 2 = removed, 0 = not a winner) or in the arena (a
// kept level of an earlier depth).  self = 1 when both sides are the same
// candidates: a set is not its own witness, and since the winners are
// distinct sets, inclusion between two of them is proper.  Witnesses are
// never filtered by marks (a removed set still removes its supersets or
// subsets, as in Alg. 1 where both reductions test the deduplicated list),
// so the result does not depend on the order in which tiles run; targets
// already removed are skipped.
struct MarkJob {
    int64_t tile_off;          // first tile of this job
    int64_t ntc;               // chunk tiles
    int64_t r_off, r_cnt;      // rows: candidate ids (r_cand) or arena indices
    int64_t c_off, c_cnt;      // chunk: candidate ids (c_cand) or arena indices
    int64_t ge_off;            // arena chunk sorted by decreasing cardinality: its ge table, or -1
    int32_t r_cand, c_cand, col, self;
    int32_t r_perm;            // arena rows of a forward level, visited through its permutation
    int32_t pad;               // (increasing cardinality), so a warp stops at its first row too large
};

// Inclusion marking by vertical bitmaps, as k_meet_bm: the chunk (up to
// Bm<LW>::kRows sets) is transposed into one bitmap per state in shared
// memory, and a warp ANDs the bitmaps of a row's states, two per step (a
// three-input LOP3 per word), voting after the fourth state and after every
// second one from there on.  A row whose intersection survives lies inside
// the surviving chunk sets.  Tiles of tr_rows rows x one chunk are drawn
// from the counter ntiles_p[1] (zeroed by the host).  counters: [0] AND
// steps, [1] chunk rows transposed, [2] (row, chunk set) pairs covered.
template <int W, int LW, int NT>
__global__ void __launch_bounds__(NT) k_mark_bm(const MarkJob *__restrict__ jobs, int njobs,
                                                int64_t *__restrict__ ntiles_p, int tr_rows, int n_cap,
                                                const uint64_t *__restrict__ sets,
                                                const uint64_t *__restrict__ cand_sets, uint8_t *flag,
                                                const int32_t *__restrict__ meta,
                                                const uint32_t *__restrict__ perm,
                                                unsigned long long *counters) {
    constexpr int HN = card_slots(W);
    using G = Bm<LW>;
    constexpr int HW = G::U / 2;
    constexpr int NW = NT / 32;
    constexpr int NWORD = 2 * LW;  // 32-bit words of the running AND per lane
    const int64_t ntiles = ntiles_p[0];
    unsigned long long *next_tile = reinterpret_cast<unsigned long long *>(ntiles_p + 1);
    extern __shared__ __align__(16) uint32_t sT[];
    __shared__ int64_t s_tile;
    __shared__ int s_job, s_maxcard;
    __shared__ uint32_t s_hit[32 * NWORD];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long my_steps = 0, my_rows = 0, my_pairs = 0;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(next_tile, 1ull);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;
        if (threadIdx.x == 0) {
            int lo = 0, hi = njobs - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (jobs[mid].tile_off <= tile) lo = mid; else hi = mid - 1;
            }
            s_job = lo;
            s_maxcard = -1;
        }
        for (int t = threadIdx.x; t < 32 * NWORD; t += NT) s_hit[t] = 0;
        __syncthreads();
        const MarkJob &J = jobs[s_job];
        const int64_t local = tile - J.tile_off;
        const int64_t tr = local / J.ntc;
        const int64_t b0 = (local - tr * J.ntc) * G::kRows;
        const int nb = (int)min((int64_t)G::kRows, J.c_cnt - b0);
        const int64_t i0 = tr * tr_rows, i1 = min(i0 + tr_rows, J.r_cnt);
        // 1. the chunk, transposed; in candidate space only the winners
        //    (witnesses) or the winners still kept (targets) take part
        const uint64_t *csrc = J.c_cand ? cand_sets : sets;
        int wmax = -1;
        for (int g = warp; g < G::kRows / 32; g += NW) {
            const int row = g * 32 + lane;
            uint64_t y[W];
#pragma unroll
            for (int w = 0; w < W; ++w) y[w] = 0;
            if (row < nb) {
                const int64_t idx = J.c_off + b0 + row;
                bool in = true;
                if (J.c_cand) {
                    const uint8_t fl = flag[idx];
                    in = J.col ? fl == 1 : fl != 0;
                }
                if (in) {
                    load_set<W>(csrc + idx * W, y);
                    int pc = 0;
#pragma unroll
                    for (int w = 0; w < W; ++w) pc += __popcll(y[w]);
                    wmax = max(wmax, pc);
                }
            }
#pragma unroll
            for (int h = 0; h < 2 * W; ++h) {
                if (32 * h >= n_cap) break;
                uint32_t v = (h & 1) ? (uint32_t)(y[h >> 1] >> 32) : (uint32_t)y[h >> 1];
                uint32_t c = warp_transpose32(v, lane);
                if (32 * h + lane < n_cap) sT[G::pos(32 * h + lane, g)] = c;
            }
        }
        for (int o = 16; o; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        if (lane == 0 && wmax >= 0) atomicMax(&s_maxcard, wmax);
        if (threadIdx.x == 0) my_rows += (unsigned long long)max(nb, 0);
        __syncthreads();
        const int maxcard = s_maxcard;
        const int32_t *ge = J.ge_off >= 0 ? meta + J.ge_off : nullptr;
        const uint64_t *rsrc = J.r_cand ? cand_sets : sets;
        const uint32_t *lbase = sT + lane * G::U;
        uint32_t hit[NWORD];
#pragma unroll
        for (int j = 0; j < NWORD; ++j) hit[j] = 0;
        // 2. rows, one per warp at a time
        for (int64_t i = i0 + warp; maxcard >= 0 && i < i1; i += NW) {
            const int64_t ridx = J.r_perm ? J.r_off + (int64_t)__ldg(perm + J.r_off + i) : J.r_off + i;
            if (J.r_cand) {
                // lane 0 reads the flag; the warp follows its decision
                int fl = lane == 0 ? (int)flag[ridx] : 0;
                fl = __shfl_sync(0xffffffffu, fl, 0);
                if (J.col ? fl == 0 : fl != 1) continue;
            }
            uint64_t x[W];
            load_set<W>(rsrc + ridx * W, x);
            int card = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) card += __popcll(x[w]);
            if (card > maxcard) {  // no chunk set is large enough to hold it
                if (J.r_perm) break;  // nor any later row of this warp (increasing cardinality)
                continue;
            }
            int limit = nb;
            if (ge) limit = (int)min((int64_t)nb, (int64_t)__ldg(ge + min(card, HN - 1)) - b0);
            if (limit <= 0) continue;
            uint32_t acc[NWORD];
#pragma unroll
            for (int j = 0; j < LW; ++j) {
                const int lim = limit - (G::row0(lane, j / HW) + 64 * (j % HW));
                const uint64_t m = lim >= 64 ? ~0ull : (lim > 0 ? ((1ull << lim) - 1) : 0ull);
                acc[2 * j] = (uint32_t)m;
                acc[2 * j + 1] = (uint32_t)(m >> 32);
            }
            if (J.self) {  // a set is not its own witness
                const int64_t own = ridx - (J.c_off + b0);
                if (own >= 0 && own < nb) {
                    const int o = (int)own;
                    const int u = o / (32 * G::U), e = o % (32 * G::U);
                    if ((u & 31) == lane) {
                        const int jj = 2 * ((u >> 5) * HW + e / 64) + ((e % 64) >> 5);
#pragma unroll
                        for (int t = 0; t < NWORD; ++t)
                            if (t == jj) acc[t] &= ~(1u << (e & 31));
                    }
                }
            }
            my_pairs += (unsigned long long)limit;
            struct Frag {
                uint32_t w[NWORD];
            };
            // as in the meet kernel: a lane with `on` false keeps fr's old
            // words (its intersection is already zero)
            auto load_into = [&](Frag &fr, int q, bool on) {
                const uint32_t *rowp = lbase + q * G::kStride;
#pragma unroll
                for (int h = 0; h < G::UPL; ++h) {
                    const uint32_t *p = rowp + 32 * h * G::U;
                    if constexpr (G::U == 4) {
                        if (on) {
                            const uint4 v = *reinterpret_cast<const uint4 *>(p);
                            fr.w[4 * h] = v.x;
                            fr.w[4 * h + 1] = v.y;
                            fr.w[4 * h + 2] = v.z;
                            fr.w[4 * h + 3] = v.w;
                        }
                    } else {
                        if (on) {
                            const uint2 v = *reinterpret_cast<const uint2 *>(p);
                            fr.w[2 * h] = v.x;
                            fr.w[2 * h + 1] = v.y;
                        }
                    }
                }
            };
            Frag fa, fb;
#pragma unroll
            for (int j = 0; j < NWORD; ++j) fa.w[j] = fb.w[j] = 0;
            bool la = true, alive = true;
            int walked = 0, pend = -1;
            // the row's states in increasing order, ANDed two at a time
#pragma unroll
            for (int h = 0; h < 2 * W; ++h) {
                uint32_t bits = (h & 1) ? (uint32_t)(x[h >> 1] >> 32) : (uint32_t)x[h >> 1];
                while (bits && alive) {
                    const int q = 32 * h + __ffs(bits) - 1;
                    bits &= bits - 1;
                    if (pend < 0) {
                        pend = q;
                        continue;
                    }
                    load_into(fa, pend, la);
                    load_into(fb, q, la);
#pragma unroll
                    for (int j = 0; j < NWORD; ++j) acc[j] &= fa.w[j] & fb.w[j];
                    pend = -1;
                    walked += 2;
                    if (walked >= 4) {
                        uint32_t any = 0;
#pragma unroll
                        for (int j = 0; j < NWORD; ++j) any |= acc[j];
                        la = any != 0;
                        alive = __any_sync(0xffffffffu, la);
                    }
                }
            }
            if (alive && pend >= 0) {
                load_into(fa, pend, la);
#pragma unroll
                for (int j = 0; j < NWORD; ++j) acc[j] &= fa.w[j];
                ++walked;
            }
            if (alive) {
                uint32_t any = 0;
#pragma unroll
                for (int j = 0; j < NWORD; ++j) any |= acc[j];
                la = any != 0;
                alive = __any_sync(0xffffffffu, la);
            }
            my_steps += (unsigned long long)walked;
            if (alive) {  // every state of the row processed: it lies inside the surviving chunk sets
                if (!J.col) {
                    if (lane == 0) flag[ridx] = 2;
                } else {
#pragma unroll
                    for (int j = 0; j < NWORD; ++j) hit[j] |= acc[j];
                }
            }
        }
        if (J.col) {
#pragma unroll
            for (int j = 0; j < NWORD; ++j)
                if (hit[j]) atomicOr(&s_hit[lane * NWORD + j], hit[j]);
            __syncthreads();
            for (int t = threadIdx.x; t < 32 * NWORD; t += NT) {
                uint32_t bits = s_hit[t];
                const int ln = t / NWORD, jj = t % NWORD, j = jj >> 1;
                const int base = G::row0(ln, j / HW) + 64 * (j % HW) + 32 * (jj & 1);
                while (bits) {
                    const int b = base + __ffs(bits) - 1;
                    bits &= bits - 1;
                    if (b < nb) flag[J.c_off + b0 + b] = 2;
                }
            }
        }
        __syncthreads();
    }
    if (lane == 0) {
        if (my_steps) atomicAdd(counters, my_steps);
        if (my_pairs) atomicAdd(counters + 2, my_pairs);
    }
    if (threadIdx.x == 0 && my_rows) atomicAdd(counters + 1, my_rows);
}

// ------------------------------------------------------------ word recovery

// One CTA per met instance.  The prefix x is the forward parent chain of the
// meeting set X (the predecessor pointers of Section 2).  The suffix y is
// the least word of length j mapping X to one state: letter by letter, the
// smallest a such that delta(S, a) lies inside some set of B_m, m = the
// letters still to come (a set inside a depth-m backward set is exactly a
// set that m more letters can map to one state, and by minimality of r that
// backward set was first reached at depth m).  Finally |delta(Q, xy)| = 1 is
// checked.  word_status[slot]: 0 ok, else kStatusWordFail/kStatusVerifyFail.
// blevels holds (offset, count, cardinality table or -1) per backward level.
template <int W, int NT>
__global__ void __launch_bounds__(NT) k_words(const WordJob *__restrict__ jobs,
                                              const int64_t *__restrict__ blevels,
                                              const uint16_t *__restrict__ delta16,
                                              const uint64_t *__restrict__ sets,
                                              const uint64_t *__restrict__ link, const int32_t *__restrict__ meta,
                                              uint8_t *__restrict__ words, uint32_t *__restrict__ word_status) {
    constexpr int HN = card_slots(W);
    const WordJob J = jobs[blockIdx.x];
    uint8_t *out = words + J.word_off;
    __shared__ int s_choice;
    __shared__ uint32_t s_fail;
    __shared__ volatile int s_found;
    if (threadIdx.x == 0) {
        s_fail = 0;
        uint64_t g = (uint64_t)J.f_arena;
        for (int d = J.i - 1; d >= 0; --d) {
            uint64_t l = link[g];
            out[d] = (uint8_t)(l & 0xFF);
            g = l >> 8;
        }
    }
    uint64_t S[W];
    load_set<W>(sets + J.f_arena * W, S);
    __syncthreads();
    for (int t = 0; t < J.j; ++t) {
        int m = J.j - 1 - t;
        const int64_t *lv = blevels + 3 * (J.blev + m);
        int64_t off = lv[0], cnt = lv[1], ge = lv[2];
        if (threadIdx.x == 0) s_choice = -1;
        __syncthreads();
        for (int a = 0; a < J.k; ++a) {
            uint64_t T[W];
            image<W>(S, delta16 + J.delta_off + (int64_t)a * J.n, T);
            // the level is in decreasing cardinality: only its first ge[|T|]
            // sets can contain T
            int card = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) card += __popcll(T[w]);
            int64_t lim = ge >= 0 ? (int64_t)meta[ge + min(card, HN - 1)] : cnt;
            if (threadIdx.x == 0) s_found = 0;
            __syncthreads();
            int found = 0;
            for (int64_t b = threadIdx.x; b < lim && !s_found; b += NT) {
                const uint64_t *y = sets + (off + b) * W;
                uint64_t acc = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) acc |= T[w] & ~y[w];
                if (acc == 0) {
                    found = 1;
                    s_found = 1;
                }
            }
            if (__syncthreads_or(found)) {
                if (threadIdx.x == 0) s_choice = a;
                __syncthreads();
                break;
            }
        }
        int a = s_choice;
        if (a < 0) {
            if (threadIdx.x == 0) s_fail = kStatusWordFail;
            break;
        }
        uint64_t T[W];
        image<W>(S, delta16 + J.delta_off + (int64_t)a * J.n, T);
#pragma unroll
        for (int w = 0; w < W; ++w) S[w] = T[w];
        if (threadIdx.x == 0) out[J.i + t] = (uint8_t)a;
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t st = s_fail;
        if (!st) {  // verify: delta(Q, word) is a singleton
            uint64_t Q[W], T[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                int lo = w * 64;
                Q[w] = (J.n >= lo + 64) ? ~0ull : (J.n > lo ? ((1ull << (J.n - lo)) - 1) : 0ull);
            }
            for (int t = 0; t < J.i + J.j; ++t) {
                image<W>(Q, delta16 + J.delta_off + (int64_t)out[t] * J.n, T);
#pragma unroll
                for (int w = 0; w < W; ++w) Q[w] = T[w];
            }
            int pc = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) pc += __popcll(Q[w]);
            if (pc != 1) st = kStatusVerifyFail;
        }
        word_status[J.slot] = st;
    }
}

// Preimage tables of one instance per blockIdx.y: pre[(a*n + t)*W ..] is the
// bitset {p : delta(p, a) = t}.  The rows are cleared first, then every
// (a, p) sets its bit.
struct PreJob {
    int64_t delta_off;   // the instance's [k][n] entries; its table starts at delta_off * W
    int32_t n, k;
};

template <int W>
__global__ void k_pre_clear(const PreJob *__restrict__ jobs, uint64_t *__restrict__ pre) {
    const PreJob J = jobs[blockIdx.y];
    const int64_t len = (int64_t)J.k * J.n * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        pre[J.delta_off * W + i] = 0;
}

template <int W>
__global__ void k_pre_fill(const PreJob *__restrict__ jobs, const uint16_t *__restrict__ delta16,
                           uint64_t *__restrict__ pre) {
    const PreJob J = jobs[blockIdx.y];
    const int64_t len = (int64_t)J.k * J.n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = i / J.n, p = i - a * J.n;
        const int t = delta16[J.delta_off + i];
        atomicOr((unsigned long long *)(pre + (J.delta_off + a * J.n + t) * W + (p >> 6)),
                 1ull << (p & 63));
    }
}

// int32 [k][n] tables -> uint16 (device-resident input path); one CTA row
// (blockIdx.y) per instance.
struct ConvJob {
    int64_t src_off, dst_off, count;
    int32_t n, pad;
};

__global__ void k_delta_to_u16(const ConvJob *__restrict__ jobs, const int32_t *__restrict__ src,
                               uint16_t *__restrict__ dst, uint32_t *bad) {
    const ConvJob J = jobs[blockIdx.y];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < J.count;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = src[J.src_off + i];
        if (v < 0 || v >= J.n) atomicOr(bad, 1u);
        dst[J.dst_off + i] = (uint16_t)(v < 0 || v >= J.n ? 0 : v);
    }
}

}  // namespace sw
