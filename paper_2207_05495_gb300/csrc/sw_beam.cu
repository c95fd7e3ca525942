// The heuristic upper bound R of Section 2.1.3 on the GPU: an inverse BFS
// from the singletons that keeps, at every depth, only the `beam` largest
// distinct preimages (the cut-off inverse BFS the paper cites; it runs it
// with beam size n log n up to n = 5000 in Section 3).  The first depth at
// which Q itself is kept gives a reset word y (delta^{-1}({q}, y) = Q, so
// delta(Q, y) = {q}) and R = |y| >= r.
//
// Sets have nw = ceil(n / 64) 64-bit words, nw chosen at run time (up to
// SW_BEAM_MAX_STATES states), so this path serves automata far larger than
// the exact search.  One level is made by:
//   k_beam_expand  one warp per candidate (parent p, letter a), c = p*k + a:
//                  lanes take 32 states q at a time and a ballot of
//                  "delta(q, a) is in S" gives 32 bits of the preimage; the
//                  candidate then enters this level's hash table (among
//                  equal sets the smallest c keeps the slot);
//   k_beam_flag    winners and the histogram of their cardinalities;
//   k_beam_cut     the cardinality c* at which the beam fills up, and how
//                  many sets of exactly c* states still fit (quota);
//   k_beam_rank    keeps every winner above c* and the first `quota`
//                  winners of exactly c* states in candidate order (two
//                  block-count scans give the ranks), and compacts the kept
//                  sets in candidate order with their candidate ids, noting
//                  the first position of Q.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "sw.h"
#include "sw_internal.h"

namespace {

constexpr uint64_t kBEmpty = ~0ull;
constexpr int kBBlock = 512;    // candidates per block of the flag/rank scans
constexpr int kBThreads = 256;  // threads of those blocks (two candidates each)
constexpr int kBMaxProbe = 1 << 14;

__device__ __forceinline__ uint64_t bmix(uint64_t x) {
    // MurmurHash3 finalizer (Appleby), a published 64-bit mixer
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Level 0: the n singletons, in state order.
__global__ void k_beam_roots(int n, int nw, uint64_t *__restrict__ sets) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * nw;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / nw), w = (int)(e % nw);
        sets[e] = (w == q / 64) ? (1ull << (q % 64)) : 0ull;
    }
}

// Preimages delta^{-1}(S, a) of the level's sets, entered into the table.
// slot[c] = the table slot, or -1 for an empty preimage (dropped) or a
// table overflow (status bit 1).
__global__ void __launch_bounds__(256) k_beam_expand(int n, int k, int nw, const uint16_t *__restrict__ d16,
                                                     const uint64_t *__restrict__ cur, int64_t ncand,
                                                     uint64_t *cand, int32_t *__restrict__ card,
                                                     int64_t *__restrict__ slot, uint64_t *table, int64_t tab_cap,
                                                     uint32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t c = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); c < ncand; c += warps) {
        const int64_t p = c / k;
        const int a = (int)(c - p * k);
        const uint64_t *S = cur + p * nw;
        const uint16_t *da = d16 + (int64_t)a * n;
        uint32_t *T32 = reinterpret_cast<uint32_t *>(cand + c * nw);
        int cnt = 0;
        uint64_t hpart = 0;
        for (int half = 0; half < 2 * nw; ++half) {
            const int q = 32 * half + lane;
            uint32_t bit = 0;
            if (q < n) {
                const int t = da[q];
                bit = (uint32_t)(__ldg(S + (t >> 6)) >> (t & 63)) & 1u;
            }
            const uint32_t ball = __ballot_sync(0xffffffffu, bit);
            cnt += __popc(ball);
            if (lane == (half & 31)) {
                T32[half] = ball;
                hpart ^= bmix((uint64_t)ball + 0x9E3779B97F4A7C15ull * (uint64_t)(half + 1));
            }
        }
        for (int o = 16; o; o >>= 1) hpart ^= __shfl_xor_sync(0xffffffffu, hpart, o);
        if (lane == 0) card[c] = cnt;
        if (cnt == 0) {  // an empty preimage contains no nonempty set
            if (lane == 0) slot[c] = -1;
            continue;
        }
        __threadfence();  // publish the set before its id can be seen in the table
        __syncwarp();
        uint64_t pos = __umul64hi(bmix(hpart), (uint64_t)tab_cap);
        int64_t result = -1;
        int probe = 0;
        for (; probe < kBMaxProbe; ++probe) {
            uint64_t v = 0;
            int won = 0;
            if (lane == 0) {
                v = *(volatile uint64_t *)(table + pos);
                if (v == kBEmpty) {
                    unsigned long long old =
                        atomicCAS((unsigned long long *)(table + pos), kBEmpty, (unsigned long long)c);
                    won = old == kBEmpty;
                    v = old;
                }
            }
            won = __shfl_sync(0xffffffffu, won, 0);
            if (won) {
                result = (int64_t)pos;
                break;
            }
            v = __shfl_sync(0xffffffffu, v, 0);
            __threadfence();  // read the other set after observing its id
            const uint64_t *O = cand + (int64_t)v * nw;
            const uint64_t *Tm = cand + c * nw;
            bool eq = true;
            for (int w = lane; w < nw; w += 32) eq &= (__ldcg(O + w) == __ldcg(Tm + w));
            if (__all_sync(0xffffffffu, eq)) {
                if (lane == 0) atomicMin((unsigned long long *)(table + pos), (unsigned long long)c);
                result = (int64_t)pos;
                break;
            }
            pos = (pos + 1 == (uint64_t)tab_cap) ? 0 : pos + 1;
        }
        if (lane == 0) {
            if (probe == kBMaxProbe) atomicOr(status, 1u);
            slot[c] = result;
        }
    }
}

// flag[c] = 1 for a winner (it owns its slot); hist[card] counts them.
__global__ void __launch_bounds__(kBThreads) k_beam_flag(int64_t ncand, const int64_t *__restrict__ slot,
                                                         const uint64_t *__restrict__ table,
                                                         const int32_t *__restrict__ card,
                                                         uint8_t *__restrict__ flag, uint32_t *__restrict__ hist) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncand; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = slot[c];
        const uint8_t f = (s >= 0 && table[s] == (uint64_t)c) ? 1 : 0;
        flag[c] = f;
        if (f) atomicAdd(&hist[card[c]], 1u);
    }
}

// cut[0] = c*, cut[1] = quota: all winners of more than c* states are kept,
// and the first quota of exactly c*; c* = -1 keeps every winner.
__global__ void k_beam_cut(int n, int64_t beam, const uint32_t *__restrict__ hist, int64_t *__restrict__ cut) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t above = 0;
    for (int c = n; c >= 1; --c) {
        if (above + (int64_t)hist[c] >= beam) {
            cut[0] = c;
            cut[1] = beam - above;
            return;
        }
        above += hist[c];
    }
    cut[0] = -1;
    cut[1] = 0;
}

// The rank of every flagged candidate inside its block (candidate order),
// for 512 candidates per block and 256 threads; returns the block total.
__device__ __forceinline__ uint32_t block_rank2(uint32_t f0, uint32_t f1, uint32_t *r0, uint32_t *r1,
                                                uint32_t *ws) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t mine = f0 + f1;
    uint32_t x = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int i = 0; i < kBThreads / 32; ++i) {
        if (i < warp) before += ws[i];
        total += ws[i];
    }
    __syncthreads();
    const uint32_t first = before + x - mine;
    *r0 = first;
    *r1 = first + f0;
    return total;
}

// Pass 1 (mode 0): per block, the winners of exactly c* states.
// Pass 2 (mode 1): which winners are kept (flag stays 1 or becomes 0), and
// per block how many.
__global__ void __launch_bounds__(kBThreads) k_beam_rank(int64_t ncand, int mode, const int32_t *__restrict__ card,
                                                         uint8_t *__restrict__ flag, const int64_t *__restrict__ cut,
                                                         const uint64_t *__restrict__ eq_off,
                                                         uint32_t *__restrict__ block_cnt) {
    __shared__ uint32_t ws[kBThreads / 32];
    const int64_t c0 = (int64_t)blockIdx.x * kBBlock + 2 * threadIdx.x;
    const int64_t cstar = cut[0], quota = cut[1];
    uint32_t f[2], e[2];
    for (int i = 0; i < 2; ++i) {
        const int64_t c = c0 + i;
        f[i] = (c < ncand) ? flag[c] : 0;
        e[i] = (f[i] && card[c] == cstar) ? 1 : 0;
    }
    uint32_t r[2];
    const uint32_t eq_total = block_rank2(e[0], e[1], &r[0], &r[1], ws);
    if (mode == 0) {
        if (threadIdx.x == 0) block_cnt[blockIdx.x] = eq_total;
        return;
    }
    uint32_t keep[2];
    for (int i = 0; i < 2; ++i) {
        keep[i] = 0;
        if (!f[i]) continue;
        const int64_t c = c0 + i;
        if (cstar < 0 || card[c] > cstar) keep[i] = 1;
        else if (e[i] && (int64_t)(eq_off[blockIdx.x] + r[i]) < quota) keep[i] = 1;
        flag[c] = (uint8_t)keep[i];
    }
    uint32_t k0, k1;
    const uint32_t kept = block_rank2(keep[0], keep[1], &k0, &k1, ws);
    if (threadIdx.x == 0) block_cnt[blockIdx.x] = kept;
}

// Exclusive scan of per-block counts in one CTA; off[nb] = total.
__global__ void __launch_bounds__(1024) k_beam_scan(int64_t nb, const uint32_t *__restrict__ cnt,
                                                    uint64_t *__restrict__ off) {
    __shared__ uint64_t wsum[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const uint64_t v = i < nb ? cnt[i] : 0;
        uint64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint64_t s = wsum[threadIdx.x];
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (threadIdx.x >= o) s += y;
            }
            wsum[threadIdx.x] = s;
        }
        __syncthreads();
        const uint64_t before = carry + (threadIdx.x >= 32 ? wsum[(threadIdx.x >> 5) - 1] : 0) + x - v;
        if (i < nb) off[i] = before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[nb] = carry;
}

// The kept sets, in candidate order, to the next level, with their
// candidate ids; hit = the smallest position of a set of n states (Q).
__global__ void __launch_bounds__(kBThreads) k_beam_compact(int64_t ncand, int n, int nw,
                                                            const uint8_t *__restrict__ flag,
                                                            const uint64_t *__restrict__ keep_off,
                                                            const uint64_t *__restrict__ cand,
                                                            const int32_t *__restrict__ card,
                                                            uint64_t *__restrict__ next, int64_t *__restrict__ link,
                                                            int64_t cap, unsigned long long *hit) {
    __shared__ uint32_t ws[kBThreads / 32];
    const int64_t c0 = (int64_t)blockIdx.x * kBBlock + 2 * threadIdx.x;
    uint32_t f[2];
    for (int i = 0; i < 2; ++i) f[i] = (c0 + i < ncand) ? flag[c0 + i] : 0;
    uint32_t r[2];
    block_rank2(f[0], f[1], &r[0], &r[1], ws);
    for (int i = 0; i < 2; ++i) {
        if (!f[i]) continue;
        const int64_t c = c0 + i;
        const int64_t pos = (int64_t)keep_off[blockIdx.x] + r[i];
        if (pos >= cap) continue;  // more kept sets than the level buffers hold: the host fails the call
        for (int w = 0; w < nw; ++w) next[pos * nw + w] = cand[c * nw + w];
        link[pos] = c;
        if (card[c] == n) atomicMin(hit, (unsigned long long)pos);
    }
}

// The word: from the first Q of level R back along the candidate ids; the
// letter of the level-d set is letter R - d of the word.  Then every state
// is mapped through it: out[0] = 1 when they all end in one state.
__global__ void k_beam_word(int R, int k, int64_t hit, const int64_t *__restrict__ level_link,
                            const int64_t *__restrict__ links, uint8_t *__restrict__ word) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t pos = hit;
    for (int d = R; d > 0; --d) {
        const int64_t c = links[level_link[d] + pos];
        word[R - d] = (uint8_t)(c % k);
        pos = c / k;
    }
}

__global__ void k_beam_verify(int n, int R, const uint16_t *__restrict__ d16, const uint8_t *__restrict__ word,
                              int32_t *__restrict__ ends) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        int s = q;
        for (int t = 0; t < R; ++t) s = d16[(int64_t)word[t] * n + s];
        atomicMin(ends, s);
        atomicMax(ends + 1, s);
    }
}

int64_t up256(int64_t b) { return (b + 255) & ~(int64_t)255; }

struct BeamLayout {
    uint16_t *d16;
    uint64_t *lev[2];
    uint64_t *cand;
    int32_t *card;
    int64_t *slot;
    uint8_t *flag;
    uint64_t *table;
    int64_t tab_cap;
    uint32_t *hist;
    uint32_t *bcnt;
    uint64_t *boff;
    int64_t *cut;
    unsigned long long *hit;
    uint32_t *status;
    int32_t *ends;
    uint8_t *word;
    int64_t *level_link;
    int64_t *links;
    int64_t links_cap;
};

}  // namespace

extern "C" int32_t sw_beam(int32_t n, int32_t k, const int32_t *delta, void *stream, void *workspace,
                           size_t ws_bytes, int64_t beam, int32_t max_depth, int32_t *R_out, uint8_t *word,
                           int32_t word_cap) {
    if (n < 1 || n > SW_BEAM_MAX_STATES || k < 1 || k > SW_MAX_LETTERS || !delta || !workspace || !R_out ||
        beam < 1 || max_depth < 0 || word_cap < 0 || ((uintptr_t)workspace & 255) != 0)
        return sw_internal_fail(SW_EINVAL);
    for (int64_t i = 0; i < (int64_t)n * k; ++i)
        if (delta[i] < 0 || delta[i] >= n) return sw_internal_fail(SW_EINVAL);
    if (n == 1) {
        *R_out = 0;
        return sw_internal_ok();
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nw = (n + 63) / 64;
    // the level buffers hold min(beam, what about 60% of the workspace
    // allows) sets; a level that keeps more fails the call with SW_ENOMEM
    const double per_set = 16.0 * nw + k * (8.0 * nw + 13.0 + 16.0);
    const int64_t fit = (int64_t)(0.6 * (double)ws_bytes / per_set);
    const int64_t lev_cap = std::max<int64_t>(n, std::min<int64_t>(beam, fit));
    const int64_t ncap = lev_cap * k;
    const int64_t nblk = (ncap + kBBlock - 1) / kBBlock;
    int64_t tab_cap = 2 * ncap + 64;
    // carve the workspace; what is left holds the candidate ids of every
    // level (the word is read back through them)
    char *base = (char *)workspace;
    size_t used = 0;
    bool ok = true;
    auto take = [&](int64_t bytes) -> char * {
        const int64_t b = up256(bytes);
        if (used + (size_t)b > ws_bytes) {
            ok = false;
            return base;
        }
        char *p = base + used;
        used += (size_t)b;
        return p;
    };
    BeamLayout L;
    L.d16 = (uint16_t *)take((int64_t)n * k * 2);
    L.lev[0] = (uint64_t *)take(lev_cap * nw * 8);
    L.lev[1] = (uint64_t *)take(lev_cap * nw * 8);
    L.cand = (uint64_t *)take(ncap * nw * 8);
    L.card = (int32_t *)take(ncap * 4);
    L.slot = (int64_t *)take(ncap * 8);
    L.flag = (uint8_t *)take(ncap);
    L.table = (uint64_t *)take(tab_cap * 8);
    L.tab_cap = tab_cap;
    L.hist = (uint32_t *)take((int64_t)(n + 1) * 4);
    L.bcnt = (uint32_t *)take(nblk * 4);
    L.boff = (uint64_t *)take((nblk + 1) * 8 * 2);  // equal-cardinality offsets, then kept offsets
    L.cut = (int64_t *)take(16);
    L.hit = (unsigned long long *)take(8);
    L.status = (uint32_t *)take(4);
    L.ends = (int32_t *)take(8);
    L.word = (uint8_t *)take(std::max<int64_t>(max_depth, 1));
    L.level_link = (int64_t *)take((int64_t)(max_depth + 1) * 8);
    if (!ok) return sw_internal_fail(SW_ENOMEM);
    L.links_cap = (int64_t)((ws_bytes - used) / 8);
    L.links = (int64_t *)(base + used);
    if (L.links_cap < n) return sw_internal_fail(SW_ENOMEM);
    uint64_t *eq_off = L.boff, *keep_off = L.boff + (nblk + 1);

#define BCK(x)                                                  \
    do {                                                        \
        if ((x) != cudaSuccess) return sw_internal_fail(SW_ECUDA); \
    } while (0)
    std::vector<uint16_t> d16((size_t)n * k);
    for (size_t i = 0; i < d16.size(); ++i) d16[i] = (uint16_t)delta[i];
    BCK(cudaMemcpyAsync(L.d16, d16.data(), d16.size() * 2, cudaMemcpyHostToDevice, st));
    BCK(cudaMemsetAsync(L.status, 0, 4, st));
    k_beam_roots<<<(unsigned)std::min<int64_t>(((int64_t)n * nw + 255) / 256, 4096), 256, 0, st>>>(n, nw, L.lev[0]);
    BCK(cudaGetLastError());
    std::vector<int64_t> level_link((size_t)max_depth + 1, 0);
    int64_t m = n, links_used = 0;
    int cur = 0, R = -1;
    int64_t hit = -1;
    struct Down {
        uint64_t kept;
        unsigned long long hit;
        uint32_t status;
    } down{};
    for (int d = 1; d <= max_depth; ++d) {
        const int64_t nc = m * k;
        const int64_t nb = (nc + kBBlock - 1) / kBBlock;
        if (links_used + std::min(nc, lev_cap) > L.links_cap) return sw_internal_fail(SW_ENOMEM);
        level_link[d] = links_used;
        BCK(cudaMemsetAsync(L.table, 0xFF, (size_t)tab_cap * 8, st));
        BCK(cudaMemsetAsync(L.hist, 0, (size_t)(n + 1) * 4, st));
        BCK(cudaMemsetAsync(L.hit, 0xFF, 8, st));
        const unsigned wblocks = (unsigned)std::min<int64_t>((nc + 7) / 8, 152 * 64);
        k_beam_expand<<<wblocks, 256, 0, st>>>(n, k, nw, L.d16, L.lev[cur], nc, L.cand, L.card, L.slot, L.table,
                                               tab_cap, L.status);
        k_beam_flag<<<(unsigned)std::min<int64_t>((nc + 255) / 256, 152 * 32), 256, 0, st>>>(
            nc, L.slot, L.table, L.card, L.flag, L.hist);
        k_beam_cut<<<1, 32, 0, st>>>(n, beam, L.hist, L.cut);
        k_beam_rank<<<(unsigned)nb, kBThreads, 0, st>>>(nc, 0, L.card, L.flag, L.cut, eq_off, L.bcnt);
        k_beam_scan<<<1, 1024, 0, st>>>(nb, L.bcnt, eq_off);
        k_beam_rank<<<(unsigned)nb, kBThreads, 0, st>>>(nc, 1, L.card, L.flag, L.cut, eq_off, L.bcnt);
        k_beam_scan<<<1, 1024, 0, st>>>(nb, L.bcnt, keep_off);
        k_beam_compact<<<(unsigned)nb, kBThreads, 0, st>>>(nc, n, nw, L.flag, keep_off, L.cand, L.card, L.lev[1 - cur],
                                                           L.links + links_used, lev_cap, L.hit);
        BCK(cudaGetLastError());
        BCK(cudaMemcpyAsync(&down.kept, keep_off + nb, 8, cudaMemcpyDeviceToHost, st));
        BCK(cudaMemcpyAsync(&down.hit, L.hit, 8, cudaMemcpyDeviceToHost, st));
        BCK(cudaMemcpyAsync(&down.status, L.status, 4, cudaMemcpyDeviceToHost, st));
        BCK(cudaStreamSynchronize(st));
        if (down.status) return sw_internal_fail(SW_EINTERNAL);  // a level's table overflowed
        if ((int64_t)down.kept > lev_cap) return sw_internal_fail(SW_ENOMEM);
        m = (int64_t)down.kept;
        links_used += m;
        cur = 1 - cur;
        if (m == 0) return sw_internal_fail(SW_ENOTSYNC);
        if (down.hit != ~0ull) {
            R = d;
            hit = (int64_t)down.hit;
            break;
        }
    }
    if (R < 0) return sw_internal_fail(SW_ENOTFOUND);
    *R_out = R;
    if (R > word_cap) return sw_internal_fail(SW_EWORDCAP);
    BCK(cudaMemcpyAsync(L.level_link, level_link.data(), (size_t)(R + 1) * 8, cudaMemcpyHostToDevice, st));
    k_beam_word<<<1, 32, 0, st>>>(R, k, hit, L.level_link, L.links, L.word);
    const int32_t init[2] = {INT32_MAX, -1};
    BCK(cudaMemcpyAsync(L.ends, init, 8, cudaMemcpyHostToDevice, st));
    k_beam_verify<<<(unsigned)std::min(((int64_t)n + 255) / 256, (int64_t)1024), 256, 0, st>>>(n, R, L.d16, L.word,
                                                                                               L.ends);
    BCK(cudaGetLastError());
    int32_t ends[2];
    BCK(cudaMemcpyAsync(ends, L.ends, 8, cudaMemcpyDeviceToHost, st));
    if (word) BCK(cudaMemcpyAsync(word, L.word, (size_t)R, cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    if (ends[0] != ends[1]) return sw_internal_fail(SW_EINTERNAL);
#undef BCK
    return sw_internal_ok();
}
