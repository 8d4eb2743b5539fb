// IC large path, grouped: the large RRR sets of a batch are sampled 64 at a
// time by the whole GPU as one multi-source reverse BFS (Generate_RRRsets,
// EfficientIMM Alg. 3, for many roots at once).
//
// Each vertex carries three 64-bit masks over the sets of the group: vis (the
// sets whose BFS has expanded it) and the frontier masks of the current and
// the next level.  Level by level, a frontier vertex v with mask F adds F to
// vis[v], reads its in-edge thresholds and sources once and flips the coins
// of every set in F: in-edge e = (u -> v) of set s is live iff word e&3 of
// Philox(s, e>>2) passes e's threshold (the same draw as the one-set-per-CTA
// path, so every set equals the reverse-reachable closure of its root under
// its own coins, whatever the traversal order).  Live bits that u holds
// neither in vis[u] nor in its current-frontier mask are ored into u's
// next-frontier mask, and u is queued for the next level when that mask
// leaves zero.  A visit that races with u's own expansion may see neither
// mask updated and queue bits u already expands; u then sweeps them once more
// with no effect on any set (the sets are read from vis), so the race costs
// work, never correctness.  The giant sets of a power-law graph walk the same
// high-degree core within a level or two of each other, so the per-vertex
// work (edge range, threshold and source loads, quad bookkeeping) is shared
// by the sets that reach v at the same level.
//
// A vertex is sorted when it is queued: vertices with >= 32 in-edge quads go
// to a large list with a running chunk count, the others to a small list.
// The kernel is persistent (cooperative launch, one 1024-thread CTA per SM)
// and advances in steps separated by grid barriers.  In a BFS step warps
// claim work items from one counter: first 32-vertex chunks of the small
// list, whose quads are flattened across lanes (one quad per lane, its owner
// found from per-warp run records in shared memory; up to 31 windows of 32
// quads per item), then the one-window 32-quad chunks of the large vertices
// (owner found by a 32-way search over the chunk prefix), which even out the
// end of the step.  A large vertex's mask is merged into vis by the warp that
// sweeps its last chunk.
//
// When no frontier is left, two dense passes over vis give every set its
// size and in-edge sum, reserve its output (member list, or an n-bit bitmap
// when the list would be larger; Sec. IV-C), write it, and clear vis.
//
// Two groups are in flight, in two slots of the arrays: every step serves
// both (their items share the counter), so one group's small levels, level
// ends and extraction passes overlap the other group's big levels.
#include "imm_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace imm {

namespace cg = cooperative_groups;

constexpr int kGroupThreads = 1024;  // threads per CTA
constexpr int kGroupBlocks = 1;      // CTAs per SM (the cooperative grid is SMs x this)
constexpr int kGroupChains = 2;      // independent Philox chains per lane in a sweep
constexpr int kGroupWarps = kGroupThreads / 32;
constexpr uint32_t kGroupHeavyQ = 32;  // in-edge quads from which a vertex is swept in 32-quad chunks
constexpr unsigned long long kLow40 = (1ull << 40) - 1;
constexpr uint32_t kHeavySmem = 6144;  // chunk prefix entries per slot searched in shared memory

__device__ __forceinline__ uint32_t lanemask_le_g()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t lanemask_lt_g()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void range_of(const DevGraph& g, uint32_t v, uint32_t& rs, uint32_t& re)
{
    rs = (uint32_t)__ldg(g.row + v);
    re = (uint32_t)__ldg(g.row + v + 1);
}

__device__ __forceinline__ uint32_t nquads(uint32_t rs, uint32_t re)
{
    return re > rs ? ((re - 1) >> 2) - (rs >> 2) + 1 : 0u;
}

// Live sets of the four in-edges of one quad: lo[t] / hi[t] hold the sets
// 0..31 / 32..63 of the group for which edge 4*quad + t is live.
struct QuadLive {
    uint32_t lo[4], hi[4];
    uint4 src;  // tails of the four in-edges
};

// One half (32 sets) of the mask: coins of every set in `mask` for the quad
// whose round-0 product is `a`; with two chains, two sets per step so that
// two independent Philox evaluations are in flight.
__device__ __forceinline__ void sweep_half(uint32_t mask, uint64_t a, uint4 tm, const PhiloxSet* ps,
                                           const PhiloxKeys& rk, uint32_t* acc)
{
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    while (mask) {
        const int s1 = 31 - __clz(mask);
        mask ^= 1u << s1;
        const uint32_t b1 = 1u << s1;
        const uint4 w1 = philox_xa(a, ps[s1], rk);
        if (kGroupChains == 2) {
            const bool two = mask != 0;
            const int s2 = two ? 31 - __clz(mask) : s1;
            const uint32_t b2 = two ? 1u << s2 : 0u;
            mask ^= b2;
            const uint4 w2 = philox_xa(a, ps[s2], rk);
            if (w2.x <= tm.x) a0 |= b2;
            if (w2.y <= tm.y) a1 |= b2;
            if (w2.z <= tm.z) a2 |= b2;
            if (w2.w <= tm.w) a3 |= b2;
        }
        if (w1.x <= tm.x) a0 |= b1;
        if (w1.y <= tm.y) a1 |= b1;
        if (w1.z <= tm.z) a2 |= b1;
        if (w1.w <= tm.w) a3 |= b1;
    }
    acc[0] = a0;
    acc[1] = a1;
    acc[2] = a2;
    acc[3] = a3;
}

// Coins of all sets in F for the in-edges of `quad` that lie in [rs, re).
// The coin is live iff the 24-bit draw w >> 8 is below the threshold th,
// i.e. iff w <= 256 th - 1; th = 0 (never live) wraps to 2^32 - 1 there and
// is cleared through `valid` instead.
__device__ __forceinline__ void sweep_quad(const DevGraph& g, const PhiloxKeys& rk, const PhiloxSet* ps,
                                           uint32_t quad, uint32_t rs, uint32_t re, unsigned long long F,
                                           QuadLive& ql)
{
    // the sources are loaded here so that their latency hides under the sweep
    ql.src = __ldg(reinterpret_cast<const uint4*>(g.src) + quad);
    const uint4 th = __ldg(reinterpret_cast<const uint4*>(g.thr) + quad);
    const uint4 tm = make_uint4((th.x << 8) - 1u, (th.y << 8) - 1u, (th.z << 8) - 1u, (th.w << 8) - 1u);
    uint32_t valid = (th.x ? 1u : 0u) | (th.y ? 2u : 0u) | (th.z ? 4u : 0u) | (th.w ? 8u : 0u);
    const uint32_t e0 = quad << 2;
    if (e0 < rs) valid &= 0xFu << (rs - e0);
    if (e0 + 4 > re) valid &= 0xFu >> (e0 + 4 - re);
    const uint64_t a = (uint64_t)kPhiloxM1 * (uint64_t)quad;
    sweep_half((uint32_t)F, a, tm, ps, rk, ql.lo);
    sweep_half((uint32_t)(F >> 32), a, tm, ps + 32, rk, ql.hi);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (!((valid >> t) & 1u)) {
            ql.lo[t] = 0;
            ql.hi[t] = 0;
        }
    }
}

// Where a level's visits queue the next frontier.
struct LevelOut {
    unsigned long long* hpack;  // large vertices << 40 | their chunks
    uint32_t* lcount;           // small vertices
    uint32_t* lq;               // small vertex ids
    uint32_t* hb;               // first chunk of each large vertex
    uint4* he;                  // large vertices: (v, rs, re, chunks not yet swept)
};

// Sort a vertex that just entered the next frontier into the large or small
// list; returns true when it went to the small list (queued by the caller).
__device__ __forceinline__ bool queue_large(const LevelOut& o, uint32_t u, uint32_t rs, uint32_t re)
{
    const uint32_t nq = nquads(rs, re);
    if (nq < kGroupHeavyQ) return true;
    const uint32_t nch = (nq + 31) >> 5;
    const unsigned long long old = atomicAdd(o.hpack, (1ull << 40) | (unsigned long long)nch);
    const uint32_t i = (uint32_t)(old >> 40);
    o.hb[i] = (uint32_t)(old & kLow40);
    o.he[i] = make_uint4(u, rs, re, nch);
    return false;
}

// Apply the live bits of one quad per lane: bits u neither expanded nor has
// in the current frontier go to u's next-frontier mask; u is queued when that
// mask leaves zero.  Every lane's four lookups, then its four atomics, are
// independent, so each step costs one memory round trip.  Called by the
// whole warp.
__device__ __forceinline__ void visit_quad(const DevGraph& g, const unsigned long long* vis,
                                           const unsigned long long* fcur, unsigned long long* fnext,
                                           const LevelOut& o, const QuadLive& ql, uint32_t lane)
{
    const uint32_t u[4] = {ql.src.x, ql.src.y, ql.src.z, ql.src.w};
    unsigned long long m[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) m[t] = ((unsigned long long)ql.hi[t] << 32) | ql.lo[t];
    unsigned long long known[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) known[t] = m[t] ? __ldcg(vis + u[t]) | __ldcg(fcur + u[t]) : ~0ull;
    bool push[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        m[t] &= ~known[t];
        push[t] = m[t] ? atomicOr(fnext + u[t], m[t]) == 0ull : false;
    }
    uint32_t np = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (push[t]) {
            uint32_t rs, re;
            range_of(g, u[t], rs, re);
            push[t] = queue_large(o, u[t], rs, re);
            np += push[t] ? 1u : 0u;
        }
    }
    uint32_t incl = np;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t x = __shfl_up_sync(kFull, incl, d);
        if ((int)lane >= d) incl += x;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(o.lcount, total);
    base = __shfl_sync(kFull, base, 31) + incl - np;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (push[t]) o.lq[base++] = u[t];
}

// Arrays of one group slot (slot 1's lie `stride` bytes after slot 0's).
struct SlotArrays {
    unsigned long long *vis, *fr0, *fr1;
    uint32_t *lq0, *lq1, *hb0, *hb1;
    uint4 *he0, *he1;
    GroupCounters* ct;
};

__device__ __forceinline__ SlotArrays slot_arrays(const GroupScratch& gs, uint32_t k)
{
    const uint64_t d = k ? gs.stride : 0;
    auto at = [d](auto* p) { return reinterpret_cast<decltype(p)>(reinterpret_cast<char*>(p) + d); };
    SlotArrays a;
    a.vis = at(gs.vis);
    a.fr0 = at(gs.fr0);
    a.fr1 = at(gs.fr1);
    a.lq0 = at(gs.lq0);
    a.lq1 = at(gs.lq1);
    a.hb0 = at(gs.hb0);
    a.hb1 = at(gs.hb1);
    a.he0 = at(gs.he0);
    a.he1 = at(gs.he1);
    a.ct = gs.ctr + k;
    return a;
}

// What a slot does in the current step (the same in every CTA: each CTA's
// thread 0 advances its copy from the same global counters).
constexpr uint32_t kIdle = 0, kInit = 1, kBfs = 2, kCount = 3, kReserve = 4, kWrite = 5;
struct SlotStep {
    uint32_t phase;
    uint32_t level;  // BFS level being expanded (kBfs)
    uint32_t g0, G;  // the group: large-queue entries g0 .. g0 + G - 1
    uint32_t nl, nch, nh;  // small vertices, large-vertex chunks, large vertices of the level
    uint32_t items;
};
constexpr uint32_t kWordsPerItem = 8;  // bitmap words per extraction item

// One BFS level's view of a slot.
struct LevelView {
    const unsigned long long* fcur;
    unsigned long long* fnext;
    const uint32_t* lq;
    const uint32_t* hb;
    uint4* he;
    LevelOut o;
};

__device__ __forceinline__ LevelView level_view(const SlotArrays& a, uint32_t level)
{
    const bool odd = level & 1u;
    const uint32_t nxt = (level + 1) % 3;
    LevelView v;
    v.fcur = odd ? a.fr1 : a.fr0;
    v.fnext = odd ? a.fr0 : a.fr1;
    v.lq = odd ? a.lq1 : a.lq0;
    v.hb = odd ? a.hb1 : a.hb0;
    v.he = odd ? a.he1 : a.he0;
    v.o = {&a.ct->hpack[nxt], &a.ct->lcount[nxt], odd ? a.lq0 : a.lq1, odd ? a.hb0 : a.hb1, odd ? a.he0 : a.he1};
    return v;
}

// 32-quad chunk hc of the level's large vertices.  Owner: the last lo with
// hb[lo] <= hc (invariant hb[lo] <= hc < hb[lo + span]; lane 0 probes lo
// itself, so the ballot is never empty).
__device__ __forceinline__ void large_item(const DevGraph& g, const PhiloxKeys& rk, const PhiloxSet* ps,
                                           const SlotArrays& a, const LevelView& lv, const uint32_t* s_hb,
                                           bool hsm, uint32_t nh, uint32_t hc, uint32_t lane)
{
    uint32_t lo = 0, span = nh;
    while (span > 1) {
        const uint32_t step = (span + 31) >> 5;
        const uint32_t off = lane * step;
        const bool le = off < span && (hsm ? s_hb[lo + off] : __ldcg(lv.hb + lo + off)) <= hc;
        const uint32_t t = 31 - __clz(__ballot_sync(kFull, le));
        lo += t * step;
        span = min(step, span - t * step);
    }
    const uint4 e = __ldcg(lv.he + lo);
    const uint32_t first = hsm ? s_hb[lo] : __ldcg(lv.hb + lo);
    const unsigned long long F = __ldcg(lv.fcur + e.x);
    const uint32_t quad = (e.y >> 2) + (hc - first) * 32 + lane;
    QuadLive ql = {};
    if (quad <= ((e.z - 1) >> 2)) sweep_quad(g, rk, ps, quad, e.y, e.z, F, ql);
    visit_quad(g, a.vis, lv.fcur, lv.fnext, lv.o, ql, lane);
    // the warp that sweeps the vertex's last chunk merges its mask
    if (lane == 0 && atomicSub(&lv.he[lo].w, 1u) == 1u) {
        __stcg(a.vis + e.x, __ldcg(a.vis + e.x) | F);
        __stcg(const_cast<unsigned long long*>(lv.fcur) + e.x, 0ull);
    }
}

// 32 small vertices from lq[v0 ..): their quads flattened across lanes, in
// windows of 32.  In a window, the run of each lane that meets it is
// recorded at its first slot there; a slot's owner is the last recorded
// start at or before it.
__device__ __forceinline__ void small_item(const DevGraph& g, const PhiloxKeys& rk, const PhiloxSet* ps,
                                           const SlotArrays& a, const LevelView& lv, uint32_t nl, uint32_t v0,
                                           uint4* rec, unsigned long long* recF, uint32_t lane)
{
    const uint32_t nf = min(nl - v0, 32u);
    uint32_t rs = 0, re = 0, nq = 0;
    unsigned long long F = 0;
    if (lane < nf) {
        const uint32_t v = __ldcg(lv.lq + v0 + lane);
        F = __ldcg(lv.fcur + v);
        __stcg(a.vis + v, __ldcg(a.vis + v) | F);
        __stcg(const_cast<unsigned long long*>(lv.fcur) + v, 0ull);
        range_of(g, v, rs, re);
        nq = nquads(rs, re);
    }
    uint32_t incl = nq;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, d);
        if ((int)lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - nq;
    for (uint32_t j0 = 0; j0 < total; j0 += 32) {
        const bool meets = nq != 0 && excl < j0 + 32 && incl > j0;
        const uint32_t st = excl > j0 ? excl - j0 : 0u;
        if (meets) {
            rec[st] = make_uint4(rs, re, excl, 0u);
            recF[st] = F;
        }
        const uint32_t starts = __reduce_or_sync(kFull, meets ? 1u << st : 0u);
        __syncwarp();
        const uint32_t j = j0 + lane;
        QuadLive ql = {};
        if (j < total) {
            const uint32_t pos = 31 - __clz(starts & lanemask_le_g());
            const uint4 r = rec[pos];
            const uint32_t quad = (r.x >> 2) + (j - r.z);
            sweep_quad(g, rk, ps, quad, r.x, r.y, recF[pos], ql);
        }
        visit_quad(g, a.vis, lv.fcur, lv.fnext, lv.o, ql, lane);
        __syncwarp();
    }
}

// Count pass over words [w0, w0 + kWordsPerItem): members and in-edge sums
// of the group's sets, into the CTA's shared accumulators.
__device__ __forceinline__ void count_item(const DevGraph& g, const SlotArrays& a, uint32_t G, uint32_t words,
                                           uint32_t w0, uint32_t* s_cnt, uint32_t* s_edg, uint32_t lane)
{
    const uint32_t w1 = min(w0 + kWordsPerItem, words);
    for (uint32_t w = w0; w < w1; ++w) {
        const uint32_t u = (w << 5) + lane;
        const unsigned long long m = u < g.n ? __ldcg(a.vis + u) : 0ull;
        if (!__any_sync(kFull, m != 0ull)) continue;
        uint32_t d = 0;
        if (m) {
            uint32_t rs, re;
            range_of(g, u, rs, re);
            d = re - rs;
        }
        for (uint32_t s = 0; s < G; ++s) {
            const bool in = (m >> s) & 1ull;
            const uint32_t bal = __ballot_sync(kFull, in);
            if (bal) {
                const uint32_t e = __reduce_add_sync(kFull, in ? d : 0u);
                if (lane == 0) {
                    atomicAdd(&s_cnt[s], (uint32_t)__popc(bal));
                    atomicAdd(&s_edg[s], e);
                }
            }
        }
    }
}

// Write pass over words [w0, w0 + kWordsPerItem): member lists and bitmap
// words of the group's sets; clears vis.
__device__ __forceinline__ void write_item(const DevGraph& g, const SampleBatch& b, const SlotArrays& a,
                                           uint32_t G, uint32_t words, uint32_t w0, const uint32_t* s_kind,
                                           const unsigned long long* s_pos, uint32_t lane)
{
    const uint32_t w1 = min(w0 + kWordsPerItem, words);
    for (uint32_t w = w0; w < w1; ++w) {
        const uint32_t u = (w << 5) + lane;
        unsigned long long m = 0;
        if (u < g.n) {
            m = __ldcg(a.vis + u);
            if (m) __stcg(a.vis + u, 0ull);
        }
        uint32_t mine0 = 0, mine1 = 0;  // bitmap word w of sets lane and lane + 32
        if (__any_sync(kFull, m != 0ull)) {
            for (uint32_t s = 0; s < G; ++s) {
                const bool in = (m >> s) & 1ull;
                const uint32_t bal = __ballot_sync(kFull, in);
                if (lane == (s & 31)) {
                    if (s < 32) mine0 = bal;
                    else mine1 = bal;
                }
                if (bal && s_kind[s] == 0) {
                    uint32_t base = 0;
                    if (lane == 0) base = (uint32_t)atomicAdd(&a.ct->lcur[s], (unsigned long long)__popc(bal));
                    base = __shfl_sync(kFull, base, 0);
                    if (in) b.big[s_pos[s] + base + __popc(bal & lanemask_lt_g())] = u;
                }
            }
        }
        if (lane < G && s_kind[lane] == 1) b.big[s_pos[lane] + w] = mine0;
        if (lane + 32 < G && s_kind[lane + 32] == 1) b.big[s_pos[lane + 32] + w] = mine1;
    }
}

// Two groups are in flight: a step (between grid barriers) serves both
// slots, so one group's small levels, level ends and extraction passes
// overlap the other's big levels.
__global__ void __launch_bounds__(kGroupThreads, kGroupBlocks)
ic_group_kernel(DevGraph g, SampleBatch b, GroupScratch gs)
{
    extern __shared__ uint32_t s_hbase[];  // [2][kHeavySmem] copies of the levels' chunk prefixes
    __shared__ PhiloxSet s_ps[2][kGroupSets];
    __shared__ uint4 s_rec[kGroupWarps][32];                // run records: rs, re, first slot
    __shared__ unsigned long long s_recF[kGroupWarps][32];  // run records: frontier mask
    __shared__ uint32_t s_cnt[2][kGroupSets], s_edg[2][kGroupSets], s_kind[2][kGroupSets];
    __shared__ unsigned long long s_pos[2][kGroupSets];
    __shared__ SlotStep s_st[2];
    __shared__ uint32_t s_next;

    cg::grid_group grid = cg::this_grid();
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31, wid = tid >> 5;
    const uint32_t large_count = b.sc->large_count;  // final: written by the previous launch
    const uint32_t words = b.words;
    const uint32_t witems = (words + kWordsPerItem - 1) / kWordsPerItem;
    uint32_t* claim = gs.ctr[0].claim;

    if (tid == 0) {
        s_st[0].phase = kIdle;
        s_st[1].phase = kIdle;
        s_next = 0;
    }
    for (uint32_t step = 0;; ++step) {
        // ---- advance both slots (thread 0 of every CTA, same inputs)
        if (tid == 0) {
            for (uint32_t k = 0; k < 2; ++k) {
                SlotStep& v = s_st[k];
                const GroupCounters* ct = gs.ctr + k;
                if (v.phase == kBfs) ++v.level;
                else if (v.phase == kInit) {
                    v.phase = kBfs;
                    v.level = 0;
                } else if (v.phase == kCount) v.phase = kReserve;
                else if (v.phase == kReserve) v.phase = kWrite;
                else if (v.phase == kWrite) v.phase = kIdle;
                if (v.phase == kBfs) {
                    const uint32_t cur = v.level % 3;
                    const unsigned long long hp = __ldcg(&ct->hpack[cur]);
                    v.nh = (uint32_t)(hp >> 40);
                    v.nch = (uint32_t)(hp & kLow40);
                    v.nl = __ldcg(&ct->lcount[cur]);
                    if (v.nch == 0 && v.nl == 0) v.phase = kCount;
                }
                if (v.phase == kIdle && s_next < large_count) {
                    v.phase = kInit;
                    v.g0 = s_next;
                    v.G = min(kGroupSets, large_count - s_next);
                    s_next += kGroupSets;
                }
                v.items = v.phase == kBfs ? (v.nl + 31) / 32 + v.nch
                                          : (v.phase == kCount || v.phase == kWrite ? witems : 0u);
            }
        }
        __syncthreads();
        if (s_st[0].phase == kIdle && s_st[1].phase == kIdle) {
            // every CTA is past the last barrier: leave the claim counters
            // zero for the next launch
            if (blockIdx.x == 0 && tid < 3) claim[tid] = 0;
            break;
        }

        // ---- per-CTA preparation of each slot's step
        if (blockIdx.x == 0 && tid == 0) claim[(step + 2) % 3] = 0;  // the step before this one's
        for (uint32_t k = 0; k < 2; ++k) {
            const SlotStep v = s_st[k];
            const SlotArrays a = slot_arrays(gs, k);
            if (v.phase == kInit) {
                if (tid < v.G) {
                    const uint64_t s = b.base + b.large_q[v.g0 + tid];
                    s_ps[k][tid] = philox_set((uint32_t)s, (uint32_t)(s >> 32), kTagIC, b.rk);
                }
                if (blockIdx.x == 0) {
                    if (tid < 3) {
                        a.ct->hpack[tid] = 0;
                        a.ct->lcount[tid] = 0;
                    }
                    if (tid < kGroupSets) {
                        a.ct->cnt[tid] = 0;
                        a.ct->edges[tid] = 0;
                        a.ct->lcur[tid] = 0;
                    }
                    __syncthreads();
                    if (tid < v.G) {
                        const uint64_t s = b.base + b.large_q[v.g0 + tid];
                        const uint32_t root = draw_root(b.rk, s, g.n);
                        if (atomicOr(a.fr0 + root, 1ull << tid) == 0ull) {
                            const LevelOut o = {&a.ct->hpack[0], &a.ct->lcount[0], a.lq0, a.hb0, a.he0};
                            uint32_t rs, re;
                            range_of(g, root, rs, re);
                            if (queue_large(o, root, rs, re)) a.lq0[atomicAdd(&a.ct->lcount[0], 1u)] = root;
                        }
                    }
                }
            } else if (v.phase == kBfs) {
                if (blockIdx.x == 0 && tid == 0) {
                    // counters of the level before this one: read by everybody
                    // before the last barrier; they serve the level after next
                    const uint32_t old = (v.level + 2) % 3;
                    a.ct->hpack[old] = 0;
                    a.ct->lcount[old] = 0;
                }
                if (v.nh <= kHeavySmem) {
                    const uint32_t* hb = (v.level & 1u) ? a.hb1 : a.hb0;
                    for (uint32_t i = tid; i < v.nh; i += kGroupThreads) s_hbase[k * kHeavySmem + i] = __ldcg(hb + i);
                }
            } else if (v.phase == kCount) {
                if (tid < kGroupSets) {
                    s_cnt[k][tid] = 0;
                    s_edg[k][tid] = 0;
                }
            } else if (v.phase == kReserve) {
                if (blockIdx.x == 0 && tid < v.G) {
                    const uint32_t rel = b.large_q[v.g0 + tid];
                    const uint32_t len = __ldcg(&a.ct->cnt[tid]);
                    b.set_edges[rel] = __ldcg(&a.ct->edges[tid]);
                    const uint32_t kind = len > words ? 1u : 0u;
                    uint64_t pos = 0;
                    const bool ok = reserve_big(b, rel, len, kind, &pos);
                    a.ct->kind[tid] = ok ? kind : 2u;
                    a.ct->pos[tid] = pos;
                }
            } else if (v.phase == kWrite) {
                if (tid < v.G) {
                    s_kind[k][tid] = __ldcg(&a.ct->kind[tid]);
                    s_pos[k][tid] = __ldcg(&a.ct->pos[tid]);
                }
            }
        }
        __syncthreads();

        // ---- work items of both slots from one counter
        const uint32_t i0 = s_st[0].items, total = i0 + s_st[1].items;
        uint32_t* cl = claim + step % 3;
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(cl, 1u);
        c = __shfl_sync(kFull, c, 0);
        while (c < total) {
            uint32_t cn = 0;  // the next claim, in flight while this item runs
            if (lane == 0) cn = atomicAdd(cl, 1u);
            const uint32_t k = c < i0 ? 0u : 1u;
            const uint32_t ci = c - (k ? i0 : 0u);
            const SlotStep& v = s_st[k];
            const SlotArrays a = slot_arrays(gs, k);
            if (v.phase == kBfs) {
                const LevelView lv = level_view(a, v.level);
                const uint32_t nlc = (v.nl + 31) / 32;
                // small-vertex chunks first (up to 31 windows each), then the
                // one-window chunks of the large vertices
                if (ci < nlc) small_item(g, b.rk, s_ps[k], a, lv, v.nl, ci * 32, s_rec[wid], s_recF[wid], lane);
                else large_item(g, b.rk, s_ps[k], a, lv, s_hbase + k * kHeavySmem, v.nh <= kHeavySmem, v.nh,
                                ci - nlc, lane);
            } else if (v.phase == kCount) {
                count_item(g, a, v.G, words, ci * kWordsPerItem, s_cnt[k], s_edg[k], lane);
            } else {
                write_item(g, b, a, v.G, words, ci * kWordsPerItem, s_kind[k], s_pos[k], lane);
            }
            c = __shfl_sync(kFull, cn, 0);
        }
        __syncthreads();
        for (uint32_t k = 0; k < 2; ++k) {
            if (s_st[k].phase == kCount && tid < s_st[k].G) {
                GroupCounters* ct = gs.ctr + k;
                atomicAdd(&ct->cnt[tid], s_cnt[k][tid]);
                atomicAdd(&ct->edges[tid], s_edg[k][tid]);
            }
        }
        grid.sync();
    }
}

constexpr size_t kGroupDynSmem = 2 * kHeavySmem * 4;

int ic_group_supported(const DeviceInfo& di)
{
    if (!di.cooperative) return 0;
    if (cudaFuncSetAttribute(ic_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGroupDynSmem) !=
        cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ic_group_kernel, kGroupThreads, kGroupDynSmem) !=
        cudaSuccess)
        return 0;
    return per_sm >= kGroupBlocks ? 1 : 0;
}

uint64_t ic_group_heavy_cap(uint32_t n, uint64_t m)
{
    // a vertex with >= 32 in-edge quads has >= 122 in-edges
    return std::min<uint64_t>((uint64_t)n, m / 122 + 1);
}

cudaError_t launch_ic_group(const DevGraph& g, const SampleBatch& b, const GroupScratch& gs, const DeviceInfo& di,
                            cudaStream_t st)
{
    DevGraph ga = g;
    SampleBatch ba = b;
    GroupScratch sa = gs;
    void* args[] = {&ga, &ba, &sa};
    return cudaLaunchCooperativeKernel((const void*)ic_group_kernel, dim3((unsigned)(di.sms * kGroupBlocks)),
                                       dim3(kGroupThreads), args, kGroupDynSmem, st);
}

}  // namespace imm
