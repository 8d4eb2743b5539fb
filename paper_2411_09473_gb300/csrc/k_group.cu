// IC large path, grouped: the large RRR sets of a batch are sampled 64 at a
// time by the whole GPU as one multi-source reverse BFS (Generate_RRRsets,
// EfficientIMM Alg. 3, for many roots at once).
//
// Each vertex carries two 64-bit masks over the sets of the group: vis (the
// sets that reached it in earlier levels) and fn (the sets that reached it in
// the level being expanded).  A level takes two steps:
//   expand  every vertex v of the level, with its new sets F, reads its
//           in-edge thresholds and sources once and flips the coins of every
//           set in F: in-edge e = (u -> v) of set s is live iff word e&3 of
//           Philox(s, e>>2) passes e's threshold (the same draw as the
//           one-set-per-CTA path, so every set is the reverse-reachable
//           closure of its root under its own coins, whatever the traversal
//           order).  Live bits u lacks in vis[u] are ored into fn[u], with no
//           value returned.
//   scan    a dense pass over fn merges every nonzero fn[v] into vis[v],
//           clears it and lists v with F = fn[v] for the next expansion:
//           vertices with >= 32 in-edge quads in a large list with a running
//           count of 64-quad chunks, the others in a small list with their
//           offsets in the level's small quads (and, for each window of 32
//           of those quads, its first vertex).
// vis changes only in scan steps, so expansions read it without races.  The
// giant sets of a power-law graph walk the same high-degree core within a
// level or two of each other, so the per-vertex work (edge range, threshold
// and source loads, quad bookkeeping) is shared by the sets that reach v at
// the same level.
//
// The kernel is persistent (cooperative launch, one 1024-thread CTA per SM)
// and advances in steps separated by grid barriers; warps claim work items
// from one counter.  Expansion items are windows of 32 of the small
// vertices' quads, one quad per lane (its owner found from per-warp run
// records in shared memory), and 64-quad chunks of the large vertices, two
// quads per lane sharing each set's bookkeeping (owner read from a per-chunk
// table the scan step writes).
//
// When no vertex is listed, two dense passes over vis give every set its
// size and in-edge sum, reserve its output (member list, or an n-bit bitmap
// when the list would be larger; Sec. IV-C), write it, and clear vis.
//
// kGroupSlots groups are in flight, in slots of the arrays, each started a
// few steps after the previous one: every step serves all of them (long
// items first, then the large-vertex chunks, which even out the end of the
// step), so the fixed cost of a step (its last item and the grid barrier) is
// shared by several groups, and one group's small levels, scans and
// extraction passes overlap the others' big levels.
#include "imm_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace imm {

namespace cg = cooperative_groups;

constexpr int kGroupThreads = 1024;  // threads per CTA
constexpr int kGroupBlocks = 1;      // CTAs per SM (the cooperative grid is SMs x this)
constexpr int kGroupChains = 2;      // independent Philox chains per lane in a sweep
constexpr int kGroupWarps = kGroupThreads / 32;
constexpr uint32_t kGroupHeavyQ = 32;  // in-edge quads from which a vertex is swept in chunks
constexpr uint32_t kChunkQuads = 64;   // quads of a large vertex per work item (two per lane)
// packed list counters: entries << 36 | quads (small list) or chunks (large list)
constexpr int kPackShift = 36;
constexpr unsigned long long kPackLow = (1ull << kPackShift) - 1;

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
// two independent Philox evaluations are in flight.  A set's bit enters each
// accumulator at most once, so the live bits are added rather than ored
// (the adds may issue on the multiply-add pipe, which the xors leave idle).
__device__ __forceinline__ void sweep_half(uint32_t mask, uint64_t a, uint4 tm, const PhiloxSet* ps,
                                           const PhiloxKeys& rk, uint32_t* acc)
{
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    while (mask) {
        const int s1 = 31 - __clz(mask);
        const uint32_t b1 = 1u << s1;
        mask -= b1;  // b1 is set in mask: the same as clearing it
        const uint4 w1 = philox_xa(a, ps[s1], rk);
        if (kGroupChains == 2) {
            const bool two = mask != 0;
            const int s2 = two ? 31 - __clz(mask) : s1;
            const uint32_t b2 = two ? 1u << s2 : 0u;
            mask -= b2;
            const uint4 w2 = philox_xa(a, ps[s2], rk);
            if (w2.x <= tm.x) a0 += b2;
            if (w2.y <= tm.y) a1 += b2;
            if (w2.z <= tm.z) a2 += b2;
            if (w2.w <= tm.w) a3 += b2;
        }
        if (w1.x <= tm.x) a0 += b1;
        if (w1.y <= tm.y) a1 += b1;
        if (w1.z <= tm.z) a2 += b1;
        if (w1.w <= tm.w) a3 += b1;
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

// One half (32 sets) for two quads of the same vertex (same sets): per set,
// the two quads' Philox evaluations are the two independent chains, and the
// set's bookkeeping is shared by both.
__device__ __forceinline__ void sweep_half2(uint32_t mask, uint64_t aa, uint64_t ab, uint4 ta, uint4 tb,
                                            const PhiloxSet* ps, const PhiloxKeys& rk, uint32_t* acc_a,
                                            uint32_t* acc_b)
{
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
    while (mask) {
        const int s = 31 - __clz(mask);
        const uint32_t bit = 1u << s;
        mask -= bit;  // bit is set in mask: the same as clearing it
        const PhiloxSet p = ps[s];
        const uint4 wa = philox_xa(aa, p, rk);
        const uint4 wb = philox_xa(ab, p, rk);
        if (wa.x <= ta.x) a0 += bit;
        if (wa.y <= ta.y) a1 += bit;
        if (wa.z <= ta.z) a2 += bit;
        if (wa.w <= ta.w) a3 += bit;
        if (wb.x <= tb.x) b0 += bit;
        if (wb.y <= tb.y) b1 += bit;
        if (wb.z <= tb.z) b2 += bit;
        if (wb.w <= tb.w) b3 += bit;
    }
    acc_a[0] = a0;
    acc_a[1] = a1;
    acc_a[2] = a2;
    acc_a[3] = a3;
    acc_b[0] = b0;
    acc_b[1] = b1;
    acc_b[2] = b2;
    acc_b[3] = b3;
}

// Thresholds of a quad as the compare bounds of sweep_half, and the mask of
// its in-edges that are in [rs, re) and can be live (th > 0).
__device__ __forceinline__ uint4 quad_bounds(const DevGraph& g, uint32_t quad, uint32_t rs, uint32_t re,
                                             uint32_t* valid)
{
    const uint4 th = __ldg(reinterpret_cast<const uint4*>(g.thr) + quad);
    uint32_t v = (th.x ? 1u : 0u) | (th.y ? 2u : 0u) | (th.z ? 4u : 0u) | (th.w ? 8u : 0u);
    const uint32_t e0 = quad << 2;
    if (e0 < rs) v &= 0xFu << (rs - e0);
    if (e0 + 4 > re) v &= 0xFu >> (e0 + 4 - re);
    *valid = v;
    return make_uint4((th.x << 8) - 1u, (th.y << 8) - 1u, (th.z << 8) - 1u, (th.w << 8) - 1u);
}

__device__ __forceinline__ void mask_invalid(QuadLive& ql, uint32_t valid)
{
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (!((valid >> t) & 1u)) {
            ql.lo[t] = 0;
            ql.hi[t] = 0;
        }
    }
}

// Coins of all sets in F for quads qa and qb = qa + 32 of one vertex (qb
// beyond the vertex's last quad when !hb: its results are cleared).
__device__ __forceinline__ void sweep_two(const DevGraph& g, const PhiloxKeys& rk, const PhiloxSet* ps,
                                          uint32_t qa, uint32_t qb, bool hb, uint32_t rs, uint32_t re,
                                          unsigned long long F, QuadLive& la, QuadLive& lb)
{
    la.src = __ldg(reinterpret_cast<const uint4*>(g.src) + qa);
    lb.src = hb ? __ldg(reinterpret_cast<const uint4*>(g.src) + qb) : make_uint4(0, 0, 0, 0);
    uint32_t va, vb;
    const uint4 ta = quad_bounds(g, qa, rs, re, &va);
    uint4 tb = make_uint4(0, 0, 0, 0);
    vb = 0;
    if (hb) tb = quad_bounds(g, qb, rs, re, &vb);
    const uint64_t aa = (uint64_t)kPhiloxM1 * (uint64_t)qa, ab = (uint64_t)kPhiloxM1 * (uint64_t)qb;
    sweep_half2((uint32_t)F, aa, ab, ta, tb, ps, rk, la.lo, lb.lo);
    sweep_half2((uint32_t)(F >> 32), aa, ab, ta, tb, ps + 32, rk, la.hi, lb.hi);
    mask_invalid(la, va);
    mask_invalid(lb, vb);
}

// Apply the live bits of one quad per lane: they are ored into fn[u] with no
// value returned, so nothing waits on the visit.  Bits of sets that have
// already reached u are dropped by the next scan step, which lists u only
// with the sets it is new to.
__device__ __forceinline__ void visit_quad(unsigned long long* fn, const QuadLive& ql)
{
    const uint32_t u[4] = {ql.src.x, ql.src.y, ql.src.z, ql.src.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const unsigned long long m = ((unsigned long long)ql.hi[t] << 32) | ql.lo[t];
        if (m) atomicOr(fn + u[t], m);
    }
}

// Arrays of one group slot (slot k's lie k * `stride` bytes after slot 0's).
struct SlotArrays {
    unsigned long long *vis, *fn;
    uint4 *lq, *he;
    uint32_t *lpre, *wst, *hb, *cown;
    GroupCounters* ct;
    uint32_t lcap, wcap, hcap, ccap;  // entries of lq / lpre, wst, hb / he, cown
    unsigned long long* err;          // checked builds: the batch's error word
};

__device__ __forceinline__ SlotArrays slot_arrays(const GroupScratch& gs, uint32_t k)
{
    const uint64_t d = (uint64_t)k * gs.stride;
    auto at = [d](auto* p) { return reinterpret_cast<decltype(p)>(reinterpret_cast<char*>(p) + d); };
    SlotArrays a;
    a.vis = at(gs.vis);
    a.fn = at(gs.fn);
    a.lq = at(gs.lq);
    a.he = at(gs.he);
    a.lpre = at(gs.lpre);
    a.wst = at(gs.wst);
    a.hb = at(gs.hb);
    a.cown = at(gs.cown);
    a.ct = gs.ctr + k;
    a.lcap = gs.lcap;
    a.wcap = gs.wcap;
    a.hcap = gs.hcap;
    a.ccap = gs.ccap;
    a.err = gs.bounds;
    return a;
}

// A vertex with >= 32 in-edge quads and new bits F enters the level's large
// list (64-quad chunks; chunk prefix in hb).
__device__ __forceinline__ void list_large(const SlotArrays& a, uint32_t par, uint32_t rs, uint32_t re,
                                           uint32_t nq, unsigned long long F)
{
    const uint32_t nch = (nq + kChunkQuads - 1) / kChunkQuads;
    const unsigned long long old = atomicAdd(&a.ct->hpack[par], (1ull << kPackShift) | (unsigned long long)nch);
    const uint32_t i = (uint32_t)(old >> kPackShift);
    if (!IMM_IN_BOUNDS(i, a.hcap, a.err, kChkGroupLarge)) return;
    const uint32_t first = (uint32_t)(old & kPackLow);
    a.hb[i] = first;
    a.he[i] = make_uint4(rs, re, (uint32_t)F, (uint32_t)(F >> 32));
    // the owner of each of its chunks, so a chunk item finds its vertex in one load
    for (uint32_t c = 0; c < nch; ++c)
        if (IMM_IN_BOUNDS(first + c, a.ccap, a.err, kChkGroupLarge)) a.cown[first + c] = i;
}

// Small-list entry i of a vertex with 1..31 in-edge quads at quad offset off
// of the level's small quads.  The windows of 32 quads that the expansion
// sweeps start at multiples of 32; the one window start inside
// [off, off + nq), if any, records i as that window's first entry.
__device__ __forceinline__ void list_small(const SlotArrays& a, uint32_t i, uint32_t off, uint32_t rs,
                                           uint32_t re, uint32_t nq, unsigned long long F)
{
    if (!IMM_IN_BOUNDS(i, a.lcap, a.err, kChkGroupSmall)) return;
    a.lq[i] = make_uint4(rs, re, (uint32_t)F, (uint32_t)(F >> 32));
    a.lpre[i] = off;
    const uint32_t w = (off + 31) >> 5;
    if ((w << 5) < off + nq && IMM_IN_BOUNDS(w, a.wcap, a.err, kChkGroupWin)) a.wst[w] = i;
}

// What a slot does in the current step (the same in every CTA: each CTA's
// thread 0 advances its copy from the same global counters).
constexpr uint32_t kIdle = 0, kInit = 1, kScan = 2, kExpand = 3, kCount = 4, kReserve = 5, kWrite = 6;
struct SlotStep {
    uint32_t phase;
    uint32_t level;        // BFS level listed (kScan) or expanded (kExpand)
    uint32_t g0, G;        // the group: large-queue entries g0 .. g0 + G - 1
    uint32_t nl, nlq;      // kExpand: small vertices and their quads
    uint32_t nch, nh;      // kExpand: large-vertex chunks, large vertices
    uint32_t nlong, nshort;  // work items: windows of small quads (or scan / extraction items), large chunks
};
constexpr uint32_t kWordsPerItem = 8;     // bitmap words per extraction item
constexpr uint32_t kScanPerItem = 256;    // vertices per scan item
constexpr uint32_t kSlotOffset = 2;       // steps by which slot k starts after slot k - 1

// Scan of vertices [v0, v0 + kScanPerItem): every vertex with bits in fn has
// fn cleared; the sets among them that had not reached it yet (F) are merged
// into vis, and the vertex is listed for their expansion unless it has no
// in-edges.
__device__ __forceinline__ void scan_item(const DevGraph& g, const SlotArrays& a, uint32_t par, uint32_t v0,
                                          uint32_t lane)
{
    // the item's fn words are loaded at once (one round trip, not eight)
    unsigned long long Fs[kScanPerItem / 32];
#pragma unroll
    for (uint32_t r = 0; r < kScanPerItem / 32; ++r) {
        const uint32_t v = v0 + r * 32 + lane;
        Fs[r] = v < g.n ? __ldcg(a.fn + v) : 0ull;
    }
#pragma unroll
    for (uint32_t r8 = 0; r8 < kScanPerItem / 32; ++r8) {
        const uint32_t r = r8 * 32;
        const uint32_t v = v0 + r + lane;
        unsigned long long F = Fs[r8];
        if (!__any_sync(kFull, F != 0ull)) continue;
        if (F) {
            __stcg(a.fn + v, 0ull);
            const unsigned long long old = __ldcg(a.vis + v);
            F &= ~old;
            if (F) __stcg(a.vis + v, old | F);
        }
        uint32_t rs = 0, re = 0, nq = 0;
        if (F) {
            range_of(g, v, rs, re);
            nq = nquads(rs, re);
            if (nq >= kGroupHeavyQ) {
                list_large(a, par, rs, re, nq, F);
                nq = 0;
            }
        }
        // small vertices of the warp: one packed reservation of entries and quads
        uint32_t incl = nq;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, d);
            if ((int)lane >= d) incl += t;
        }
        const uint32_t bal = __ballot_sync(kFull, nq != 0);
        if (bal) {
            unsigned long long base = 0;
            if (lane == 31)
                base = atomicAdd(&a.ct->lpack[par],
                                 ((unsigned long long)__popc(bal) << kPackShift) | (unsigned long long)incl);
            base = __shfl_sync(kFull, base, 31);
            if (nq)
                list_small(a, (uint32_t)(base >> kPackShift) + __popc(bal & lanemask_lt_g()),
                           (uint32_t)(base & kPackLow) + incl - nq, rs, re, nq, F);
        }
    }
}

// 64-quad chunk hc of the level's large vertices: lane t sweeps quads t and
// t + 32 of the chunk (the second only when some lane has one there).  Its
// vertex is the large-list entry the scan step recorded as its owner.
__device__ __forceinline__ void large_item(const DevGraph& g, const PhiloxKeys& rk, const PhiloxSet* ps,
                                           const SlotArrays& a, uint32_t hc, uint32_t lane)
{
    const uint32_t lo = __ldcg(a.cown + hc);
    const uint4 e = __ldcg(a.he + lo);
    const uint32_t first = __ldcg(a.hb + lo);
    const uint32_t qa = (e.x >> 2) + (hc - first) * kChunkQuads + lane, qb = qa + 32;
    const uint32_t qlast = (e.y - 1) >> 2;
    const unsigned long long F = ((unsigned long long)e.w << 32) | e.z;
    const bool ha = qa <= qlast, hb = qb <= qlast;
    QuadLive la = {};
    if (__any_sync(kFull, hb)) {
        QuadLive lb = {};
        if (ha) sweep_two(g, rk, ps, qa, qb, hb, e.x, e.y, F, la, lb);
        visit_quad(a.fn, la);
        visit_quad(a.fn, lb);
    } else {
        if (ha) sweep_quad(g, rk, ps, qa, e.x, e.y, F, la);
        visit_quad(a.fn, la);
    }
}

// Window c of the level's small quads: quads [32c, 32c + 32) of the small
// list, one per lane.  Its first entry is wst[c]; every entry has at least
// one quad, so the window meets at most the 32 entries from there.  The run
// of each entry that meets the window is recorded at its first slot there;
// a slot's owner is the last recorded start at or before it.
__device__ __forceinline__ void window_item(const DevGraph& g, const PhiloxKeys& rk, const PhiloxSet* ps,
                                            const SlotArrays& a, uint32_t nl, uint32_t nlq, uint32_t c,
                                            uint4* rec, unsigned long long* recF, uint32_t lane)
{
    const uint32_t w0 = c << 5;
    const uint32_t i = __ldcg(a.wst + c) + lane;
    uint4 e = make_uint4(0, 0, 0, 0);
    uint32_t off = 0, nq = 0;
    if (i < nl) {
        off = __ldcg(a.lpre + i);
        if (off < w0 + 32) {
            e = __ldcg(a.lq + i);
            nq = nquads(e.x, e.y);
        }
    }
    const bool meets = nq != 0 && off + nq > w0;
    const uint32_t st = off > w0 ? off - w0 : 0u;
    if (meets) {
        rec[st] = make_uint4(e.x, e.y, off, 0u);
        recF[st] = ((unsigned long long)e.w << 32) | e.z;
    }
    const uint32_t starts = __reduce_or_sync(kFull, meets ? 1u << st : 0u);
    __syncwarp();
    const uint32_t j = w0 + lane;
    QuadLive ql = {};
    if (j < nlq) {
        const uint32_t pos = 31 - __clz(starts & lanemask_le_g());
        const uint4 r = rec[pos];
        const uint32_t quad = (r.x >> 2) + (j - r.z);
        sweep_quad(g, rk, ps, quad, r.x, r.y, recF[pos], ql);
    }
    visit_quad(a.fn, ql);
    __syncwarp();
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
                    const uint64_t at = s_pos[s] + base + __popc(bal & lanemask_lt_g());
                    if (in && IMM_IN_BOUNDS(at, b.big_cap, a.err, kChkBig)) b.big[at] = u;
                }
            }
        }
        if (lane < G && s_kind[lane] == 1 && IMM_IN_BOUNDS(s_pos[lane] + w, b.big_cap, a.err, kChkBig))
            b.big[s_pos[lane] + w] = mine0;
        if (lane + 32 < G && s_kind[lane + 32] == 1 && IMM_IN_BOUNDS(s_pos[lane + 32] + w, b.big_cap, a.err, kChkBig))
            b.big[s_pos[lane + 32] + w] = mine1;
    }
}

__global__ void __launch_bounds__(kGroupThreads, kGroupBlocks)
ic_group_kernel(DevGraph g, SampleBatch b, GroupScratch gs)
{
    __shared__ PhiloxSet s_ps[kGroupSlots][kGroupSets];
    __shared__ uint4 s_rec[kGroupWarps][32];                // run records: rs, re, first slot
    __shared__ unsigned long long s_recF[kGroupWarps][32];  // run records: new bits
    __shared__ uint32_t s_cnt[kGroupSlots][kGroupSets], s_edg[kGroupSlots][kGroupSets];
    __shared__ uint32_t s_kind[kGroupSlots][kGroupSets];
    __shared__ unsigned long long s_pos[kGroupSlots][kGroupSets];
    __shared__ SlotStep s_st[kGroupSlots];
    __shared__ uint32_t s_lbase[kGroupSlots + 1], s_sbase[kGroupSlots + 1];  // item ranges of the step
    __shared__ uint32_t s_next;

    cg::grid_group grid = cg::this_grid();
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31, wid = tid >> 5;
    const uint32_t large_count = b.sc->large_count;  // final: written by the previous launch
    const uint32_t words = b.words;
    const uint32_t witems = (words + kWordsPerItem - 1) / kWordsPerItem;
    const uint32_t sitems = (g.n + kScanPerItem - 1) / kScanPerItem;
    uint32_t* claim = gs.ctr[0].claim;

    if (tid == 0) {
        for (uint32_t k = 0; k < kGroupSlots; ++k) s_st[k].phase = kIdle;
        s_next = 0;
    }
    for (uint32_t step = 0;; ++step) {
        // ---- advance every slot (thread 0 of every CTA, same inputs)
        if (tid == 0) {
            for (uint32_t k = 0; k < kGroupSlots; ++k) {
                SlotStep& v = s_st[k];
                const GroupCounters* ct = gs.ctr + k;
                const uint32_t was = v.phase;
                if (was == kInit) {
                    v.phase = kExpand;
                    v.level = 0;
                } else if (was == kScan) {
                    v.phase = kExpand;
                } else if (was == kExpand) {
                    v.phase = kScan;
                    ++v.level;
                } else if (was == kCount) {
                    v.phase = kReserve;
                } else if (was == kReserve) {
                    v.phase = kWrite;
                } else if (was == kWrite) {
                    v.phase = kIdle;
                }
                if (v.phase == kExpand) {
                    const uint32_t par = v.level & 1u;
                    const unsigned long long hp = __ldcg(&ct->hpack[par]);
                    const unsigned long long lp = __ldcg(&ct->lpack[par]);
                    v.nh = (uint32_t)(hp >> kPackShift);
                    v.nch = (uint32_t)(hp & kPackLow);
                    v.nl = (uint32_t)(lp >> kPackShift);
                    v.nlq = (uint32_t)(lp & kPackLow);
                    if (v.nch == 0 && v.nl == 0) v.phase = kCount;
                }
                if (v.phase == kIdle && s_next < large_count && step >= k * kSlotOffset) {
                    v.phase = kInit;
                    v.g0 = s_next;
                    v.G = min(kGroupSets, large_count - s_next);
                    s_next += kGroupSets;
                }
                v.nlong = v.phase == kExpand ? (v.nlq + 31) / 32
                        : v.phase == kScan ? sitems
                        : (v.phase == kCount || v.phase == kWrite) ? witems : 0u;
                v.nshort = v.phase == kExpand ? v.nch : 0u;
            }
            // item ranges: the long items of all slots, then the large-vertex chunks
            uint32_t x = 0;
            for (uint32_t k = 0; k < kGroupSlots; ++k) {
                s_lbase[k] = x;
                x += s_st[k].nlong;
            }
            s_lbase[kGroupSlots] = x;
            for (uint32_t k = 0; k < kGroupSlots; ++k) {
                s_sbase[k] = x;
                x += s_st[k].nshort;
            }
            s_sbase[kGroupSlots] = x;
        }
        __syncthreads();
        bool idle = s_next >= large_count;
        for (uint32_t k = 0; k < kGroupSlots; ++k) idle = idle && s_st[k].phase == kIdle;
        if (idle) {
            // every CTA is past the last barrier: leave the claim counters
            // zero for the next launch
            if (blockIdx.x == 0 && tid < 3) claim[tid] = 0;
            break;
        }

        // ---- per-CTA preparation of each slot's step
        if (blockIdx.x == 0 && tid == 0) claim[(step + 2) % 3] = 0;  // the step before this one's
        for (uint32_t k = 0; k < kGroupSlots; ++k) {
            const SlotStep v = s_st[k];
            const SlotArrays a = slot_arrays(gs, k);
            if (v.phase == kInit) {
                if (tid < v.G) {
                    const uint64_t s = b.base + b.large_q[v.g0 + tid];
                    s_ps[k][tid] = philox_set((uint32_t)s, (uint32_t)(s >> 32), kTagIC, b.rk);
                }
                if (blockIdx.x == 0) {
                    // level 0: the roots, listed directly
                    if (tid < 2) {
                        a.ct->hpack[tid] = 0;
                        a.ct->lpack[tid] = 0;
                    }
                    if (tid < kGroupSets) {
                        a.ct->cnt[tid] = 0;
                        a.ct->edges[tid] = 0;
                        a.ct->lcur[tid] = 0;
                    }
                    uint32_t root = 0;
                    bool first = false;
                    if (tid < v.G) {
                        const uint64_t s = b.base + b.large_q[v.g0 + tid];
                        root = draw_root(b.rk, s, g.n);
                        first = atomicOr(a.fn + root, 1ull << tid) == 0ull;
                    }
                    __syncthreads();
                    if (first) {
                        const unsigned long long F = __ldcg(a.fn + root);
                        __stcg(a.fn + root, 0ull);
                        __stcg(a.vis + root, F);
                        uint32_t rs, re;
                        range_of(g, root, rs, re);
                        const uint32_t nq = nquads(rs, re);
                        if (nq >= kGroupHeavyQ) {
                            list_large(a, 0, rs, re, nq, F);
                        } else if (nq) {
                            const unsigned long long old =
                                atomicAdd(&a.ct->lpack[0], (1ull << kPackShift) | (unsigned long long)nq);
                            list_small(a, (uint32_t)(old >> kPackShift), (uint32_t)(old & kPackLow), rs, re, nq, F);
                        }
                    }
                }
            } else if (v.phase == kExpand) {
                if (blockIdx.x == 0 && tid == 0) {
                    // the next scan's counters: last read at the top of the
                    // previous expansion step
                    const uint32_t np = (v.level + 1) & 1u;
                    a.ct->hpack[np] = 0;
                    a.ct->lpack[np] = 0;
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

        // ---- work items of all slots from one counter: the long items of
        // every slot first, then the large-vertex chunks (they even out the end)
        const uint32_t total = s_sbase[kGroupSlots];
        uint32_t* cl = claim + step % 3;
        // a claim takes two items while many remain (half the traffic on the
        // one counter), one item near the end of the step (a shorter tail)
        const uint32_t pair_until = total > 8u * kGroupWarps * gridDim.x ? total - 8u * kGroupWarps * gridDim.x : 0u;
        uint32_t c0 = 0, take = pair_until ? 2u : 1u;
        if (lane == 0) c0 = atomicAdd(cl, take);
        c0 = __shfl_sync(kFull, c0, 0);
        while (c0 < total) {
            const uint32_t c1 = min(c0 + take, total);
            take = c1 < pair_until ? 2u : 1u;
            uint32_t cn = 0;  // the next claim, in flight while these items run
            if (lane == 0) cn = atomicAdd(cl, take);
          for (uint32_t c = c0; c < c1; ++c) {
            const bool lng = c < s_lbase[kGroupSlots];
            const uint32_t* base = lng ? s_lbase : s_sbase;
            uint32_t k = 0;
            while (c >= base[k + 1]) ++k;
            const uint32_t ci = c - base[k];
            const SlotStep& v = s_st[k];
            const SlotArrays a = slot_arrays(gs, k);
            if (!lng) {
                large_item(g, b.rk, s_ps[k], a, ci, lane);
            } else if (v.phase == kExpand) {
                window_item(g, b.rk, s_ps[k], a, v.nl, v.nlq, ci, s_rec[wid], s_recF[wid], lane);
            } else if (v.phase == kScan) {
                scan_item(g, a, v.level & 1u, ci * kScanPerItem, lane);
            } else if (v.phase == kCount) {
                count_item(g, a, v.G, words, ci * kWordsPerItem, s_cnt[k], s_edg[k], lane);
            } else {
                write_item(g, b, a, v.G, words, ci * kWordsPerItem, s_kind[k], s_pos[k], lane);
            }
          }
            c0 = __shfl_sync(kFull, cn, 0);
        }
        __syncthreads();
        for (uint32_t k = 0; k < kGroupSlots; ++k) {
            if (s_st[k].phase == kCount && tid < s_st[k].G) {
                GroupCounters* ct = gs.ctr + k;
                atomicAdd(&ct->cnt[tid], s_cnt[k][tid]);
                atomicAdd(&ct->edges[tid], s_edg[k][tid]);
            }
        }
        grid.sync();
    }
}

constexpr size_t kGroupDynSmem = 0;

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
