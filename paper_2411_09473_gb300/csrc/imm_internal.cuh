// Internal declarations shared by the CUDA translation units of the IMM
// library (device structs, the Philox device function, launch wrappers).
// Not part of the public ABI (include/imm.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace imm {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kLenPending = 0xFFFFFFFEu;  // set handed to the block / long-walk path
constexpr uint32_t kLenFailed = 0xFFFFFFFFu;   // staging reservation failed; resample later
constexpr uint32_t kTagRoot = 1, kTagIC = 2, kTagLT = 3;
constexpr uint32_t kQ24 = 1u << 24;

// Device error bits (written to BatchScalars::error).
constexpr int kErrHashProbe = 1;
constexpr int kErrQueue = 2;
constexpr int kErrBadGraph = 4;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// -> 64-bit products whose halves are xored with the other counter words and
// the round key; the key advances by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// The ten round keys of one 64-bit key: k[2r], k[2r+1] are round r's words.
// Kernels receive them as parameters, so every round's xor reads its key
// straight from the constant bank instead of advancing it in registers.
struct PhiloxKeys {
    uint32_t k[20];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint64_t seed)
{
    PhiloxKeys rk;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k[2 * r] = k0;
        rk.k[2 * r + 1] = k1;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return rk;
}

__host__ __device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1)
{
    const uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)c.x;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)c.z;
    return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
}

__host__ __device__ __forceinline__ uint4 philox(uint4 c, const PhiloxKeys& rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) c = philox_round(c, rk.k[2 * r], rk.k[2 * r + 1]);
    return c;
}

// All draws of one RRR set use counters (s_lo, s_hi, x, tag) that differ in
// word 2 only.  Round 0 multiplies words 0 and 2, so its half fed by word 0
// (and word 3) is the same for every x; round 1 then multiplies that half's
// output again.  PhiloxSet holds those x-independent values, pre-xored with
// the round keys they meet, so a draw costs 1 + 1 + 2 x 8 products instead of
// 2 x 10 (the result is bit-identical to philox()).
struct PhiloxSet {
    uint32_t r0;    // round 0, word 0: s_hi ^ k0(0)
    uint32_t r1a;   // round 1, word 0: hi(M1 * a2) ^ k0(1)
    uint32_t r1b;   // round 1, word 2: a3 ^ k1(1)
    uint32_t r2;    // round 2, word 0: lo(M1 * a2) ^ k0(2)
};

__host__ __device__ __forceinline__ PhiloxSet philox_set(uint32_t s_lo, uint32_t s_hi, uint32_t tag,
                                                        const PhiloxKeys& rk)
{
    const uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)s_lo;
    const uint32_t a2 = (uint32_t)(p0 >> 32) ^ tag ^ rk.k[1];  // round 0, word 2
    const uint32_t a3 = (uint32_t)p0;                          // round 0, word 3
    const uint64_t b = (uint64_t)kPhiloxM1 * (uint64_t)a2;       // round 1, product of word 2
    PhiloxSet ps;
    ps.r0 = s_hi ^ rk.k[0];
    ps.r1a = (uint32_t)(b >> 32) ^ rk.k[2];
    ps.r1b = a3 ^ rk.k[3];
    ps.r2 = (uint32_t)b ^ rk.k[4];
    return ps;
}

// philox((s_lo, s_hi, x, tag), key) for the set `ps` was built from, given
// a = M1 * x (round 0's product of word 2, which is the same for every set:
// sweeping many sets over one x computes it once).
__host__ __device__ __forceinline__ uint4 philox_xa(uint64_t a, const PhiloxSet& ps, const PhiloxKeys& rk)
{
    // round 0: only the product of word 2 (= x) depends on x
    const uint32_t x0 = (uint32_t)(a >> 32) ^ ps.r0, x1 = (uint32_t)a;
    // round 1: counter (x0, x1, a2, a3); the product of a2 is in ps
    const uint64_t p = (uint64_t)kPhiloxM0 * (uint64_t)x0;
    // round 2: counter (y0, lo(M1 a2), y2, y3)
    const uint32_t y0 = x1 ^ ps.r1a, y2 = (uint32_t)(p >> 32) ^ ps.r1b, y3 = (uint32_t)p;
    const uint64_t q0 = (uint64_t)kPhiloxM0 * (uint64_t)y0;
    const uint64_t q1 = (uint64_t)kPhiloxM1 * (uint64_t)y2;
    uint4 c = make_uint4((uint32_t)(q1 >> 32) ^ ps.r2, (uint32_t)q1, (uint32_t)(q0 >> 32) ^ y3 ^ rk.k[5],
                         (uint32_t)q0);
#pragma unroll
    for (int r = 3; r < 10; ++r) c = philox_round(c, rk.k[2 * r], rk.k[2 * r + 1]);
    return c;
}

__host__ __device__ __forceinline__ uint4 philox_x(uint32_t x, const PhiloxSet& ps, const PhiloxKeys& rk)
{
    return philox_xa((uint64_t)kPhiloxM1 * (uint64_t)x, ps, rk);
}

// Root of set s: uniform over [0, n) by multiply-shift of a 64-bit draw.
__device__ __forceinline__ uint32_t draw_root(const PhiloxKeys& rk, uint64_t s, uint32_t n)
{
    const uint4 w = philox(make_uint4((uint32_t)s, (uint32_t)(s >> 32), 0u, kTagRoot), rk);
    const uint64_t x = ((uint64_t)w.y << 32) | w.x;
    return (uint32_t)__umul64hi(x, (uint64_t)n);
}

// ---------------------------------------------------------------------------
// Device-side views.
// ---------------------------------------------------------------------------
struct DevGraph {
    uint32_t n;
    uint64_t m;
    const uint64_t* row;  // n+1 in-edge offsets (CSR of G^T)
    const uint32_t* src;  // m (padded to a multiple of 4): tail of each in-edge
    const uint32_t* thr;  // m (padded, zeros): IC threshold or LT cumulative threshold
    const uint4* guide;     // LT only, m: guide[row[v] + b] = (j, cthr[j] | indeg(u) << 25,
                            // u = src[j], row[u]) for j the first in-edge of v with
                            // cthr[j] > ceil(b * 2^24 / indeg(v)), b < indeg(v)
                            // (no such j: j = row[v+1], the rest 0); j and indeg(u)
                            // packed as kGuideRelMax / kGuideDegRel / kGuideDegAbs say
};

// Counters and flags of one sampling batch (device memory, zeroed per batch
// except first_fail, set to kEmpty).
struct BatchScalars {
    uint32_t cursor;        // next batch-relative set id for the small-set path
    uint32_t large_count;   // sets handed to the large-set path
    uint32_t large_cursor;  // next entry of the large-set queue
    uint32_t first_fail;    // lowest batch-relative id whose output reservation failed
    unsigned long long stage_cursor;  // small-set staging (exact capacity)
    unsigned long long big_cursor;    // large-set outputs (lists or bitmaps)
    unsigned long long edges;         // IC: in-edges of the members; LT: walk steps
    unsigned long long committed;     // sets kept (min(first_fail, count)), by the scan
    unsigned long long list_members;  // members of kept sets stored as lists
    unsigned long long all_members;   // members of all kept sets
    unsigned long long nbitmaps;      // kept sets stored as bitmaps
    int error;
    int pad;
    unsigned long long bounds[3];     // checked builds: first failed index check (where, index, bound)
    uint32_t long_count;    // LT: walks handed on to the bitmap path
    uint32_t long_cursor;   // next entry of that queue
    uint32_t mid_claim;     // LT: per-walk tables claimed by the lane path
    uint32_t pad2;
};

// Index checks of the bounds-checked build (-DIMM_BOUNDS_CHECK): an index at
// or above its buffer's bound is not used; the first such index is recorded
// as (where, index, bound) in a device error word that the host reads after
// the launch and reports.  In the normal build the check is `true` and
// compiles away.
#ifdef IMM_BOUNDS_CHECK
__device__ __forceinline__ bool imm_in_bounds(uint64_t idx, uint64_t bound, unsigned long long* err, uint32_t where)
{
    if (idx < bound) return true;
    if (atomicCAS(err, 0ull, (unsigned long long)where) == 0ull) {
        err[1] = idx;
        err[2] = bound;
    }
    return false;
}
#define IMM_IN_BOUNDS(idx, bound, err, where) \
    ::imm::imm_in_bounds((uint64_t)(idx), (uint64_t)(bound), (err), (uint32_t)(where))
constexpr bool kBoundsChecked = true;
#else
#define IMM_IN_BOUNDS(idx, bound, err, where) true
constexpr bool kBoundsChecked = false;
#endif
// LT guide entries (one per in-edge): heads of at most kGuideRelMax in-edges
// store the candidate edge relative to their first in-edge in 16 bits and
// the tail's in-degree in 23 (kGuideDegRel: unknown, read the row); larger
// heads store it absolutely and the degree in 7 bits (kGuideDegAbs)
constexpr uint32_t kGuideRelMax = 0xFFFFu;
constexpr uint32_t kGuideDegRel = (1u << 23) - 1u;
constexpr uint32_t kGuideDegAbs = 127u;

// where codes of the checks
enum : uint32_t {
    kChkStage = 1, kChkLargeQ, kChkSlotQueue, kChkSlotBitmap, kChkBig, kChkArena, kChkInv, kChkGroupSmall,
    kChkGroupWin, kChkGroupLarge, kChkNewly, kChkCand, kChkUbmp, kChkCounts, kChkLongQ
};

constexpr uint64_t kBigFlag = 1ull << 63;  // set_pos points into the large-output buffer

struct SampleBatch {
    uint64_t seed;
    PhiloxKeys rk;        // round keys of `seed`
    uint64_t base;        // first set id of the batch
    uint32_t count;       // sets in the batch
    uint32_t words;       // ceil(n / 32): words of one n-bit bitmap
    uint32_t* set_len;    // [count] members
    uint64_t* set_pos;    // [count] output position (kBigFlag: large-output buffer)
    uint32_t* set_edges;  // [count] IC: in-edges of the members; LT: walk steps
    uint32_t* set_kind;   // [count] 0 = member list, 1 = n-bit bitmap
    uint32_t* stage;      // small-set member lists
    uint64_t stage_cap;
    uint32_t* big;        // large-set outputs
    uint64_t big_cap;
    uint32_t* large_q;    // [count] batch-relative ids for the large-set path
    uint32_t* long_q;     // [count] LT: ids of walks too long for a per-walk table
    BatchScalars* sc;
};

// Reserve space for a large set's output (list of len members, or a bitmap
// of b.words words).  When the buffer is full the set is marked failed; it
// and every later set of the batch are resampled by the next batch.
__device__ __forceinline__ bool reserve_big(const SampleBatch& b, uint32_t rel, uint32_t len, uint32_t kind,
                                            uint64_t* pos)
{
    const uint64_t size = kind ? (uint64_t)b.words : (uint64_t)len;
    const unsigned long long p = atomicAdd(&b.sc->big_cursor, (unsigned long long)size);
    if (p + size > b.big_cap) {
        b.set_len[rel] = kLenFailed;
        atomicMin(&b.sc->first_fail, rel);
        return false;
    }
    *pos = p;
    b.set_pos[rel] = p | kBigFlag;
    b.set_len[rel] = len;
    b.set_kind[rel] = kind;
    return true;
}

// Per-CTA scratch of the large-set path: a member queue of n entries and,
// when the visited bitmap does not fit in shared memory, an n-bit bitmap.
struct LargeSlots {
    uint32_t* queues;
    uint64_t queue_cap;
    uint32_t* bitmaps;
    uint64_t bitmap_words;
    uint32_t nslots;
};

// Per-walk tables of LT walks past the lane path's kLtCap members: an
// open-addressing table of kLtMidHash entries (member + 1, 0 = empty; zero
// between walks) in global memory, and the members it holds with their
// table slots in walk order.  The lane path claims them for the walks it
// continues (members kLtCap.. go to the table); the per-walk-table kernel
// uses them for walks it samples whole.  A walk longer than kLtMidCap
// members (or than a list of n/32 members) goes on to the bitmap path.
constexpr uint32_t kLtMidHashBits = 11;
constexpr uint32_t kLtMidHash = 1u << kLtMidHashBits;  // load factor at most 1/2
constexpr uint32_t kLtMidCap = 1024;
constexpr uint32_t kLtMidSlotsMax = 8192;  // 16 KB each
struct MidSlots {
    uint32_t* tab;   // [nslots][kLtMidHash]
    uint32_t* path;  // [nslots][kLtMidCap]
    uint32_t* hpos;  // [nslots][kLtMidCap]
    uint32_t nslots;
};

// One segment of the inverted index over the list-stored sets of one batch:
// inv[voff[v] .. voff[v+1]) = ids of the segment's sets that contain v.
struct DevSegment {
    const uint64_t* voff;
    const uint32_t* inv;
};

// Where the batch's kept sets go once the scan has run.
struct BatchOut {
    uint64_t* off;        // stream list offsets (off[base .. base+committed])
    uint32_t* arena;      // stream member lists
    uint32_t* set_bmp;    // [nsets] bitmap id of each set, kEmpty for lists
    uint32_t* bmp;        // bitmap arena, `words` words per bitmap
    uint32_t* bmp_set;    // [nbmp] set id of each bitmap
    uint32_t* bmp_len;    // [nbmp] members of each bitmap set
    uint32_t* bmp_rel;    // [count] batch-relative id of the batch's r-th bitmap
    uint64_t bmp_base;    // bitmaps stored before this batch
    uint64_t arena_cap;   // entries of arena
    unsigned long long* bounds;  // checked builds: the batch's error word (BatchScalars::bounds)
};

// ---------------------------------------------------------------------------
// Launch wrappers (defined in the .cu files).
// ---------------------------------------------------------------------------
struct DeviceInfo {
    int sms;
    int max_smem_optin;
    int cooperative;  // cooperative launches supported
};

// graph
cudaError_t launch_validate_graph(const uint64_t* row, const uint32_t* src, const float* w, uint32_t n,
                                  uint64_t m, int model, int* d_flags, cudaStream_t st);
cudaError_t launch_thresholds(const uint64_t* row, const float* w, uint32_t n, uint64_t m, int model,
                              uint32_t* thr, int* d_flags, cudaStream_t st);
cudaError_t launch_lt_guide(const uint64_t* row, const uint32_t* cthr, const uint32_t* src, uint32_t n, uint4* guide,
                            cudaStream_t st);

// sampling
uint32_t small_cap(int model);  // members a small-path set may hold (staging per set)
int ic_large_uses_smem(uint32_t n, const DeviceInfo& di);
cudaError_t launch_ic_small(const DevGraph& g, const SampleBatch& b, const DeviceInfo& di, cudaStream_t st);
cudaError_t launch_ic_large(const DevGraph& g, const SampleBatch& b, const LargeSlots& ls,
                            const DeviceInfo& di, cudaStream_t st);
cudaError_t launch_lt_small(const DevGraph& g, const SampleBatch& b, const MidSlots& ms, const DeviceInfo& di,
                            cudaStream_t st);
cudaError_t launch_lt_mid(const DevGraph& g, const SampleBatch& b, const MidSlots& ms, cudaStream_t st);
cudaError_t launch_lt_long(const DevGraph& g, const SampleBatch& b, const LargeSlots& ls,
                           const DeviceInfo& di, cudaStream_t st);
// Grouped IC large path: the large sets of a batch, 64 at a time, as one
// multi-source BFS over the whole GPU (cooperative launch), kGroupSlots
// groups in flight (slots of the arrays below).
constexpr uint32_t kGroupSets = 64;
constexpr uint32_t kGroupSlots = 8;  // groups in flight
struct GroupCounters {
    unsigned long long hpack[2];      // listed large vertices << 36 | their chunks, by level parity
    unsigned long long lpack[2];      // listed small vertices << 36 | their quads, by level parity
    uint32_t claim[3];                // work items claimed, by step mod 3 (zero between launches)
    uint32_t cnt[kGroupSets];         // members per set
    uint32_t edges[kGroupSets];       // in-edges of the members per set
    uint32_t kind[kGroupSets];        // 0 list, 1 bitmap, 2 reservation failed
    unsigned long long pos[kGroupSets];   // output position in the large-output buffer
    unsigned long long lcur[kGroupSets];  // list entries written
};
struct GroupScratch {
    unsigned long long* vis;  // [n] sets of the group that expanded v (zero between groups)
    unsigned long long* fn;   // [n] sets that reached v in the level being expanded (zero otherwise)
    uint4* lq;                // [n] small vertices of the level: (rs, re, F lo, F hi)
    uint32_t* lpre;           // [n] their offsets in the level's small quads
    uint32_t* wst;            // [wcap] first small entry of each 32-quad window
    uint32_t* hb;             // [hcap] first chunk of each large vertex of the level
    uint4* he;                // [hcap] large vertices: (rs, re, F lo, F hi)
    uint32_t* cown;           // [ccap] large-list entry owning each chunk of the level
    uint64_t stride;          // bytes from each slot's arrays to the next slot's
    GroupCounters* ctr;       // [kGroupSlots], one per slot (ctr[0].claim serves all)
    uint32_t wcap, hcap;      // entries of wst and of hb / he
    uint32_t ccap;            // entries of cown
    uint32_t lcap;            // entries of lq / lpre (n)
    unsigned long long* bounds;  // checked builds: the batch's error word
};
int ic_group_supported(const DeviceInfo& di);
uint64_t ic_group_heavy_cap(uint32_t n, uint64_t m);
cudaError_t launch_ic_group(const DevGraph& g, const SampleBatch& b, const GroupScratch& gs, const DeviceInfo& di,
                            cudaStream_t st);
// Scan of the kept sets: list offsets into off[], bitmap ranks, totals.
uint64_t scan_tmp_words(uint32_t count);
cudaError_t launch_batch_scan(const SampleBatch& b, const BatchOut& o, uint64_t* tmp, const DeviceInfo& di,
                              cudaStream_t st);
cudaError_t launch_compact(const SampleBatch& b, const BatchOut& o, uint64_t committed, uint32_t* seg_hist,
                           const DeviceInfo& di, cudaStream_t st);
cudaError_t launch_bitmap_store(const SampleBatch& b, const BatchOut& o, uint64_t nbitmaps, uint32_t n,
                                uint32_t* cnt, const DeviceInfo& di, cudaStream_t st);
// cnt[v] += number of bitmaps first .. first+count-1 holding v, skipping
// bitmaps whose set is flagged in skip[] (nullable)
cudaError_t launch_bitmap_count(const uint32_t* bmp, uint32_t words, uint32_t n, uint64_t first, uint64_t count,
                                const uint8_t* skip, const uint32_t* bmp_set, uint32_t* cnt, const DeviceInfo& di,
                                cudaStream_t st);
// voff = exclusive scan of hist; cnt[v] += hist[v] and cnt2[v] += hist[v]
// (each nullable); cursor zeroed
cudaError_t launch_vertex_scan(const uint32_t* hist, uint32_t n, uint64_t* voff, uint32_t* cnt, uint32_t* cnt2,
                               uint32_t* cursor, uint64_t* tmp, const DeviceInfo& di, cudaStream_t st);
cudaError_t launch_index_scatter(uint64_t set_begin, uint64_t set_end, const uint64_t* off, const uint32_t* arena,
                                 const uint64_t* voff, uint32_t* cursor, uint32_t* inv, uint64_t inv_cap,
                                 unsigned long long* err, const DeviceInfo& di, cudaStream_t st);

// selection
struct SelectState {
    uint32_t n;
    uint32_t words;
    uint64_t nsets;
    uint64_t total_members;   // all members (lists and bitmaps)
    uint64_t list_members;    // members of list-stored sets
    const uint64_t* off;
    const uint32_t* arena;
    const uint32_t* set_bmp;  // [nsets] bitmap id or kEmpty
    const uint32_t* bmp;      // bitmap arena
    const uint32_t* bmp_set;  // [nbmp]
    const uint32_t* bmp_len;  // [nbmp]
    uint32_t nbmp;
    uint32_t* work;      // n mutable counts
    uint8_t* picked;     // n
    uint8_t* covered;    // nsets
    uint32_t* newly;     // nsets: ids covered in the current round
    unsigned long long* keys;      // k: packed (count, ~v) argmax per round
    unsigned long long* newly_n;   // k: sets covered per round
    unsigned long long* vol_cov;   // k: members of the sets covered per round
    unsigned long long* vol_list;  // k: of which in list-stored sets
    unsigned long long* bmp_cov;   // k: bitmap sets covered per round
    uint32_t* ubmp;                // nbmp: uncovered bitmap ids gathered for a rebuild
    unsigned long long* ubmp_n;    // k: entries of ubmp gathered in round j
    uint32_t* seeds;     // k
    const DevSegment* segs;
    uint32_t nsegs;
    int force_mode;      // 0: decrement or recount chosen per round; 1: always decrement; 2: always recount
    uint32_t* cand;      // n (nullable): argmax candidates, the unpicked vertices with counts >= tau
    uint32_t* cstate;    // 4: candidates, tau, list valid, count of the last list that came out too long
    unsigned long long* bounds;  // 3: checked builds, first failed index check (where, index, bound)
};
cudaError_t launch_select_round(const SelectState& s, uint32_t j, const DeviceInfo& di, cudaStream_t st,
                                uint64_t* launches);
// counts of the stream's first `prefix` sets into work (zero on entry);
// list_end = off[prefix]; *members receives their total members
cudaError_t launch_prefix_count(const SelectState& s, uint64_t prefix, uint64_t list_end,
                                unsigned long long* members, const DeviceInfo& di, cudaStream_t st);
// all k rounds in one cooperative launch over the whole GPU (one instance)
cudaError_t launch_select_all(const SelectState& s, uint32_t k, const DeviceInfo& di, cudaStream_t st);
// all k rounds of many instances in one launch, one cluster of kClusterSel
// CTAs per instance (states and ks in device memory); cudaErrorCooperative-
// LaunchTooLarge if no cluster of that size fits the device
constexpr uint32_t kClusterSel = 8;
cudaError_t launch_select_clusters(const SelectState* d_states, const uint32_t* d_ks, uint32_t count,
                                   const DeviceInfo& di, cudaStream_t st);
// all k rounds of many instances in one launch, one CTA per instance
// (states and ks in device memory)
cudaError_t launch_select_batch(const SelectState* d_states, const uint32_t* d_ks, uint32_t count,
                                const DeviceInfo& di, cudaStream_t st);

// Seed-set coverage of a stored stream (k_opim.cu): sets [0, nsets) holding
// a vertex whose flag is nonzero (list-stored sets) or one of the k seeds
// (bitmap-stored sets); the count goes to *out.
struct CoverageArgs {
    uint64_t nsets;
    uint32_t words;
    uint32_t k;
    const uint64_t* off;
    const uint32_t* arena;
    const uint32_t* set_bmp;
    const uint32_t* bmp;
    const uint8_t* flag;      // [n] 1 for the seeds
    const uint32_t* seeds;    // [k]
    unsigned long long* out;
};
cudaError_t launch_coverage(const CoverageArgs& a, const DeviceInfo& di, cudaStream_t st);

}  // namespace imm
