// Greedy max-coverage seed selection (Find_Most_Influential_Set, EfficientIMM
// Alg. 2) over the RRR-set stream.  One round = five launches on the stream:
//
//   argmax        PARALLEL_REDUCTION (Sec. IV-A): max over vertices not yet
//                 picked of key = (count << 32) | (2^32 - 1 - v), so ties go to
//                 the lowest id; thread -> warp shuffle -> block -> atomicMax.
//   cover         every set holding the pick that is not yet covered is
//                 marked covered and appended to this round's list; its size
//                 is summed.  List-stored sets are found through the inverted
//                 index segments, bitmap-stored sets by one bit test each.
//   decrement     Alg. 2's update: one atomic decrement per member of each
//                 newly covered set ...
//   rebuild       ... or, when those members outnumber the members of the
//                 sets still uncovered, the counts are rebuilt from the
//                 uncovered sets (Sec. IV-C adaptive counter update).
// The decrement/rebuild choice is taken on the device from the round's
// volumes, so no host round trip is needed; both give the same counts.
#include <cooperative_groups.h>

#include "imm_internal.cuh"

namespace imm {

constexpr int kModeDecrement = 0;
constexpr int kModeRebuild = 1;

__device__ __forceinline__ uint64_t shfl64s(uint64_t x, int srcLane)
{
    const uint32_t lo = __shfl_sync(kFull, (uint32_t)x, srcLane);
    const uint32_t hi = __shfl_sync(kFull, (uint32_t)(x >> 32), srcLane);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t shfl64s_up(uint64_t x, int d)
{
    const uint32_t lo = __shfl_up_sync(kFull, (uint32_t)x, d);
    const uint32_t hi = __shfl_up_sync(kFull, (uint32_t)(x >> 32), d);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint32_t owner_lane(uint32_t j, uint32_t incl)
{
    uint32_t o = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const uint32_t c = __shfl_sync(kFull, incl, o + step - 1);
        if (c <= j) o += step;
    }
    return o;
}

// atomicAdd(&work[u], delta) for every member u of one set (arena[start ..
// start + len)), strided over the lanes of the calling warp with eight member
// loads in flight per lane: a set of a few hundred members costs one or two
// load round trips, not one per 32 members.
constexpr uint32_t kNoMember = 0xFFFFFFFFu;  // never a vertex id (n < 2^32)
__device__ __forceinline__ void warp_apply_one(const uint32_t* arena, uint64_t start, uint32_t len, uint32_t* work,
                                               uint32_t delta, uint32_t lane)
{
    for (uint32_t x0 = lane; x0 < len; x0 += 32u * 8u) {
        uint32_t m[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t x = x0 + 32u * u;
            m[u] = x < len ? __ldg(arena + start + x) : kNoMember;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (m[u] != kNoMember) atomicAdd(&work[m[u]], delta);
    }
}

// Every member u of the sets given by (start, len) per lane gets
// atomicAdd(&work[u], delta).  Warp-cooperative: sets of >= 32 members one at
// a time across the warp, shorter ones flattened across lanes (four member
// loads in flight per lane).
__device__ __forceinline__ void warp_apply_sets(const uint32_t* arena, uint64_t start, uint32_t len, uint32_t* work,
                                                uint32_t delta)
{
    const uint32_t lane = threadIdx.x & 31;
    const bool big = len >= 32;
    uint32_t bigmask = __ballot_sync(kFull, big);
    while (bigmask) {
        const int o = __ffs(bigmask) - 1;
        bigmask &= bigmask - 1;
        const uint32_t L = __shfl_sync(kFull, len, o);
        const uint64_t A = shfl64s(start, o);
        warp_apply_one(arena, A, L, work, delta, lane);
    }
    const uint32_t sl = big ? 0u : len;
    uint32_t incl = sl;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, d);
        if ((int)lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - sl;
    for (uint32_t j0 = 0; j0 < total; j0 += 32u * 4u) {
        uint32_t m[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t j = j0 + 32u * u + lane;
            const uint32_t o = owner_lane(j, incl);
            const uint64_t A = shfl64s(start, o);
            const uint32_t ex = __shfl_sync(kFull, excl, o);
            m[u] = j < total ? __ldg(arena + A + (j - ex)) : kNoMember;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (m[u] != kNoMember) atomicAdd(&work[m[u]], delta);
    }
}

// Decrement when the newly covered sets hold fewer members than a recount
// would read: vol_cov <= list members still uncovered afterwards + words/8 per
// uncovered bitmap + n/8 + sets/8.
__device__ int round_mode(const SelectState& s, uint32_t j)
{
    if (s.force_mode == 1) return kModeDecrement;
    if (s.force_mode == 2) return kModeRebuild;
    uint64_t before_list = 0, before_b = 0;
    for (uint32_t i = 0; i < j; ++i) {
        before_list += s.vol_list[i];
        before_b += s.bmp_cov[i];
    }
    const uint64_t cov = s.vol_cov[j];
    const uint64_t unc_list = s.list_members - before_list - s.vol_list[j];
    const uint64_t unc_bmp = (uint64_t)s.nbmp - before_b - s.bmp_cov[j];
    const uint64_t rebuild_cost = unc_list + unc_bmp * (s.words >> 3) + (s.n >> 3) + (s.nsets >> 3);
    return cov > rebuild_cost ? kModeRebuild : kModeDecrement;
}

__global__ void __launch_bounds__(256)
argmax_kernel(const uint32_t* work, const uint8_t* picked, uint32_t n, unsigned long long* out)
{
    __shared__ unsigned long long s_best[8];
    unsigned long long best = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (!picked[v]) {
            const unsigned long long key = ((unsigned long long)work[v] << 32) | (0xFFFFFFFFu - v);
            best = key > best ? key : best;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, best, d);
        best = o > best ? o : best;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_best[wid] = best;
    __syncthreads();
    if (wid == 0) {
        best = lane < (int)(blockDim.x >> 5) ? s_best[lane] : 0ull;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(kFull, best, d);
            best = o > best ? o : best;
        }
        if (lane == 0 && best) atomicMax(out, best);
    }
}

__global__ void __launch_bounds__(256)
cover_kernel(SelectState s, uint32_t j)
{
    const unsigned long long key = s.keys[j];
    const uint32_t v = 0xFFFFFFFFu - (uint32_t)key;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.picked[v] = 1;
        s.seeds[j] = v;
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long vol = 0, nb = 0;
    for (uint32_t g = 0; g < s.nsegs; ++g) {
        const uint64_t a = s.segs[g].voff[v], b = s.segs[g].voff[v + 1];
        const uint32_t* inv = s.segs[g].inv;
        for (uint64_t i = a + tid; i < b; i += stride) {
            const uint32_t sid = inv[i];
            // a set holds v at most once, so only this thread can see sid here
            if (!s.covered[sid]) {
                s.covered[sid] = 1;
                const unsigned long long p = atomicAdd(&s.newly_n[j], 1ull);
                if (IMM_IN_BOUNDS(p, s.nsets, s.bounds, kChkNewly)) s.newly[p] = sid;
                vol += s.off[(uint64_t)sid + 1] - s.off[sid];
            }
        }
    }
    if (vol) {
        atomicAdd(&s.vol_cov[j], vol);
        atomicAdd(&s.vol_list[j], vol);
    }
    vol = 0;
    const uint32_t wv = v >> 5, bit = 1u << (v & 31);
    for (uint64_t b = tid; b < s.nbmp; b += stride) {
        const uint32_t sid = s.bmp_set[b];
        if (!s.covered[sid] && (s.bmp[b * s.words + wv] & bit)) {
            s.covered[sid] = 1;
            const unsigned long long p = atomicAdd(&s.newly_n[j], 1ull);
            if (IMM_IN_BOUNDS(p, s.nsets, s.bounds, kChkNewly)) s.newly[p] = sid;
            vol += s.bmp_len[b];
            ++nb;
        }
    }
    if (vol) atomicAdd(&s.vol_cov[j], vol);
    if (nb) atomicAdd(&s.bmp_cov[j], nb);
}

__global__ void __launch_bounds__(256)
decrement_kernel(SelectState s, uint32_t j)
{
    __shared__ int s_mode;
    if (threadIdx.x == 0) s_mode = round_mode(s, j);
    __syncthreads();
    if (s_mode != kModeDecrement) return;
    const uint64_t cnt = s.newly_n[j];
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t first = gw * 32; first < cnt; first += nw * 32) {
        const uint64_t i = first + lane;
        uint64_t start = 0;
        uint32_t len = 0, bid = kEmpty;
        if (i < cnt) {
            const uint32_t sid = s.newly[i];
            start = s.off[sid];
            len = (uint32_t)(s.off[(uint64_t)sid + 1] - start);
            bid = s.set_bmp[sid];
        }
        warp_apply_sets(s.arena, start, len, s.work, 0xFFFFFFFFu);  // += -1
        // bitmap-stored sets: the warp walks the set bits of each one
        uint32_t bm = __ballot_sync(kFull, bid != kEmpty);
        while (bm) {
            const int o = __ffs(bm) - 1;
            bm &= bm - 1;
            const uint32_t B = __shfl_sync(kFull, bid, o);
            const uint32_t* row = s.bmp + (uint64_t)B * s.words;
            for (uint32_t w = lane; w < s.words; w += 32) {
                uint32_t x = row[w];
                while (x) {
                    const int t = __ffs(x) - 1;
                    x &= x - 1;
                    atomicAdd(&s.work[w * 32 + t], 0xFFFFFFFFu);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256)
rebuild_zero_kernel(SelectState s, uint32_t j)
{
    __shared__ int s_mode;
    if (threadIdx.x == 0) s_mode = round_mode(s, j);
    __syncthreads();
    if (s_mode != kModeRebuild) return;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < s.n; v += stride) s.work[v] = 0;
}

__global__ void __launch_bounds__(256)
rebuild_add_kernel(SelectState s, uint32_t j)
{
    __shared__ int s_mode;
    if (threadIdx.x == 0) s_mode = round_mode(s, j);
    __syncthreads();
    if (s_mode != kModeRebuild) return;
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t first = gw * 32; first < s.nsets; first += nw * 32) {
        const uint64_t sid = first + lane;
        uint64_t start = 0;
        uint32_t len = 0;
        if (sid < s.nsets && !s.covered[sid]) {
            start = s.off[sid];
            len = (uint32_t)(s.off[sid + 1] - start);
        }
        warp_apply_sets(s.arena, start, len, s.work, 1u);
    }
}

// Rebuild, bitmap-stored part: counts of the uncovered bitmap sets added by
// columns (each thread owns the 32 vertices of one bitmap word).
__global__ void __launch_bounds__(256)
rebuild_bitmap_kernel(SelectState s, uint32_t j, uint64_t per_chunk)
{
    __shared__ int s_mode;
    if (threadIdx.x == 0) s_mode = round_mode(s, j);
    __syncthreads();
    if (s_mode != kModeRebuild) return;
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t b0 = (uint64_t)blockIdx.y * per_chunk;
    uint64_t b1 = b0 + per_chunk;
    if (b1 > s.nbmp) b1 = s.nbmp;
    if (w >= s.words) return;
    uint32_t c[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) c[i] = 0;
    for (uint64_t b = b0; b < b1; ++b) {
        if (s.covered[s.bmp_set[b]]) continue;
        const uint32_t x = __ldg(s.bmp + b * s.words + w);
        if (!x) continue;
#pragma unroll
        for (int i = 0; i < 32; ++i) c[i] += (x >> i) & 1u;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const uint32_t v = w * 32 + i;
        if (c[i] && v < s.n) atomicAdd(&s.work[v], c[i]);
    }
}

// ===========================================================================
// Persistent selection: all k rounds in one launch.  The phases above become
// device functions run by a "team": the whole cooperative grid (one
// instance, imm_select) or one CTA (many instances per launch, batches).
// ===========================================================================
namespace cg = cooperative_groups;

struct GridTeam {
    __device__ __forceinline__ uint64_t rank() const { return (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ uint64_t size() const { return (uint64_t)gridDim.x * blockDim.x; }
    __device__ __forceinline__ void sync() const { cg::this_grid().sync(); }
};

struct BlockTeam {
    __device__ __forceinline__ uint64_t rank() const { return threadIdx.x; }
    __device__ __forceinline__ uint64_t size() const { return blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// A thread-block cluster (kClusterSel CTAs on as many SMs of one GPC) as the
// team of one instance: its barrier is the cluster's, with release/acquire
// semantics at cluster scope, far cheaper than a grid barrier.
struct ClusterTeam {
    __device__ __forceinline__ uint64_t rank() const
    {
        return (uint64_t)cg::this_cluster().block_rank() * blockDim.x + threadIdx.x;
    }
    __device__ __forceinline__ uint64_t size() const { return (uint64_t)cg::this_cluster().num_blocks() * blockDim.x; }
    __device__ __forceinline__ void sync() const { cg::this_cluster().sync(); }
};

// s_red: one slot per warp of the block; the block's best key goes to the
// round's key with one atomic (not one per warp: they all hit one address).
template <class Team>
__device__ void team_argmax(const SelectState& s, uint32_t j, Team t, unsigned long long* s_red)
{
    // Four vertices per load with 16-byte count loads (work is 256-byte
    // aligned), eight loads issued before any is used (the counts sit in L2:
    // the pass is bound by load latency and issue, not bandwidth).  A thread
    // meets its vertices in increasing order, so among equal counts the
    // first one it meets is the lowest id and a strict comparison keeps it:
    // (count, vertex) is packed into the round's key once per thread, not
    // per vertex.  bc holds count + 1 (0: no unpicked vertex met yet).
    constexpr int kU = 8;
    uint32_t bc = 0, bv = 0;
    const uint64_t n4 = s.n >> 2;
    const uint4* w4 = reinterpret_cast<const uint4*>(s.work);
    const uint32_t* p4 = reinterpret_cast<const uint32_t*>(s.picked);
    const uint64_t stride = t.size();
    for (uint64_t i0 = t.rank(); i0 < n4; i0 += kU * stride) {
        uint4 w[kU];
        uint32_t pk[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint64_t i = i0 + u * stride;
            w[u] = i < n4 ? w4[i] : make_uint4(0u, 0u, 0u, 0u);
            pk[u] = i < n4 ? p4[i] : 0x01010101u;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t v = (uint32_t)((i0 + u * stride) << 2);
            const uint32_t c[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
            if (pk[u] == 0u) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t cq = c[q] + 1u;
                    if (cq > bc) {
                        bc = cq;
                        bv = v + q;
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t cq = c[q] + 1u;
                    if (!((pk[u] >> (8 * q)) & 0xFFu) && cq > bc) {
                        bc = cq;
                        bv = v + q;
                    }
                }
            }
        }
    }
    for (uint64_t v = (n4 << 2) + t.rank(); v < s.n; v += t.size()) {
        const uint32_t cq = s.work[v] + 1u;
        if (!s.picked[v] && cq > bc) {
            bc = cq;
            bv = (uint32_t)v;
        }
    }
    unsigned long long best = bc ? ((unsigned long long)(bc - 1u) << 32) | (0xFFFFFFFFu - bv) : 0ull;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, best, d);
        best = o > best ? o : best;
    }
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane == 0) s_red[wid] = best;
    __syncthreads();
    if (wid == 0) {
        best = lane < nwarps ? s_red[lane] : 0ull;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(kFull, best, d);
            best = o > best ? o : best;
        }
        if (lane == 0 && best) atomicMax(&s.keys[j], best);
    }
}

// Argmax over the candidate list (same key and reduction as team_argmax).
// Counts never increase during a selection, so when every vertex left off
// the list held fewer than tau occurrences at the time it was built, the
// list's best key is the global one whenever its count is at least tau:
// every vertex holding that count is on the list, so the lowest id among
// them is the lowest overall.
template <class Team>
__device__ void team_argmax_cand(const SelectState& s, uint32_t j, Team t, unsigned long long* s_red)
{
    unsigned long long best = 0;
    const uint32_t nc = __ldcg(s.cstate);
    for (uint64_t i = t.rank(); i < nc; i += t.size()) {
        const uint32_t v = s.cand[i];
        if (!s.picked[v]) {
            const unsigned long long key = ((unsigned long long)s.work[v] << 32) | (0xFFFFFFFFu - v);
            best = key > best ? key : best;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, best, d);
        best = o > best ? o : best;
    }
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane == 0) s_red[wid] = best;
    __syncthreads();
    if (wid == 0) {
        best = lane < nwarps ? s_red[lane] : 0ull;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(kFull, best, d);
            best = o > best ? o : best;
        }
        if (lane == 0 && best) atomicMax(&s.keys[j], best);
    }
    __syncthreads();  // s_red is reused by the next reduction
}

// The candidate list: unpicked vertices with counts >= tau (one append
// atomic per warp).
template <class Team>
__device__ void team_build_cand(const SelectState& s, uint32_t tau, Team t)
{
    const uint64_t lane = threadIdx.x & 31;
    for (uint64_t v0 = t.rank() - lane; v0 < s.n; v0 += t.size()) {
        const uint64_t v = v0 + lane;
        const bool take = v < s.n && !s.picked[v] && s.work[v] >= tau;
        const uint32_t bal = __ballot_sync(kFull, take);
        if (!bal) continue;
        const int leader = __ffs(bal) - 1;
        uint32_t base = 0;
        if ((int)lane == leader) base = atomicAdd(s.cstate, (uint32_t)__popc(bal));
        base = __shfl_sync(kFull, base, leader);
        const uint64_t at = base + __popc(bal & ((1u << lane) - 1u));
        if (take && IMM_IN_BOUNDS(at, s.n, s.bounds, kChkCand)) s.cand[at] = (uint32_t)v;
    }
}

// Appends the set ids of a warp's `take` lanes to the round's newly covered
// list with one atomic per warp (the list's counter is a single address).
__device__ __forceinline__ void append_newly(const SelectState& s, uint32_t j, bool take, uint32_t sid)
{
    const uint32_t bal = __ballot_sync(kFull, take);
    if (!bal) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(bal) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&s.newly_n[j], (unsigned long long)__popc(bal));
    base = __shfl_sync(kFull, base, leader);
    const uint64_t at = base + __popc(bal & ((1u << lane) - 1u));
    if (take && IMM_IN_BOUNDS(at, s.nsets, s.bounds, kChkNewly)) s.newly[at] = sid;
}

template <class Team>
__device__ void team_cover(const SelectState& s, uint32_t j, Team t)
{
    const unsigned long long key = s.keys[j];
    const uint32_t v = 0xFFFFFFFFu - (uint32_t)key;
    if (t.rank() == 0) {
        s.picked[v] = 1;
        s.seeds[j] = v;
    }
    // warp-uniform loops (lane i of a warp takes element first + i), so the
    // appends can be aggregated per warp
    const uint64_t lane = threadIdx.x & 31;
    const uint64_t wfirst = t.rank() - lane, tsize = t.size();
    unsigned long long vol = 0, nb = 0;
    for (uint32_t g = 0; g < s.nsegs; ++g) {
        const uint64_t a = s.segs[g].voff[v], b = s.segs[g].voff[v + 1];
        const uint32_t* inv = s.segs[g].inv;
        for (uint64_t i0 = a + wfirst; i0 < b; i0 += tsize) {
            const uint64_t i = i0 + lane;
            bool take = false;
            uint32_t sid = 0;
            if (i < b) {
                sid = inv[i];
                if (!s.covered[sid]) {
                    s.covered[sid] = 1;
                    take = true;
                    vol += s.off[(uint64_t)sid + 1] - s.off[sid];
                }
            }
            append_newly(s, j, take, sid);
        }
    }
    if (vol) {
        atomicAdd(&s.vol_cov[j], vol);
        atomicAdd(&s.vol_list[j], vol);
    }
    vol = 0;
    const uint32_t wv = v >> 5, bit = 1u << (v & 31);
    for (uint64_t b0 = wfirst; b0 < s.nbmp; b0 += tsize) {
        const uint64_t b = b0 + lane;
        bool take = false;
        uint32_t sid = 0;
        if (b < s.nbmp) {
            sid = s.bmp_set[b];
            if (!s.covered[sid] && (s.bmp[b * s.words + wv] & bit)) {
                s.covered[sid] = 1;
                take = true;
                vol += s.bmp_len[b];
                ++nb;
            }
        }
        append_newly(s, j, take, sid);
    }
    if (vol) atomicAdd(&s.vol_cov[j], vol);
    if (nb) atomicAdd(&s.bmp_cov[j], nb);
}

// Shared memory of a selection block: the argmax reduction, the round's
// update mode, and the picked vertex's ranges in every index segment.
constexpr uint32_t kSegTab = 64;
struct SelShared {
    unsigned long long red[32];
    uint64_t seg_a[kSegTab];    // first entry of the pick's list in segment g
    uint64_t seg_end[kSegTab];  // end of segment g's part of the flattened lists
    const uint32_t* seg_inv[kSegTab];   // the segments, loaded once per selection
    const uint64_t* seg_voff[kSegTab];
    int mode;
};

// Set id at position f of the pick's flattened lists; g is the segment of
// the caller's previous (smaller) position.
__device__ __forceinline__ uint32_t flat_set(const SelShared* sh, uint64_t f, uint32_t& g)
{
    while (f >= sh->seg_end[g]) ++g;
    const uint64_t first = g ? sh->seg_end[g - 1] : 0;
    return sh->seg_inv[g][sh->seg_a[g] + (f - first)];
}

// Streams without bitmap-stored sets (small sets: decrementing is always the
// cheaper update): cover and decrement in one pass, so a round needs one grid
// barrier less; counts are identical to cover-then-decrement.  The picked
// vertex's lists in all index segments are read as one flattened range,
// their bounds loaded once per block, so no thread walks the segments one
// after another.  A range with few entries per warp of the team goes one
// entry per warp (the set's members strided over the lanes), so the round's
// covered sets spread over all warps; a long one goes 32 entries per warp
// with the members of those sets flattened across the lanes.
template <class Team>
__device__ void team_cover_decrement(const SelectState& s, uint32_t j, Team t, SelShared* sh)
{
    const unsigned long long key = s.keys[j];
    const uint32_t v = 0xFFFFFFFFu - (uint32_t)key;
    if (t.rank() == 0) {
        s.picked[v] = 1;
        s.seeds[j] = v;
    }
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t gw = t.rank() >> 5, nw = t.size() >> 5;
    unsigned long long vol = 0, nnew = 0;
    if (s.nsegs <= kSegTab) {
        if (threadIdx.x < 32) {
            uint64_t a[2] = {0, 0}, len[2] = {0, 0};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t g = lane + 32u * h;
                if (g < s.nsegs) {
                    const uint64_t* voff = sh->seg_voff[g];
                    a[h] = voff[v];
                    len[h] = voff[v + 1] - a[h];
                }
            }
            uint64_t run = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint64_t incl = len[h];
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint64_t o = shfl64s_up(incl, d);
                    if ((int)lane >= d) incl += o;
                }
                const uint32_t g = lane + 32u * h;
                sh->seg_a[g] = a[h];
                sh->seg_end[g] = run + incl;  // past nsegs: the total
                run += shfl64s(incl, 31);
            }
        }
        __syncthreads();
        const uint64_t total = sh->seg_end[kSegTab - 1];
        uint32_t g = 0;
        if (total <= 4 * nw) {
            for (uint64_t f = gw; f < total; f += nw) {
                uint32_t take = 0;
                uint64_t start = 0;
                uint32_t len = 0;
                if (lane == 0) {
                    // the set's covered flag and extent are read together
                    const uint32_t sid = flat_set(sh, f, g);
                    const uint8_t cv = s.covered[sid];
                    const uint64_t o0 = __ldg(s.off + sid), o1 = __ldg(s.off + (uint64_t)sid + 1);
                    if (!cv) {
                        s.covered[sid] = 1;
                        take = 1;
                        start = o0;
                        len = (uint32_t)(o1 - o0);
                    }
                }
                take = __shfl_sync(kFull, take, 0);
                if (!take) continue;
                start = shfl64s(start, 0);
                len = __shfl_sync(kFull, len, 0);
                warp_apply_one(s.arena, start, len, s.work, 0xFFFFFFFFu, lane);
                if (lane == 0) {
                    vol += len;
                    ++nnew;
                }
            }
        } else {
            for (uint64_t f0 = gw * 32; f0 < total; f0 += nw * 32) {
                const uint64_t f = f0 + lane;
                uint64_t start = 0;
                uint32_t len = 0;
                bool take = false;
                if (f < total) {
                    const uint32_t sid = flat_set(sh, f, g);
                    const uint8_t cv = s.covered[sid];
                    const uint64_t o0 = __ldg(s.off + sid), o1 = __ldg(s.off + (uint64_t)sid + 1);
                    if (!cv) {
                        s.covered[sid] = 1;
                        take = true;
                        start = o0;
                        len = (uint32_t)(o1 - o0);
                        vol += len;
                        ++nnew;
                    }
                }
                if (__any_sync(kFull, take)) warp_apply_sets(s.arena, start, len, s.work, 0xFFFFFFFFu);
            }
        }
    }
    for (uint32_t g = 0; s.nsegs > kSegTab && g < s.nsegs; ++g) {
        const uint64_t a = s.segs[g].voff[v], b = s.segs[g].voff[v + 1];
        const uint32_t* inv = s.segs[g].inv;
        if (b - a <= 4 * nw) {
            for (uint64_t i = a + gw; i < b; i += nw) {
                uint32_t take = 0;
                uint64_t start = 0;
                uint32_t len = 0;
                if (lane == 0) {
                    const uint32_t sid = inv[i];
                    if (!s.covered[sid]) {
                        s.covered[sid] = 1;
                        take = 1;
                        start = s.off[sid];
                        len = (uint32_t)(s.off[(uint64_t)sid + 1] - start);
                    }
                }
                take = __shfl_sync(kFull, take, 0);
                if (!take) continue;
                start = shfl64s(start, 0);
                len = __shfl_sync(kFull, len, 0);
                warp_apply_one(s.arena, start, len, s.work, 0xFFFFFFFFu, lane);
                if (lane == 0) {
                    vol += len;
                    ++nnew;
                }
            }
        } else {
            for (uint64_t i0 = a + gw * 32; i0 < b; i0 += nw * 32) {
                const uint64_t i = i0 + lane;
                uint64_t start = 0;
                uint32_t len = 0;
                bool take = false;
                if (i < b) {
                    const uint32_t sid = inv[i];
                    if (!s.covered[sid]) {
                        s.covered[sid] = 1;
                        take = true;
                        start = s.off[sid];
                        len = (uint32_t)(s.off[(uint64_t)sid + 1] - start);
                        vol += len;
                        ++nnew;
                    }
                }
                if (__any_sync(kFull, take)) warp_apply_sets(s.arena, start, len, s.work, 0xFFFFFFFFu);
            }
        }
    }
    if (nnew) atomicAdd(&s.newly_n[j], nnew);
    if (vol) {
        atomicAdd(&s.vol_cov[j], vol);
        atomicAdd(&s.vol_list[j], vol);
    }
}

template <class Team>
__device__ void team_decrement(const SelectState& s, uint32_t j, Team t)
{
    const uint64_t cnt = s.newly_n[j];
    const int lane = threadIdx.x & 31;
    const uint64_t gw = t.rank() >> 5, nw = t.size() >> 5;
    for (uint64_t first = gw * 32; first < cnt; first += nw * 32) {
        const uint64_t i = first + lane;
        uint64_t start = 0;
        uint32_t len = 0, bid = kEmpty;
        if (i < cnt) {
            const uint32_t sid = s.newly[i];
            start = s.off[sid];
            len = (uint32_t)(s.off[(uint64_t)sid + 1] - start);
            bid = s.set_bmp[sid];
        }
        warp_apply_sets(s.arena, start, len, s.work, 0xFFFFFFFFu);
        uint32_t bm = __ballot_sync(kFull, bid != kEmpty);
        while (bm) {
            const int o = __ffs(bm) - 1;
            bm &= bm - 1;
            const uint32_t B = __shfl_sync(kFull, bid, o);
            const uint32_t* row = s.bmp + (uint64_t)B * s.words;
            for (uint32_t w = lane; w < s.words; w += 32) {
                uint32_t x = row[w];
                while (x) {
                    const int tt = __ffs(x) - 1;
                    x &= x - 1;
                    atomicAdd(&s.work[w * 32 + tt], 0xFFFFFFFFu);
                }
            }
        }
    }
}

template <class Team>
__device__ void team_rebuild_add(const SelectState& s, Team t)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = t.rank() >> 5, nw = t.size() >> 5;
    for (uint64_t first = gw * 32; first < s.nsets; first += nw * 32) {
        const uint64_t sid = first + lane;
        uint64_t start = 0;
        uint32_t len = 0;
        if (sid < s.nsets && !s.covered[sid]) {
            start = s.off[sid];
            len = (uint32_t)(s.off[sid + 1] - start);
        }
        warp_apply_sets(s.arena, start, len, s.work, 1u);
    }
}

// Rebuild, bitmap part: gather the uncovered bitmaps of round j into ubmp,
// then add them by columns (items = (word, chunk of gathered bitmaps)).
template <class Team>
__device__ void team_gather_uncovered(const SelectState& s, uint32_t j, Team t)
{
    // warp-uniform loop with one append atomic per warp
    const uint64_t lane = threadIdx.x & 31;
    for (uint64_t b0 = t.rank() - lane; b0 < s.nbmp; b0 += t.size()) {
        const uint64_t b = b0 + lane;
        const bool take = b < s.nbmp && !s.covered[s.bmp_set[b]];
        const uint32_t bal = __ballot_sync(kFull, take);
        if (!bal) continue;
        const int leader = __ffs(bal) - 1;
        unsigned long long base = 0;
        if ((int)lane == leader) base = atomicAdd(&s.ubmp_n[j], (unsigned long long)__popc(bal));
        base = __shfl_sync(kFull, base, leader);
        const uint64_t at = base + __popc(bal & ((1u << lane) - 1u));
        if (take && IMM_IN_BOUNDS(at, s.nbmp, s.bounds, kChkUbmp)) s.ubmp[at] = (uint32_t)b;
    }
}

template <class Team>
__device__ void team_count_uncovered(const SelectState& s, uint32_t j, Team t)
{
    const uint64_t nb = s.ubmp_n[j];
    if (nb == 0) return;
    uint64_t chunks = t.size() / s.words;
    if (chunks == 0) chunks = 1;
    if (chunks > nb) chunks = nb;
    const uint64_t per = (nb + chunks - 1) / chunks;
    const uint64_t items = (uint64_t)s.words * chunks;
    for (uint64_t it = t.rank(); it < items; it += t.size()) {
        const uint32_t w = (uint32_t)(it % s.words);
        const uint64_t b0 = (it / s.words) * per;
        const uint64_t b1 = b0 + per < nb ? b0 + per : nb;
        uint32_t c[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) c[i] = 0;
        for (uint64_t bi = b0; bi < b1; ++bi) {
            const uint32_t x = s.bmp[(uint64_t)s.ubmp[bi] * s.words + w];
            if (!x) continue;
#pragma unroll
            for (int i = 0; i < 32; ++i) c[i] += (x >> i) & 1u;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const uint32_t v = w * 32 + i;
            if (c[i] && v < s.n) atomicAdd(&s.work[v], c[i]);
        }
    }
}

// The argmax of a round scans the candidate list when one is valid and its
// best count reaches tau; otherwise all n vertices, and the list is rebuilt
// with tau = a quarter of that round's best count.  A list longer than n/8
// is dropped (scanning it would cost about as much as the full pass), and no
// new one is built until the best count has halved since.  The picks are
// those of the full scan in every round.
template <class Team>
__device__ void team_pick(const SelectState& s, uint32_t j, Team t, unsigned long long* s_red)
{
    if (s.cand && __ldcg(s.cstate + 2)) {
        team_argmax_cand(s, j, t, s_red);
        t.sync();
        const unsigned long long key = __ldcg(&s.keys[j]);
        if (key != 0ull && (uint32_t)(key >> 32) >= __ldcg(s.cstate + 1)) return;
        t.sync();  // every thread has read the key before it is reset
        if (t.rank() == 0) {
            s.keys[j] = 0ull;
            s.cstate[2] = 0u;
        }
        t.sync();
    }
    team_argmax(s, j, t, s_red);
    t.sync();
    if (!s.cand) return;
    const uint32_t best = (uint32_t)(__ldcg(&s.keys[j]) >> 32);
    const uint32_t last_long = __ldcg(s.cstate + 3);
    if (best == 0u || (last_long && best > last_long / 2)) return;
    const uint32_t tau = best >> 2 ? best >> 2 : 1u;
    if (t.rank() == 0) {
        s.cstate[0] = 0u;
        s.cstate[1] = tau;
    }
    t.sync();
    team_build_cand(s, tau, t);
    t.sync();
    if (t.rank() == 0) {
        const uint32_t nc = s.cstate[0];
        const bool keep = (uint64_t)nc * 8 <= s.n;
        s.cstate[2] = keep ? 1u : 0u;
        s.cstate[3] = keep ? 0u : best;
    }
    t.sync();
}

template <class Team>
__device__ void select_rounds(const SelectState& s, uint32_t k, Team t, SelShared* sh)
{
    int* s_mode = &sh->mode;
    if (s.nsegs <= kSegTab && threadIdx.x < s.nsegs) {
        const DevSegment sg = s.segs[threadIdx.x];
        sh->seg_voff[threadIdx.x] = sg.voff;
        sh->seg_inv[threadIdx.x] = sg.inv;
    }
    __syncthreads();
    for (uint32_t j = 0; j < k; ++j) {
        team_pick(s, j, t, sh->red);
        if (s.nbmp == 0 && s.force_mode != 2) {
            team_cover_decrement(s, j, t, sh);
            t.sync();
            continue;
        }
        team_cover(s, j, t);
        t.sync();
        if (threadIdx.x == 0) *s_mode = round_mode(s, j);
        __syncthreads();
        if (*s_mode == kModeDecrement) {
            team_decrement(s, j, t);
        } else {
            for (uint64_t v = t.rank(); v < s.n; v += t.size()) s.work[v] = 0;
            if (s.nbmp) team_gather_uncovered(s, j, t);
            t.sync();
            team_rebuild_add(s, t);
            if (s.nbmp) team_count_uncovered(s, j, t);
        }
        t.sync();
    }
}

// One 1024-thread CTA per SM: half the CTAs of two 512-thread ones, so each
// grid barrier gathers half the arrivals.
constexpr int kCoopThreads = 1024;

__global__ void __launch_bounds__(kCoopThreads, 1)
select_coop_kernel(SelectState s, uint32_t k)
{
    __shared__ SelShared sh;
    select_rounds(s, k, GridTeam{}, &sh);
}

__global__ void __launch_bounds__(512, 1)
select_cta_kernel(const SelectState* states, const uint32_t* ks, uint32_t count)
{
    __shared__ SelShared sh;
    for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
        select_rounds(states[i], ks[i], BlockTeam{}, &sh);
        __syncthreads();
    }
}

// Counts of the first `prefix` sets of the stream (a selection over a prefix
// of a longer resident stream sees only those sets): list-stored sets of ids
// below the prefix occupy arena[0, off[prefix]); bitmap-stored ones are
// those with bmp_set[b] < prefix, one block per (bitmap, chunk of words).
// work must be zero on entry; *members receives the prefix's total members.
__global__ void __launch_bounds__(256)
prefix_list_count_kernel(const uint32_t* arena, uint64_t end, uint32_t* work, unsigned long long* members)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end; i += stride)
        atomicAdd(&work[arena[i]], 1u);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(members, (unsigned long long)end);
}

__global__ void __launch_bounds__(256)
prefix_bitmap_count_kernel(SelectState s, uint64_t prefix, unsigned long long* members)
{
    const uint32_t b = blockIdx.y;
    if (b >= s.nbmp || s.bmp_set[b] >= prefix) return;
    const uint32_t* row = s.bmp + (uint64_t)b * s.words;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < s.words; w += gridDim.x * blockDim.x) {
        uint32_t x = row[w];
        while (x) {
            const int t = __ffs(x) - 1;
            x &= x - 1;
            atomicAdd(&s.work[w * 32 + t], 1u);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(members, (unsigned long long)s.bmp_len[b]);
}

cudaError_t launch_prefix_count(const SelectState& s, uint64_t prefix, uint64_t list_end,
                                unsigned long long* members, const DeviceInfo& di, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(members, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    uint64_t blocks = (list_end + 255) / 256;
    if (blocks > (uint64_t)di.sms * 8) blocks = (uint64_t)di.sms * 8;
    if (blocks == 0) blocks = 1;
    prefix_list_count_kernel<<<(unsigned)blocks, 256, 0, st>>>(s.arena, list_end, s.work, members);
    if (s.nbmp) {
        const uint32_t bx = (s.words + 255 * 8) / (256 * 8) + 1;
        for (uint32_t b0 = 0; b0 < s.nbmp; b0 += 65535) {
            SelectState sc = s;
            sc.bmp_set += b0;
            sc.bmp += (uint64_t)b0 * s.words;
            sc.bmp_len += b0;
            sc.nbmp = s.nbmp - b0 < 65535 ? s.nbmp - b0 : 65535;
            prefix_bitmap_count_kernel<<<dim3(bx, sc.nbmp), 256, 0, st>>>(sc, prefix, members);
        }
    }
    return cudaGetLastError();
}

// All k rounds of many instances in one launch, one cluster per instance.
__global__ void __launch_bounds__(512, 1)
select_cluster_kernel(const SelectState* states, const uint32_t* ks, uint32_t count)
{
    __shared__ SelShared sh;
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t nb = cl.num_blocks();
    const uint32_t cid = blockIdx.x / nb, ncl = gridDim.x / nb;
    for (uint32_t i = cid; i < count; i += ncl) {
        select_rounds(states[i], ks[i], ClusterTeam{}, &sh);
        cl.sync();
    }
}

cudaError_t launch_select_clusters(const SelectState* d_states, const uint32_t* d_ks, uint32_t count,
                                   const DeviceInfo& di, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterSel;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(kClusterSel);
    int fit = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&fit, select_cluster_kernel, &cfg);
    if (e != cudaSuccess) return e;
    if (fit < 1) return cudaErrorCooperativeLaunchTooLarge;
    const uint32_t ncl = count < (uint32_t)fit ? count : (uint32_t)fit;
    cfg.gridDim = dim3(ncl * kClusterSel);
    return cudaLaunchKernelEx(&cfg, select_cluster_kernel, d_states, d_ks, count);
}

cudaError_t launch_select_all(const SelectState& s, uint32_t k, const DeviceInfo& di, cudaStream_t st)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_coop_kernel, kCoopThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    unsigned grid = (unsigned)di.sms;
    SelectState sc = s;
    uint32_t kk = k;
    void* args[] = {&sc, &kk};
    return cudaLaunchCooperativeKernel((void*)select_coop_kernel, dim3(grid), dim3(kCoopThreads), args, 0, st);
}

cudaError_t launch_select_batch(const SelectState* d_states, const uint32_t* d_ks, uint32_t count,
                                const DeviceInfo& di, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    select_cta_kernel<<<count, 512, 0, st>>>(d_states, d_ks, count);
    return cudaGetLastError();
}

cudaError_t launch_select_round(const SelectState& s, uint32_t j, const DeviceInfo& di, cudaStream_t st,
                                uint64_t* launches)
{
    const uint32_t sms = (uint32_t)di.sms;
    uint32_t ab = (s.n + 255) / 256;
    if (ab > sms * 4) ab = sms * 4;
    argmax_kernel<<<ab, 256, 0, st>>>(s.work, s.picked, s.n, s.keys + j);
    cover_kernel<<<sms * 2, 256, 0, st>>>(s, j);
    decrement_kernel<<<sms * 8, 256, 0, st>>>(s, j);
    uint32_t zb = (s.n + 255) / 256;
    if (zb > sms * 4) zb = sms * 4;
    rebuild_zero_kernel<<<zb, 256, 0, st>>>(s, j);
    uint64_t rb = (s.nsets + 255) / 256;
    if (rb > sms * 8) rb = sms * 8;
    if (rb == 0) rb = 1;
    rebuild_add_kernel<<<(unsigned)rb, 256, 0, st>>>(s, j);
    int n = 5;
    if (s.nbmp) {
        const uint32_t bx = (s.words + 255) / 256;
        uint64_t chunks = ((uint64_t)sms * 8 + bx - 1) / bx;
        if (chunks > s.nbmp) chunks = s.nbmp;
        if (chunks > 65535) chunks = 65535;
        const uint64_t per = (s.nbmp + chunks - 1) / chunks;
        chunks = (s.nbmp + per - 1) / per;
        rebuild_bitmap_kernel<<<dim3(bx, (unsigned)chunks), 256, 0, st>>>(s, j, per);
        ++n;
    }
    if (launches) *launches += n;
    return cudaGetLastError();
}

}  // namespace imm
