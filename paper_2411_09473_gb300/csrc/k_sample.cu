// RRR-set sampling kernels (Generate_RRRsets, EfficientIMM Alg. 3) and the
// storage of the sampled sets.
//
// A batch of consecutive set ids is sampled in two passes:
//   small path  one warp per set (IC) or one lane per walk (LT); the visited
//               state lives in shared memory (open-addressing hash / path
//               list).  A set that outgrows it is handed to the large path.
//   large path  one CTA per set (IC): level-synchronous BFS whose warps claim
//               32-vertex chunks of the frontier; vertices with >= 32 in-edge
//               quads are swept by the whole warp, the rest are flattened
//               across lanes.  The n-bit visited bitmap sits in shared memory
//               when it fits, else in a per-CTA global slot.  LT long walks
//               run one per thread with a global bitmap.
// Storage follows the adaptive representation of Sec. IV-C: a set is kept
// as a member list unless its list would be larger than an n-bit bitmap, in
// which case the bitmap is kept (O(1) membership tests during selection).
// The batch scan turns list lengths into arena offsets (prefix-sum
// compaction); the compaction kernel copies lists into the arena in set-id
// order while counting occurrences, and bitmap sets are counted by a
// column-popcount kernel (Alg. 3's fused count).
#include "imm_internal.cuh"

namespace imm {

__device__ __forceinline__ uint64_t shfl64(uint64_t x, int srcLane)
{
    const uint32_t lo = __shfl_sync(kFull, (uint32_t)x, srcLane);
    const uint32_t hi = __shfl_sync(kFull, (uint32_t)(x >> 32), srcLane);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t shfl64_up(uint64_t x, int d)
{
    const uint32_t lo = __shfl_up_sync(kFull, (uint32_t)x, d);
    const uint32_t hi = __shfl_up_sync(kFull, (uint32_t)(x >> 32), d);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint4 load_thr4(const uint32_t* thr, uint32_t quad)
{
    return __ldg(reinterpret_cast<const uint4*>(thr) + quad);
}

// in-edge range of v (m < 2^32, so the offsets fit 32 bits)
__device__ __forceinline__ void edge_range(const DevGraph& g, uint32_t v, uint32_t& rs, uint32_t& re)
{
    rs = (uint32_t)__ldg(g.row + v);
    re = (uint32_t)__ldg(g.row + v + 1);
}

__device__ __forceinline__ uint32_t quads_of(uint32_t rs, uint32_t re)
{
    return re > rs ? ((re - 1) >> 2) - (rs >> 2) + 1 : 0u;
}

// IC coins of the four in-edges of `quad` for set (s_hi, s_lo), restricted
// to [rs, re): bit t is set iff edge 4*quad + t is live.
__device__ __forceinline__ uint32_t live_mask(uint4 w, uint4 th, uint32_t quad, uint32_t rs, uint32_t re)
{
    uint32_t live = ((w.x >> 8) < th.x ? 1u : 0u) | ((w.y >> 8) < th.y ? 2u : 0u) |
                    ((w.z >> 8) < th.z ? 4u : 0u) | ((w.w >> 8) < th.w ? 8u : 0u);
    const uint32_t e0 = quad << 2;
    if (e0 < rs) live &= 0xFu << (rs - e0);
    if (e0 + 4 > re) live &= 0xFu >> (e0 + 4 - re);
    return live & 0xFu;
}

// Reserve space in the small-set staging.  Its capacity is sized from the
// running mean set size; a set that does not fit is marked failed and, with
// every later set of the batch, resampled by the next batch.
__device__ __forceinline__ bool reserve_small(const SampleBatch& b, uint32_t rel, uint32_t len, uint64_t* pos)
{
    const unsigned long long p = atomicAdd(&b.sc->stage_cursor, (unsigned long long)len);
    if (p + len > b.stage_cap) {
        b.set_len[rel] = kLenFailed;
        atomicMin(&b.sc->first_fail, rel);
        return false;
    }
    *pos = p;
    b.set_pos[rel] = p;
    b.set_len[rel] = len;
    b.set_kind[rel] = 0;
    return true;
}

// ===========================================================================
// IC, small path: one warp per set.
// ===========================================================================
constexpr int kSmallWarps = 6;               // 7 KB of shared memory per warp
constexpr uint32_t kSmallCap = 512;          // members a warp keeps before handing off
constexpr int kSmallHashBits = 10;
constexpr uint32_t kSmallHash = 1u << kSmallHashBits;  // > kSmallCap + 4*32 (one inner step)

constexpr uint32_t kLtCap = 160;              // path length a lane keeps before handing off
                                              // (its revisit test scans the path: a few hundred
                                              // compares cost less than a step's memory reads)

uint32_t small_cap(int model)
{
    return model == 0 ? kSmallCap : kLtCap;
}

__device__ __forceinline__ uint32_t small_slot(uint32_t v)
{
    return (v * 0x9E3779B1u) >> (32 - kSmallHashBits);
}

__global__ void __launch_bounds__(kSmallWarps * 32)
ic_small_kernel(DevGraph g, SampleBatch b)
{
    __shared__ uint32_t sh_list[kSmallWarps][kSmallCap];
    __shared__ uint16_t sh_slot[kSmallWarps][kSmallCap];
    __shared__ uint32_t sh_hash[kSmallWarps][kSmallHash];
    const int wid = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    uint32_t* list = sh_list[wid];
    uint16_t* lslot = sh_slot[wid];
    uint32_t* hash = sh_hash[wid];
    const uint32_t ltm = lanemask_lt();

    for (uint32_t i = lane; i < kSmallHash; i += 32) hash[i] = kEmpty;
    __syncwarp();

    for (;;) {
        uint32_t rel = 0;
        if (lane == 0) rel = atomicAdd(&b.sc->cursor, 1u);
        rel = __shfl_sync(kFull, rel, 0);
        if (rel >= b.count) break;
        const uint64_t s = b.base + rel;
        const PhiloxSet ps = philox_set((uint32_t)s, (uint32_t)(s >> 32), kTagIC, b.rk);
        if (lane == 0) {
            const uint32_t root = draw_root(b.rk, s, g.n);
            const uint32_t sl = small_slot(root);
            hash[sl] = root;
            list[0] = root;
            lslot[0] = (uint16_t)sl;
        }
        __syncwarp();

        uint32_t head = 0, tail = 1;
        uint32_t edges = 0;  // lane-partial sum of in-degrees of expanded members
        bool overflow = false;
        while (head < tail && !overflow) {
            // Up to 32 frontier vertices; their in-edge quads are flattened
            // across the warp so short and long adjacency lists share lanes.
            const uint32_t nf = min(tail - head, 32u);
            uint32_t rs = 0, re = 0, nq = 0;
            if ((uint32_t)lane < nf) {
                edge_range(g, list[head + lane], rs, re);
                nq = quads_of(rs, re);
                edges += re - rs;
            }
            uint32_t incl = nq;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, incl, d);
                if (lane >= d) incl += t;
            }
            const uint32_t total = __shfl_sync(kFull, incl, 31);
            const uint32_t excl = incl - nq;

            for (uint32_t j0 = 0; j0 < total && !overflow; j0 += 32) {
                const uint32_t j = j0 + lane;
                // owner lane: number of lanes whose inclusive prefix is <= j
                uint32_t o = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t c = __shfl_sync(kFull, incl, o + step - 1);
                    if (c <= j) o += step;
                }
                const uint32_t ors = __shfl_sync(kFull, rs, o);
                const uint32_t ore = __shfl_sync(kFull, re, o);
                const uint32_t oex = __shfl_sync(kFull, excl, o);
                uint32_t live = 0, quad = 0;
                if (j < total) {
                    quad = (ors >> 2) + (j - oex);
                    const uint4 th = load_thr4(g.thr, quad);
                    const uint4 w = philox_x(quad, ps, b.rk);
                    live = live_mask(w, th, quad, ors, ore);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    bool isnew = false;
                    uint32_t u = 0, sl = 0;
                    if ((live >> t) & 1u) {
                        u = __ldg(g.src + (quad << 2) + t);
                        sl = small_slot(u);
                        uint32_t probe = 0;
                        for (; probe < kSmallHash; ++probe) {
                            const uint32_t prev = atomicCAS(&hash[sl], kEmpty, u);
                            if (prev == kEmpty) {
                                isnew = true;
                                break;
                            }
                            if (prev == u) break;
                            sl = (sl + 1) & (kSmallHash - 1);
                        }
                        if (probe == kSmallHash) atomicOr(&b.sc->error, kErrHashProbe);
                    }
                    const uint32_t nm = __ballot_sync(kFull, isnew);
                    if (isnew) {
                        const uint32_t pos = tail + __popc(nm & ltm);
                        if (pos < kSmallCap) {
                            list[pos] = u;
                            lslot[pos] = (uint16_t)sl;
                        }
                    }
                    tail += __popc(nm);
                }
                if (tail > kSmallCap) overflow = true;
                __syncwarp();
            }
            head += nf;
            __syncwarp();
        }

        if (overflow) {
            if (lane == 0) {
                const uint32_t qi = atomicAdd(&b.sc->large_count, 1u);
                if (IMM_IN_BOUNDS(qi, b.count, b.sc->bounds, kChkLargeQ)) b.large_q[qi] = rel;
                b.set_len[rel] = kLenPending;
            }
            for (uint32_t i = lane; i < kSmallHash; i += 32) hash[i] = kEmpty;
        } else {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) edges += __shfl_xor_sync(kFull, edges, d);
            uint64_t pos = 0;
            int ok = 0;
            if (lane == 0) {
                b.set_edges[rel] = edges;
                ok = reserve_small(b, rel, tail, &pos) ? 1 : 0;
            }
            ok = __shfl_sync(kFull, ok, 0);
            pos = shfl64(pos, 0);
            if (ok)
                for (uint32_t i = lane; i < tail; i += 32)
                    if (IMM_IN_BOUNDS(pos + i, b.stage_cap, b.sc->bounds, kChkStage)) b.stage[pos + i] = list[i];
            for (uint32_t i = lane; i < tail; i += 32) hash[lslot[i]] = kEmpty;
        }
        __syncwarp();
    }
}

cudaError_t launch_ic_small(const DevGraph& g, const SampleBatch& b, const DeviceInfo& di, cudaStream_t st)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ic_small_kernel, kSmallWarps * 32, 0);
    if (e != cudaSuccess) return e;
    const uint64_t want = ((uint64_t)b.count + kSmallWarps - 1) / kSmallWarps;
    uint64_t grid = (uint64_t)di.sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    if (grid > want) grid = want;
    if (grid == 0) grid = 1;
    ic_small_kernel<<<(unsigned)grid, kSmallWarps * 32, 0, st>>>(g, b);
    return cudaGetLastError();
}

// ===========================================================================
// IC, large path: one CTA per set, level-synchronous BFS.
// ===========================================================================
constexpr int kLargeThreads = 1024;

// Test-and-set of u in the visited bitmap; appends u to the member queue when
// it was not yet visited.  Bits only ever go from 0 to 1, so a plain read
// that sees the bit set is final and saves the atomic.
__device__ __forceinline__ void visit(uint32_t u, uint32_t* bm, uint32_t* q, uint32_t* s_tail,
                                      unsigned long long* err, uint32_t qcap)
{
    const uint32_t bit = 1u << (u & 31);
    uint32_t* word = bm + (u >> 5);
    if (*reinterpret_cast<volatile uint32_t*>(word) & bit) return;
    const uint32_t old = atomicOr(word, bit);
    if (!(old & bit)) {
        const uint32_t at = atomicAdd(s_tail, 1u);
        if (IMM_IN_BOUNDS(at, qcap, err, kChkSlotQueue)) q[at] = u;
    }
}

__device__ __forceinline__ void visit_live(uint32_t live, uint32_t quad, const uint32_t* src, uint32_t* bm,
                                           uint32_t* q, uint32_t* s_tail, unsigned long long* err, uint32_t qcap)
{
    while (live) {
        const int t = __ffs(live) - 1;
        live &= live - 1;
        visit(__ldg(src + (quad << 2) + t), bm, q, s_tail, err, qcap);
    }
}

constexpr uint32_t kWarpBuf = 128;
__device__ __forceinline__ void expand_pair(uint32_t qa, bool ha, uint32_t rsa, uint32_t rea, uint32_t qb, bool hb,
                                            uint32_t rsb, uint32_t reb, const PhiloxSet& ps, const PhiloxKeys& rk,
                                            const DevGraph& g, uint32_t* bm, uint32_t* q, uint32_t* s_tail,
                                            uint32_t* wbuf, unsigned long long* err, uint32_t qcap)
{
    uint4 tha = make_uint4(0, 0, 0, 0), thb = tha, wa = tha, wb = tha;
    if (ha) tha = load_thr4(g.thr, qa);
    if (hb) thb = load_thr4(g.thr, qb);
    if (ha) wa = philox_x(qa, ps, rk);
    if (hb) wb = philox_x(qb, ps, rk);
    uint32_t la = ha ? live_mask(wa, tha, qa, rsa, rea) : 0u;
    uint32_t lb = hb ? live_mask(wb, thb, qb, rsb, reb) : 0u;
    const int lane = threadIdx.x & 31;
    const uint32_t cnt = __popc(la) + __popc(lb);
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    if (total > kWarpBuf) {
        visit_live(la, qa, g.src, bm, q, s_tail, err, qcap);
        visit_live(lb, qb, g.src, bm, q, s_tail, err, qcap);
        return;
    }
    uint32_t p = incl - cnt;
    while (la) { const int t = __ffs(la) - 1; la &= la - 1; wbuf[p++] = (qa << 2) + t; }
    while (lb) { const int t = __ffs(lb) - 1; lb &= lb - 1; wbuf[p++] = (qb << 2) + t; }
    __syncwarp();
    for (uint32_t i = lane; i < total; i += 32) visit(__ldg(g.src + wbuf[i]), bm, q, s_tail, err, qcap);
    __syncwarp();
}

constexpr uint32_t kHeavyQuads = 64;    // vertices with this many in-edge quads are split
constexpr uint32_t kChunkQuads = 64;    // quads of a heavy vertex per claimed chunk (2 per lane)
constexpr uint32_t kHeavyMax = 8192;    // heavy vertices listed per level (more: swept in place)

// Dynamic shared memory of the large path: [bitmap words (when it fits)]
// [heavy vertex ids: hcap][heavy chunk prefix: hcap + 1].
__host__ __device__ __forceinline__ size_t bitmap_smem_bytes(uint32_t n)
{
    const uint64_t words = ((uint64_t)n + 31) >> 5;
    return (size_t)(((words * 4) + 15) / 16 * 16);
}

template <bool kSmemBitmap>
__global__ void __launch_bounds__(kLargeThreads, 1)
ic_large_kernel(DevGraph g, SampleBatch b, LargeSlots ls, uint32_t hcap)
{
    unsigned long long* const err = b.sc->bounds;
    const uint32_t qcap = (uint32_t)ls.queue_cap;
    extern __shared__ __align__(16) uint32_t dyn[];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_wbuf[32][kWarpBuf];
    __shared__ uint32_t s_tail, s_next, s_end, s_claim, s_nheavy, s_hnext;
    __shared__ int s_ok;
    __shared__ unsigned long long s_pos;
    __shared__ unsigned long long s_edges;

    const uint32_t tid = threadIdx.x;
    const int lane = tid & 31;
    const int wid = tid >> 5;
    uint32_t* wbuf = s_wbuf[wid];
    const uint32_t words = b.words;
    const uint32_t bm_words = kSmemBitmap ? (uint32_t)(bitmap_smem_bytes(g.n) / 4) : 0u;
    uint32_t* bm = kSmemBitmap ? dyn : ls.bitmaps + (uint64_t)blockIdx.x * ls.bitmap_words;
    uint32_t* s_hv = dyn + bm_words;
    uint32_t* s_hpre = s_hv + hcap;
    uint32_t* q = ls.queues + (uint64_t)blockIdx.x * ls.queue_cap;
    const uint32_t large_count = b.sc->large_count;  // final: written by the previous launch

    if (kSmemBitmap)
        for (uint32_t i = tid; i < words; i += kLargeThreads) bm[i] = 0;

    for (;;) {
        if (tid == 0) {
            s_claim = atomicAdd(&b.sc->large_cursor, 1u);
            s_edges = 0;
        }
        __syncthreads();
        const uint32_t idx = s_claim;
        if (idx >= large_count) break;
        const uint32_t rel = b.large_q[idx];
        const uint64_t s = b.base + rel;
        const PhiloxSet ps = philox_set((uint32_t)s, (uint32_t)(s >> 32), kTagIC, b.rk);
        if (tid == 0) {
            const uint32_t root = draw_root(b.rk, s, g.n);
            q[0] = root;
            bm[root >> 5] |= 1u << (root & 31);
            s_tail = 1;
            s_next = 0;
            s_end = 1;
            s_nheavy = 0;
            s_hnext = 0;
        }
        __syncthreads();

        uint32_t edges = 0;
        uint32_t end = s_end;
        for (;;) {
            // ---- level q[.. end): warps claim 32-vertex chunks; light
            // vertices are expanded at once, heavy ones are listed
            for (;;) {
                uint32_t c = 0;
                if (lane == 0) c = atomicAdd(&s_next, 32u);
                c = __shfl_sync(kFull, c, 0);
                if (c >= end) break;
                const uint32_t nf = min(end - c, 32u);
                uint32_t v = 0, rs = 0, re = 0, nq = 0;
                if ((uint32_t)lane < nf) {
                    v = q[c + lane];
                    edge_range(g, v, rs, re);
                    nq = quads_of(rs, re);
                    edges += re - rs;
                }
                if (nq >= kHeavyQuads) {
                    const uint32_t hp = atomicAdd(&s_nheavy, 1u);
                    if (hp < hcap) {
                        s_hv[hp] = v;
                        nq = 0;
                    }
                }
                // leftovers when the heavy list is full: swept by this warp
                uint32_t bigm = __ballot_sync(kFull, nq >= kHeavyQuads);
                while (bigm) {
                    const int o = __ffs(bigm) - 1;
                    bigm &= bigm - 1;
                    const uint32_t ors = __shfl_sync(kFull, rs, o);
                    const uint32_t ore = __shfl_sync(kFull, re, o);
                    const uint32_t q1 = (ore - 1) >> 2;
                    for (uint32_t q0 = (ors >> 2); q0 <= q1; q0 += 64) {
                        const uint32_t qa = q0 + lane;
                        expand_pair(qa, qa <= q1, ors, ore, qa + 32, qa + 32 <= q1, ors, ore, ps, b.rk, g, bm,
                                    q, &s_tail, wbuf, err, qcap);
                    }
                }
                // light vertices: quads flattened across lanes, two per lane
                const uint32_t sq = nq >= kHeavyQuads ? 0u : nq;
                uint32_t incl = sq;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t t = __shfl_up_sync(kFull, incl, d);
                    if (lane >= d) incl += t;
                }
                const uint32_t total = __shfl_sync(kFull, incl, 31);
                const uint32_t excl = incl - sq;
                for (uint32_t j0 = 0; j0 < total; j0 += 64) {
                    const uint32_t ja = j0 + lane, jb = ja + 32;
                    uint32_t oa = 0, ob = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const uint32_t ca = __shfl_sync(kFull, incl, oa + step - 1);
                        const uint32_t cb = __shfl_sync(kFull, incl, ob + step - 1);
                        if (ca <= ja) oa += step;
                        if (cb <= jb) ob += step;
                    }
                    const uint32_t rsa = __shfl_sync(kFull, rs, oa), rea = __shfl_sync(kFull, re, oa);
                    const uint32_t rsb = __shfl_sync(kFull, rs, ob), reb = __shfl_sync(kFull, re, ob);
                    const uint32_t exa = __shfl_sync(kFull, excl, oa), exb = __shfl_sync(kFull, excl, ob);
                    const bool ha = ja < total, hb = jb < total;
                    const uint32_t qa = (rsa >> 2) + (ja - exa);
                    const uint32_t qb = (rsb >> 2) + (jb - exb);
                    expand_pair(qa, ha, rsa, rea, qb, hb, rsb, reb, ps, b.rk, g, bm, q, &s_tail, wbuf, err, qcap);
                }
            }
            __syncthreads();
            // ---- heavy vertices of the level: 64-quad chunks shared by all warps
            const uint32_t nh = min(s_nheavy, hcap);
            if (nh) {
                // block-wide exclusive scan of the chunk counts (hcap / 1024 per thread)
                const uint32_t per = (nh + kLargeThreads - 1) / kLargeThreads;
                const uint32_t i0 = tid * per;
                uint32_t local = 0;
                for (uint32_t i = i0; i < i0 + per && i < nh; ++i) {
                    uint32_t hrs, hre;
                    edge_range(g, s_hv[i], hrs, hre);
                    local += (quads_of(hrs, hre) + kChunkQuads - 1) / kChunkQuads;
                }
                uint32_t incl = local;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t t = __shfl_up_sync(kFull, incl, d);
                    if (lane >= d) incl += t;
                }
                if (lane == 31) s_warp[wid] = incl;
                __syncthreads();
                if (wid == 0) {
                    uint32_t x = s_warp[lane];
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const uint32_t t = __shfl_up_sync(kFull, x, d);
                        if (lane >= d) x += t;
                    }
                    s_warp[lane] = x;
                }
                __syncthreads();
                uint32_t run = incl - local + (wid ? s_warp[wid - 1] : 0u);
                for (uint32_t i = i0; i < i0 + per && i < nh; ++i) {
                    s_hpre[i] = run;
                    uint32_t hrs, hre;
                    edge_range(g, s_hv[i], hrs, hre);
                    run += (quads_of(hrs, hre) + kChunkQuads - 1) / kChunkQuads;
                }
                if (tid == 0) s_hpre[nh] = s_warp[31];
                __syncthreads();
                const uint32_t nchunks = s_hpre[nh];
                for (;;) {
                    uint32_t c = 0;
                    if (lane == 0) c = atomicAdd(&s_hnext, 1u);
                    c = __shfl_sync(kFull, c, 0);
                    if (c >= nchunks) break;
                    // owner: the last lo with s_hpre[lo] <= c, by a 32-way search
                    // (invariant s_hpre[lo] <= c < s_hpre[lo + span]; lane 0's
                    // probe is s_hpre[lo] itself, so the ballot is never empty)
                    uint32_t lo = 0, span = nh;
                    while (span > 1) {
                        const uint32_t step = (span + 31) >> 5;
                        const uint32_t off = (uint32_t)lane * step;
                        const bool le = off < span && s_hpre[lo + off] <= c;
                        const uint32_t t = 31 - __clz(__ballot_sync(kFull, le));
                        lo += t * step;
                        span = min(step, span - t * step);
                    }
                    uint32_t hrs, hre;
                    edge_range(g, s_hv[lo], hrs, hre);
                    const uint32_t q1 = (hre - 1) >> 2;
                    const uint32_t qa = (hrs >> 2) + (c - s_hpre[lo]) * kChunkQuads + lane;
                    expand_pair(qa, qa <= q1, hrs, hre, qa + 32, qa + 32 <= q1, hrs, hre, ps, b.rk, g, bm, q,
                                &s_tail, wbuf, err, qcap);
                }
            }
            __syncthreads();
            if (tid == 0) {
                s_next = end;
                s_end = s_tail;
                s_nheavy = 0;
                s_hnext = 0;
            }
            __syncthreads();
            const uint32_t ne = s_end;
            if (ne == end) break;
            end = ne;
        }

        // set done: record, store as list or bitmap, clear the visited bits
        const uint32_t len = end;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) edges += __shfl_xor_sync(kFull, edges, d);
        if (lane == 0 && edges) atomicAdd(&s_edges, (unsigned long long)edges);
        __syncthreads();
        const uint32_t kind = len > words ? 1u : 0u;
        if (tid == 0) {
            b.set_edges[rel] = (uint32_t)s_edges;
            uint64_t pos = 0;
            s_ok = reserve_big(b, rel, len, kind, &pos) ? 1 : 0;
            s_pos = pos;
        }
        __syncthreads();
        if (s_ok) {
            uint32_t* out = b.big + s_pos;
            if (kind) {
                for (uint32_t i = tid; i < words; i += kLargeThreads)
                    if (IMM_IN_BOUNDS(s_pos + i, b.big_cap, err, kChkBig)) out[i] = bm[i];
            } else {
                for (uint32_t i = tid; i < len; i += kLargeThreads)
                    if (IMM_IN_BOUNDS(s_pos + i, b.big_cap, err, kChkBig)) out[i] = q[i];
            }
        }
        __syncthreads();
        if (kSmemBitmap || (uint64_t)len * 8 >= words) {
            for (uint32_t i = tid; i < words; i += kLargeThreads) bm[i] = 0;
        } else {
            for (uint32_t i = tid; i < len; i += kLargeThreads) bm[q[i] >> 5] = 0;
        }
        __syncthreads();
    }
}

static size_t large_smem_bytes(uint32_t n)
{
    return bitmap_smem_bytes(n);
}

int ic_large_uses_smem(uint32_t n, const DeviceInfo& di)
{
    // the bitmap plus a heavy-vertex list of at least 1024 entries
    return large_smem_bytes(n) + 8 * 1024 + 1024 <= (size_t)di.max_smem_optin;
}

// heavy-list capacity that fits beside the bitmap (or alone)
static uint32_t heavy_cap(uint32_t n, bool smem_bitmap, const DeviceInfo& di)
{
    const size_t used = (smem_bitmap ? large_smem_bytes(n) : 0) + 1024 + 32 * kWarpBuf * 4;
    const size_t room = (size_t)di.max_smem_optin > used ? (size_t)di.max_smem_optin - used : 0;
    size_t cap = room / 8;
    if (cap > kHeavyMax) cap = kHeavyMax;
    return (uint32_t)(cap > 16 ? cap - 1 : 0);
}

cudaError_t launch_ic_large(const DevGraph& g, const SampleBatch& b, const LargeSlots& ls, const DeviceInfo& di,
                            cudaStream_t st)
{
    const unsigned grid = ls.nslots;
    const bool smem_bm = ic_large_uses_smem(g.n, di) != 0;
    const uint32_t hcap = heavy_cap(g.n, smem_bm, di);
    const size_t smem = (smem_bm ? large_smem_bytes(g.n) : 0) + (size_t)(2 * hcap + 1) * 4;
    // The opt-in limit is set to one fixed value (the device maximum less the
    // kernel's static shared memory) whatever this launch needs, so host
    // threads launching for graphs of different sizes never undercut each
    // other's setting.
    cudaFuncAttributes fa;
    cudaError_t fe = smem_bm ? cudaFuncGetAttributes(&fa, ic_large_kernel<true>)
                             : cudaFuncGetAttributes(&fa, ic_large_kernel<false>);
    if (fe != cudaSuccess) return fe;
    const int max_dyn = di.max_smem_optin - (int)fa.sharedSizeBytes;
    if ((int)smem > max_dyn) return cudaErrorInvalidValue;
    if (smem_bm) {
        cudaError_t e =
            cudaFuncSetAttribute(ic_large_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
        if (e != cudaSuccess) return e;
        ic_large_kernel<true><<<grid, kLargeThreads, smem, st>>>(g, b, ls, hcap);
    } else {
        cudaError_t e =
            cudaFuncSetAttribute(ic_large_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
        if (e != cudaSuccess) return e;
        ic_large_kernel<false><<<grid, kLargeThreads, smem, st>>>(g, b, ls, hcap);
    }
    return cudaGetLastError();
}

// ===========================================================================
// LT, small path: one lane per walk, path kept in shared memory.
// ===========================================================================
constexpr int kLtThreads = 64;  // path and filter stay within static shared memory

// One step of the reverse walk at a vertex with in-edge range [lo, hi): the
// first j in [lo, hi) with r < cthr[j] (cthr is nondecreasing), or hi; the
// tail u of j and u's in-edge range [*ulo, *uhi).  The guide entry of r's
// bucket is the answer when r is below its threshold, and it carries u and
// (unless u's in-degree is too large for its field) u's range; otherwise a
// short scan and row reads.
constexpr uint32_t kCthrMask = (1u << 25) - 1;

// The guide entry a walk step at a vertex with in-edges [lo, hi) and draw r
// starts from (nothing to load for a vertex without in-edges).
__device__ __forceinline__ uint4 lt_guide_load(const DevGraph& g, uint32_t lo, uint32_t hi, uint32_t r)
{
    if (hi == lo) return make_uint4(hi, 0u, 0u, 0u);
    return __ldg(g.guide + lo + (uint32_t)(((uint64_t)r * (hi - lo)) >> 24));
}

// The step itself, from that entry: the picked in-edge j (hi when none) and
// its tail u with u's in-edge range.  Memory is read only when the entry's
// candidate is not the pick or the tail's range is not in the entry.
__device__ __forceinline__ uint32_t lt_resolve(const DevGraph& g, uint32_t lo, uint32_t hi, uint32_t r, uint4 e,
                                               uint32_t* u, uint32_t* ulo, uint32_t* uhi)
{
    if (hi == lo) return hi;
    const bool rel = hi - lo <= kGuideRelMax;
    uint32_t j = rel ? lo + (e.x & 0xFFFFu) : e.x;
    if (j < hi && r < (e.y & kCthrMask)) {
        *u = e.z;
        const uint32_t du = rel ? (e.y >> 25) | ((e.x >> 16) << 7) : e.y >> 25;
        if (du < (rel ? kGuideDegRel : kGuideDegAbs)) {
            *ulo = e.w;
            *uhi = e.w + du;
        } else {
            edge_range(g, e.z, *ulo, *uhi);
        }
        return j;
    }
    if (j < hi) ++j;
    while (j < hi && r >= __ldg(g.thr + j)) ++j;
    if (j < hi) {
        *u = __ldg(g.src + j);
        edge_range(g, *u, *ulo, *uhi);
    }
    return j;
}

// Walks that outgrow the lane's path go on in a per-walk table claimed from
// the pool (MidSlots; the pool's tables are zero between walks): members
// kLtCap.. are kept there, and a step's table probe is issued together with
// the next guide entry.  A lane whose claim finds the pool used up hands the
// walk to the per-walk-table kernel, which samples it again from its root.
// A lane's path has a 1024-bit membership filter, so the path is scanned
// only when the filter holds the vertex's bit (a revisit, or 1 in 7 steps at
// most while the path fills).
constexpr int kLtFiltWords = 32;
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

// One thread's copy of src[0, len) to dst + pos (dst's bound cap) and
// clearing of tab[slots[0, len)], eight loads in flight at a time: a walk of
// hundreds of members costs tens of round trips, not hundreds.
__device__ __forceinline__ void thread_copy(uint32_t* dst, uint64_t pos, uint64_t cap, const uint32_t* src,
                                            uint32_t len, unsigned long long* err, uint32_t where)
{
    for (uint32_t i0 = 0; i0 < len; i0 += 8) {
        uint32_t t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = i0 + u < len ? src[i0 + u] : 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (i0 + u < len && IMM_IN_BOUNDS(pos + i0 + u, cap, err, where)) dst[pos + i0 + u] = t[u];
    }
    (void)err;
    (void)where;
}

__device__ __forceinline__ void thread_clear(uint32_t* tab, const uint32_t* slots, uint32_t len)
{
    for (uint32_t i0 = 0; i0 < len; i0 += 8) {
        uint32_t t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = i0 + u < len ? slots[i0 + u] : 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (i0 + u < len) tab[t[u]] = 0u;
    }
}

__device__ __forceinline__ uint32_t lt_mid_hash(uint32_t u)
{
    return (u * 0x9E3779B1u) >> (32 - kLtMidHashBits);
}

__device__ __forceinline__ uint32_t lt_filt_bit(uint32_t u)
{
    return (u * 0x85EBCA6Bu) >> 22;  // 10 bits
}

__global__ void __launch_bounds__(kLtThreads)
lt_small_kernel(DevGraph g, SampleBatch b, MidSlots ms)
{
    __shared__ uint32_t path[kLtCap][kLtThreads];
    __shared__ uint32_t filt[kLtFiltWords][kLtThreads];
    const uint32_t tid = threadIdx.x;
    const int lane = tid & 31;
    const uint32_t ltm = lanemask_lt();
    // total members a walk may reach here: a list of at most n/32 members
    // and the table's capacity (no continuation when that is below kLtCap)
    const uint32_t cap = b.words < kLtMidCap ? b.words : kLtMidCap;
#pragma unroll
    for (int w = 0; w < kLtFiltWords; ++w) filt[w][tid] = 0u;
    bool busy = false, done = false;
    uint32_t rel = 0, len = 0, v = 0, lo = 0, hi = 0;  // walk position and its in-edge range
    uint32_t dr = 0;                                   // the draw at v
    uint4 e = make_uint4(0, 0, 0, 0);                  // its guide entry (loaded one step ahead)
    uint32_t slot = kNoSlot;                           // pool slot of a continued walk
    PhiloxSet ps{};
    for (;;) {
        const uint32_t need = __ballot_sync(kFull, !busy && !done);
        if (need) {
            const int leader = __ffs(need) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&b.sc->cursor, (uint32_t)__popc(need));
            base = __shfl_sync(kFull, base, leader);
            if (!busy && !done) {
                const uint32_t r = base + __popc(need & ltm);
                if (r < b.count) {
                    rel = r;
                    busy = true;
                    const uint64_t s = b.base + rel;
                    ps = philox_set((uint32_t)s, (uint32_t)(s >> 32), kTagLT, b.rk);
                    v = draw_root(b.rk, s, g.n);
                    edge_range(g, v, lo, hi);
                    dr = philox_x(v, ps, b.rk).x >> 8;
                    e = lt_guide_load(g, lo, hi, dr);
                    path[0][tid] = v;
                    const uint32_t fb = lt_filt_bit(v);
                    filt[fb >> 5][tid] |= 1u << (fb & 31);
                    len = 1;
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(kFull, done)) break;
        if (!busy) continue;
        uint32_t* tab = ms.tab + (slot != kNoSlot ? (uint64_t)slot * kLtMidHash : 0ull);
        // one step of the reverse walk at v (in-edges [lo, hi)); the next
        // step's guide entry and the table probe are loaded before the
        // revisit test on the path, which then runs while they are in flight
        uint32_t u = 0, ulo = 0, uhi = 0;
        const uint32_t pick = lt_resolve(g, lo, hi, dr, e, &u, &ulo, &uhi);
        bool stop = pick == hi;
        uint32_t r2 = 0, h = 0;
        uint4 e2 = make_uint4(0, 0, 0, 0);
        if (!stop) {
            r2 = philox_x(u, ps, b.rk).x >> 8;
            e2 = lt_guide_load(g, ulo, uhi, r2);
            uint32_t t = 0;
            if (slot != kNoSlot) {
                h = lt_mid_hash(u);
                t = tab[h];
            }
            const uint32_t fb = lt_filt_bit(u);
            if (filt[fb >> 5][tid] & (1u << (fb & 31))) {
                const uint32_t pl = len < kLtCap ? len : kLtCap;
                for (uint32_t i = 0; i < pl; ++i)
                    if (path[i][tid] == u) {
                        stop = true;
                        break;
                    }
            }
            if (!stop && slot != kNoSlot) {
                // linear probing ends: the table holds at most cap - kLtCap
                // <= half its entries
                while (t != 0u && t != u + 1u) {
                    h = (h + 1u) & (kLtMidHash - 1u);
                    t = tab[h];
                }
                stop = t != 0u;
            }
        }
        if (!stop) {
            bool keep = true;
            if (len < kLtCap) {
                path[len][tid] = u;
                const uint32_t fb = lt_filt_bit(u);
                filt[fb >> 5][tid] |= 1u << (fb & 31);
            } else if (len == cap || (slot == kNoSlot && cap <= kLtCap)) {
                // longer than a list or a table holds: the bitmap path
                const uint32_t o = atomicAdd(&b.sc->long_count, 1u);
                if (IMM_IN_BOUNDS(o, b.count, b.sc->bounds, kChkLongQ)) b.long_q[o] = rel;
                b.set_len[rel] = kLenPending;
                keep = false;
            } else {
                if (slot == kNoSlot) {
                    const uint32_t sl = atomicAdd(&b.sc->mid_claim, 1u);
                    if (sl < ms.nslots) {
                        slot = sl;
                        tab = ms.tab + (uint64_t)slot * kLtMidHash;
                        h = lt_mid_hash(u);  // the table is empty
                    } else {
                        const uint32_t qi = atomicAdd(&b.sc->large_count, 1u);
                        if (IMM_IN_BOUNDS(qi, b.count, b.sc->bounds, kChkLargeQ)) b.large_q[qi] = rel;
                        b.set_len[rel] = kLenPending;
                        keep = false;
                    }
                }
                if (keep) {
                    const uint64_t at = (uint64_t)slot * kLtMidCap + (len - kLtCap);
                    tab[h] = u + 1u;
                    ms.hpos[at] = h;
                    ms.path[at] = u;
                }
            }
            if (keep) {
                ++len;
                v = u;
                lo = ulo;
                hi = uhi;
                dr = r2;
                e = e2;
                continue;
            }
        } else {
            b.set_edges[rel] = len;
            uint64_t pos = 0;
            if (reserve_small(b, rel, len, &pos)) {
                const uint32_t pl = len < kLtCap ? len : kLtCap;
                for (uint32_t i = 0; i < pl; ++i)
                    if (IMM_IN_BOUNDS(pos + i, b.stage_cap, b.sc->bounds, kChkStage)) b.stage[pos + i] = path[i][tid];
                if (len > pl)
                    thread_copy(b.stage, pos + pl, b.stage_cap, ms.path + (uint64_t)slot * kLtMidCap, len - pl,
                                b.sc->bounds, kChkStage);
            }
        }
        // the walk ends here (stored, or handed on): clear its table entries
        // and its filter
        if (slot != kNoSlot) {
            if (len > kLtCap) thread_clear(tab, ms.hpos + (uint64_t)slot * kLtMidCap, len - kLtCap);
            slot = kNoSlot;
        }
#pragma unroll
        for (int w = 0; w < kLtFiltWords; ++w) filt[w][tid] = 0u;
        busy = false;
    }
}

cudaError_t launch_lt_small(const DevGraph& g, const SampleBatch& b, const MidSlots& ms, const DeviceInfo& di,
                            cudaStream_t st)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lt_small_kernel, kLtThreads, 0);
    if (e != cudaSuccess) return e;
    const uint64_t want = ((uint64_t)b.count + kLtThreads - 1) / kLtThreads;
    uint64_t grid = (uint64_t)di.sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    if (grid > want) grid = want;
    if (grid == 0) grid = 1;
    lt_small_kernel<<<(unsigned)grid, kLtThreads, 0, st>>>(g, b, ms);
    return cudaGetLastError();
}

// ===========================================================================
// LT, walks past the lane path's capacity: one thread per walk (every walk
// of the batch at once, up to kLtMidSlotsMax), visited set in a per-walk
// table.  Each step's table probe is issued together with the next step's
// guide entry, so a step costs one memory round trip as on the other paths.
// ===========================================================================
constexpr int kLtMidThreads = 128;

__global__ void __launch_bounds__(kLtMidThreads)
lt_mid_kernel(DevGraph g, SampleBatch b, MidSlots ms)
{
    const uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= ms.nslots) return;
    uint32_t* tab = ms.tab + (uint64_t)slot * kLtMidHash;
    uint32_t* path = ms.path + (uint64_t)slot * kLtMidCap;
    uint32_t* hpos = ms.hpos + (uint64_t)slot * kLtMidCap;
    const uint32_t large_count = b.sc->large_count;
    // a walk longer than a list of n/32 members is stored as a bitmap: the
    // bitmap path takes it
    const uint32_t cap = b.words < kLtMidCap ? b.words : kLtMidCap;
    for (uint32_t idx = slot; idx < large_count; idx += ms.nslots) {
        const uint32_t rel = b.large_q[idx];
        const uint64_t s = b.base + rel;
        const PhiloxSet ps = philox_set((uint32_t)s, (uint32_t)(s >> 32), kTagLT, b.rk);
        uint32_t v = draw_root(b.rk, s, g.n);
        uint32_t lo, hi;
        edge_range(g, v, lo, hi);
        uint32_t h = lt_mid_hash(v);
        tab[h] = v + 1;
        hpos[0] = h;
        path[0] = v;
        uint32_t len = 1;
        bool over = false;
        uint32_t r = philox_x(v, ps, b.rk).x >> 8;
        uint4 e = lt_guide_load(g, lo, hi, r);
        for (;;) {
            uint32_t u = 0, ulo = 0, uhi = 0;
            const uint32_t pick = lt_resolve(g, lo, hi, r, e, &u, &ulo, &uhi);
            if (pick == hi) break;
            h = lt_mid_hash(u);
            uint32_t t = tab[h];
            const uint32_t r2 = philox_x(u, ps, b.rk).x >> 8;
            const uint4 e2 = lt_guide_load(g, ulo, uhi, r2);
            // linear probing ends: the table holds at most cap <= half its
            // entries
            while (t != 0u && t != u + 1u) {
                h = (h + 1u) & (kLtMidHash - 1u);
                t = tab[h];
            }
            if (t) break;  // u is on the walk already
            if (len == cap) {
                over = true;
                break;
            }
            tab[h] = u + 1u;
            hpos[len] = h;
            path[len] = u;
            ++len;
            lo = ulo;
            hi = uhi;
            r = r2;
            e = e2;
        }
        thread_clear(tab, hpos, len);
        if (over) {
            const uint32_t o = atomicAdd(&b.sc->long_count, 1u);
            if (IMM_IN_BOUNDS(o, b.count, b.sc->bounds, kChkLongQ)) b.long_q[o] = rel;
            continue;
        }
        b.set_edges[rel] = len;
        uint64_t pos = 0;
        if (reserve_big(b, rel, len, 0u, &pos)) {
            thread_copy(b.big, pos, b.big_cap, path, len, b.sc->bounds, kChkBig);
        }
    }
}

cudaError_t launch_lt_mid(const DevGraph& g, const SampleBatch& b, const MidSlots& ms, cudaStream_t st)
{
    const unsigned grid = (ms.nslots + kLtMidThreads - 1) / kLtMidThreads;
    lt_mid_kernel<<<grid, kLtMidThreads, 0, st>>>(g, b, ms);
    return cudaGetLastError();
}

// ===========================================================================
// LT, walks longer still: one thread per walk with an n-bit global bitmap
// slot; the member queue holds the first n/32 + 1 members (a longer walk is
// stored as the bitmap).
// ===========================================================================
__global__ void __launch_bounds__(32)
lt_long_kernel(DevGraph g, SampleBatch b, LargeSlots ls)
{
    const int lane = threadIdx.x;
    uint32_t* bm = ls.bitmaps + (uint64_t)blockIdx.x * ls.bitmap_words;
    uint32_t* q = ls.queues + (uint64_t)blockIdx.x * ls.queue_cap;
    const uint32_t long_count = b.sc->long_count;
    const uint32_t words = b.words;
    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(&b.sc->long_cursor, 1u);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= long_count) break;
        const uint32_t rel = b.long_q[idx];
        const uint64_t s = b.base + rel;
        uint32_t len = 0;
        if (lane == 0) {
            const PhiloxSet ps = philox_set((uint32_t)s, (uint32_t)(s >> 32), kTagLT, b.rk);
            const uint32_t v = draw_root(b.rk, s, g.n);
            uint32_t lo, hi;
            edge_range(g, v, lo, hi);
            q[0] = v;
            bm[v >> 5] |= 1u << (v & 31);
            len = 1;
            uint32_t r = philox_x(v, ps, b.rk).x >> 8;
            uint4 e = lt_guide_load(g, lo, hi, r);
            for (;;) {
                uint32_t u = 0, ulo = 0, uhi = 0;
                const uint32_t pick = lt_resolve(g, lo, hi, r, e, &u, &ulo, &uhi);
                if (pick == hi) break;
                // the visited word and the next step's guide entry (loaded on
                // the chance that u is new) are in flight together: one round
                // trip per step
                const uint32_t bit = 1u << (u & 31);
                const uint32_t word = bm[u >> 5];
                const uint32_t r2 = philox_x(u, ps, b.rk).x >> 8;
                const uint4 e2 = lt_guide_load(g, ulo, uhi, r2);
                if (word & bit) break;
                bm[u >> 5] = word | bit;
                if (len < ls.queue_cap) q[len] = u;
                ++len;
                lo = ulo;
                hi = uhi;
                r = r2;
                e = e2;
            }
            b.set_edges[rel] = len;
        }
        len = __shfl_sync(kFull, len, 0);
        __syncwarp();
        const uint32_t kind = len > words ? 1u : 0u;
        uint64_t pos = 0;
        int ok = 0;
        if (lane == 0) ok = reserve_big(b, rel, len, kind, &pos) ? 1 : 0;
        ok = __shfl_sync(kFull, ok, 0);
        pos = shfl64(pos, 0);
        if (ok) {
            uint32_t* out = b.big + pos;
            if (kind)
                for (uint32_t i = lane; i < words; i += 32) {
                    if (IMM_IN_BOUNDS(pos + i, b.big_cap, b.sc->bounds, kChkBig)) out[i] = bm[i];
                }
            else
                for (uint32_t i = lane; i < len; i += 32)
                    if (IMM_IN_BOUNDS(pos + i, b.big_cap, b.sc->bounds, kChkBig)) out[i] = q[i];
        }
        __syncwarp();
        if (kind)
            for (uint32_t i = lane; i < words; i += 32) bm[i] = 0;
        else
            for (uint32_t i = lane; i < len; i += 32) bm[q[i] >> 5] = 0;
        __syncwarp();
    }
}

cudaError_t launch_lt_long(const DevGraph& g, const SampleBatch& b, const LargeSlots& ls, const DeviceInfo& di,
                           cudaStream_t st)
{
    (void)di;
    lt_long_kernel<<<ls.nslots, 32, 0, st>>>(g, b, ls);
    return cudaGetLastError();
}

// ===========================================================================
// Batch scan over the kept sets [0, committed), committed = min(first_fail,
// count): list offsets into off[], bitmap ranks, and the batch totals.
// ===========================================================================
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr uint32_t kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t warp_incl_scan64(uint64_t x, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t t = shfl64_up(x, d);
        if (lane >= d) x += t;
    }
    return x;
}

uint64_t scan_tmp_words(uint32_t count)
{
    return 4 * ((uint64_t)count / kScanTile + 2) + 8;
}

__device__ __forceinline__ uint32_t batch_committed(const SampleBatch& b)
{
    const uint32_t f = b.sc->first_fail;
    return f < b.count ? f : b.count;
}

// Block-wide exclusive scan of one value per thread (uint64).  Returns the
// exclusive prefix; *total receives the block sum.
__device__ uint64_t block_excl_scan64(uint64_t x, uint64_t* s_warp, uint64_t* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t incl = warp_incl_scan64(x, lane);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        uint64_t y = lane < nw ? s_warp[lane] : 0;
        y = warp_incl_scan64(y, lane);
        if (lane < nw) s_warp[lane] = y;
    }
    __syncthreads();
    const uint64_t wb = wid ? s_warp[wid - 1] : 0;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return wb + incl - x;
}

// per tile: [0] list members, [1] bitmap sets, [2] all members, [3] edges
__global__ void __launch_bounds__(kScanThreads)
batch_tile_sum_kernel(SampleBatch b, uint64_t* tiles, uint32_t ntiles)
{
    __shared__ uint64_t s_warp[32];
    const uint32_t committed = batch_committed(b);
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTile;
    uint64_t sum[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t r = t0 + (uint64_t)threadIdx.x * kScanItems + i;
        if (r < committed) {
            const uint32_t len = b.set_len[r];
            const uint32_t kind = b.set_kind[r];
            sum[0] += kind ? 0u : len;
            sum[1] += kind;
            sum[2] += len;
            sum[3] += b.set_edges[r];
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint64_t tot;
        block_excl_scan64(sum[c], s_warp, &tot);
        if (threadIdx.x == 0) tiles[(uint64_t)c * ntiles + blockIdx.x] = tot;
    }
}

// one block: exclusive scans of the tile sums (lists, bitmaps) and totals
__global__ void __launch_bounds__(kScanThreads)
batch_tile_scan_kernel(SampleBatch b, uint64_t* tiles, uint32_t ntiles)
{
    __shared__ uint64_t s_warp[32];
    __shared__ uint64_t s_carry[2];
    if (threadIdx.x < 2) s_carry[threadIdx.x] = 0;
    __syncthreads();
    uint64_t all = 0, edges = 0;
    for (uint32_t t0 = 0; t0 < ntiles; t0 += kScanThreads) {
        const uint32_t t = t0 + threadIdx.x;
        if (t < ntiles) {
            all += tiles[2ull * ntiles + t];
            edges += tiles[3ull * ntiles + t];
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint64_t x = t < ntiles ? tiles[(uint64_t)c * ntiles + t] : 0;
            uint64_t tot;
            const uint64_t ex = block_excl_scan64(x, s_warp, &tot);
            if (t < ntiles) tiles[(uint64_t)c * ntiles + t] = s_carry[c] + ex;
            __syncthreads();
            if (threadIdx.x == 0) s_carry[c] += tot;
            __syncthreads();
        }
    }
    uint64_t tot_all, tot_edges;
    block_excl_scan64(all, s_warp, &tot_all);
    block_excl_scan64(edges, s_warp, &tot_edges);
    if (threadIdx.x == 0) {
        b.sc->list_members = s_carry[0];
        b.sc->nbitmaps = s_carry[1];
        b.sc->all_members = tot_all;
        b.sc->edges = tot_edges;
        b.sc->committed = batch_committed(b);
    }
}

__global__ void __launch_bounds__(kScanThreads)
batch_tile_write_kernel(SampleBatch b, BatchOut o, const uint64_t* tiles, uint32_t ntiles)
{
    __shared__ uint64_t s_warp[32];
    const uint32_t committed = batch_committed(b);
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTile;
    uint32_t ln[kScanItems], kd[kScanItems];
    uint64_t a = 0, c = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t r = t0 + (uint64_t)threadIdx.x * kScanItems + i;
        ln[i] = 0;
        kd[i] = 0;
        if (r < committed) {
            kd[i] = b.set_kind[r];
            ln[i] = kd[i] ? 0u : b.set_len[r];
        }
        a += ln[i];
        c += kd[i];
    }
    uint64_t tot;
    uint64_t ex = block_excl_scan64(a, s_warp, &tot);
    uint64_t exb = block_excl_scan64(c, s_warp, &tot);
    const uint64_t base = o.off[b.base] + tiles[blockIdx.x];
    const uint64_t bbase = tiles[(uint64_t)ntiles + blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t r = t0 + (uint64_t)threadIdx.x * kScanItems + i;
        if (r < committed) {
            const uint64_t rank = bbase + exb;
            o.set_bmp[b.base + r] = kd[i] ? (uint32_t)(o.bmp_base + rank) : kEmpty;
            if (kd[i]) o.bmp_rel[rank] = (uint32_t)r;
        }
        ex += ln[i];
        exb += kd[i];
        if (r < committed) o.off[b.base + r + 1] = base + ex;
    }
}

cudaError_t launch_batch_scan(const SampleBatch& b, const BatchOut& o, uint64_t* tmp, const DeviceInfo& di,
                              cudaStream_t st)
{
    (void)di;
    const uint32_t ntiles = (uint32_t)(((uint64_t)b.count + kScanTile - 1) / kScanTile);
    batch_tile_sum_kernel<<<ntiles, kScanThreads, 0, st>>>(b, tmp, ntiles);
    batch_tile_scan_kernel<<<1, kScanThreads, 0, st>>>(b, tmp, ntiles);
    batch_tile_write_kernel<<<ntiles, kScanThreads, 0, st>>>(b, o, tmp, ntiles);
    return cudaGetLastError();
}

// ===========================================================================
// Compaction of the list-stored sets: staging -> arena in set-id order, fused
// occurrence count.  A warp takes 32 consecutive sets: sets of >= 32 members
// are copied by the whole warp one at a time; the shorter ones are flattened.
// ===========================================================================
__device__ __forceinline__ uint32_t owner_of(uint32_t j, uint32_t incl)
{
    uint32_t o = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const uint32_t c = __shfl_sync(kFull, incl, o + step - 1);
        if (c <= j) o += step;
    }
    return o;
}

__device__ __forceinline__ const uint32_t* source_of(const SampleBatch& b, uint64_t pos)
{
    return (pos & kBigFlag) ? b.big + (pos & ~kBigFlag) : b.stage + pos;
}

__global__ void __launch_bounds__(256)
compact_kernel(SampleBatch b, BatchOut ob, uint64_t committed, uint32_t* hist)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t first = gw * 32; first < committed; first += nw * 32) {
        const uint64_t rel = first + lane;
        uint32_t len = 0;
        const uint32_t* src = nullptr;
        uint64_t dst = 0;
        if (rel < committed && b.set_kind[rel] == 0) {
            len = b.set_len[rel];
            src = source_of(b, b.set_pos[rel]);
            dst = ob.off[b.base + rel];
        }
        const bool big = len >= 32;
        uint32_t bigmask = __ballot_sync(kFull, big);
        while (bigmask) {
            const int o = __ffs(bigmask) - 1;
            bigmask &= bigmask - 1;
            const uint32_t L = __shfl_sync(kFull, len, o);
            const uint32_t* S = reinterpret_cast<const uint32_t*>(shfl64(reinterpret_cast<uint64_t>(src), o));
            const uint64_t D = shfl64(dst, o);
            for (uint32_t i = lane; i < L; i += 32) {
                const uint32_t u = S[i];
                if (IMM_IN_BOUNDS(D + i, ob.arena_cap, ob.bounds, kChkArena)) ob.arena[D + i] = u;
                atomicAdd(&hist[u], 1u);
            }
        }
        const uint32_t sl = big ? 0u : len;
        uint32_t incl = sl;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += t;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        const uint32_t excl = incl - sl;
        for (uint32_t j0 = 0; j0 < total; j0 += 32) {
            const uint32_t j = j0 + lane;
            const uint32_t o = owner_of(j, incl);
            const uint32_t* S = reinterpret_cast<const uint32_t*>(shfl64(reinterpret_cast<uint64_t>(src), o));
            const uint64_t D = shfl64(dst, o);
            const uint32_t ex = __shfl_sync(kFull, excl, o);
            if (j < total) {
                const uint32_t u = S[j - ex];
                if (IMM_IN_BOUNDS(D + (j - ex), ob.arena_cap, ob.bounds, kChkArena)) ob.arena[D + (j - ex)] = u;
                atomicAdd(&hist[u], 1u);
            }
        }
    }
}

cudaError_t launch_compact(const SampleBatch& b, const BatchOut& o, uint64_t committed, uint32_t* hist,
                           const DeviceInfo& di, cudaStream_t st)
{
    if (committed == 0) return cudaSuccess;
    const uint64_t warps = (committed + 31) / 32;
    uint64_t blocks = (warps + 7) / 8;
    const uint64_t cap = (uint64_t)di.sms * 16;
    if (blocks > cap) blocks = cap;
    compact_kernel<<<(unsigned)blocks, 256, 0, st>>>(b, o, committed, hist);
    return cudaGetLastError();
}

// ===========================================================================
// Bitmap-stored sets: copy into the bitmap arena, then count them into cnt[]
// by columns (each thread owns 32 vertices of one bitmap word and sums the
// bits of a chunk of bitmaps in registers).
// ===========================================================================
__global__ void __launch_bounds__(256)
bitmap_copy_kernel(SampleBatch b, BatchOut o, uint64_t nbitmaps)
{
    for (uint64_t r = blockIdx.x; r < nbitmaps; r += gridDim.x) {
        const uint32_t rel = o.bmp_rel[r];
        const uint32_t* src = b.big + (b.set_pos[rel] & ~kBigFlag);
        const uint64_t gid = o.bmp_base + r;
        uint32_t* dst = o.bmp + gid * b.words;
        for (uint32_t i = threadIdx.x; i < b.words; i += blockDim.x) dst[i] = src[i];
        if (threadIdx.x == 0) {
            o.bmp_set[gid] = (uint32_t)(b.base + rel);
            o.bmp_len[gid] = b.set_len[rel];
        }
    }
}

__global__ void __launch_bounds__(256)
bitmap_count_kernel(const uint32_t* bmp, uint32_t words, uint32_t n, uint64_t first, uint64_t count,
                    uint64_t per_chunk, const uint8_t* skip, const uint32_t* bmp_set, uint32_t* cnt)
{
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t b0 = first + (uint64_t)blockIdx.y * per_chunk;
    uint64_t b1 = b0 + per_chunk;
    if (b1 > first + count) b1 = first + count;
    if (w >= words) return;
    uint32_t c[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) c[i] = 0;
    for (uint64_t bi = b0; bi < b1; ++bi) {
        if (skip && skip[bmp_set[bi]]) continue;
        const uint32_t x = __ldg(bmp + bi * words + w);
        if (!x) continue;
#pragma unroll
        for (int i = 0; i < 32; ++i) c[i] += (x >> i) & 1u;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const uint32_t v = w * 32 + i;
        if (c[i] && v < n) atomicAdd(&cnt[v], c[i]);
    }
}

cudaError_t launch_bitmap_count(const uint32_t* bmp, uint32_t words, uint32_t n, uint64_t first, uint64_t count,
                                const uint8_t* skip, const uint32_t* bmp_set, uint32_t* cnt, const DeviceInfo& di,
                                cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    const uint32_t bx = (words + 255) / 256;
    uint64_t chunks = ((uint64_t)di.sms * 8 + bx - 1) / bx;
    if (chunks > count) chunks = count;
    if (chunks > 65535) chunks = 65535;
    if (chunks == 0) chunks = 1;
    const uint64_t per = (count + chunks - 1) / chunks;
    chunks = (count + per - 1) / per;
    bitmap_count_kernel<<<dim3(bx, (unsigned)chunks), 256, 0, st>>>(bmp, words, n, first, count, per, skip, bmp_set,
                                                                      cnt);
    return cudaGetLastError();
}

cudaError_t launch_bitmap_store(const SampleBatch& b, const BatchOut& o, uint64_t nbitmaps, uint32_t n, uint32_t* cnt,
                                const DeviceInfo& di, cudaStream_t st)
{
    if (nbitmaps == 0) return cudaSuccess;
    uint64_t grid = nbitmaps;
    if (grid > (uint64_t)di.sms * 8) grid = (uint64_t)di.sms * 8;
    bitmap_copy_kernel<<<(unsigned)grid, 256, 0, st>>>(b, o, nbitmaps);
    return launch_bitmap_count(o.bmp, b.words, n, o.bmp_base, nbitmaps, nullptr, nullptr, cnt, di, st);
}

// ===========================================================================
// Vertex scan: voff = exclusive prefix of a segment's per-vertex counts;
// also adds them into the stream's counter and zeroes the scatter cursors.
// ===========================================================================
__global__ void __launch_bounds__(kScanThreads)
vtx_tile_sum_kernel(const uint32_t* hist, uint32_t n, uint64_t* tile_sum)
{
    __shared__ uint64_t s_warp[32];
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTile;
    uint64_t a = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t v = t0 + (uint64_t)threadIdx.x * kScanItems + i;
        if (v < n) a += hist[v];
    }
    uint64_t tot;
    block_excl_scan64(a, s_warp, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads)
tile_excl_scan_kernel(uint64_t* tile, uint32_t ntiles)
{
    __shared__ uint64_t s_warp[32];
    __shared__ uint64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t t0 = 0; t0 < ntiles; t0 += kScanThreads) {
        const uint32_t t = t0 + threadIdx.x;
        const uint64_t x = t < ntiles ? tile[t] : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_scan64(x, s_warp, &tot);
        if (t < ntiles) tile[t] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads)
vtx_tile_write_kernel(const uint32_t* hist, uint32_t n, const uint64_t* tile_off, uint64_t* voff, uint32_t* cnt,
                      uint32_t* cnt2, uint32_t* cursor)
{
    __shared__ uint64_t s_warp[32];
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTile;
    uint32_t h[kScanItems];
    uint64_t a = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t v = t0 + (uint64_t)threadIdx.x * kScanItems + i;
        h[i] = v < n ? hist[v] : 0;
        a += h[i];
    }
    uint64_t tot;
    uint64_t ex = block_excl_scan64(a, s_warp, &tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t v = t0 + (uint64_t)threadIdx.x * kScanItems + i;
        if (v < n) {
            voff[v] = ex;
            if (cnt) cnt[v] += h[i];
            if (cnt2) cnt2[v] += h[i];
            cursor[v] = 0;
        }
        ex += h[i];
        if (v + 1 == n) voff[n] = ex;
    }
}

cudaError_t launch_vertex_scan(const uint32_t* hist, uint32_t n, uint64_t* voff, uint32_t* cnt, uint32_t* cnt2,
                               uint32_t* cursor, uint64_t* tmp, const DeviceInfo& di, cudaStream_t st)
{
    (void)di;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kScanTile - 1) / kScanTile);
    vtx_tile_sum_kernel<<<ntiles, kScanThreads, 0, st>>>(hist, n, tmp);
    tile_excl_scan_kernel<<<1, kScanThreads, 0, st>>>(tmp, ntiles);
    vtx_tile_write_kernel<<<ntiles, kScanThreads, 0, st>>>(hist, n, tmp, voff, cnt, cnt2, cursor);
    return cudaGetLastError();
}

// ===========================================================================
// Inverted index scatter over list-stored sets: for every member u of set s
// in [set_begin, set_end), inv[voff[u] + cursor[u]++] = s (one-pass counting
// sort by vertex; bitmap sets have empty lists and add nothing).
// ===========================================================================
__global__ void __launch_bounds__(256)
index_scatter_kernel(uint64_t set_begin, uint64_t set_end, const uint64_t* off, const uint32_t* arena,
                     const uint64_t* voff, uint32_t* cursor, uint32_t* inv, uint64_t inv_cap,
                     unsigned long long* err)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t first = set_begin + gw * 32; first < set_end; first += nw * 32) {
        const uint64_t s = first + lane;
        uint32_t len = 0;
        uint64_t a = 0;
        if (s < set_end) {
            a = off[s];
            len = (uint32_t)(off[s + 1] - a);
        }
        const bool big = len >= 32;
        uint32_t bigmask = __ballot_sync(kFull, big);
        while (bigmask) {
            const int o = __ffs(bigmask) - 1;
            bigmask &= bigmask - 1;
            const uint32_t L = __shfl_sync(kFull, len, o);
            const uint64_t A = shfl64(a, o);
            const uint32_t sid = (uint32_t)(first + o);
            for (uint32_t i = lane; i < L; i += 32) {
                const uint32_t u = arena[A + i];
                const uint64_t at = voff[u] + atomicAdd(&cursor[u], 1u);
                if (IMM_IN_BOUNDS(at, inv_cap, err, kChkInv)) inv[at] = sid;
            }
        }
        const uint32_t sl = big ? 0u : len;
        uint32_t incl = sl;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += t;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        const uint32_t excl = incl - sl;
        for (uint32_t j0 = 0; j0 < total; j0 += 32) {
            const uint32_t j = j0 + lane;
            const uint32_t o = owner_of(j, incl);
            const uint64_t A = shfl64(a, o);
            const uint32_t ex = __shfl_sync(kFull, excl, o);
            if (j < total) {
                const uint32_t u = arena[A + (j - ex)];
                const uint64_t at = voff[u] + atomicAdd(&cursor[u], 1u);
                if (IMM_IN_BOUNDS(at, inv_cap, err, kChkInv)) inv[at] = (uint32_t)(first + o);
            }
        }
    }
}

cudaError_t launch_index_scatter(uint64_t set_begin, uint64_t set_end, const uint64_t* off, const uint32_t* arena,
                                 const uint64_t* voff, uint32_t* cursor, uint32_t* inv, uint64_t inv_cap,
                                 unsigned long long* err, const DeviceInfo& di, cudaStream_t st)
{
    if (set_end <= set_begin) return cudaSuccess;
    const uint64_t warps = (set_end - set_begin + 31) / 32;
    uint64_t blocks = (warps + 7) / 8;
    const uint64_t cap = (uint64_t)di.sms * 16;
    if (blocks > cap) blocks = cap;
    index_scatter_kernel<<<(unsigned)blocks, 256, 0, st>>>(set_begin, set_end, off, arena, voff, cursor, inv, inv_cap,
                                                           err);
    return cudaGetLastError();
}

}  // namespace imm
