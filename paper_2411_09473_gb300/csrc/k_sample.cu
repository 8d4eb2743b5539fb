// RRR-set sampling kernels (Generate_RRRsets, EfficientIMM Alg. 3) and the
// prefix-sum compaction of the sampled sets into the device arena.
//
// A batch of consecutive set ids is sampled in two passes:
//   small path  one warp per set (IC) or one lane per walk (LT); the visited
//               state lives in shared memory (open-addressing hash / path
//               list).  A set that outgrows it is handed to the large path.
//   large path  one CTA per set (IC) with an n-bit visited bitmap in shared
//               memory when it fits, else in a per-CTA global slot; one thread
//               per walk (LT) with a global bitmap.
// Each finished set is written to a staging buffer; the batch scan turns the
// set lengths into arena offsets and the compaction kernel copies members to
// the arena in set-id order while counting occurrences (Alg. 3 fused count).
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

__device__ __forceinline__ uint4 load_thr4(const uint32_t* thr, uint64_t quad)
{
    return __ldg(reinterpret_cast<const uint4*>(thr) + quad);
}

// Reserve staging space for a finished set.  On overflow the set is marked
// failed; it and every later set of the batch are resampled by the next batch.
__device__ __forceinline__ bool reserve_stage(const SampleBatch& b, uint32_t rel, uint32_t len, uint64_t* pos)
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
    return true;
}

// ===========================================================================
// IC, small path: one warp per set.
// ===========================================================================
constexpr int kSmallWarps = 8;
constexpr uint32_t kSmallCap = 256;          // members a warp keeps before handing off
constexpr int kSmallHashBits = 9;
constexpr uint32_t kSmallHash = 1u << kSmallHashBits;  // > kSmallCap + 4*32 (one inner step)

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
    const uint2 key = philox_key(b.seed);

    for (uint32_t i = lane; i < kSmallHash; i += 32) hash[i] = kEmpty;
    __syncwarp();

    for (;;) {
        uint32_t rel = 0;
        if (lane == 0) rel = atomicAdd(&b.sc->cursor, 1u);
        rel = __shfl_sync(kFull, rel, 0);
        if (rel >= b.count) break;
        const uint64_t s = b.base + rel;
        const uint32_t s_lo = (uint32_t)s, s_hi = (uint32_t)(s >> 32);
        if (lane == 0) {
            const uint32_t root = draw_root(b.seed, s, g.n);
            const uint32_t sl = small_slot(root);
            hash[sl] = root;
            list[0] = root;
            lslot[0] = (uint16_t)sl;
        }
        __syncwarp();

        uint32_t head = 0, tail = 1;
        uint64_t edges = 0;  // lane-partial sum of in-degrees of expanded members
        bool overflow = false;
        while (head < tail && !overflow) {
            // Up to 32 frontier vertices; their in-edge quads are flattened
            // across the warp so short and long adjacency lists share lanes.
            const uint32_t nf = min(tail - head, 32u);
            uint64_t rs = 0, re = 0;
            uint32_t nq = 0;
            if ((uint32_t)lane < nf) {
                const uint32_t v = list[head + lane];
                rs = g.row[v];
                re = g.row[v + 1];
                if (re > rs) nq = (uint32_t)(((re - 1) >> 2) - (rs >> 2) + 1);
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
                const uint64_t ors = shfl64(rs, o);
                const uint64_t ore = shfl64(re, o);
                const uint32_t oex = __shfl_sync(kFull, excl, o);
                const bool active = j < total;
                uint4 w = make_uint4(0, 0, 0, 0), th = make_uint4(0, 0, 0, 0);
                uint64_t e0 = 0;
                if (active) {
                    const uint64_t quad = (ors >> 2) + (j - oex);
                    e0 = quad << 2;
                    w = philox(make_uint4(s_lo, s_hi, (uint32_t)quad, kTagIC), key);
                    th = load_thr4(g.thr, quad);
                }
                const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
                const uint32_t tv[4] = {th.x, th.y, th.z, th.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint64_t e = e0 + t;
                    const bool live = active && e >= ors && e < ore && (wv[t] >> 8) < tv[t];
                    bool isnew = false;
                    uint32_t u = 0, sl = 0;
                    if (live) {
                        u = __ldg(g.src + e);
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
                b.large_q[qi] = rel;
                b.set_len[rel] = kLenPending;
            }
            for (uint32_t i = lane; i < kSmallHash; i += 32) hash[i] = kEmpty;
        } else {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) edges += __shfl_xor_sync(kFull, edges, d);
            uint64_t pos = 0;
            int ok = 0;
            if (lane == 0) {
                b.set_edges[rel] = (uint32_t)edges;
                ok = reserve_stage(b, rel, tail, &pos) ? 1 : 0;
            }
            ok = __shfl_sync(kFull, ok, 0);
            pos = shfl64(pos, 0);
            if (ok)
                for (uint32_t i = lane; i < tail; i += 32) b.stage[pos + i] = list[i];
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
// IC, large path: one CTA per set, queue-driven BFS.
// ===========================================================================
constexpr int kLargeThreads = 1024;
constexpr int kLargeWarps = kLargeThreads / 32;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += t;
    }
    return x;
}

template <bool kSmemBitmap>
__global__ void __launch_bounds__(kLargeThreads, 1)
ic_large_kernel(DevGraph g, SampleBatch b, LargeSlots ls)
{
    extern __shared__ __align__(16) uint32_t dyn_bitmap[];
    __shared__ uint64_t s_rs[kLargeThreads];
    __shared__ uint64_t s_re[kLargeThreads];
    __shared__ uint32_t s_excl[kLargeThreads + 1];
    __shared__ uint32_t s_warp[kLargeWarps];
    __shared__ uint32_t s_tail;
    __shared__ uint32_t s_claim;
    __shared__ int s_ok;
    __shared__ unsigned long long s_pos;
    __shared__ unsigned long long s_edges;

    const uint32_t tid = threadIdx.x;
    const int lane = tid & 31;
    const int wid = tid >> 5;
    const uint32_t ltm = lanemask_lt();
    const uint64_t words = ((uint64_t)g.n + 31) >> 5;
    uint32_t* bm = kSmemBitmap ? dyn_bitmap : ls.bitmaps + (uint64_t)blockIdx.x * ls.bitmap_words;
    uint32_t* q = ls.queues + (uint64_t)blockIdx.x * ls.queue_cap;
    const uint2 key = philox_key(b.seed);
    const uint32_t large_count = b.sc->large_count;  // final: written by the previous launch

    if (kSmemBitmap)
        for (uint64_t i = tid; i < words; i += kLargeThreads) bm[i] = 0;

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
        const uint32_t s_lo = (uint32_t)s, s_hi = (uint32_t)(s >> 32);
        if (tid == 0) {
            const uint32_t root = draw_root(b.seed, s, g.n);
            q[0] = root;
            bm[root >> 5] |= 1u << (root & 31);
            s_tail = 1;
        }
        __syncthreads();

        uint32_t head = 0, tail = 1;
        uint64_t edges = 0;
        while (head < tail) {
            const uint32_t nf = min(tail - head, (uint32_t)kLargeThreads);
            uint32_t nq = 0;
            if (tid < nf) {
                const uint32_t v = q[head + tid];
                const uint64_t rs = g.row[v], re = g.row[v + 1];
                s_rs[tid] = rs;
                s_re[tid] = re;
                if (re > rs) nq = (uint32_t)(((re - 1) >> 2) - (rs >> 2) + 1);
                edges += re - rs;
            }
            const uint32_t incl = warp_incl_scan(nq, lane);
            if (lane == 31) s_warp[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                const uint32_t x = warp_incl_scan(s_warp[lane], lane);
                s_warp[lane] = x;
            }
            __syncthreads();
            const uint32_t wbase = wid ? s_warp[wid - 1] : 0u;
            s_excl[tid] = wbase + incl - nq;
            const uint32_t total = s_warp[kLargeWarps - 1];
            if (tid == 0) s_excl[kLargeThreads] = total;
            __syncthreads();

            for (uint32_t j0 = (uint32_t)wid * 32u; j0 < total; j0 += kLargeThreads) {
                const uint32_t j = j0 + lane;
                const bool active = j < total;
                uint4 w = make_uint4(0, 0, 0, 0), th = make_uint4(0, 0, 0, 0);
                uint64_t e0 = 0, ors = 0, ore = 0;
                if (active) {
                    // owner: last frontier slot whose exclusive prefix is <= j
                    uint32_t lo = 0, hi = nf;
                    while (hi - lo > 1) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (s_excl[mid] <= j) lo = mid;
                        else hi = mid;
                    }
                    ors = s_rs[lo];
                    ore = s_re[lo];
                    const uint64_t quad = (ors >> 2) + (j - s_excl[lo]);
                    e0 = quad << 2;
                    w = philox(make_uint4(s_lo, s_hi, (uint32_t)quad, kTagIC), key);
                    th = load_thr4(g.thr, quad);
                }
                const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
                const uint32_t tv[4] = {th.x, th.y, th.z, th.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint64_t e = e0 + t;
                    const bool live = active && e >= ors && e < ore && (wv[t] >> 8) < tv[t];
                    bool isnew = false;
                    uint32_t u = 0;
                    if (live) {
                        u = __ldg(g.src + e);
                        const uint32_t bit = 1u << (u & 31);
                        const uint32_t old = atomicOr(&bm[u >> 5], bit);
                        isnew = (old & bit) == 0;
                    }
                    const uint32_t nm = __ballot_sync(kFull, isnew);
                    if (nm) {
                        uint32_t base = 0;
                        if (lane == 0) base = atomicAdd(&s_tail, (uint32_t)__popc(nm));
                        base = __shfl_sync(kFull, base, 0);
                        if (isnew) q[base + __popc(nm & ltm)] = u;
                    }
                }
            }
            __syncthreads();
            head += nf;
            tail = s_tail;
        }

        // set done: record, stage, clear the visited bits
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) edges += __shfl_xor_sync(kFull, edges, d);
        if (lane == 0 && edges) atomicAdd(&s_edges, (unsigned long long)edges);
        __syncthreads();
        if (tid == 0) {
            b.set_edges[rel] = (uint32_t)s_edges;
            uint64_t pos = 0;
            s_ok = reserve_stage(b, rel, tail, &pos) ? 1 : 0;
            s_pos = pos;
        }
        __syncthreads();
        if (s_ok) {
            const uint64_t pos = s_pos;
            for (uint32_t i = tid; i < tail; i += kLargeThreads) b.stage[pos + i] = q[i];
        }
        if (kSmemBitmap || (uint64_t)tail * 8 >= words) {
            for (uint64_t i = tid; i < words; i += kLargeThreads) bm[i] = 0;
        } else {
            for (uint32_t i = tid; i < tail; i += kLargeThreads) bm[q[i] >> 5] = 0;
        }
        __syncthreads();
    }
}

static size_t large_smem_bytes(uint32_t n)
{
    const uint64_t words = ((uint64_t)n + 31) >> 5;
    return (size_t)(((words * 4) + 15) / 16 * 16);
}

int ic_large_uses_smem(uint32_t n, const DeviceInfo& di)
{
    // static shared memory of the kernel is ~20.7 KB; keep 1 KB of slack
    const size_t static_bytes = sizeof(uint64_t) * 2 * kLargeThreads + sizeof(uint32_t) * (kLargeThreads + 1) +
                                sizeof(uint32_t) * kLargeWarps + 64;
    return large_smem_bytes(n) + static_bytes + 1024 <= (size_t)di.max_smem_optin;
}

cudaError_t launch_ic_large(const DevGraph& g, const SampleBatch& b, const LargeSlots& ls, const DeviceInfo& di,
                            cudaStream_t st)
{
    const unsigned grid = ls.nslots;
    if (ic_large_uses_smem(g.n, di)) {
        const size_t smem = large_smem_bytes(g.n);
        cudaError_t e = cudaFuncSetAttribute(ic_large_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        ic_large_kernel<true><<<grid, kLargeThreads, smem, st>>>(g, b, ls);
    } else {
        ic_large_kernel<false><<<grid, kLargeThreads, 0, st>>>(g, b, ls);
    }
    return cudaGetLastError();
}

// ===========================================================================
// LT, small path: one lane per walk, path kept in shared memory.
// ===========================================================================
constexpr int kLtThreads = 128;
constexpr uint32_t kLtCap = 48;

// first j in [lo, hi) with r < cthr[j] (cthr is nondecreasing), or hi
__device__ __forceinline__ uint64_t lt_pick(const uint32_t* cthr, uint64_t lo, uint64_t hi, uint32_t r)
{
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (r < __ldg(cthr + mid)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kLtThreads)
lt_small_kernel(DevGraph g, SampleBatch b)
{
    __shared__ uint32_t path[kLtCap][kLtThreads];
    const uint32_t tid = threadIdx.x;
    const int lane = tid & 31;
    const uint32_t ltm = lanemask_lt();
    const uint2 key = philox_key(b.seed);
    bool busy = false, done = false;
    uint32_t rel = 0, len = 0, v = 0;
    uint64_t s = 0;
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
                    s = b.base + rel;
                    v = draw_root(b.seed, s, g.n);
                    path[0][tid] = v;
                    len = 1;
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(kFull, done)) break;
        if (!busy) continue;
        // one step of the reverse walk at v
        const uint4 w = philox(make_uint4((uint32_t)s, (uint32_t)(s >> 32), v, kTagLT), key);
        const uint64_t lo = g.row[v], hi = g.row[v + 1];
        const uint64_t pick = lt_pick(g.thr, lo, hi, w.x >> 8);
        bool stop = pick == hi;
        uint32_t u = 0;
        if (!stop) {
            u = __ldg(g.src + pick);
            for (uint32_t i = 0; i < len; ++i)
                if (path[i][tid] == u) {
                    stop = true;
                    break;
                }
        }
        if (!stop) {
            if (len == kLtCap) {
                const uint32_t qi = atomicAdd(&b.sc->large_count, 1u);
                b.large_q[qi] = rel;
                b.set_len[rel] = kLenPending;
                busy = false;
            } else {
                path[len][tid] = u;
                ++len;
                v = u;
            }
        } else {
            b.set_edges[rel] = len;
            uint64_t pos = 0;
            if (reserve_stage(b, rel, len, &pos))
                for (uint32_t i = 0; i < len; ++i) b.stage[pos + i] = path[i][tid];
            busy = false;
        }
    }
}

cudaError_t launch_lt_small(const DevGraph& g, const SampleBatch& b, const DeviceInfo& di, cudaStream_t st)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lt_small_kernel, kLtThreads, 0);
    if (e != cudaSuccess) return e;
    const uint64_t want = ((uint64_t)b.count + kLtThreads - 1) / kLtThreads;
    uint64_t grid = (uint64_t)di.sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    if (grid > want) grid = want;
    if (grid == 0) grid = 1;
    lt_small_kernel<<<(unsigned)grid, kLtThreads, 0, st>>>(g, b);
    return cudaGetLastError();
}

// ===========================================================================
// LT, long walks: one thread per walk with an n-bit global bitmap slot.
// ===========================================================================
__global__ void __launch_bounds__(32)
lt_long_kernel(DevGraph g, SampleBatch b, LargeSlots ls)
{
    const int lane = threadIdx.x;
    uint32_t* bm = ls.bitmaps + (uint64_t)blockIdx.x * ls.bitmap_words;
    uint32_t* q = ls.queues + (uint64_t)blockIdx.x * ls.queue_cap;
    const uint2 key = philox_key(b.seed);
    const uint32_t large_count = b.sc->large_count;
    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(&b.sc->large_cursor, 1u);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= large_count) break;
        const uint32_t rel = b.large_q[idx];
        const uint64_t s = b.base + rel;
        uint32_t len = 0;
        if (lane == 0) {
            uint32_t v = draw_root(b.seed, s, g.n);
            q[0] = v;
            bm[v >> 5] |= 1u << (v & 31);
            len = 1;
            for (;;) {
                const uint4 w = philox(make_uint4((uint32_t)s, (uint32_t)(s >> 32), v, kTagLT), key);
                const uint64_t lo = g.row[v], hi = g.row[v + 1];
                const uint64_t pick = lt_pick(g.thr, lo, hi, w.x >> 8);
                if (pick == hi) break;
                const uint32_t u = __ldg(g.src + pick);
                const uint32_t bit = 1u << (u & 31);
                if (bm[u >> 5] & bit) break;
                bm[u >> 5] |= bit;
                q[len++] = u;
                v = u;
            }
            b.set_edges[rel] = len;
        }
        len = __shfl_sync(kFull, len, 0);
        uint64_t pos = 0;
        int ok = 0;
        if (lane == 0) ok = reserve_stage(b, rel, len, &pos) ? 1 : 0;
        ok = __shfl_sync(kFull, ok, 0);
        pos = shfl64(pos, 0);
        __syncwarp();
        if (ok)
            for (uint32_t i = lane; i < len; i += 32) b.stage[pos + i] = q[i];
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
// Batch scan: exclusive prefix of the kept sets' lengths -> arena offsets.
// Kept sets are ids [0, committed), committed = min(first_fail, count).
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
    return 2 * ((uint64_t)count / kScanTile + 2) + 8;
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

__global__ void __launch_bounds__(kScanThreads)
batch_tile_sum_kernel(SampleBatch b, uint64_t* tile_len, uint64_t* tile_edges)
{
    __shared__ uint64_t s_warp[32];
    const uint32_t committed = batch_committed(b);
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTile;
    uint64_t a = 0, ed = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t r = t0 + (uint64_t)threadIdx.x * kScanItems + i;
        if (r < committed) {
            a += b.set_len[r];
            ed += b.set_edges[r];
        }
    }
    uint64_t tot_a, tot_e;
    block_excl_scan64(a, s_warp, &tot_a);
    block_excl_scan64(ed, s_warp, &tot_e);
    if (threadIdx.x == 0) {
        tile_len[blockIdx.x] = tot_a;
        tile_edges[blockIdx.x] = tot_e;
    }
}

// one block: exclusive scan of the tile sums, and the batch totals
__global__ void __launch_bounds__(kScanThreads)
batch_tile_scan_kernel(SampleBatch b, uint64_t* tile_len, const uint64_t* tile_edges, uint32_t ntiles)
{
    __shared__ uint64_t s_warp[32];
    __shared__ uint64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    uint64_t edges = 0;
    for (uint32_t t0 = 0; t0 < ntiles; t0 += kScanThreads) {
        const uint32_t t = t0 + threadIdx.x;
        const uint64_t x = t < ntiles ? tile_len[t] : 0;
        if (t < ntiles) edges += tile_edges[t];
        uint64_t tot;
        const uint64_t ex = block_excl_scan64(x, s_warp, &tot);
        if (t < ntiles) tile_len[t] = s_carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
    uint64_t tot_e;
    block_excl_scan64(edges, s_warp, &tot_e);
    if (threadIdx.x == 0) {
        b.sc->members = s_carry;
        b.sc->committed = batch_committed(b);
        b.sc->edges = tot_e;
    }
}

__global__ void __launch_bounds__(kScanThreads)
batch_tile_write_kernel(SampleBatch b, const uint64_t* tile_off, uint64_t* off)
{
    __shared__ uint64_t s_warp[32];
    const uint32_t committed = batch_committed(b);
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTile;
    uint64_t v[kScanItems];
    uint64_t a = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t r = t0 + (uint64_t)threadIdx.x * kScanItems + i;
        v[i] = r < committed ? b.set_len[r] : 0;
        a += v[i];
    }
    uint64_t tot;
    uint64_t ex = block_excl_scan64(a, s_warp, &tot);
    const uint64_t base = off[b.base] + tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t r = t0 + (uint64_t)threadIdx.x * kScanItems + i;
        ex += v[i];
        if (r < committed) off[b.base + r + 1] = base + ex;
    }
}

cudaError_t launch_batch_scan(const SampleBatch& b, uint64_t* off, uint64_t* tmp, const DeviceInfo& di,
                              cudaStream_t st)
{
    (void)di;
    const uint32_t ntiles = (uint32_t)(((uint64_t)b.count + kScanTile - 1) / kScanTile);
    uint64_t* tile_len = tmp;
    uint64_t* tile_edges = tmp + ntiles + 1;
    batch_tile_sum_kernel<<<ntiles, kScanThreads, 0, st>>>(b, tile_len, tile_edges);
    batch_tile_scan_kernel<<<1, kScanThreads, 0, st>>>(b, tile_len, tile_edges, ntiles);
    batch_tile_write_kernel<<<ntiles, kScanThreads, 0, st>>>(b, tile_len, off);
    return cudaGetLastError();
}

// ===========================================================================
// Compaction: staging -> arena in set-id order, fused occurrence count.
// A warp takes 32 consecutive sets: sets of >= 32 members are copied by the
// whole warp one at a time; the shorter ones are flattened across lanes.
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

__global__ void __launch_bounds__(256)
compact_kernel(SampleBatch b, uint64_t committed, const uint64_t* off, uint32_t* arena, uint32_t* hist)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t first = gw * 32; first < committed; first += nw * 32) {
        const uint64_t rel = first + lane;
        uint32_t len = 0;
        uint64_t pos = 0, dst = 0;
        if (rel < committed) {
            len = b.set_len[rel];
            pos = b.set_pos[rel];
            dst = off[b.base + rel];
        }
        const bool big = len >= 32;
        uint32_t bigmask = __ballot_sync(kFull, big);
        while (bigmask) {
            const int o = __ffs(bigmask) - 1;
            bigmask &= bigmask - 1;
            const uint32_t L = __shfl_sync(kFull, len, o);
            const uint64_t P = shfl64(pos, o), D = shfl64(dst, o);
            for (uint32_t i = lane; i < L; i += 32) {
                const uint32_t u = b.stage[P + i];
                arena[D + i] = u;
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
            const uint64_t P = shfl64(pos, o), D = shfl64(dst, o);
            const uint32_t ex = __shfl_sync(kFull, excl, o);
            if (j < total) {
                const uint32_t u = b.stage[P + (j - ex)];
                arena[D + (j - ex)] = u;
                atomicAdd(&hist[u], 1u);
            }
        }
    }
}

cudaError_t launch_compact(const SampleBatch& b, uint64_t committed, const uint64_t* off, uint32_t* arena,
                           uint32_t* hist, const DeviceInfo& di, cudaStream_t st)
{
    if (committed == 0) return cudaSuccess;
    uint64_t warps = (committed + 31) / 32;
    uint64_t blocks = (warps + 7) / 8;
    const uint64_t cap = (uint64_t)di.sms * 16;
    if (blocks > cap) blocks = cap;
    compact_kernel<<<(unsigned)blocks, 256, 0, st>>>(b, committed, off, arena, hist);
    return cudaGetLastError();
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
tile_excl_scan_kernel(uint64_t* tile, uint32_t ntiles, uint64_t* grand_total)
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
    if (threadIdx.x == 0 && grand_total) *grand_total = s_carry;
}

__global__ void __launch_bounds__(kScanThreads)
vtx_tile_write_kernel(const uint32_t* hist, uint32_t n, const uint64_t* tile_off, uint64_t* voff, uint32_t* cnt,
                      uint32_t* cursor)
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
            cursor[v] = 0;
        }
        ex += h[i];
        if (v + 1 == n) voff[n] = ex;
    }
}

cudaError_t launch_vertex_scan(const uint32_t* hist, uint32_t n, uint64_t* voff, uint32_t* cnt, uint32_t* cursor,
                               uint64_t* tmp, const DeviceInfo& di, cudaStream_t st)
{
    (void)di;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kScanTile - 1) / kScanTile);
    vtx_tile_sum_kernel<<<ntiles, kScanThreads, 0, st>>>(hist, n, tmp);
    tile_excl_scan_kernel<<<1, kScanThreads, 0, st>>>(tmp, ntiles, nullptr);
    vtx_tile_write_kernel<<<ntiles, kScanThreads, 0, st>>>(hist, n, tmp, voff, cnt, cursor);
    return cudaGetLastError();
}

// ===========================================================================
// Inverted index scatter: for every member u of set s in [set_begin,
// set_end), inv[voff[u] + cursor[u]++] = s (one-pass counting sort by vertex).
// ===========================================================================
__global__ void __launch_bounds__(256)
index_scatter_kernel(uint64_t set_begin, uint64_t set_end, const uint64_t* off, const uint32_t* arena,
                     const uint64_t* voff, uint32_t* cursor, uint32_t* inv)
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
                inv[voff[u] + atomicAdd(&cursor[u], 1u)] = sid;
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
                inv[voff[u] + atomicAdd(&cursor[u], 1u)] = (uint32_t)(first + o);
            }
        }
    }
}

cudaError_t launch_index_scatter(uint64_t set_begin, uint64_t set_end, const uint64_t* off, const uint32_t* arena,
                                 const uint64_t* voff, uint32_t* cursor, uint32_t* inv, const DeviceInfo& di,
                                 cudaStream_t st)
{
    if (set_end <= set_begin) return cudaSuccess;
    const uint64_t warps = (set_end - set_begin + 31) / 32;
    uint64_t blocks = (warps + 7) / 8;
    const uint64_t cap = (uint64_t)di.sms * 16;
    if (blocks > cap) blocks = cap;
    index_scatter_kernel<<<(unsigned)blocks, 256, 0, st>>>(set_begin, set_end, off, arena, voff, cursor, inv);
    return cudaGetLastError();
}

}  // namespace imm
