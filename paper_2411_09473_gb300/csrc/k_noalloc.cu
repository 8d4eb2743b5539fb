// imm_select_noalloc: greedy max-coverage selection over a caller-provided,
// device-resident RRR-set system that allocates no device memory.
//
// Some callers cannot allocate device memory at run time: a plugin living
// inside another framework whose pool owns all of the GPU's memory, or a
// service whose memory footprint is fixed when it starts.  This entry point
// serves them.  Its scratch (per-vertex counts, picked and covered flags, the
// per-round argmax keys and the covered total) lives in one file-scope
// __device__ array of fixed size, which every GPU that loads the library
// holds until the process exits.  The caller passes the sets and the output
// buffers; nothing is allocated or freed.
//
// The kernels are a variant of the library's selection kernels: instead of
// an inverted index (which would need memory proportional to the stream),
// each round scans the uncovered sets for the pick, one warp per set.
#include <mutex>

#include "imm.h"
#include "imm_internal.cuh"

namespace imm {
namespace {

constexpr uint64_t kMaxN = IMM_NOALLOC_MAX_N;
constexpr uint64_t kMaxSets = IMM_NOALLOC_MAX_SETS;
constexpr uint64_t kMaxK = IMM_NOALLOC_MAX_K;

// scratch layout (bytes, each part 256-byte aligned)
constexpr uint64_t kOffCounts = 0;                                   // uint32[kMaxN]
constexpr uint64_t kOffPicked = kOffCounts + kMaxN * 4;              // uint8[kMaxN]
constexpr uint64_t kOffCovered = kOffPicked + kMaxN;                 // uint8[kMaxSets]
constexpr uint64_t kOffKeys = kOffCovered + kMaxSets;                // uint64[kMaxK]
constexpr uint64_t kOffTotal = kOffKeys + kMaxK * 8;                 // uint64
constexpr uint64_t kOffBad = kOffTotal + 8;                          // uint32: a member id >= n was seen
constexpr uint64_t kScratchBytes = kOffTotal + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Scratch {
    uint32_t* counts;
    uint8_t* picked;
    uint8_t* covered;
    unsigned long long* keys;
    unsigned long long* total;
    uint32_t* bad;
};

// Device address of g_scratch and the SM count, looked up once per device
// (with that device current); the host-side symbol itself is not a device
// address.  The cached address is not refreshed after a device reset.
std::mutex g_mu;
void* g_addr[256];
unsigned g_sms[256];
bool g_ready[256];

int scratch_for_current_device(Scratch* s, unsigned* sms)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return IMM_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
        void* p = nullptr;
        int count = 0;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr ||
            cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || count <= 0) {
            cudaGetLastError();
            return IMM_ECUDA;
        }
        g_addr[dev] = p;
        g_sms[dev] = (unsigned)count;
        g_ready[dev] = true;
    }
    *sms = g_sms[dev];
    unsigned char* base = static_cast<unsigned char*>(g_addr[dev]);
    s->counts = reinterpret_cast<uint32_t*>(base + kOffCounts);
    s->picked = base + kOffPicked;
    s->covered = base + kOffCovered;
    s->keys = reinterpret_cast<unsigned long long*>(base + kOffKeys);
    s->total = reinterpret_cast<unsigned long long*>(base + kOffTotal);
    s->bad = reinterpret_cast<uint32_t*>(base + kOffBad);
    return IMM_OK;
}

__global__ void na_clear_kernel(Scratch s, uint32_t n, uint64_t nsets, uint32_t k)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = t; i < n; i += stride) {
        s.counts[i] = 0;
        s.picked[i] = 0;
    }
    for (uint64_t i = t; i < nsets; i += stride) s.covered[i] = 0;
    for (uint64_t i = t; i < k; i += stride) s.keys[i] = 0;
    if (t == 0) {
        *s.total = 0;
        *s.bad = 0;
    }
}

// occurrence counts: one atomic increment per member; a member id >= n is
// not counted and raises the `bad` flag
__global__ void na_count_kernel(Scratch s, uint32_t n, uint64_t nsets, const uint64_t* off, const uint32_t* mem)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t set = gw; set < nsets; set += nw) {
        const uint64_t a = off[set], b = off[set + 1];
        for (uint64_t i = a + lane; i < b; i += 32) {
            const uint32_t u = mem[i];
            if (u < n) atomicAdd(&s.counts[u], 1u);
            else *s.bad = 1;
        }
    }
}

// argmax over vertices not yet picked; key = (count << 32) | (2^32 - 1 - v)
__global__ void na_argmax_kernel(Scratch s, uint32_t n, uint32_t j)
{
    __shared__ unsigned long long s_best[8];
    unsigned long long best = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (!s.picked[v]) {
            const unsigned long long key = ((unsigned long long)s.counts[v] << 32) | (0xFFFFFFFFu - v);
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
        if (lane == 0 && best) atomicMax(&s.keys[j], best);
    }
}

// every uncovered set holding the pick: mark covered, decrement its members
__global__ void na_cover_kernel(Scratch s, uint32_t n, uint64_t nsets, const uint64_t* off, const uint32_t* mem,
                                uint32_t j, uint32_t* seeds_out)
{
    const uint32_t v = 0xFFFFFFFFu - (uint32_t)s.keys[j];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.picked[v] = 1;
        seeds_out[j] = v;
    }
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long covered = 0;
    for (uint64_t set = gw; set < nsets; set += nw) {
        if (s.covered[set]) continue;
        const uint64_t a = off[set], b = off[set + 1];
        bool has = false;
        for (uint64_t i0 = a; i0 < b && !has; i0 += 32) {
            const uint64_t i = i0 + lane;
            has = __any_sync(kFull, i < b && mem[i] == v);
        }
        if (!has) continue;
        for (uint64_t i = a + lane; i < b; i += 32) {
            const uint32_t u = mem[i];
            if (u < n) atomicSub(&s.counts[u], 1u);
        }
        if (lane == 0) {
            s.covered[set] = 1;
            ++covered;
        }
    }
    if (lane == 0 && covered) atomicAdd(s.total, covered);
}

// the covered total; a set system with a member id >= n gets the error
// pattern instead (every seed 0xFFFFFFFF, covered 2^64 - 1)
__global__ void na_finish_kernel(Scratch s, uint32_t k, uint32_t* seeds_out, unsigned long long* covered_out)
{
    const bool bad = *s.bad != 0;
    if (bad)
        for (uint32_t j = threadIdx.x; j < k; j += blockDim.x) seeds_out[j] = 0xFFFFFFFFu;
    if (covered_out && threadIdx.x == 0) *covered_out = bad ? ~0ull : *s.total;
}

}  // namespace
}  // namespace imm

extern "C" int imm_select_noalloc(uint32_t n, uint64_t nsets, const uint64_t* d_off, const uint32_t* d_members,
                                  uint32_t k, uint32_t* d_seeds_out, unsigned long long* d_covered_out, void* stream)
{
    using namespace imm;
    if (n == 0 || n > kMaxN || nsets > kMaxSets || k == 0 || k > n || k > kMaxK) return IMM_EINVAL;
    if (!d_off || !d_seeds_out || (nsets > 0 && !d_members)) return IMM_EINVAL;
    // a launch error left by earlier, unrelated work on this host thread is
    // cleared here, so that it is not reported as this call's failure
    cudaGetLastError();
    Scratch s;
    unsigned sms = 0;
    const int rc = scratch_for_current_device(&s, &sms);
    if (rc != IMM_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    na_clear_kernel<<<sms * 4, 256, 0, st>>>(s, n, nsets, k);
    if (nsets) na_count_kernel<<<sms * 8, 256, 0, st>>>(s, n, nsets, d_off, d_members);
    if (cudaGetLastError() != cudaSuccess) return IMM_ECUDA;
    unsigned ab = (n + 255) / 256;
    if (ab > sms * 4) ab = sms * 4;
    for (uint32_t j = 0; j < k; ++j) {
        na_argmax_kernel<<<ab, 256, 0, st>>>(s, n, j);
        na_cover_kernel<<<sms * 8, 256, 0, st>>>(s, n, nsets, d_off, d_members, j, d_seeds_out);
        // a failed launch stops the call before the later rounds are enqueued
        if (cudaGetLastError() != cudaSuccess) return IMM_ECUDA;
    }
    na_finish_kernel<<<1, 256, 0, st>>>(s, k, d_seeds_out, d_covered_out);
    return cudaGetLastError() == cudaSuccess ? IMM_OK : IMM_ECUDA;
}
