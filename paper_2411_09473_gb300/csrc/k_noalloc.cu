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
constexpr uint64_t kScratchBytes = kOffTotal + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Scratch {
    uint32_t* counts;
    uint8_t* picked;
    uint8_t* covered;
    unsigned long long* keys;
    unsigned long long* total;
};

// Device address of g_scratch, looked up once per device (with that device
// current); the host-side symbol itself is not a device address.
std::mutex g_mu;
void* g_addr[256];
bool g_ready[256];

int scratch_for_current_device(Scratch* s)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return IMM_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return IMM_ECUDA;
        }
        g_addr[dev] = p;
        g_ready[dev] = true;
    }
    unsigned char* base = static_cast<unsigned char*>(g_addr[dev]);
    s->counts = reinterpret_cast<uint32_t*>(base + kOffCounts);
    s->picked = base + kOffPicked;
    s->covered = base + kOffCovered;
    s->keys = reinterpret_cast<unsigned long long*>(base + kOffKeys);
    s->total = reinterpret_cast<unsigned long long*>(base + kOffTotal);
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
    if (t == 0) *s.total = 0;
}

// occurrence counts: one atomic increment per member
__global__ void na_count_kernel(Scratch s, uint64_t nsets, const uint64_t* off, const uint32_t* mem)
{
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t set = gw; set < nsets; set += nw) {
        const uint64_t a = off[set], b = off[set + 1];
        for (uint64_t i = a + lane; i < b; i += 32) atomicAdd(&s.counts[mem[i]], 1u);
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
__global__ void na_cover_kernel(Scratch s, uint64_t nsets, const uint64_t* off, const uint32_t* mem, uint32_t j,
                                uint32_t* seeds_out)
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
        for (uint64_t i = a + lane; i < b; i += 32) atomicSub(&s.counts[mem[i]], 1u);
        if (lane == 0) {
            s.covered[set] = 1;
            ++covered;
        }
    }
    if (lane == 0 && covered) atomicAdd(s.total, covered);
}

__global__ void na_finish_kernel(Scratch s, unsigned long long* covered_out)
{
    if (covered_out) *covered_out = *s.total;
}

}  // namespace
}  // namespace imm

extern "C" int imm_select_noalloc(uint32_t n, uint64_t nsets, const uint64_t* d_off, const uint32_t* d_members,
                                  uint32_t k, uint32_t* d_seeds_out, unsigned long long* d_covered_out, void* stream)
{
    using namespace imm;
    if (n == 0 || n > kMaxN || nsets > kMaxSets || k == 0 || k > n || k > kMaxK) return IMM_EINVAL;
    if (!d_off || !d_seeds_out || (nsets > 0 && !d_members)) return IMM_EINVAL;
    Scratch s;
    const int rc = scratch_for_current_device(&s);
    if (rc != IMM_OK) return rc;
    cudaDeviceProp prop;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return IMM_ECUDA;
    }
    const unsigned sms = (unsigned)prop.multiProcessorCount;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    na_clear_kernel<<<sms * 4, 256, 0, st>>>(s, n, nsets, k);
    if (nsets) na_count_kernel<<<sms * 8, 256, 0, st>>>(s, nsets, d_off, d_members);
    unsigned ab = (n + 255) / 256;
    if (ab > sms * 4) ab = sms * 4;
    for (uint32_t j = 0; j < k; ++j) {
        na_argmax_kernel<<<ab, 256, 0, st>>>(s, n, j);
        na_cover_kernel<<<sms * 8, 256, 0, st>>>(s, nsets, d_off, d_members, j, d_seeds_out);
    }
    na_finish_kernel<<<1, 1, 0, st>>>(s, d_covered_out);
    return cudaGetLastError() == cudaSuccess ? IMM_OK : IMM_ECUDA;
}
