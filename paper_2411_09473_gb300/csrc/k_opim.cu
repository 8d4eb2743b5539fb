// Coverage of a seed set over a stored RRR-set stream: the number of sets
// that hold at least one of the seeds.  OPIM's early stop (Sec. VI cites
// OPIM, Tang et al. 2018) measures the greedy's seed set on a second,
// independent collection with it, as the lower confidence bound on the set's
// spread needs that collection's coverage.
//
// One warp per set.  A list-stored set is scanned for a member whose flag is
// set (flags: one byte per vertex, 1 for the seeds); a bitmap-stored set
// tests the seeds' bits, one seed per lane.  Each warp adds its count once.
#include "imm_internal.cuh"

namespace imm {

__global__ void __launch_bounds__(256)
coverage_kernel(CoverageArgs a)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long hits = 0;
    for (uint64_t s = gw; s < a.nsets; s += nw) {
        const uint32_t bid = a.set_bmp[s];
        bool hit = false;
        if (bid == kEmpty) {
            const uint64_t b = a.off[s], e = a.off[s + 1];
            for (uint64_t i0 = b; i0 < e && !hit; i0 += 32) {
                const uint64_t i = i0 + lane;
                hit = __any_sync(kFull, i < e && a.flag[a.arena[i]] != 0);
            }
        } else {
            const uint32_t* words = a.bmp + (uint64_t)bid * a.words;
            for (uint32_t j0 = 0; j0 < a.k && !hit; j0 += 32) {
                const uint32_t j = j0 + lane;
                bool in = false;
                if (j < a.k) {
                    const uint32_t v = a.seeds[j];
                    in = (words[v >> 5] >> (v & 31u)) & 1u;
                }
                hit = __any_sync(kFull, in);
            }
        }
        hits += hit ? 1u : 0u;
    }
    if (lane == 0 && hits) atomicAdd(a.out, hits);
}

cudaError_t launch_coverage(const CoverageArgs& a, const DeviceInfo& di, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(a.out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (a.nsets == 0) return cudaSuccess;
    const uint64_t warps = a.nsets;
    uint64_t blocks = (warps + 7) / 8;
    const uint64_t cap = (uint64_t)di.sms * 8;
    if (blocks > cap) blocks = cap;
    coverage_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace imm
