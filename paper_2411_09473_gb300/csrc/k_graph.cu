// Graph load kernels: CSR validation and per-edge integer thresholds.
//
// IC (Sec. II-A): in-edge e is live with probability p_e.  The coin compares
// a 24-bit draw with thr[e] = ceilf(p_e * 2^24); the product by a power of two
// is exact in fp32, so thr/2^24 is p_e rounded up to the 24-bit grid.
// LT (Sec. II-A): a head keeps at most one in-edge, edge j with probability
// w_j.  cthr[j] = min(ceil(cw_j * 2^24), 2^24) where cw_j is the fp64 running
// sum of the head's fp32 weights in CSR order; the first j with draw < cthr[j]
// is the kept edge.
#include "imm_internal.cuh"

namespace imm {

constexpr int kFlagRow = 1;      // row not monotone / row[0] != 0 / row[n] != m
constexpr int kFlagSrc = 2;      // src >= n
constexpr int kFlagWeight = 4;   // NaN, < 0 or > 1
constexpr int kFlagLtSum = 8;    // LT head sum > 1 + 1e-6

__global__ void validate_rows_kernel(const uint64_t* row, uint32_t n, uint64_t m, int* flags)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (row[v + 1] < row[v]) atomicOr(flags, kFlagRow);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (row[0] != 0 || row[n] != m) atomicOr(flags, kFlagRow);
    }
}

__global__ void validate_edges_kernel(const uint32_t* src, const float* w, uint32_t n, uint64_t m, int* flags)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    int f = 0;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        if (src[e] >= n) f |= kFlagSrc;
        const float x = w[e];
        if (!(x >= 0.0f && x <= 1.0f)) f |= kFlagWeight;
    }
    if (f) atomicOr(flags, f);
}

cudaError_t launch_validate_graph(const uint64_t* row, const uint32_t* src, const float* w, uint32_t n,
                                  uint64_t m, int model, int* d_flags, cudaStream_t st)
{
    (void)model;
    validate_rows_kernel<<<1024, 256, 0, st>>>(row, n, m, d_flags);
    if (m) validate_edges_kernel<<<2048, 256, 0, st>>>(src, w, n, m, d_flags);
    return cudaGetLastError();
}

__global__ void ic_threshold_kernel(const float* w, uint64_t m, uint32_t* thr)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        thr[e] = (uint32_t)ceilf(__fmul_rn(w[e], 16777216.0f));
    }
}

// One warp per head.  The running sum is sequential by definition, but when
// every weight of the head is 0 or at least 2^-29 (so a multiple of 2^-52)
// and the head's sum is below 2, every partial sum is a multiple of 2^-52
// below 2, which fp64 holds exactly: no addition rounds, and a warp scan in
// any order gives the sequential sums bit for bit.  Other heads take the
// sequential loop on one lane.
__global__ void __launch_bounds__(256)
lt_threshold_kernel(const uint64_t* row, const float* w, uint32_t n, uint32_t* cthr, int* flags)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = gw; v < n; v += nw) {
        const uint64_t lo = row[v], hi = row[v + 1];
        bool ok = true;
        double part = 0.0;
        for (uint64_t e = lo + lane; e < hi; e += 32) {
            const float x = w[e];
            ok = ok && (x == 0.0f || (x >= 0x1p-29f && x <= 1.0f));
            part = __dadd_rn(part, (double)x);
        }
        ok = __all_sync(kFull, ok);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) part = __dadd_rn(part, __shfl_xor_sync(kFull, part, d));
        if (ok && part < 2.0) {
            double carry = 0.0;
            for (uint64_t e0 = lo; e0 < hi; e0 += 32) {
                const uint64_t e = e0 + lane;
                double x = e < hi ? (double)w[e] : 0.0;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const double y = __shfl_up_sync(kFull, x, d);
                    if ((int)lane >= d) x = __dadd_rn(x, y);
                }
                if (e < hi) {
                    const double t = ceil(__dmul_rn(__dadd_rn(carry, x), 16777216.0));
                    cthr[e] = t > 16777216.0 ? kQ24 : (uint32_t)t;
                }
                carry = __dadd_rn(carry, __shfl_sync(kFull, x, 31));
            }
            if (lane == 0 && part > 1.0 + 1e-6) atomicOr(flags, kFlagLtSum);
        } else if (lane == 0) {
            double cw = 0.0;
            for (uint64_t e = lo; e < hi; ++e) {
                cw = __dadd_rn(cw, (double)w[e]);
                const double t = ceil(__dmul_rn(cw, 16777216.0));
                cthr[e] = t > 16777216.0 ? kQ24 : (uint32_t)t;
            }
            if (cw > 1.0 + 1e-6) atomicOr(flags, kFlagLtSum);
        }
    }
}

cudaError_t launch_thresholds(const uint64_t* row, const float* w, uint32_t n, uint64_t m, int model,
                              uint32_t* thr, int* d_flags, cudaStream_t st)
{
    if (model == 0) {
        if (m) ic_threshold_kernel<<<2048, 256, 0, st>>>(w, m, thr);
    } else {
        uint64_t blocks = ((uint64_t)n + 7) / 8;  // 8 warps (heads) per block
        if (blocks > 65535ull * 16) blocks = 65535ull * 16;
        if (blocks == 0) blocks = 1;
        lt_threshold_kernel<<<(unsigned)blocks, 256, 0, st>>>(row, w, n, thr, d_flags);
    }
    return cudaGetLastError();
}

// LT guide table (index-assisted inverse transform; Chen & Asau 1974): for a
// head v of in-degree d, bucket b < d covers the 24-bit draws r with
// floor(r * d / 2^24) = b, whose smallest is lo_b = ceil(b * 2^24 / d).  The
// entry of bucket b is (j, cthr[j], src[j], 0) for j = the first in-edge of v
// with cthr[j] > lo_b, packed with u = src[j] as (j, cthr[j] | deg(u) << 25,
// u, row[u]): the tail u and u's in-edge range, which the walk's next step
// needs.  deg(u) takes the 7 bits above cthr and, for heads of fewer than
// 2^16 in-edges (j stored relative to row[v] in the low 16 bits of x), the 16
// high bits of x as well; its top value stands for "read u's row".  A draw r in bucket b
// has its answer (the first j with r < cthr[j]) at that j whenever r <
// cthr[j], which the entry tells with the next vertex in hand; otherwise the
// scan continues over cthr from j + 1.  The same answer as a search over all
// of v's in-edges, usually in one read.

// Number of buckets b of a head of in-degree d whose smallest draw
// lo_b = ceil(b * 2^24 / d) is below t: floor((t - 1) d / 2^24) + 1 (0 for
// t = 0).  In-edge j is the entry of exactly the buckets with
// cthr[j-1] <= lo_b < cthr[j], i.e. b in [nb(cthr[j-1]), nb(cthr[j])) (the
// first in-edge from 0); buckets from nb(cthr[last]) on have no in-edge.
__device__ __forceinline__ uint64_t guide_nb(uint32_t t, uint64_t d)
{
    return t == 0u ? 0ull : (((uint64_t)(t - 1u) * d) >> 24) + 1ull;
}

// One warp per head, its lanes over the in-edges: each in-edge writes the
// buckets it answers (one on average), so a head of 10^5 in-edges is not one
// thread's serial loop.
__global__ void __launch_bounds__(256)
lt_guide_kernel(const uint64_t* row, const uint32_t* cthr, const uint32_t* src, uint32_t n, uint4* guide)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = gw; v < n; v += nw) {
        const uint32_t rs = (uint32_t)row[v], re = (uint32_t)row[v + 1];
        const uint64_t d = re - rs;
        // heads with fewer than 2^16 in-edges keep j relative to their
        // first in-edge in 16 bits, which leaves 16 more bits for the
        // tail's in-degree (23 in all; the top value means "read the row")
        const bool rel = d <= kGuideRelMax;
        for (uint32_t j = rs + lane; j < re; j += 32) {
            const uint32_t tj = cthr[j];
            const uint64_t b0 = guide_nb(j > rs ? cthr[j - 1] : 0u, d);
            const uint64_t b1 = guide_nb(tj, d) < d ? guide_nb(tj, d) : d;
            if (b0 < b1) {
                const uint32_t u = src[j];
                const uint64_t du = row[u + 1] - row[u];
                const uint32_t dmax = rel ? kGuideDegRel : kGuideDegAbs;
                const uint32_t dc = du < dmax ? (uint32_t)du : dmax;
                const uint32_t x = rel ? (j - rs) | ((dc >> 7) << 16) : j;
                const uint4 e = make_uint4(x, tj | ((dc & 127u) << 25), u, (uint32_t)row[u]);
                for (uint64_t b = b0; b < b1; ++b) guide[rs + b] = e;
            }
            if (j == re - 1u) {
                const uint4 none = make_uint4(rel ? re - rs : re, 0u, 0u, 0u);
                for (uint64_t b = b1; b < d; ++b) guide[rs + b] = none;
            }
        }
    }
}

cudaError_t launch_lt_guide(const uint64_t* row, const uint32_t* cthr, const uint32_t* src, uint32_t n,
                            uint4* guide, cudaStream_t st)
{
    uint64_t blocks = ((uint64_t)n + 7) / 8;  // 8 warps (heads) per block
    if (blocks > 65535ull * 16) blocks = 65535ull * 16;
    if (blocks == 0) blocks = 1;
    lt_guide_kernel<<<(unsigned)blocks, 256, 0, st>>>(row, cthr, src, n, guide);
    return cudaGetLastError();
}

}  // namespace imm
