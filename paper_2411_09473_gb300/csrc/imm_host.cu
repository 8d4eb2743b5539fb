// Host runtime behind include/imm.h: context, device memory (pooled arena),
// sampling batches, selection rounds and the IMM theta control.
//
// The theta control follows EfficientIMM Alg. 1 with the three steps it names
// from Tang, Shi & Xiao (SIGMOD 2015): Theta_Estimation (lambda'), the
// OPT_Lower_Bound test and Set_Theta (lambda*).  It runs in host fp64 with no
// FMA contraction (-ffp-contract=off), so theta, LB and the ladder are
// bit-identical to any other IEEE evaluation in the same order.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "imm.h"
#include "imm_internal.cuh"

using namespace imm;

namespace {

struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct Segment {
    uint64_t set_begin = 0, set_end = 0;
    DBuf voff;  // n+1 uint64
    DBuf inv;   // members uint32
};

constexpr double kE = 2.71828182845904523536;  // the double nearest e
constexpr uint32_t kSelectCtaMaxN = 1u << 17;  // default: graphs this small select in one CTA

imm_tuning default_tuning()
{
    imm_tuning t;
    t.batch_sets = 1u << 22;
    t.group_min_mean = 4096;
    t.select_cta_max_n = kSelectCtaMaxN;
    t.cluster_min_n = 1u << 15;
    t.select_cand = 1;
    t.solo_cluster = 0;
    return t;
}

// tests: environment overrides of two knobs (read once per process)
uint32_t env_u32(const char* name, uint32_t dflt)
{
    const char* e = std::getenv(name);
    return e ? (uint32_t)std::strtoul(e, nullptr, 10) : dflt;
}
constexpr size_t kServerIdlePerGraph = 8;       // workers a server keeps for reuse per graph

}  // namespace

struct imm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    imm_alloc alloc{};
    bool has_alloc = false;
    DeviceInfo di{};
    std::string err = "no error";

    // graph (a worker context of a batch borrows its parent's graph arrays)
    bool loaded = false;
    bool borrowed = false;
    bool own_stream = false;
    DBuf bstates;  // batch engine: device copies of the selection states
    uint32_t n = 0;
    uint64_t m = 0;
    int model = IMM_IC;
    DBuf row, src, thr, guide;

    // RRR-set stream
    bool have_stream = false;
    uint64_t seed = 0;
    uint64_t nsets = 0;
    uint64_t nmembers = 0;
    DBuf off;   // uint64 [off_cap + 1]
    uint64_t off_cap = 0;
    DBuf arena;  // uint32 [arena_cap]: member lists of list-stored sets
    uint64_t arena_cap = 0;
    uint64_t list_members = 0;
    DBuf set_bmp;  // uint32 [off_cap]: bitmap id of each set, or kEmpty
    DBuf bmp;      // bitmap arena: words uint32 per bitmap-stored set
    DBuf bmp_set, bmp_len;  // uint32 [bmp_cap]
    uint64_t bmp_cap = 0, nbmp = 0;
    DBuf cnt;       // uint32 [n]: occurrences over all sets
    DBuf cnt_list;  // uint32 [n]: occurrences over list-stored sets (index sizes)
    std::vector<Segment> segs;
    uint64_t index_bytes = 0;

    // sampling scratch
    DBuf set_len, set_pos, set_edges, set_kind, large_q, long_q, bmp_rel;
    uint32_t batch_cap = 0;
    DBuf stage;
    uint64_t stage_cap = 0;
    DBuf big;
    uint64_t big_cap = 0;
    DBuf scalars;
    DBuf scan_tmp;
    DBuf slot_q, slot_bm;
    DBuf grp;  // grouped IC large path: masks, frontier lists, large-vertex list, counters
    DBuf mid;  // LT walks with per-walk tables (tables zero between launches)
    uint32_t nslots = 0, mid_slots = 0;
    uint64_t slot_words = 0, slot_qcap = 0;
    DBuf hist, cursor, vtmp;

    // selection scratch
    DBuf work, picked, covered, newly, keys, newly_n, vol_cov, vol_list, bmp_cov, ubmp, ubmp_n, seeds, dsegs, dstate;
    DBuf cand, cstate;

    DBuf flags;
    imm_tuning tune = default_tuning();
    uint64_t arena_limit = 0;
    uint64_t dev_bytes = 0;  // device bytes this context holds
    uint32_t next_batch = 1u << 22;  // reset to tune.batch_sets with the stream
    double avg_len = 0.0;
    double small_mean = 0.0;  // running mean members per small-path set
    double lt_cont = 0.0;     // LT: fraction of the last batch's walks past the lane path
    double large_mean = 0.0;  // running mean members per large-path set

    // accounting for imm_stats
    double acc_sample_ms = 0, acc_select_ms = 0, acc_index_ms = 0;
    uint64_t acc_sample_launches = 0, acc_launches = 0, acc_edges = 0, acc_sample_members = 0;
    cudaEvent_t ev[8] = {};
    bool index_timed = false;

    // batch in flight (phases 1-3) and pinned host slots for its read-backs
    SampleBatch fb{};
    BatchOut fo{};
    uint32_t fb_large = 0;
    struct Pinned {
        uint32_t k;
        BatchScalars sc;
        SelectState state;
    };
    Pinned* pin = nullptr;
    uint32_t* pin_seeds = nullptr;
    unsigned long long* pin_newly = nullptr;
    uint32_t pin_k = 0;
    void* pin_stage = nullptr;  // batch engine: selection states staged for the device
    size_t pin_stage_bytes = 0;
};

namespace {

int set_err(imm_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
    return code;
}

int cuda_err(imm_ctx* c, cudaError_t e, const char* where)
{
    return set_err(c, IMM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_err(c, e_, #call);     \
    } while (0)

#define TRY(call)                     \
    do {                              \
        int r_ = (call);              \
        if (r_ != IMM_OK) return r_;  \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

void dfree(imm_ctx* c, DBuf& b)
{
    if (b.p) {
        c->dev_bytes -= std::min<uint64_t>(c->dev_bytes, b.bytes);
        if (c->has_alloc) c->alloc.free(c->alloc.user, b.p, b.bytes, c->stream);
        else cudaFreeAsync(b.p, c->stream);
    }
    b = DBuf{};
}

// The library's own stream-ordered memory pool of a device (contexts without
// an allocator, and batch and server workers, allocate from it).  Freed
// memory stays in the pool for the next allocation instead of going back to
// the driver at every synchronisation, as a caching allocator would keep it;
// the pool lives until the process exits.  Null if the device has none.
cudaMemPool_t lib_pool(int device)
{
    static std::mutex mu;
    static std::unordered_map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(device);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pool = nullptr;
    } else {
        uint64_t keep = ~0ull;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
        // memory freed on one worker's stream is not handed to another
        // worker's stream by making that stream wait for the first: batch and
        // server workers must not serialise on each other
        int no = 0;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no) != cudaSuccess)
            cudaGetLastError();
    }
    pools[device] = pool;
    return pool;
}

int dalloc(imm_ctx* c, DBuf& b, size_t bytes)
{
    dfree(c, b);
    if (bytes < 16) bytes = 16;
    bytes = (bytes + 255) / 256 * 256;
    void* p = nullptr;
    if (c->has_alloc) {
        p = c->alloc.alloc(c->alloc.user, bytes, c->stream);
    } else {
        cudaMemPool_t pool = lib_pool(c->device);
        const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, c->stream)
                                   : cudaMallocAsync(&p, bytes, c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (!p) return set_err(c, IMM_ENOMEM, "device allocation of %zu bytes failed", bytes);
    b.p = p;
    b.bytes = bytes;
    c->dev_bytes += bytes;
    return IMM_OK;
}

// grow (contents discarded)
int ensure(imm_ctx* c, DBuf& b, size_t bytes)
{
    if (b.bytes >= bytes) return IMM_OK;
    size_t want = std::max(bytes, b.bytes + b.bytes / 2);
    return dalloc(c, b, want);
}

// grow keeping the first `used` bytes
int grow_keep(imm_ctx* c, DBuf& b, size_t need, size_t used)
{
    if (b.bytes >= need) return IMM_OK;
    DBuf nb;
    size_t want = std::max(need, b.bytes + b.bytes / 2);
    if (dalloc(c, nb, want) != IMM_OK) {
        if (dalloc(c, nb, need) != IMM_OK) return IMM_ENOMEM;
    }
    if (used) {
        cudaError_t e = cudaMemcpyAsync(nb.p, b.p, used, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) {
            dfree(c, nb);
            return cuda_err(c, e, "arena copy");
        }
    }
    dfree(c, b);
    b = nb;
    return IMM_OK;
}

template <typename T>
T* P(const DBuf& b)
{
    return reinterpret_cast<T*>(b.p);
}

// device time between two recorded events; 0 unless both have completed
double elapsed(imm_ctx* c, int a, int b)
{
    if (cudaEventQuery(c->ev[b]) != cudaSuccess || cudaEventQuery(c->ev[a]) != cudaSuccess) return 0.0;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) != cudaSuccess) return 0.0;
    return (double)ms;
}

void drop_stream(imm_ctx* c)
{
    for (auto& s : c->segs) {
        dfree(c, s.voff);
        dfree(c, s.inv);
    }
    c->segs.clear();
    c->index_bytes = 0;
    c->have_stream = false;
    c->nsets = 0;
    c->nmembers = 0;
    c->list_members = 0;
    c->nbmp = 0;
    c->avg_len = 0.0;
    c->small_mean = 0.0;
    c->large_mean = 0.0;
    c->lt_cont = 0.0;
    c->next_batch = c->tune.batch_sets;
    if (c->off.p) cudaMemsetAsync(c->off.p, 0, sizeof(uint64_t), c->stream);
    if (c->cnt.p) cudaMemsetAsync(c->cnt.p, 0, (size_t)c->n * 4, c->stream);
    if (c->cnt_list.p) cudaMemsetAsync(c->cnt_list.p, 0, (size_t)c->n * 4, c->stream);
}

void free_graph(imm_ctx* c)
{
    drop_stream(c);
    if (c->borrowed) {
        c->row = c->src = c->thr = c->guide = DBuf{};
        c->borrowed = false;
    }
    dfree(c, c->row);
    dfree(c, c->src);
    dfree(c, c->thr);
    dfree(c, c->guide);
    dfree(c, c->cnt);
    dfree(c, c->cnt_list);
    dfree(c, c->hist);
    dfree(c, c->cursor);
    dfree(c, c->vtmp);
    dfree(c, c->work);
    dfree(c, c->picked);
    dfree(c, c->cand);
    dfree(c, c->slot_q);
    dfree(c, c->slot_bm);
    dfree(c, c->grp);
    dfree(c, c->mid);
    c->nslots = 0;
    c->slot_qcap = 0;
    c->mid_slots = 0;
    c->loaded = false;
}

DevGraph dev_graph(imm_ctx* c)
{
    DevGraph g;
    g.n = c->n;
    g.m = c->m;
    g.row = P<uint64_t>(c->row);
    g.src = P<uint32_t>(c->src);
    g.thr = P<uint32_t>(c->thr);
    g.guide = P<uint4>(c->guide);
    return g;
}

uint64_t device_free_bytes()
{
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return fr;
}

int load_graph_common(imm_ctx* c, uint32_t n, uint64_t m, const void* row, const void* src, const void* w,
                      int model, cudaMemcpyKind kind)
{
    if (n < 2 || n == 0xFFFFFFFFu) return set_err(c, IMM_EINVAL, "n must be in [2, 2^32-2], got %u", n);
    if (m >= 0xFFFFFFFFull) return set_err(c, IMM_EINVAL, "m must be < 2^32-1");
    if (model != IMM_IC && model != IMM_LT) return set_err(c, IMM_EINVAL, "unknown model %d", model);
    if (!row || (m && (!src || !w))) return set_err(c, IMM_EINVAL, "null graph array");
    free_graph(c);
    const uint64_t m_pad = std::max<uint64_t>((m + 3) & ~3ull, 4);
    DBuf wbuf;
    TRY(dalloc(c, c->row, ((size_t)n + 1) * 8));
    TRY(dalloc(c, c->src, m_pad * 4));
    TRY(dalloc(c, c->thr, m_pad * 4));
    TRY(dalloc(c, wbuf, std::max<uint64_t>(m, 1) * 4));
    TRY(ensure(c, c->flags, 64));
    CK(cudaMemcpyAsync(c->row.p, row, ((size_t)n + 1) * 8, kind, c->stream));
    CK(cudaMemsetAsync(c->src.p, 0, m_pad * 4, c->stream));
    CK(cudaMemsetAsync(c->thr.p, 0, m_pad * 4, c->stream));
    if (m) {
        CK(cudaMemcpyAsync(c->src.p, src, m * 4, kind, c->stream));
        CK(cudaMemcpyAsync(wbuf.p, w, m * 4, kind, c->stream));
    }
    CK(cudaMemsetAsync(c->flags.p, 0, 64, c->stream));
    CK(launch_validate_graph(P<uint64_t>(c->row), P<uint32_t>(c->src), P<float>(wbuf), n, m, model,
                             P<int>(c->flags), c->stream));
    int flags = 0;
    CK(cudaMemcpyAsync(&flags, c->flags.p, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (flags) {
        dfree(c, wbuf);
        free_graph(c);
        return set_err(c, IMM_EINVAL, "malformed graph (flags 0x%x: 1=row offsets, 2=src >= n, 4=weight)",
                       flags);
    }
    CK(launch_thresholds(P<uint64_t>(c->row), P<float>(wbuf), n, m, model, P<uint32_t>(c->thr),
                         P<int>(c->flags), c->stream));
    CK(cudaMemcpyAsync(&flags, c->flags.p, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    dfree(c, wbuf);
    if (flags) {
        free_graph(c);
        return set_err(c, IMM_EINVAL, "LT in-weights of some head sum to more than 1 + 1e-6");
    }
    if (model == IMM_LT) {
        TRY(dalloc(c, c->guide, m_pad * 16));
        CK(launch_lt_guide(P<uint64_t>(c->row), P<uint32_t>(c->thr), P<uint32_t>(c->src), n, P<uint4>(c->guide),
                           c->stream));
    }
    c->n = n;
    c->m = m;
    c->model = model;
    TRY(dalloc(c, c->cnt, (size_t)n * 4));
    CK(cudaMemsetAsync(c->cnt.p, 0, (size_t)n * 4, c->stream));
    TRY(dalloc(c, c->cnt_list, (size_t)n * 4));
    CK(cudaMemsetAsync(c->cnt_list.p, 0, (size_t)n * 4, c->stream));
    TRY(dalloc(c, c->off, 8 * 1024));
    TRY(dalloc(c, c->set_bmp, 4 * 1024));
    c->off_cap = 1023;
    CK(cudaMemsetAsync(c->off.p, 0, 8, c->stream));
    // the graph is complete before the call returns: contexts that borrow it
    // run on other streams
    CK(cudaStreamSynchronize(c->stream));
    c->loaded = true;
    return IMM_OK;
}

// Per-CTA slots of the large-set paths: a member queue of qcap entries and,
// when asked for, an n-bit bitmap (zero between launches).
int ensure_slots(imm_ctx* c, uint32_t want_slots, bool need_bitmap, uint64_t qcap)
{
    const uint64_t words = ((uint64_t)c->n + 31) / 32;
    if (c->nslots >= want_slots && c->slot_qcap >= qcap &&
        (!need_bitmap || c->slot_bm.bytes >= (size_t)want_slots * words * 4))
        return IMM_OK;
    want_slots = std::max(want_slots, c->nslots);
    qcap = std::max(qcap, c->slot_qcap);
    c->nslots = 0;  // nothing usable until both are allocated
    c->slot_qcap = 0;
    TRY(dalloc(c, c->slot_q, (size_t)want_slots * qcap * 4));
    if (need_bitmap) {
        TRY(dalloc(c, c->slot_bm, (size_t)want_slots * words * 4));
        CK(cudaMemsetAsync(c->slot_bm.p, 0, (size_t)want_slots * words * 4, c->stream));
    }
    c->nslots = want_slots;
    c->slot_qcap = qcap;
    c->slot_words = words;
    return IMM_OK;
}

// Per-walk tables of the LT walks past the lane path (zeroed once; every
// walk clears the entries it set); ms covers all of them.
int ensure_mid(imm_ctx* c, uint32_t want_slots, MidSlots* ms)
{
    const size_t per = (size_t)(kLtMidHash + 2 * kLtMidCap) * 4;
    if (c->mid_slots < want_slots) {
        const uint32_t cap = std::min<uint32_t>((want_slots + 1023u) / 1024u * 1024u, kLtMidSlotsMax);
        c->mid_slots = 0;
        TRY(dalloc(c, c->mid, (size_t)cap * per));
        CK(cudaMemsetAsync(c->mid.p, 0, (size_t)cap * per, c->stream));
        c->mid_slots = cap;
    }
    uint32_t* base = P<uint32_t>(c->mid);
    ms->tab = base;
    ms->path = base + (size_t)c->mid_slots * kLtMidHash;
    ms->hpos = ms->path + (size_t)c->mid_slots * kLtMidCap;
    ms->nslots = c->mid_slots;
    return IMM_OK;
}

// Cooperative kernels (the grouped sampler, the whole-grid selection) each
// need every SM at once.  Two of them running side by side (contexts driven
// from different host threads) could each hold SMs the other's CTAs wait
// for, so on every device they run one after another: a launch waits for
// the event recorded after the previous one.  Other kernels overlap freely.
struct CoopOrder {
    std::mutex mu;
    cudaEvent_t last = nullptr;
};

CoopOrder& coop_order(int device)
{
    static std::mutex table_mu;
    static std::unordered_map<int, CoopOrder*> table;
    std::lock_guard<std::mutex> lk(table_mu);
    CoopOrder*& o = table[device];
    if (!o) o = new CoopOrder();  // lives for the process
    return *o;
}

// Runs `launch` (which enqueues one cooperative kernel on st) after every
// cooperative kernel enqueued before it on this device.
template <class F>
cudaError_t coop_launch(int device, cudaStream_t st, F&& launch)
{
    CoopOrder& o = coop_order(device);
    std::lock_guard<std::mutex> lk(o.mu);
    if (!o.last) {
        const cudaError_t e = cudaEventCreateWithFlags(&o.last, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    } else {
        const cudaError_t e = cudaStreamWaitEvent(st, o.last, 0);
        if (e != cudaSuccess) return e;
    }
    const cudaError_t le = launch();
    if (le != cudaSuccess) return le;
    return cudaEventRecord(o.last, st);
}

// The error word of the bounds-checked build inside the batch scalars.
unsigned long long* batch_bounds(imm_ctx* c)
{
    return reinterpret_cast<unsigned long long*>(static_cast<char*>(c->scalars.p) + offsetof(BatchScalars, bounds));
}

// Scratch of the grouped IC large path (carved from one buffer; the masks
// start at zero and every launch leaves them zero).
int ensure_group(imm_ctx* c, GroupScratch* gs)
{
    const uint64_t n = c->n;
    const uint64_t hcap = ic_group_heavy_cap(c->n, c->m);
    auto up = [](uint64_t x) { return (x + 255) & ~255ull; };
    // one slot: vis and fn (zeroed once; every launch leaves them zero), lists
    // windows of 32 small quads per level: a vertex has at most (indeg + 6) / 4 quads
    const uint64_t wcap = (c->m + 6 * n) / 128 + 2;
    const uint64_t o_fn = up(n * 8), o_lq = o_fn + up(n * 8), o_lpre = o_lq + up(n * 16);
    // chunks of one level: sum over its large vertices of ceil(quads / 64)
    const uint64_t ccap = c->m / 256 + 2 * hcap + 64;
    const uint64_t o_wst = o_lpre + up(n * 4), o_hb = o_wst + up(wcap * 4);
    const uint64_t o_he = o_hb + up(hcap * 4), o_co = o_he + up(hcap * 16), slot = o_co + up(ccap * 4);
    const uint64_t o_ct = kGroupSlots * slot;
    const uint64_t bytes = o_ct + up(kGroupSlots * sizeof(GroupCounters));
    char* p;
    if (c->grp.bytes < bytes) {
        TRY(dalloc(c, c->grp, bytes));
        p = static_cast<char*>(c->grp.p);
        for (uint32_t k = 0; k < kGroupSlots; ++k) CK(cudaMemsetAsync(p + k * slot, 0, o_lq, c->stream));
        CK(cudaMemsetAsync(p + o_ct, 0, kGroupSlots * sizeof(GroupCounters), c->stream));
    }
    p = static_cast<char*>(c->grp.p);
    gs->vis = reinterpret_cast<unsigned long long*>(p);
    gs->fn = reinterpret_cast<unsigned long long*>(p + o_fn);
    gs->lq = reinterpret_cast<uint4*>(p + o_lq);
    gs->lpre = reinterpret_cast<uint32_t*>(p + o_lpre);
    gs->wst = reinterpret_cast<uint32_t*>(p + o_wst);
    gs->hb = reinterpret_cast<uint32_t*>(p + o_hb);
    gs->he = reinterpret_cast<uint4*>(p + o_he);
    gs->cown = reinterpret_cast<uint32_t*>(p + o_co);
    gs->ccap = (uint32_t)ccap;
    gs->stride = slot;
    gs->ctr = reinterpret_cast<GroupCounters*>(p + o_ct);
    gs->wcap = (uint32_t)wcap;
    gs->hcap = (uint32_t)hcap;
    gs->lcap = c->n;
    gs->bounds = batch_bounds(c);
    return IMM_OK;
}

// The grouped path pays dense passes over n and grid barriers per BFS level
// for every group of 64 sets; it wins when the sets are giant and share the
// graph's core (thousands of members and more).  So it is taken when there
// are enough large sets and their mean size, from the previous batches, is at
// least max(4096, n/64); before any batch has told, on graphs of >= 2^19
// vertices only.  It launches cooperatively, so contexts whose streams run
// beside others' (batch and server workers) keep the one-set-per-CTA path.
// IMM_IC_LARGE=cta|group overrides the choice (both give the same sets).
bool use_group(const imm_ctx* c, uint32_t large_count)
{
    if (c->model != IMM_IC || c->borrowed || large_count == 0) return false;
    const char* force = getenv("IMM_IC_LARGE");
    if (force && strcmp(force, "cta") == 0) return false;
    if (!ic_group_supported(c->di)) return false;
    if (force && strcmp(force, "group") == 0) return true;
    if (large_count < kGroupSets) return false;
    if (c->large_mean > 0.0) return c->large_mean >= std::max((double)c->tune.group_min_mean, (double)c->n / 64.0);
    return c->n >= (1u << 19);
}

// Checked builds: the first failed index check recorded by the kernels
// enqueued so far on the context's stream (`err` is a device error word);
// IMM_ECUDA naming it, else IMM_OK.  A no-op in normal builds.
int bounds_verdict(imm_ctx* c, const unsigned long long* err, const char* where)
{
    if (!kBoundsChecked) return IMM_OK;
    unsigned long long h[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(h, err, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (h[0])
        return set_err(c, IMM_ECUDA, "%s: index check %llu failed (index %llu, bound %llu)", where, h[0], h[1], h[2]);
    return IMM_OK;
}

int index_limit_ok(imm_ctx* c, uint64_t more_bytes)
{
    if (!c->arena_limit) return IMM_OK;
    const uint64_t used = c->arena_cap * 4 + c->index_bytes + c->bmp.bytes;
    if (used + more_bytes > c->arena_limit)
        return set_err(c, IMM_ENOMEM, "arena limit of %llu bytes reached", (unsigned long long)c->arena_limit);
    return IMM_OK;
}

// Rebuild the inverted index as a single segment over the whole stream.
int merge_segments(imm_ctx* c)
{
    for (auto& s : c->segs) {
        dfree(c, s.voff);
        dfree(c, s.inv);
    }
    c->segs.clear();
    c->index_bytes = 0;
    Segment seg;
    seg.set_begin = 0;
    seg.set_end = c->nsets;
    TRY(dalloc(c, seg.voff, ((size_t)c->n + 1) * 8));
    TRY(dalloc(c, seg.inv, std::max<uint64_t>(c->list_members, 1) * 4));
    CK(launch_vertex_scan(P<uint32_t>(c->cnt_list), c->n, P<uint64_t>(seg.voff), nullptr, nullptr,
                          P<uint32_t>(c->cursor), P<uint64_t>(c->vtmp), c->di, c->stream));
    CK(launch_index_scatter(0, c->nsets, P<uint64_t>(c->off), P<uint32_t>(c->arena), P<uint64_t>(seg.voff),
                            P<uint32_t>(c->cursor), P<uint32_t>(seg.inv), std::max<uint64_t>(c->list_members, 1),
                            batch_bounds(c), c->di, c->stream));
    c->acc_launches += 4;
    c->index_bytes = seg.voff.bytes + seg.inv.bytes;
    c->segs.push_back(seg);
    return IMM_OK;
}

// ---------------------------------------------------------------------------
// Generate_RRRsets, one batch of consecutive set ids in three phases so that
// many contexts (each on its own stream) can advance together:
//   phase 1  buffers, small-set path launch, large-set count -> pinned host
//   phase 2  (after the stream drained) large-set path and batch scan,
//            batch scalars -> pinned host
//   phase 3  (after the stream drained) grow the arena / bitmap arena, launch
//            compaction, bitmap store, vertex scan and index scatter
// ---------------------------------------------------------------------------
int begin_stream(imm_ctx* c, uint64_t theta, uint64_t seed)
{
    if (!c->loaded) return set_err(c, IMM_ESTATE, "no graph loaded");
    if (theta >= 0xFFFFFFFFull) return set_err(c, IMM_EINVAL, "theta must be < 2^32-1");
    if (c->have_stream && c->nsets > 0 && c->seed != seed)
        return set_err(c, IMM_ESTATE, "rng seed differs from the current stream's; reset first");
    c->have_stream = true;
    c->seed = seed;
    TRY(ensure(c, c->scalars, sizeof(BatchScalars)));
    TRY(ensure(c, c->hist, (size_t)c->n * 4));
    TRY(ensure(c, c->cursor, (size_t)c->n * 4));
    TRY(ensure(c, c->vtmp, scan_tmp_words(c->n) * 8));
    return IMM_OK;
}

void take_index_time(imm_ctx* c)
{
    // the stream has drained since the index launches were recorded
    if (c->index_timed && cudaEventQuery(c->ev[7]) == cudaSuccess) {
        c->acc_index_ms += elapsed(c, 6, 7);
        c->index_timed = false;
    }
}

int batch_phase1(imm_ctx* c, uint64_t theta)
{
    take_index_time(c);
    const uint32_t words = (uint32_t)(((uint64_t)c->n + 31) / 32);
    const uint64_t want = theta - c->nsets;
    uint32_t count = (uint32_t)std::min<uint64_t>(want, c->next_batch);
    if (count == 0) count = 1;
    if (c->batch_cap < count) {
        const uint32_t cap = std::max(count, c->batch_cap + c->batch_cap / 2);
        TRY(dalloc(c, c->set_len, (size_t)cap * 4));
        TRY(dalloc(c, c->set_pos, (size_t)cap * 8));
        TRY(dalloc(c, c->set_edges, (size_t)cap * 4));
        TRY(dalloc(c, c->set_kind, (size_t)cap * 4));
        TRY(dalloc(c, c->large_q, (size_t)cap * 4));
        TRY(dalloc(c, c->long_q, (size_t)cap * 4));
        TRY(dalloc(c, c->bmp_rel, (size_t)cap * 4));
        TRY(dalloc(c, c->scan_tmp, scan_tmp_words(cap) * 8));
        c->batch_cap = cap;
    }
    // small-path staging: sized from the running mean small-set size (sets
    // past it are resampled), never above count * small_cap, and always
    // enough for one full small set
    {
        const double mean = c->small_mean > 0 ? c->small_mean * 1.5 + 8.0 : 64.0;
        const uint64_t cap_all = (uint64_t)count * small_cap(c->model);
        uint64_t need = std::min<uint64_t>(cap_all, (uint64_t)(mean * (double)count) + 4096);
        need = std::max<uint64_t>(need, small_cap(c->model) + 4096);
        if (c->stage_cap < need) {
            TRY(ensure(c, c->stage, need * 4));
            c->stage_cap = c->stage.bytes / 4;
        }
    }
    // per-set arrays of the stream: room for base + count sets
    if (c->off_cap < c->nsets + count) {
        const uint64_t need = c->nsets + count;
        const uint64_t cap = std::max(need, c->off_cap + c->off_cap / 2);
        TRY(grow_keep(c, c->off, (cap + 1) * 8, (c->nsets + 1) * 8));
        TRY(grow_keep(c, c->set_bmp, cap * 4, c->nsets * 4));
        c->off_cap = cap;
    }
    BatchScalars* sc = P<BatchScalars>(c->scalars);
    CK(cudaMemsetAsync(sc, 0, sizeof(BatchScalars), c->stream));
    CK(cudaMemsetAsync(&sc->first_fail, 0xFF, 4, c->stream));
    SampleBatch& b = c->fb;
    b.seed = c->seed;
    b.rk = philox_keys(c->seed);
    b.base = c->nsets;
    b.count = count;
    b.words = words;
    b.set_len = P<uint32_t>(c->set_len);
    b.set_pos = P<uint64_t>(c->set_pos);
    b.set_edges = P<uint32_t>(c->set_edges);
    b.set_kind = P<uint32_t>(c->set_kind);
    b.stage = P<uint32_t>(c->stage);
    b.stage_cap = c->stage_cap;
    b.big = P<uint32_t>(c->big);
    b.big_cap = 0;
    b.large_q = P<uint32_t>(c->large_q);
    b.long_q = P<uint32_t>(c->long_q);
    b.sc = sc;
    const DevGraph g = dev_graph(c);
    MidSlots ms{};
    if (c->model == IMM_LT) {
        // tables for the walks that outgrow the lane path, sized from the
        // last batch's share of them (a walk that finds none left is sampled
        // again by the per-walk-table kernel)
        const double f = c->lt_cont > 0 ? c->lt_cont : 0.1;
        const double want = std::min<double>((double)kLtMidSlotsMax, (double)count * f * 1.25 + 256.0);
        TRY(ensure_mid(c, std::min<uint32_t>((uint32_t)want, count), &ms));
    }
    CK(cudaEventRecord(c->ev[0], c->stream));
    if (c->model == IMM_IC) CK(launch_ic_small(g, b, c->di, c->stream));
    else CK(launch_lt_small(g, b, ms, c->di, c->stream));
    CK(cudaEventRecord(c->ev[1], c->stream));
    // the batch scalars in one read-back: phase 2 needs the hand-off counts
    CK(cudaMemcpyAsync(&c->pin->sc, sc, sizeof(BatchScalars), cudaMemcpyDeviceToHost, c->stream));
    c->acc_sample_launches += 1;
    c->acc_launches += 1;
    return IMM_OK;
}

int batch_phase2(imm_ctx* c)
{
    c->acc_sample_ms += elapsed(c, 0, 1);
    SampleBatch& b = c->fb;
    const uint32_t large_count = c->pin->sc.large_count;
    const uint32_t long_count = c->pin->sc.long_count;  // LT walks already bound for the bitmap slots
    const uint32_t words = b.words;
    c->fb_large = large_count + long_count;
    if (large_count + long_count) {
        // outputs of the large path: a list or a bitmap of `words` words
        // each; capped by a memory budget (sets past the cap are resampled)
        const uint64_t fr = device_free_bytes() + c->big.bytes;
        const uint64_t budget = std::max<uint64_t>((uint64_t)words * 4,
                                                   std::min<uint64_t>(fr / 4, 16ull << 30) / 4);
        const uint64_t need = std::min<uint64_t>((uint64_t)(large_count + long_count) * words, budget);
        if (c->big_cap < need) {
            TRY(ensure(c, c->big, need * 4));
            c->big_cap = c->big.bytes / 4;
        }
        b.big = P<uint32_t>(c->big);
        b.big_cap = c->big_cap;
        // IMM_BIG_CAP_WORDS (tests): a smaller output buffer, at least one
        // bitmap, drives the reservation-failure and resampling path
        if (const char* cap = std::getenv("IMM_BIG_CAP_WORDS"))
            b.big_cap = std::min<uint64_t>(b.big_cap, std::max<uint64_t>(std::strtoull(cap, nullptr, 10), words));
        const bool ic = c->model == IMM_IC;
        const DevGraph g = dev_graph(c);
        if (use_group(c, large_count)) {
            GroupScratch gs;
            TRY(ensure_group(c, &gs));
            CK(cudaEventRecord(c->ev[2], c->stream));
            CK(coop_launch(c->device, c->stream, [&] { return launch_ic_group(g, b, gs, c->di, c->stream); }));
            CK(cudaEventRecord(c->ev[3], c->stream));
        } else {
            const uint32_t want_slots = std::min<uint32_t>(
                large_count + long_count, ic ? (uint32_t)c->di.sms : (uint32_t)std::min(c->di.sms * 2, 1024));
            MidSlots ms{};
            if (ic) {
                const bool smem = ic_large_uses_smem(c->n, c->di) != 0;
                TRY(ensure_slots(c, want_slots, !smem, c->n));
            } else {
                TRY(ensure_slots(c, want_slots, true, (uint64_t)words + 1));
                if (large_count) {
                    TRY(ensure_mid(c, std::min<uint32_t>(large_count, kLtMidSlotsMax), &ms));
                    ms.nslots = std::min<uint32_t>(ms.nslots, large_count);
                }
            }
            LargeSlots ls;
            ls.queues = P<uint32_t>(c->slot_q);
            ls.queue_cap = c->slot_qcap;
            ls.bitmaps = P<uint32_t>(c->slot_bm);
            ls.bitmap_words = words;
            ls.nslots = std::min<uint32_t>(c->nslots, large_count + long_count);
            CK(cudaEventRecord(c->ev[2], c->stream));
            if (ic) {
                CK(launch_ic_large(g, b, ls, c->di, c->stream));
            } else {
                // walks the lane path handed back (its tables were used up)
                // with per-walk tables; walks longer than a table or a list
                // holds on the bitmap slots
                if (large_count) {
                    CK(launch_lt_mid(g, b, ms, c->stream));
                    c->acc_sample_launches += 1;
                    c->acc_launches += 1;
                }
                CK(launch_lt_long(g, b, ls, c->di, c->stream));
            }
            CK(cudaEventRecord(c->ev[3], c->stream));
        }
        c->acc_sample_launches += 1;
        c->acc_launches += 1;
    }
    BatchOut& o = c->fo;
    o.off = P<uint64_t>(c->off);
    o.arena = P<uint32_t>(c->arena);
    o.set_bmp = P<uint32_t>(c->set_bmp);
    o.bmp = P<uint32_t>(c->bmp);
    o.bmp_set = P<uint32_t>(c->bmp_set);
    o.bmp_len = P<uint32_t>(c->bmp_len);
    o.bmp_rel = P<uint32_t>(c->bmp_rel);
    o.bmp_base = c->nbmp;
    o.arena_cap = c->arena_cap;
    o.bounds = batch_bounds(c);
    CK(launch_batch_scan(b, o, P<uint64_t>(c->scan_tmp), c->di, c->stream));
    c->acc_launches += 3;
    CK(cudaMemcpyAsync(&c->pin->sc, b.sc, sizeof(BatchScalars), cudaMemcpyDeviceToHost, c->stream));
    return IMM_OK;
}

// returns IMM_OK; *progress = false when the batch kept no set (retry smaller)
int batch_phase3(imm_ctx* c, bool* progress)
{
    if (c->fb_large) c->acc_sample_ms += elapsed(c, 2, 3);
    SampleBatch& b = c->fb;
    BatchOut& o = c->fo;
    const BatchScalars& hs = c->pin->sc;
    const uint32_t words = b.words;
    const uint32_t count = b.count;
    *progress = false;
    if (hs.error) return set_err(c, IMM_ECUDA, "sampler reported device error 0x%x", hs.error);
    if (hs.bounds[0])
        return set_err(c, IMM_ECUDA, "sampling: index check %llu failed (index %llu, bound %llu)", hs.bounds[0],
                       hs.bounds[1], hs.bounds[2]);
    const uint64_t committed = hs.committed;
    const uint64_t lm = hs.list_members;
    const uint64_t nb = hs.nbitmaps;
    if (committed == 0) {
        if (count == 1) return set_err(c, IMM_ENOMEM, "output buffer cannot hold one RRR set");
        c->next_batch = std::max<uint32_t>(1, count / 4);
        return IMM_OK;
    }
    // arena for the lists, bitmap arena, this batch's index segment
    const uint64_t seg_bytes = ((uint64_t)c->n + 1) * 8 + lm * 4;
    const uint64_t bmp_bytes = nb * words * 4;
    if (c->arena_cap < c->list_members + lm) {
        const uint64_t need = c->list_members + lm;
        uint64_t cap = std::max(need, c->arena_cap + c->arena_cap / 2);
        if (c->arena_limit && (cap * 4 + c->index_bytes + c->bmp.bytes + seg_bytes + bmp_bytes > c->arena_limit))
            cap = need;
        TRY(index_limit_ok(c, (cap - c->arena_cap) * 4 + seg_bytes + bmp_bytes));
        TRY(grow_keep(c, c->arena, cap * 4, c->list_members * 4));
        c->arena_cap = cap;
    } else {
        TRY(index_limit_ok(c, seg_bytes + bmp_bytes));
    }
    if (c->bmp_cap < c->nbmp + nb) {
        const uint64_t need = c->nbmp + nb;
        const uint64_t cap = std::max(need, c->bmp_cap + c->bmp_cap / 2);
        TRY(grow_keep(c, c->bmp, cap * words * 4, c->nbmp * words * 4));
        TRY(grow_keep(c, c->bmp_set, cap * 4, c->nbmp * 4));
        TRY(grow_keep(c, c->bmp_len, cap * 4, c->nbmp * 4));
        c->bmp_cap = cap;
    }
    o.arena = P<uint32_t>(c->arena);
    o.bmp = P<uint32_t>(c->bmp);
    o.bmp_set = P<uint32_t>(c->bmp_set);
    o.bmp_len = P<uint32_t>(c->bmp_len);
    o.arena_cap = c->arena_cap;
    Segment seg;
    seg.set_begin = c->nsets;
    seg.set_end = c->nsets + committed;
    TRY(dalloc(c, seg.voff, ((size_t)c->n + 1) * 8));
    if (dalloc(c, seg.inv, std::max<uint64_t>(lm, 1) * 4) != IMM_OK) {
        dfree(c, seg.voff);
        return IMM_ENOMEM;
    }
    CK(cudaEventRecord(c->ev[6], c->stream));
    CK(cudaMemsetAsync(c->hist.p, 0, (size_t)c->n * 4, c->stream));
    CK(launch_compact(b, o, committed, P<uint32_t>(c->hist), c->di, c->stream));
    CK(launch_bitmap_store(b, o, nb, c->n, P<uint32_t>(c->cnt), c->di, c->stream));
    CK(launch_vertex_scan(P<uint32_t>(c->hist), c->n, P<uint64_t>(seg.voff), P<uint32_t>(c->cnt),
                          P<uint32_t>(c->cnt_list), P<uint32_t>(c->cursor), P<uint64_t>(c->vtmp), c->di,
                          c->stream));
    CK(launch_index_scatter(seg.set_begin, seg.set_end, P<uint64_t>(c->off), P<uint32_t>(c->arena),
                            P<uint64_t>(seg.voff), P<uint32_t>(c->cursor), P<uint32_t>(seg.inv), std::max<uint64_t>(lm, 1),
                            batch_bounds(c), c->di, c->stream));
    CK(cudaEventRecord(c->ev[7], c->stream));
    c->index_timed = true;
    c->acc_launches += nb ? 7 : 5;
    c->index_bytes += seg.voff.bytes + seg.inv.bytes;
    c->segs.push_back(seg);
    c->nsets += committed;
    c->list_members += lm;
    c->nmembers += hs.all_members;
    c->nbmp += nb;
    c->acc_edges += hs.edges;
    c->acc_sample_members += hs.all_members;
    c->next_batch = committed < count ? std::max<uint32_t>(256, (uint32_t)committed) : c->tune.batch_sets;
    // running mean of the small-path set sizes of this batch
    if (count > c->fb_large) {
        const double m = (double)hs.stage_cursor / (double)(count - c->fb_large);
        c->small_mean = c->small_mean > 0 ? std::max(m, 0.5 * (c->small_mean + m)) : m;
    }
    if (c->model == IMM_LT) c->lt_cont = (double)hs.mid_claim / (double)count;
    if (c->fb_large && hs.all_members > hs.stage_cursor) {
        const double m = (double)(hs.all_members - hs.stage_cursor) / (double)c->fb_large;
        c->large_mean = c->large_mean > 0 ? 0.5 * (c->large_mean + m) : m;
    }
    if (c->segs.size() > 48) TRY(merge_segments(c));
    TRY(bounds_verdict(c, batch_bounds(c), "compaction and index"));
    *progress = true;
    return IMM_OK;
}

// Generate_RRRsets: extend the stream to theta sets (solo path).
int sample_to(imm_ctx* c, uint64_t theta, uint64_t seed)
{
    TRY(begin_stream(c, theta, seed));
    while (c->nsets < theta) {
        TRY(batch_phase1(c, theta));
        CK(cudaStreamSynchronize(c->stream));
        TRY(batch_phase2(c));
        CK(cudaStreamSynchronize(c->stream));
        bool progress = false;
        TRY(batch_phase3(c, &progress));
    }
    CK(cudaStreamSynchronize(c->stream));
    take_index_time(c);
    return IMM_OK;
}

// ---------------------------------------------------------------------------
// Find_Most_Influential_Set: buffers and state (prepare), one launch, and
// the read-back of seeds and per-round coverage (collect).
// ---------------------------------------------------------------------------
// prefix < nsets: the selection sees only sets [0, prefix) of the stream
// (the others start covered and the counts are those of the prefix), so its
// result is that of a stream of `prefix` sets.
int select_prepare(imm_ctx* c, uint32_t k, SelectState* out, uint64_t prefix = ~0ull)
{
    if (!c->loaded) return set_err(c, IMM_ESTATE, "no graph loaded");
    if (k == 0 || k > c->n) return set_err(c, IMM_EINVAL, "k must be in [1, n]");
    const uint64_t R = c->nsets;
    const bool part = prefix < R;
    TRY(ensure(c, c->work, (size_t)c->n * 4));
    TRY(ensure(c, c->picked, (size_t)c->n));
    TRY(ensure(c, c->covered, std::max<uint64_t>(R, 1)));
    TRY(ensure(c, c->newly, std::max<uint64_t>(R, 1) * 4));
    TRY(ensure(c, c->keys, (size_t)k * 8));
    TRY(ensure(c, c->newly_n, (size_t)k * 8));
    TRY(ensure(c, c->vol_cov, (size_t)k * 8));
    TRY(ensure(c, c->vol_list, (size_t)k * 8));
    TRY(ensure(c, c->bmp_cov, (size_t)k * 8));
    TRY(ensure(c, c->ubmp, std::max<uint64_t>(c->nbmp, 1) * 4));
    TRY(ensure(c, c->ubmp_n, (size_t)k * 8));
    TRY(ensure(c, c->seeds, (size_t)k * 4));
    TRY(ensure(c, c->cand, (size_t)c->n * 4));
    TRY(ensure(c, c->cstate, 64));
    std::vector<DevSegment> hsegs;
    for (auto& sg : c->segs) hsegs.push_back(DevSegment{P<uint64_t>(sg.voff), P<uint32_t>(sg.inv)});
    TRY(ensure(c, c->dsegs, std::max<size_t>(hsegs.size(), 1) * sizeof(DevSegment)));

    uint64_t list_end = 0;
    if (part) {
        TRY(ensure(c, c->flags, 64));
        CK(cudaMemcpyAsync(&c->pin->sc.list_members, P<uint64_t>(c->off) + prefix, 8, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        list_end = c->pin->sc.list_members;
    }
    CK(cudaEventRecord(c->ev[4], c->stream));
    if (!hsegs.empty())
        CK(cudaMemcpyAsync(c->dsegs.p, hsegs.data(), hsegs.size() * sizeof(DevSegment), cudaMemcpyHostToDevice,
                           c->stream));
    if (part) CK(cudaMemsetAsync(c->work.p, 0, (size_t)c->n * 4, c->stream));
    else CK(cudaMemcpyAsync(c->work.p, c->cnt.p, (size_t)c->n * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemsetAsync(c->picked.p, 0, (size_t)c->n, c->stream));
    if (R) CK(cudaMemsetAsync(c->covered.p, 0, part ? prefix : R, c->stream));
    if (part) CK(cudaMemsetAsync(P<uint8_t>(c->covered) + prefix, 1, R - prefix, c->stream));
    DBuf* zero_k[] = {&c->keys, &c->newly_n, &c->vol_cov, &c->vol_list, &c->bmp_cov, &c->ubmp_n};
    for (DBuf* z : zero_k) CK(cudaMemsetAsync(z->p, 0, (size_t)k * 8, c->stream));
    CK(cudaMemsetAsync(c->cstate.p, 0, 64, c->stream));

    SelectState& s = *out;
    s.n = c->n;
    s.words = (uint32_t)(((uint64_t)c->n + 31) / 32);
    s.nsets = R;
    s.total_members = c->nmembers;
    s.list_members = c->list_members;
    s.off = P<uint64_t>(c->off);
    s.arena = P<uint32_t>(c->arena);
    s.set_bmp = P<uint32_t>(c->set_bmp);
    s.bmp = P<uint32_t>(c->bmp);
    s.bmp_set = P<uint32_t>(c->bmp_set);
    s.bmp_len = P<uint32_t>(c->bmp_len);
    s.nbmp = (uint32_t)c->nbmp;
    s.work = P<uint32_t>(c->work);
    s.picked = P<uint8_t>(c->picked);
    s.covered = P<uint8_t>(c->covered);
    s.newly = P<uint32_t>(c->newly);
    s.keys = P<unsigned long long>(c->keys);
    s.newly_n = P<unsigned long long>(c->newly_n);
    s.vol_cov = P<unsigned long long>(c->vol_cov);
    s.vol_list = P<unsigned long long>(c->vol_list);
    s.bmp_cov = P<unsigned long long>(c->bmp_cov);
    s.ubmp = P<uint32_t>(c->ubmp);
    s.ubmp_n = P<unsigned long long>(c->ubmp_n);
    s.seeds = P<uint32_t>(c->seeds);
    s.segs = P<DevSegment>(c->dsegs);
    s.nsegs = (uint32_t)hsegs.size();
    // IMM_SELECT_CAND=0 (tests) overrides the tuning: every argmax scans all n vertices
    static const uint32_t cand_env = env_u32("IMM_SELECT_CAND", 1u);
    const bool cand = c->tune.select_cand && cand_env;
    s.cand = cand ? P<uint32_t>(c->cand) : nullptr;
    s.cstate = P<uint32_t>(c->cstate);
    s.bounds = reinterpret_cast<unsigned long long*>(static_cast<char*>(c->cstate.p) + 32);
    // IMM_SELECT_MODE=decrement|rebuild (tests): one counter update for every
    // round; the two give the same counts (Sec. IV-C), which the tests check
    s.force_mode = 0;
    if (const char* fm = std::getenv("IMM_SELECT_MODE"))
        s.force_mode = std::strcmp(fm, "decrement") == 0 ? 1 : std::strcmp(fm, "rebuild") == 0 ? 2 : 0;
    if (part) {
        s.list_members = list_end;
        CK(launch_prefix_count(s, prefix, list_end, P<unsigned long long>(c->flags) + 1, c->di, c->stream));
        c->acc_launches += 2 + (c->nbmp + 65534) / 65535;
    }
    return IMM_OK;
}

// Members of the stream's first `prefix` sets, as counted by the last
// prefix selection's set-up (read after the stream has drained).
int prefix_members(imm_ctx* c, uint64_t* out)
{
    CK(cudaMemcpyAsync(&c->pin->sc.list_members, P<unsigned long long>(c->flags) + 1, 8, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *out = c->pin->sc.list_members;
    return IMM_OK;
}

// enqueue the read-back of seeds and per-round coverage on `st`
int select_readback(imm_ctx* c, uint32_t k, cudaStream_t st)
{
    if (c->pin_k < k) {
        // grown geometrically: freeing pinned memory synchronises the whole
        // device, which would stall every other stream of a batch or server
        const uint32_t cap = std::max<uint32_t>(k, std::max<uint32_t>(256u, c->pin_k * 2u));
        if (c->pin_seeds) cudaFreeHost(c->pin_seeds);
        if (c->pin_newly) cudaFreeHost(c->pin_newly);
        c->pin_seeds = nullptr;
        c->pin_newly = nullptr;
        c->pin_k = 0;
        CK(cudaMallocHost(&c->pin_seeds, (size_t)cap * 4));
        CK(cudaMallocHost(&c->pin_newly, (size_t)cap * 8));
        c->pin_k = cap;
    }
    CK(cudaMemcpyAsync(c->pin_seeds, c->seeds.p, (size_t)k * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(c->pin_newly, c->newly_n.p, (size_t)k * 8, cudaMemcpyDeviceToHost, st));
    return IMM_OK;
}

uint64_t select_covered(imm_ctx* c, uint32_t k, uint32_t* seeds_out)
{
    uint64_t cov = 0;
    for (uint32_t j = 0; j < k; ++j) cov += c->pin_newly[j];
    if (seeds_out) std::memcpy(seeds_out, c->pin_seeds, (size_t)k * 4);
    return cov;
}

int select_k(imm_ctx* c, uint32_t k, uint32_t* seeds_out, uint64_t* covered_out)
{
    if (!seeds_out) return set_err(c, IMM_EINVAL, "seeds_out is NULL");
    SelectState s;
    TRY(select_prepare(c, k, &s));
    // all k rounds in one launch: one CTA for small graphs (block barriers),
    // the whole cooperative grid otherwise; per-round launches if the device
    // refuses a cooperative grid of that size
    // tune.solo_cluster: streams without bitmap-stored sets on larger graphs
    // select on one 8-CTA cluster instead of the whole grid (off by default:
    // on the 4M-vertex LT workload the cluster's full scans took 14.8 ms per
    // run against 4.5-5 ms for the grid)
    const bool cluster = c->n > c->tune.select_cta_max_n && c->nbmp == 0 && c->tune.solo_cluster;
    bool done = false;
    if (c->n <= c->tune.select_cta_max_n || cluster) {
        TRY(ensure(c, c->dstate, sizeof(SelectState) + 16));
        c->pin->k = k;
        c->pin->state = s;
        CK(cudaMemcpyAsync(c->dstate.p, &c->pin->state, sizeof(SelectState), cudaMemcpyHostToDevice, c->stream));
        uint32_t* dk = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(c->dstate.p) + sizeof(SelectState));
        CK(cudaMemcpyAsync(dk, &c->pin->k, 4, cudaMemcpyHostToDevice, c->stream));
        if (cluster) {
            const cudaError_t ce = launch_select_clusters(P<SelectState>(c->dstate), dk, 1, c->di, c->stream);
            if (ce == cudaSuccess) {
                done = true;
            } else if (ce == cudaErrorCooperativeLaunchTooLarge || ce == cudaErrorNotSupported) {
                cudaGetLastError();
            } else {
                CK(ce);
            }
        } else {
            CK(launch_select_batch(P<SelectState>(c->dstate), dk, 1, c->di, c->stream));
            done = true;
        }
        if (done) c->acc_launches += 1;
    }
    if (!done) {
        // the whole-grid rounds are bound by their grid barriers, not by the
        // argmax scan, so they scan every vertex (no candidate list, which
        // costs barriers of its own)
        s.cand = nullptr;
        const cudaError_t ce =
            coop_launch(c->device, c->stream, [&] { return launch_select_all(s, k, c->di, c->stream); });
        if (ce == cudaErrorCooperativeLaunchTooLarge || ce == cudaErrorNotSupported) {
            cudaGetLastError();
            for (uint32_t j = 0; j < k; ++j) CK(launch_select_round(s, j, c->di, c->stream, &c->acc_launches));
        } else {
            CK(ce);
            c->acc_launches += 1;
        }
    }
    CK(cudaEventRecord(c->ev[5], c->stream));
    TRY(select_readback(c, k, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    TRY(bounds_verdict(c, reinterpret_cast<unsigned long long*>(static_cast<char*>(c->cstate.p) + 32), "selection"));
    c->acc_select_ms += elapsed(c, 4, 5);
    const uint64_t cov = select_covered(c, k, seeds_out);
    if (covered_out) *covered_out = cov;
    return IMM_OK;
}

// Theta_Estimation constants (Tang et al.), same operation order as any plain
// fp64 evaluation of the formulas; shared by imm_run and the batch engine so
// both produce bit-identical ladders.
struct ThetaPlan {
    double nd, ln_n, lam_p, lam_s, eps_p;
    uint32_t rounds;
};

ThetaPlan theta_plan(uint32_t n, uint32_t k, double epsilon, double ell)
{
    ThetaPlan p;
    p.nd = (double)n;
    p.ln_n = std::log(p.nd);
    const double ell_p = ell * (1.0 + std::log(2.0) / p.ln_n);
    p.eps_p = std::sqrt(2.0) * epsilon;
    double lnC = 0.0;
    for (uint32_t i = 1; i <= k; i++) lnC += std::log((double)(n - k + i)) - std::log((double)i);
    p.lam_p = (2.0 + 2.0 * p.eps_p / 3.0) * (lnC + ell_p * p.ln_n + std::log(std::log2(p.nd))) * p.nd /
              (p.eps_p * p.eps_p);
    const double g = 1.0 - 1.0 / kE;
    const double alpha = std::sqrt(ell_p * p.ln_n + std::log(2.0));
    const double beta = std::sqrt(g * (lnC + ell_p * p.ln_n + std::log(2.0)));
    const double t = g * alpha + beta;
    p.lam_s = 2.0 * p.nd * t * t / (epsilon * epsilon);
    uint32_t lg = 0;
    while (lg < 32 && ((uint64_t)1 << lg) < (uint64_t)n) lg++;
    p.rounds = lg >= 1 ? lg - 1 : 0;
    return p;
}

void reset_acc(imm_ctx* c)
{
    c->acc_sample_ms = c->acc_select_ms = c->acc_index_ms = 0;
    c->acc_sample_launches = c->acc_launches = c->acc_edges = c->acc_sample_members = 0;
}

// ---------------------------------------------------------------------------
// Batch engine: many IMM queries advance together in waves.  Each query runs
// on a worker context that borrows its graph's device arrays and owns its
// stream and RRR-set state.  A wave runs one sampling batch of every query
// still sampling (phases 1-3 for all of them, one host drain per phase) and
// then one selection launch covering every query that reached its target
// (one CTA per query).  Every query executes exactly the solo path's steps,
// so its result is the same as imm_run's on the same inputs.
// ---------------------------------------------------------------------------
int make_worker(imm_ctx* g, imm_ctx** out, bool own_allocator = false)
{
    *out = nullptr;
    imm_ctx* w = new imm_ctx();
    w->device = g->device;
    w->di = g->di;
    w->alloc = g->alloc;
    w->has_alloc = g->has_alloc && !own_allocator;
    if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete w;
        return set_err(g, IMM_ECUDA, "stream creation failed");
    }
    w->own_stream = true;
    bool ok = cudaMallocHost(&w->pin, sizeof(imm_ctx::Pinned)) == cudaSuccess;
    for (auto& e : w->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        *out = w;  // caller destroys
        return set_err(g, IMM_ECUDA, "event or pinned allocation failed");
    }
    w->n = g->n;
    w->m = g->m;
    w->model = g->model;
    w->row = g->row;
    w->src = g->src;
    w->thr = g->thr;
    w->guide = g->guide;
    w->borrowed = true;
    w->arena_limit = g->arena_limit;
    w->tune = g->tune;
    w->next_batch = w->tune.batch_sets;
    *out = w;
    int rc = dalloc(w, w->cnt, (size_t)w->n * 4);
    if (rc == IMM_OK) rc = dalloc(w, w->cnt_list, (size_t)w->n * 4);
    if (rc == IMM_OK) rc = dalloc(w, w->off, 8 * 1024);
    if (rc == IMM_OK) rc = dalloc(w, w->set_bmp, 4 * 1024);
    if (rc != IMM_OK) return set_err(g, rc, "worker allocation failed: %s", w->err.c_str());
    w->off_cap = 1023;
    cudaMemsetAsync(w->cnt.p, 0, (size_t)w->n * 4, w->stream);
    cudaMemsetAsync(w->cnt_list.p, 0, (size_t)w->n * 4, w->stream);
    cudaMemsetAsync(w->off.p, 0, 8, w->stream);
    w->loaded = true;
    return IMM_OK;
}

void destroy_worker(imm_ctx* w);

struct Job {
    imm_ctx* w = nullptr;
    uint32_t k = 0;
    double eps = 0, ell = 0;
    uint64_t seed = 0;
    ThetaPlan plan{};
    double lb = 1.0;
    uint32_t i = 1;
    int stage = 0;  // 0 sample round i, 1 select round i, 2 sample final, 3 select final, 4 done, 5 failed
    uint64_t target = 0;      // sets of the stream the next selection sees
    uint64_t round_sets = 0;  // sets of the last estimation round's selection
    imm_stats st{};
    int status = IMM_OK;
    std::string err;
    std::chrono::steady_clock::time_point t0;
    uint32_t* seeds_out = nullptr;  // host, k entries
};

void job_fail(Job& j, int rc)
{
    j.status = rc;
    j.err = j.w ? j.w->err : std::string("no worker");
    j.stage = 5;
}

int job_final_target(Job& j)
{
    const double tf = std::ceil(j.plan.lam_s / j.lb);
    if (tf >= 4294967295.0) return set_err(j.w, IMM_EINVAL, "theta exceeds 2^32-2");
    j.st.lb = j.lb;
    j.st.theta = (uint64_t)tf;
    j.target = std::max<uint64_t>(j.st.theta, j.round_sets);
    j.stage = 2;
    return IMM_OK;
}

int job_round_target(Job& j)
{
    const double x = std::ldexp(j.plan.nd, -(int)j.i);
    const double th = std::ceil(j.plan.lam_p / x);
    if (th >= 4294967295.0) return set_err(j.w, IMM_EINVAL, "theta_%u exceeds 2^32-2", j.i);
    j.target = (uint64_t)th;
    j.stage = 0;
    return IMM_OK;
}

// keep_stream: a worker whose resident stream was drawn with the query's own
// seed keeps it; the query's selections then see prefixes of it (sets are a
// pure function of graph, seed and set id, so a prefix of the resident stream
// is exactly the stream the query would sample).
int job_start(Job& j, bool keep_stream = false)
{
    imm_ctx* w = j.w;
    j.t0 = std::chrono::steady_clock::now();
    const bool keep = keep_stream && w->have_stream && w->seed == j.seed && w->nsets > 0;
    if (!keep) drop_stream(w);
    reset_acc(w);
    std::memset(&j.st, 0, sizeof(j.st));
    j.st.reused_sets = keep ? w->nsets : 0;
    j.round_sets = 0;
    j.plan = theta_plan(w->n, j.k, j.eps, j.ell);
    j.st.lambda_prime = j.plan.lam_p;
    j.st.lambda_star = j.plan.lam_s;
    j.lb = 1.0;
    j.i = 1;
    TRY(j.plan.rounds >= 1 ? job_round_target(j) : job_final_target(j));
    return begin_stream(w, j.target, j.seed);
}

int job_after_select(Job& j, uint64_t cov)
{
    imm_ctx* w = j.w;
    if (j.stage == 1) {
        const double x = std::ldexp(j.plan.nd, -(int)j.i);
        const double nF = j.plan.nd * (double)cov / (double)j.target;
        if (j.i - 1 < IMM_MAX_ROUNDS) {
            j.st.theta_i[j.i - 1] = j.target;
            j.st.covered_i[j.i - 1] = cov;
            j.st.sets_i[j.i - 1] = j.target;
        }
        j.st.rounds = j.i;
        j.round_sets = j.target;
        if (nF >= (1.0 + j.plan.eps_p) * x) {
            j.lb = nF / (1.0 + j.plan.eps_p);
            j.st.stopped_early = 1;
        } else if (j.i < j.plan.rounds) {
            ++j.i;
            return job_round_target(j);
        }
        TRY(job_final_target(j));
        // theta within this round's sets: the final selection sees exactly
        // this round's sets, so this round's seeds and coverage are final
        if (j.target != j.round_sets) return IMM_OK;
    }
    // final selection
    std::memcpy(j.seeds_out, w->pin_seeds, (size_t)j.k * 4);
    j.st.num_sets = j.target;
    j.st.covered = cov;
    j.st.members = w->nmembers;
    if (j.target < w->nsets) TRY(prefix_members(w, &j.st.members));
    j.st.edges_examined = w->acc_edges;
    j.st.ms_sample = w->acc_sample_ms;
    j.st.ms_select = w->acc_select_ms;
    j.st.ms_index = w->acc_index_ms;
    j.st.sample_launches = w->acc_sample_launches;
    j.st.kernel_launches = w->acc_launches;
    j.st.sample_edges = w->acc_edges;
    j.st.sample_members = w->acc_sample_members;
    j.st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - j.t0).count();
    j.stage = 4;
    return IMM_OK;
}

// One wave over the active jobs.  `master` is the stream of the selection
// launch; `host` is the context that owns the device copy of the states.
// Per-wave trace lines on stderr when the environment sets IMM_TRACE.
bool trace_on()
{
    static const bool on = std::getenv("IMM_TRACE") != nullptr;
    return on;
}

double ms_since(std::chrono::steady_clock::time_point t)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
}

// The selection launched by one wave runs while the next wave samples the
// other queries; that wave collects it (waiting only if it is still running)
// before it launches its own.  The jobs of an in-flight selection neither
// sample nor select until collected.
// Instances on graphs of at least tune.cluster_min_n vertices select with a
// cluster of CTAs (IMM_SELECT_CLUSTER_MIN_N overrides every tuning; tests use
// 0 to send every instance there, and a value above every n keeps one CTA
// per instance).
uint32_t select_cluster_min_n(const imm_ctx* w)
{
    static const char* e = std::getenv("IMM_SELECT_CLUSTER_MIN_N");
    return e ? (uint32_t)std::strtoul(e, nullptr, 10) : w->tune.cluster_min_n;
}

struct WaveState {
    std::vector<Job*> inflight;
    cudaEvent_t done = nullptr;  // recorded on the master stream after the selection's read-backs
    ~WaveState()
    {
        if (done) cudaEventDestroy(done);
    }
};

int collect_selection(WaveState& ws, imm_ctx* host)
{
    if (ws.inflight.empty()) return IMM_OK;
    std::vector<Job*> L;
    L.swap(ws.inflight);
    const cudaError_t e = cudaEventSynchronize(ws.done);
    if (e != cudaSuccess) {
        for (Job* j : L) job_fail(*j, IMM_ECUDA);
        return cuda_err(host, e, "batched selection");
    }
    for (Job* j : L) {
        const uint64_t cov = select_covered(j->w, j->k, nullptr);
        int rc = bounds_verdict(j->w, reinterpret_cast<unsigned long long*>(static_cast<char*>(j->w->cstate.p) + 32),
                                "selection");
        if (rc == IMM_OK) rc = job_after_select(*j, cov);
        if (rc == IMM_OK && (j->stage == 0 || j->stage == 2)) rc = begin_stream(j->w, j->target, j->seed);
        if (rc != IMM_OK) job_fail(*j, rc);
    }
    return IMM_OK;
}

int run_wave(std::vector<Job*>& jobs, imm_ctx* host, cudaStream_t master, uint64_t* launches, WaveState& ws)
{
    std::vector<Job*> S;
    for (Job* j : jobs) {
        if (j->stage != 0 && j->stage != 2) continue;
        if (j->w->nsets >= j->target) {
            ++j->stage;
            continue;
        }
        S.push_back(j);
    }
    // phase-major: every job's launches are issued before any stream is
    // drained, so the jobs' kernels overlap on the GPU
    const auto tw0 = std::chrono::steady_clock::now();
    double t_sync = 0.0, t_p[3] = {0.0, 0.0, 0.0};
    for (Job* j : S) {
        const int rc = batch_phase1(j->w, j->target);
        if (rc != IMM_OK) job_fail(*j, rc);
    }
    t_p[0] = ms_since(tw0);
    for (Job* j : S) {
        if (j->stage == 5) continue;
        const auto ta = std::chrono::steady_clock::now();
        int rc = cudaStreamSynchronize(j->w->stream) == cudaSuccess ? IMM_OK : IMM_ECUDA;
        t_sync += ms_since(ta);
        if (rc == IMM_OK) rc = batch_phase2(j->w);
        if (rc != IMM_OK) job_fail(*j, rc);
    }
    t_p[1] = ms_since(tw0) - t_p[0];
    for (Job* j : S) {
        if (j->stage == 5) continue;
        bool progress = false;
        const auto ta = std::chrono::steady_clock::now();
        int rc = cudaStreamSynchronize(j->w->stream) == cudaSuccess ? IMM_OK : IMM_ECUDA;
        t_sync += ms_since(ta);
        if (rc == IMM_OK) rc = batch_phase3(j->w, &progress);
        if (rc != IMM_OK) job_fail(*j, rc);
        else if (j->w->nsets >= j->target) ++j->stage;
    }
    const double t_sample = ms_since(tw0);
    t_p[2] = t_sample - t_p[0] - t_p[1];
    if (trace_on() && !S.empty())
        fprintf(stderr, "imm wave phases: %.2f / %.2f / %.2f ms, of which waiting on streams %.2f ms\n", t_p[0], t_p[1],
                t_p[2], t_sync);
    // the previous wave's selection has run beside these phases
    const auto tc0 = std::chrono::steady_clock::now();
    const size_t collected = ws.inflight.size();
    TRY(collect_selection(ws, host));
    const double t_collect = ms_since(tc0);
    std::vector<Job*> L;
    for (Job* j : jobs)
        if (j->stage == 1 || j->stage == 3) L.push_back(j);
    if (L.empty()) {
        if (trace_on())
            fprintf(stderr, "imm wave: sample %zu jobs %.2f ms | collect %zu %.2f ms\n", S.size(), t_sample,
                    collected, t_collect);
        return IMM_OK;
    }
    const auto tp0 = std::chrono::steady_clock::now();
    // selection: prepare each job's state on its stream, one launch for all
    const size_t rec = sizeof(SelectState);
    std::vector<SelectState> states(L.size());
    std::vector<uint32_t> ks(L.size());
    std::vector<Job*> ok;
    std::vector<SelectState> prep(L.size());
    std::vector<int> prc(L.size(), IMM_OK);
    for (size_t t = 0; t < L.size(); ++t) {
        prc[t] = select_prepare(L[t]->w, L[t]->k, &prep[t], L[t]->target);
        if (prc[t] == IMM_OK) cudaEventRecord(L[t]->w->ev[4], L[t]->w->stream);
    }
    // instances on graphs of >= their tuning's cluster_min_n vertices select
    // with a cluster of CTAs each, the others with one CTA; the small ones
    // come first
    auto big = [](const Job* j) { return j->w->n >= select_cluster_min_n(j->w); };
    for (int pass = 0; pass < 2; ++pass) {
        for (size_t t = 0; t < L.size(); ++t) {
            Job* j = L[t];
            if (prc[t] != IMM_OK) {
                if (pass == 0) job_fail(*j, prc[t]);
                continue;
            }
            if (big(j) != (pass == 1)) continue;
            states[ok.size()] = prep[t];
            ks[ok.size()] = j->k;
            cudaStreamWaitEvent(master, j->w->ev[4], 0);
            ok.push_back(j);
        }
    }
    if (ok.empty()) return IMM_OK;
    uint32_t nsmall = 0;
    while (nsmall < ok.size() && !big(ok[nsmall])) ++nsmall;
    const size_t nbytes = ok.size() * (rec + 4) + 16;
    TRY(ensure(host, host->bstates, nbytes));
    // the states are staged through pinned memory the host context keeps
    // (grown geometrically: freeing pinned memory synchronises the device);
    // the previous selection has been collected, so both are free
    if (host->pin_stage_bytes < nbytes) {
        const size_t cap = std::max(nbytes, host->pin_stage_bytes * 2);
        if (host->pin_stage) cudaFreeHost(host->pin_stage);
        host->pin_stage = nullptr;
        host->pin_stage_bytes = 0;
        if (cudaMallocHost(&host->pin_stage, cap) != cudaSuccess) {
            cudaGetLastError();
            return set_err(host, IMM_ECUDA, "pinned staging allocation failed");
        }
        host->pin_stage_bytes = cap;
    }
    if (!ws.done && cudaEventCreateWithFlags(&ws.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ws.done = nullptr;
        return set_err(host, IMM_ECUDA, "event creation failed");
    }
    void* hbuf = host->pin_stage;
    std::memcpy(hbuf, states.data(), ok.size() * rec);
    std::memcpy(static_cast<char*>(hbuf) + ok.size() * rec, ks.data(), ok.size() * 4);
    cudaError_t e = cudaMemcpyAsync(host->bstates.p, hbuf, ok.size() * (rec + 4), cudaMemcpyHostToDevice, master);
    const SelectState* dst = P<SelectState>(host->bstates);
    const uint32_t* dks = reinterpret_cast<const uint32_t*>(static_cast<char*>(host->bstates.p) + ok.size() * rec);
    const uint32_t nbig = (uint32_t)ok.size() - nsmall;
    if (e == cudaSuccess && nsmall) e = launch_select_batch(dst, dks, nsmall, host->di, master);
    if (e == cudaSuccess && nbig) {
        e = launch_select_clusters(dst + nsmall, dks + nsmall, nbig, host->di, master);
        if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
            cudaGetLastError();
            e = launch_select_batch(dst + nsmall, dks + nsmall, nbig, host->di, master);
        }
    }
    if (launches) *launches += (nsmall ? 1 : 0) + (nbig ? 1 : 0);
    for (Job* j : ok) {
        if (e != cudaSuccess) break;
        j->w->acc_launches += 1;
        if (select_readback(j->w, j->k, master) != IMM_OK) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = cudaEventRecord(ws.done, master);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(master);
        for (Job* j : ok) job_fail(*j, IMM_ECUDA);
        return cuda_err(host, e, "batched selection");
    }
    ws.inflight = ok;
    if (trace_on()) {
        uint32_t kmax = 0, nmax = 0;
        for (Job* j : ok) {
            kmax = std::max(kmax, j->k);
            nmax = std::max(nmax, j->w->n);
        }
        fprintf(stderr, "imm wave: sample %zu jobs %.2f ms | collect %zu %.2f ms | select %zu jobs: launch %.2f ms "
                        "(k<=%u, n<=%u)\n", S.size(), t_sample, collected, t_collect, ok.size(), ms_since(tp0), kmax,
                nmax);
    }
    return IMM_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int imm_create(imm_ctx** out, int device, const imm_alloc* alloc, void* stream)
{
    if (!out) return IMM_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return IMM_EINVAL;
    }
    imm_ctx* c = new imm_ctx();
    c->device = device;
    DeviceGuard guard(device);
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    if (alloc && alloc->alloc && alloc->free) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return IMM_ECUDA;
    }
    c->di.sms = prop.multiProcessorCount;
    c->di.max_smem_optin = (int)prop.sharedMemPerBlockOptin;
    c->di.cooperative = prop.cooperativeLaunch;
    for (auto& e : c->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            delete c;
            return IMM_ECUDA;
        }
    }
    if (cudaMallocHost(&c->pin, sizeof(imm_ctx::Pinned)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return IMM_ECUDA;
    }
    *out = c;
    return IMM_OK;
}

void imm_destroy(imm_ctx* c)
{
    if (!c) return;
    DeviceGuard guard(c->device);
    free_graph(c);
    DBuf* bufs[] = {&c->off,      &c->arena,   &c->set_len,  &c->set_pos, &c->set_edges, &c->set_kind,
                    &c->large_q,  &c->long_q,  &c->bmp_rel,  &c->stage,   &c->big,       &c->scalars,   &c->scan_tmp,
                    &c->covered,  &c->newly,   &c->keys,     &c->newly_n, &c->vol_cov,   &c->vol_list,
                    &c->bmp_cov,  &c->ubmp,    &c->ubmp_n,   &c->seeds,   &c->dsegs,     &c->flags,
                    &c->set_bmp,  &c->bmp,     &c->dstate,
                    &c->bmp_set,  &c->bmp_len, &c->cand,     &c->cstate};
    for (DBuf* b : bufs) dfree(c, *b);
    cudaStreamSynchronize(c->stream);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->pin) cudaFreeHost(c->pin);
    if (c->pin_seeds) cudaFreeHost(c->pin_seeds);
    if (c->pin_newly) cudaFreeHost(c->pin_newly);
    if (c->pin_stage) cudaFreeHost(c->pin_stage);
    delete c;
}

const char* imm_last_error(imm_ctx* c)
{
    return c ? c->err.c_str() : "null context";
}

int imm_load_graph(imm_ctx* c, uint32_t n, uint64_t m, const uint64_t* in_row, const uint32_t* in_src,
                   const float* weight, int model)
{
    if (!c) return IMM_EINVAL;
    DeviceGuard guard(c->device);
    return load_graph_common(c, n, m, in_row, in_src, weight, model, cudaMemcpyHostToDevice);
}

int imm_load_graph_device(imm_ctx* c, uint32_t n, uint64_t m, const uint64_t* d_in_row, const uint32_t* d_in_src,
                          const float* d_weight, int model)
{
    if (!c) return IMM_EINVAL;
    DeviceGuard guard(c->device);
    return load_graph_common(c, n, m, d_in_row, d_in_src, d_weight, model, cudaMemcpyDeviceToDevice);
}

int imm_sample(imm_ctx* c, int model, uint64_t theta, uint64_t rng_seed)
{
    if (!c) return IMM_EINVAL;
    DeviceGuard guard(c->device);
    if (!c->loaded) return set_err(c, IMM_ESTATE, "no graph loaded");
    if (model != c->model) return set_err(c, IMM_EINVAL, "model %d differs from the loaded graph's", model);
    return sample_to(c, theta, rng_seed);
}

int imm_select(imm_ctx* c, uint32_t k, uint32_t* seeds_out, uint64_t* covered_out)
{
    if (!c) return IMM_EINVAL;
    DeviceGuard guard(c->device);
    return select_k(c, k, seeds_out, covered_out);
}

int imm_reset_sets(imm_ctx* c)
{
    if (!c) return IMM_EINVAL;
    DeviceGuard guard(c->device);
    drop_stream(c);
    return IMM_OK;
}

int imm_stream_size(imm_ctx* c, uint64_t* num_sets, uint64_t* num_members)
{
    if (!c) return IMM_EINVAL;
    if (num_sets) *num_sets = c->nsets;
    if (num_members) *num_members = c->nmembers;
    return IMM_OK;
}

int imm_set_arena_limit(imm_ctx* c, uint64_t bytes)
{
    if (!c) return IMM_EINVAL;
    c->arena_limit = bytes;
    return IMM_OK;
}

int imm_run(imm_ctx* c, int model, uint32_t k, double epsilon, double ell, uint64_t rng_seed, uint32_t* seeds_out,
            imm_stats* stats_out)
{
    return imm_run_ex(c, model, k, epsilon, ell, rng_seed, 0u, seeds_out, stats_out);
}

int imm_run_ex(imm_ctx* c, int model, uint32_t k, double epsilon, double ell, uint64_t rng_seed, uint32_t flags,
               uint32_t* seeds_out, imm_stats* stats_out)
{
    if (!c) return IMM_EINVAL;
    if (flags & ~IMM_RUN_FRESH_FINAL) return set_err(c, IMM_EINVAL, "unknown flags 0x%x", flags);
    DeviceGuard guard(c->device);
    const auto t0 = std::chrono::steady_clock::now();
    if (!c->loaded) return set_err(c, IMM_ESTATE, "no graph loaded");
    if (model != c->model) return set_err(c, IMM_EINVAL, "model %d differs from the loaded graph's", model);
    if (k == 0 || k > c->n) return set_err(c, IMM_EINVAL, "k must be in [1, n]");
    if (!(epsilon > 0.0 && epsilon < 1.0)) return set_err(c, IMM_EINVAL, "epsilon must be in (0, 1)");
    if (!(ell > 0.0)) return set_err(c, IMM_EINVAL, "ell must be > 0");
    if (!seeds_out) return set_err(c, IMM_EINVAL, "seeds_out is NULL");
    drop_stream(c);
    reset_acc(c);
    imm_stats st;
    std::memset(&st, 0, sizeof(st));

    const ThetaPlan tp = theta_plan(c->n, k, epsilon, ell);
    const double nd = tp.nd, lam_p = tp.lam_p, lam_s = tp.lam_s, eps_p = tp.eps_p;
    const uint32_t rounds = tp.rounds;
    st.lambda_prime = lam_p;
    st.lambda_star = lam_s;

    double lb = 1.0;
    uint64_t last_cov = 0, last_sets = 0;  // the last round's selection
    for (uint32_t i = 1; i <= rounds; i++) {
        const double x = std::ldexp(nd, -(int)i);
        const double th = std::ceil(lam_p / x);
        if (th >= 4294967295.0) return set_err(c, IMM_EINVAL, "theta_%u exceeds 2^32-2", i);
        const uint64_t theta_i = (uint64_t)th;
        TRY(sample_to(c, theta_i, rng_seed));
        uint64_t cov = 0;
        TRY(select_k(c, k, seeds_out, &cov));
        last_cov = cov;
        last_sets = c->nsets;
        const double nF = nd * (double)cov / (double)c->nsets;
        if (i - 1 < IMM_MAX_ROUNDS) {
            st.theta_i[i - 1] = theta_i;
            st.covered_i[i - 1] = cov;
            st.sets_i[i - 1] = c->nsets;
        }
        st.rounds = i;
        if (nF >= (1.0 + eps_p) * x) {
            lb = nF / (1.0 + eps_p);
            st.stopped_early = 1;
            break;
        }
    }
    const double tf = std::ceil(lam_s / lb);
    if (tf >= 4294967295.0) return set_err(c, IMM_EINVAL, "theta exceeds 2^32-2");
    const uint64_t theta = (uint64_t)tf;
    st.lb = lb;
    st.theta = theta;
    bool reuse = false;
    if (flags & IMM_RUN_FRESH_FINAL) {
        drop_stream(c);
        TRY(sample_to(c, theta, rng_seed ^ IMM_FRESH_FINAL_KEY));
    } else {
        TRY(sample_to(c, std::max<uint64_t>(theta, c->nsets), rng_seed));
        // theta within the stream the last round selected over: the final
        // selection's sets are that round's, so its seeds (already in
        // seeds_out) and coverage are the final ones
        reuse = last_sets > 0 && c->nsets == last_sets;
    }
    uint64_t cov = last_cov;
    if (!reuse) TRY(select_k(c, k, seeds_out, &cov));
    st.num_sets = c->nsets;
    st.covered = cov;
    st.members = c->nmembers;
    st.edges_examined = c->acc_edges;
    st.ms_sample = c->acc_sample_ms;
    st.ms_select = c->acc_select_ms;
    st.ms_index = c->acc_index_ms;
    st.sample_launches = c->acc_sample_launches;
    st.kernel_launches = c->acc_launches;
    st.sample_edges = c->acc_edges;
    st.sample_members = c->acc_sample_members;
    st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats_out) *stats_out = st;
    return IMM_OK;
}

// OPIM-style early stop (Sec. VI cites OPIM, Tang et al. SIGMOD 2018; this
// follows its OPIM-C procedure).  R1 is the context's own stream under
// rng_seed; R2 lives in a worker context on the same graph under rng_seed ^
// IMM_OPIM_KEY.  Both double each round; the greedy over R1 gives the seeds
// and R1 coverage (upper confidence bound on OPT, the optimum's coverage
// bounded by the greedy's over 1 - (1 - 1/k)^k), the seeds' R2 coverage gives
// a lower confidence bound on their spread, and sampling stops once
// lower / upper >= 1 - 1/e - eps.  delta = n^-ell.  Host fp64, no FMA
// contraction, in the same operation order as any plain evaluation.
int imm_run_opim(imm_ctx* c, int model, uint32_t k, double epsilon, double ell, uint64_t rng_seed,
                 uint32_t* seeds_out, imm_opim_stats* stats_out)
{
    if (!c) return IMM_EINVAL;
    DeviceGuard guard(c->device);
    const auto t0c = std::chrono::steady_clock::now();
    if (!c->loaded) return set_err(c, IMM_ESTATE, "no graph loaded");
    if (model != c->model) return set_err(c, IMM_EINVAL, "model %d differs from the loaded graph's", model);
    if (k == 0 || k > c->n) return set_err(c, IMM_EINVAL, "k must be in [1, n]");
    if (!(epsilon > 0.0 && epsilon < 1.0)) return set_err(c, IMM_EINVAL, "epsilon must be in (0, 1)");
    if (!(ell > 0.0)) return set_err(c, IMM_EINVAL, "ell must be > 0");
    if (!seeds_out) return set_err(c, IMM_EINVAL, "seeds_out is NULL");
    const double nd = (double)c->n;
    const double ln_n = std::log(nd);
    const double delta = std::exp(-ell * ln_n);
    double lnC = 0.0;
    for (uint32_t i = 1; i <= k; i++) lnC += std::log((double)(c->n - k + i)) - std::log((double)i);
    const double g = 1.0 - 1.0 / kE;
    const double l6 = std::log(6.0 / delta);
    const double tt = g * std::sqrt(l6) + std::sqrt(g * (lnC + l6));
    const double theta_max = 2.0 * nd * tt * tt / (epsilon * epsilon * (double)k);
    const double theta_0 = theta_max * epsilon * epsilon * (double)k / nd;
    double im = std::ceil(std::log2(theta_max / theta_0));
    if (im < 1.0) im = 1.0;
    const double a2 = std::log(3.0 * im / delta);
    const double a1 = a2 + lnC;
    const uint32_t i_max = (uint32_t)im;
    const double t0 = std::ceil(theta_0);
    if (t0 * std::ldexp(1.0, (int)i_max - 1) >= 4294967295.0)
        return set_err(c, IMM_EINVAL, "the last round's collections would reach 2^32-1 sets");
    const double ratio = 1.0 - std::pow(1.0 - 1.0 / (double)k, (double)k);
    const double target = 1.0 - 1.0 / kE - epsilon;

    imm_opim_stats st;
    std::memset(&st, 0, sizeof(st));
    st.i_max = i_max;
    st.theta_max = theta_max;
    st.theta_0 = theta_0;
    drop_stream(c);
    reset_acc(c);
    TRY(ensure(c, c->flags, 64));
    imm_ctx* w = nullptr;
    int rc = make_worker(c, &w);
    uint64_t cov_launches = 0;
    for (uint32_t i = 1; rc == IMM_OK && i <= i_max; i++) {
        const uint64_t theta = (uint64_t)(t0 * std::ldexp(1.0, (int)i - 1));
        rc = sample_to(c, theta, rng_seed);
        if (rc == IMM_OK && (rc = sample_to(w, theta, rng_seed ^ IMM_OPIM_KEY)) != IMM_OK)
            rc = set_err(c, rc, "second collection: %s", w->err.c_str());
        uint64_t cov1 = 0, cov2 = 0;
        if (rc == IMM_OK) rc = select_k(c, k, seeds_out, &cov1);
        if (rc == IMM_OK) {
            // the selection left picked[v] = 1 exactly for the k seeds
            CoverageArgs a;
            a.nsets = w->nsets;
            a.words = (uint32_t)(((uint64_t)c->n + 31) / 32);
            a.k = k;
            a.off = P<uint64_t>(w->off);
            a.arena = P<uint32_t>(w->arena);
            a.set_bmp = P<uint32_t>(w->set_bmp);
            a.bmp = P<uint32_t>(w->bmp);
            a.flag = P<uint8_t>(c->picked);
            a.seeds = P<uint32_t>(c->seeds);
            a.out = P<unsigned long long>(c->flags);
            cudaError_t e = launch_coverage(a, c->di, c->stream);
            unsigned long long hc = 0;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, c->flags.p, 8, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) rc = cuda_err(c, e, "seed-set coverage of the second collection");
            cov2 = hc;
            cov_launches += 1;
        }
        if (rc != IMM_OK) break;
        const double th = (double)theta;
        const double lam_u = (double)cov1 / ratio;
        const double up = std::sqrt(lam_u + a1 / 2.0) + std::sqrt(a1 / 2.0);
        const double lo = std::sqrt((double)cov2 + 2.0 * a2 / 9.0) - std::sqrt(a2 / 2.0);
        const double upper = up * up * nd / th;
        const double lower = (lo * lo - a2 / 18.0) * nd / th;
        const double alpha = lower / upper;
        if (i - 1 < IMM_MAX_ROUNDS) {
            st.sets_i[i - 1] = theta;
            st.cov1_i[i - 1] = cov1;
            st.cov2_i[i - 1] = cov2;
            st.upper_i[i - 1] = upper;
            st.lower_i[i - 1] = lower;
        }
        st.rounds = i;
        st.alpha = alpha;
        if (alpha >= target) {
            st.stopped_early = i < i_max ? 1u : 0u;
            break;
        }
    }
    if (w) {
        st.kernel_launches = w->acc_launches;
        destroy_worker(w);
    }
    if (rc != IMM_OK) return rc;
    st.kernel_launches += c->acc_launches + cov_launches;
    st.ms_sample = c->acc_sample_ms;
    st.ms_select = c->acc_select_ms;
    st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0c).count();
    if (stats_out) *stats_out = st;
    return IMM_OK;
}

// Members of one stored set, sorted ascending (lists are sorted here, bitmaps
// are expanded in id order).
static int fetch_set(imm_ctx* c, uint64_t id, std::vector<uint32_t>& out)
{
    uint64_t o[2];
    uint32_t bid = kEmpty;
    CK(cudaMemcpyAsync(o, P<uint64_t>(c->off) + id, 16, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&bid, P<uint32_t>(c->set_bmp) + id, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out.clear();
    if (bid == kEmpty) {
        out.resize(o[1] - o[0]);
        if (!out.empty()) {
            CK(cudaMemcpyAsync(out.data(), P<uint32_t>(c->arena) + o[0], out.size() * 4, cudaMemcpyDeviceToHost,
                               c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        std::sort(out.begin(), out.end());
    } else {
        const uint64_t words = ((uint64_t)c->n + 31) / 32;
        std::vector<uint32_t> bits(words);
        CK(cudaMemcpyAsync(bits.data(), P<uint32_t>(c->bmp) + (uint64_t)bid * words, words * 4,
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (uint64_t w = 0; w < words; ++w)
            for (uint32_t x = bits[w]; x; x &= x - 1) out.push_back((uint32_t)(w * 32 + __builtin_ctz(x)));
    }
    return IMM_OK;
}

int imm_get_set(imm_ctx* c, uint64_t set_id, uint32_t* buf, uint32_t cap, uint32_t* len)
{
    if (!c) return IMM_EINVAL;
    DeviceGuard guard(c->device);
    if (set_id >= c->nsets || !len) return set_err(c, IMM_EINVAL, "set id out of range");
    std::vector<uint32_t> m;
    TRY(fetch_set(c, set_id, m));
    *len = (uint32_t)m.size();
    if (m.size() > cap || (!m.empty() && !buf))
        return set_err(c, IMM_EINVAL, "set has %zu members, cap %u", m.size(), cap);
    std::copy(m.begin(), m.end(), buf);
    return IMM_OK;
}

int imm_get_sets(imm_ctx* c, uint64_t first, uint64_t count, uint64_t* off_out, uint32_t* mem_out, uint64_t cap)
{
    if (!c) return IMM_EINVAL;
    DeviceGuard guard(c->device);
    if (first > c->nsets || count > c->nsets - first || !off_out)
        return set_err(c, IMM_EINVAL, "range outside the stream");
    std::vector<uint64_t> lo(count + 1);
    std::vector<uint32_t> bid(count ? count : 1);
    CK(cudaMemcpyAsync(lo.data(), P<uint64_t>(c->off) + first, (count + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    if (count)
        CK(cudaMemcpyAsync(bid.data(), P<uint32_t>(c->set_bmp) + first, count * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // true sizes: list lengths, and bitmap sizes for bitmap-stored sets
    std::vector<uint32_t> blen(count ? count : 1, 0);
    for (uint64_t i = 0; i < count; ++i) {
        if (bid[i] != kEmpty) {
            CK(cudaMemcpyAsync(&blen[i], P<uint32_t>(c->bmp_len) + bid[i], 4, cudaMemcpyDeviceToHost, c->stream));
        }
    }
    CK(cudaStreamSynchronize(c->stream));
    off_out[0] = 0;
    for (uint64_t i = 0; i < count; ++i)
        off_out[i + 1] = off_out[i] + (bid[i] == kEmpty ? lo[i + 1] - lo[i] : (uint64_t)blen[i]);
    const uint64_t total = off_out[count];
    if (total > cap || (total && !mem_out))
        return set_err(c, IMM_EINVAL, "range holds %llu members, cap %llu", (unsigned long long)total,
                       (unsigned long long)cap);
    // lists in stored (traversal) order, bitmaps expanded in id order
    std::vector<uint32_t> lists(lo[count] - lo[0]);
    if (!lists.empty()) {
        CK(cudaMemcpyAsync(lists.data(), P<uint32_t>(c->arena) + lo[0], lists.size() * 4, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    std::vector<uint32_t> tmp;
    for (uint64_t i = 0; i < count; ++i) {
        if (bid[i] == kEmpty) {
            std::copy(lists.begin() + (lo[i] - lo[0]), lists.begin() + (lo[i + 1] - lo[0]), mem_out + off_out[i]);
        } else {
            TRY(fetch_set(c, first + i, tmp));
            std::copy(tmp.begin(), tmp.end(), mem_out + off_out[i]);
        }
    }
    return IMM_OK;
}

int imm_get_counts(imm_ctx* c, uint32_t* cnt_out)
{
    if (!c) return IMM_EINVAL;
    DeviceGuard guard(c->device);
    if (!c->loaded) return set_err(c, IMM_ESTATE, "no graph loaded");
    if (!cnt_out) return set_err(c, IMM_EINVAL, "cnt_out is NULL");
    CK(cudaMemcpyAsync(cnt_out, c->cnt.p, (size_t)c->n * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return IMM_OK;
}

}  // extern "C"

namespace {
void destroy_worker(imm_ctx* w)
{
    if (!w) return;
    cudaStream_t st = w->own_stream ? w->stream : nullptr;
    imm_destroy(w);
    if (st) cudaStreamDestroy(st);
}
}  // namespace

extern "C" int imm_run_batch(const imm_query* queries, uint32_t nq, uint32_t* seeds_out, imm_stats* stats_out,
                             int* status_out)
{
    if (nq == 0) return IMM_OK;
    if (!queries || !seeds_out) return IMM_EINVAL;
    imm_ctx* g0 = queries[0].graph;
    if (!g0) return IMM_EINVAL;
    DeviceGuard guard(g0->device);
    for (uint32_t q = 0; q < nq; ++q) {
        const imm_query& Q = queries[q];
        if (!Q.graph || !Q.graph->loaded || Q.graph->device != g0->device)
            return set_err(g0, IMM_EINVAL, "query %u: graph context missing, not loaded or on another device", q);
        if (Q.k == 0 || Q.k > Q.graph->n || !(Q.epsilon > 0.0 && Q.epsilon < 1.0) || !(Q.ell > 0.0))
            return set_err(g0, IMM_EINVAL, "query %u: bad k, epsilon or ell", q);
    }
    // every graph finished loading before any worker stream reads it
    for (uint32_t q = 0; q < nq; ++q) {
        const cudaError_t e = cudaStreamSynchronize(queries[q].graph->stream);
        if (e != cudaSuccess) return cuda_err(g0, e, "graph stream");
    }
    std::vector<Job> jobs(nq);
    std::vector<Job*> active;
    uint64_t off = 0;
    int rc = IMM_OK;
    const auto tb0 = std::chrono::steady_clock::now();
    for (uint32_t q = 0; q < nq; ++q) {
        Job& j = jobs[q];
        j.k = queries[q].k;
        j.eps = queries[q].epsilon;
        j.ell = queries[q].ell;
        j.seed = queries[q].rng_seed;
        j.seeds_out = seeds_out + off;
        off += j.k;
        // workers allocate through the graph context's allocator when it has
        // one (a caching allocator hands each call's buffers back to the next
        // call at once, which stream-ordered pool allocations from new
        // streams measured about 2x slower)
        rc = make_worker(queries[q].graph, &j.w);
        if (rc != IMM_OK) break;
        rc = job_start(j);
        if (rc != IMM_OK) job_fail(j, rc);
        active.push_back(&j);
        rc = IMM_OK;
    }
    uint64_t launches = 0;
    const double t_setup = ms_since(tb0);
    const auto tb1 = std::chrono::steady_clock::now();
    {
        // the queries go in two cohorts one wave apart: while one cohort's
        // batched selection runs, the other samples (in one cohort every
        // query would wait for the selection before sampling again)
        std::vector<Job*> later;
        if (active.size() >= 8) {
            std::vector<Job*> first;
            for (size_t t = 0; t < active.size(); ++t) (t % 2 ? later : first).push_back(active[t]);
            active.swap(first);
        }
        WaveState ws;
        while (rc == IMM_OK) {
            bool any = !later.empty();
            for (Job* j : active) any = any || (j->stage < 4);
            if (!any) break;
            rc = run_wave(active, g0, g0->stream, &launches, ws);
            if (!later.empty()) {
                active.insert(active.end(), later.begin(), later.end());
                later.clear();
            }
        }
        // nothing may still run on the workers' buffers when they are freed
        cudaStreamSynchronize(g0->stream);
    }
    const double t_waves = ms_since(tb1);
    const auto tb2 = std::chrono::steady_clock::now();
    for (uint32_t q = 0; q < nq; ++q) {
        if (status_out) status_out[q] = jobs[q].stage == 4 ? IMM_OK : (jobs[q].status ? jobs[q].status : rc);
        if (stats_out) stats_out[q] = jobs[q].st;
        destroy_worker(jobs[q].w);
    }
    if (trace_on())
        fprintf(stderr, "imm batch: %u queries: set-up %.2f ms, waves %.2f ms, tear-down %.2f ms\n", nq, t_setup,
                t_waves, ms_since(tb2));
    return rc;
}

extern "C" int imm_build_flags(void)
{
    return kBoundsChecked ? IMM_BUILD_BOUNDS_CHECK : 0;
}

extern "C" int imm_set_tuning(imm_ctx* c, const imm_tuning* t)
{
    if (!c || !t) return IMM_EINVAL;
    if (t->batch_sets < 256) return set_err(c, IMM_EINVAL, "batch_sets must be >= 256");
    c->tune = *t;
    if (c->nsets == 0) c->next_batch = c->tune.batch_sets;
    return IMM_OK;
}

extern "C" int imm_get_tuning(imm_ctx* c, imm_tuning* out)
{
    if (!c || !out) return IMM_EINVAL;
    *out = c->tune;
    return IMM_OK;
}

// The autotuner's grid: the selection team threshold of batched instances
// (cluster from 2^12, 2^14, 2^16 vertices, or never) crossed with the
// candidate-list argmax on or off and two sampling batch sizes.
static void tune_candidates(const imm_tuning& base, imm_tuning* out)
{
    const uint32_t cmin[4] = {1u << 12, 1u << 14, 1u << 16, 0xFFFFFFFFu};
    const uint32_t cand[3] = {1u, 0u, 1u};
    const uint32_t bsets[3] = {1u << 22, 1u << 22, 1u << 16};
    int i = 0;
    for (uint32_t a = 0; a < 4; ++a) {
        for (uint32_t b = 0; b < 3; ++b) {
            imm_tuning t = base;
            t.cluster_min_n = cmin[a];
            t.select_cand = cand[b];
            t.batch_sets = bsets[b];
            out[i++] = t;
        }
    }
}

extern "C" int imm_autotune_batch(const imm_query* queries, uint32_t nq, uint32_t reps, imm_tuning* best_out,
                                  double* times_ms_out, imm_tuning* candidates_out)
{
    if (nq == 0 || !queries) return IMM_EINVAL;
    std::vector<imm_ctx*> graphs;
    uint64_t total_k = 0;
    for (uint32_t q = 0; q < nq; ++q) {
        if (!queries[q].graph) return IMM_EINVAL;
        if (std::find(graphs.begin(), graphs.end(), queries[q].graph) == graphs.end())
            graphs.push_back(queries[q].graph);
        total_k += queries[q].k;
    }
    if (reps == 0) reps = 1;
    std::vector<imm_tuning> saved;
    for (imm_ctx* g : graphs) saved.push_back(g->tune);
    imm_tuning cands[IMM_TUNE_CANDIDATES];
    tune_candidates(graphs[0]->tune, cands);
    std::vector<uint32_t> seeds(std::max<uint64_t>(total_k, 1));
    std::vector<int> status(nq);
    double best_ms = 0.0;
    int best = -1, rc = IMM_OK;
    for (int i = 0; i < IMM_TUNE_CANDIDATES && rc == IMM_OK; ++i) {
        for (imm_ctx* g : graphs) g->tune = cands[i];
        double sum = 0.0;
        uint32_t timed = 0;
        const uint32_t runs = reps > 1 ? reps + 1 : 1;
        for (uint32_t r = 0; r < runs && rc == IMM_OK; ++r) {
            const auto t0 = std::chrono::steady_clock::now();
            rc = imm_run_batch(queries, nq, seeds.data(), nullptr, status.data());
            const double ms = ms_since(t0);
            for (uint32_t q = 0; q < nq && rc == IMM_OK; ++q)
                if (status[q] != IMM_OK) rc = status[q];
            if (reps == 1 || r > 0) {
                sum += ms;
                ++timed;
            }
        }
        const double mean = timed ? sum / timed : 0.0;
        if (times_ms_out) times_ms_out[i] = mean;
        if (rc == IMM_OK && (best < 0 || mean < best_ms)) {
            best = i;
            best_ms = mean;
        }
    }
    if (rc != IMM_OK || best < 0) {
        for (size_t i = 0; i < graphs.size(); ++i) graphs[i]->tune = saved[i];
        return rc != IMM_OK ? rc : IMM_EINVAL;
    }
    for (imm_ctx* g : graphs) g->tune = cands[best];
    if (best_out) *best_out = cands[best];
    if (candidates_out) std::memcpy(candidates_out, cands, sizeof(cands));
    return IMM_OK;
}

// ===========================================================================
// Served IMM: a continuous-batching loop on a host thread.  Queries are
// submitted at any time; between waves the loop admits pending queries (up
// to max_active in flight and while the workers' device memory stays under
// the budget), runs one wave over every admitted query, and retires the
// finished ones with their latency.  Admitted queries join the next wave, so
// newcomers overlap on the GPU with queries already in flight.  Each result
// equals the query's solo imm_run.  Server workers allocate with the
// library's own stream-ordered allocator, so the loop thread never calls back
// into the caller's allocator.
// ===========================================================================
namespace {

struct ServedQuery {
    uint64_t id = 0;
    uint32_t graph = 0;
    Job job;
    std::vector<uint32_t> seeds;
    std::chrono::steady_clock::time_point submitted, admitted, finished;
};

}  // namespace

struct imm_server {
    std::vector<imm_ctx*> graphs;
    imm_server_config cfg{};
    imm_ctx* host = nullptr;  // master stream + device copy of selection states
    std::vector<std::vector<imm_ctx*>> idle;  // per graph: workers ready for reuse
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServedQuery*> pending;
    std::vector<ServedQuery*> active;
    std::deque<ServedQuery*> done;
    std::unordered_map<uint64_t, ServedQuery*> finished;
    std::atomic<bool> stop{false};
    std::thread loop;
    uint64_t next_id = 1;
    uint64_t waves = 0, launches = 0;
    int fatal = IMM_OK;
    std::string err;
    WaveState wave;  // the selection in flight between waves
};

namespace {

uint64_t active_bytes(imm_server* s)
{
    uint64_t b = s->host ? s->host->dev_bytes : 0;
    for (ServedQuery* q : s->active) b += q->job.w ? q->job.w->dev_bytes : 0;
    for (auto& v : s->idle)
        for (imm_ctx* w : v) b += w->dev_bytes;
    return b;
}

void server_loop(imm_server* s)
{
    DeviceGuard guard(s->host->device);
    while (!s->stop.load()) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->active.empty() && s->pending.empty())
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
            // admission: concurrency and device memory.  Idle workers are
            // reclaimed when memory blocks admission, and one query is always
            // admitted when none is in flight, so the queue always drains.
            while (!s->pending.empty() && s->active.size() < s->cfg.max_active) {
                if (s->cfg.memory_budget_bytes && active_bytes(s) >= s->cfg.memory_budget_bytes) {
                    for (auto& v : s->idle) {
                        for (imm_ctx* w : v) destroy_worker(w);
                        v.clear();
                    }
                    if (!s->active.empty() && active_bytes(s) >= s->cfg.memory_budget_bytes) break;
                }
                ServedQuery* q = s->pending.front();
                s->pending.pop_front();
                q->admitted = std::chrono::steady_clock::now();
                imm_ctx* w = nullptr;
                auto& pool = s->idle[q->graph];
                int rc = IMM_OK;
                if (!pool.empty()) {
                    // with shared streams, an idle worker holding a stream
                    // drawn with this query's seed is taken first
                    size_t pick = pool.size() - 1;
                    if (s->cfg.share_streams) {
                        for (size_t i = 0; i < pool.size(); ++i) {
                            if (pool[i]->have_stream && pool[i]->seed == q->job.seed && pool[i]->nsets > 0) {
                                pick = i;
                                break;
                            }
                        }
                    }
                    w = pool[pick];
                    pool.erase(pool.begin() + (long)pick);
                } else {
                    rc = make_worker(s->graphs[q->graph], &w, true);
                }
                q->job.w = w;
                if (rc == IMM_OK && s->cfg.memory_budget_bytes) w->arena_limit = s->cfg.memory_budget_bytes / 2;
                if (rc == IMM_OK) rc = job_start(q->job, s->cfg.share_streams != 0);
                if (rc != IMM_OK) job_fail(q->job, rc);
                s->active.push_back(q);
            }
        }
        if (s->active.empty()) continue;
        std::vector<Job*> jobs;
        for (ServedQuery* q : s->active) jobs.push_back(&q->job);
        const int rc = run_wave(jobs, s->host, s->host->stream, &s->launches, s->wave);
        ++s->waves;
        std::lock_guard<std::mutex> lk(s->mu);
        if (rc != IMM_OK) {
            // no selection may still run on a worker that is freed below
            cudaStreamSynchronize(s->host->stream);
            s->wave.inflight.clear();
            // the loop stops: every query in flight or still queued completes
            // with the error, so no client waits forever
            s->fatal = rc;
            s->err = s->host->err;
            for (ServedQuery* q : s->active) {
                if (q->job.stage < 4) job_fail(q->job, rc);
            }
            while (!s->pending.empty()) {
                ServedQuery* q = s->pending.front();
                s->pending.pop_front();
                q->admitted = q->finished = std::chrono::steady_clock::now();
                job_fail(q->job, rc);
                s->done.push_back(q);
                s->finished[q->id] = q;
            }
        }
        std::vector<ServedQuery*> still;
        for (ServedQuery* q : s->active) {
            if (q->job.stage >= 4) {
                q->finished = std::chrono::steady_clock::now();
                if (q->job.w) {
                    // shared streams: the idle worker keeps the query's stream
                    // for a later query with the same seed
                    if (!s->cfg.share_streams || q->job.stage != 4) drop_stream(q->job.w);
                    cudaStreamSynchronize(q->job.w->stream);
                    if (q->job.stage == 4 && s->idle[q->graph].size() < kServerIdlePerGraph)
                        s->idle[q->graph].push_back(q->job.w);
                    else
                        destroy_worker(q->job.w);
                    q->job.w = nullptr;
                }
                s->done.push_back(q);
                s->finished[q->id] = q;
            } else {
                still.push_back(q);
            }
        }
        s->active.swap(still);
        if (rc != IMM_OK) break;
    }
}

}  // namespace

extern "C" {

int imm_server_create(imm_server** out, imm_ctx* const* graphs, uint32_t ngraphs, const imm_server_config* cfg)
{
    if (!out || !graphs || ngraphs == 0) return IMM_EINVAL;
    *out = nullptr;
    for (uint32_t i = 0; i < ngraphs; ++i)
        if (!graphs[i] || !graphs[i]->loaded || graphs[i]->device != graphs[0]->device) return IMM_EINVAL;
    DeviceGuard guard(graphs[0]->device);
    for (uint32_t i = 0; i < ngraphs; ++i)
        if (cudaStreamSynchronize(graphs[i]->stream) != cudaSuccess) return IMM_ECUDA;
    imm_server* s = new imm_server();
    s->graphs.assign(graphs, graphs + ngraphs);
    s->idle.resize(ngraphs);
    if (cfg) s->cfg = *cfg;
    if (s->cfg.max_active == 0) s->cfg.max_active = 64;
    int rc = make_worker(graphs[0], &s->host, true);
    if (rc != IMM_OK) {
        destroy_worker(s->host);
        delete s;
        return rc;
    }
    s->loop = std::thread(server_loop, s);
    *out = s;
    return IMM_OK;
}

int imm_server_submit(imm_server* s, uint32_t graph, uint32_t k, double epsilon, double ell, uint64_t rng_seed,
                      uint64_t* id_out)
{
    if (!s || graph >= s->graphs.size()) return IMM_EINVAL;
    imm_ctx* g = s->graphs[graph];
    if (k == 0 || k > g->n || !(epsilon > 0.0 && epsilon < 1.0) || !(ell > 0.0)) return IMM_EINVAL;
    ServedQuery* q = new ServedQuery();
    q->graph = graph;
    q->job.k = k;
    q->job.eps = epsilon;
    q->job.ell = ell;
    q->job.seed = rng_seed;
    q->seeds.assign(k, 0);
    q->job.seeds_out = q->seeds.data();
    q->submitted = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal != IMM_OK) {
            delete q;
            return s->fatal;
        }
        q->id = s->next_id++;
        s->pending.push_back(q);
    }
    s->cv.notify_one();
    if (id_out) *id_out = q->id;
    return IMM_OK;
}

int imm_server_poll(imm_server* s, imm_completion* out, uint32_t cap, uint32_t* n_out)
{
    if (!s || !n_out || (cap && !out)) return IMM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    uint32_t n = 0;
    while (n < cap && !s->done.empty()) {
        ServedQuery* q = s->done.front();
        s->done.pop_front();
        imm_completion& c = out[n++];
        c.id = q->id;
        c.status = q->job.stage == 4 ? IMM_OK : (q->job.status ? q->job.status : IMM_ECUDA);
        c.latency_ms = std::chrono::duration<double, std::milli>(q->finished - q->submitted).count();
        c.queue_ms = std::chrono::duration<double, std::milli>(q->admitted - q->submitted).count();
    }
    *n_out = n;
    return IMM_OK;
}

int imm_server_take(imm_server* s, uint64_t id, uint32_t* seeds_out, uint32_t k, imm_stats* stats_out)
{
    if (!s) return IMM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->finished.find(id);
    if (it == s->finished.end()) return IMM_ESTATE;
    ServedQuery* q = it->second;
    if (q->job.stage != 4) {
        const int st = q->job.status ? q->job.status : IMM_ECUDA;
        s->finished.erase(it);
        delete q;
        return st;
    }
    if (seeds_out) {
        if (k < q->job.k) return IMM_EINVAL;
        std::memcpy(seeds_out, q->seeds.data(), (size_t)q->job.k * 4);
    }
    if (stats_out) *stats_out = q->job.st;
    s->finished.erase(it);
    delete q;
    return IMM_OK;
}

int imm_server_info(imm_server* s, uint64_t* pending, uint64_t* active, uint64_t* waves, uint64_t* device_bytes)
{
    if (!s) return IMM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (pending) *pending = s->pending.size();
    if (active) *active = s->active.size();
    if (waves) *waves = s->waves;
    if (device_bytes) *device_bytes = active_bytes(s);
    return s->fatal;
}

void imm_server_destroy(imm_server* s)
{
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_one();
    if (s->loop.joinable()) s->loop.join();
    DeviceGuard guard(s->host->device);
    cudaStreamSynchronize(s->host->stream);  // a selection may still be in flight
    for (ServedQuery* q : s->active) {
        destroy_worker(q->job.w);
        delete q;
    }
    for (ServedQuery* q : s->pending) delete q;
    for (auto& kv : s->finished) delete kv.second;
    for (auto& v : s->idle)
        for (imm_ctx* w : v) destroy_worker(w);
    destroy_worker(s->host);
    delete s;
}

}  // extern "C"
