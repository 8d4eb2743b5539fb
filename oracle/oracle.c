/*
 * IMM oracle: a plain, slow, single-threaded CPU implementation of what the
 * GPU hot path computes.  TEST INFRASTRUCTURE ONLY: tests/, the smoke check
 * and the benchmark's CPU-baseline leg may call it; the product path never
 * does.  It shares no code, header or table with the CUDA library.
 *
 * What it follows (EfficientIMM, arXiv 2411.09473):
 *   - Algorithm 1 (IMM workflow, Sec. II-B): sampling rounds that estimate
 *     theta, extend the RRR-set stream and lower-bound OPT, then a final
 *     selection.  The three named-but-undefined steps (Theta_Estimation,
 *     OPT_Lower_Bound, Set_Theta) follow Tang, Shi & Xiao, SIGMOD 2015 (the
 *     paper's reference for IMM), restated in orc_theta_params below.
 *   - Algorithm 3 (Generate_RRRsets with kernel fusion, Sec. IV-B): BFS from a
 *     uniformly drawn root over in-edges, an unvisited in-neighbour joining
 *     when the diffusion coin says so, then one counter increment per member.
 *   - Algorithm 2 (Find_Most_Influential_Set, Sec. IV-A): global occurrence
 *     counter, k rounds of argmax, and for every remaining set holding the
 *     pick, decrement all its members' counters and drop the set.
 *   - IC and LT models as defined in Sec. II-A.
 *
 * Readings where the paper is silent (all fixed identically on both sides):
 *   - RNG: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed
 *     low 32, seed high 32).  Root of set s: (w0,w1) = P(s_lo,s_hi,0,1),
 *     root = ((w1<<32|w0) * n) >> 64.  IC coin of in-edge e for set s:
 *     w = P(s_lo,s_hi,e>>2,2)[e&3], live iff (w>>8) < thr[e].  LT draw at
 *     vertex v for set s: r = P(s_lo,s_hi,v,3)[0] >> 8.
 *   - IC threshold thr[e] = ceilf(p_e * 2^24) in fp32 (exact), so
 *     P(live) = thr/2^24; p=1 always live, p=0 never.
 *   - LT: cthr_j = min(ceil(cw_j * 2^24), 2^24) where cw_j is the fp64
 *     left-to-right running sum of the head's fp32 in-edge weights in CSR
 *     order (an fp32 running sum drifts by ~1e-3 over 10^5 in-edges).  The walk picks
 *     the first j with r < cthr_j; none -> stop; an already-visited source ->
 *     stop; else the source joins and the walk continues from it.
 *   - Greedy: ties go to the lowest vertex id, already-picked vertices are
 *     excluded, and picking continues at count 0 so |S| = k.
 *   - theta control: loop i = 1 .. ceil(log2 n) - 1, theta_i = ceil(lambda'/x),
 *     stop test ">=", sets reused in the final selection, lambda* uses eps.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_IC 0
#define ORC_LT 1
/* Euler's number, the double nearest e. */
#define ORC_E 2.71828182845904523536

/* ------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition (SC'11).      */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += W0; k1 += W1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_for(uint64_t seed, uint64_t set_id, uint32_t c2, uint32_t tag, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)set_id, (uint32_t)(set_id >> 32), c2, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Alg. 3 / Sec. II-B: the start vertex is drawn uniformly from V. */
uint32_t orc_root(uint64_t seed, uint64_t set_id, uint32_t n)
{
    uint32_t w[4];
    philox_for(seed, set_id, 0u, 1u, w);
    uint64_t x = ((uint64_t)w[1] << 32) | w[0];
    /* (x * n) >> 64 with a 128-bit product written out in 32-bit halves. */
    uint64_t xl = x & 0xFFFFFFFFull, xh = x >> 32;
    uint64_t lo = xl * (uint64_t)n;
    uint64_t hi = xh * (uint64_t)n + (lo >> 32);
    return (uint32_t)(hi >> 32);
}

/* IC threshold (reading: fp32, 24-bit). */
uint32_t orc_ic_threshold(float p)
{
    return (uint32_t)ceilf(p * 16777216.0f);
}

/* IC coin of in-edge e in set set_id (Sec. II-A: edge live w.p. p_uv). */
int orc_ic_live(uint64_t seed, uint64_t set_id, uint32_t e, uint32_t thr)
{
    uint32_t w[4];
    philox_for(seed, set_id, e >> 2, 2u, w);
    return (w[e & 3u] >> 8) < thr;
}

/* LT 24-bit draw at vertex v in set set_id. */
uint32_t orc_lt_draw(uint64_t seed, uint64_t set_id, uint32_t v)
{
    uint32_t w[4];
    philox_for(seed, set_id, v, 3u, w);
    return w[0] >> 8;
}

/* ------------------------------------------------------------------ */
/* theta control (Alg. 1; Tang, Shi, Xiao 2015).                       */
/* out: [0] ell', [1] eps', [2] ln C(n,k), [3] lambda', [4] lambda*,   */
/*      [5] alpha, [6] beta, [7] number of sampling rounds             */
/* ------------------------------------------------------------------ */
void orc_theta_params(uint32_t n, uint32_t k, double eps, double ell, double out[8])
{
    const double nd = (double)n;
    const double ln_n = log(nd);
    const double ell_p = ell * (1.0 + log(2.0) / ln_n);
    const double eps_p = sqrt(2.0) * eps;
    double lnC = 0.0;
    for (uint32_t i = 1; i <= k; i++) lnC += log((double)(n - k + i)) - log((double)i);
    const double lam_p = (2.0 + 2.0 * eps_p / 3.0) * (lnC + ell_p * ln_n + log(log2(nd))) * nd
                         / (eps_p * eps_p);
    const double one_m_inv_e = 1.0 - 1.0 / ORC_E;
    const double alpha = sqrt(ell_p * ln_n + log(2.0));
    const double beta = sqrt(one_m_inv_e * (lnC + ell_p * ln_n + log(2.0)));
    const double t = one_m_inv_e * alpha + beta;
    const double lam_s = 2.0 * nd * t * t / (eps * eps);
    uint32_t lg = 0;
    while (lg < 32 && ((uint64_t)1 << lg) < (uint64_t)n) lg++;
    out[0] = ell_p;
    out[1] = eps_p;
    out[2] = lnC;
    out[3] = lam_p;
    out[4] = lam_s;
    out[5] = alpha;
    out[6] = beta;
    out[7] = (double)(lg >= 1 ? lg - 1 : 0);
}

/* ------------------------------------------------------------------ */
/* Context: graph, thresholds, RRR-set stream, counters.               */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t n;
    uint64_t m;
    int model;
    uint64_t* row;   /* n+1: in-edge offsets of G^T */
    uint32_t* src;   /* m: tail of each in-edge */
    uint32_t* thr;   /* m: IC threshold, or LT cumulative threshold */
    int have_stream;
    uint64_t seed;
    uint64_t nsets, cap_sets;
    uint64_t* off;   /* nsets+1 */
    uint64_t cap_mem;
    uint32_t* mem;   /* members, BFS order inside a set */
    uint32_t* cnt;   /* n: occurrences over all sets (fused count, Alg. 3) */
    uint8_t* visited;
    uint32_t* queue;
} orc_ctx;

typedef struct {
    uint32_t rounds;
    uint32_t stopped_early;   /* 1 if the LB test fired */
    uint64_t theta_i[64];
    uint64_t covered_i[64];
    uint64_t sets_i[64];
    double lb;
    uint64_t theta;
    uint64_t num_sets;
    uint64_t covered;
    double lambda_prime;
    double lambda_star;
} orc_stats;

void orc_destroy(orc_ctx* c)
{
    if (!c) return;
    free(c->row); free(c->src); free(c->thr); free(c->off); free(c->mem);
    free(c->cnt); free(c->visited); free(c->queue); free(c);
}

orc_ctx* orc_create(uint32_t n, uint64_t m, const uint64_t* row, const uint32_t* src,
                    const float* weight, int model, int* err)
{
    *err = ORC_EINVAL;
    if (n < 2 || (model != ORC_IC && model != ORC_LT) || row == NULL) return NULL;
    if (m > 0xFFFFFFFFull || (m > 0 && (src == NULL || weight == NULL))) return NULL;
    if (row[0] != 0 || row[n] != m) return NULL;
    for (uint32_t v = 0; v < n; v++) if (row[v + 1] < row[v]) return NULL;
    for (uint64_t e = 0; e < m; e++) {
        if (src[e] >= n) return NULL;
        float w = weight[e];
        if (!(w >= 0.0f && w <= 1.0f)) return NULL;
    }
    orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    *err = ORC_ENOMEM;
    if (!c) return NULL;
    c->n = n; c->m = m; c->model = model;
    c->row = (uint64_t*)malloc(((uint64_t)n + 1) * sizeof(uint64_t));
    c->src = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    c->thr = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    c->cnt = (uint32_t*)calloc(n, sizeof(uint32_t));
    c->visited = (uint8_t*)calloc(n, 1);
    c->queue = (uint32_t*)malloc((uint64_t)n * sizeof(uint32_t));
    c->cap_sets = 1024;
    c->off = (uint64_t*)malloc((c->cap_sets + 1) * sizeof(uint64_t));
    c->cap_mem = 1 << 16;
    c->mem = (uint32_t*)malloc(c->cap_mem * sizeof(uint32_t));
    if (!c->row || !c->src || !c->thr || !c->cnt || !c->visited || !c->queue || !c->off || !c->mem) {
        orc_destroy(c);
        return NULL;
    }
    memcpy(c->row, row, ((uint64_t)n + 1) * sizeof(uint64_t));
    if (m) memcpy(c->src, src, m * sizeof(uint32_t));
    c->off[0] = 0;
    if (model == ORC_IC) {
        for (uint64_t e = 0; e < m; e++) c->thr[e] = orc_ic_threshold(weight[e]);
    } else {
        for (uint32_t v = 0; v < n; v++) {
            double cw = 0.0;
            for (uint64_t e = row[v]; e < row[v + 1]; e++) {
                cw = cw + (double)weight[e];
                double t = ceil(cw * 16777216.0);
                c->thr[e] = t > 16777216.0 ? 16777216u : (uint32_t)t;
            }
            /* Sec. II-A: sum of a vertex's in-weights must not exceed 1. */
            if (cw > 1.0 + 1e-6) { *err = ORC_EINVAL; orc_destroy(c); return NULL; }
        }
    }
    *err = ORC_OK;
    return c;
}

static int reserve_mem(orc_ctx* c, uint64_t need)
{
    if (need <= c->cap_mem) return ORC_OK;
    uint64_t cap = c->cap_mem;
    while (cap < need) cap *= 2;
    uint32_t* p = (uint32_t*)realloc(c->mem, cap * sizeof(uint32_t));
    if (!p) return ORC_ENOMEM;
    c->mem = p;
    c->cap_mem = cap;
    return ORC_OK;
}

static int reserve_sets(orc_ctx* c, uint64_t need)
{
    if (need <= c->cap_sets) return ORC_OK;
    uint64_t cap = c->cap_sets;
    while (cap < need) cap *= 2;
    uint64_t* p = (uint64_t*)realloc(c->off, (cap + 1) * sizeof(uint64_t));
    if (!p) return ORC_ENOMEM;
    c->off = p;
    c->cap_sets = cap;
    return ORC_OK;
}

/*
 * One RRR set, written to `out` (BFS order, root first); returns its size.
 * `out` must hold n entries.  visited[] is all-zero on entry and on exit.
 */
static uint32_t sample_set(orc_ctx* c, uint64_t seed, uint64_t s, uint32_t* out)
{
    const uint32_t root = orc_root(seed, s, c->n);
    uint32_t len = 0;
    if (c->model == ORC_IC) {
        /* Alg. 3: BFS over in-neighbours; an unvisited in-neighbour u of the
           dequeued vertex joins when its edge's coin comes up live. */
        uint32_t head = 0;
        out[len++] = root;
        c->visited[root] = 1;
        while (head < len) {
            uint32_t v = out[head++];
            for (uint64_t e = c->row[v]; e < c->row[v + 1]; e++) {
                uint32_t u = c->src[e];
                if (!c->visited[u] && orc_ic_live(seed, s, (uint32_t)e, c->thr[e])) {
                    c->visited[u] = 1;
                    out[len++] = u;
                }
            }
        }
    } else {
        /* Reverse LT walk: each vertex keeps at most one live in-edge
           (Sec. II-A live-edge reading of LT); follow it from the root. */
        uint32_t v = root;
        out[len++] = root;
        c->visited[root] = 1;
        for (;;) {
            uint32_t r = orc_lt_draw(seed, s, v);
            uint64_t pick = c->row[v + 1];
            for (uint64_t e = c->row[v]; e < c->row[v + 1]; e++) {
                if (r < c->thr[e]) { pick = e; break; }
            }
            if (pick == c->row[v + 1]) break;   /* no in-edge chosen */
            uint32_t u = c->src[pick];
            if (c->visited[u]) break;           /* walk closed a cycle */
            c->visited[u] = 1;
            out[len++] = u;
            v = u;
        }
    }
    for (uint32_t i = 0; i < len; i++) c->visited[out[i]] = 0;
    return len;
}

/* Generate_RRRsets: extend the stream to theta sets (ids nsets..theta-1),
   counting each member as the set is produced (Alg. 3, fused count). */
int orc_sample(orc_ctx* c, uint64_t theta, uint64_t seed)
{
    if (theta >= 0xFFFFFFFFull) return ORC_EINVAL;
    if (c->have_stream && c->seed != seed) return ORC_EINVAL;
    c->have_stream = 1;
    c->seed = seed;
    if (theta <= c->nsets) return ORC_OK;
    if (reserve_sets(c, theta) != ORC_OK) return ORC_ENOMEM;
    for (uint64_t s = c->nsets; s < theta; s++) {
        uint64_t at = c->off[s];
        if (reserve_mem(c, at + c->n) != ORC_OK) return ORC_ENOMEM;
        uint32_t len = sample_set(c, seed, s, c->mem + at);
        for (uint32_t i = 0; i < len; i++) c->cnt[c->mem[at + i]] += 1;
        c->off[s + 1] = at + len;
        c->nsets = s + 1;
    }
    return ORC_OK;
}

int orc_reset(orc_ctx* c)
{
    c->nsets = 0;
    c->off[0] = 0;
    c->have_stream = 0;
    memset(c->cnt, 0, (uint64_t)c->n * sizeof(uint32_t));
    return ORC_OK;
}

/*
 * Find_Most_Influential_Set (Alg. 2) over an explicit set system
 * (nsets sets, members mem[off[s]..off[s+1])).  Writes k picks in order and
 * the number of sets covered.
 */
int orc_select_sets(uint32_t n, uint64_t nsets, const uint64_t* off, const uint32_t* mem,
                    uint32_t k, uint32_t* seeds, uint64_t* covered_out)
{
    if (k == 0 || k > n) return ORC_EINVAL;
    uint32_t* counter = (uint32_t*)calloc(n, sizeof(uint32_t));
    uint8_t* removed = (uint8_t*)calloc(nsets ? nsets : 1, 1);
    uint8_t* picked = (uint8_t*)calloc(n, 1);
    if (!counter || !removed || !picked) { free(counter); free(removed); free(picked); return ORC_ENOMEM; }
    /* counter[v] = number of sets containing v */
    for (uint64_t s = 0; s < nsets; s++)
        for (uint64_t i = off[s]; i < off[s + 1]; i++) counter[mem[i]] += 1;
    uint64_t covered = 0;
    for (uint32_t j = 0; j < k; j++) {
        /* PARALLEL_REDUCTION written as a plain scan: the largest counter
           among vertices not yet picked, lowest id on ties. */
        uint32_t best = 0xFFFFFFFFu, best_cnt = 0;
        for (uint32_t v = 0; v < n; v++) {
            if (picked[v]) continue;
            if (best == 0xFFFFFFFFu || counter[v] > best_cnt) { best = v; best_cnt = counter[v]; }
        }
        picked[best] = 1;
        seeds[j] = best;
        /* every remaining set holding the pick: decrement its members, drop it */
        for (uint64_t s = 0; s < nsets; s++) {
            if (removed[s]) continue;
            int has = 0;
            for (uint64_t i = off[s]; i < off[s + 1]; i++)
                if (mem[i] == best) { has = 1; break; }
            if (!has) continue;
            for (uint64_t i = off[s]; i < off[s + 1]; i++) counter[mem[i]] -= 1;
            removed[s] = 1;
            covered += 1;
        }
    }
    *covered_out = covered;
    free(counter); free(removed); free(picked);
    return ORC_OK;
}

int orc_select(orc_ctx* c, uint32_t k, uint32_t* seeds, uint64_t* covered)
{
    return orc_select_sets(c->n, c->nsets, c->off, c->mem, k, seeds, covered);
}

/* Key of the fresh final stream (Chen 2018): the estimation phase's sets are
 * dropped and theta new ones drawn under a second key, seed xor this odd
 * constant (2^64 / golden ratio), so they are independent of the sets that
 * fixed theta.  The paper reuses the sets (Alg. 1); the constant is a reading. */
#define ORC_FRESH_KEY 0x9E3779B97F4A7C15ull
#define ORC_FRESH_FINAL 1u

/* Alg. 1 with Tang et al.'s Theta_Estimation / OPT_Lower_Bound / Set_Theta;
 * flags & ORC_FRESH_FINAL: the final selection runs on a fresh stream of
 * exactly theta sets. */
int orc_run_ex(orc_ctx* c, uint32_t k, double eps, double ell, uint64_t seed, uint32_t flags,
               uint32_t* seeds, orc_stats* st)
{
    if (k == 0 || k > c->n || !(eps > 0.0 && eps < 1.0) || !(ell > 0.0)) return ORC_EINVAL;
    orc_reset(c);
    double prm[8];
    orc_theta_params(c->n, k, eps, ell, prm);
    const double eps_p = prm[1], lam_p = prm[3], lam_s = prm[4];
    const uint32_t rounds = (uint32_t)prm[7];
    memset(st, 0, sizeof(*st));
    st->lambda_prime = lam_p;
    st->lambda_star = lam_s;
    double lb = 1.0;
    int rc;
    for (uint32_t i = 1; i <= rounds; i++) {
        const double x = ldexp((double)c->n, -(int)i);
        const double th = ceil(lam_p / x);
        if (th >= 4294967295.0) return ORC_EINVAL;
        const uint64_t theta_i = (uint64_t)th;
        if ((rc = orc_sample(c, theta_i, seed)) != ORC_OK) return rc;
        uint64_t cov = 0;
        if ((rc = orc_select(c, k, seeds, &cov)) != ORC_OK) return rc;
        const double nF = (double)c->n * (double)cov / (double)c->nsets;
        if (i - 1 < 64) {
            st->theta_i[i - 1] = theta_i;
            st->covered_i[i - 1] = cov;
            st->sets_i[i - 1] = c->nsets;
        }
        st->rounds = i;
        if (nF >= (1.0 + eps_p) * x) {
            lb = nF / (1.0 + eps_p);
            st->stopped_early = 1;
            break;
        }
    }
    const double tf = ceil(lam_s / lb);
    if (tf >= 4294967295.0) return ORC_EINVAL;
    const uint64_t theta = (uint64_t)tf;
    st->lb = lb;
    st->theta = theta;
    uint64_t target = theta > c->nsets ? theta : c->nsets;
    if (flags & ORC_FRESH_FINAL) {
        orc_reset(c);
        seed ^= ORC_FRESH_KEY;
        target = theta;
    }
    if ((rc = orc_sample(c, target, seed)) != ORC_OK) return rc;
    uint64_t cov = 0;
    if ((rc = orc_select(c, k, seeds, &cov)) != ORC_OK) return rc;
    st->num_sets = c->nsets;
    st->covered = cov;
    return ORC_OK;
}

int orc_run(orc_ctx* c, uint32_t k, double eps, double ell, uint64_t seed, uint32_t* seeds, orc_stats* st)
{
    return orc_run_ex(c, k, eps, ell, seed, 0u, seeds, st);
}

/* ------------------------------------------------------------------ */
/* OPIM-style early stop (Sec. VI cites OPIM: Tang, Tang, Xiao, Yuan,   */
/* SIGMOD 2018, whose OPIM-C procedure this follows).  Two independent  */
/* RR-set collections of equal size, R1 (key seed) and R2 (key seed xor */
/* ORC_OPIM_KEY), double each round; the greedy picks S on R1; R1's     */
/* coverage gives an upper confidence bound on OPT and R2's coverage of */
/* S a lower confidence bound on the spread of S; sampling stops once   */
/* their ratio reaches 1 - 1/e - eps (or at the last round).            */
/* Readings where the paper (which only cites OPIM) is silent:          */
/*   - the failure probability is delta = n^-ell (IMM's ell);           */
/*   - theta_0 is rounded up; round i holds ceil(theta_0) * 2^(i-1)     */
/*     sets per collection; i_max = max(1, ceil(log2(theta_max /       */
/*     theta_0)));                                                      */
/*   - the bound on the optimum's R1 coverage is the greedy's coverage  */
/*     over 1 - (1 - 1/k)^k (OPIM-C's tighter marginal-gain bound is    */
/*     not used);                                                       */
/*   - R2's key is seed xor ORC_OPIM_KEY (an odd constant).             */
/* ------------------------------------------------------------------ */
#define ORC_OPIM_KEY 0xD1B54A32D192ED03ull

/* out: [0] delta, [1] ln C(n,k), [2] theta_max, [3] theta_0, [4] i_max,
 *      [5] a1, [6] a2 */
void orc_opim_params(uint32_t n, uint32_t k, double eps, double ell, double out[7])
{
    const double nd = (double)n;
    const double ln_n = log(nd);
    const double delta = exp(-ell * ln_n);
    double lnC = 0.0;
    for (uint32_t i = 1; i <= k; i++) lnC += log((double)(n - k + i)) - log((double)i);
    const double g = 1.0 - 1.0 / ORC_E;
    const double l6 = log(6.0 / delta);
    const double t = g * sqrt(l6) + sqrt(g * (lnC + l6));
    const double theta_max = 2.0 * nd * t * t / (eps * eps * (double)k);
    const double theta_0 = theta_max * eps * eps * (double)k / nd;
    double im = ceil(log2(theta_max / theta_0));
    if (im < 1.0) im = 1.0;
    const double a2 = log(3.0 * im / delta);
    out[0] = delta;
    out[1] = lnC;
    out[2] = theta_max;
    out[3] = theta_0;
    out[4] = im;
    out[5] = a2 + lnC;
    out[6] = a2;
}

/* Confidence bounds of one round: cov1 = R1 coverage of the greedy's set,
 * cov2 = its R2 coverage, theta = sets per collection.
 * out: [0] upper bound on OPT, [1] lower bound on the set's spread. */
void orc_opim_bounds(uint32_t n, uint32_t k, double a1, double a2, uint64_t theta, uint64_t cov1, uint64_t cov2,
                     double out[2])
{
    const double nd = (double)n, th = (double)theta;
    const double ratio = 1.0 - pow(1.0 - 1.0 / (double)k, (double)k);
    const double lam_u = (double)cov1 / ratio;
    const double up = sqrt(lam_u + a1 / 2.0) + sqrt(a1 / 2.0);
    const double lo = sqrt((double)cov2 + 2.0 * a2 / 9.0) - sqrt(a2 / 2.0);
    out[0] = up * up * nd / th;
    out[1] = (lo * lo - a2 / 18.0) * nd / th;
}

typedef struct {
    uint32_t rounds;
    uint32_t stopped_early;   /* 1 if the ratio test fired before the last round */
    uint32_t i_max;
    uint64_t sets_i[64];      /* sets per collection in round i */
    uint64_t cov1_i[64];      /* R1 coverage of the greedy's set */
    uint64_t cov2_i[64];      /* R2 coverage of the same set */
    double upper_i[64];
    double lower_i[64];
    double theta_max;
    double theta_0;
    double alpha;             /* lower / upper of the last round */
} orc_opim_stats;

int orc_opim_run(orc_ctx* c, uint32_t k, double eps, double ell, uint64_t seed, uint32_t* seeds,
                 orc_opim_stats* st)
{
    if (k == 0 || k > c->n || !(eps > 0.0 && eps < 1.0) || !(ell > 0.0)) return ORC_EINVAL;
    double prm[7];
    orc_opim_params(c->n, k, eps, ell, prm);
    const double theta_max = prm[2], theta_0 = prm[3], a1 = prm[5], a2 = prm[6];
    const uint32_t i_max = (uint32_t)prm[4];
    const double t0 = ceil(theta_0);
    if (t0 * ldexp(1.0, (int)i_max - 1) >= 4294967295.0) return ORC_EINVAL;
    /* R2: a second context on the same graph (thresholds copied) */
    orc_ctx* r2 = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    if (!r2) return ORC_ENOMEM;
    r2->n = c->n; r2->m = c->m; r2->model = c->model;
    r2->row = (uint64_t*)malloc(((uint64_t)c->n + 1) * sizeof(uint64_t));
    r2->src = (uint32_t*)malloc((c->m ? c->m : 1) * sizeof(uint32_t));
    r2->thr = (uint32_t*)malloc((c->m ? c->m : 1) * sizeof(uint32_t));
    r2->cnt = (uint32_t*)calloc(c->n, sizeof(uint32_t));
    r2->visited = (uint8_t*)calloc(c->n, 1);
    r2->queue = (uint32_t*)malloc((uint64_t)c->n * sizeof(uint32_t));
    r2->cap_sets = 1024;
    r2->off = (uint64_t*)malloc((r2->cap_sets + 1) * sizeof(uint64_t));
    r2->cap_mem = 1 << 16;
    r2->mem = (uint32_t*)malloc(r2->cap_mem * sizeof(uint32_t));
    if (!r2->row || !r2->src || !r2->thr || !r2->cnt || !r2->visited || !r2->queue || !r2->off || !r2->mem) {
        orc_destroy(r2);
        return ORC_ENOMEM;
    }
    memcpy(r2->row, c->row, ((uint64_t)c->n + 1) * sizeof(uint64_t));
    if (c->m) memcpy(r2->src, c->src, c->m * sizeof(uint32_t));
    if (c->m) memcpy(r2->thr, c->thr, c->m * sizeof(uint32_t));
    r2->off[0] = 0;
    orc_reset(c);
    memset(st, 0, sizeof(*st));
    st->i_max = i_max;
    st->theta_max = theta_max;
    st->theta_0 = theta_0;
    uint8_t* in_s = (uint8_t*)calloc(c->n, 1);
    if (!in_s) { orc_destroy(r2); return ORC_ENOMEM; }
    int rc = ORC_OK;
    for (uint32_t i = 1; i <= i_max; i++) {
        const uint64_t theta = (uint64_t)(t0 * ldexp(1.0, (int)i - 1));
        if ((rc = orc_sample(c, theta, seed)) != ORC_OK) break;
        if ((rc = orc_sample(r2, theta, seed ^ ORC_OPIM_KEY)) != ORC_OK) break;
        uint64_t cov1 = 0;
        if ((rc = orc_select(c, k, seeds, &cov1)) != ORC_OK) break;
        /* R2 coverage of the greedy's set: sets holding any of its members */
        for (uint32_t j = 0; j < k; j++) in_s[seeds[j]] = 1;
        uint64_t cov2 = 0;
        for (uint64_t s = 0; s < r2->nsets; s++) {
            for (uint64_t e = r2->off[s]; e < r2->off[s + 1]; e++)
                if (in_s[r2->mem[e]]) { cov2++; break; }
        }
        for (uint32_t j = 0; j < k; j++) in_s[seeds[j]] = 0;
        double b[2];
        orc_opim_bounds(c->n, k, a1, a2, theta, cov1, cov2, b);
        const double alpha = b[1] / b[0];
        if (i - 1 < 64) {
            st->sets_i[i - 1] = theta;
            st->cov1_i[i - 1] = cov1;
            st->cov2_i[i - 1] = cov2;
            st->upper_i[i - 1] = b[0];
            st->lower_i[i - 1] = b[1];
        }
        st->rounds = i;
        st->alpha = alpha;
        if (alpha >= 1.0 - 1.0 / ORC_E - eps) {
            st->stopped_early = i < i_max ? 1u : 0u;
            break;
        }
    }
    free(in_s);
    orc_destroy(r2);
    return rc;
}

/* ---- accessors for tests ---- */
uint64_t orc_num_sets(const orc_ctx* c) { return c->nsets; }
uint64_t orc_num_members(const orc_ctx* c) { return c->off[c->nsets]; }

static int cmp_u32(const void* a, const void* b)
{
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/* Members of stored set `id`, sorted ascending. */
int orc_get_set(const orc_ctx* c, uint64_t id, uint32_t* buf, uint32_t cap, uint32_t* len)
{
    if (id >= c->nsets) return ORC_EINVAL;
    uint64_t l = c->off[id + 1] - c->off[id];
    *len = (uint32_t)l;
    if (l > cap) return ORC_EINVAL;
    memcpy(buf, c->mem + c->off[id], l * sizeof(uint32_t));
    qsort(buf, l, sizeof(uint32_t), cmp_u32);
    return ORC_OK;
}

/* One set sampled on its own (not stored), sorted ascending; buf holds n. */
int orc_sample_one(orc_ctx* c, uint64_t seed, uint64_t id, uint32_t* buf, uint32_t* len)
{
    uint32_t l = sample_set(c, seed, id, buf);
    qsort(buf, l, sizeof(uint32_t), cmp_u32);
    *len = l;
    return ORC_OK;
}

void orc_get_counts(const orc_ctx* c, uint32_t* out)
{
    memcpy(out, c->cnt, (uint64_t)c->n * sizeof(uint32_t));
}

/* Whole stream: off[nsets+1] and members (BFS order inside each set). */
void orc_get_arena(const orc_ctx* c, uint64_t* off, uint32_t* mem)
{
    memcpy(off, c->off, (c->nsets + 1) * sizeof(uint64_t));
    memcpy(mem, c->mem, c->off[c->nsets] * sizeof(uint32_t));
}

void orc_get_thresholds(const orc_ctx* c, uint32_t* out)
{
    memcpy(out, c->thr, c->m * sizeof(uint32_t));
}
