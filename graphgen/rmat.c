/*
 * Seeded synthetic input generator: R-MAT directed graphs in transposed CSR,
 * plus fp32 edge weights.  Both the oracle tests and the CUDA path read their
 * inputs from here; nothing in this file computes any step of IMM itself
 * (no thresholds, no coins, no RRR sets, no counts).
 *
 * R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): each edge draw descends
 * `scale` levels of the adjacency matrix, picking one quadrant per level with
 * probabilities (a, b, c, d).  Quadrant a = (row bit 0, col bit 0), b = (0, 1),
 * c = (1, 0), d = (1, 1); the row is the edge's tail u, the column its head v.
 * Self-loops and draws outside [0, n) are skipped, duplicate (u, v) pairs are
 * merged, and draws continue in index order until exactly m distinct edges
 * exist.  The edges are then grouped by head v (CSR of the transposed graph),
 * tails ascending within each head.
 *
 * Random words come from a stateless counter hash: the splitmix64 output
 * function (Steele, Lea, Flood, OOPSLA 2014) applied to a Weyl sequence keyed
 * by (seed, draw index, word index).  Plain C, fixed-width integers only, so
 * x86-64 and aarch64 produce the same graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t gg_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Word w of draw i under `seed`. */
uint64_t gg_word(uint64_t seed, uint64_t i, uint32_t w)
{
    uint64_t x = gg_mix64(seed * 0x9E3779B97F4A7C15ULL + 0x632BE59BD9B4E019ULL);
    x += (i * 64u + (uint64_t)w + 1u) * 0xD1B54A32D192ED03ULL;
    return gg_mix64(x);
}

static uint32_t ceil_log2_u32(uint32_t n)
{
    uint32_t s = 0;
    while (s < 32 && ((uint64_t)1 << s) < (uint64_t)n) s++;
    return s;
}

static int cmp_u32(const void* a, const void* b)
{
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Fills row[n+1] (in-edge offsets per head v) and src[m] (tails, ascending
 * within a head).  a, b, c are quadrant probabilities (d = 1 - a - b - c).
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure,
 * -3 if m distinct edges could not be drawn within 64*m + 2^20 draws.
 */
int gg_rmat(uint32_t n, uint64_t m, double a, double b, double c, uint64_t seed,
            uint64_t* row, uint32_t* src)
{
    if (n < 2 || row == NULL || (m > 0 && src == NULL)) return -1;
    if (m > (uint64_t)n * (uint64_t)(n - 1)) return -1;
    if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return -1;
    const uint32_t scale = ceil_log2_u32(n);
    /* 24-bit integer cut points for the quadrant pick. */
    const uint32_t ta = (uint32_t)(a * 16777216.0 + 0.5);
    const uint32_t tb = (uint32_t)((a + b) * 16777216.0 + 0.5);
    const uint32_t tc = (uint32_t)((a + b + c) * 16777216.0 + 0.5);

    uint64_t cap = 1;
    while (cap < 2 * m + 16) cap <<= 1;
    uint64_t* table = (uint64_t*)malloc(cap * sizeof(uint64_t));
    uint64_t* keys = (uint64_t*)malloc((m ? m : 1) * sizeof(uint64_t));
    if (!table || !keys) { free(table); free(keys); return -2; }
    const uint64_t EMPTY = ~(uint64_t)0;
    memset(table, 0xFF, cap * sizeof(uint64_t));

    uint64_t have = 0, draw = 0;
    const uint64_t max_draws = 64 * m + (1u << 20);
    while (have < m) {
        if (draw >= max_draws) { free(table); free(keys); return -3; }
        uint32_t u = 0, v = 0;
        uint64_t word = 0;
        for (uint32_t lvl = 0; lvl < scale; lvl++) {
            if ((lvl & 1) == 0) word = gg_word(seed, draw, lvl >> 1);
            uint32_t r = (uint32_t)((lvl & 1) ? (word >> 32) : word) & 0xFFFFFFu;
            uint32_t bit = scale - 1 - lvl;
            if (r < ta) {
            } else if (r < tb) {
                v |= 1u << bit;
            } else if (r < tc) {
                u |= 1u << bit;
            } else {
                u |= 1u << bit;
                v |= 1u << bit;
            }
        }
        draw++;
        if (u >= n || v >= n || u == v) continue;
        uint64_t key = ((uint64_t)u << 32) | v;
        uint64_t h = gg_mix64(key) & (cap - 1);
        int dup = 0;
        while (table[h] != EMPTY) {
            if (table[h] == key) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        table[h] = key;
        keys[have++] = key;
    }
    free(table);

    /* Counting sort by head v, then tails ascending inside each head. */
    memset(row, 0, ((uint64_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < m; i++) row[(uint32_t)keys[i] + 1]++;
    for (uint32_t v = 0; v < n; v++) row[v + 1] += row[v];
    uint64_t* cur = (uint64_t*)malloc((uint64_t)n * sizeof(uint64_t));
    if (!cur) { free(keys); return -2; }
    memcpy(cur, row, (uint64_t)n * sizeof(uint64_t));
    for (uint64_t i = 0; i < m; i++) {
        uint32_t v = (uint32_t)keys[i];
        src[cur[v]++] = (uint32_t)(keys[i] >> 32);
    }
    free(cur);
    free(keys);
    for (uint32_t v = 0; v < n; v++) {
        uint64_t lo = row[v], hi = row[v + 1];
        if (hi - lo > 1) qsort(src + lo, hi - lo, sizeof(uint32_t), cmp_u32);
    }
    return 0;
}

/* Weighted cascade / uniform LT weights: w_e = 1 / indeg(head), in fp32. */
void gg_weights_inv_indeg(uint32_t n, const uint64_t* row, float* w)
{
    for (uint32_t v = 0; v < n; v++) {
        uint64_t lo = row[v], hi = row[v + 1];
        if (hi == lo) continue;
        float p = 1.0f / (float)(hi - lo);
        for (uint64_t e = lo; e < hi; e++) w[e] = p;
    }
}

/* w_e = (u24 * 2^-24) * pmax in fp32, u24 drawn from (seed, e). */
void gg_weights_uniform(uint64_t m, float pmax, uint64_t seed, float* w)
{
    for (uint64_t e = 0; e < m; e++) {
        uint32_t r = (uint32_t)(gg_word(seed ^ 0xA5A5A5A55A5A5A5AULL, e, 0) >> 40);
        float u = (float)r * (1.0f / 16777216.0f);
        w[e] = u * pmax;
    }
}

/* n uniform doubles in [0, 1) with 53 random bits each, drawn from (seed, i). */
void gg_uniform_f64(uint64_t count, uint64_t seed, uint64_t first, double* out)
{
    for (uint64_t i = 0; i < count; i++) {
        uint64_t x = gg_word(seed, first + i, 63) >> 11;
        out[i] = (double)x * (1.0 / 9007199254740992.0);
    }
}
