/* Barabasi-Albert preferential-attachment edge list (input generator only).
 *
 * Seed: a clique on k+1 nodes.  Each later node v joins k distinct earlier nodes, each
 * drawn uniformly from the list of all edge endpoints so far (so with probability
 * proportional to degree); a draw that repeats a target already chosen for v is redrawn.
 * Random numbers come from splitmix64 (Steele, Lea and Flood, 2014), so the output is the
 * same on every machine for a given seed.
 */
#include <stdint.h>
#include <stdlib.h>

static uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Returns the number of edges written (each undirected edge once) or -1 on error. */
int64_t ba_edges(int64_t n, int32_t k, uint64_t seed, int32_t *src, int32_t *dst) {
    if (k < 1 || n <= k + 1) return -1;
    int64_t ne_total = (int64_t)(k + 1) * k / 2 + (n - k - 1) * (int64_t)k;
    int32_t *ends = (int32_t *)malloc(sizeof(int32_t) * 2 * ne_total);
    int32_t *pick = (int32_t *)malloc(sizeof(int32_t) * k);
    if (!ends || !pick) { free(ends); free(pick); return -1; }
    uint64_t s = seed;
    int64_t ne = 0, nends = 0;
    for (int32_t i = 0; i <= k; ++i)
        for (int32_t j = i + 1; j <= k; ++j) {
            src[ne] = i; dst[ne] = j; ++ne;
            ends[nends++] = i; ends[nends++] = j;
        }
    for (int64_t v = k + 1; v < n; ++v) {
        int32_t got = 0;
        while (got < k) {
            int32_t t = ends[splitmix64(&s) % (uint64_t)nends];
            int dup = 0;
            for (int32_t q = 0; q < got; ++q) if (pick[q] == t) { dup = 1; break; }
            if (!dup) pick[got++] = t;
        }
        for (int32_t q = 0; q < k; ++q) {
            src[ne] = (int32_t)v; dst[ne] = pick[q]; ++ne;
            ends[nends++] = (int32_t)v; ends[nends++] = pick[q];
        }
    }
    free(ends); free(pick);
    return ne;
}
