/*
 * Seeded synthetic protein families: the input generator shared by the tests,
 * the CPU oracle checks and the benchmark. It produces inputs only and holds
 * none of the method's arithmetic (no k-mer counting, ranking, partitioning or
 * alignment).
 *
 * The paper evaluates on rose-generated families (N = 5000/10000/20000,
 * L ~ 300) and on 2000 genome proteins of mean length 316 (Section 4). Neither
 * dataset is available, so families are evolved here from a random root along
 * a random binary (Yule) tree with substitutions and geometric indels.
 *
 * PRNG: xoshiro256** (Blackman & Vigna, 2018), state seeded by splitmix64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t* x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t next_u64(rng_t* r) {
    uint64_t* s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return res;
}
static void rng_seed(rng_t* r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
/* uniform double in [0, 1) with 53 random bits */
static double uni(rng_t* r) { return (double)(next_u64(r) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, n), n >= 1 (multiply-high; bias < 2^-32 for n < 2^32) */
static uint32_t below(rng_t* r, uint32_t n) {
    return (uint32_t)(((unsigned __int128)next_u64(r) * n) >> 64);
}
static int geometric_ge1(rng_t* r, double mean) {
    /* P(g) = (1-q)^(g-1) q with q = 1/mean, support g >= 1 */
    double q = 1.0 / mean;
    int g = 1;
    while (uni(r) >= q && g < 1000000) g++;
    return g;
}
static double std_normal(rng_t* r) {
    /* Box-Muller; 1 - u keeps the log argument in (0, 1] */
    double u1 = 1.0 - uni(r), u2 = uni(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* length distributions */
enum { LEN_UNIFORM = 0, LEN_NORMAL = 1, LEN_LOGNORMAL = 2 };

static int32_t draw_length(rng_t* r, int32_t dist, double p1, double p2, int32_t lo, int32_t hi) {
    double v;
    if (dist == LEN_UNIFORM) return lo + (int32_t)below(r, (uint32_t)(hi - lo + 1));
    if (dist == LEN_NORMAL) v = p1 + p2 * std_normal(r);
    else v = p1 * exp(p2 * std_normal(r));          /* median p1, log-sd p2 */
    long iv = lround(v);
    if (iv < lo) iv = lo;
    if (iv > hi) iv = hi;
    return (int32_t)iv;
}

typedef struct { uint8_t* a; int32_t len, cap; } seq_t;

static void seq_reserve(seq_t* s, int32_t cap) {
    if (cap <= s->cap) return;
    int32_t nc = s->cap ? s->cap : 64;
    while (nc < cap) nc *= 2;
    s->a = (uint8_t*)realloc(s->a, (size_t)nc);
    s->cap = nc;
}

/* One edge of the tree: per-site substitution with probability qs (to a uniform
 * different letter), then per-site indel events with probability qi, half
 * insertions after the site and half deletions starting at it, each of
 * geometric length (mean indel_mean, support >= 1). */
static void evolve_edge(rng_t* r, const seq_t* par, seq_t* out, double qs, double qi,
                        double indel_mean, int32_t A) {
    out->len = 0;
    seq_reserve(out, par->len + 16);
    int32_t i = 0;
    while (i < par->len) {
        uint8_t c = par->a[i];
        if (uni(r) < qs) c = (uint8_t)((c + 1 + below(r, (uint32_t)(A - 1))) % A);
        if (uni(r) < qi) {
            int g = geometric_ge1(r, indel_mean);
            if (uni(r) < 0.5) {                 /* insertion after this site */
                seq_reserve(out, out->len + 1 + g);
                out->a[out->len++] = c;
                for (int t = 0; t < g; t++) out->a[out->len++] = (uint8_t)below(r, (uint32_t)A);
                i += 1;
            } else {                            /* deletion of g sites from here */
                i += g;
            }
            continue;
        }
        seq_reserve(out, out->len + 1);
        out->a[out->len++] = c;
        i += 1;
    }
}

/*
 * Generate sum(family_sizes) sequences. Each family: random root of length
 * root_len, a Yule tree with family_sizes[f] leaves, evolution along every edge
 * with per-edge rates chosen so that the rates compound to sub_total and
 * indel_total over the mean root-to-leaf depth, then each leaf is truncated or
 * extended with uniform residues to a length drawn from the length
 * distribution. The final set is shuffled by a seeded permutation.
 *
 * residues_out: capacity res_capacity bytes; offsets_out: n+1 entries.
 * Returns the total residue count, or -1 if res_capacity is too small.
 */
int64_t synth_families(uint64_t seed, int32_t n_families, const int32_t* family_sizes,
                       int32_t root_len, int32_t len_dist, double p1, double p2,
                       int32_t lo, int32_t hi, double sub_total, double indel_total,
                       double indel_mean, int32_t alphabet,
                       uint8_t* residues_out, int64_t res_capacity, int64_t* offsets_out) {
    rng_t rng; rng_seed(&rng, seed);
    int64_t n = 0;
    for (int f = 0; f < n_families; f++) n += family_sizes[f];
    seq_t* leaves = (seq_t*)calloc((size_t)(n ? n : 1), sizeof(seq_t));
    int64_t leaf_base = 0;
    for (int f = 0; f < n_families; f++) {
        int32_t m = family_sizes[f];
        if (m <= 0) continue;
        /* Yule tree: nodes 0..2m-2; parent[], depth[]; leaves are split uniformly */
        int32_t nn = 2 * m - 1;
        int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * nn);
        int32_t* depth = (int32_t*)malloc(sizeof(int32_t) * nn);
        int32_t* leafs = (int32_t*)malloc(sizeof(int32_t) * m);
        int32_t nl = 1, used = 1;
        parent[0] = -1; depth[0] = 0; leafs[0] = 0;
        while (nl < m) {
            int32_t pick = (int32_t)below(&rng, (uint32_t)nl);
            int32_t node = leafs[pick];
            int32_t c1 = used++, c2 = used++;
            parent[c1] = node; parent[c2] = node;
            depth[c1] = depth[c2] = depth[node] + 1;
            leafs[pick] = c1; leafs[nl++] = c2;
        }
        double mean_depth = 0;
        for (int32_t t = 0; t < m; t++) mean_depth += depth[leafs[t]];
        mean_depth /= m;
        if (mean_depth < 1) mean_depth = 1;
        double qs = 1.0 - pow(1.0 - sub_total, 1.0 / mean_depth);
        double qi = 1.0 - pow(1.0 - indel_total, 1.0 / mean_depth);
        /* nodes are created parent-before-child, so a forward sweep evolves all */
        seq_t* seqs = (seq_t*)calloc((size_t)nn, sizeof(seq_t));
        seq_reserve(&seqs[0], root_len);
        seqs[0].len = root_len;
        for (int32_t t = 0; t < root_len; t++) seqs[0].a[t] = (uint8_t)below(&rng, (uint32_t)alphabet);
        for (int32_t v = 1; v < used; v++)
            evolve_edge(&rng, &seqs[parent[v]], &seqs[v], qs, qi, indel_mean, alphabet);
        for (int32_t t = 0; t < m; t++) {
            seq_t* src = &seqs[leafs[t]];
            seq_t* dst = &leaves[leaf_base + t];
            int32_t target = draw_length(&rng, len_dist, p1, p2, lo, hi);
            seq_reserve(dst, target > 0 ? target : 1);
            int32_t keep = src->len < target ? src->len : target;
            memcpy(dst->a, src->a, (size_t)keep);
            for (int32_t q = keep; q < target; q++) dst->a[q] = (uint8_t)below(&rng, (uint32_t)alphabet);
            dst->len = target;
        }
        for (int32_t v = 0; v < nn; v++) free(seqs[v].a);
        free(seqs); free(parent); free(depth); free(leafs);
        leaf_base += m;
    }
    /* seeded Fisher-Yates shuffle of the sequence order */
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    for (int64_t t = 0; t < n; t++) perm[t] = t;
    for (int64_t t = n - 1; t > 0; t--) {
        int64_t j = (int64_t)below(&rng, (uint32_t)(t + 1));
        int64_t tmp = perm[t]; perm[t] = perm[j]; perm[j] = tmp;
    }
    int64_t total = 0;
    for (int64_t t = 0; t < n; t++) total += leaves[perm[t]].len;
    if (total > res_capacity) {
        for (int64_t t = 0; t < n; t++) free(leaves[t].a);
        free(leaves); free(perm);
        return -1;
    }
    int64_t pos = 0;
    offsets_out[0] = 0;
    for (int64_t t = 0; t < n; t++) {
        seq_t* s = &leaves[perm[t]];
        memcpy(residues_out + pos, s->a, (size_t)s->len);
        pos += s->len;
        offsets_out[t + 1] = pos;
    }
    for (int64_t t = 0; t < n; t++) free(leaves[t].a);
    free(leaves); free(perm);
    return total;
}

/* Seeded symmetric substitution matrix: diagonal uniform in [dlo, dhi],
 * off-diagonal uniform in [olo, ohi]; row-major alphabet x alphabet int8. */
void synth_subst(uint64_t seed, int32_t alphabet, int32_t dlo, int32_t dhi,
                 int32_t olo, int32_t ohi, int8_t* out) {
    rng_t rng; rng_seed(&rng, seed);
    for (int a = 0; a < alphabet; a++) {
        out[a * alphabet + a] = (int8_t)(dlo + (int32_t)below(&rng, (uint32_t)(dhi - dlo + 1)));
        for (int b = a + 1; b < alphabet; b++) {
            int8_t v = (int8_t)(olo + (int32_t)below(&rng, (uint32_t)(ohi - olo + 1)));
            out[a * alphabet + b] = v;
            out[b * alphabet + a] = v;
        }
    }
}

/* Uniform random residues (no family structure), for adversarial and unit inputs. */
void synth_uniform(uint64_t seed, int64_t count, int32_t alphabet, uint8_t* out) {
    rng_t rng; rng_seed(&rng, seed);
    for (int64_t t = 0; t < count; t++) out[t] = (uint8_t)below(&rng, (uint32_t)alphabet);
}

/* Raw uniform doubles in [0,1), e.g. for Poisson arrival times of serving jobs. */
void synth_uniform_f64(uint64_t seed, int64_t count, double* out) {
    rng_t rng; rng_seed(&rng, seed);
    for (int64_t t = 0; t < count; t++) out[t] = uni(&rng);
}
