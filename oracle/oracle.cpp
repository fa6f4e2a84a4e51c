/*
 * CPU oracle for the Sample-Align-D data-parallel core.
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, obviously correct statement
 * of what the GPU path computes. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does. It
 * shares no code, headers or tables with the CUDA library.
 *
 * Every result is an exact integer definition:
 *   - k-mer similarity numerator a_ij = sum over k-mers tau of
 *     min(n_xi(tau), n_xj(tau)), denominator b_ij = min(|x_i|, |x_j|) - k + 1
 *     (Section 2, equation for r_ij; the stray factor tau printed inside the
 *     sum is read as a typesetting error).
 *   - average k-mer similarity D_i (Section 2, equation for D_i) in fixed point:
 *     D^_i = sum_j floor(a_ij * 2^32 / b_ij); the 1/N factor is dropped because it
 *     never changes an order inside one set. A term with b_ij <= 0 is 0.
 *   - the k-mer rank R_i = log(0.1 + D_i) (Section 2) is monotone in the ratio,
 *     so ranks are ordered by the exact key (a_i, b_i, i) with a_i/b_i compared
 *     by 64-bit cross-multiplication and ties broken by the index.
 *   - local ancestor of block b = argmax of the local D^ over the block
 *     (medoid, lowest index on ties); global ancestor = medoid of the local
 *     ancestors (Algorithm Sample-Align-D: local ancestors gathered at the root,
 *     the global ancestor broadcast back; Section 2.3.3).
 *   - regular-sampling redistribution (Section 2.3.2): blocks sorted by rank,
 *     p-1 evenly spaced samples per block, p(p-1) samples sorted, p-1 pivots,
 *     bucket = number of pivots strictly below the key.
 *   - per-bucket all-pairs global alignment scores with affine gaps (Gotoh),
 *     the aligner each processor runs on its bucket (Section 2.3.3; the paper
 *     allows any sequential aligner), as the textbook three-state recursion.
 *   - per-bucket guide tree, the first step of the progressive aligner that
 *     runs on each bucket (Section 2.3.3): average linkage (UPGMA) on the
 *     integer distances d_uv = S_uu + S_vv - 2 S_uv of the bucket's scores,
 *     the distance of two clusters being the pair sum over the product of
 *     their sizes, compared as exact rationals; ties go to the lexicographically
 *     smallest pair of cluster ids (leaves 0..nb-1, merge k creates nb + k).
 *   - per-bucket progressive alignment along that tree (Section 2.3.3): each
 *     merge aligns the two clusters' profiles with the three-state affine-gap
 *     recursion, a column pair scoring the sum of the substitution scores of
 *     the letter pairs across the profiles and a new gap run costing the
 *     member-count product times the pairwise run cost; the tie order and the
 *     column bookkeeping are stated at orc_progressive.
 *   - realignment of every bucket's alignment against the global ancestor and
 *     the glue of all buckets through the ancestor's positions (the last steps
 *     of the algorithm box), stated at orc_ancestor_glue.
 */
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using KmerCounts = std::unordered_map<uint64_t, int64_t>;

const int64_t NEG_INF = INT64_MIN / 4;

// Count every contiguous length-k window of sequence s (residues mapped
// through class_map when given). The code of a k-mer is its base-A' number.
KmerCounts count_kmers(const uint8_t* s, int64_t len, const uint8_t* class_map,
                       int32_t kmer_alphabet, int32_t k) {
    KmerCounts c;
    for (int64_t start = 0; start + k <= len; start++) {
        uint64_t code = 0;
        for (int32_t t = 0; t < k; t++) {
            uint64_t letter = class_map ? class_map[s[start + t]] : s[start + t];
            code = code * (uint64_t)kmer_alphabet + letter;
        }
        c[code] += 1;
    }
    return c;
}

int64_t shared_kmers(const KmerCounts& x, const KmerCounts& y) {
    const KmerCounts& small = x.size() <= y.size() ? x : y;
    const KmerCounts& big = x.size() <= y.size() ? y : x;
    int64_t a = 0;
    for (const auto& kv : small) {
        auto it = big.find(kv.first);
        if (it != big.end()) a += std::min(kv.second, it->second);
    }
    return a;
}

// floor(a * 2^32 / b) for 0 <= a <= b; 0 when b <= 0 (no k-mer fits).
uint64_t fixed_ratio(int64_t a, int64_t b) {
    if (b <= 0) return 0;
    return ((uint64_t)a << 32) / (uint64_t)b;
}

int64_t denom(int64_t li, int64_t lj, int32_t k) { return std::min(li, lj) - k + 1; }

template <class F>
void parallel_for(int64_t count, int32_t nthreads, F fn) {
    if (nthreads <= 1 || count < 2) {
        for (int64_t t = 0; t < count; t++) fn(t);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> pool;
    for (int32_t w = 0; w < nthreads; w++)
        pool.emplace_back([&]() {
            for (;;) {
                int64_t t = next.fetch_add(1);
                if (t >= count) break;
                fn(t);
            }
        });
    for (auto& th : pool) th.join();
}

int64_t block_begin(int64_t b, int64_t n, int64_t p) { return b * n / p; }

// Rank key order: a_i/b_i ascending (cross-multiplied), then index ascending.
struct KeyLess {
    const int32_t* ka;
    const int32_t* kb;
    bool operator()(int32_t i, int32_t j) const {
        int64_t lhs = (int64_t)ka[i] * (int64_t)kb[j];
        int64_t rhs = (int64_t)ka[j] * (int64_t)kb[i];
        if (lhs != rhs) return lhs < rhs;
        return i < j;
    }
};

}  // namespace

/* Regular-sampling redistribution (Section 2.3.2) under a strict total order
 * `less` on sequence indices. Each of the p contiguous blocks is sorted, p-1
 * regular samples are taken per non-empty block (positions floor(j*w/p)),
 * all samples are sorted, and pivot m (1-based) is the sample at 1-based
 * position (m-1)*q + max(1, floor(q/2)) where q counts the non-empty blocks.
 * A sequence goes to the bucket numbered by how many pivots rank strictly
 * below it. */
template <class Less>
void regular_sampling(int32_t n, int32_t p, Less less, int32_t* bucket_offsets, int32_t* order,
                      int32_t* pivot_idx) {
    std::vector<int32_t> samples;
    int32_t q = 0;  // blocks that hold at least one sequence
    for (int32_t b = 0; b < p; b++) {
        int64_t lo = block_begin(b, n, p), hi = block_begin(b + 1, n, p);
        int64_t w = hi - lo;
        if (w == 0) continue;
        q++;
        std::vector<int32_t> blk;
        for (int64_t i = lo; i < hi; i++) blk.push_back((int32_t)i);
        std::sort(blk.begin(), blk.end(), less);
        for (int64_t j = 1; j <= p - 1; j++) samples.push_back(blk[(j * w) / p]);
    }
    std::sort(samples.begin(), samples.end(), less);
    std::vector<int32_t> piv;
    for (int32_t m = 1; m <= p - 1; m++) {
        if (q == 0) { pivot_idx[m - 1] = -1; continue; }
        int64_t pos1 = (int64_t)(m - 1) * q + std::max(1, q / 2);  // 1-based
        int32_t s = samples[pos1 - 1];
        pivot_idx[m - 1] = s;
        piv.push_back(s);
    }
    std::vector<int32_t> bucket(n);
    std::vector<int32_t> count(p, 0);
    for (int32_t i = 0; i < n; i++) {
        int32_t c = 0;
        for (int32_t s : piv) if (less(s, i)) c++;
        bucket[i] = c;
        count[c]++;
    }
    bucket_offsets[0] = 0;
    for (int32_t b = 0; b < p; b++) bucket_offsets[b + 1] = bucket_offsets[b] + count[b];
    std::vector<int32_t> fill(bucket_offsets, bucket_offsets + p);
    for (int32_t i = 0; i < n; i++) order[fill[bucket[i]]++] = i;
}

extern "C" {

/* Per-sequence k-mer histograms flattened as (sequence, code, count) triples,
 * sorted by sequence then code. Returns the triple count, or -1 if cap_triples
 * is too small (then nothing is written). */
int64_t orc_kmer_histograms(const uint8_t* res, const int64_t* offs, int32_t n,
                            const uint8_t* class_map, int32_t kmer_alphabet, int32_t k,
                            int64_t* out_triples, int64_t cap_triples) {
    std::vector<std::vector<std::pair<uint64_t, int64_t>>> all(n);
    int64_t total = 0;
    for (int32_t i = 0; i < n; i++) {
        KmerCounts c = count_kmers(res + offs[i], offs[i + 1] - offs[i], class_map, kmer_alphabet, k);
        all[i].assign(c.begin(), c.end());
        std::sort(all[i].begin(), all[i].end());
        total += (int64_t)all[i].size();
    }
    if (total > cap_triples) return -1;
    int64_t w = 0;
    for (int32_t i = 0; i < n; i++)
        for (auto& kv : all[i]) {
            out_triples[3 * w] = i;
            out_triples[3 * w + 1] = (int64_t)kv.first;
            out_triples[3 * w + 2] = kv.second;
            w++;
        }
    return total;
}

/* k-mer rank stage. Outputs (all host, caller-owned):
 *   A      nullable, n*n int32 row-major: a_ij
 *   dloc   n: sum over j in block(i) of floor(a_ij 2^32 / b_ij)
 *   dcen   n: the same sum over all j
 *   la     p: local ancestor of each block (-1 for an empty block)
 *   ga     1: global ancestor (-1 when n == 0)
 *   key_a, key_b  n: a(i, GA) and b(i, GA) (key (0, 1) when b(i, GA) <= 0)
 * Returns 0, or -1 on invalid arguments. */
int orc_kmer_rank(const uint8_t* res, const int64_t* offs, int32_t n, int32_t alphabet,
                  const uint8_t* class_map, int32_t kmer_alphabet, int32_t k, int32_t p,
                  int32_t nthreads, int32_t* A, uint64_t* dloc, uint64_t* dcen, int32_t* la,
                  int32_t* ga, int32_t* key_a, int32_t* key_b) {
    if (n < 0 || k < 1 || p < 1 || alphabet < 1 || kmer_alphabet < 1) return -1;
    for (int32_t i = 0; i < n; i++)
        for (int64_t t = offs[i]; t < offs[i + 1]; t++) {
            if (res[t] >= alphabet) return -1;
            if (class_map && class_map[res[t]] >= kmer_alphabet) return -1;
            if (!class_map && res[t] >= kmer_alphabet) return -1;
        }
    std::vector<KmerCounts> cnt(n);
    std::vector<int64_t> len(n);
    parallel_for(n, nthreads, [&](int64_t i) {
        len[i] = offs[i + 1] - offs[i];
        cnt[i] = count_kmers(res + offs[i], len[i], class_map, kmer_alphabet, k);
    });
    auto block_of = [&](int64_t i) {
        // largest b with floor(b n / p) <= i
        int64_t b = (i * p) / n;
        while (b + 1 < p && block_begin(b + 1, n, p) <= i) b++;
        while (b > 0 && block_begin(b, n, p) > i) b--;
        return b;
    };
    parallel_for(n, nthreads, [&](int64_t i) {
        uint64_t sl = 0, sc = 0;
        int64_t bi = block_of(i);
        for (int32_t j = 0; j < n; j++) {
            int64_t a = shared_kmers(cnt[i], cnt[j]);
            if (A) A[(int64_t)i * n + j] = (int32_t)a;
            uint64_t term = fixed_ratio(a, denom(len[i], len[j], k));
            sc += term;
            if (block_of(j) == bi) sl += term;
        }
        dloc[i] = sl;
        dcen[i] = sc;
    });
    for (int32_t b = 0; b < p; b++) {
        int64_t lo = block_begin(b, n, p), hi = block_begin(b + 1, n, p);
        int32_t best = -1;
        for (int64_t i = lo; i < hi; i++)
            if (best < 0 || dloc[i] > dloc[best]) best = (int32_t)i;
        la[b] = best;
    }
    int32_t g = -1;
    uint64_t gbest = 0;
    for (int32_t b = 0; b < p; b++) {
        if (la[b] < 0) continue;
        uint64_t s = 0;
        for (int32_t b2 = 0; b2 < p; b2++) {
            if (la[b2] < 0) continue;
            int64_t a = shared_kmers(cnt[la[b]], cnt[la[b2]]);
            s += fixed_ratio(a, denom(len[la[b]], len[la[b2]], k));
        }
        if (g < 0 || s > gbest) { g = la[b]; gbest = s; }
    }
    *ga = g;
    for (int32_t i = 0; i < n; i++) {
        int64_t b = denom(len[i], len[g], k);
        if (b <= 0) { key_a[i] = 0; key_b[i] = 1; continue; }
        key_a[i] = (int32_t)shared_kmers(cnt[i], cnt[g]);
        key_b[i] = (int32_t)b;
    }
    return 0;
}

/* Selected rows of the k-mer stage, for inputs too large to redo in full:
 * for each listed sequence i, a_ij for every j (A_rows, nrows x n) and its
 * two fixed-point D sums, exactly as orc_kmer_rank defines them.
 * Returns 0, or -1 on invalid arguments. */
int orc_kmer_rows(const uint8_t* res, const int64_t* offs, int32_t n, int32_t alphabet,
                  const uint8_t* class_map, int32_t kmer_alphabet, int32_t k, int32_t p,
                  const int32_t* rows, int32_t nrows, int32_t nthreads, int32_t* A_rows,
                  uint64_t* dloc, uint64_t* dcen) {
    if (n < 1 || k < 1 || p < 1) return -1;
    std::vector<KmerCounts> cnt(n);
    std::vector<int64_t> len(n);
    parallel_for(n, nthreads, [&](int64_t i) {
        len[i] = offs[i + 1] - offs[i];
        cnt[i] = count_kmers(res + offs[i], len[i], class_map, kmer_alphabet, k);
    });
    auto block_of = [&](int64_t i) {
        int64_t b = (i * p) / n;
        while (b + 1 < p && block_begin(b + 1, n, p) <= i) b++;
        while (b > 0 && block_begin(b, n, p) > i) b--;
        return b;
    };
    for (int32_t r = 0; r < nrows; r++)
        if (rows[r] < 0 || rows[r] >= n) return -1;
    parallel_for(nrows, nthreads, [&](int64_t r) {
        const int32_t i = rows[r];
        uint64_t sl = 0, sc = 0;
        const int64_t bi = block_of(i);
        for (int32_t j = 0; j < n; j++) {
            const int64_t a = shared_kmers(cnt[i], cnt[j]);
            A_rows[r * (int64_t)n + j] = (int32_t)a;
            const uint64_t term = fixed_ratio(a, denom(len[i], len[j], k));
            sc += term;
            if (block_of(j) == bi) sl += term;
        }
        dloc[r] = sl;
        dcen[r] = sc;
    });
    return 0;
}

/* Globalized k-mer rank (Section 2.3.1; algorithm box: a sample set of s
 * sequences per processor, sent to all processors, every sequence ranked
 * against the s*p samples). Each block is sorted by its local rank (dloc, then
 * index); its samples are the members at 0-based positions
 * floor((2j+1) w_b / (2s)), j = 0..s-1 (evenly spaced strata; a member may be
 * taken twice when w_b < s). G_i = sum over the s*p samples sigma of
 * floor(a_i,sigma 2^32 / b_i,sigma), a sample taken twice counting twice.
 * sample_idx: p*s entries, -1 for the slots of an empty block.
 * Returns 0, or -1 on invalid arguments. */
int orc_global_rank(const uint8_t* res, const int64_t* offs, int32_t n, const uint8_t* class_map,
                    int32_t kmer_alphabet, int32_t k, int32_t p, int32_t s, int32_t nthreads,
                    const uint64_t* dloc, uint64_t* G, int32_t* sample_idx) {
    if (n < 0 || k < 1 || p < 1 || s < 1) return -1;
    std::vector<int32_t> samples;
    for (int32_t b = 0; b < p; b++) {
        const int64_t lo = block_begin(b, n, p), hi = block_begin(b + 1, n, p), w = hi - lo;
        std::vector<int32_t> blk;
        for (int64_t i = lo; i < hi; i++) blk.push_back((int32_t)i);
        std::sort(blk.begin(), blk.end(), [&](int32_t x, int32_t y) {
            return dloc[x] != dloc[y] ? dloc[x] < dloc[y] : x < y;
        });
        for (int32_t j = 0; j < s; j++) {
            int32_t v = -1;
            if (w > 0) {
                v = blk[(size_t)(((int64_t)(2 * j + 1) * w) / (2 * (int64_t)s))];
                samples.push_back(v);
            }
            sample_idx[(int64_t)b * s + j] = v;
        }
    }
    std::vector<KmerCounts> cnt(n);
    std::vector<int64_t> len(n);
    parallel_for(n, nthreads, [&](int64_t i) {
        len[i] = offs[i + 1] - offs[i];
        cnt[i] = count_kmers(res + offs[i], len[i], class_map, kmer_alphabet, k);
    });
    parallel_for(n, nthreads, [&](int64_t i) {
        uint64_t g = 0;
        for (int32_t v : samples) g += fixed_ratio(shared_kmers(cnt[i], cnt[v]), denom(len[i], len[v], k));
        G[i] = g;
    });
    return 0;
}

/* Regular sampling on 64-bit integer rank keys (the globalized rank G), ties
 * by index. Returns 0, or -1 on invalid arguments. */
int orc_partition_keys64(int32_t n, const uint64_t* keys, int32_t p, int32_t* bucket_offsets,
                         int32_t* order, int32_t* pivot_idx) {
    if (n < 0 || p < 1) return -1;
    auto less = [&](int32_t i, int32_t j) { return keys[i] != keys[j] ? keys[i] < keys[j] : i < j; };
    regular_sampling(n, p, less, bucket_offsets, order, pivot_idx);
    return 0;
}

/* Regular-sampling redistribution by the rational rank key a/b (Section
 * 2.3.2). bucket_offsets: p+1; order: n (members of a bucket ascending by
 * index); pivot_idx: p-1 sequence indices of the pivots (-1 when there is
 * none). Returns 0, or -1 on invalid arguments. */
int orc_partition(int32_t n, const int32_t* key_a, const int32_t* key_b, int32_t p,
                  int32_t* bucket_offsets, int32_t* order, int32_t* pivot_idx) {
    if (n < 0 || p < 1) return -1;
    for (int32_t i = 0; i < n; i++)
        if (key_a[i] < 0 || key_b[i] < 1 || key_a[i] > key_b[i]) return -1;
    regular_sampling(n, p, KeyLess{key_a, key_b}, bucket_offsets, order, pivot_idx);
    return 0;
}

}  // extern "C"

namespace {

/* The three score tables of the global affine-gap alignment: M, X and Y hold
 * the best score of an alignment of x[0..i) with y[0..j) whose last column is
 * a match column (M), x_i against a gap (X) or a gap against y_j (Y). A gap
 * run of length g costs go + g*ge (go, ge <= 0); end gaps cost the same as
 * internal ones; a run of X columns may directly follow a run of Y columns,
 * each opening its own gap. 64-bit arithmetic; NEG_INF marks no alignment. */
struct GotohTables {
    int64_t W;
    std::vector<int64_t> M, X, Y;
    int64_t at(int64_t i, int64_t j) const { return i * W + j; }
};

GotohTables fill_gotoh(const uint8_t* x, int32_t m, const uint8_t* y, int32_t n, const int8_t* S,
                       int32_t alphabet, int32_t go, int32_t ge) {
    GotohTables t;
    t.W = (int64_t)n + 1;
    t.M.assign((size_t)(m + 1) * t.W, NEG_INF);
    t.X.assign((size_t)(m + 1) * t.W, NEG_INF);
    t.Y.assign((size_t)(m + 1) * t.W, NEG_INF);
    std::vector<int64_t>&M = t.M, &X = t.X, &Y = t.Y;
    auto at = [&](int64_t i, int64_t j) { return t.at(i, j); };
    M[at(0, 0)] = 0;  // the empty alignment
    for (int32_t i = 0; i <= m; i++)
        for (int32_t j = 0; j <= n; j++) {
            if (i == 0 && j == 0) continue;
            if (i > 0 && j > 0) {
                int64_t prev = std::max({M[at(i - 1, j - 1)], X[at(i - 1, j - 1)], Y[at(i - 1, j - 1)]});
                if (prev > NEG_INF) M[at(i, j)] = prev + S[x[i - 1] * alphabet + y[j - 1]];
            }
            if (i > 0) {
                int64_t open = std::max(M[at(i - 1, j)], Y[at(i - 1, j)]);
                int64_t v = NEG_INF;
                if (open > NEG_INF) v = open + go + ge;
                if (X[at(i - 1, j)] > NEG_INF) v = std::max(v, X[at(i - 1, j)] + ge);
                X[at(i, j)] = v;
            }
            if (j > 0) {
                int64_t open = std::max(M[at(i, j - 1)], X[at(i, j - 1)]);
                int64_t v = NEG_INF;
                if (open > NEG_INF) v = open + go + ge;
                if (Y[at(i, j - 1)] > NEG_INF) v = std::max(v, Y[at(i, j - 1)] + ge);
                Y[at(i, j)] = v;
            }
        }
    return t;
}

/* One optimal alignment of profile P (m columns, np members; counts
 * cp[column * alphabet + letter]) with profile Q (w columns, nq members): the
 * three-state recursion of fill_gotoh in which a column pair scores the sum of
 * S over the letter pairs across the two profiles and a new gap run of length
 * g costs np nq (go + g ge); the traceback takes the tie order of orc_align.
 * Writes the optimum and the columns ('M', 'X': P's column against a gap, 'Y')
 * first to last; false when the tables are inconsistent. */
bool profile_align(const std::vector<int64_t>& cp, int64_t np, int64_t m, const std::vector<int64_t>& cq, int64_t nq,
                   int64_t w, const int8_t* S, int32_t alphabet, int32_t go, int32_t ge, int64_t* score_out,
                   std::string* cols) {
    // sum_b S[a][b] cntQ[j][b] for every column j and letter a (a factor of s(i, j))
    std::vector<int64_t> sq((size_t)w * alphabet, 0);
    for (int64_t j = 0; j < w; j++)
        for (int32_t a = 0; a < alphabet; a++)
            for (int32_t c = 0; c < alphabet; c++) sq[j * alphabet + a] += S[a * alphabet + c] * cq[j * alphabet + c];
    auto s = [&](int64_t i, int64_t j) {  // 1-based column indices
        int64_t v = 0;
        for (int32_t a = 0; a < alphabet; a++) v += cp[(i - 1) * alphabet + a] * sq[(j - 1) * alphabet + a];
        return v;
    };
    const int64_t gop = (int64_t)go * np * nq, gex = (int64_t)ge * np * nq;
    // the three tables, as in fill_gotoh
    const int64_t W = w + 1;
    std::vector<int64_t> TM((size_t)(m + 1) * W, NEG_INF), TX(TM), TY(TM);
    auto at = [&](int64_t i, int64_t j) { return i * W + j; };
    TM[at(0, 0)] = 0;
    for (int64_t i = 0; i <= m; i++)
        for (int64_t j = 0; j <= w; j++) {
            if (i == 0 && j == 0) continue;
            if (i > 0 && j > 0) {
                const int64_t prev = std::max({TM[at(i - 1, j - 1)], TX[at(i - 1, j - 1)], TY[at(i - 1, j - 1)]});
                if (prev > NEG_INF) TM[at(i, j)] = prev + s(i, j);
            }
            if (i > 0) {
                const int64_t open = std::max(TM[at(i - 1, j)], TY[at(i - 1, j)]);
                int64_t v = NEG_INF;
                if (open > NEG_INF) v = open + gop + gex;
                if (TX[at(i - 1, j)] > NEG_INF) v = std::max(v, TX[at(i - 1, j)] + gex);
                TX[at(i, j)] = v;
            }
            if (j > 0) {
                const int64_t open = std::max(TM[at(i, j - 1)], TX[at(i, j - 1)]);
                int64_t v = NEG_INF;
                if (open > NEG_INF) v = open + gop + gex;
                if (TY[at(i, j - 1)] > NEG_INF) v = std::max(v, TY[at(i, j - 1)] + gex);
                TY[at(i, j)] = v;
            }
        }
    // traceback with the tie order of orc_align
    auto best_of = [&](int64_t i, int64_t j, bool useM, bool useX, bool useY, int64_t want, int64_t add) {
        if (useM && TM[at(i, j)] > NEG_INF && TM[at(i, j)] + add == want) return 'M';
        if (useX && TX[at(i, j)] > NEG_INF && TX[at(i, j)] + add == want) return 'X';
        if (useY && TY[at(i, j)] > NEG_INF && TY[at(i, j)] + add == want) return 'Y';
        return '?';
    };
    const int64_t score = std::max({TM[at(m, w)], TX[at(m, w)], TY[at(m, w)]});
    char state = best_of(m, w, true, true, true, score, 0);
    std::string rev;
    int64_t i = m, j = w;
    while (i > 0 || j > 0) {
        rev.push_back(state);
        if (state == 'M') {
            state = best_of(i - 1, j - 1, true, true, true, TM[at(i, j)] - s(i, j), 0);
            i--;
            j--;
        } else if (state == 'X') {
            const int64_t v = TX[at(i, j)];
            const char ext = best_of(i - 1, j, false, true, false, v, gex);
            state = ext == 'X' ? 'X' : best_of(i - 1, j, true, false, true, v, gop + gex);
            i--;
        } else if (state == 'Y') {
            const int64_t v = TY[at(i, j)];
            const char ext = best_of(i, j - 1, false, false, true, v, gex);
            state = ext == 'Y' ? 'Y' : best_of(i, j - 1, true, true, false, v, gop + gex);
            j--;
        } else {
            return false;
        }
    }
    *score_out = score;
    cols->assign(rev.rbegin(), rev.rend());
    return true;
}

}  // namespace

extern "C" {

/* Global alignment score with affine gaps (the three tables above). */
int64_t orc_gotoh(const uint8_t* x, int32_t m, const uint8_t* y, int32_t n, const int8_t* S,
                  int32_t alphabet, int32_t go, int32_t ge) {
    const GotohTables t = fill_gotoh(x, m, y, n, S, alphabet, go, ge);
    return std::max({t.M[t.at(m, n)], t.X[t.at(m, n)], t.Y[t.at(m, n)]});
}

/* One optimal global alignment: columns 'M' (x_i with y_j), 'X' (x_i against a
 * gap) and 'Y' (a gap against y_j), first column first, written to ops
 * (capacity m + n); *len receives the column count. Traced back through the
 * tables from the best state at (m, n), preferring M, then X, then Y among
 * equal predecessors. Returns the score. */
int64_t orc_align(const uint8_t* x, int32_t m, const uint8_t* y, int32_t n, const int8_t* S, int32_t alphabet,
                  int32_t go, int32_t ge, char* ops, int32_t* len) {
    const GotohTables t = fill_gotoh(x, m, y, n, S, alphabet, go, ge);
    auto subst = [&](uint8_t a, uint8_t b) { return (int64_t)S[(int64_t)a * alphabet + b]; };
    auto best_of = [&](int64_t i, int64_t j, bool useM, bool useX, bool useY, int64_t want, int64_t add) {
        if (useM && t.M[t.at(i, j)] > NEG_INF && t.M[t.at(i, j)] + add == want) return 'M';
        if (useX && t.X[t.at(i, j)] > NEG_INF && t.X[t.at(i, j)] + add == want) return 'X';
        if (useY && t.Y[t.at(i, j)] > NEG_INF && t.Y[t.at(i, j)] + add == want) return 'Y';
        return '?';
    };
    const int64_t score = std::max({t.M[t.at(m, n)], t.X[t.at(m, n)], t.Y[t.at(m, n)]});
    char state = best_of(m, n, true, true, true, score, 0);
    std::string rev;
    int64_t i = m, j = n;
    while (i > 0 || j > 0) {
        rev.push_back(state);
        if (state == 'M') {
            const int64_t v = t.M[t.at(i, j)] - subst(x[i - 1], y[j - 1]);
            state = best_of(i - 1, j - 1, true, true, true, v, 0);
            i--;
            j--;
        } else if (state == 'X') {
            const int64_t v = t.X[t.at(i, j)];
            const char ext = best_of(i - 1, j, false, true, false, v, ge);
            state = ext == 'X' ? 'X' : best_of(i - 1, j, true, false, true, v, go + ge);
            i--;
        } else if (state == 'Y') {
            const int64_t v = t.Y[t.at(i, j)];
            const char ext = best_of(i, j - 1, false, false, true, v, ge);
            state = ext == 'Y' ? 'Y' : best_of(i, j - 1, true, true, false, v, go + ge);
            j--;
        } else {
            return NEG_INF;  // cannot happen for a consistent table
        }
    }
    *len = (int32_t)rev.size();
    for (size_t c = 0; c < rev.size(); c++) ops[c] = rev[rev.size() - 1 - c];
    return score;
}

/* Score of a given alignment (columns as in orc_align): the sum of S over the
 * M columns plus go + g*ge for every maximal run of g X columns and every
 * maximal run of g Y columns. Returns 0 and *score, or -1 when the columns do
 * not consume exactly x[0..m) and y[0..n) or hold another letter. */
int orc_alignment_score(const uint8_t* x, int32_t m, const uint8_t* y, int32_t n, const char* ops,
                        int32_t len, const int8_t* S, int32_t alphabet, int32_t go, int32_t ge,
                        int64_t* score) {
    int64_t total = 0, i = 0, j = 0;
    for (int32_t c = 0; c < len; c++) {
        const char op = ops[c];
        if (op == 'M') {
            if (i >= m || j >= n) return -1;
            total += S[x[i] * alphabet + y[j]];
            i++;
            j++;
        } else if (op == 'X' || op == 'Y') {
            if (op == 'X' && i >= m) return -1;
            if (op == 'Y' && j >= n) return -1;
            if (c == 0 || ops[c - 1] != op) total += go;  // a new run opens
            total += ge;
            if (op == 'X') i++;
            else j++;
        } else {
            return -1;
        }
    }
    if (i != m || j != n) return -1;
    *score = total;
    return 0;
}

/* All pairs u <= v inside every bucket. score_offsets: p+1 (filled);
 * scores[score_offsets[b] + u*nb - u*(u-1)/2 + (v-u)] = S(x_order[..u], x_order[..v]).
 * Returns 0, or -1 on invalid arguments. */
int orc_bucket_pair_scores(const uint8_t* res, const int64_t* offs, int32_t n,
                           const int32_t* bucket_offsets, const int32_t* order, int32_t p,
                           const int8_t* S, int32_t alphabet, int32_t go, int32_t ge,
                           int32_t nthreads, int64_t* score_offsets, int32_t* scores) {
    if (p < 1 || go > 0 || ge > 0) return -1;
    for (int32_t a = 0; a < alphabet; a++)
        for (int32_t b = 0; b < alphabet; b++)
            if (S[a * alphabet + b] != S[b * alphabet + a]) return -1;
    score_offsets[0] = 0;
    for (int32_t b = 0; b < p; b++) {
        int64_t nb = bucket_offsets[b + 1] - bucket_offsets[b];
        score_offsets[b + 1] = score_offsets[b] + nb * (nb + 1) / 2;
    }
    std::vector<std::pair<int32_t, int64_t>> rows;  // (bucket, u)
    for (int32_t b = 0; b < p; b++)
        for (int64_t u = 0; u < bucket_offsets[b + 1] - bucket_offsets[b]; u++) rows.push_back({b, u});
    parallel_for((int64_t)rows.size(), nthreads, [&](int64_t r) {
        int32_t b = rows[r].first;
        int64_t u = rows[r].second;
        int64_t nb = bucket_offsets[b + 1] - bucket_offsets[b];
        int32_t xi = order[bucket_offsets[b] + u];
        for (int64_t v = u; v < nb; v++) {
            int32_t yi = order[bucket_offsets[b] + v];
            int64_t s = orc_gotoh(res + offs[xi], (int32_t)(offs[xi + 1] - offs[xi]), res + offs[yi],
                                  (int32_t)(offs[yi + 1] - offs[yi]), S, alphabet, go, ge);
            scores[score_offsets[b] + u * nb - u * (u - 1) / 2 + (v - u)] = (int32_t)s;
        }
    });
    return 0;
}

/* Average-linkage guide tree of every bucket from its pair scores (layout of
 * orc_bucket_pair_scores). merge_offsets: p+1 (filled; bucket b's merges are
 * [merge_offsets[b], merge_offsets[b+1]), nb - 1 of them when nb >= 1). Merge k
 * of a bucket joins clusters left < right into cluster nb + k at distance
 * num / den (num = sum of d_uv over the pairs between the two clusters, den =
 * the product of their sizes). Plain O(nb^3): every step scans every pair of
 * live clusters. Returns 0. */
int orc_guide_trees(const int32_t* bucket_offsets, int32_t p, const int64_t* score_offsets,
                    const int32_t* scores, int64_t* merge_offsets, int32_t* left, int32_t* right,
                    int64_t* num, int64_t* den) {
    merge_offsets[0] = 0;
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = bucket_offsets[b + 1] - bucket_offsets[b];
        merge_offsets[b + 1] = merge_offsets[b] + (nb > 0 ? nb - 1 : 0);
    }
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = bucket_offsets[b + 1] - bucket_offsets[b];
        if (nb < 2) continue;
        const int32_t* sc = scores + score_offsets[b];
        auto S = [&](int64_t u, int64_t v) {  // u <= v
            return (int64_t)sc[u * nb - u * (u - 1) / 2 + (v - u)];
        };
        // clusters: id, size, alive; W[i][j] = sum of d over member pairs of clusters i, j
        const int64_t cap = 2 * nb - 1;
        std::vector<int64_t> size(cap, 0);
        std::vector<char> alive(cap, 0);
        std::vector<std::vector<int64_t>> W(cap, std::vector<int64_t>(cap, 0));
        for (int64_t u = 0; u < nb; u++) {
            size[u] = 1;
            alive[u] = 1;
            for (int64_t v = 0; v < nb; v++)
                if (u != v) W[u][v] = S(u, u) + S(v, v) - 2 * S(std::min(u, v), std::max(u, v));
        }
        for (int64_t k = 0; k < nb - 1; k++) {
            int64_t bi = -1, bj = -1;
            for (int64_t i = 0; i < nb + k; i++) {
                if (!alive[i]) continue;
                for (int64_t j = i + 1; j < nb + k; j++) {
                    if (!alive[j]) continue;
                    if (bi < 0) {
                        bi = i;
                        bj = j;
                        continue;
                    }
                    // W[i][j] / (size_i size_j) < W[bi][bj] / (size_bi size_bj), exactly
                    const __int128 lhs = (__int128)W[i][j] * (size[bi] * size[bj]);
                    const __int128 rhs = (__int128)W[bi][bj] * (size[i] * size[j]);
                    if (lhs < rhs) {  // on equality the pair met first (smaller ids) stays
                        bi = i;
                        bj = j;
                    }
                }
            }
            const int64_t c = nb + k, m = merge_offsets[b] + k;
            left[m] = (int32_t)bi;
            right[m] = (int32_t)bj;
            num[m] = W[bi][bj];
            den[m] = size[bi] * size[bj];
            size[c] = size[bi] + size[bj];
            alive[c] = 1;
            alive[bi] = alive[bj] = 0;
            for (int64_t x = 0; x < c; x++) {
                if (!alive[x]) continue;
                W[c][x] = W[x][c] = W[bi][x] + W[bj][x];
            }
        }
    }
    return 0;
}

/* Progressive alignment of every bucket along its guide tree (the aligner
 * each processor runs on its bucket, Section 2.3.3), merge by merge in the
 * tree's order. A cluster is a multiple alignment of its members: its profile
 * column c holds, per letter a, the number of members with letter a in column
 * c. Merge k aligns the profile P of cluster left[k] (rows) with the profile Q
 * of cluster right[k] (columns) by the three-state global affine-gap
 * recursion of orc_align, where pairing column i of P with column j of Q
 * scores the sum of S over the letter pairs across the two profiles,
 *   s(i, j) = sum_a sum_b cntP[i][a] cntQ[j][b] S[a][b]
 * (a gap in an existing column pairs with nothing), and a new gap run of
 * length g costs nP nQ (go + g ge), nP and nQ being the member counts: every
 * cross pair of members receives the run. Ties are taken as in orc_align. The
 * merged cluster has one column per alignment column, in order; its members
 * are P's followed by Q's, each residue moved to the column its old column
 * went to. Outputs: widths[b] = the number of columns of bucket b's final
 * alignment (the root cluster; a one-member bucket is its sequence, an empty
 * one 0); merge_scores / merge_widths per merge (layout of orc_guide_trees);
 * colmap = the final column of every residue, over the residues of order[0],
 * order[1], ... in turn. Returns 0, or -1 on a tree that is not a tree. */
int orc_progressive(const uint8_t* res, const int64_t* offs, int32_t n, const int32_t* bucket_offsets,
                    const int32_t* order, int32_t p, const int64_t* merge_offsets, const int32_t* left,
                    const int32_t* right, const int8_t* S, int32_t alphabet, int32_t go, int32_t ge,
                    int32_t nthreads, int32_t* widths, int64_t* merge_scores, int32_t* merge_widths,
                    int32_t* colmap) {
    if (p < 1 || n < 0) return -1;
    // where each bucket position's residues start in colmap (positions 0 .. bucket_offsets[p])
    const int32_t npos = bucket_offsets[p];
    std::vector<int64_t> pos_off((size_t)npos + 1, 0);
    for (int32_t q = 0; q < npos; q++) {
        if (order[q] < 0 || order[q] >= n) return -1;
        pos_off[q + 1] = pos_off[q] + (offs[order[q] + 1] - offs[order[q]]);
    }
    std::atomic<int> bad(0);
    parallel_for(p, nthreads, [&](int64_t b) {
        const int32_t boff = bucket_offsets[b];
        const int64_t nb = bucket_offsets[b + 1] - boff;
        struct Cluster {
            std::vector<int32_t> members;           // bucket positions
            std::vector<std::vector<int64_t>> col;  // per member: the column of each residue
            int64_t width = 0;
            bool alive = false;
        };
        std::vector<Cluster> cl(nb > 0 ? 2 * nb - 1 : 0);
        for (int64_t u = 0; u < nb; u++) {
            const int32_t sq = order[boff + u];
            const int64_t len = offs[sq + 1] - offs[sq];
            cl[u].members = {(int32_t)u};
            std::vector<int64_t> c(len);
            for (int64_t r = 0; r < len; r++) c[r] = r;
            cl[u].col = {c};
            cl[u].width = len;
            cl[u].alive = true;
        }
        auto residues_of = [&](int32_t u) { return res + offs[order[boff + u]]; };
        auto profile = [&](const Cluster& c) {  // counts[col * alphabet + letter]
            std::vector<int64_t> cnt((size_t)c.width * alphabet, 0);
            for (size_t t = 0; t < c.members.size(); t++) {
                const uint8_t* x = residues_of(c.members[t]);
                for (size_t r = 0; r < c.col[t].size(); r++) cnt[c.col[t][r] * alphabet + x[r]]++;
            }
            return cnt;
        };
        for (int64_t k = 0; k + 1 < nb; k++) {
            const int64_t mi = merge_offsets[b] + k;
            const int32_t li = left[mi], ri = right[mi];
            if (li < 0 || ri < 0 || li >= nb + k || ri >= nb + k || li == ri || !cl[li].alive || !cl[ri].alive) {
                bad = 1;
                return;
            }
            Cluster &P = cl[li], &Q = cl[ri];
            const int64_t m = P.width, w = Q.width;
            const int64_t np = (int64_t)P.members.size(), nq = (int64_t)Q.members.size();
            const std::vector<int64_t> cp = profile(P), cq = profile(Q);
            int64_t score = 0;
            std::string fwd;
            if (!profile_align(cp, np, m, cq, nq, w, S, alphabet, go, ge, &score, &fwd)) {
                bad = 1;
                return;
            }
            // the merged cluster: alignment column c takes P's column and/or Q's column
            const int64_t len = (int64_t)fwd.size();
            std::vector<int64_t> mapP(m), mapQ(w);
            int64_t pi = 0, qj = 0;
            for (int64_t c = 0; c < len; c++) {
                const char op = fwd[c];
                if (op == 'M' || op == 'X') mapP[pi++] = c;
                if (op == 'M' || op == 'Y') mapQ[qj++] = c;
            }
            Cluster& R = cl[nb + k];
            R.members = P.members;
            R.members.insert(R.members.end(), Q.members.begin(), Q.members.end());
            for (auto c : P.col) {
                for (auto& v : c) v = mapP[v];
                R.col.push_back(c);
            }
            for (auto c : Q.col) {
                for (auto& v : c) v = mapQ[v];
                R.col.push_back(c);
            }
            R.width = len;
            R.alive = true;
            P.alive = Q.alive = false;
            P.col.clear();
            Q.col.clear();
            merge_scores[mi] = score;
            merge_widths[mi] = (int32_t)len;
        }
        if (nb == 0) {
            widths[b] = 0;
            return;
        }
        const Cluster& root = cl[2 * nb - 2];
        widths[b] = (int32_t)root.width;
        for (size_t t = 0; t < root.members.size(); t++) {
            const int64_t q = boff + root.members[t];
            for (size_t r = 0; r < root.col[t].size(); r++) colmap[pos_off[q] + r] = (int32_t)root.col[t][r];
        }
    });
    return bad ? -1 : 0;
}

/* Realignment against the global ancestor and the glue, the last steps of
 * Algorithm Sample-Align-D (Section 2.3.3: every processor's aligned sequences
 * are aligned with the ancestor's profile, and the aligned sets are joined
 * through it). Bucket b's alignment (widths[b] columns; colmap as written by
 * orc_progressive) is kept fixed and aligned, as a profile of its nb members,
 * with the ancestor sequence ga as a profile of one member by profile_align
 * (the bucket's columns are the rows). A bucket column matched to ancestor
 * position g is anchored at g (anchors[...] = g); one against a gap in the
 * ancestor is an insertion in slot s, s being the number of ancestor positions
 * before it (anchors[...] = -(s + 1)); anchors holds bucket b's columns at
 * offset widths[0] + ... + widths[b - 1]. The joined alignment has, for s = 0,
 * 1, ..., |ga|, the insertions of slot s (bucket by bucket in bucket order,
 * inside a bucket in column order) followed by the anchor column of ancestor
 * position s (for s < |ga|), shared by every bucket column anchored there;
 * columns holding no residue are then dropped. Outputs: ga_scores[b] (the
 * optimum of bucket b's alignment with the ancestor; 0 for an empty bucket),
 * *global_width, global_colmap (the joined column of every residue, in the
 * layout of colmap). Returns 0, or -1 on invalid arguments. */
int orc_ancestor_glue(const uint8_t* res, const int64_t* offs, int32_t n, const int32_t* bucket_offsets,
                      const int32_t* order, int32_t p, const int32_t* widths, const int32_t* colmap, int32_t ga,
                      const int8_t* S, int32_t alphabet, int32_t go, int32_t ge, int32_t nthreads,
                      int64_t* ga_scores, int32_t* anchors, int32_t* global_width, int32_t* global_colmap) {
    if (p < 1 || n < 1 || ga < 0 || ga >= n) return -1;
    const int32_t npos = bucket_offsets[p];
    std::vector<int64_t> pos_off((size_t)npos + 1, 0), col_off((size_t)p + 1, 0);
    for (int32_t q = 0; q < npos; q++) {
        if (order[q] < 0 || order[q] >= n) return -1;
        pos_off[q + 1] = pos_off[q] + (offs[order[q] + 1] - offs[order[q]]);
    }
    for (int32_t b = 0; b < p; b++) col_off[b + 1] = col_off[b] + widths[b];
    for (int32_t b = 0; b < p; b++)
        for (int32_t q = bucket_offsets[b]; q < bucket_offsets[b + 1]; q++)
            for (int64_t t = pos_off[q]; t < pos_off[q + 1]; t++)
                if (colmap[t] < 0 || colmap[t] >= widths[b]) return -1;
    const int64_t lg = offs[ga + 1] - offs[ga];
    std::vector<int64_t> cg((size_t)lg * alphabet, 0);  // the ancestor as a profile of one member
    for (int64_t r = 0; r < lg; r++) cg[r * alphabet + res[offs[ga] + r]] = 1;
    std::atomic<int> bad(0);
    parallel_for(p, nthreads, [&](int64_t b) {
        const int64_t nb = bucket_offsets[b + 1] - bucket_offsets[b], w = widths[b];
        ga_scores[b] = 0;
        if (nb == 0) return;
        std::vector<int64_t> cp((size_t)w * alphabet, 0);  // the bucket's profile from its alignment
        for (int32_t q = bucket_offsets[b]; q < bucket_offsets[b + 1]; q++) {
            const uint8_t* x = res + offs[order[q]];
            for (int64_t t = pos_off[q]; t < pos_off[q + 1]; t++) cp[(int64_t)colmap[t] * alphabet + x[t - pos_off[q]]]++;
        }
        int64_t score = 0;
        std::string cols;
        if (!profile_align(cp, nb, w, cg, 1, lg, S, alphabet, go, ge, &score, &cols)) {
            bad = 1;
            return;
        }
        ga_scores[b] = score;
        int64_t c = 0, g = 0;
        for (char op : cols) {
            if (op == 'M') anchors[col_off[b] + c++] = (int32_t)g++;
            else if (op == 'X') anchors[col_off[b] + c++] = -(int32_t)(g + 1);
            else g++;
        }
    });
    if (bad) return -1;
    // the joined layout: per slot s the insertions of every bucket, then anchor s
    std::vector<int64_t> ins((size_t)(lg + 1) * p, 0);
    for (int32_t b = 0; b < p; b++)
        for (int64_t c = 0; c < widths[b]; c++) {
            const int32_t a = anchors[col_off[b] + c];
            if (a < 0) ins[(int64_t)(-a - 1) * p + b]++;
        }
    std::vector<int64_t> start((size_t)(lg + 1) * p, 0), anchor_col((size_t)lg, 0);
    int64_t col = 0;
    for (int64_t sl = 0; sl <= lg; sl++) {
        for (int32_t b = 0; b < p; b++) {
            start[sl * p + b] = col;
            col += ins[sl * p + b];
        }
        if (sl < lg) anchor_col[sl] = col++;
    }
    // each bucket column's joined column (insertions of a slot are consecutive in a bucket)
    std::vector<int64_t> joined((size_t)col_off[p], 0);
    for (int32_t b = 0; b < p; b++) {
        std::vector<int64_t> rank((size_t)lg + 1, 0);
        for (int64_t c = 0; c < widths[b]; c++) {
            const int32_t a = anchors[col_off[b] + c];
            joined[col_off[b] + c] = a >= 0 ? anchor_col[a] : start[(int64_t)(-a - 1) * p + b] + rank[-a - 1]++;
        }
    }
    // drop the columns that hold no residue
    std::vector<int64_t> used((size_t)col + 1, 0);
    for (int32_t b = 0; b < p; b++)
        for (int32_t q = bucket_offsets[b]; q < bucket_offsets[b + 1]; q++)
            for (int64_t t = pos_off[q]; t < pos_off[q + 1]; t++) used[joined[col_off[b] + colmap[t]]] = 1;
    std::vector<int64_t> renum((size_t)col + 1, 0);
    int64_t kept = 0;
    for (int64_t x = 0; x < col; x++) {
        renum[x] = kept;
        kept += used[x];
    }
    *global_width = (int32_t)kept;
    for (int32_t b = 0; b < p; b++)
        for (int32_t q = bucket_offsets[b]; q < bucket_offsets[b + 1]; q++)
            for (int64_t t = pos_off[q]; t < pos_off[q + 1]; t++)
                global_colmap[t] = (int32_t)renum[joined[col_off[b] + colmap[t]]];
    return 0;
}

}  // extern "C"
