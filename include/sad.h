/*
 * sad.h -- C ABI of the GB300-native Sample-Align-D data-parallel core.
 *
 * Two stages of the method (Saeed & Khokhar, "Sample-Align-D"):
 *   1. k-mer-rank partitioning (Section 2 "k-mer Rank", the algorithm box,
 *      Section 2.3.2 "Redistribution Based on k-mer Rank"):
 *        sad_kmer_rank   counts, all-pairs k-mer similarity, local and global
 *                        ancestors, rank keys against the global ancestor
 *                        and, optionally, the globalized rank against the
 *                        sample sets of all blocks (Section 2.3.1)
 *        sad_partition   regular-sampling splitters and p buckets
 *                        (sad_partition_keys64 for the globalized rank)
 *   2. per-bucket alignment (algorithm box "align sequences in each processor
 *      using any sequential multiple alignment system", Section 2.3.3):
 *        sad_bucket_pair_scores  all-pairs global affine-gap (Gotoh) scores
 *                                inside every bucket
 *        sad_align_pairs         the alignments themselves (traceback) of
 *                                given pairs
 *        sad_guide_trees         average-linkage guide tree of every bucket
 *                                from its pair scores
 *        sad_progressive_align   one multiple alignment per bucket, profile
 *                                against profile along its guide tree
 *        sad_ancestor_glue       every bucket realigned against the global
 *                                ancestor and all joined through its positions
 * plus sad_pipeline (both stages in one call) and a continuous-batching
 * serving loop (sad_server_*).
 *
 * Conventions shared by every call
 *   - Status: 0 (SAD_OK) or a negative SAD_E* code; sad_last_error() gives a
 *     message for the calling thread's last failure.
 *   - Memory: each call takes `mem`. With SAD_MEM_DEVICE every data array
 *     argument (sequences, offsets, keys, buckets, outputs) is a device
 *     pointer on the current device; with SAD_MEM_HOST every one is a host
 *     pointer, the library stages it through device memory and the call
 *     returns after the results are back in host memory. Parameter tables
 *     (substitution matrix, class map) are always host pointers.
 *   - The caller owns every argument buffer. The library allocates only its
 *     own workspaces, which a sad_ctx caches (grow-only) between calls.
 *   - `ctx` may be NULL: a default context per device is used. One context
 *     must not be used by two calls at the same time.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Device-mode
 *     calls enqueue their kernels on it; calls that must plan on the host
 *     (sad_bucket_pair_scores, sad_pipeline) synchronise it once to read the
 *     bucket layout.
 *   - Nothing here falls back to the CPU: without a usable sm_103 GPU every
 *     compute call fails with SAD_ECUDA.
 */
#ifndef SAD_H
#define SAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SAD_OK 0
#define SAD_EINVAL (-1)    /* invalid argument (message in sad_last_error) */
#define SAD_ENOMEM (-2)    /* device or host allocation failed */
#define SAD_ECUDA (-3)     /* a CUDA runtime call or kernel failed */
#define SAD_ETIMEOUT (-4)  /* a bounded device-side wait gave up */
#define SAD_EBUSY (-5)     /* serving: no slot or memory for the job now */
#define SAD_ERANGE (-6)    /* an output buffer is too small; the size is reported */
#define SAD_ENOTFOUND (-7) /* serving: unknown job id */
#define SAD_ECANCELED (-8) /* serving: the job was cancelled */

#define SAD_MEM_HOST 0
#define SAD_MEM_DEVICE 1

/* Limits of this build (checked; violating one gives SAD_EINVAL). */
#define SAD_MAX_ALPHABET 32     /* residue codes 0..alphabet-1 */
#define SAD_MAX_KMER_SPACE 49152 /* kmer_alphabet^k on the dense count-row paths */
#define SAD_MAX_SPARSE_KMER_SPACE 2147483647 /* kmer_alphabet^k on the sorted-list path */
#define SAD_MAX_SPARSE_KMERS 8192 /* |x| - k + 1 of any sequence on the sorted-list path */

typedef struct sad_ctx sad_ctx;

/* A set of n sequences: residues[offsets[i] .. offsets[i+1]) is sequence i.
 * offsets has n+1 nondecreasing entries with offsets[0] = 0; every residue
 * is a code < alphabet ("N sequences of amino acids x1..xN", algorithm box
 * input). Both arrays live where the call's `mem` says. */
typedef struct sad_seqset {
    const uint8_t* residues;
    const int64_t* offsets;
    int32_t n;
    int32_t alphabet; /* 1..SAD_MAX_ALPHABET */
} sad_seqset;

/* k-mer parameters (Section 2: "a k-mer is a contiguous subsequence of length
 * k"). Residue r is counted as letter class_map[r] of a kmer_alphabet-letter
 * alphabet (class_map NULL: identity, kmer_alphabet = alphabet).
 *   cap = 0: all-pairs similarity on saturating uint8 count vectors (the
 *            plain CUDA-core path; exact for any count via a residual pass).
 *   cap > 0: the same similarity as threshold planes,
 *            min(c, c') = sum_{t=1..cap} [c >= t][c' >= t] + residual above
 *            cap, contracted on the tensor cores; exact for any count. */
typedef struct sad_kmer_params {
    int32_t k;               /* >= 1 */
    int32_t kmer_alphabet;   /* >= 1; kmer_alphabet^k <= SAD_MAX_KMER_SPACE, or
                              * SAD_MAX_SPARSE_KMER_SPACE on the sorted-list path */
    const uint8_t* class_map; /* host, `alphabet` entries, or NULL */
    int32_t cap;             /* k-mer similarity path:
                              *   0      uint8 count rows, CUDA cores (the sorted-list
                              *          path when kmer_alphabet^k > SAD_MAX_KMER_SPACE)
                              *   1..8   threshold planes [count >= t], t <= cap, on the
                              *          tensor cores, counts above cap by a residual
                              *   SAD_KMER_SPARSE  sorted (k-mer, count) lists per
                              *          sequence, work proportional to the distinct
                              *          k-mers (any kmer_alphabet^k up to
                              *          SAD_MAX_SPARSE_KMER_SPACE; every sequence at
                              *          most SAD_MAX_SPARSE_KMERS k-mers)
                              * every path gives identical results */
    int32_t p;               /* number of blocks / buckets, >= 1 */
    int32_t global_samples;  /* 0, or s in 1..SAD_MAX_GLOBAL_SAMPLES: also compute the
                              * globalized rank G against s samples per block
                              * (sad_rank_out.G); sad_pipeline then partitions by G */
} sad_kmer_params;

#define SAD_KMER_SPARSE (-1)

#define SAD_MAX_GLOBAL_SAMPLES 1024

/* Outputs of sad_kmer_rank (caller-owned, in `mem` space).
 * With b_ij = min(|x_i|,|x_j|) - k + 1 and a_ij = sum_tau min(n_xi(tau), n_xj(tau))
 * (Section 2, r_ij = a_ij / b_ij; a term with b_ij <= 0 counts as 0):
 *   dloc[n]  sum over j in block(i) of floor(a_ij * 2^32 / b_ij), blocks
 *            [floor(bN/p), floor((b+1)N/p)) ("N/p sequences on each of the
 *            p processors"); the fixed-point form of the local D_i (the 1/N
 *            factor of D_i is dropped, it never changes an order)
 *   dcen[n]  the same sum over all j (the centralised D_i)
 *   la[p]    local ancestor of each block: argmax dloc in the block, lowest
 *            index on ties; -1 for an empty block
 *   ga[1]    global ancestor: the local ancestor with the largest fixed-point
 *            similarity sum to all local ancestors (lowest index on ties)
 *   key_a[n], key_b[n]  rank key of sequence i: a(i, GA) and b(i, GA);
 *            (0, 1) when b(i, GA) <= 0. The k-mer rank R_i = log(0.1 + D)
 *            of Section 2 is monotone, so sequences are ordered by
 *            key_a/key_b (compared by 64-bit cross-multiplication), then by
 *            index.
 *   A        NULL, or n*n int32 row-major receiving a_ij.
 * With params->global_samples = s >= 1, the globalized rank of Section 2.3.1
 * (each processor sends a sample set of s sequences to all others, and every
 * sequence is ranked against all s*p samples):
 *   sample_idx[p*s]  the samples of block b at [b*s, (b+1)*s): the block is
 *            ordered by (dloc, index) ascending and sample j (j = 0..s-1) is
 *            its member at 0-based position floor((2j+1) w_b / (2s)), w_b the
 *            block size (evenly spaced strata; with w_b < s a member is taken
 *            more than once); -1 for every slot of an empty block
 *   G[n]     sum over the p*s sample slots sigma (a slot taken twice counts
 *            twice, -1 slots count 0) of floor(a_i,sigma 2^32 / b_i,sigma);
 *            below 2^52. Sorted ascending with ties by index it gives the
 *            globalized order (sad_partition_keys64).
 * Both may be NULL when global_samples = 0. */
typedef struct sad_rank_out {
    uint64_t* dloc;
    uint64_t* dcen;
    int32_t* la;
    int32_t* ga;
    int32_t* key_a;
    int32_t* key_b;
    int32_t* A;
    uint64_t* G;
    int32_t* sample_idx;
} sad_rank_out;

/* ---- context ---------------------------------------------------------- */

/* Create a context bound to CUDA device `device`; it owns cached device
 * workspaces. Returns SAD_OK and *out, or an error. */
int sad_ctx_create(int32_t device, sad_ctx** out);
/* Free a context and its workspaces (synchronises its device). */
int sad_ctx_destroy(sad_ctx* ctx);

/* Thread-local message for the last failure of this thread ("" if none). */
const char* sad_last_error(void);
/* Library version string. */
const char* sad_version(void);

/* ---- tracing ------------------------------------------------------------ */

/* Stages whose device time the tracer records (CUDA events on the call's
 * stream around the stage's kernels). */
#define SAD_STAGE_PREPARE 0    /* staging and padding of the sequences */
#define SAD_STAGE_COUNT 1      /* k-mer counts, planes, excess lists, residual matrix */
#define SAD_STAGE_ALLPAIRS 2   /* all-pairs similarity with the fused D sums */
#define SAD_STAGE_RANK 3       /* ancestors and rank keys */
#define SAD_STAGE_PARTITION 4  /* regular-sampling partition */
#define SAD_STAGE_SCORES 5     /* alignment-score kernels, 32-bit DP */
#define SAD_STAGE_SCORES_PACKED 6 /* alignment-score kernels, two problems per 16x2 lane */
#define SAD_STAGE_GLOBAL 7     /* globalized rank: sample selection and sums against the samples */
#define SAD_STAGE_ALIGN 8      /* alignments with traceback (sad_align_pairs) */
#define SAD_STAGE_TREE 9       /* guide trees (sad_guide_trees) */
#define SAD_STAGE_PROG 10      /* progressive alignment (sad_progressive_align) */
#define SAD_STAGE_PLANE_GEMM 11 /* the threshold-plane GEMM launch alone (inside SAD_STAGE_ALLPAIRS) */
#define SAD_NUM_STAGES 12

/* Turn event tracing of `ctx` on (1) or off (0); turning it on clears the
 * accumulated times. */
int sad_trace_enable(sad_ctx* ctx, int32_t on);
/* Wait for the recorded events, then write per stage the accumulated device
 * milliseconds (ms[s]) and the number of traced intervals (counts[s]) for
 * s < nstages, and clear them. */
int sad_trace_read(sad_ctx* ctx, double* ms, int32_t* counts, int32_t nstages);
/* The intervals that the last sad_trace_read consumed, in start order: for
 * entry t its stage (stage[t]) and its device start and end (t0_ms[t],
 * t1_ms[t]) in milliseconds after the start of the first of them. Gaps between
 * consecutive intervals of one call are device idle time (host work between
 * launches, host synchronisation). Writes min(n, max_entries) entries and sets
 * *n_entries = n. Host arrays, caller-owned. */
int sad_trace_timeline(sad_ctx* ctx, int32_t* stage, double* t0_ms, double* t1_ms, int32_t max_entries,
                       int32_t* n_entries);
/* Number of kernels this library has launched in this process. */
uint64_t sad_launch_count(void);

/* Tensor-core work of the last threshold-plane GEMM that ctx ran (cap > 0):
 * *mma_flops = 2 x 128 x 128 x (k-blocks x tile width) of the MMAs issued, and
 * *dense_flops the same over every k-block of every tile. A tile skips the
 * 128-byte k-blocks that are zero in all rows of its row or of its column
 * panel (the planes of counts >= 3 are mostly zero); they add nothing, so the
 * result is the same. Synchronises the device; host outputs. */
int sad_kmer_gemm_work(sad_ctx* ctx, int64_t* mma_flops, int64_t* dense_flops);

/* ---- pipe probe ---------------------------------------------------------- */

/* Instruction mixes of sad_probe_alu. */
#define SAD_PROBE_VIADDMAX_S32 0   /* __viaddmax_s32 alone */
#define SAD_PROBE_VIMAX3_S32 1     /* __vimax3_s32 alone */
#define SAD_PROBE_VIADDMAX_S16X2 2 /* __viaddmax_s16x2 alone */
#define SAD_PROBE_VIMAX3_S16X2 3   /* __vimax3_s16x2 alone */
#define SAD_PROBE_IADD 4           /* plain 32-bit adds alone */
#define SAD_PROBE_ROW_DPX3_ADD2 5  /* one packed DP row: 2 add-max, 1 3-way max, 2 adds */
#define SAD_PROBE_ROW_DPX5 6       /* the same row with both adds as add-max against -inf */
#define SAD_PROBE_ROW_DPX3 7       /* the row's 3 DPX instructions without the adds */
#define SAD_PROBE_NUM_MIXES 8

/* Register-only throughput of an integer instruction mix on the current
 * device. This is not a step of the paper's method: it measures the rate that
 * the alignment kernels' roofline is derived for (SMs x DPX lanes per clock x
 * clock). One CTA per SM with warps_per_sm warps (1..32), each thread running
 * 8 independent chains for iters x 16 steps; the SM-clock cycles of the median
 * CTA give *lanes_per_clk_sm (instructions x 32 lanes per warp instruction,
 * per clock per SM; for the row mixes the DPX instructions only) and, for the
 * row mixes, *rows_per_clk_sm (DP rows of two 16-bit problems per clock per
 * SM, else 0). Host outputs; synchronises the device; allocates two small
 * device buffers for the call. Errors: SAD_EINVAL (unknown mix, warps or iters
 * out of range, a NULL output), SAD_ENOMEM, SAD_ECUDA. */
int sad_probe_alu(int32_t mix, int32_t warps_per_sm, int32_t iters, double* lanes_per_clk_sm,
                  double* rows_per_clk_sm);

/* ---- stage 1: k-mer rank ----------------------------------------------- */

/* All-pairs k-mer similarity and the rank keys (Section 2 equations r_ij,
 * D_i, R_i; algorithm box steps "locally compute k-mer rank", local and
 * global ancestor). Errors: SAD_EINVAL for n < 0, alphabet out of range,
 * k < 1, p < 1, cap out of range, kmer space too large, a class_map entry
 * >= kmer_alphabet, bad offsets, or (detected on the device) a residue >=
 * alphabet; SAD_ENOMEM; SAD_ECUDA. On error the outputs are unspecified. */
int sad_kmer_rank(sad_ctx* ctx, const sad_seqset* seqs, const sad_kmer_params* params,
                  const sad_rank_out* out, int32_t mem, void* stream);

/* ---- stage 1: partition ------------------------------------------------- */

/* Regular-sampling redistribution by rank key (Section 2.3.2):
 * block b = [floor(bN/p), floor((b+1)N/p)) is sorted by key; p-1 samples are
 * taken at 0-based positions floor(j*w_b/p), j = 1..p-1 of every non-empty
 * block; the q(p-1) samples (q = non-empty blocks) are sorted into Y; pivot m
 * (m = 1..p-1) is Y at 1-based position (m-1)q + max(1, floor(q/2)), which is
 * (m-1)p + floor(p/2) whenever N >= p; sequence i goes to bucket
 * #{pivots strictly below key_i}.
 * Inputs key_a[n], key_b[n] (0 <= key_a <= key_b, key_b >= 1).
 * Outputs: bucket_offsets[p+1] (CSR), order[n] (members of each bucket in
 * ascending index), pivot_idx[p-1] (sequence index of each pivot; may be
 * NULL). Errors: SAD_EINVAL (n < 0, p < 1, p > 1024, a bad key), SAD_ECUDA. */
int sad_partition(sad_ctx* ctx, int32_t n, const int32_t* key_a, const int32_t* key_b,
                  int32_t p, int32_t* bucket_offsets, int32_t* order, int32_t* pivot_idx,
                  int32_t mem, void* stream);

/* The same regular-sampling partition on unsigned 64-bit integer rank keys
 * (the globalized rank G of sad_rank_out), ascending, ties by index.
 * keys[n], bucket_offsets[p+1], order[n], pivot_idx[p-1] (nullable) in `mem`
 * space. Errors: SAD_EINVAL (n < 0, p outside 1..1024, a NULL pointer),
 * SAD_ECUDA. */
int sad_partition_keys64(sad_ctx* ctx, int32_t n, const uint64_t* keys, int32_t p,
                         int32_t* bucket_offsets, int32_t* order, int32_t* pivot_idx,
                         int32_t mem, void* stream);

/* ---- stage 1: partition without any allocation ------------------------- */

#define SAD_NOALLOC_MAX_N 262144 /* keys per call of sad_partition_noalloc */
#define SAD_NOALLOC_MAX_P 256    /* buckets per call of sad_partition_noalloc */

/* The same partition as sad_partition, for callers that cannot call
 * cudaMalloc: code that runs where a device allocation is forbidden or would
 * stall other work (a real-time or latency-critical loop, a host callback,
 * an embedding whose device memory is owned and capped by another framework).
 * The paper has no counterpart; this is an interface for those callers.
 * It allocates nothing: no device memory, no pinned or heap host memory, no
 * context. Its scratch is one fixed array in device memory of about 5 MiB,
 * which every GPU that loads the library holds until the process exits.
 * The array belongs to the library's device code, and CUDA reserves it when it
 * loads that code on a device: with lazy module loading (CUDA's default) that
 * is the first call of this function on the device, or an earlier call of
 * sad_partition or sad_partition_keys64, which share that code. A caller that
 * may never allocate should therefore make one warm-up call at set-up; later
 * calls leave the device's free memory unchanged.
 *   key_a, key_b [n], bucket_offsets [p+1], order [n], pivot_idx [p-1]
 *   (nullable): device pointers on the current device, same meaning as in
 *   sad_partition; n <= SAD_NOALLOC_MAX_N and 1 <= p <= SAD_NOALLOC_MAX_P,
 *   otherwise SAD_EINVAL before any device work.
 * The first call on a device looks up the array's device address (again after
 * a device reset, which gives the device a new context and a new copy of the
 * array); make that first call before any stream capture. Every call reuses
 * the same array, and each call clears the parts that must start at zero; two
 * calls that overlap on the GPU (other threads or streams at the same time)
 * race and give wrong results, so serialise them. The call synchronises `stream` to report bad
 * keys (SAD_EINVAL), like sad_partition. */
int sad_partition_noalloc(int32_t n, const int32_t* key_a, const int32_t* key_b, int32_t p,
                          int32_t* bucket_offsets, int32_t* order, int32_t* pivot_idx,
                          void* stream);

/* ---- stage 2: per-bucket all-pairs alignment scores -------------------- */

/* Number of scores for a bucket layout: sum_b n_b (n_b + 1) / 2, where
 * n_b = bucket_offsets[b+1] - bucket_offsets[b]; bucket_offsets is in `mem`
 * space. Returns SAD_OK and *total. */
int sad_scores_size(const int32_t* bucket_offsets, int32_t p, int32_t mem, int64_t* total);

#define SAD_SCORES_PER_BUCKET 0  /* one kernel launch per bucket, 32-bit DP */
#define SAD_SCORES_PERSISTENT 1  /* one persistent launch over a length-binned
                                    queue of every bucket, CUDA-graph replayed;
                                    two problems per 16x2 lane when a bias fits */
#define SAD_SCORES_PERSISTENT_32 2 /* the batched form in 32-bit DP: one
                                      persistent launch over every bucket's
                                      query rows, longest first */

/* Global alignment score with affine gaps for every pair u <= v inside every
 * bucket (the diagonal is the self-score). A gap run of length g scores
 * gap_open + g * gap_extend (gap_open, gap_extend <= 0, written as negative
 * numbers, e.g. -11 and -1); end gaps score like internal ones; a gap in x
 * may directly follow a gap in y, each run with its own opening.
 * subst: host, alphabet x alphabet int8, row-major, symmetric.
 * Layout: bucket b's members are order[bucket_offsets[b] .. bucket_offsets[b+1]);
 * score_offsets[p+1] (written) holds each bucket's start in `scores`; the pair
 * of local positions (u, v), u <= v, of bucket b with n_b members is at
 * scores[score_offsets[b] + u*n_b - u*(u-1)/2 + (v-u)].
 * scores_capacity is the length of `scores`; if it is smaller than the total,
 * nothing is computed, score_offsets is still written and SAD_ERANGE returned.
 * Errors: SAD_EINVAL (bad layout or order, asymmetric subst, positive gap
 * costs, unknown mode), SAD_ERANGE, SAD_ENOMEM, SAD_ECUDA. */
int sad_bucket_pair_scores(sad_ctx* ctx, const sad_seqset* seqs, const int32_t* bucket_offsets,
                           const int32_t* order, int32_t p, const int8_t* subst,
                           int32_t gap_open, int32_t gap_extend, int32_t mode,
                           int64_t* score_offsets, int32_t* scores, int64_t scores_capacity,
                           int32_t mem, void* stream);

/* Variant table of the packed alignment kernel (SAD_SCORES_PERSISTENT mode
 * when every score provably fits 16 bits). The pair of queries at length-order
 * positions 2q, 2q+1 of a bucket with `rows` = the longer length uses the first
 * bin b with rows <= upper[b]: R[b] query rows per lane (8, 12, 16, 20, 24 or
 * 32) and G[b] lanes per subject (8, 16 or 32); rows beyond every bin use the
 * built-in cost model. With an empty table (nbins = 0, the default) each pair
 * takes the variant of least padding whose one strip of G x R rows holds it
 * (the smallest G R >= rows; then R <= 24; then G nearest 16), and only pairs
 * longer than every strip use the cost model. Bounds must increase; at most 16
 * bins. The table only changes speed, never a score.
 * get: copies up to max_bins entries and the bin count. */
int sad_scores_set_variants(sad_ctx* ctx, const int32_t* upper, const int32_t* R, const int32_t* G,
                            int32_t nbins);
int sad_scores_get_variants(sad_ctx* ctx, int32_t* upper, int32_t* R, int32_t* G, int32_t max_bins,
                            int32_t* nbins);

/* Autotuner: on the caller's own sequences and bucket layout (arguments as
 * sad_bucket_pair_scores), time every packed-kernel variant on the query
 * pairs of each length bin (rows in (bin_upper[b-1], bin_upper[b]]), `reps`
 * times after one warm-up run, with CUDA events on `stream`, and store the
 * fastest variant of every non-empty bin. The variants of different bins run
 * side by side, so it then times whole score stages (each a full
 * sad_bucket_pair_scores call on these arguments, into buffers of its own; the
 * mean of at least seven runs): it starts from the better of that per-bin table
 * and the least-padding table (see sad_scores_set_variants), changes one bin at
 * a time while that gains 0.5 % twice, and keeps the result only if it still
 * beats its start. The table ends in ctx's variant table (read it with
 * sad_scores_get_variants; save and restore it with set). A variant that
 * cannot hold some pair of a bin in shared memory is not eligible for that
 * bin. Synchronises `stream`. SAD_EINVAL when the inputs need the 32-bit
 * kernel (nothing to tune). */
int sad_scores_autotune(sad_ctx* ctx, const sad_seqset* seqs, const int32_t* bucket_offsets,
                        const int32_t* order, int32_t p, const int8_t* subst, int32_t gap_open,
                        int32_t gap_extend, const int32_t* bin_upper, int32_t nbins, int32_t reps,
                        int32_t mem, void* stream);

/* ---- guide trees ------------------------------------------------------------ */

/* Average-linkage (UPGMA) guide tree of every bucket from its pair scores: the
 * first step of the progressive multiple aligner that each processor runs on
 * its bucket (Section 2.3.3 lets it be any sequential aligner). Inside bucket b
 * (nb members, local positions 0..nb-1 as in sad_bucket_pair_scores) the
 * distance of u and v is d_uv = S_uu + S_vv - 2 S_uv; two clusters are at
 * W / (|A| |B|), W the sum of d over their member pairs; the closest pair is
 * joined first (exact rational comparison), ties to the smallest pair of
 * cluster ids (lower id, then higher id); merge k creates cluster nb + k.
 * Inputs: bucket_offsets[p+1], score_offsets[p+1] and scores as written by
 * sad_bucket_pair_scores. Outputs (caller-owned, `mem` space):
 * merge_offsets[p+1] (filled: bucket b's merges are [merge_offsets[b],
 * merge_offsets[b+1]), nb - 1 of them for nb >= 1), and per merge m: left[m] <
 * right[m] (cluster ids joined), num[m] and den[m] (their distance num / den;
 * den = |A| |B|). M = sum over buckets of max(nb - 1, 0) = n minus the number of
 * non-empty buckets. Errors: SAD_EINVAL (offsets that do not describe upper
 * triangles, a bucket above 2^20 members), SAD_ENOMEM (the buckets' nb x nb
 * cluster matrices above 12 GiB), SAD_ECUDA. */
int sad_guide_trees(sad_ctx* ctx, const int32_t* bucket_offsets, int32_t p, const int64_t* score_offsets,
                    const int32_t* scores, int64_t* merge_offsets, int32_t* left, int32_t* right, int64_t* num,
                    int64_t* den, int32_t mem, void* stream);

/* Progressive alignment of every bucket along its guide tree (the
 * per-processor multiple aligner of Section 2.3.3; the paper allows any
 * sequential one). Inputs: the buckets (bucket_offsets[p+1], order[npos],
 * npos = bucket_offsets[p], positions of sequence ids of seqs, as
 * sad_partition writes them) and their trees (merge_offsets[p+1],
 * left/right[M], as sad_guide_trees writes them: merge k of bucket b joins
 * clusters left < right into nb + k; leaves are the bucket positions 0..nb-1).
 * Merge k aligns the multiple alignment of cluster left[k] (profile P, nP
 * members) with that of right[k] (profile Q, nQ members), both kept fixed, by
 * the global affine-gap recursion of sad_align_pairs in which pairing a column
 * of P with a column of Q scores the sum of subst over the letter pairs across
 * them (a gap already in a column pairs with nothing) and a new run of g gap
 * columns costs nP nQ (gap_open + g gap_extend). The optimal alignment is
 * taken with fixed ties: a cell's best state is match, then a gap in Q's
 * columns, then a gap in P's; a gap column extends its run before it opens
 * one and opens from a match before the other gap state. Outputs (caller-
 * owned, `mem` space): widths[p] (columns of bucket b's alignment; a
 * one-member bucket is its sequence, an empty one 0), merge_scores[M] (int64
 * optimum of each merge), merge_widths[M] (columns of each merged cluster),
 * colmap[sum of the lengths of order[0..npos)] (the column of every residue
 * in its bucket's alignment, over the residues of order[0], order[1], ... in
 * turn). Errors: SAD_EINVAL (layout or tree inconsistent, a bucket above
 * 65535 members, nP nQ max|subst| >= 2^31, an asymmetric subst, gap costs
 * > 0 or below -1000, a residue >= alphabet), SAD_ENOMEM, SAD_ECUDA. The host
 * reads the new widths back after every tree level (one synchronisation of
 * `stream` per level). */
int sad_progressive_align(sad_ctx* ctx, const sad_seqset* seqs, const int32_t* bucket_offsets,
                          const int32_t* order, int32_t p, const int64_t* merge_offsets, const int32_t* left,
                          const int32_t* right, const int8_t* subst, int32_t gap_open, int32_t gap_extend,
                          int32_t* widths, int64_t* merge_scores, int32_t* merge_widths, int32_t* colmap,
                          int32_t mem, void* stream);

/* Tuning of the profile DP of sad_progressive_align and sad_ancestor_glue:
 * columns = 1 or 2 subject columns per DP lane step for every batch, 0 (the
 * default) lets each batch choose (two when it holds at least one merge per
 * SM or a profile of 1024 columns or more). Results do not depend on it.
 * Errors: SAD_EINVAL for other values. */
int sad_progressive_columns(sad_ctx* ctx, int32_t columns);

/* Bound of the one device-side wait of the profile DP (sad_progressive_align,
 * sad_ancestor_glue): a warp that aligns a strip of rows waits for the strip
 * above to finish each column it needs, polling every 32 ns at most `polls`
 * times. A wait that runs out sets the context's status, the kernel goes on
 * with whatever the boundary holds (every access stays in bounds) and the call
 * returns SAD_ETIMEOUT; the context stays usable. polls = 0 restores the
 * default bound (2^22 polls, about 0.15 s of waiting per column); a small bound
 * makes a multi-strip merge give up, which is how the timeout path is tested.
 * Errors: SAD_EINVAL for polls < 0. */
int sad_progressive_wait_limit(sad_ctx* ctx, int64_t polls);

/* Realignment against the global ancestor and the glue, the last steps of
 * Algorithm Sample-Align-D (Section 2.3.3): the alignment of every bucket
 * (widths[p] and colmap as sad_progressive_align writes them, over the
 * residues of order[0..npos) in turn) is kept fixed and aligned, as a profile
 * of its members (rows), with sequence ga as a profile of one member
 * (columns), by the recursion and tie order of sad_progressive_align. A bucket
 * column matched to position g of ga is anchored there (anchors[...] = g), one
 * against a gap in ga is an insertion of slot s, s being the number of ga's
 * positions before it (anchors[...] = -(s + 1)); bucket b's columns sit at
 * offset widths[0] + ... + widths[b-1] of anchors. The joined alignment holds,
 * for s = 0 .. |ga|, the insertions of slot s (bucket by bucket in bucket
 * order, inside a bucket in column order) and then the anchor column of
 * position s (s < |ga|), shared by every bucket column anchored there; columns
 * holding no residue are dropped. Outputs (caller-owned, `mem` space):
 * ga_scores[p] (int64 optimum of each bucket against ga; 0 for an empty
 * bucket), anchors[sum widths], *global_width, global_colmap (the joined
 * column of every residue, in the layout of colmap). Errors: SAD_EINVAL
 * (layout inconsistent, ga outside 0..n-1, a colmap entry outside its
 * bucket's width, a bucket above 65535 members, member products x max|subst|
 * >= 2^31, an asymmetric subst, gap costs > 0 or below -1000, a residue >=
 * alphabet), SAD_ENOMEM, SAD_ECUDA. */
int sad_ancestor_glue(sad_ctx* ctx, const sad_seqset* seqs, const int32_t* bucket_offsets, const int32_t* order,
                      int32_t p, const int32_t* widths, const int32_t* colmap, int32_t ga, const int8_t* subst,
                      int32_t gap_open, int32_t gap_extend, int64_t* ga_scores, int32_t* anchors,
                      int32_t* global_width, int32_t* global_colmap, int32_t mem, void* stream);

/* ---- alignments (traceback) ----------------------------------------------- */

/* Column codes of an alignment. */
#define SAD_COL_MATCH 'M'  /* x_i aligned with y_j */
#define SAD_COL_XGAP 'X'   /* x_i against a gap */
#define SAD_COL_YGAP 'Y'   /* a gap against y_j */

/* Optimal global affine-gap alignments (not only their scores) of the pairs
 * (x, y) = (pairs[2k], pairs[2k+1]), sequence ids of seqs; the same gap model
 * and score as sad_bucket_pair_scores (a run of g gap columns of one kind costs
 * gap_open + g * gap_extend). The per-processor aligner of Section 2.3.3 turns
 * pair scores into alignments; among equally good alignments any one may be
 * returned. Outputs (caller-owned, `mem` space): scores[npairs],
 * ops_offsets[npairs+1] (filled: pair k owns ops[ops_offsets[k] ..
 * ops_offsets[k] + |x| + |y|)), ops[ops_capacity] (pair k's columns, first
 * column first, SAD_COL_* bytes, at the start of its slot), ops_len[npairs]
 * (columns of pair k). The direction bits of every cell are kept: 4 bits per
 * cell, |x| |y| / 2 bytes per pair, pairs in batches whose bits fit 1 GiB
 * (sad_align_pairs_linear needs memory linear in the lengths). Errors:
 * SAD_EINVAL (a pair id outside 0..n-1, gap costs > 0 or below -1000, a
 * residue >= alphabet), SAD_ERANGE (ops_capacity below sum |x| + |y|;
 * ops_offsets is filled), SAD_ENOMEM, SAD_ECUDA. */
int sad_align_pairs(sad_ctx* ctx, const sad_seqset* seqs, const int32_t* pairs, int32_t npairs,
                    const int8_t* subst, int32_t gap_open, int32_t gap_extend, int32_t* scores,
                    int64_t* ops_offsets, uint8_t* ops, int64_t ops_capacity, int32_t* ops_len,
                    int32_t mem, void* stream);
/* The same alignments in linear space: memory per pair grows with the
 * length of the sequences, not with their product. Rows are split at the
 * middle (Hirschberg's divide and conquer with Myers and Miller's affine-gap
 * bookkeeping: the best crossing of the middle row is taken from a forward
 * pass over the top half and a pass over the reversed bottom half, with a
 * vertical gap allowed to span the cut at one opening), down to blocks of at
 * most 256 rows, which are solved with their direction bits. The shorter
 * sequence of a pair is taken as the rows. Arguments, outputs and errors as
 * sad_align_pairs; any optimal alignment may be returned (the two calls may
 * return different ones of the same score). The device scratch is
 * sad_align_linear_bytes_per_warp(L) bytes for each of up to 16 warps per SM,
 * L the longest sequence of the pairs; a pass sums two 32-bit DP values, so
 * (max|subst| + |gap_open| + |gap_extend|) x 2 x (L + 1) must stay below 2^28
 * (SAD_EINVAL otherwise). */
int sad_align_pairs_linear(sad_ctx* ctx, const sad_seqset* seqs, const int32_t* pairs, int32_t npairs,
                           const int8_t* subst, int32_t gap_open, int32_t gap_extend, int32_t* scores,
                           int64_t* ops_offsets, uint8_t* ops, int64_t ops_capacity, int32_t* ops_len,
                           int32_t mem, void* stream);
/* Device bytes one warp of sad_align_pairs_linear uses for pairs whose longer
 * sequence has max_len residues: 6 x (max_len + 2) int32 (the middle-row
 * vectors and a strip boundary) and (max_len + 34) x 32 direction words; -1
 * for max_len < 0. */
int64_t sad_align_linear_bytes_per_warp(int32_t max_len);

/* ---- both stages ------------------------------------------------------- */

/* sad_kmer_rank, sad_partition and sad_bucket_pair_scores in one call, with
 * every intermediate kept on the device. rank (may have NULL members: those
 * outputs are skipped), bucket_offsets[p+1], order[n], score_offsets[p+1],
 * scores[scores_capacity] are in `mem` space. SAD_ERANGE when the scores do
 * not fit (score_offsets then holds the layout). With
 * params->global_samples >= 1 the buckets come from the globalized rank G
 * (sad_partition_keys64) instead of the keys against the global ancestor. */
int sad_pipeline(sad_ctx* ctx, const sad_seqset* seqs, const sad_kmer_params* params,
                 const int8_t* subst, int32_t gap_open, int32_t gap_extend, int32_t mode,
                 const sad_rank_out* rank, int32_t* bucket_offsets, int32_t* order,
                 int64_t* score_offsets, int32_t* scores, int64_t scores_capacity,
                 int32_t mem, void* stream);

/* ---- serving: continuous batching of partition-and-score jobs ----------- */

/* A stream of jobs (each a full sad_pipeline: k-mer rank, partition, bucket
 * scores) of different sizes on one GPU. The server runs `slots` jobs at once,
 * each on its own stream with its own workspaces, so their kernels overlap on
 * the device; a queued job is admitted as soon as a slot is free and its
 * device-memory estimate fits in what the running jobs leave of `hbm_budget`
 * (the first queued job that fits goes first). Results stay in server-owned
 * host memory until released. Every result is bit-identical to the same job
 * run alone. The paper has no serving layer; this is the batching of its
 * per-processor work across independent requests. */
typedef struct sad_server sad_server;

typedef struct sad_server_config {
    int32_t device;          /* CUDA device */
    int32_t slots;           /* jobs in flight at once, 1..64 */
    int64_t hbm_budget;      /* bytes of device memory jobs may hold at once; 0 = 90% of free */
    int32_t queue_capacity;  /* queued jobs; submit returns SAD_EBUSY beyond it */
} sad_server_config;

/* One job; every array is host memory and is copied by sad_server_submit. */
typedef struct sad_job {
    const uint8_t* residues;
    const int64_t* offsets;  /* n+1 */
    int32_t n;
    int32_t alphabet;
    sad_kmer_params kmer;
    const int8_t* subst;     /* alphabet x alphabet, symmetric */
    int32_t gap_open;
    int32_t gap_extend;
} sad_job;

#define SAD_JOB_QUEUED 0
#define SAD_JOB_RUNNING 1
#define SAD_JOB_DONE 2
#define SAD_JOB_FAILED 3
#define SAD_JOB_CANCELLED 4

typedef struct sad_server_stats {
    int64_t done, failed, cancelled, queued;
    int32_t running;
    double p50_ms, p99_ms, mean_ms;  /* submit-to-done latency of finished jobs */
    double jobs_per_s;               /* finished jobs / (last finish - first submit) */
    int64_t budget_bytes, reserved_bytes;
} sad_server_stats;

/* Start the workers. Errors: SAD_EINVAL, SAD_ECUDA, SAD_ENOMEM. */
int sad_server_create(const sad_server_config* cfg, sad_server** out);
/* Validate and queue a job; *job_id identifies it. SAD_ENOMEM when the job's
 * estimate exceeds the whole budget, SAD_EBUSY when the queue is full,
 * SAD_EINVAL for bad parameters (bad residue codes surface later as the job's
 * own failure). */
int sad_server_submit(sad_server* s, const sad_job* job, uint64_t* job_id);
/* *state = SAD_JOB_*; returns the job's error code if it failed. */
int sad_server_poll(sad_server* s, uint64_t job_id, int32_t* state);
/* Wait until the job ends (timeout_ms < 0: no limit). SAD_OK when done,
 * SAD_EBUSY on timeout, SAD_ECANCELED, or the job's own error code. */
int sad_server_wait(sad_server* s, uint64_t job_id, int64_t timeout_ms);
/* Copy a finished job's bucket_offsets[p+1], order[n], score_offsets[p+1] and
 * scores (layout as sad_bucket_pair_scores); any output pointer may be NULL.
 * *n_scores receives the score count, *latency_ms (nullable) the job's
 * submit-to-done time. SAD_ERANGE if capacity < *n_scores. */
int sad_server_result(sad_server* s, uint64_t job_id, int32_t* bucket_offsets, int32_t* order,
                      int64_t* score_offsets, int32_t* scores, int64_t capacity, int64_t* n_scores,
                      double* latency_ms);
/* Forget a finished job and free its results. */
int sad_server_release(sad_server* s, uint64_t job_id);
/* Cancel: a queued job is dropped now; a running one stops between stages. */
int sad_server_cancel(sad_server* s, uint64_t job_id);
int sad_server_get_stats(sad_server* s, sad_server_stats* out);
/* Device interval of a finished job: *t0_ms and *t1_ms are the times, in ms
 * after the server was created, at which its first device operation started
 * and its last one ended on its worker's stream (CUDA events around the job).
 * Two jobs whose intervals intersect were on the device at the same time.
 * SAD_EBUSY for a job that is not done. */
int sad_server_job_span(sad_server* s, uint64_t job_id, double* t0_ms, double* t1_ms);
/* Stop the workers (running jobs finish, queued jobs are cancelled) and free
 * everything. */
int sad_server_destroy(sad_server* s);

#ifdef __cplusplus
}
#endif

#endif /* SAD_H */
