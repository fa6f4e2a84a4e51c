// Sorted-list k-mer similarity (Section 2, r_ij; the "w^2 L" cost the paper
// gives the k-mer rank step): each sequence becomes the list of its distinct
// k-mer codes with their counts, so the work per pair follows the number of
// distinct k-mers instead of the size A^k of the k-mer space. This path serves
// k-mer spaces too large for dense count rows (k = 4, 5 over 20 letters) and
// gives the same numerators a_ij = sum_tau min(n_xi(tau), n_xj(tau)) as the
// dense paths.
//
// Counting: one CTA per sequence computes every window's code into shared
// memory, sorts them (bitonic) and run-length encodes the sorted codes.
//
// All pairs: a CTA takes TI <= 8 "row" sequences and a range of columns, and
// each warp streams one column's list against the rows at a time. Two forms:
//  - k-mer spaces that fit shared memory as one byte per k-mer code (up to
//    about 2^17.7 codes, e.g. k = 4 over 20 letters): bit r of byte c says that
//    row r holds k-mer c. A lane reads the byte of each of its column entries
//    and adds its two 4-row halves, spread to one byte per row by a multiply
//    (((x & 15) * 0x00204081) & 0x01010101: the four 4-bit copies sit 7 bits
//    apart, so none overlaps), to per-lane byte counters: no probing, no
//    divergence. This counts sum_tau [c_i >= 1][c_j >= 1]; the rest of
//    min(c_i, c_j) is the residual of the counts above 1 (threshold 1).
//  - larger spaces: a shared-memory hash table keyed by k-mer code whose value
//    holds one byte per row (the count clamped to 255); a hit adds
//    min(row byte, column count) for all rows at once (two vminu4 on the packed
//    bytes); counts above 255 go to the residual (threshold 255).
// Both accumulate the rows' numerators as 16-bit halves, and counts above the
// threshold are exact through the residual matrix of the sequences whose lists
// hold such counts, as on the uint8 dense path. The epilogue is the exact
// fixed-point D-sum epilogue.
#include <algorithm>
#include <cstring>

#include "kmer_common.cuh"
#include "kmer_stage.cuh"
#include "sad_internal.cuh"

namespace sad {

namespace {

constexpr int kSortThreads = 1024;
constexpr uint32_t kEmpty = 0xffffffffu;
constexpr int kPairThreads = 256;
constexpr int kPairThreadsBytes = 1024;  // a byte table of most of an SM's shared memory: one CTA, 32 warps
constexpr int64_t kBigTable = 48 * 1024;  // byte tables above this size take the 1024-thread CTAs
constexpr int kRowsMax = 8;       // rows per CTA: one byte each in an 8-byte table value
constexpr int32_t kColChunkMin = kPairThreads / 32;  // one column per warp
constexpr int32_t kColChunkMax = 2048;

// Exclusive block-wide prefix of a per-thread flag; *total receives the sum.
__device__ __forceinline__ int32_t block_scan_flag(bool f, int32_t* warp_tot, int32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_tot[w] = __popc(bal);
    __syncthreads();
    int32_t before = 0, tot = 0;
    for (int q = 0; q < nw; q++) {
        const int32_t v = warp_tot[q];
        before += q < w ? v : 0;
        tot += v;
    }
    __syncthreads();
    *total = tot;
    return before + __popc(bal & ((1u << lane) - 1u));
}

// One CTA per sequence: sorted (code, count) list and excess entries above T.
__global__ void __launch_bounds__(kSortThreads)
k_sparse_count(const uint8_t* __restrict__ res, const int64_t* __restrict__ pad_off,
               const int32_t* __restrict__ len, int32_t k, int32_t A2, ClassMap cm, int32_t T,
               const int64_t* __restrict__ loff, uint2* __restrict__ lists, int32_t* __restrict__ nd,
               const int64_t* __restrict__ ex_off, int32_t* __restrict__ ex_tau,
               int32_t* __restrict__ ex_val, int32_t* __restrict__ nex) {
    extern __shared__ uint32_t codes[];
    __shared__ int32_t warp_tot[kSortThreads / 32];
    __shared__ uint8_t cls[SAD_MAX_ALPHABET];
    if (threadIdx.x < SAD_MAX_ALPHABET) cls[threadIdx.x] = cm.c[threadIdx.x];
    __syncthreads();
    const int32_t i = blockIdx.x;
    const int32_t nk = len[i] - k + 1;
    if (nk <= 0) {
        if (threadIdx.x == 0) {
            nd[i] = 0;
            nex[i] = 0;
        }
        return;
    }
    int32_t P = 1;
    while (P < nk) P <<= 1;
    const uint8_t* x = res + pad_off[i];
    for (int32_t t = threadIdx.x; t < P; t += blockDim.x) {
        uint32_t code = kEmpty;
        if (t < nk) {
            code = 0;
            for (int32_t q = 0; q < k; q++) code = code * (uint32_t)A2 + cls[x[t + q]];
        }
        codes[t] = code;
    }
    __syncthreads();
    // bitonic sort, ascending; the padding (kEmpty) ends up behind the codes
    for (int32_t size = 2; size <= P; size <<= 1)
        for (int32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (int32_t t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int32_t lo = 2 * t - (t & (stride - 1));
                const int32_t hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint32_t a = codes[lo], b = codes[hi];
                if ((a > b) == up) {
                    codes[lo] = b;
                    codes[hi] = a;
                }
            }
            __syncthreads();
        }
    // run-length encoding: the first element of every run writes (code, run length)
    const int64_t lo0 = loff[i], eo = ex_off[i];
    int32_t base = 0, base_h = 0;
    for (int32_t t0 = 0; t0 < nk; t0 += blockDim.x) {
        const int32_t t = t0 + threadIdx.x;
        const bool in = t < nk;
        const uint32_t c = in ? codes[t] : 0u;
        const bool st = in && (t == 0 || codes[t - 1] != c);
        int32_t cnt = 0;
        if (st) {
            cnt = 1;
            while (t + cnt < nk && codes[t + cnt] == c) cnt++;
        }
        int32_t tot = 0, tot_h = 0;
        const int32_t u = block_scan_flag(st, warp_tot, &tot);
        const bool heavy = st && cnt > T;
        const int32_t uh = block_scan_flag(heavy, warp_tot, &tot_h);
        if (st) lists[lo0 + base + u] = make_uint2(c, (uint32_t)cnt);
        if (heavy) {
            ex_tau[eo + base_h + uh] = (int32_t)c;
            ex_val[eo + base_h + uh] = cnt - T;
        }
        base += tot;
        base_h += tot_h;
    }
    if (threadIdx.x == 0) {
        nd[i] = base;
        nex[i] = base_h;
    }
}

__device__ __forceinline__ uint32_t hash_slot(uint32_t code, int log2S) {
    return (code * 0x9E3779B1u) >> (32 - log2S);
}

// Epilogues of the rows x columns kernel.
enum SparseMode : int {
    kDSums = 0,    // rows = columns = all sequences, pairs i <= j: D sums (and A)
    kGSums = 1,    // rows = sample slots: G_j += the slots' terms
    kKeys = 2,     // one row (the global ancestor): rank key of every column
    kRowSums = 3,  // rows = columns = the local ancestors: per-row sum of the terms
};

struct PairOut {
    uint64_t* dloc;
    uint64_t* dcen;
    int32_t* A;
    uint64_t* G;
    int32_t* key_a;
    int32_t* key_b;
    uint64_t* row_sums;
};

// Rows x columns through a per-CTA table of the rows' lists (kBytes: one byte
// per k-mer code, log2S unused and V the table's codes; else a hash table of
// 2^log2S slots). Rows are the row positions [blockIdx.x*TI, +TI) (sequence
// row_ids[pos], or pos itself when row_ids is NULL; -1 is an empty row); columns
// are the positions [blockIdx.y*cw, +cw) (sequence col_ids[pos] or pos; -1
// skipped). Each lane fetches four list entries before it looks them up, so
// four L2 loads are in flight.
template <int kMode, bool kBytes, int kThreads>
__global__ void __launch_bounds__(kThreads)
k_sparse_pairs(int32_t n, int32_t nrows, const int32_t* __restrict__ row_ids, int32_t ncols,
               const int32_t* __restrict__ col_ids, int32_t TI, int32_t cw, int32_t log2S, int32_t V,
               SparseLists L, SeqTables tab, PairOut out) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ unsigned long long rowc[kRowsMax], rowl[kRowsMax];
    const int32_t S = 1 << log2S;
    uint32_t* keys = sm;
    uint32_t* vals = sm + S;  // two words per slot: bytes of rows 0-3 and 4-7
    const uint8_t* pres = (const uint8_t*)sm;  // kBytes: bit r of byte c = row r holds k-mer c
    const int32_t r0 = blockIdx.x * TI;
    const int32_t jbeg = max(kMode == kDSums ? r0 : 0, (int32_t)blockIdx.y * cw);
    const int32_t jend = min(ncols, (int32_t)(blockIdx.y + 1) * cw);
    if (jbeg >= jend) return;  // whole CTA (uniform)
    if constexpr (kBytes) {
        const int32_t nw16 = (V + 15) / 16;
        for (int32_t t = threadIdx.x; t < nw16; t += blockDim.x) ((uint4*)sm)[t] = make_uint4(0u, 0u, 0u, 0u);
    } else {
        for (int32_t t = threadIdx.x; t < S; t += blockDim.x) {
            keys[t] = kEmpty;
            vals[2 * t] = 0;
            vals[2 * t + 1] = 0;
        }
    }
    if (threadIdx.x < kRowsMax) {
        rowc[threadIdx.x] = 0;
        rowl[threadIdx.x] = 0;
    }
    __syncthreads();
    // build
    for (int r = 0; r < TI && r0 + r < nrows; r++) {
        const int32_t q = row_ids ? row_ids[r0 + r] : r0 + r;
        if (q < 0) continue;
        const uint2* lq = L.lists + L.loff[q];
        const int32_t nq = L.nd[q];
        for (int32_t t = threadIdx.x; t < nq; t += blockDim.x) {
            const uint2 e = lq[t];
            if constexpr (kBytes) {
                atomicOr(&sm[e.x >> 2], 1u << (8 * (e.x & 3) + r));
            } else {
                uint32_t slot = hash_slot(e.x, log2S);
                for (int32_t probe = 0; probe < S; probe++) {
                    const uint32_t prev = atomicCAS(&keys[slot], kEmpty, e.x);
                    if (prev == kEmpty || prev == e.x) break;
                    slot = (slot + 1) & (uint32_t)(S - 1);
                }
                atomicOr(&vals[2 * slot + (r >> 2)], min(e.y, 255u) << (8 * (r & 3)));
            }
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // per-lane row constants (lane r < TI serves row r)
    int32_t my = -1;
    if (lane < TI && r0 + lane < nrows) my = row_ids ? row_ids[r0 + lane] : r0 + lane;
    const int32_t nki = my >= 0 ? tab.nkb[my] : 0;
    const uint64_t qi = my >= 0 ? tab.q32[my] : 0;
    const uint32_t ri = my >= 0 ? tab.r32[my] : 0;
    const int32_t bli = my >= 0 ? tab.blk[my] : -2;
    const int32_t hxi = my >= 0 ? tab.hidx[my] : -1;
    const float inv_i = my >= 0 ? tab.inv[my] : 0.0f;
    uint64_t rs_c = 0, rs_l = 0;
    for (int32_t jc = jbeg + warp; jc < jend; jc += nwarps) {
        const int32_t j = col_ids ? col_ids[jc] : jc;
        if (j < 0) continue;  // uniform in the warp
        const uint2* lj = L.lists + L.loff[j];
        const int32_t nj = L.nd[j];
        uint32_t acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
        if constexpr (kBytes) {
            // per-lane byte counters of rows 0-3 (lo) and 4-7 (hi); a lane adds at
            // most 4 per round and at most 63 rounds before folding: <= 252 per byte
            uint32_t lo = 0, hi = 0;
            int32_t rounds = 0;
            for (int32_t t0 = 0; t0 < nj; t0 += 4 * 32) {
                uint32_t code[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int32_t t = t0 + u * 32 + lane;
                    code[u] = t < nj ? lj[t].x : kEmpty;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const uint32_t b = code[u] != kEmpty ? (uint32_t)pres[code[u]] : 0u;
                    lo += ((b & 15u) * 0x00204081u) & 0x01010101u;
                    hi += ((b >> 4) * 0x00204081u) & 0x01010101u;
                }
                if (++rounds == 63) {
                    acc0 += lo & 0x00ff00ffu;
                    acc1 += (lo >> 8) & 0x00ff00ffu;
                    acc2 += hi & 0x00ff00ffu;
                    acc3 += (hi >> 8) & 0x00ff00ffu;
                    lo = hi = 0;
                    rounds = 0;
                }
            }
            acc0 += lo & 0x00ff00ffu;         // rows 0 and 2
            acc1 += (lo >> 8) & 0x00ff00ffu;  // rows 1 and 3
            acc2 += hi & 0x00ff00ffu;         // rows 4 and 6
            acc3 += (hi >> 8) & 0x00ff00ffu;  // rows 5 and 7
        }
        for (int32_t t0 = 0; !kBytes && t0 < nj; t0 += 4 * 32) {
            uint2 e[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int32_t t = t0 + u * 32 + lane;
                e[u] = t < nj ? lj[t] : make_uint2(kEmpty, 0u);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (e[u].x == kEmpty) continue;
                uint32_t slot = hash_slot(e[u].x, log2S);
                uint32_t key = keys[slot];
                for (int32_t probe = 0; key != e[u].x && key != kEmpty && probe < S; probe++) {
                    slot = (slot + 1) & (uint32_t)(S - 1);
                    key = keys[slot];
                }
                if (key == e[u].x) {
                    const uint2 v = *(const uint2*)&vals[2 * slot];
                    const uint32_t c4 = min(e[u].y, 255u) * 0x01010101u;
                    const uint32_t m0 = __vminu4(v.x, c4), m1 = __vminu4(v.y, c4);
                    acc0 += m0 & 0x00ff00ffu;          // rows 0 and 2
                    acc1 += (m0 >> 8) & 0x00ff00ffu;   // rows 1 and 3
                    acc2 += m1 & 0x00ff00ffu;          // rows 4 and 6
                    acc3 += (m1 >> 8) & 0x00ff00ffu;   // rows 5 and 7
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
            acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
            acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
            acc3 += __shfl_xor_sync(0xffffffffu, acc3, o);
        }
        // numerator of row `lane`
        const uint32_t w = (lane & 4) ? ((lane & 1) ? acc3 : acc2) : ((lane & 1) ? acc1 : acc0);
        const uint32_t part = (lane & 2) ? (w >> 16) : (w & 0xffffu);
        uint64_t col = 0, coll = 0;
        if (my >= 0 && (kMode != kDSums || my <= j)) {
            const uint32_t a = part + (uint32_t)residual_at(tab, hxi, tab.hidx[j]);
            if (kMode == kKeys) {
                const int32_t b = min(nki, tab.nkb[j]);
                out.key_a[j] = b <= 0 ? 0 : (int32_t)a;
                out.key_b[j] = b <= 0 ? 1 : b;
            } else {
                const uint64_t term = fixed_term_fast(a, nki, qi, ri, inv_i, tab.nkb[j], tab.q32[j], tab.r32[j],
                                                      tab.inv[j]);
                if (kMode == kDSums) {
                    const uint64_t tl = bli == tab.blk[j] ? term : 0;
                    rs_c += term;
                    rs_l += tl;
                    if (my != j) {
                        col = term;
                        coll = tl;
                    }
                    if (out.A) {
                        out.A[(int64_t)my * n + j] = (int32_t)a;
                        out.A[(int64_t)j * n + my] = (int32_t)a;
                    }
                } else if (kMode == kGSums) {
                    col = term;
                } else {
                    rs_c += term;
                }
            }
        }
        if (kMode == kDSums || kMode == kGSums) {
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                col += __shfl_xor_sync(0xffffffffu, col, o);
                coll += __shfl_xor_sync(0xffffffffu, coll, o);
            }
            if (lane == 0) {
                if (kMode == kDSums) {
                    if (col) atomicAdd((unsigned long long*)&out.dcen[j], (unsigned long long)col);
                    if (coll) atomicAdd((unsigned long long*)&out.dloc[j], (unsigned long long)coll);
                } else if (col) {
                    atomicAdd((unsigned long long*)&out.G[j], (unsigned long long)col);
                }
            }
        }
    }
    if (kMode == kDSums || kMode == kRowSums) {
        if (lane < kRowsMax && my >= 0) {
            if (rs_c) atomicAdd(&rowc[lane], (unsigned long long)rs_c);
            if (rs_l) atomicAdd(&rowl[lane], (unsigned long long)rs_l);
        }
        __syncthreads();
        const int32_t rp = r0 + threadIdx.x;
        if (threadIdx.x < TI && rp < nrows) {
            if (kMode == kDSums) {
                if (rowc[threadIdx.x]) atomicAdd((unsigned long long*)&out.dcen[rp], rowc[threadIdx.x]);
                if (rowl[threadIdx.x]) atomicAdd((unsigned long long*)&out.dloc[rp], rowl[threadIdx.x]);
            } else if (rowc[threadIdx.x]) {
                atomicAdd((unsigned long long*)&out.row_sums[rp], rowc[threadIdx.x]);
            }
        }
    }
}

int log2_ceil(int64_t v) {
    int l = 0;
    while ((1ll << l) < v) l++;
    return l;
}

// Launch shape of the rows x columns kernel: the byte table (8 rows) when the
// k-mer space fits shared memory at one byte per code; else the largest TI in
// {8, 4, 2, 1} whose hash table (a power of two with the rows' distinct k-mers,
// bounded by the k-mer space, filling at most 0.6 of it; at least 16 slots)
// fits; and a column chunk that leaves a few waves of CTAs (a wider chunk
// amortises the table's clear and build).
struct PairShape {
    int32_t TI, log2S, cw;
    size_t smem;
    bool bytes;
    int32_t V;
};

int pair_shape(sad_ctx* ctx, int64_t keys8, int64_t per_row, int64_t V, int64_t nrows, int64_t ncols,
               bool triangle, PairShape* sh) {
    const int64_t limit = (int64_t)ctx->smem_optin - 1024;
    sh->TI = 0;
    sh->bytes = sparse_byte_table(ctx, V);
    sh->V = sh->bytes ? (int32_t)V : 0;
    if (sh->bytes) {
        sh->TI = kRowsMax;
        sh->log2S = 0;
        sh->smem = (size_t)round_up(V, 16);
    }
    for (int t = kRowsMax; t >= 1 && !sh->bytes; t >>= 1) {
        int64_t keys = t == kRowsMax ? keys8 : std::min(keys8, per_row * t);
        keys = std::min(keys, V);
        const int l = std::max(4, log2_ceil(std::max<int64_t>((5 * keys + 2) / 3, 16)));
        if ((int64_t)12 << l <= limit) {
            sh->TI = t;
            sh->log2S = l;
            break;
        }
    }
    SAD_CHECK(sh->TI > 0, SAD_EINVAL, "a sequence has too many distinct k-mers for the sorted-list hash table");
    if (!sh->bytes) sh->smem = (size_t)12 << sh->log2S;
    // the widest chunk (up to 2048 columns) that still gives 8 CTAs per SM (4 of
    // the 1024-thread CTAs of a big byte table), else the narrowest (one column
    // per warp)
    const int64_t rb = (nrows + sh->TI - 1) / sh->TI;
    const bool big = sh->bytes && (int64_t)sh->smem > kBigTable;
    const int64_t want = (big ? 4ll : 8ll) * ctx->num_sms;
    sh->cw = kColChunkMax;
    while (sh->cw > (big ? kPairThreadsBytes / 32 : kColChunkMin) &&
           rb * ((ncols + sh->cw - 1) / sh->cw) / (triangle ? 2 : 1) < want)
        sh->cw /= 2;
    return SAD_OK;
}

template <int kMode, bool kBytes, int kThreads>
int launch_pairs_t(sad_ctx* ctx, int32_t n, int32_t nrows, const int32_t* row_ids, int32_t ncols,
                   const int32_t* col_ids, const PairShape& sh, const SparseLists& L, const SeqTables& tab,
                   const PairOut& out, cudaStream_t stream) {
    if (sh.smem > 40 * 1024)
        SAD_RET(allow_max_dynamic_smem(ctx, (const void*)k_sparse_pairs<kMode, kBytes, kThreads>));
    const dim3 grid((unsigned)((nrows + sh.TI - 1) / sh.TI), (unsigned)((ncols + sh.cw - 1) / sh.cw));
    k_sparse_pairs<kMode, kBytes, kThreads><<<grid, kThreads, sh.smem, stream>>>(
        n, nrows, row_ids, ncols, col_ids, sh.TI, sh.cw, sh.log2S, sh.V, L, tab, out);
    SAD_LAUNCHED();
    return SAD_OK;
}

template <int kMode>
int launch_pairs(sad_ctx* ctx, int32_t n, int32_t nrows, const int32_t* row_ids, int32_t ncols,
                 const int32_t* col_ids, const PairShape& sh, const SparseLists& L, const SeqTables& tab,
                 const PairOut& out, cudaStream_t stream) {
    if (!sh.bytes)
        return launch_pairs_t<kMode, false, kPairThreads>(ctx, n, nrows, row_ids, ncols, col_ids, sh, L, tab, out,
                                                          stream);
    if ((int64_t)sh.smem > kBigTable)
        return launch_pairs_t<kMode, true, kPairThreadsBytes>(ctx, n, nrows, row_ids, ncols, col_ids, sh, L, tab,
                                                              out, stream);
    return launch_pairs_t<kMode, true, kPairThreads>(ctx, n, nrows, row_ids, ncols, col_ids, sh, L, tab, out,
                                                     stream);
}

}  // namespace

bool sparse_byte_table(const sad_ctx* ctx, int64_t V) {
    return V >= 1 && round_up(V, 16) <= (int64_t)ctx->smem_optin - 2048;
}

int sparse_count(sad_ctx* ctx, const DevSeqs& S, int32_t k, int32_t A2, const ClassMap& cm, int32_t T,
                 const int64_t* loff, uint2* lists, int32_t* nd, const int64_t* ex_off, int32_t* ex_tau,
                 int32_t* ex_val, int32_t* nex, cudaStream_t stream) {
    const int32_t nk_max = S.max_len - k + 1;
    int32_t P = 1;
    while (P < nk_max) P <<= 1;
    const size_t smem = sizeof(uint32_t) * (size_t)P;
    if (smem > 40 * 1024) SAD_RET(allow_max_dynamic_smem(ctx, (const void*)k_sparse_count));
    k_sparse_count<<<S.n, kSortThreads, smem, stream>>>(S.res, S.pad_off, S.len, k, A2, cm, T, loff, lists, nd,
                                                        ex_off, ex_tau, ex_val, nex);
    SAD_LAUNCHED();
    return SAD_OK;
}

int sparse_allpairs(sad_ctx* ctx, int32_t n, const SparseLists& L, const SeqTables& tab, const int32_t* h_nd,
                    int64_t V, uint64_t* dloc, uint64_t* dcen, int32_t* A, cudaStream_t stream) {
    // bound of the distinct k-mers of any 8 consecutive rows, and of one row
    int64_t worst8 = 0, per_row = 0;
    for (int32_t b0 = 0; b0 < n; b0 += kRowsMax) {
        int64_t s = 0;
        for (int32_t i = b0; i < std::min(n, b0 + kRowsMax); i++) {
            const int64_t c = std::max(h_nd[i], 0);
            s += c;
            per_row = std::max(per_row, c);
        }
        worst8 = std::max(worst8, s);
    }
    PairShape sh;
    SAD_RET(pair_shape(ctx, worst8, per_row, V, n, n, true, &sh));
    const PairOut out{dloc, dcen, A, nullptr, nullptr, nullptr, nullptr};
    return launch_pairs<kDSums>(ctx, n, n, nullptr, n, nullptr, sh, L, tab, out, stream);
}

int sparse_sample_sums(sad_ctx* ctx, int32_t n, int32_t nslots, const int32_t* samples, const SparseLists& L,
                       const SeqTables& tab, int32_t max_nd, int64_t V, uint64_t* G, cudaStream_t stream) {
    const int64_t per_row = std::max<int64_t>(max_nd, 1);
    PairShape sh;
    SAD_RET(pair_shape(ctx, per_row * kRowsMax, per_row, V, nslots, n, false, &sh));
    const PairOut out{nullptr, nullptr, nullptr, G, nullptr, nullptr, nullptr};
    return launch_pairs<kGSums>(ctx, n, nslots, samples, n, nullptr, sh, L, tab, out, stream);
}

int sparse_ga_sums(sad_ctx* ctx, int32_t n, int32_t p, const int32_t* la, const SparseLists& L,
                   const SeqTables& tab, int32_t max_nd, int64_t V, uint64_t* gsum, cudaStream_t stream) {
    const int64_t per_row = std::max<int64_t>(max_nd, 1);
    PairShape sh;
    SAD_RET(pair_shape(ctx, per_row * kRowsMax, per_row, V, p, p, false, &sh));
    SAD_CUDA(cudaMemsetAsync(gsum, 0, 8ull * p, stream));
    const PairOut out{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, gsum};
    return launch_pairs<kRowSums>(ctx, n, p, la, p, la, sh, L, tab, out, stream);
}

int sparse_key_column(sad_ctx* ctx, int32_t n, const int32_t* ga, const SparseLists& L, const SeqTables& tab,
                      int32_t max_nd, int64_t V, int32_t* key_a, int32_t* key_b, cudaStream_t stream) {
    const int64_t per_row = std::max<int64_t>(max_nd, 1);
    PairShape sh;
    SAD_RET(pair_shape(ctx, per_row, per_row, V, 1, n, false, &sh));
    const PairOut out{nullptr, nullptr, nullptr, nullptr, key_a, key_b, nullptr};
    return launch_pairs<kKeys>(ctx, n, 1, ga, n, nullptr, sh, L, tab, out, stream);
}

}  // namespace sad
