// Progressive alignment of every bucket along its guide tree: the aligner
// each processor runs on its bucket (Section 2.3.3 lets it be any sequential
// multiple aligner; a progressive aligner joins the members two clusters at a
// time, in guide-tree order, each join aligning two fixed alignments).
//
// Definition (exact integers). A cluster is a multiple alignment of its
// members; column c of its profile counts, per letter a, the members with
// letter a there. Merge k aligns the profile P of cluster left[k] (rows,
// width m, nP members) with the profile Q of cluster right[k] (columns, width
// n, nQ members) by the three-state global affine-gap recursion
//   M(i,j) = max(M, X, Y)(i-1, j-1) + s(i, j)
//   X(i,j) = max(max(M, Y)(i-1, j) + go' + ge', X(i-1, j) + ge')
//   Y(i,j) = max(max(M, X)(i, j-1) + go' + ge', Y(i, j-1) + ge')
// with s(i, j) = sum_a sum_b cntP[i][a] cntQ[j][b] S[a][b] (letter pairs
// across the two profiles; gaps already in a column pair with nothing) and
// go' = nP nQ go, ge' = nP nQ ge (every cross pair of members receives a new
// gap run). One optimal alignment is taken back from (m, n) with the ties
// fixed: a cell's best state is M, then X, then Y; an X or Y column extends
// its run before it opens one, and opens from M before the other gap state.
// The merged cluster has one column per alignment column; every residue moves
// to the column its old column went to.
//
// GPU mapping. The merges of a bucket depend on each other only through the
// tree, so the host runs them level by level (a merge's level is one more
// than its children's), all buckets' merges of a level in one batch, and
// reads the new widths back after each level. Per batch:
//   k_prof_scores  tiles of 64 rows x 32 columns over all SMs: PB[j][a] =
//                  sum_b S[a][b] cntQ[j][b] in shared memory, then s(i, j) =
//                  sum_a cntP[i][a] PB[j][a], laid out as one stream per DP lane
//   k_prof_dp<T>   one CTA per merge: its rows are cut into strips of 64, one
//                  warp per strip (up to 8 side by side, each following the one
//                  above through a shared boundary row); the lanes hold 2 rows
//                  each and sweep the columns as a diagonal wavefront (M, X and
//                  Y of a lane's bottom row move one lane down per step); a lane
//                  loads its scores 8 steps ahead; every cell stores one byte of
//                  tie-resolved directions; warp 0 walks them back through a
//                  shared window, then all warps write the column maps and the
//                  merged profile. T is int32 when the host proves every value
//                  fits, else int64.
// At the end k_colmap composes each residue's column maps up the tree.
//
// sad_ancestor_glue (the last steps of the algorithm box: every bucket's
// alignment realigned with the global ancestor's profile, then all buckets
// joined through it) reuses the same score and DP kernels, one merge per
// bucket against the ancestor as a one-member profile; k_anchors turns the
// column maps into anchors, k_glue_layout and k_joined lay out the joined
// alignment, k_glue_residues drops its empty columns and writes the columns.
// Profiles (uint16 counts, the alphabet padded to 8) and column maps live in
// an arena of device chunks that only grows during a call.
#include <algorithm>
#include <type_traits>
#include <cstring>
#include <vector>

#include "sad_internal.cuh"

namespace sad {

namespace {

constexpr int kPrR = 2;                  // rows per lane
constexpr int kPrG = 32;                 // lanes per merge (one warp)
constexpr int kPrStrip = kPrR * kPrG;    // rows per strip
constexpr int kPrWarps = 8;              // most warps (strips side by side) per merge

// One merge of a batch.
struct ProgJob {
    const uint16_t* prof_p;  // P: m columns of Ap counts
    const uint16_t* prof_q;  // Q: n columns
    uint16_t* prof_r;        // the merged cluster (capacity m + n columns)
    int32_t* map;            // m entries for P's columns, then n for Q's
    int64_t s_off;           // cell-score streams (int4): strips x 32 lanes x (ceil(n/2) + 31) steps, then padding
    int64_t d_off;           // direction words (uint32, strips x (ceil(n/2) + 31) x 32)
    int32_t m, n, np, nq;
    int32_t merge;           // index into the per-merge outputs
    int32_t tile0;           // first score tile (a job has strips x ceil(n / 32) of them)
};

struct ProgArgs {
    const ProgJob* jobs;
    int32_t njobs;
    int32_t ntiles;
    int32_t Ap;              // counts per profile column
    int32_t alphabet;
    int32_t go, ge;
    const int8_t* subst;
    void* S;                 // int2 (one column per lane step) or int4 (two) score streams
    void* dirs;              // uint16 or uint32 direction words
    long long* scores;       // per merge
    int32_t* widths;         // per merge
    uint32_t* status;
    int64_t spin_limit;      // bound of the strip hand-off wait (polls of 32 ns)
    int32_t maxw;            // widest profile of the batch
    int32_t warp_smem;       // dynamic shared bytes of one DP CTA
};

// steps of direction words the traceback holds in shared memory (8 KB either way)
template <int C>
__host__ __device__ constexpr int win_steps() { return C == 1 ? 128 : 64; }
constexpr int kPrPre = 8;        // steps of cell scores a lane loads ahead

template <typename T>
__device__ __forceinline__ T neg_inf();
template <>
__device__ __forceinline__ int32_t neg_inf<int32_t>() { return -(1 << 30); }
template <>
__device__ __forceinline__ long long neg_inf<long long>() { return -(1ll << 60); }

template <typename T>
__device__ __forceinline__ T max3(T a, T b, T c) { return max(a, max(b, c)); }

// max(a, b) and whether a >= b: one DPX instruction for 32-bit values.
__device__ __forceinline__ int32_t bmax(int32_t a, int32_t b, bool& ge) { return __vibmax_s32(a, b, &ge); }
__device__ __forceinline__ long long bmax(long long a, long long b, bool& ge) {
    ge = a >= b;
    return ge ? a : b;
}

// Shared-memory layout of one DP warp: strip boundary (3 values per column),
// the traceback's window of direction words, the alignment columns.
template <typename T>
__host__ __device__ inline int64_t bnd_bytes(int32_t maxw) {
    return (3ll * (maxw + 2) * (int64_t)sizeof(T) + 15) / 16 * 16;
}
__host__ __device__ inline int64_t win_bytes() { return 8192; }
__host__ __device__ inline int64_t ops_bytes(int32_t maxw) { return (2ll * maxw + 16 + 15) / 16 * 16; }
// chunks of 32 alignment columns (at most 2 maxw columns), rounded to 4 for alignment
__host__ __device__ inline int32_t chunk_count(int32_t maxw) { return ((2 * maxw + 31) / 32 + 4) / 4 * 4; }

// Leaf profiles: one column per residue, a count of 1 for its letter.
__global__ void k_leaf_profiles(const uint8_t* __restrict__ res, const int64_t* __restrict__ pad_off,
                                const int32_t* __restrict__ len, const int32_t* __restrict__ order, int32_t npos,
                                const int64_t* __restrict__ pos_off, int32_t Ap, uint16_t* __restrict__ prof) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = wid; q < npos; q += nw) {
        const int32_t sq = order[q];
        const uint8_t* x = res + pad_off[sq];
        uint16_t* out = prof + pos_off[q] * Ap;
        const int64_t cells = (int64_t)len[sq] * Ap;
        for (int64_t t = lane; t < cells; t += 32) {
            const int64_t r = t / Ap;
            out[t] = (uint16_t)((t - r * Ap) == x[r] ? 1 : 0);
        }
    }
}

// Cell scores of one tile: 64 rows (one strip) x 32 columns of one merge.
// PB[j][a] = sum_b S[a][b] cntQ[j][b] is formed in shared memory for the
// tile's columns, then s(i, j) = sum_a cntP[i][a] PB[j][a]; thread (g, c4)
// holds rows 2g, 2g+1 and columns 4c4..4c4+3. Lane g of the DP warp reads its
// rows' scores as one stream over its steps: column j (1-based) sits at step
// tau = j - 1 + g.
constexpr int kScThreads = 256;
template <int C>
__global__ void __launch_bounds__(kScThreads)
k_prof_scores(ProgArgs a) {
    __shared__ int32_t sub[SAD_MAX_ALPHABET * SAD_MAX_ALPHABET];
    __shared__ int32_t cps[kPrStrip * (SAD_MAX_ALPHABET + 1)];
    __shared__ int32_t pbs[32 * (SAD_MAX_ALPHABET + 1)];
    const int32_t A = a.alphabet, Ap = a.Ap, st = A + 1;
    for (int t = threadIdx.x; t < A * A; t += blockDim.x) sub[t] = a.subst[t];
    for (int32_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        // the job holding this tile: the last one whose first tile is <= tile
        int32_t lo = 0, hi = a.njobs - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (a.jobs[mid].tile0 <= tile) lo = mid;
            else hi = mid - 1;
        }
        const ProgJob& jb = a.jobs[lo];
        const int32_t m = jb.m, n = jb.n;
        const int32_t cblocks = (n + 31) / 32, nsteps = C == 1 ? n + kPrG - 1 : (n + 1) / 2 + kPrG - 1;
        const int32_t tt = tile - jb.tile0, s = tt / cblocks, cb = tt - s * cblocks;
        __syncthreads();  // the previous tile's reads of cps / pbs are done (and sub is loaded)
        // a profile of one member is one letter per column (its count is 1): the
        // sums over letters then reduce to lookups (the same integers)
        const bool one_p = jb.np == 1, one_q = jb.nq == 1;
        if (one_p) {
            for (int r = threadIdx.x; r < kPrStrip; r += blockDim.x) {
                const int64_t i = (int64_t)s * kPrStrip + r;
                int32_t letter = -1;
                if (i < m)
                    for (int32_t l = 0; l < A; l++) letter = jb.prof_p[i * Ap + l] ? l : letter;
                cps[r] = letter;
            }
        } else {
            for (int t = threadIdx.x; t < kPrStrip * A; t += blockDim.x) {
                const int32_t r = t / A, l = t - r * A;
                const int64_t i = (int64_t)s * kPrStrip + r;
                cps[r * st + l] = i < m ? (int32_t)jb.prof_p[i * Ap + l] : 0;
            }
        }
        for (int t = threadIdx.x; t < 32 * A; t += blockDim.x) {
            const int32_t c = t / A, l = t - c * A;
            const int64_t j = (int64_t)cb * 32 + c;
            int32_t v = 0;
            if (j < n) {
                const uint16_t* cq = jb.prof_q + j * Ap;
                if (one_q) {
                    for (int32_t b = 0; b < A; b++) v = cq[b] ? sub[l * A + b] : v;
                } else {
                    for (int32_t b = 0; b < A; b++) v += sub[l * A + b] * (int32_t)cq[b];
                }
            }
            pbs[c * st + l] = v;
        }
        __syncthreads();
        const int g = threadIdx.x >> 3, c4 = threadIdx.x & 7;
        int32_t acc[kPrR][4];
#pragma unroll
        for (int r = 0; r < kPrR; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[r][c] = 0;
        if (one_p) {
#pragma unroll
            for (int r = 0; r < kPrR; r++) {
                const int32_t letter = cps[g * kPrR + r];
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = letter >= 0 ? pbs[(c4 * 4 + c) * st + letter] : 0;
            }
        } else {
            for (int32_t l = 0; l < A; l++) {
                int32_t pv[kPrR], qv[4];
#pragma unroll
                for (int r = 0; r < kPrR; r++) pv[r] = cps[(g * kPrR + r) * st + l];
#pragma unroll
                for (int c = 0; c < 4; c++) qv[c] = pbs[(c4 * 4 + c) * st + l];
#pragma unroll
                for (int r = 0; r < kPrR; r++)
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[r][c] += pv[r] * qv[c];
            }
        }
        if constexpr (C == 1) {  // column j0 at step j0 + g
            int2* out = (int2*)a.S + jb.s_off + ((int64_t)s * kPrG + g) * nsteps;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int32_t j0 = cb * 32 + c4 * 4 + c;  // 0-based column
                if (j0 < n) out[j0 + g] = make_int2(acc[0][c], acc[1][c]);
            }
        } else {  // column pair qp (columns 2qp, 2qp + 1) at step qp + g
            int4* out = (int4*)a.S + jb.s_off + ((int64_t)s * kPrG + g) * nsteps;
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const int32_t qp = cb * 16 + c4 * 2 + e;
                if (2 * qp < n)
                    out[qp + g] = make_int4(acc[0][2 * e], acc[1][2 * e], acc[0][2 * e + 1], acc[1][2 * e + 1]);
            }
        }
    }
}


__device__ __forceinline__ int32_t take_row(const int2& v, int r) { return r == 0 ? v.x : v.y; }

// Direction byte of a cell: bits 0-1 its best state (0 M, 1 X, 2 Y); bit 2
// X extends; bit 3 X opens from M (else from Y); bit 4 Y extends; bit 5 Y
// opens from M (else from X).
//
// One CTA per merge, W = blockDim.x / 32 warps: warp w takes strips w, w + W,
// ... in order. The bottom row of strip s goes to boundary slot s mod W with
// a progress count (the last column written); the warp of strip s + 1 reads
// it one column at a time once the count has passed that column. A slot is
// rewritten by strip s + W, which reaches a column only after strip s + 1 has
// read it, so W slots suffice. Then warp 0 walks the directions back.
constexpr int kMaxStrips = 256;
constexpr int64_t kSpinLimit = 1ll << 22;

template <typename T, int C>
__global__ void __launch_bounds__(kPrG * kPrWarps)
k_prof_dp(ProgArgs a) {
    using DirT = typename std::conditional<C == 1, uint16_t, uint32_t>::type;
    constexpr int kWin = win_steps<C>();
    extern __shared__ __align__(16) unsigned char psm[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int64_t slot_bytes = bnd_bytes<T>(a.maxw);
    volatile int32_t* prog = (volatile int32_t*)(psm + W * slot_bytes);
    T* score_sh = (T*)(psm + W * slot_bytes + 4 * kMaxStrips);
    int32_t* len_sh = (int32_t*)(psm + W * slot_bytes + 4 * kMaxStrips + 8);
    DirT* win = (DirT*)(psm + W * slot_bytes + 4 * kMaxStrips + 16);
    uint8_t* ops = psm + W * slot_bytes + 4 * kMaxStrips + 16 + win_bytes();
    int32_t* chP = (int32_t*)(ops + ops_bytes(a.maxw));
    int32_t* chQ = chP + chunk_count(a.maxw);
    const T NEG = neg_inf<T>();
    const int32_t Ap = a.Ap;
    for (int64_t k = blockIdx.x; k < a.njobs; k += gridDim.x) {
        const ProgJob& jb = a.jobs[k];
        const int32_t m = jb.m, n = jb.n;
        const T w = (T)jb.np * (T)jb.nq;
        const T gop = w * (T)a.go, gex = w * (T)a.ge, goe = gop + gex;
        const int32_t cap = m + n;
        const int32_t strips = (m + kPrStrip - 1) / kPrStrip;
        const int32_t nsteps = C == 1 ? n + kPrG - 1 : (n + 1) / 2 + kPrG - 1;  // C columns per lane step
        DirT* dirs = (DirT*)a.dirs + jb.d_off;
        const bool cells = m > 0 && n > 0;
        for (int t = threadIdx.x; t < strips; t += blockDim.x) prog[t] = 0;
        __syncthreads();
        // one cell: diagonal hd = H(i-1, j-1), (am, ax, ay) = (M, X, Y)(i-1, j),
        // (lm, lx, ly) = (M, X, Y)(i, j-1); returns the direction byte
        auto cell = [&](T hd, T am, T ax, T ay, T lm, T lx, T ly, int32_t sc, T& M, T& X, T& Y, T& H) -> uint32_t {
            bool xs, xe, ys, ye, xy, mb;
            M = hd + (T)sc;
            X = bmax(ax + gex, bmax(am, ay, xs) + goe, xe);
            Y = bmax(ly + gex, bmax(lm, lx, ys) + goe, ye);
            H = bmax(M, bmax(X, Y, xy), mb);
            return (mb ? 0u : (xy ? 1u : 2u)) | (xe ? 4u : 0u) | (xs ? 8u : 0u) | (ye ? 16u : 0u) | (ys ? 32u : 0u);
        };
        if constexpr (C == 1) {
            for (int32_t s = warp; cells && s < strips; s += W) {
                const T* bin = (const T*)(psm + ((s + W - 1) % W) * slot_bytes);
                T* bout = (T*)(psm + (s % W) * slot_bytes);
                const int32_t row0 = s * kPrStrip + lane * kPrR;  // rows row0+1 .. row0+2 (1-based)
                T mm[kPrR], xx[kPrR], yy[kPrR], hh[kPrR];          // values at the previous column
    #pragma unroll
                for (int r = 0; r < kPrR; r++) {
                    mm[r] = NEG;
                    xx[r] = gop + (T)(row0 + r + 1) * gex;  // X(i, 0)
                    yy[r] = NEG;
                    hh[r] = xx[r];
                }
                T hdiag = row0 == 0 ? (T)0 : gop + (T)row0 * gex;  // H(row0, 0)
                T min_ = NEG, xin = NEG, yin = NEG;                // (row0, j) from above
                const bool last_strip = s == strips - 1;
                int32_t avail = s == 0 ? n : 0;                    // columns of the strip above known written
                // this lane's score stream (the job's padding keeps the look-ahead in bounds)
                const int2* Sl = (const int2*)a.S + jb.s_off + ((int64_t)s * kPrG + lane) * nsteps;
                int2 cur[kPrPre], nxt[kPrPre];
    #pragma unroll
                for (int u = 0; u < kPrPre; u++) cur[u] = Sl[u];
                for (int32_t tau0 = 0; tau0 < nsteps; tau0 += kPrPre) {
    #pragma unroll
                    for (int u = 0; u < kPrPre; u++) nxt[u] = Sl[tau0 + kPrPre + u];
    #pragma unroll
                    for (int u = 0; u < kPrPre; u++) {
                        const int32_t tau = tau0 + u;
                        if (tau >= nsteps) break;
                        if (lane == 0 && tau < n) {
                            if (s == 0) {
                                min_ = NEG;
                                xin = NEG;
                                yin = gop + (T)(tau + 1) * gex;  // Y(0, j)
                            } else {
                                if (avail < tau + 1) {  // wait (bounded) for the strip above
                                    int64_t spins = 0;
                                    while ((avail = prog[s - 1]) < tau + 1 && ++spins < a.spin_limit) __nanosleep(32);
                                    if (spins >= a.spin_limit) {
                                        atomicOr(a.status, STATUS_TIMEOUT);
                                        avail = n;
                                    }
                                    __threadfence_block();
                                }
                                const volatile T* vb = bin;
                                min_ = vb[3 * (tau + 1)];
                                xin = vb[3 * (tau + 1) + 1];
                                yin = vb[3 * (tau + 1) + 2];
                            }
                        }
                        const int32_t j = tau - lane + 1;
                        T mo = min_, xo = xin, yo = yin;
                        if (j >= 1 && j <= n) {
                            const int2 sv = cur[u];
                            T hd = hdiag, am = min_, ax = xin, ay = yin;
                            uint32_t bits = 0;
    #pragma unroll
                            for (int r = 0; r < kPrR; r++) {
                                bool xs, xe, ys, ye, xy, mb;
                                const T M = hd + (T)take_row(sv, r);
                                const T X = bmax(ax + gex, bmax(am, ay, xs) + goe, xe);
                                const T Y = bmax(yy[r] + gex, bmax(mm[r], xx[r], ys) + goe, ye);
                                const T H = bmax(M, bmax(X, Y, xy), mb);
                                const uint32_t b = (mb ? 0u : (xy ? 1u : 2u)) | (xe ? 4u : 0u) | (xs ? 8u : 0u) |
                                                   (ye ? 16u : 0u) | (ys ? 32u : 0u);
                                bits |= b << (8 * r);
                                hd = hh[r];  // H(i, j-1): the next row's diagonal
                                mm[r] = M;
                                xx[r] = X;
                                yy[r] = Y;
                                hh[r] = H;
                                am = M;
                                ax = X;
                                ay = Y;
                            }
                            dirs[((int64_t)s * nsteps + tau) * kPrG + lane] = (uint16_t)bits;
                            hdiag = max3(min_, xin, yin);  // H(row0, j): the next column's diagonal
                            mo = am;
                            xo = ax;
                            yo = ay;
                            if (!last_strip && lane == kPrG - 1) {
                                volatile T* vb = bout;
                                vb[3 * j] = mo;
                                vb[3 * j + 1] = xo;
                                vb[3 * j + 2] = yo;
                                __threadfence_block();
                                prog[s] = j;
                            }
                        }
                        min_ = __shfl_up_sync(0xffffffffu, mo, 1);
                        xin = __shfl_up_sync(0xffffffffu, xo, 1);
                        yin = __shfl_up_sync(0xffffffffu, yo, 1);
                    }
    #pragma unroll
                    for (int u = 0; u < kPrPre; u++) cur[u] = nxt[u];
                }
                if (last_strip) {
                    // (named values: a select over the array would put it in local memory)
                    static_assert(kPrR == 2, "two rows per lane");
                    const int32_t rr = (m - 1) - s * kPrStrip;
                    const T v = (rr % kPrR) == 0 ? hh[0] : hh[1];
                    const T sc = __shfl_sync(0xffffffffu, v, rr / kPrR);
                    if (lane == 0) *score_sh = sc;
                }
                __syncwarp();
            }
        } else {
            for (int32_t s = warp; cells && s < strips; s += W) {
                const T* bin = (const T*)(psm + ((s + W - 1) % W) * slot_bytes);
                T* bout = (T*)(psm + (s % W) * slot_bytes);
                const int32_t row0 = s * kPrStrip + lane * kPrR;  // rows row0+1 .. row0+2 (1-based)
                T mm[kPrR], xx[kPrR], yy[kPrR], hh[kPrR];          // values at the previous column
    #pragma unroll
                for (int r = 0; r < kPrR; r++) {
                    mm[r] = NEG;
                    xx[r] = gop + (T)(row0 + r + 1) * gex;  // X(i, 0)
                    yy[r] = NEG;
                    hh[r] = xx[r];
                }
                T hdiag = row0 == 0 ? (T)0 : gop + (T)row0 * gex;  // H(row0, 0)
                // (row0, j0) and (row0, j1) from above, j0 = 2q + 1, j1 = 2q + 2 for pair q
                T a0m = NEG, a0x = NEG, a0y = NEG, a1m = NEG, a1x = NEG, a1y = NEG;
                const bool last_strip = s == strips - 1;
                int32_t avail = s == 0 ? n : 0;                    // columns of the strip above known written
                // this lane's score stream (the job's padding keeps the look-ahead in bounds)
                const int4* Sl = (const int4*)a.S + jb.s_off + ((int64_t)s * kPrG + lane) * nsteps;
                int4 cur[kPrPre], nxt[kPrPre];
    #pragma unroll
                for (int u = 0; u < kPrPre; u++) cur[u] = Sl[u];
                for (int32_t tau0 = 0; tau0 < nsteps; tau0 += kPrPre) {
    #pragma unroll
                    for (int u = 0; u < kPrPre; u++) nxt[u] = Sl[tau0 + kPrPre + u];
    #pragma unroll
                    for (int u = 0; u < kPrPre; u++) {
                        const int32_t tau = tau0 + u;
                        if (tau >= nsteps) break;
                        const int32_t lj0 = 2 * tau + 1;  // lane 0's columns this step
                        if (lane == 0 && lj0 <= n) {
                            const int32_t lj1 = min(lj0 + 1, n);
                            if (s == 0) {
                                a0m = a0x = a1m = a1x = NEG;
                                a0y = gop + (T)lj0 * gex;  // Y(0, j)
                                a1y = gop + (T)(lj0 + 1) * gex;
                            } else {
                                if (avail < lj1) {  // wait (bounded) for the strip above
                                    int64_t spins = 0;
                                    while ((avail = prog[s - 1]) < lj1 && ++spins < a.spin_limit) __nanosleep(32);
                                    if (spins >= a.spin_limit) {
                                        atomicOr(a.status, STATUS_TIMEOUT);
                                        avail = n;
                                    }
                                    __threadfence_block();
                                }
                                const volatile T* vb = bin;
                                a0m = vb[3 * lj0];
                                a0x = vb[3 * lj0 + 1];
                                a0y = vb[3 * lj0 + 2];
                                a1m = vb[3 * lj1];  // (lj1 = n when lj0 = n: not used then)
                                a1x = vb[3 * lj1 + 1];
                                a1y = vb[3 * lj1 + 2];
                            }
                        }
                        const int32_t q = tau - lane;
                        const int32_t j0 = 2 * q + 1;
                        T o0m = a0m, o0x = a0x, o0y = a0y, o1m = a1m, o1x = a1x, o1y = a1y;
                        if (q >= 0 && j0 <= n) {
                            const bool two = j0 < n;
                            const int4 sv = cur[u];
                            T M00, X00, Y00, H00, M10, X10, Y10, H10, M01, X01, Y01, H01, M11, X11, Y11, H11;
                            // the two chains (one per column) interleave: (r0,c0); (r1,c0) with (r0,c1); (r1,c1)
                            const uint32_t b00 = cell(hdiag, a0m, a0x, a0y, mm[0], xx[0], yy[0], sv.x, M00, X00, Y00, H00);
                            const uint32_t b10 = cell(hh[0], M00, X00, Y00, mm[1], xx[1], yy[1], sv.y, M10, X10, Y10, H10);
                            const T hup = max3(a0m, a0x, a0y);  // H(row0, j0)
                            const uint32_t b01 = cell(hup, a1m, a1x, a1y, M00, X00, Y00, sv.z, M01, X01, Y01, H01);
                            const uint32_t b11 = cell(H00, M01, X01, Y01, M10, X10, Y10, sv.w, M11, X11, Y11, H11);
                            dirs[((int64_t)s * nsteps + tau) * kPrG + lane] =
                                b00 | (b10 << 8) | (two ? (b01 << 16) | (b11 << 24) : 0u);
                            o0m = M10;
                            o0x = X10;
                            o0y = Y10;
                            if (two) {
                                mm[0] = M01;
                                xx[0] = X01;
                                yy[0] = Y01;
                                hh[0] = H01;
                                mm[1] = M11;
                                xx[1] = X11;
                                yy[1] = Y11;
                                hh[1] = H11;
                                hdiag = max3(a1m, a1x, a1y);  // H(row0, j1): the next pair's diagonal
                                o1m = M11;
                                o1x = X11;
                                o1y = Y11;
                            } else {
                                mm[0] = M00;
                                xx[0] = X00;
                                yy[0] = Y00;
                                hh[0] = H00;
                                mm[1] = M10;
                                xx[1] = X10;
                                yy[1] = Y10;
                                hh[1] = H10;
                            }
                            if (!last_strip && lane == kPrG - 1) {
                                volatile T* vb = bout;
                                vb[3 * j0] = o0m;
                                vb[3 * j0 + 1] = o0x;
                                vb[3 * j0 + 2] = o0y;
                                if (two) {
                                    vb[3 * j0 + 3] = o1m;
                                    vb[3 * j0 + 4] = o1x;
                                    vb[3 * j0 + 5] = o1y;
                                }
                                __threadfence_block();
                                prog[s] = two ? j0 + 1 : j0;
                            }
                        }
                        a0m = __shfl_up_sync(0xffffffffu, o0m, 1);
                        a0x = __shfl_up_sync(0xffffffffu, o0x, 1);
                        a0y = __shfl_up_sync(0xffffffffu, o0y, 1);
                        a1m = __shfl_up_sync(0xffffffffu, o1m, 1);
                        a1x = __shfl_up_sync(0xffffffffu, o1x, 1);
                        a1y = __shfl_up_sync(0xffffffffu, o1y, 1);
                    }
    #pragma unroll
                    for (int u = 0; u < kPrPre; u++) cur[u] = nxt[u];
                }
                if (last_strip) {
                    // (named values: a select over the array would put it in local memory)
                    static_assert(kPrR == 2, "two rows per lane");
                    const int32_t rr = (m - 1) - s * kPrStrip;
                    const T v = (rr % kPrR) == 0 ? hh[0] : hh[1];
                    const T sc = __shfl_sync(0xffffffffu, v, rr / kPrR);
                    if (lane == 0) *score_sh = sc;
                }
                __syncwarp();
            }
        }
        __syncthreads();  // every strip's directions are written
        if (warp == 0) {
            T score = 0;
            int32_t L = 0;
            if (!cells) {  // one gap run, or nothing
                for (int32_t c = lane; c < cap; c += 32) ops[c] = m == 0 ? 'Y' : 'X';
                score = cap == 0 ? (T)0 : gop + (T)cap * gex;
                L = cap;
            } else {
                score = *score_sh;
                // traceback, one column per step: every lane walks the same path (the
                // direction words come from a shared window of kWin steps of one
                // strip, reloaded by the whole warp when the path leaves it); lane 0
                // writes the columns backwards from the end of the slot. The cell
                // (i, jj) sits in strip s, lane t, row r of the lane, step tau.
                // The walk goes a run at a time: in state M the cells ahead are the
                // diagonal (i-k, jj-k), k >= 1, and the run goes on while a cell's best
                // state is M; in state X (Y) they are (i-k, jj) ((i, jj-k)), k >= 0, and
                // the run goes on while the cell extends its gap. Lane l looks at the
                // l-th cell ahead; a ballot finds where the run ends. A cell outside the
                // shared window (another strip, or steps not loaded) ends the look-ahead
                // without ending the run; state 3 means the current cell's best state is
                // still to be read.
                int32_t i = m, jj = n, state = 3;
                int32_t ws = -1, wt0 = 0;
                int64_t guard = 2ll * cap + 4;
                while (i > 0 && jj > 0 && guard-- > 0) {
                    const int32_t k = state == 0 ? lane + 1 : (state == 3 ? 0 : lane);
                    const int32_t ci = i - (state != 2 ? k : 0), cj = jj - (state != 1 ? k : 0);
                    const bool valid = ci > 0 && cj > 0 && (state != 3 || lane == 0);
                    const uint32_t q = (uint32_t)(ci - 1);
                    const int32_t cs = (int32_t)(q / kPrStrip), ct = (int32_t)((q % kPrStrip) / kPrR);
                    const int32_t ctau = (C == 1 ? cj - 1 : (cj - 1) / 2) + ct;  // C columns per lane step
                    bool inwin = valid && cs == ws && ctau >= wt0 && ctau < wt0 + kWin;
                    // the first cell ahead must be in the window: reload around it
                    const bool need = __shfl_sync(0xffffffffu, valid && !inwin, 0);
                    if (need) {
                        ws = __shfl_sync(0xffffffffu, cs, 0);
                        wt0 = max(0, __shfl_sync(0xffffffffu, ctau, 0) - kWin + 1);
                        __syncwarp();
                        // kWin steps x 32 lanes of DirT, in 16-byte chunks (kChunks per step)
                        constexpr int kChunks = 2 * (int)sizeof(DirT);
                        for (int e = lane; e < kWin * kChunks; e += 32) {
                            const int32_t u = e / kChunks, part = e % kChunks;
                            if (wt0 + u < nsteps)
                                ((uint4*)win)[e] = *(const uint4*)(dirs + ((int64_t)ws * nsteps + wt0 + u) * kPrG +
                                                                   part * (16 / (int)sizeof(DirT)));
                        }
                        __syncwarp();
                        inwin = valid && cs == ws && ctau >= wt0 && ctau < wt0 + kWin;
                    }
                    // byte of the cell: row r; with two columns per step, column half h = (cj - 1) & 1
                    // holds bytes 2h (row 0) and 2h + 1
                    const int32_t byte = C == 1 ? (int32_t)(q % kPrR) : 2 * ((cj - 1) & 1) + (int32_t)(q % kPrR);
                    const uint32_t bb = inwin ? (((uint32_t)win[(ctau - wt0) * kPrG + ct] >> (8 * byte)) & 0xffu) : 0u;
                    if (state == 3) {
                        state = (int32_t)(__shfl_sync(0xffffffffu, bb, 0) & 3u);
                        continue;
                    }
                    const bool cont = inwin && (state == 0 ? (bb & 3u) == 0 : (state == 1 ? (bb & 4u) != 0
                                                                                           : (bb & 16u) != 0));
                    const unsigned stop = ~__ballot_sync(0xffffffffu, cont);
                    const int32_t f = stop ? __ffs(stop) - 1 : 32;  // first lane whose cell ends the look-ahead
                    const uint32_t bf = __shfl_sync(0xffffffffu, bb, f & 31);
                    const bool real = f < 32 && __shfl_sync(0xffffffffu, inwin ? 1 : 0, f & 31);
                    int32_t E, nstate;
                    if (state == 0) {  // M at (i, jj), then the continuing diagonal cells
                        E = f + 1;
                        nstate = real ? (int32_t)(bf & 3u) : 3;
                    } else if (state == 1) {
                        E = real ? f + 1 : f;
                        nstate = real ? ((bf & 8u) ? 0 : 2) : 1;
                    } else {
                        E = real ? f + 1 : f;
                        nstate = real ? ((bf & 32u) ? 0 : 1) : 2;
                    }
                    const uint8_t opc = state == 0 ? 'M' : (state == 1 ? 'X' : 'Y');
                    for (int32_t e = lane; e < E; e += 32) ops[cap - 1 - L - e] = opc;
                    L += E;
                    i -= state != 2 ? E : 0;
                    jj -= state != 1 ? E : 0;
                    state = nstate;
                }
                if (guard < 0 && lane == 0) atomicOr(a.status, STATUS_CAPACITY);
                // the border: X(i, 0) and Y(0, j) are single gap runs
                for (int32_t c = lane; c < i; c += 32) ops[cap - 1 - L - c] = 'X';
                L += i;
                for (int32_t c = lane; c < jj; c += 32) ops[cap - 1 - L - c] = 'Y';
                L += jj;
                L = min(L, cap);
            }
            if (lane == 0) {
                *len_sh = L;
                a.scores[jb.merge] = (long long)score;
                a.widths[jb.merge] = L;
            }
        }
        __syncthreads();
        // the column maps and the merged profile, 32 columns per warp step: the
        // P and Q columns before each chunk come from a prefix over the chunks
        {
            const int32_t L = *len_sh;
            const uint8_t* col = ops + (cap - L);
            const int32_t nch = (L + 31) / 32;
            for (int32_t c0 = warp * 32; c0 < L; c0 += W * 32) {
                const int32_t c = c0 + lane;
                const uint8_t op = c < L ? col[c] : 0;
                const unsigned bp = __ballot_sync(0xffffffffu, c < L && op != 'Y');
                const unsigned bq = __ballot_sync(0xffffffffu, c < L && op != 'X');
                if (lane == 0) {
                    chP[c0 / 32] = __popc(bp);
                    chQ[c0 / 32] = __popc(bq);
                }
            }
            __syncthreads();
            if (warp == 0) {  // exclusive prefix over the chunks
                int32_t carryP = 0, carryQ = 0;
                for (int32_t c0 = 0; c0 < nch; c0 += 32) {
                    const int32_t c = c0 + lane;
                    const int32_t vP = c < nch ? chP[c] : 0, vQ = c < nch ? chQ[c] : 0;
                    int32_t iP = vP, iQ = vQ;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int32_t xP = __shfl_up_sync(0xffffffffu, iP, o), xQ = __shfl_up_sync(0xffffffffu, iQ, o);
                        if (lane >= o) {
                            iP += xP;
                            iQ += xQ;
                        }
                    }
                    __syncwarp();
                    if (c < nch) {
                        chP[c] = carryP + iP - vP;
                        chQ[c] = carryQ + iQ - vQ;
                    }
                    carryP += __shfl_sync(0xffffffffu, iP, 31);
                    carryQ += __shfl_sync(0xffffffffu, iQ, 31);
                }
            }
            __syncthreads();
            int32_t* mapP = jb.map;
            int32_t* mapQ = jb.map + m;
            const unsigned below = (1u << lane) - 1u;
            for (int32_t c0 = warp * 32; c0 < L; c0 += W * 32) {
                const int32_t c = c0 + lane;
                const uint8_t op = c < L ? col[c] : 0;
                const bool inP = c < L && op != 'Y', inQ = c < L && op != 'X';
                const unsigned bp = __ballot_sync(0xffffffffu, inP), bq = __ballot_sync(0xffffffffu, inQ);
                const int32_t i = chP[c0 / 32] + __popc(bp & below), j = chQ[c0 / 32] + __popc(bq & below);
                if (inP) mapP[i] = c;
                if (inQ) mapQ[j] = c;
                if (c < L) {
                    const uint4* cp = (const uint4*)(jb.prof_p + (int64_t)i * Ap);
                    const uint4* cq = (const uint4*)(jb.prof_q + (int64_t)j * Ap);
                    uint4* cr = (uint4*)(jb.prof_r + (int64_t)c * Ap);
                    for (int32_t h = 0; h < Ap / 8; h++) {
                        const uint4 u = inP ? cp[h] : make_uint4(0, 0, 0, 0);
                        const uint4 v = inQ ? cq[h] : make_uint4(0, 0, 0, 0);
                        // two 16-bit counts per word; their sums stay below 2^16
                        cr[h] = make_uint4(u.x + v.x, u.y + v.y, u.z + v.z, u.w + v.w);
                    }
                }
            }
        }
        __syncthreads();  // shared memory is reused by the next merge
    }
}

// Final columns: each residue's leaf column, moved through the column map of
// every merge on its way to the root. One warp per bucket position.
__global__ void k_colmap(int32_t npos, const int32_t* __restrict__ order, const int32_t* __restrict__ len,
                         const int64_t* __restrict__ pos_off, const int32_t* __restrict__ leaf_gc,
                         const int32_t* __restrict__ par_merge, const int32_t* __restrict__ par_gc,
                         const uint8_t* __restrict__ par_side, int32_t* const* __restrict__ map_ptr,
                         const int32_t* __restrict__ map_split, int32_t max_depth, int32_t* __restrict__ colmap) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = wid; q < npos; q += nw) {
        const int32_t L = len[order[q]];
        for (int32_t r = lane; r < L; r += 32) {
            int32_t c = r, g = leaf_gc[q];
            for (int32_t d = 0; d < max_depth; d++) {
                const int32_t k = par_merge[g];
                if (k < 0) break;
                c = map_ptr[k][(par_side[g] ? map_split[k] : 0) + c];
                g = par_gc[g];
            }
            colmap[pos_off[q] + r] = c;
        }
    }
}

// Bump allocation over a grow-only list of device chunks (profiles and
// column maps; what a merge writes must outlive its batch).
struct Arena {
    sad_ctx* ctx;
    size_t cur = 0, off = 0;
    int alloc(size_t bytes, void** out) {
        bytes = (size_t)round_up((int64_t)std::max<size_t>(bytes, 16), 256);
        while (cur < ctx->prog_chunks.size() && off + bytes > ctx->prog_chunks[cur].bytes) {
            cur++;
            off = 0;
        }
        if (cur == ctx->prog_chunks.size()) {
            Buffer b;
            b.bytes = std::max<size_t>(bytes, (size_t)64 << 20);
            cudaError_t e = cudaMalloc(&b.ptr, b.bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                set_error("cudaMalloc of %zu bytes for the alignment arena failed: %s", b.bytes,
                          cudaGetErrorString(e));
                return SAD_ENOMEM;
            }
            ctx->prog_chunks.push_back(b);
            off = 0;
        }
        *out = (char*)ctx->prog_chunks[cur].ptr + off;
        off += bytes;
        return SAD_OK;
    }
};

// A batch of independent merges: every job's offsets into the batch's score
// streams, direction words and score tiles, and what the launch needs.
struct Batch {
    int C = 1;  // columns per DP lane step (1 or 2)
    std::vector<ProgJob> jobs;
    int64_t s_vecs = 0, d_words = 0, maxw = 1, max_strips = 0;
    int32_t tiles = 0;
    bool wide = false;
    int64_t steps(int64_t n) const { return (C == 1 ? n : (n + 1) / 2) + kPrG - 1; }  // C columns per lane step
    int64_t streams(int64_t m, int64_t n) const {  // score streams plus the look-ahead of the last lane
        return (m > 0 && n > 0) ? (m + kPrStrip - 1) / kPrStrip * kPrG * steps(n) + 2 * kPrPre : 0;
    }
    int64_t words(int64_t m, int64_t n) const {
        return (m > 0 && n > 0) ? (m + kPrStrip - 1) / kPrStrip * steps(n) * kPrG : 0;
    }
    // bytes of scores (8 C per stream element) and directions (2 C per word) once a merge of m x n is added
    int64_t bytes_with(int64_t m, int64_t n) const {
        return 8ll * C * (s_vecs + streams(m, n)) + 2ll * C * (d_words + words(m, n));
    }
    // checks the merge's ranges (SAD_EINVAL) and appends it
    int add(ProgJob jb, int64_t smax, int64_t cmax) {
        const int64_t m = jb.m, n = jb.n, strips = (m + kPrStrip - 1) / kPrStrip;
        SAD_CHECK(strips <= kMaxStrips, SAD_EINVAL, "merge %d: a profile of %lld columns (at most %d)", jb.merge,
                  (long long)m, kMaxStrips * kPrStrip);
        const int64_t pq = (int64_t)jb.np * jb.nq;
        SAD_CHECK(pq * smax < (1ll << 31), SAD_EINVAL,
                  "merge %d: %lld member pairs x max |S| exceed the 32-bit cell scores", jb.merge, (long long)pq);
        if ((m + n + 2 * kPrStrip) * pq * cmax >= (1ll << 28)) wide = true;
        jb.s_off = s_vecs;
        jb.d_off = d_words;
        jb.tile0 = tiles;
        jobs.push_back(jb);
        s_vecs += streams(m, n);
        d_words += words(m, n);
        tiles += (m > 0 && n > 0) ? (int32_t)(strips * ((n + 31) / 32)) : 0;
        maxw = std::max(maxw, std::max(m, n));
        max_strips = std::max(max_strips, strips);
        return SAD_OK;
    }
};

// Columns per DP lane step for a batch of `jobs` merges whose widest column
// profile has `maxn` columns (the context can force one form).
int pick_columns(const sad_ctx* ctx, int64_t jobs, int64_t maxn) {
    if (ctx->prog_columns == 1 || ctx->prog_columns == 2) return ctx->prog_columns;
    return (jobs >= ctx->num_sms || maxn >= 1024) ? 2 : 1;
}

// Launches one batch (score tiles, then the DP: one CTA per merge, one warp
// per strip up to kPrWarps); `pa` carries the call's parameters and outputs.
int run_batch(sad_ctx* ctx, const Batch& bt, ProgArgs pa, cudaStream_t stream, ProgJob* pin_jobs) {
    const int32_t nj = (int32_t)bt.jobs.size();
    if (nj == 0) return SAD_OK;
    // shared memory: one boundary slot per warp, the progress counts, the
    // traceback window, the columns and their chunk counts
    const int64_t slot = bt.wide ? bnd_bytes<long long>((int32_t)bt.maxw) : bnd_bytes<int32_t>((int32_t)bt.maxw);
    const int64_t fixed = 4 * kMaxStrips + 16 + win_bytes() + ops_bytes((int32_t)bt.maxw) +
                          8ll * chunk_count((int32_t)bt.maxw);
    int64_t warps_cta = std::min<int64_t>(kPrWarps, std::max<int64_t>(1, bt.max_strips));
    while (warps_cta > 1 && warps_cta * slot + fixed > (int64_t)ctx->smem_optin - 1024) warps_cta--;
    SAD_CHECK(slot + fixed <= (int64_t)ctx->smem_optin - 1024, SAD_EINVAL,
              "profiles of %lld columns exceed the DP kernel's shared memory", (long long)bt.maxw);
    const int64_t cta_smem = warps_cta * slot + fixed;
    const int64_t grid_dp = std::min<int64_t>(nj, (int64_t)ctx->num_sms * 16);
    size_t lo = 0;
    auto lcarve = [&](size_t bytes) {
        const size_t o = lo;
        lo = (size_t)round_up((int64_t)(lo + bytes), 256);
        return o;
    };
    const size_t l_jobs = lcarve(sizeof(ProgJob) * nj), l_s = lcarve(8ull * bt.C * bt.s_vecs + 16),
                 l_d = lcarve(2ull * bt.C * bt.d_words + 4);
    void* lv_ws = nullptr;
    SAD_RET(workspace(ctx, WS_PROG_LEVEL, lo, stream, &lv_ws));
    char* lw = (char*)lv_ws;
    // the job table through pinned memory (the caller synchronises before the next batch reuses it)
    memcpy(pin_jobs, bt.jobs.data(), sizeof(ProgJob) * nj);
    SAD_CUDA(cudaMemcpyAsync(lw + l_jobs, pin_jobs, sizeof(ProgJob) * nj, cudaMemcpyHostToDevice, stream));
    pa.jobs = (const ProgJob*)(lw + l_jobs);
    pa.njobs = nj;
    pa.ntiles = bt.tiles;
    pa.S = lw + l_s;
    pa.dirs = lw + l_d;
    pa.maxw = (int32_t)bt.maxw;
    pa.warp_smem = (int32_t)cta_smem;
    void (*dp)(ProgArgs) = bt.C == 1 ? (bt.wide ? k_prof_dp<long long, 1> : k_prof_dp<int32_t, 1>)
                                      : (bt.wide ? k_prof_dp<long long, 2> : k_prof_dp<int32_t, 2>);
    SAD_RET(allow_max_dynamic_smem(ctx, (const void*)dp));
    if (bt.tiles > 0) {
        const unsigned g1 = (unsigned)std::min<int64_t>(bt.tiles, (int64_t)ctx->num_sms * 8);
        if (bt.C == 1) k_prof_scores<1><<<g1, kScThreads, 0, stream>>>(pa);
        else k_prof_scores<2><<<g1, kScThreads, 0, stream>>>(pa);
        SAD_LAUNCHED();
    }
    dp<<<(unsigned)grid_dp, (unsigned)(kPrG * warps_cta), (size_t)cta_smem, stream>>>(pa);
    SAD_LAUNCHED();
    return SAD_OK;
}


// ---- realignment against the global ancestor and the glue ----------------

// Profile of every bucket from its alignment: position q's residue r adds 1 to
// column colmap[pos_off[q] + r] of its bucket (two 16-bit counts per word; a
// column never counts more than the bucket's members). A column outside the
// bucket's width is reported, not counted.
__global__ void k_bucket_profiles(const uint8_t* __restrict__ res, const int64_t* __restrict__ pad_off,
                                  const int32_t* __restrict__ len, const int32_t* __restrict__ order, int32_t npos,
                                  const int64_t* __restrict__ pos_off, const int32_t* __restrict__ pos_bucket,
                                  const int64_t* __restrict__ col_off, const int32_t* __restrict__ widths,
                                  const int32_t* __restrict__ colmap, int32_t Ap, uint32_t* __restrict__ prof,
                                  uint32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = wid; q < npos; q += nw) {
        const int32_t sq = order[q], b = pos_bucket[q];
        const uint8_t* x = res + pad_off[sq];
        for (int32_t r = lane; r < len[sq]; r += 32) {
            const int32_t c = colmap[pos_off[q] + r];
            if (c < 0 || c >= widths[b]) {
                atomicOr(status, STATUS_BAD_INPUT);
                continue;
            }
            if (x[r] >= Ap) continue;  // a residue code the sequence check reports
            const int64_t e = (col_off[b] + c) * Ap + x[r];
            atomicAdd(prof + (e >> 1), 1u << (16 * (e & 1)));
        }
    }
}

// Anchor of every bucket column from its realignment's column maps: with P's
// column i at alignment column mapP[i] and ancestor position g at mapQ[g]
// (increasing), s = #{g : mapQ[g] < mapP[i]}; the column is anchored at s when
// mapQ[s] == mapP[i], else it is an insertion of slot s (stored -(s + 1),
// counted in ins[s * p + b], the slot's first such column of the bucket in
// first[s * p + b]).
__global__ void k_anchors(int32_t p, const int64_t* __restrict__ col_off, int32_t* const* __restrict__ map_ptr,
                          int32_t lg, int32_t* __restrict__ anchors, int32_t* __restrict__ ins,
                          int32_t* __restrict__ first) {
    const int64_t total = col_off[p];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = p - 1;  // the bucket holding column t: the last with col_off <= t
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (col_off[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const int32_t b = lo;
        const int64_t m = col_off[b + 1] - col_off[b], i = t - col_off[b];
        const int32_t* mapP = map_ptr[b];
        const int32_t* mapQ = mapP + m;
        const int32_t c = mapP[i];
        int32_t a = 0, z = lg;  // lower bound of c in mapQ
        while (a < z) {
            const int32_t mid = (a + z) >> 1;
            if (mapQ[mid] < c) a = mid + 1;
            else z = mid;
        }
        if (a < lg && mapQ[a] == c) {
            anchors[t] = a;
        } else {
            anchors[t] = -(a + 1);
            atomicAdd(&ins[(int64_t)a * p + b], 1);
            atomicMin(&first[(int64_t)a * p + b], (int32_t)i);
        }
    }
}

// Exclusive prefix sums of x[0..n) into y (y[n] = the total), by one CTA.
__device__ void block_scan(const int32_t* x, int64_t n, int32_t* y) {
    __shared__ int32_t warp_sum[32];
    __shared__ int32_t carry_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry_sh = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < n; c0 += blockDim.x) {
        const int64_t t = c0 + threadIdx.x;
        const int32_t v = t < n ? x[t] : 0;
        int32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) warp_sum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            int32_t ws = lane < nw ? warp_sum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t u = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += u;
            }
            if (lane < nw) warp_sum[lane] = ws;  // inclusive over warps
        }
        __syncthreads();
        const int32_t before = carry_sh + (warp > 0 ? warp_sum[warp - 1] : 0);
        if (t < n) y[t] = before + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) carry_sh += warp_sum[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) y[n] = carry_sh;
}

// The joined layout: slot s holds the insertions of bucket 0, 1, ..., then the
// anchor of ancestor position s. sizes[s * (p + 1) + b] = ins[s * p + b] for
// b < p and 1 for the anchor (0 after the last position); start = their
// exclusive prefix sums.
__global__ void k_glue_layout(int32_t p, int32_t lg, const int32_t* __restrict__ ins, int32_t* __restrict__ sizes,
                              int32_t* __restrict__ start) {
    const int64_t cells = (int64_t)(lg + 1) * (p + 1);
    for (int64_t t = threadIdx.x; t < cells; t += blockDim.x) {
        const int64_t s = t / (p + 1), b = t - s * (p + 1);
        sizes[t] = b < p ? ins[s * p + b] : (s < lg ? 1 : 0);
    }
    __syncthreads();
    block_scan(sizes, cells, start);
}

// Joined column of every bucket column: its anchor's column, or the slot's
// start for its bucket plus its rank among the bucket's insertions of that
// slot (they are consecutive columns: rank = i - the first of them).
__global__ void k_joined(int32_t p, const int64_t* __restrict__ col_off, const int32_t* __restrict__ anchors,
                         const int32_t* __restrict__ start, const int32_t* __restrict__ first,
                         int32_t* __restrict__ joined) {
    const int64_t total = col_off[p];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = p - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (col_off[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const int32_t b = lo, a = anchors[t];
        const int64_t i = t - col_off[b];
        if (a >= 0) {
            joined[t] = start[(int64_t)a * (p + 1) + p];
        } else {
            const int64_t sl = -a - 1;
            joined[t] = start[sl * (p + 1) + b] + (int32_t)(i - first[sl * p + b]);
        }
    }
}

// used[joined column of each residue] = 1 (mode 0), or the residue's final
// column renum[...] (mode 1). One warp per bucket position.
__global__ void k_glue_residues(int32_t mode, const int32_t* __restrict__ order, int32_t npos,
                                const int32_t* __restrict__ len, const int64_t* __restrict__ pos_off,
                                const int32_t* __restrict__ pos_bucket, const int64_t* __restrict__ col_off,
                                const int32_t* __restrict__ widths, const int32_t* __restrict__ colmap,
                                const int32_t* __restrict__ joined, int32_t* __restrict__ used,
                                const int32_t* __restrict__ renum, int32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = wid; q < npos; q += nw) {
        const int32_t b = pos_bucket[q];
        for (int32_t r = lane; r < len[order[q]]; r += 32) {
            const int32_t c = colmap[pos_off[q] + r];
            if (c < 0 || c >= widths[b]) continue;  // reported by k_bucket_profiles
            const int32_t g = joined[col_off[b] + c];
            if (mode == 0) used[g] = 1;
            else out[pos_off[q] + r] = renum[g];
        }
    }
}

__global__ void k_scan_one(const int32_t* __restrict__ x, int64_t n, int32_t* __restrict__ y) { block_scan(x, n, y); }
}  // namespace

}  // namespace sad

extern "C" int sad_progressive_align(sad_ctx* ctx_in, const sad_seqset* seqs, const int32_t* bucket_offsets,
                                     const int32_t* order, int32_t p, const int64_t* merge_offsets,
                                     const int32_t* left, const int32_t* right, const int8_t* subst,
                                     int32_t gap_open, int32_t gap_extend, int32_t* widths, int64_t* merge_scores,
                                     int32_t* merge_widths, int32_t* colmap, int32_t mem, void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mem == SAD_MEM_HOST || mem == SAD_MEM_DEVICE, SAD_EINVAL, "mem = %d", mem);
    SAD_CHECK(p >= 1, SAD_EINVAL, "p = %d < 1", p);
    SAD_CHECK(seqs && subst && bucket_offsets && merge_offsets && widths, SAD_EINVAL, "a required pointer is NULL");
    SAD_CHECK(gap_open <= 0 && gap_extend <= 0, SAD_EINVAL, "gap costs must be <= 0");
    SAD_CHECK(gap_open >= -1000 && gap_extend >= -1000, SAD_EINVAL, "gap costs below -1000");
    const int32_t A = seqs->alphabet;
    SAD_CHECK(A >= 1 && A <= SAD_MAX_ALPHABET, SAD_EINVAL, "alphabet %d outside 1..%d", A, SAD_MAX_ALPHABET);
    for (int32_t x = 0; x < A; x++)
        for (int32_t y = 0; y < A; y++)
            SAD_CHECK(subst[x * A + y] == subst[y * A + x], SAD_EINVAL, "the substitution matrix is not symmetric");
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    SAD_RET(status_clear(ctx, stream));
    DevSeqs S;
    SAD_RET(prepare_seqs(ctx, seqs, mem, stream, &S));
    // the layout and the trees on the host
    std::vector<int32_t> bo((size_t)p + 1);
    std::vector<int64_t> mo((size_t)p + 1);
    SAD_RET(arg_to_host(bucket_offsets, 4ull * (p + 1), mem, stream, bo.data()));
    SAD_RET(arg_to_host(merge_offsets, 8ull * (p + 1), mem, stream, mo.data()));
    SAD_CHECK(bo[0] == 0 && mo[0] == 0, SAD_EINVAL, "bucket_offsets and merge_offsets must start at 0");
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = bo[b + 1] - bo[b];
        SAD_CHECK(nb >= 0, SAD_EINVAL, "bucket_offsets decreases at %d", b);
        SAD_CHECK(nb < 65536, SAD_EINVAL, "bucket %d has %lld members (at most 65535)", b, (long long)nb);
        SAD_CHECK(mo[b + 1] - mo[b] == (nb > 0 ? nb - 1 : 0), SAD_EINVAL,
                  "merge_offsets of bucket %d do not hold its %lld merges", b, (long long)(nb > 0 ? nb - 1 : 0));
    }
    const int32_t npos = bo[p];
    const int64_t M = mo[p];
    SAD_CHECK(npos == 0 || order, SAD_EINVAL, "order is NULL");
    SAD_CHECK(M == 0 || (left && right && merge_scores && merge_widths), SAD_EINVAL, "a required pointer is NULL");
    std::vector<int32_t> od((size_t)npos), lt((size_t)M), rt((size_t)M);
    SAD_RET(arg_to_host(order, 4ull * npos, mem, stream, od.data()));
    SAD_RET(arg_to_host(left, 4ull * M, mem, stream, lt.data()));
    SAD_RET(arg_to_host(right, 4ull * M, mem, stream, rt.data()));
    std::vector<int64_t> pos_off((size_t)npos + 1, 0);
    for (int32_t q = 0; q < npos; q++) {
        SAD_CHECK(od[q] >= 0 && od[q] < S.n, SAD_EINVAL, "order[%d] = %d outside 0..%d", q, od[q], S.n - 1);
        pos_off[q + 1] = pos_off[q] + S.h_len[od[q]];
    }
    const int64_t T_res = pos_off[npos];
    SAD_CHECK(T_res == 0 || colmap, SAD_EINVAL, "colmap is NULL");
    // clusters: global id cl_off[b] + local id (leaves 0..nb-1, merge k -> nb + k)
    std::vector<int64_t> cl_off((size_t)p + 1, 0);
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = bo[b + 1] - bo[b];
        cl_off[b + 1] = cl_off[b] + (nb > 0 ? 2 * nb - 1 : 0);
    }
    const int64_t C = cl_off[p];
    std::vector<int32_t> width((size_t)C, 0), nmem((size_t)C, 0), level((size_t)C, 0), par_merge((size_t)C, -1),
        par_gc((size_t)C, -1), leaf_gc((size_t)npos, 0);
    std::vector<uint8_t> par_side((size_t)C, 0), alive((size_t)C, 0);
    std::vector<int32_t> merge_level((size_t)M, 0), merge_bucket((size_t)M, 0);
    int32_t max_level = 0, max_depth = 1;
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = bo[b + 1] - bo[b];
        for (int64_t u = 0; u < nb; u++) {
            const int64_t g = cl_off[b] + u;
            width[g] = S.h_len[od[bo[b] + u]];
            nmem[g] = 1;
            alive[g] = 1;
            leaf_gc[bo[b] + u] = (int32_t)g;
        }
        for (int64_t k = 0; k + 1 < nb; k++) {
            const int64_t mi = mo[b] + k;
            const int32_t l = lt[mi], r = rt[mi];
            SAD_CHECK(l >= 0 && r >= 0 && l < nb + k && r < nb + k && l != r, SAD_EINVAL,
                      "merge %lld of bucket %d joins clusters %d and %d, not two of 0..%lld", (long long)k, b, l, r,
                      (long long)(nb + k - 1));
            const int64_t gl = cl_off[b] + l, gr = cl_off[b] + r, gn = cl_off[b] + nb + k;
            SAD_CHECK(alive[gl] && alive[gr], SAD_EINVAL, "merge %lld of bucket %d reuses a merged cluster",
                      (long long)k, b);
            alive[gl] = alive[gr] = 0;
            alive[gn] = 1;
            nmem[gn] = nmem[gl] + nmem[gr];
            level[gn] = 1 + std::max(level[gl], level[gr]);
            merge_level[mi] = level[gn];
            merge_bucket[mi] = b;
            max_level = std::max(max_level, level[gn]);
            par_merge[gl] = par_merge[gr] = (int32_t)mi;
            par_gc[gl] = par_gc[gr] = (int32_t)gn;
            par_side[gl] = 0;
            par_side[gr] = 1;
        }
    }
    max_depth = max_level + 1;
    int32_t smax = 0;
    for (int32_t t = 0; t < A * A; t++) smax = std::max(smax, (int32_t)std::abs((int)subst[t]));
    const int64_t cmax = std::max<int64_t>(smax, (int64_t)-gap_open - gap_extend);
    const int32_t Ap = (int32_t)round_up(A, 8);
    // device tables of the call (copied once), outputs staged in host mode
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_sub = carve(1024), o_od = carve(4ull * (npos + 1)), o_pos = carve(8ull * (npos + 1)),
                 o_leaf = carve(4ull * (npos + 1)), o_pm = carve(4ull * (C + 1)), o_pg = carve(4ull * (C + 1)),
                 o_ps = carve(C + 16), o_mp = carve(8ull * (M + 1)), o_ms = carve(4ull * (M + 1)),
                 o_sc = carve(8ull * (M + 1)), o_w = carve(4ull * (M + 1)),
                 o_cm = carve(mem == SAD_MEM_HOST ? 4ull * (T_res + 1) : 0);
    void* wsp = nullptr;
    SAD_RET(workspace(ctx, WS_PROG, off, stream, &wsp));
    char* w = (char*)wsp;
    int8_t* d_sub = (int8_t*)(w + o_sub);
    int32_t* d_od = (int32_t*)(w + o_od);
    int64_t* d_pos = (int64_t*)(w + o_pos);
    long long* d_sc = mem == SAD_MEM_HOST ? (long long*)(w + o_sc) : (long long*)merge_scores;
    int32_t* d_mw = mem == SAD_MEM_HOST ? (int32_t*)(w + o_w) : merge_widths;
    int32_t* d_cm = mem == SAD_MEM_HOST ? (int32_t*)(w + o_cm) : colmap;
    if (M == 0) {
        d_sc = (long long*)(w + o_sc);
        d_mw = (int32_t*)(w + o_w);
    }
    SAD_CUDA(cudaMemcpyAsync(d_sub, subst, (size_t)A * A, cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync(d_od, od.data(), 4ull * npos, cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync(d_pos, pos_off.data(), 8ull * (npos + 1), cudaMemcpyHostToDevice, stream));
    // leaf profiles
    Arena arena{ctx};
    void* leaf_prof = nullptr;
    SAD_RET(arena.alloc(2ull * Ap * std::max<int64_t>(T_res, 1), &leaf_prof));
    std::vector<const uint16_t*> prof((size_t)C, nullptr);
    for (int32_t b = 0; b < p; b++)
        for (int32_t u = 0; u < bo[b + 1] - bo[b]; u++)
            prof[cl_off[b] + u] = (const uint16_t*)leaf_prof + pos_off[bo[b] + u] * Ap;
    TraceScope ts(ctx, SAD_STAGE_PROG, stream);
    if (npos > 0) {
        const int64_t blocks = std::min<int64_t>(((int64_t)npos * 32 + 255) / 256, (int64_t)ctx->num_sms * 16);
        k_leaf_profiles<<<(unsigned)blocks, 256, 0, stream>>>(S.res, S.pad_off, S.len, d_od, npos, d_pos, Ap,
                                                              (uint16_t*)leaf_prof);
        SAD_LAUNCHED();
    }
    // merges level by level
    std::vector<std::vector<int32_t>> by_level((size_t)max_level + 1);
    for (int64_t mi = 0; mi < M; mi++) by_level[merge_level[mi]].push_back((int32_t)mi);
    std::vector<int32_t*> map_ptr((size_t)M, nullptr);
    std::vector<int32_t> map_split((size_t)M, 0);
    // pinned host staging: a batch's job table, and the merge widths read back per level
    void* pin = nullptr;
    const size_t pin_jobs_bytes = (size_t)round_up((int64_t)sizeof(ProgJob) * std::max<int64_t>(M, 1), 256);
    SAD_RET(pinned(ctx, pin_jobs_bytes + 4ull * (M + 1), stream, &pin));
    ProgJob* pin_jobs = (ProgJob*)pin;
    int32_t* h_mw = (int32_t*)((char*)pin + pin_jobs_bytes);
    const int64_t budget = (int64_t)1 << 30;  // bytes of cell scores and directions per batch
    ProgArgs base{};
    base.Ap = Ap;
    base.alphabet = A;
    base.go = gap_open;
    base.ge = gap_extend;
    base.subst = d_sub;
    base.scores = d_sc;
    base.widths = d_mw;
    base.status = ctx->d_status;
    base.spin_limit = ctx->prog_spin_limit > 0 ? ctx->prog_spin_limit : kSpinLimit;
    for (int32_t lv = 1; lv <= max_level; lv++) {
        const std::vector<int32_t>& ms = by_level[lv];
        // columns per DP lane step: two when the level holds enough merges to fill the GPU or
        // wide profiles (fewer instructions per cell), else one (a shorter lag between strips)
        int64_t maxn = 0;
        for (int32_t mi : ms) {
            const int32_t b = merge_bucket[mi];
            maxn = std::max<int64_t>(maxn, width[cl_off[b] + rt[mi]]);
        }
        const int level_c = pick_columns(ctx, (int64_t)ms.size(), maxn);
        for (size_t j0 = 0; j0 < ms.size();) {
            Batch bt;
            bt.C = level_c;
            size_t j1 = j0;
            while (j1 < ms.size()) {
                const int32_t mi = ms[j1];
                const int32_t b = merge_bucket[mi];
                const int64_t nb = bo[b + 1] - bo[b];
                const int64_t k = mi - mo[b];
                const int64_t gl = cl_off[b] + lt[mi], gr = cl_off[b] + rt[mi], gn = cl_off[b] + nb + k;
                const int64_t m = width[gl], n = width[gr];
                if (j1 > j0 && bt.bytes_with(m, n) > budget) break;
                ProgJob jb{};
                jb.prof_p = prof[gl];
                jb.prof_q = prof[gr];
                void* pr = nullptr;
                SAD_RET(arena.alloc(2ull * Ap * (m + n), &pr));
                jb.prof_r = (uint16_t*)pr;
                void* mp = nullptr;
                SAD_RET(arena.alloc(4ull * (m + n), &mp));
                jb.map = (int32_t*)mp;
                jb.m = (int32_t)m;
                jb.n = (int32_t)n;
                jb.np = nmem[gl];
                jb.nq = nmem[gr];
                jb.merge = mi;
                SAD_RET(bt.add(jb, smax, cmax));
                prof[gn] = jb.prof_r;
                map_ptr[mi] = jb.map;
                map_split[mi] = (int32_t)m;
                j1++;
            }
            SAD_RET(run_batch(ctx, bt, base, stream, pin_jobs));
            const std::vector<ProgJob>& jobs = bt.jobs;
            // the new widths, for the next level's layout (the jobs' table copy
            // from pageable memory has been consumed when this returns)
            SAD_CUDA(cudaMemcpyAsync(h_mw, d_mw, 4ull * std::max<int64_t>(M, 1), cudaMemcpyDeviceToHost,
                                     stream));
            SAD_CUDA(cudaStreamSynchronize(stream));
            for (const ProgJob& jb : jobs) {
                const int32_t b = merge_bucket[jb.merge];
                const int64_t nb = bo[b + 1] - bo[b];
                const int64_t gn = cl_off[b] + nb + (jb.merge - mo[b]);
                SAD_CHECK(h_mw[jb.merge] >= std::max(jb.m, jb.n) && h_mw[jb.merge] <= jb.m + jb.n, SAD_ECUDA,
                          "merge %d returned width %d for widths %d and %d", jb.merge, h_mw[jb.merge], jb.m, jb.n);
                width[gn] = h_mw[jb.merge];
            }
            j0 = j1;
        }
    }
    // the final column of every residue, and the widths of the buckets' alignments
    std::vector<int32_t> h_w((size_t)p, 0);
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = bo[b + 1] - bo[b];
        h_w[b] = nb > 0 ? width[cl_off[b] + 2 * nb - 2] : 0;
    }
    if (npos > 0) {
        int32_t* d_leaf = (int32_t*)(w + o_leaf);
        int32_t* d_pm = (int32_t*)(w + o_pm);
        int32_t* d_pg = (int32_t*)(w + o_pg);
        uint8_t* d_ps = (uint8_t*)(w + o_ps);
        int32_t** d_mp = (int32_t**)(w + o_mp);
        int32_t* d_msp = (int32_t*)(w + o_ms);
        SAD_CUDA(cudaMemcpyAsync(d_leaf, leaf_gc.data(), 4ull * npos, cudaMemcpyHostToDevice, stream));
        SAD_CUDA(cudaMemcpyAsync(d_pm, par_merge.data(), 4ull * C, cudaMemcpyHostToDevice, stream));
        SAD_CUDA(cudaMemcpyAsync(d_pg, par_gc.data(), 4ull * C, cudaMemcpyHostToDevice, stream));
        SAD_CUDA(cudaMemcpyAsync(d_ps, par_side.data(), (size_t)C, cudaMemcpyHostToDevice, stream));
        if (M > 0) {
            SAD_CUDA(cudaMemcpyAsync(d_mp, map_ptr.data(), 8ull * M, cudaMemcpyHostToDevice, stream));
            SAD_CUDA(cudaMemcpyAsync(d_msp, map_split.data(), 4ull * M, cudaMemcpyHostToDevice, stream));
        }
        const int64_t blocks = std::min<int64_t>(((int64_t)npos * 32 + 255) / 256, (int64_t)ctx->num_sms * 16);
        k_colmap<<<(unsigned)blocks, 256, 0, stream>>>(npos, d_od, S.len, d_pos, d_leaf, d_pm, d_pg, d_ps, d_mp,
                                                       d_msp, max_depth, d_cm);
        SAD_LAUNCHED();
    }
    // outputs (host mode: copied back; device mode: widths from the host table)
    if (mem == SAD_MEM_HOST) {
        memcpy(widths, h_w.data(), 4ull * p);
        if (M > 0) {
            SAD_CUDA(cudaMemcpyAsync(merge_scores, d_sc, 8ull * M, cudaMemcpyDeviceToHost, stream));
            SAD_CUDA(cudaMemcpyAsync(merge_widths, d_mw, 4ull * M, cudaMemcpyDeviceToHost, stream));
        }
        if (T_res > 0) SAD_CUDA(cudaMemcpyAsync(colmap, d_cm, 4ull * T_res, cudaMemcpyDeviceToHost, stream));
    } else {
        SAD_CUDA(cudaMemcpyAsync(widths, h_w.data(), 4ull * p, cudaMemcpyHostToDevice, stream));
    }
    SAD_RET(status_check(ctx, stream));
    return SAD_OK;
}

extern "C" int sad_ancestor_glue(sad_ctx* ctx_in, const sad_seqset* seqs, const int32_t* bucket_offsets,
                                 const int32_t* order, int32_t p, const int32_t* widths, const int32_t* colmap,
                                 int32_t ga, const int8_t* subst, int32_t gap_open, int32_t gap_extend,
                                 int64_t* ga_scores, int32_t* anchors, int32_t* global_width, int32_t* global_colmap,
                                 int32_t mem, void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mem == SAD_MEM_HOST || mem == SAD_MEM_DEVICE, SAD_EINVAL, "mem = %d", mem);
    SAD_CHECK(p >= 1, SAD_EINVAL, "p = %d < 1", p);
    SAD_CHECK(seqs && subst && bucket_offsets && widths && ga_scores && global_width, SAD_EINVAL,
              "a required pointer is NULL");
    SAD_CHECK(gap_open <= 0 && gap_extend <= 0, SAD_EINVAL, "gap costs must be <= 0");
    SAD_CHECK(gap_open >= -1000 && gap_extend >= -1000, SAD_EINVAL, "gap costs below -1000");
    const int32_t A = seqs->alphabet;
    SAD_CHECK(A >= 1 && A <= SAD_MAX_ALPHABET, SAD_EINVAL, "alphabet %d outside 1..%d", A, SAD_MAX_ALPHABET);
    for (int32_t x = 0; x < A; x++)
        for (int32_t y = 0; y < A; y++)
            SAD_CHECK(subst[x * A + y] == subst[y * A + x], SAD_EINVAL, "the substitution matrix is not symmetric");
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    SAD_RET(status_clear(ctx, stream));
    DevSeqs S;
    SAD_RET(prepare_seqs(ctx, seqs, mem, stream, &S));
    SAD_CHECK(ga >= 0 && ga < S.n, SAD_EINVAL, "ga = %d outside 0..%d", ga, S.n - 1);
    // layout on the host
    std::vector<int32_t> bo((size_t)p + 1), wd((size_t)p);
    SAD_RET(arg_to_host(bucket_offsets, 4ull * (p + 1), mem, stream, bo.data()));
    SAD_RET(arg_to_host(widths, 4ull * p, mem, stream, wd.data()));
    SAD_CHECK(bo[0] == 0, SAD_EINVAL, "bucket_offsets must start at 0");
    for (int32_t b = 0; b < p; b++) {
        SAD_CHECK(bo[b + 1] >= bo[b], SAD_EINVAL, "bucket_offsets decreases at %d", b);
        SAD_CHECK(bo[b + 1] - bo[b] < 65536, SAD_EINVAL, "bucket %d has more than 65535 members", b);
        SAD_CHECK(wd[b] >= 0 && (bo[b + 1] > bo[b] || wd[b] == 0), SAD_EINVAL, "widths[%d] = %d", b, wd[b]);
    }
    const int32_t npos = bo[p];
    SAD_CHECK(npos == 0 || order, SAD_EINVAL, "order is NULL");
    std::vector<int32_t> od((size_t)npos), pos_bucket((size_t)npos);
    SAD_RET(arg_to_host(order, 4ull * npos, mem, stream, od.data()));
    std::vector<int64_t> pos_off((size_t)npos + 1, 0), col_off((size_t)p + 1, 0);
    for (int32_t b = 0; b < p; b++) {
        col_off[b + 1] = col_off[b] + wd[b];
        for (int32_t q = bo[b]; q < bo[b + 1]; q++) {
            SAD_CHECK(od[q] >= 0 && od[q] < S.n, SAD_EINVAL, "order[%d] = %d outside 0..%d", q, od[q], S.n - 1);
            pos_off[q + 1] = pos_off[q] + S.h_len[od[q]];
            pos_bucket[q] = b;
        }
    }
    const int64_t T_res = pos_off[npos], Wtot = col_off[p];
    SAD_CHECK(T_res == 0 || (colmap && global_colmap), SAD_EINVAL, "colmap or global_colmap is NULL");
    SAD_CHECK(Wtot == 0 || anchors, SAD_EINVAL, "anchors is NULL");
    const int32_t lg = S.h_len[ga];
    const int64_t J = Wtot + lg;  // joined columns before the empty ones are dropped, at most
    int32_t smax = 0;
    for (int32_t t = 0; t < A * A; t++) smax = std::max(smax, (int32_t)std::abs((int)subst[t]));
    const int64_t cmax = std::max<int64_t>(smax, (int64_t)-gap_open - gap_extend);
    const int32_t Ap = (int32_t)round_up(A, 8);
    // device tables, scratch and (host mode) staged arrays
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const int64_t cells = (int64_t)(lg + 1) * p, lay = (int64_t)(lg + 1) * (p + 1);
    const size_t o_sub = carve(1024), o_od = carve(4ull * (npos + 1)), o_pos = carve(8ull * (npos + 1)),
                 o_pb = carve(4ull * (npos + 1)), o_coff = carve(8ull * (p + 1)), o_wd = carve(4ull * p),
                 o_mp = carve(8ull * p), o_ins = carve(4ull * cells), o_first = carve(4ull * cells),
                 o_sizes = carve(4ull * lay), o_start = carve(4ull * (lay + 1)), o_join = carve(4ull * (Wtot + 1)),
                 o_used = carve(4ull * (J + 1)), o_renum = carve(4ull * (J + 1)), o_ga = carve(16),
                 o_gpos = carve(16), o_mw = carve(4ull * p), o_sc = carve(8ull * p), o_an = carve(4ull * (Wtot + 1)),
                 o_cm = carve(mem == SAD_MEM_HOST ? 4ull * (T_res + 1) : 0),
                 o_gcm = carve(mem == SAD_MEM_HOST ? 4ull * (T_res + 1) : 0);
    void* wsp = nullptr;
    SAD_RET(workspace(ctx, WS_PROG, off, stream, &wsp));
    char* w = (char*)wsp;
    int32_t* d_od = (int32_t*)(w + o_od);
    int64_t* d_pos = (int64_t*)(w + o_pos);
    int32_t* d_pb = (int32_t*)(w + o_pb);
    int64_t* d_coff = (int64_t*)(w + o_coff);
    int32_t* d_wd = (int32_t*)(w + o_wd);
    int32_t* d_ins = (int32_t*)(w + o_ins);
    int32_t* d_first = (int32_t*)(w + o_first);
    int32_t* d_start = (int32_t*)(w + o_start);
    int32_t* d_join = (int32_t*)(w + o_join);
    int32_t* d_used = (int32_t*)(w + o_used);
    int32_t* d_renum = (int32_t*)(w + o_renum);
    long long* d_sc = mem == SAD_MEM_HOST ? (long long*)(w + o_sc) : (long long*)ga_scores;
    int32_t* d_an = (mem == SAD_MEM_HOST || Wtot == 0) ? (int32_t*)(w + o_an) : anchors;
    const int32_t* d_cm = colmap;
    int32_t* d_gcm = mem == SAD_MEM_HOST ? (int32_t*)(w + o_gcm) : global_colmap;
    if (mem == SAD_MEM_HOST) {
        if (T_res > 0) SAD_CUDA(cudaMemcpyAsync(w + o_cm, colmap, 4ull * T_res, cudaMemcpyHostToDevice, stream));
        d_cm = (const int32_t*)(w + o_cm);
    }
    const int64_t ga_pos[2] = {0, lg};
    SAD_CUDA(cudaMemcpyAsync(w + o_sub, subst, (size_t)A * A, cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync(d_od, od.data(), 4ull * npos, cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync(d_pos, pos_off.data(), 8ull * (npos + 1), cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync(d_pb, pos_bucket.data(), 4ull * npos, cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync(d_coff, col_off.data(), 8ull * (p + 1), cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync(d_wd, wd.data(), 4ull * p, cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync(w + o_ga, &ga, 4, cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync(w + o_gpos, ga_pos, 16, cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemsetAsync(d_sc, 0, 8ull * p, stream));
    SAD_CUDA(cudaMemsetAsync(d_ins, 0, 4ull * cells, stream));
    SAD_CUDA(cudaMemsetAsync(d_first, 0x7f, 4ull * cells, stream));
    SAD_CUDA(cudaMemsetAsync(d_used, 0, 4ull * (J + 1), stream));
    TraceScope ts(ctx, SAD_STAGE_PROG, stream);
    // profiles: every bucket's from its alignment, the ancestor's as one member
    Arena arena{ctx};
    void* bprof = nullptr;
    SAD_RET(arena.alloc(2ull * Ap * std::max<int64_t>(Wtot, 1), &bprof));
    SAD_CUDA(cudaMemsetAsync(bprof, 0, 2ull * Ap * std::max<int64_t>(Wtot, 1), stream));
    void* gprof = nullptr;
    SAD_RET(arena.alloc(2ull * Ap * std::max<int32_t>(lg, 1), &gprof));
    const unsigned blocks = (unsigned)std::min<int64_t>(((int64_t)std::max(npos, 1) * 32 + 255) / 256,
                                                        (int64_t)ctx->num_sms * 16);
    if (npos > 0) {
        k_bucket_profiles<<<blocks, 256, 0, stream>>>(S.res, S.pad_off, S.len, d_od, npos, d_pos, d_pb, d_coff, d_wd,
                                                      d_cm, Ap, (uint32_t*)bprof, ctx->d_status);
        SAD_LAUNCHED();
    }
    k_leaf_profiles<<<1, 32, 0, stream>>>(S.res, S.pad_off, S.len, (const int32_t*)(w + o_ga), 1,
                                          (const int64_t*)(w + o_gpos), Ap, (uint16_t*)gprof);
    SAD_LAUNCHED();
    // every non-empty bucket against the ancestor (its columns are the rows)
    std::vector<int32_t*> map_ptr((size_t)p, nullptr);
    ProgArgs base{};
    base.Ap = Ap;
    base.alphabet = A;
    base.go = gap_open;
    base.ge = gap_extend;
    base.subst = (const int8_t*)(w + o_sub);
    base.scores = d_sc;
    base.widths = (int32_t*)(w + o_mw);
    base.status = ctx->d_status;
    base.spin_limit = ctx->prog_spin_limit > 0 ? ctx->prog_spin_limit : kSpinLimit;
    const int64_t budget = (int64_t)1 << 30;
    int64_t glue_jobs = 0;
    for (int32_t b = 0; b < p; b++) glue_jobs += bo[b + 1] > bo[b] ? 1 : 0;
    void* pin = nullptr;
    SAD_RET(pinned(ctx, sizeof(ProgJob) * (size_t)std::max<int64_t>(glue_jobs, 1), stream, &pin));
    ProgJob* pin_jobs = (ProgJob*)pin;
    const int glue_c = pick_columns(ctx, glue_jobs, lg);
    for (int32_t b0 = 0; b0 < p;) {
        Batch bt;
        bt.C = glue_c;
        int32_t b1 = b0;
        for (; b1 < p; b1++) {
            const int32_t nb = bo[b1 + 1] - bo[b1];
            if (nb == 0) continue;
            if (!bt.jobs.empty() && bt.bytes_with(wd[b1], lg) > budget) break;
            ProgJob jb{};
            jb.prof_p = (const uint16_t*)bprof + col_off[b1] * Ap;
            jb.prof_q = (const uint16_t*)gprof;
            void* pr = nullptr;
            SAD_RET(arena.alloc(2ull * Ap * ((int64_t)wd[b1] + lg), &pr));
            jb.prof_r = (uint16_t*)pr;
            void* mp = nullptr;
            SAD_RET(arena.alloc(4ull * ((int64_t)wd[b1] + lg), &mp));
            jb.map = (int32_t*)mp;
            jb.m = wd[b1];
            jb.n = lg;
            jb.np = nb;
            jb.nq = 1;
            jb.merge = b1;
            SAD_RET(bt.add(jb, smax, cmax));
            map_ptr[b1] = jb.map;
        }
        SAD_RET(run_batch(ctx, bt, base, stream, pin_jobs));
        if (b1 < p) SAD_CUDA(cudaStreamSynchronize(stream));  // the next batch reuses the workspace and pinned table
        b0 = b1;
    }
    // anchors, the joined layout, the joined column of every bucket column
    int32_t** d_mp = (int32_t**)(w + o_mp);
    SAD_CUDA(cudaMemcpyAsync(d_mp, map_ptr.data(), 8ull * p, cudaMemcpyHostToDevice, stream));
    const unsigned cblocks = (unsigned)std::min<int64_t>((std::max<int64_t>(Wtot, 1) + 255) / 256,
                                                         (int64_t)ctx->num_sms * 16);
    if (Wtot > 0) {
        k_anchors<<<cblocks, 256, 0, stream>>>(p, d_coff, d_mp, lg, d_an, d_ins, d_first);
        SAD_LAUNCHED();
    }
    k_glue_layout<<<1, 1024, 0, stream>>>(p, lg, d_ins, (int32_t*)(w + o_sizes), d_start);
    SAD_LAUNCHED();
    if (Wtot > 0) {
        k_joined<<<cblocks, 256, 0, stream>>>(p, d_coff, d_an, d_start, d_first, d_join);
        SAD_LAUNCHED();
    }
    // drop the columns without residues
    if (npos > 0) {
        k_glue_residues<<<blocks, 256, 0, stream>>>(0, d_od, npos, S.len, d_pos, d_pb, d_coff, d_wd, d_cm, d_join,
                                                    d_used, nullptr, nullptr);
        SAD_LAUNCHED();
    }
    k_scan_one<<<1, 1024, 0, stream>>>(d_used, J, d_renum);
    SAD_LAUNCHED();
    if (npos > 0) {
        k_glue_residues<<<blocks, 256, 0, stream>>>(1, d_od, npos, S.len, d_pos, d_pb, d_coff, d_wd, d_cm, d_join,
                                                    nullptr, d_renum, d_gcm);
        SAD_LAUNCHED();
    }
    // outputs
    const cudaMemcpyKind k_out = mem == SAD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    SAD_CUDA(cudaMemcpyAsync(global_width, d_renum + J, 4, k_out, stream));
    if (mem == SAD_MEM_HOST) {
        SAD_CUDA(cudaMemcpyAsync(ga_scores, d_sc, 8ull * p, cudaMemcpyDeviceToHost, stream));
        if (Wtot > 0) SAD_CUDA(cudaMemcpyAsync(anchors, d_an, 4ull * Wtot, cudaMemcpyDeviceToHost, stream));
        if (T_res > 0) SAD_CUDA(cudaMemcpyAsync(global_colmap, d_gcm, 4ull * T_res, cudaMemcpyDeviceToHost, stream));
    }
    SAD_RET(status_check(ctx, stream));
    return SAD_OK;
}

extern "C" int sad_progressive_wait_limit(sad_ctx* ctx_in, int64_t polls) {
    using namespace sad;
    clear_error();
    SAD_CHECK(polls >= 0, SAD_EINVAL, "polls = %lld < 0", (long long)polls);
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->prog_spin_limit = polls;
    return SAD_OK;
}

extern "C" int sad_progressive_columns(sad_ctx* ctx_in, int32_t columns) {
    using namespace sad;
    clear_error();
    SAD_CHECK(columns >= 0 && columns <= 2, SAD_EINVAL, "columns = %d (0, 1 or 2)", columns);
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->prog_columns = columns;
    return SAD_OK;
}
