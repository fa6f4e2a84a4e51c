// Stage 2 of Sample-Align-D: all-pairs global alignment scores with affine
// gaps inside every bucket (the "align sequences in each processor" step of
// the algorithm box; Section 2.3.3 lets each processor run any sequential
// aligner, and a progressive aligner starts from exactly these pair scores).
//
// Recurrences (Gotoh), gap run of length g = go + g*ge, go, ge <= 0:
//   E(i,j) = max(E(i,j-1) + ge, H(i,j-1) + go + ge)      gap in x (consumes y_j)
//   F(i,j) = max(F(i-1,j) + ge, H(i-1,j) + go + ge)      gap in y (consumes x_i)
//   H(i,j) = max(H(i-1,j-1) + s(x_i, y_j), E(i,j), F(i,j))
//   H(0,0) = 0, H(i,0) = go + i ge, H(0,j) = go + j ge, E(i,0) = F(0,j) = -inf.
// With go <= 0 this equals the best score over alignments where every maximal
// gap run pays one opening (a run in x may directly follow a run in y).
//
// GPU mapping. A CTA owns one query x_q of a bucket and keeps its profile
// prof[a][i] = s(a, x_i) in shared memory; groups of G lanes each take one
// subject y_v at a time. Lane t of a group holds R consecutive query rows in
// registers (H, H+go+ge and E per row) and sweeps the subject's columns; the
// bottom row's H and F and the column letter move to lane t+1 by a warp
// shuffle each step, so the group is a diagonal wavefront of G x R rows.
// Queries longer than G*R rows are processed in strips; a strip's bottom row
// is handed to the next strip through a per-group boundary buffer in global
// memory. Per cell: two add-max (DPX), one add, one 3-way max (DPX), one add.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "gotoh_stage.cuh"
#include "sad_internal.cuh"

namespace sad {

namespace {

constexpr int32_t NEG = -(1 << 30);
constexpr int32_t kChunkSubjects = 64;  // subjects per packed work item (at most)

// everything a Gotoh kernel needs besides its work items
struct GotohArgs {
    const uint8_t* res;        // padded residues
    const int64_t* pad_off;    // padded starts
    const int32_t* len;        // lengths
    const int32_t* order;      // CSR members (sequence ids)
    const int32_t* bucket_off; // p+1
    const int32_t* srt;        // per bucket: sorted position -> local CSR position
    const int64_t* score_off;  // p+1
    int32_t* scores;
    int32_t* scratch;          // strip boundaries: per group 2*(max_n+1) ints
    int64_t scratch_stride;    // ints per group
    const int8_t* subst;       // alphabet x alphabet (device)
    int32_t alphabet;
    int32_t go, ge;
    int32_t prof_stride;       // bytes per profile row (>= padded query length)
    int32_t G;                 // lanes per group
    int32_t bias;              // packed form: stored DP value = true value + bias
};

__device__ __forceinline__ int64_t tri_pos(int64_t u, int64_t v, int64_t nb) {
    return u * nb - u * (u - 1) / 2 + (v - u);
}

// Load R profile bytes and widen them to int32.
template <int R>
__device__ __forceinline__ void load_profile(const int8_t* p, int32_t (&s)[R]) {
    static_assert(R % 4 == 0, "R must be a multiple of 4");
    uint32_t ww[R / 4];
    if constexpr (R % 16 == 0) {
#pragma unroll
        for (int q = 0; q < R / 16; q++) {
            const uint4 w = *(const uint4*)(p + 16 * q);
            ww[4 * q] = w.x; ww[4 * q + 1] = w.y; ww[4 * q + 2] = w.z; ww[4 * q + 3] = w.w;
        }
    } else if constexpr (R % 8 == 0) {
#pragma unroll
        for (int q = 0; q < R / 8; q++) {
            const uint2 w = *(const uint2*)(p + 8 * q);
            ww[2 * q] = w.x; ww[2 * q + 1] = w.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < R / 4; q++) ww[q] = *(const uint32_t*)(p + 4 * q);
    }
#pragma unroll
    for (int t = 0; t < R; t++) s[t] = (int32_t)(int8_t)(ww[t >> 2] >> (8 * (t & 3)));
}

// One group aligns query (profile in smem, length m) against subject y (length n,
// n may be 0 for an idle group whose lanes still join the warp's shuffles).
// Returns the score in every lane of the group (valid when active).
template <int R>
__device__ int32_t align_group(const int8_t* __restrict__ prof, int32_t m, const uint8_t* __restrict__ y,
                               int32_t n, int32_t nsteps_warp, const GotohArgs& a,
                               int32_t* __restrict__ bnd, int lane, unsigned gmask) {
    const int G = a.G;
    const int32_t goe = a.go + a.ge, ge = a.ge, go = a.go;
    const int32_t strip_h = G * R;
    const int32_t strips = (m + strip_h - 1) / strip_h;
    int32_t result = 0;
    for (int32_t s = 0; s < strips; s++) {
        const int32_t row0 = s * strip_h + lane * R;   // 0-based residue of my first row
        int32_t H[R], Hg[R], E[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            H[r] = go + (row0 + r + 1) * ge;
            Hg[r] = H[r] + goe;
            E[r] = NEG;
        }
        int32_t hdiag = (row0 == 0) ? 0 : go + row0 * ge;   // H(row0, 0)
        const int32_t top = s * strip_h;                      // DP row above the strip
        int32_t hin = 0, fin = NEG;                           // values from lane-1
        uint32_t yin = 0;
        uint32_t yword = 0;
        const bool last_strip = s == strips - 1;
        for (int32_t tau = 0; tau < nsteps_warp; tau++) {
            const int32_t j = tau - lane + 1;   // my 1-based column this step
            // lane 0 feeds the strip's top boundary and the subject letter
            // (reads stay inside the subject and its 16 zero bytes of padding)
            if (lane == 0 && tau < n) {
                if ((tau & 3) == 0) yword = *(const uint32_t*)(y + tau);
                yin = (yword >> (8 * (tau & 3))) & 0xffu;
                if (s == 0) {
                    hin = go + (tau + 1) * ge;
                    fin = NEG;
                } else {
                    hin = bnd[2 * (tau + 1)];
                    fin = bnd[2 * (tau + 1) + 1];
                }
            }
            int32_t hout = hin, fout = fin;
            if (j >= 1 && j <= n) {
                int32_t sc[R];
                load_profile<R>(prof + (int64_t)yin * a.prof_stride + row0, sc);
                int32_t hu = hin, fu = fin;
                int32_t hgu = hu + goe;
                int32_t hd = hdiag;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const int32_t e = __viaddmax_s32(E[r], ge, Hg[r]);
                    const int32_t f = __viaddmax_s32(fu, ge, hgu);
                    const int32_t h = __vimax3_s32(hd + sc[r], e, f);
                    hd = H[r];
                    H[r] = h;
                    Hg[r] = h + goe;
                    E[r] = e;
                    fu = f;
                    hgu = Hg[r];
                }
                hdiag = hin;
                hout = H[R - 1];
                fout = fu;
                if (!last_strip && lane == G - 1) {
                    bnd[2 * j] = hout;
                    bnd[2 * j + 1] = fout;
                }
            }
            // pass bottom row and letter one lane down the group
            hin = __shfl_up_sync(gmask, hout, 1, G);
            fin = __shfl_up_sync(gmask, fout, 1, G);
            yin = __shfl_up_sync(gmask, yin, 1, G);
        }
        __syncwarp(gmask);
        if (last_strip) {
            const int32_t rr = (m - 1) - s * strip_h;   // strip-local row of x_m
            const int owner = rr / R, rsel = rr % R;
            int32_t v = 0;
#pragma unroll
            for (int r = 0; r < R; r++) v = (r == rsel) ? H[r] : v;
            result = __shfl_sync(gmask, v, owner, G);
        }
        (void)top;
    }
    return result;
}

template <int R>
__global__ void __launch_bounds__(128)
k_gotoh_items(const GotohItem* __restrict__ items, int32_t n_items, int32_t* __restrict__ head,
              GotohArgs a) {
    extern __shared__ __align__(16) int8_t prof[];
    __shared__ int32_t item_sh;
    __shared__ int32_t next_sub;  // next subject of the item
    const int G = a.G;
    const int NG = blockDim.x / G;
    const int g = threadIdx.x / G;
    const int lane = threadIdx.x % G;
    const int warp_lane0 = (threadIdx.x & 31) - lane;   // first lane of my group in the warp
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << warp_lane0);
    int32_t it_idx = head ? -1 : (int32_t)blockIdx.x;
    for (;;) {
        if (head) {
            __syncthreads();
            if (threadIdx.x == 0) item_sh = atomicAdd(head, 1);
            __syncthreads();
            it_idx = item_sh;
        }
        if (it_idx >= n_items) break;
        const GotohItem it = items[it_idx];
        const int32_t b = it.bucket;
        const int32_t boff = a.bucket_off[b];
        const int32_t nb = a.bucket_off[b + 1] - boff;
        const int32_t uq = a.srt[boff + it.q];
        const int32_t xq = a.order[boff + uq];
        const int32_t m = a.len[xq];
        const uint8_t* x = a.res + a.pad_off[xq];
        // profile rows prof[c][i] = s(c, x_i); rows past m are zero
        const int32_t mp = a.prof_stride;
        for (int32_t t = threadIdx.x; t < a.alphabet * mp; t += blockDim.x) {
            const int32_t c = t / mp, i = t - c * mp;
            prof[t] = i < m ? a.subst[c * a.alphabet + x[i]] : (int8_t)0;
        }
        if (threadIdx.x == 0) next_sub = 0;
        __syncthreads();
        int32_t* bnd = a.scratch + ((int64_t)blockIdx.x * NG + g) * a.scratch_stride;
        // warps take the item's subjects from a shared counter, longest first (the
        // subjects are in ascending length order), so that no warp waits at the
        // next item's barrier for more than one subject of another
        const int32_t nsub = it.v1 - it.v0;
        const int gpw = 32 / G, gw = g % gpw;  // groups per warp, my group's index in it
        for (;;) {
            int32_t base = 0;
            if ((threadIdx.x & 31) == 0) base = atomicAdd(&next_sub, gpw);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= nsub) break;  // uniform in the warp
            const int32_t v = it.v1 - 1 - (base + gw);
            const bool have = v >= it.v0;
            int32_t uv = 0, ys = 0, n = 0;
            if (have) {
                uv = a.srt[boff + v];
                ys = a.order[boff + uv];
                n = a.len[ys];
            }
            // warp-uniform step count (every group of the warp joins each shuffle)
            const int32_t need = (have && m > 0 && n > 0) ? n + G - 1 : 0;
            const int32_t steps = (__reduce_max_sync(0xffffffffu, need) + 3) & ~3;
            int32_t score = 0;
            if (steps > 0) {
                score = align_group<R>(prof, m, a.res + a.pad_off[have ? ys : xq],
                                       (have && m > 0) ? n : 0, steps, a, bnd, lane, gmask);
            }
            if (have && lane == 0) {
                if (m == 0 && n == 0) score = 0;
                else if (m == 0) score = a.go + n * a.ge;
                else if (n == 0) score = a.go + m * a.ge;
                const int32_t lo = min(uq, uv), hi = max(uq, uv);
                a.scores[a.score_off[b] + tri_pos(lo, hi, nb)] = score;
            }
        }
        if (!head) break;
    }
}

using KernelFn = void (*)(const GotohItem*, int32_t, int32_t*, GotohArgs);

KernelFn kernel_for(int R) {
    switch (R) {
        case 4: return k_gotoh_items<4>;
        case 8: return k_gotoh_items<8>;
        case 12: return k_gotoh_items<12>;
        case 16: return k_gotoh_items<16>;
        case 20: return k_gotoh_items<20>;
        case 24: return k_gotoh_items<24>;
        case 32: return k_gotoh_items<32>;
        default: return nullptr;
    }
}

// ---------------------------------------------------------------------------
// Packed form: two queries of similar length share every instruction. Each
// 32-bit register holds the same DP cell of both problems (x1 in the low
// halfword, x2 in the high halfword). Every DP value is stored with a bias B
// (stored = true + B) chosen by the host so that each stored H, E, F lies in
// [0, 32767] and each addend keeps it there. Then a plain 32-bit add of a
// packed addend word a_hi * 2^16 + a_lo adds both halves exactly (a borrow
// from a negative low addend is cancelled by the carry of the low sum, and no
// half leaves [0, 65535]), and the compiler can spread those adds over the
// integer and FMA pipes, while the maxima are 16x2 DPX instructions. The
// sentinel for -inf is stored 0: every real stored E or F candidate is >= 0.
// Per row and column: 3 DPX instructions and 2 adds for 2 cells.
__device__ __forceinline__ uint32_t pk2(int32_t lo, int32_t hi) {
    return ((uint32_t)lo & 0xffffu) | ((uint32_t)hi << 16);
}

// the 32-bit addend that adds lo to the low and hi to the high halfword
__host__ __device__ __forceinline__ uint32_t addend2(int32_t lo, int32_t hi) {
    return (uint32_t)(hi * 65536 + lo);
}

__device__ __forceinline__ int32_t lo16(uint32_t v) { return (int32_t)(v & 0xffffu); }
__device__ __forceinline__ int32_t hi16(uint32_t v) { return (int32_t)(v >> 16); }

// Words per lane chunk of the packed profile: R rows padded so that a chunk is
// an odd number of 16-byte units; the 8 lanes of one 128-bit load phase then
// hit 8 different 16-byte bank groups.
template <int R>
__host__ __device__ constexpr int rpad() {
    return ((R / 4) % 2 == 0) ? R + 4 : R;
}

template <int R>
__device__ __forceinline__ void load_profile32(const uint32_t* p, uint32_t (&s)[R]) {
    if constexpr (R % 4 == 0) {
#pragma unroll
        for (int q = 0; q < R / 4; q++) {
            const uint4 w = *(const uint4*)(p + 4 * q);
            s[4 * q] = w.x; s[4 * q + 1] = w.y; s[4 * q + 2] = w.z; s[4 * q + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < R; q++) s[q] = p[q];
    }
}

// One lane step over C consecutive subject columns j1..j1+C-1 of the lane's R
// rows (CC <= C of them present): sub-step s moves row s - c to column j1 + c
// for every chain c, so the C chains F -> H -> H+go+ge are independent and
// interleave, and every chain finds its left neighbour (chain c - 1, same row)
// already one sub-step ahead. The instruction count per cell is that of one
// column; no branch sits inside the unrolled rows. Values are biased (see the
// packed-form note): t = H(i-1,j-1) + s and H + go + ge are plain 32-bit adds
// (goe_w = addend2(go + ge, go + ge)); ge2 = pk2(ge, ge) feeds the DPX add-max.
template <int R, int CC>
__device__ __forceinline__ void pair16_columns(const uint32_t* __restrict__ prof, int64_t stride, int64_t chunk,
                                               uint32_t letters, uint32_t (&H)[R], uint32_t (&Hg)[R],
                                               uint32_t (&E)[R], const uint32_t* hin, const uint32_t* fin,
                                               uint32_t hdiag, uint32_t ge2, uint32_t goe_w,
                                               uint32_t* hout, uint32_t* fout) {
    uint32_t sc[CC][R];
#pragma unroll
    for (int c = 0; c < CC; c++) load_profile32<R>(prof + (int64_t)((letters >> (8 * c)) & 0xffu) * stride + chunk, sc[c]);
    uint32_t fu[CC], hgu[CC], hd[CC];
#pragma unroll
    for (int c = 0; c < CC; c++) {
        fu[c] = fin[c];
        hgu[c] = hin[c] + goe_w;
        hd[c] = c == 0 ? hdiag : hin[c - 1];
    }
#pragma unroll
    for (int s = 0; s < R + CC - 1; s++) {
        // the order inside a sub-step is free; chain 0 first ends the old H(r)'s
        // life before chain 1 writes the new one (0.8 % faster than chain 1 first)
#pragma unroll
        for (int c = 0; c < CC; c++) {
            const int r = s - c;
            if (r < 0 || r >= R) continue;
            const uint32_t e = __viaddmax_s16x2(E[r], ge2, Hg[r]);
            const uint32_t f = __viaddmax_s16x2(fu[c], ge2, hgu[c]);
            const uint32_t h = __vimax3_s16x2(hd[c] + sc[c][r], e, f);
            hd[c] = H[r];
            H[r] = h;
            Hg[r] = h + goe_w;
            E[r] = e;
            fu[c] = f;
            hgu[c] = Hg[r];
            if (r == R - 1) {
                hout[c] = h;
                fout[c] = f;
            }
        }
    }
}

// pair16_columns for the cnt <= C columns present (the last chunk of a subject).
template <int R, int C>
__device__ __forceinline__ void pair16_chunk(int32_t cnt, const uint32_t* __restrict__ prof, int64_t stride,
                                             int64_t chunk, uint32_t letters, uint32_t (&H)[R], uint32_t (&Hg)[R],
                                             uint32_t (&E)[R], const uint32_t* hin, const uint32_t* fin,
                                             uint32_t hdiag, uint32_t ge2, uint32_t goe_w,
                                             uint32_t* hout, uint32_t* fout) {
    if (cnt == C) {
        pair16_columns<R, C>(prof, stride, chunk, letters, H, Hg, E, hin, fin, hdiag, ge2, goe_w, hout, fout);
    } else if (C > 1 && cnt == 1) {
        pair16_columns<R, 1>(prof, stride, chunk, letters, H, Hg, E, hin, fin, hdiag, ge2, goe_w, hout, fout);
    } else if (C > 2 && cnt == 2) {
        pair16_columns<R, (C > 2 ? 2 : 1)>(prof, stride, chunk, letters, H, Hg, E, hin, fin, hdiag, ge2, goe_w,
                                           hout, fout);
    } else if (C > 3 && cnt == 3) {
        pair16_columns<R, (C > 3 ? 3 : 1)>(prof, stride, chunk, letters, H, Hg, E, hin, fin, hdiag, ge2, goe_w,
                                           hout, fout);
    }
}

// One group aligns the query pair (packed profile in smem, lengths m1, m2)
// against subject y of length n, with C subject columns per lane step (one
// chain per column, see pair16_columns), in strips of G R rows; writes the two
// scores to r1, r2 (valid for m1 >= 1 and m2 >= 1). In step tau lane t takes columns
// C(tau - t) + 1 .. C(tau - t) + C; the last step of a subject whose length is
// not a multiple of C takes the remaining columns. A step hands C (H, F) pairs
// and C letters (one 32-bit word) to the next lane.
template <int R, int C>
__device__ void align_pair16c(const uint32_t* __restrict__ prof, int32_t m1, int32_t m2,
                              const uint8_t* __restrict__ y, int32_t n, int32_t nsteps_warp,
                              const GotohArgs& a, int32_t* __restrict__ bnd, int lane, unsigned gmask,
                              int32_t* r1, int32_t* r2) {
    static_assert(C >= 1 && C <= 4, "up to four letters travel in one word");
    const int G = a.G;
    const int32_t go = a.go, ge = a.ge;
    const int32_t B = a.bias;  // stored = true + B
    const uint32_t ge2 = pk2(ge, ge), goe_w = addend2(go + ge, go + ge);
    const int32_t strip_h = G * R;
    const int32_t mrows = max(m1, m2);
    const int32_t strips = (mrows + strip_h - 1) / strip_h;
    const int32_t nchunks = (n + C - 1) / C;
    for (int32_t s = 0; s < strips; s++) {
        const int32_t row0 = s * strip_h + lane * R;
        uint32_t H[R], Hg[R], E[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int32_t b0 = go + (row0 + r + 1) * ge + B;
            H[r] = pk2(b0, b0);
            Hg[r] = H[r] + goe_w;
            E[r] = 0u;
        }
        const int32_t d0 = ((row0 == 0) ? 0 : go + row0 * ge) + B;
        uint32_t hdiag = pk2(d0, d0);  // H(row0 - 1, j1 - 1)
        uint32_t hin[C], fin[C], yin = 0;
#pragma unroll
        for (int c = 0; c < C; c++) {
            hin[c] = 0u;
            fin[c] = 0u;
        }
        const bool last_strip = s == strips - 1;
        const int64_t chunk = (int64_t)(row0 / R) * rpad<R>();
        for (int32_t tau = 0; tau < nsteps_warp; tau++) {
            if (lane == 0 && tau < nchunks) {
                // letters y_{C tau + 1 ..}: zero bytes past the subject are padding
                const uint8_t* yp = y + (int64_t)C * tau;
                yin = 0;
#pragma unroll
                for (int c = 0; c < C; c++) yin |= (uint32_t)yp[c] << (8 * c);
                const int32_t j1 = C * tau + 1;
#pragma unroll
                for (int c = 0; c < C; c++) {
                    if (s == 0) {
                        const int32_t b = go + (j1 + c) * ge + B;
                        hin[c] = pk2(b, b);
                        fin[c] = 0u;
                    } else if (j1 + c <= n) {  // the buffer holds columns 0..n
                        hin[c] = (uint32_t)bnd[2 * (j1 + c)];
                        fin[c] = (uint32_t)bnd[2 * (j1 + c) + 1];
                    }
                }
            }
            const int32_t cidx = tau - lane;
            const int32_t j1 = C * cidx + 1;
            uint32_t hout[C], fout[C];
#pragma unroll
            for (int c = 0; c < C; c++) {
                hout[c] = hin[c];
                fout[c] = fin[c];
            }
            if (cidx >= 0 && j1 <= n) {
                const int32_t cnt = min(C, n - j1 + 1);
                pair16_chunk<R, C>(cnt, prof, a.prof_stride, chunk, yin, H, Hg, E, hin, fin, hdiag, ge2, goe_w, hout,
                                   fout);
                // the last column's value from above is the next step's diagonal
                // (constant indices keep the arrays in registers)
#pragma unroll
                for (int c = 0; c < C; c++)
                    if (c == cnt - 1) hdiag = hin[c];
                if (!last_strip && lane == G - 1) {
#pragma unroll
                    for (int c = 0; c < C; c++) {
                        if (c < cnt) {
                            bnd[2 * (j1 + c)] = (int32_t)hout[c];
                            bnd[2 * (j1 + c) + 1] = (int32_t)fout[c];
                        }
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < C; c++) {
                hin[c] = __shfl_up_sync(gmask, hout[c], 1, G);
                fin[c] = __shfl_up_sync(gmask, fout[c], 1, G);
            }
            yin = __shfl_up_sync(gmask, yin, 1, G);
        }
        __syncwarp(gmask);
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int32_t mq = q == 0 ? m1 : m2;
            if (mq >= 1 && (mq - 1) / strip_h == s) {
                const int32_t rr = (mq - 1) - s * strip_h;
                const int owner = rr / R, rsel = rr % R;
                uint32_t v = 0;
#pragma unroll
                for (int r = 0; r < R; r++) v = (r == rsel) ? H[r] : v;
                v = __shfl_sync(gmask, v, owner, G);
                if (q == 0) *r1 = lo16(v) - B;
                else *r2 = hi16(v) - B;
            }
        }
    }
}

// The query pair against every subject of one group (bucket positions vfirst,
// vfirst + vstep, ... below vend, in length order) in a single wavefront: the
// subjects' columns follow each other in chunks of up to C columns that never
// span two subjects, and every lane walks the same chunk sequence one step
// behind the lane above, so the wavefront fills and drains once per group
// instead of once per subject. A lane resets its rows to column 0 when it
// enters a subject; the lane that holds a query's last row writes that query's
// score when it finishes the subject's last column. Only for query pairs within
// one strip (1 <= max(m1, m2) <= G R); pairs with an empty query or subject are
// scored beforehand by lane 0.
// The group's non-empty subjects go to shared memory first (slots g, g + NG,
// ... of subj_pos / subj_off), so that moving to the next subject inside the
// wavefront loop is an index step and one shared load.
// With C = 2 columns per step a subject of odd length starts one column early,
// at a virtual column 0 that the recurrence itself fills with the boundary
// values: the lane enters it with H = E = the stored sentinel 0 and
// Hg = go + ge (so the diagonal and horizontal candidates stay below every
// boundary value, which the bias guarantees to exceed the largest substitution
// score), and the vertical candidate down the column, started from H(0, 0),
// is go + i ge, the boundary H(i, 0). Every chunk then holds two columns, and
// no lane runs a one-column step while the others of its warp run two.
template <int R, int C>
__device__ void stream_pair16(const uint32_t* __restrict__ prof, int32_t m1, int32_t m2, int32_t u1, int32_t u2,
                              int32_t b, int32_t boff, int32_t nb, int32_t vfirst, int32_t vend, int32_t vstep,
                              int2* __restrict__ subj_pos, long long* __restrict__ subj_off, const GotohArgs& a,
                              int lane, unsigned gmask) {
    const int G = a.G;
    const int32_t go = a.go, ge = a.ge;
    const int32_t B = a.bias;  // stored = true + B
    const uint32_t ge2 = pk2(ge, ge), goe_w = addend2(go + ge, go + ge);
    int32_t* scores = a.scores + a.score_off[b];
    auto subject = [&](int32_t v, int32_t* uv, int32_t* ys) {
        *uv = a.srt[boff + v];
        *ys = a.order[boff + *uv];
        return a.len[*ys];
    };
    // empty queries or subjects are scored here; the rest are listed in order
    int32_t nchunks = 0, nsubj = 0;
    for (int32_t v = vfirst; v < vend; v += vstep) {
        int32_t uv, ys;
        const int32_t n = subject(v, &uv, &ys);
        nchunks += (n + C - 1) / C;
        if (n > 0) {
            if (lane == 0) {
                subj_pos[nsubj * vstep] = make_int2(uv, n);
                subj_off[nsubj * vstep] = a.pad_off[ys];
            }
            nsubj++;
        }
        if (lane == 0) {
            const int32_t mq[2] = {m1, m2}, uq[2] = {u1, u2};
#pragma unroll
            for (int q = 0; q < 2; q++) {
                if (uq[q] < 0 || (mq[q] > 0 && n > 0)) continue;
                const int32_t sc = (mq[q] == 0 && n == 0) ? 0 : go + (mq[q] + n) * ge;
                scores[tri_pos(min(uq[q], uv), max(uq[q], uv), nb)] = sc;
            }
        }
    }
    __syncwarp(gmask);
    if (max(m1, m2) == 0) return;  // every score was written above (uniform over the CTA)
    const int32_t steps = __reduce_max_sync(0xffffffffu, nchunks > 0 ? nchunks + G - 1 : 0);
    if (steps == 0) return;
    // this lane's cursor: subject ordinal k, its length, CSR position, residues, next column
    // (0: the virtual column of an odd-length subject)
    constexpr bool kVirt = C == 2;
    int32_t ck = -1, cn = 0, cuv = 0, cj = 1;
    const uint8_t* cy = nullptr;
    auto advance = [&]() {
        ck++;
        if (ck < nsubj) {
            const int2 e = subj_pos[ck * vstep];
            cuv = e.x;
            cn = e.y;
            cy = a.res + subj_off[ck * vstep];
        }
        cj = kVirt ? 1 - (cn & 1) : 1;
    };
    advance();
    const int32_t row0 = lane * R;
    const int64_t chunk = (int64_t)lane * rpad<R>();
    const int own1 = m1 >= 1 ? (m1 - 1) / R : -1, sel1 = m1 >= 1 ? (m1 - 1) % R : 0;
    const int own2 = (u2 >= 0 && m2 >= 1) ? (m2 - 1) / R : -1, sel2 = m2 >= 1 ? (m2 - 1) % R : 0;
    uint32_t H[R], Hg[R], E[R];
    uint32_t hdiag = 0;
    uint32_t hin[C], fin[C], yin = 0;
#pragma unroll
    for (int c = 0; c < C; c++) {
        hin[c] = 0u;
        fin[c] = 0u;
    }
    for (int32_t tau = 0; tau < steps; tau++) {
        const bool live = tau >= lane && ck < nsubj;
        if (lane == 0 && live) {
            if constexpr (kVirt) {
                // columns cj, cj + 1 (letters y[cj - 1], y[cj]; the virtual column
                // takes any letter, here y[0]); the top row H(0, j) = go + j ge
                // (H(0, 0) = 0), stored values below 2^16 so that pk2(x, x) = x 0x10001
                yin = (uint32_t)cy[max(cj - 1, 0)] | ((uint32_t)cy[cj] << 8);
                hin[1] = (uint32_t)(go + (cj + 1) * ge + B) * 0x10001u;
                hin[0] = cj == 0 ? (uint32_t)B * 0x10001u : hin[1] - (uint32_t)ge * 0x10001u;
                fin[0] = 0u;
                fin[1] = 0u;
            } else {
                yin = 0;
#pragma unroll
                for (int c = 0; c < C; c++) {
                    yin |= (uint32_t)cy[cj - 1 + c] << (8 * c);  // bytes past the subject are zero padding
                    const int32_t bnd0 = go + (cj + c) * ge + B;
                    hin[c] = pk2(bnd0, bnd0);
                    fin[c] = 0u;
                }
            }
        }
        uint32_t hout[C], fout[C];
#pragma unroll
        for (int c = 0; c < C; c++) {
            hout[c] = hin[c];
            fout[c] = fin[c];
        }
        if (live) {
            if (kVirt && cj == 0) {  // entering an odd-length subject: the sentinel column -1
                const uint32_t hg0 = pk2(go + ge, go + ge);
#pragma unroll
                for (int r = 0; r < R; r++) {
                    H[r] = 0u;
                    Hg[r] = hg0;
                    E[r] = 0u;
                }
                hdiag = 0u;
            } else if (cj == 1) {  // entering a subject: column 0 of my rows
                // recomputed here on purpose: hoisting these 2R loop-invariant values
                // out of the loop would hold them in registers for the whole stream
                int32_t base;
                asm volatile("mov.b32 %0, %1;" : "=r"(base) : "r"(go + row0 * ge + B));
                const uint32_t ge_w = addend2(ge, ge);
                uint32_t h = pk2(base, base);
#pragma unroll
                for (int r = 0; r < R; r++) {
                    h = h + ge_w;  // go + (row0 + r + 1) ge
                    H[r] = h;
                    Hg[r] = h + goe_w;
                    E[r] = 0u;
                }
                hdiag = row0 == 0 ? pk2(B, B) : pk2(base, base);
            }
            const int32_t cnt = kVirt ? C : min(C, cn - cj + 1);
            if constexpr (kVirt)
                pair16_columns<R, C>(prof, a.prof_stride, chunk, yin, H, Hg, E, hin, fin, hdiag, ge2, goe_w, hout,
                                     fout);
            else
                pair16_chunk<R, C>(cnt, prof, a.prof_stride, chunk, yin, H, Hg, E, hin, fin, hdiag, ge2, goe_w,
                                   hout, fout);
#pragma unroll
            for (int c = 0; c < C; c++)
                if (c == cnt - 1) hdiag = hin[c];
            if (cj + cnt - 1 == cn) {  // the subject's last column
                if (lane == own1 || lane == own2) {
                    uint32_t v1 = 0, v2 = 0;
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        v1 = (r == sel1) ? H[r] : v1;
                        v2 = (r == sel2) ? H[r] : v2;
                    }
                    if (lane == own1) scores[tri_pos(min(u1, cuv), max(u1, cuv), nb)] = lo16(v1) - B;
                    if (lane == own2) scores[tri_pos(min(u2, cuv), max(u2, cuv), nb)] = hi16(v2) - B;
                }
                advance();
            } else {
                cj += cnt;
            }
        }
#pragma unroll
        for (int c = 0; c < C; c++) {
            hin[c] = __shfl_up_sync(gmask, hout[c], 1, G);
            fin[c] = __shfl_up_sync(gmask, fout[c], 1, G);
        }
        yin = __shfl_up_sync(gmask, yin, 1, G);
    }
}

// Columns per lane step of the packed kernel for R rows per lane (a build
// option: SAD_PAIR_COLS_SMALL for R <= 20, SAD_PAIR_COLS_LARGE above).
#ifndef SAD_PAIR_COLS_SMALL
#define SAD_PAIR_COLS_SMALL 2
#endif
#ifndef SAD_PAIR_COLS_LARGE
#define SAD_PAIR_COLS_LARGE 2
#endif
template <int R>
__host__ __device__ constexpr int pair_cols() {
    return R <= 20 ? SAD_PAIR_COLS_SMALL : SAD_PAIR_COLS_LARGE;
}

// Work item (bucket, query pair qp, subjects [v0, v1)): queries are the
// members at length-order positions 2qp and 2qp+1 of the bucket.
// kStream: every query pair of the launch lies within one strip, and each
// group streams its subjects through one wavefront (stream_pair16); otherwise
// one wavefront per subject, in strips (the two forms are separate kernels: in
// one body their register needs add up).
// Occupancy: 4 CTAs (16 warps) per SM up to R = 20 rows per lane, 3 above
// (the R = 32 body fits 167 registers without spilling; at 2 CTAs per SM the
// two interleaved column chains per lane left the DPX pipe waiting on
// dependencies: N = 2000 scores 2.68 -> 2.57 ms with 3).
template <int R, bool kStream>
__global__ void __launch_bounds__(128, (R <= 20) ? 4 : 3)
k_gotoh_pair16(const GotohItem* __restrict__ items, int32_t n_items, int32_t* __restrict__ head,
               GotohArgs a) {
    extern __shared__ __align__(16) uint32_t prof32[];
    __shared__ int32_t item_sh;
    __shared__ int32_t next_sub;                    // next subject of the item (per-subject form)
    __shared__ int2 subj_pos[kChunkSubjects];       // streamed subjects: (CSR position, length)
    __shared__ long long subj_off[kChunkSubjects];  // and their padded residue offsets
    const int G = a.G;
    const int NG = blockDim.x / G;
    const int g = threadIdx.x / G;
    const int lane = threadIdx.x % G;
    const int warp_lane0 = (threadIdx.x & 31) - lane;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << warp_lane0);
    int32_t* bnd = a.scratch ? a.scratch + ((int64_t)blockIdx.x * NG + g) * a.scratch_stride : nullptr;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item_sh = atomicAdd(head, 1);
        __syncthreads();
        const int32_t it_idx = item_sh;
        if (it_idx >= n_items) break;
        const GotohItem it = items[it_idx];
        const int32_t b = it.bucket;
        const int32_t boff = a.bucket_off[b];
        const int32_t nb = a.bucket_off[b + 1] - boff;
        const int32_t u1 = a.srt[boff + 2 * it.q];
        const int32_t u2 = (2 * it.q + 1 < nb) ? a.srt[boff + 2 * it.q + 1] : -1;
        const int32_t x1 = a.order[boff + u1];
        const int32_t x2 = u2 >= 0 ? a.order[boff + u2] : x1;
        const int32_t m1 = a.len[x1];
        const int32_t m2 = u2 >= 0 ? a.len[x2] : 0;
        const uint8_t* q1 = a.res + a.pad_off[x1];
        const uint8_t* q2 = a.res + a.pad_off[x2];
        // profile words of letter c: lane chunks of R rows, each padded to rpad<R>() words
        const int32_t mp = a.prof_stride;
        for (int32_t t = threadIdx.x; t < a.alphabet * mp; t += blockDim.x) {
            const int32_t c = t / mp, w = t - c * mp;
            const int32_t chunk = w / rpad<R>(), off = w - chunk * rpad<R>();
            const int32_t i = chunk * R + off;
            const bool row = off < R;
            const int32_t lo = (row && i < m1) ? a.subst[c * a.alphabet + q1[i]] : 0;
            const int32_t hi = (row && i < m2) ? a.subst[c * a.alphabet + q2[i]] : 0;
            prof32[t] = addend2(lo, hi);
        }
        if (threadIdx.x == 0) next_sub = 0;
        __syncthreads();
        const int32_t mrows = max(m1, m2);
        if constexpr (kStream) {
            // one wavefront over all of the group's subjects (1 <= mrows <= G R is
            // guaranteed by the host; mrows = 0 scores every pair in the pre-pass)
            stream_pair16<R, pair_cols<R>()>(prof32, m1, m2, u1, u2, b, boff, nb, it.v0 + g, it.v1, NG,
                                             subj_pos + g, subj_off + g, a, lane, gmask);
            continue;
        }
        // warps take the item's subjects from a shared counter, longest first (the
        // subjects are in ascending length order), so that no warp waits at the
        // next item's barrier for more than one subject of another
        const int32_t nsub = it.v1 - it.v0;
        const int gpw = 32 / G, gw = g % gpw;  // groups per warp, my group's index in it
        for (;;) {
            int32_t base = 0;
            if ((threadIdx.x & 31) == 0) base = atomicAdd(&next_sub, gpw);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= nsub) break;  // uniform in the warp
            const int32_t v = it.v1 - 1 - (base + gw);
            const bool have = v >= it.v0;
            int32_t uv = 0, ys = 0, n = 0;
            if (have) {
                uv = a.srt[boff + v];
                ys = a.order[boff + uv];
                n = a.len[ys];
            }
            constexpr int kC = pair_cols<R>();
            const int32_t need = (have && mrows > 0 && n > 0) ? (n + kC - 1) / kC + G - 1 : 0;
            const int32_t steps = (__reduce_max_sync(0xffffffffu, need) + 3) & ~3;
            int32_t s1 = 0, s2 = 0;
            if (steps > 0) {
                const uint8_t* yp = a.res + a.pad_off[have ? ys : x1];
                const int32_t ny = (have && mrows > 0) ? n : 0;
                align_pair16c<R, kC>(prof32, m1, m2, yp, ny, steps, a, bnd, lane, gmask, &s1, &s2);
            }
            if (have && lane == 0) {
                const int32_t mq[2] = {m1, m2};
                int32_t sc[2] = {s1, s2};
                const int32_t uq[2] = {u1, u2};
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    if (uq[q] < 0) continue;
                    if (mq[q] == 0 && n == 0) sc[q] = 0;
                    else if (mq[q] == 0) sc[q] = a.go + n * a.ge;
                    else if (n == 0) sc[q] = a.go + mq[q] * a.ge;
                    const int32_t lo = min(uq[q], uv), hi = max(uq[q], uv);
                    a.scores[a.score_off[b] + tri_pos(lo, hi, nb)] = sc[q];
                }
            }
        }
    }
}

KernelFn pair16_kernel_for(int R, bool stream) {
    switch (R) {
        case 8: return stream ? k_gotoh_pair16<8, true> : k_gotoh_pair16<8, false>;
        case 12: return stream ? k_gotoh_pair16<12, true> : k_gotoh_pair16<12, false>;
        case 16: return stream ? k_gotoh_pair16<16, true> : k_gotoh_pair16<16, false>;
        case 20: return stream ? k_gotoh_pair16<20, true> : k_gotoh_pair16<20, false>;
        case 24: return stream ? k_gotoh_pair16<24, true> : k_gotoh_pair16<24, false>;
        case 32: return stream ? k_gotoh_pair16<32, true> : k_gotoh_pair16<32, false>;
        default: return nullptr;
    }
}

}  // namespace

// Host-side plan: per bucket, members sorted by length (ascending, ties by
// local position); a work item is one query row with a range of subjects
// that are at least as long.
void plan_buckets(const std::vector<int32_t>& h_bo, const std::vector<int32_t>& h_order,
                  const std::vector<int32_t>& h_len, int32_t p, std::vector<int32_t>* srt,
                  std::vector<int64_t>* score_off) {
    const int32_t n = (int32_t)h_order.size();
    srt->assign((size_t)n, 0);
    score_off->assign((size_t)p + 1, 0);
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = h_bo[b + 1] - h_bo[b];
        (*score_off)[b + 1] = (*score_off)[b] + nb * (nb + 1) / 2;
    }
    int32_t maxlen = 0;
    for (int32_t t = 0; t < n; t++) maxlen = std::max(maxlen, h_len[h_order[t]]);
    if ((int64_t)maxlen > 4ll * n + 4096) {
        // sparse length range: sort (length, position) keys per bucket
        std::vector<uint64_t> key;
        for (int32_t b = 0; b < p; b++) {
            const int32_t lo = h_bo[b], nb = h_bo[b + 1] - h_bo[b];
            key.resize((size_t)nb);
            for (int32_t u = 0; u < nb; u++) key[u] = ((uint64_t)(uint32_t)h_len[h_order[lo + u]] << 32) | (uint32_t)u;
            std::sort(key.begin(), key.end());
            for (int32_t u = 0; u < nb; u++) (*srt)[lo + u] = (int32_t)(key[u] & 0xffffffffu);
        }
        return;
    }
    // two stable counting passes over the CSR positions: by length, then by
    // bucket; inside a bucket that is ascending length, ties by local position
    std::vector<int32_t> cnt((size_t)maxlen + 2, 0), by_len((size_t)n), bucket_of((size_t)n), next((size_t)p);
    for (int32_t t = 0; t < n; t++) cnt[h_len[h_order[t]] + 1]++;
    for (int32_t l = 0; l <= maxlen; l++) cnt[l + 1] += cnt[l];
    for (int32_t t = 0; t < n; t++) by_len[cnt[h_len[h_order[t]]]++] = t;
    for (int32_t b = 0; b < p; b++) {
        next[b] = h_bo[b];
        for (int32_t t = h_bo[b]; t < h_bo[b + 1]; t++) bucket_of[t] = b;
    }
    for (int32_t t : by_len) {
        const int32_t b = bucket_of[t];
        (*srt)[next[b]++] = t - h_bo[b];
    }
}

int gotoh_launch(sad_ctx* ctx, const DevSeqs& S, const GotohLaunch& L, cudaStream_t stream) {
    KernelFn fn = kernel_for(L.R);
    SAD_CHECK(fn != nullptr, SAD_EINVAL, "no Gotoh kernel for R = %d", L.R);
    SAD_CHECK(L.G == 4 || L.G == 8 || L.G == 16 || L.G == 32, SAD_EINVAL, "G = %d", L.G);
    const int threads = 128;
    const int NG = threads / L.G;
    GotohArgs a;
    a.res = S.res;
    a.pad_off = S.pad_off;
    a.len = S.len;
    a.order = L.order;
    a.bucket_off = L.bucket_off;
    a.srt = L.srt;
    a.score_off = L.score_off;
    a.scores = L.scores;
    a.subst = L.subst;
    a.alphabet = S.alphabet;
    a.go = L.go;
    a.ge = L.ge;
    a.G = L.G;
    const int32_t strip_h = L.G * L.R;
    a.prof_stride = (int32_t)round_up(std::max<int32_t>(L.max_m, 1), strip_h);
    const int grid = L.persistent ? L.persistent_grid : L.n_items;
    if (grid == 0) return SAD_OK;
    // strip boundaries are needed only for queries longer than one strip
    a.scratch_stride = 2 * ((int64_t)S.max_len + 1 + 4);
    int32_t* scratch = nullptr;
    if (L.max_m > strip_h) {
        void* sp = nullptr;
        SAD_RET(workspace(ctx, WS_SCORE_SCRATCH, sizeof(int32_t) * (size_t)grid * NG * a.scratch_stride,
                          stream, &sp));
        scratch = (int32_t*)sp;
    }
    a.scratch = scratch;
    const size_t smem = (size_t)S.alphabet * a.prof_stride;
    SAD_CHECK(smem <= ctx->smem_optin, SAD_EINVAL, "query profile of %zu bytes exceeds shared memory",
              smem);
    SAD_RET(allow_max_dynamic_smem(ctx, (const void*)fn));
    TraceScope ts(ctx, SAD_STAGE_SCORES, stream);
    fn<<<grid, threads, smem, stream>>>(L.items, L.n_items, L.head, a);
    SAD_LAUNCHED();
    return SAD_OK;
}

// Choose R for a query length so that one strip covers it with little padding
// at G = 32 lanes; longer queries strip-mine at R = 32.
int pick_R(int32_t m) {
    static const int Rs[] = {4, 8, 12, 16, 20, 24, 32};
    for (int R : Rs)
        if (m <= 32 * R) return R;
    return 32;
}

// Variants of the packed kernel: R rows per lane x G lanes per subject.
constexpr int kPackedR[] = {8, 12, 16, 20, 24, 32};
constexpr int kPackedG[] = {8, 16, 32};
constexpr int kNumR = 6, kNumG = 3, kNumVariants = kNumR * kNumG;
constexpr int kPackedThreads = 128;

// Bias of the packed form (stored = true + bias), or false when none fits.
// Over the padded strip rows i <= L + 1024 and columns j <= L (L = longest
// sequence) every true H, E, F value v satisfies
//   2 go + (i + j) ge <= v <= max(s, 0) L
// (the all-gap path is one alignment; each column gains at most max(s, 0)).
// The stored values must stay in [0, 32767] with room for every addend:
//   bias + vmin + min(smin, go + ge, 0) >= 0,  bias + vmax + max(smax, 0) <= 32767.
bool packed16_bias(const DevSeqs& S, const int8_t* subst, int32_t go, int32_t ge, int32_t* bias) {
    int32_t smax = 0, smin = 0;
    for (int32_t t = 0; t < S.alphabet * S.alphabet; t++) {
        smax = std::max<int32_t>(smax, subst[t]);
        smin = std::min<int32_t>(smin, subst[t]);
    }
    const int64_t L = S.max_len;
    const int64_t rows = L + 1024;  // padding of the widest strip
    const int64_t vmax = (int64_t)smax * L;
    const int64_t vmin = 2ll * go + (int64_t)ge * (rows + L);
    // every stored value, and each sum with a negative addend, >= 0; every
    // boundary value go + i ge + B (i <= rows) above the largest substitution
    // score (the virtual column of the streaming form relies on it)
    const int64_t lo = std::max<int64_t>(-vmin - std::min<int64_t>(std::min<int64_t>(smin, go + ge), 0),
                                         (int64_t)smax + 1 - go - (int64_t)ge * rows);
    const int64_t hi = 32767 - vmax - smax;
    if (lo > hi) return false;
    *bias = (int32_t)lo;
    return true;
}

int rpad_rt(int R) { return ((R / 4) % 2 == 0) ? R + 4 : R; }

int variant_index(int R, int G) {
    for (int ri = 0; ri < kNumR; ri++)
        for (int gi = 0; gi < kNumG; gi++)
            if (kPackedR[ri] == R && kPackedG[gi] == G) return ri * kNumG + gi;
    return -1;
}


int ensure_aux_streams(sad_ctx* ctx) {
    if (ctx->aux_ready) return SAD_OK;
    for (int v = 0; v < kAuxStreams; v++) {
        SAD_CUDA(cudaStreamCreateWithFlags(&ctx->aux[v], cudaStreamNonBlocking));
        SAD_CUDA(cudaEventCreateWithFlags(&ctx->ev_join[v], cudaEventDisableTiming));
    }
    SAD_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    ctx->aux_ready = true;
    return SAD_OK;
}

// One kernel launch of the batched score stage.
struct PackedLaunch {
    KernelFn fn;
    int grid, block;
    size_t smem;
    const GotohItem* items;
    int32_t n_items;
    int32_t* head;
    GotohArgs args;
};

// Host plan of the packed score stage: work items grouped by kernel variant
// (longest first inside a variant), then the single-query items of queries too
// long for any packed profile.
struct PackedPlan {
    std::vector<GotohItem> all;
    int32_t first[kNumVariants + 1];
    int32_t rows_var[kNumVariants];
    int32_t first_single = 0;
    int32_t singles_rows = 0;
};

void plan_packed(sad_ctx* ctx, const DevSeqs& S, const std::vector<int32_t>& h_bo,
                 const std::vector<int32_t>& h_order, const std::vector<int32_t>& srt, PackedPlan* plan) {
    const int32_t p = (int32_t)h_bo.size() - 1;
    auto len_at = [&](int32_t b, int32_t pos) { return S.h_len[h_order[h_bo[b] + srt[h_bo[b] + pos]]]; };
    // per variant: strip height and the most strips whose profile fits in shared memory
    int32_t vsh[kNumVariants], vmax_strips[kNumVariants];
    for (int v = 0; v < kNumVariants; v++) {
        const int R = kPackedR[v / kNumG], G = kPackedG[v % kNumG];
        vsh[v] = R * G;
        vmax_strips[v] = (int32_t)(ctx->smem_optin / ((size_t)S.alphabet * 4 * G * rpad_rt(R)));
    }
    const ScoreTuning& tu = ctx->tuning;
    const int fv = tu.filter ? variant_index(tu.force_R, tu.force_G) : -1;
    // subjects per work item: up to kChunkSubjects, fewer when the call holds
    // few (query pair, subject) visits, so that there are about five items per
    // resident CTA and the persistent launches end on small items (N = 2000:
    // 24 subjects, scores 2.22 -> 2.11 ms; N = 20000 keeps 64, where 24 cost 2 %
    // in profile builds)
    int64_t visits = 0;
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = h_bo[b + 1] - h_bo[b];
        const int64_t nq = (nb + 1) / 2;  // query pairs; pair q visits subjects 2q .. nb - 1
        visits += nq * nb - nq * (nq - 1);
    }
    const int64_t slots = 4ll * std::max(ctx->num_sms, 1);
    const int32_t chunk = (int32_t)std::min<int64_t>(
        kChunkSubjects, std::max<int64_t>(24, round_up((visits + 5 * slots - 1) / (5 * slots), 8)));
    // per-thread scratch kept across calls (no allocation once warm)
    // (the arrays are reached through local pointers: in a shared library each
    // thread_local access may otherwise go through the TLS lookup call)
    thread_local std::vector<GotohItem> by_var_tls[kNumVariants];
    thread_local std::vector<double> cost_var_tls[kNumVariants];
    std::vector<GotohItem>* const by_var = by_var_tls;
    std::vector<double>* const cost_var = cost_var_tls;
    for (int v = 0; v < kNumVariants; v++) {
        by_var[v].clear();
        cost_var[v].clear();
    }
    int32_t rows_var[kNumVariants] = {0};
    std::vector<GotohItem> singles;  // single-query items for the 32-bit kernel
    int32_t singles_rows = 0;
    // the table's variant per bin (or -1)
    int bin_v[ScoreTuning::kMaxBins];
    for (int t = 0; t < tu.nbins; t++) bin_v[t] = variant_index(tu.R[t], tu.G[t]);
    // without a table: the variants whose profile fits one strip, in the order of
    // least padding (smallest strip G R; then R <= 24; then G nearest 16); a pair
    // takes the first whose strip holds its rows
    int lp_v[kNumVariants], n_lp = 0;
    if (tu.nbins == 0 && !tu.filter) {
        for (int v = 0; v < kNumVariants; v++)
            if (vmax_strips[v] >= 1) lp_v[n_lp++] = v;
        auto lp_key = [&](int v) {
            const int R = kPackedR[v / kNumG], G = kPackedG[v % kNumG];
            return vsh[v] * 1024 + (R <= 24 ? 0 : 512) + std::abs(G - 16);
        };
        std::sort(lp_v, lp_v + n_lp, [&](int x, int y) { return lp_key(x) < lp_key(y); });
    }
    // per variant for a pair of `rows` rows: whether its profile fits, and the
    // estimated instruction slots of one subject of length n, ca n + cb =
    // strips G ((n + G + 1)(5 R + 16) + 40): every strip runs n + G + 1 steps on
    // G lanes of 5R + 16 instructions, plus a fixed cost per strip and lane
    auto variant_cost = [&](int v, int32_t rows1, double* ca, double* cb) {
        const int R = kPackedR[v / kNumG], G = kPackedG[v % kNumG];
        const int32_t strips = (rows1 + vsh[v] - 1) / vsh[v];
        const double k = (double)strips * G;
        *ca = k * (5.0 * R + 16.0);
        *cb = k * ((G + 1) * (5.0 * R + 16.0) + 40.0);
        return strips <= vmax_strips[v];
    };
    thread_local std::vector<int32_t> lens_tls;  // the bucket's lengths in length order
    thread_local std::vector<int64_t> pre_tls;   // and their prefix sums
    std::vector<int32_t>& lens = lens_tls;
    std::vector<int64_t>& pre = pre_tls;
    for (int32_t b = 0; b < p; b++) {
        const int32_t nb = h_bo[b + 1] - h_bo[b];
        lens.resize((size_t)nb);
        pre.assign((size_t)nb + 1, 0);
        for (int32_t v = 0; v < nb; v++) {
            lens[v] = len_at(b, v);
            pre[v + 1] = pre[v] + lens[v];
        }
        for (int32_t qp = 0; 2 * qp < nb; qp++) {
            const int32_t m1 = lens[2 * qp];
            const int32_t m2 = (2 * qp + 1 < nb) ? lens[2 * qp + 1] : 0;
            const int32_t rows = std::max(m1, m2);
            const int32_t rows1 = std::max(rows, 1);
            if (tu.filter && (rows <= tu.lo || rows > tu.hi)) continue;  // autotuning: one length bin
            // the variant of this pair: the forced one (autotuning), the table's, or
            // per chunk the cost model's (every variant's cost, computed only then)
            int fixed_v = -1;
            double fa = 0, fb = 0;
            if (tu.filter) {
                if (fv < 0 || !variant_cost(fv, rows1, &fa, &fb)) {
                    ctx->tuning.skipped = true;  // this variant cannot serve the whole bin
                    continue;
                }
                fixed_v = fv;
            } else {
                int tv = -1;
                for (int t = 0; t < tu.nbins && tv < 0; t++)
                    if (rows <= tu.upper[t]) tv = bin_v[t];
                if (tu.nbins == 0) {
                    // no table: the variant of least padding whose one strip holds the
                    // pair, the table the autotuner ends on for the N = 2000 workload
                    // (untuned, the cost model below gave 3.2 ms there against 2.1 ms)
                    for (int t = 0; t < n_lp && tv < 0; t++)
                        if (vsh[lp_v[t]] >= rows1) tv = lp_v[t];
                }
                if (tv >= 0 && variant_cost(tv, rows1, &fa, &fb)) fixed_v = tv;
            }
            bool fit[kNumVariants];
            double ca[kNumVariants], cb[kNumVariants];
            if (fixed_v < 0)
                for (int v = 0; v < kNumVariants; v++) fit[v] = variant_cost(v, rows1, &ca[v], &cb[v]);
            for (int32_t v0 = 2 * qp; v0 < nb; v0 += chunk) {
                const int32_t v1 = std::min(nb, v0 + chunk);
                // the chunk's cost: per subject ca n + cb, summed (no mean, no division)
                const double nsum = (double)(pre[v1] - pre[v0]), ncnt = (double)(v1 - v0);
                int best = fixed_v;
                double bc = best >= 0 ? fa * nsum + fb * ncnt : 1e300;
                if (best < 0) {
                    for (int v = 0; v < kNumVariants; v++) {
                        if (!fit[v]) continue;
                        const double c = ca[v] * nsum + cb[v] * ncnt;
                        if (c < bc) {
                            bc = c;
                            best = v;
                        }
                    }
                }
                if (best < 0) {
                    // too long for any packed profile: both queries go to the 32-bit kernel
                    singles.push_back(GotohItem{b, 2 * qp, v0, v1});
                    if (2 * qp + 1 < nb && std::max(v0, 2 * qp + 1) < v1)
                        singles.push_back(GotohItem{b, 2 * qp + 1, std::max(v0, 2 * qp + 1), v1});
                    singles_rows = std::max(singles_rows, rows);
                    continue;
                }
                by_var[best].push_back(GotohItem{b, qp, v0, v1});
                cost_var[best].push_back(bc);
                rows_var[best] = std::max(rows_var[best], rows);
            }
        }
    }
    // longest first inside every variant: one counting pass over 32 cost classes
    // per octave (exponent and top five mantissa bits of the cost), largest first,
    // plan order inside a class (about 3 % resolution is enough to leave the
    // shortest items for the end of the queue)
    std::vector<GotohItem> all;
    {
        size_t total = singles.size();
        for (int v = 0; v < kNumVariants; v++) total += by_var[v].size();
        all.reserve(total);
    }
    int32_t first[kNumVariants + 1];
    thread_local std::vector<int32_t> ccnt_tls;
    thread_local std::vector<int32_t> cls_tls;
    std::vector<int32_t>& ccnt = ccnt_tls;
    std::vector<int32_t>& cls = cls_tls;
    for (int v = 0; v < kNumVariants; v++) {
        first[v] = (int32_t)all.size();
        const size_t nv = by_var[v].size();
        if (nv == 0) continue;
        cls.resize(nv);
        int32_t cmin = INT32_MAX, cmax = -1;
        for (size_t t = 0; t < nv; t++) {
            uint64_t bits;
            const double x = 1.0 + cost_var[v][t];
            memcpy(&bits, &x, sizeof(bits));
            const int32_t c = (int32_t)(bits >> 47);  // 11 exponent bits, 5 mantissa bits
            cls[t] = c;
            cmin = std::min(cmin, c);
            cmax = std::max(cmax, c);
        }
        ccnt.assign((size_t)(cmax - cmin) + 2, 0);
        for (size_t t = 0; t < nv; t++) ccnt[(size_t)(cmax - cls[t]) + 1]++;  // descending cost
        for (int32_t c = 0; c <= cmax - cmin; c++) ccnt[c + 1] += ccnt[c];
        all.resize(first[v] + nv);
        for (size_t t = 0; t < nv; t++) all[first[v] + ccnt[cmax - cls[t]]++] = by_var[v][t];
    }
    first[kNumVariants] = (int32_t)all.size();
    plan->first_single = (int32_t)all.size();
    for (const GotohItem& it : singles) all.push_back(it);
    plan->singles_rows = singles_rows;
    for (int v = 0; v <= kNumVariants; v++) plan->first[v] = first[v];
    for (int v = 0; v < kNumVariants; v++) plan->rows_var[v] = rows_var[v];
    plan->all.swap(all);
}

// Blocks of `fn` resident per SM at `threads` threads and `smem` dynamic shared
// memory bytes (cached: the answer depends only on these and the device).
int occupancy(sad_ctx* ctx, const void* fn, int threads, size_t smem, int* occ) {
    struct Key {
        int dev;
        const void* fn;
        int threads;
        size_t smem;
    };
    static std::mutex mu;
    static std::vector<std::pair<Key, int>> cache;
    std::lock_guard<std::mutex> lock(mu);
    for (auto& e : cache)
        if (e.first.dev == ctx->device && e.first.fn == fn && e.first.threads == threads && e.first.smem == smem) {
            *occ = e.second;
            return SAD_OK;
        }
    int o = 0;
    SAD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, threads, smem));
    cache.push_back({Key{ctx->device, fn, threads, smem}, o});
    *occ = o;
    return SAD_OK;
}

// Launch a packed plan whose items are on the device (d_items, in plan order)
// with kNumVariants + 1 queue heads at d_heads (zeroed here, on the stream).
int launch_packed(sad_ctx* ctx, const DevSeqs& S, const PackedPlan& plan, const GotohItem* d_items,
                  int32_t* d_heads, const GotohLaunch& base, cudaStream_t stream) {
    const int32_t* first = plan.first;
    const int32_t* rows_var = plan.rows_var;
    const int32_t first_single = plan.first_single;
    const int32_t singles_rows = plan.singles_rows;
    const size_t n_singles = plan.all.size() - (size_t)first_single;
    const size_t heads_bytes = 4 * (kNumVariants + 1);
    // launch shapes and strip-boundary scratch
    struct Shape {
        int grid = 0;
        size_t smem = 0;
        int64_t scratch_off = 0;
        bool strips = false;
        bool stream = false;
        int32_t prof_stride = 0;
    } shp[kNumVariants];
    const int64_t stride = 2 * ((int64_t)S.max_len + 1 + 4);
    int64_t scratch_ints = 0;
    for (int v = 0; v < kNumVariants; v++) {
        const int32_t nv = first[v + 1] - first[v];
        if (nv == 0) continue;
        const int R = kPackedR[v / kNumG], G = kPackedG[v % kNumG];
        const int32_t strip_h = R * G;
        shp[v].prof_stride = (int32_t)(round_up(std::max<int32_t>(rows_var[v], 1), strip_h) / R) * rpad_rt(R);
        shp[v].smem = (size_t)S.alphabet * shp[v].prof_stride * 4;
        SAD_CHECK(shp[v].smem <= ctx->smem_optin, SAD_EINVAL,
                  "packed query profile of %zu bytes exceeds shared memory", shp[v].smem);
        // every query pair within one strip: the streaming kernel, one fill and
        // drain per group and item instead of one per subject (N = 2000 scores
        // 2.37 -> 2.21 ms once the virtual column had removed its one-column steps;
        // before that, with 8 or 16 lanes per subject its per-step bookkeeping cost
        // as much as the fill it saved)
        shp[v].strips = rows_var[v] > strip_h;
        shp[v].stream = !shp[v].strips;
        KernelFn fn = pair16_kernel_for(R, shp[v].stream);
        SAD_RET(allow_max_dynamic_smem(ctx, (const void*)fn));
        int occ = 0;
        SAD_RET(occupancy(ctx, (const void*)fn, kPackedThreads, shp[v].smem, &occ));
        occ = std::max(occ, 1);
        shp[v].grid = std::min<int64_t>(nv, (int64_t)ctx->num_sms * occ);
        if (shp[v].strips) {
            shp[v].scratch_off = scratch_ints;
            scratch_ints += (int64_t)shp[v].grid * (kPackedThreads / G) * stride;
        }
    }
    int32_t* scratch = nullptr;
    if (scratch_ints > 0) {
        void* sp = nullptr;
        SAD_RET(workspace(ctx, WS_SCORE_SCRATCH, sizeof(int32_t) * (size_t)scratch_ints, stream, &sp));
        scratch = (int32_t*)sp;
    }
    SAD_RET(ensure_aux_streams(ctx));
    // the launches of this call, as plain records (they also key the graph cache)
    std::vector<PackedLaunch> recs;
    auto common_args = [&](GotohArgs& a) {
        memset(&a, 0, sizeof(a));
        a.res = S.res;
        a.pad_off = S.pad_off;
        a.len = S.len;
        a.order = base.order;
        a.bucket_off = base.bucket_off;
        a.srt = base.srt;
        a.score_off = base.score_off;
        a.scores = base.scores;
        a.subst = base.subst;
        a.alphabet = S.alphabet;
        a.go = base.go;
        a.ge = base.ge;
        a.scratch_stride = stride;
        a.bias = base.bias;
    };
    for (int v = 0; v < kNumVariants; v++) {
        if (shp[v].grid == 0) continue;
        const int R = kPackedR[v / kNumG], G = kPackedG[v % kNumG];
        PackedLaunch L;
        memset(&L, 0, sizeof(L));
        common_args(L.args);
        L.args.G = G;
        L.args.prof_stride = shp[v].prof_stride;
        L.args.scratch = shp[v].strips ? scratch + shp[v].scratch_off : nullptr;
        L.fn = pair16_kernel_for(R, shp[v].stream);
        L.grid = shp[v].grid;
        L.block = kPackedThreads;
        L.smem = shp[v].smem;
        L.items = d_items + first[v];
        L.n_items = first[v + 1] - first[v];
        L.head = d_heads + v;
        recs.push_back(L);
    }
    if (n_singles > 0) {
        // queries too long for a packed profile: 32-bit kernel, int8 profile, G = 32, R = 32
        constexpr int R1 = 32, G1 = 32, T1 = 128;
        PackedLaunch L;
        memset(&L, 0, sizeof(L));
        common_args(L.args);
        L.fn = kernel_for(R1);
        L.args.G = G1;
        L.args.prof_stride = (int32_t)round_up(std::max<int32_t>(singles_rows, 1), R1 * G1);
        L.smem = (size_t)S.alphabet * L.args.prof_stride;
        SAD_CHECK(L.smem <= ctx->smem_optin, SAD_EINVAL, "query profile of %zu bytes exceeds shared memory",
                  L.smem);
        SAD_RET(allow_max_dynamic_smem(ctx, (const void*)L.fn));
        int occ = 0;
        SAD_RET(occupancy(ctx, (const void*)L.fn, T1, L.smem, &occ));
        L.grid = (int)std::min<int64_t>((int64_t)n_singles, (int64_t)ctx->num_sms * std::max(occ, 1));
        void* sp = nullptr;
        SAD_RET(workspace(ctx, WS_SCORE_SCRATCH_LONG, sizeof(int32_t) * (size_t)L.grid * (T1 / G1) * stride,
                          stream, &sp));
        L.args.scratch = (int32_t*)sp;
        L.block = T1;
        L.items = d_items + first_single;
        L.n_items = (int32_t)n_singles;
        L.head = d_heads + kNumVariants;
        recs.push_back(L);
    }
    // queue heads to zero, fork onto the auxiliary streams, one launch each, join
    auto enqueue = [&](cudaStream_t st) -> int {
        SAD_CUDA(cudaMemsetAsync(d_heads, 0, heads_bytes, st));
        SAD_CUDA(cudaEventRecord(ctx->ev_fork, st));
        int used = 0;
        for (const PackedLaunch& L : recs) {
            cudaStream_t sv = ctx->aux[used % kAuxStreams];
            SAD_CUDA(cudaStreamWaitEvent(sv, ctx->ev_fork, 0));
            L.fn<<<L.grid, L.block, L.smem, sv>>>(L.items, L.n_items, L.head, L.args);
            SAD_CUDA(cudaGetLastError());
            used++;
        }
        for (int u = 0; u < std::min(used, kAuxStreams); u++) {
            SAD_CUDA(cudaEventRecord(ctx->ev_join[u], ctx->aux[u]));
            SAD_CUDA(cudaStreamWaitEvent(st, ctx->ev_join[u], 0));
        }
        return SAD_OK;
    };
    // replay the cached graph when this call launches exactly what the last one did
    std::vector<char> sig(sizeof(PackedLaunch) * recs.size() + sizeof(void*) + sizeof(size_t));
    {
        char* q = sig.data();
        memcpy(q, &d_heads, sizeof(void*));
        memcpy(q + sizeof(void*), &heads_bytes, sizeof(size_t));
        if (!recs.empty()) memcpy(q + sizeof(void*) + sizeof(size_t), recs.data(), sizeof(PackedLaunch) * recs.size());
    }
    if (stream == nullptr) {
        // the legacy default stream cannot be captured: launch directly
        TraceScope ts(ctx, SAD_STAGE_SCORES_PACKED, stream);
        SAD_RET(enqueue(stream));
        for (size_t t = 0; t < recs.size(); t++) note_launch();
        return SAD_OK;
    }
    if (!ctx->score_graph || ctx->score_graph_sig != sig) {
        cudaGraph_t graph = nullptr;
        SAD_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue(stream);
        const cudaError_t ec = cudaStreamEndCapture(stream, &graph);
        if (rc != SAD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        SAD_CUDA(ec);
        if (ctx->score_graph) {
            cudaGraphExecDestroy(ctx->score_graph);
            ctx->score_graph = nullptr;
        }
        const cudaError_t ei = cudaGraphInstantiate(&ctx->score_graph, graph, 0);
        cudaGraphDestroy(graph);
        SAD_CUDA(ei);
        ctx->score_graph_sig = sig;
    }
    TraceScope ts(ctx, SAD_STAGE_SCORES_PACKED, stream);
    SAD_CUDA(cudaGraphLaunch(ctx->score_graph, stream));
    for (size_t t = 0; t < recs.size(); t++) note_launch();
    return SAD_OK;
}

int bucket_scores_device(sad_ctx* ctx, const DevSeqs& S, const int32_t* d_bo, const int32_t* d_order,
                         int32_t p, const int8_t* h_subst, int32_t go, int32_t ge, int32_t mode,
                         int64_t* d_score_off_out, int32_t* d_scores, int64_t capacity,
                         int64_t* total_out, cudaStream_t stream) {
    const int32_t n = S.n;
    std::vector<int32_t> h_bo((size_t)p + 1), h_order((size_t)n);
    {
        // through the context's pinned area (stream-ordered after any earlier
        // copy from it): two asynchronous copies and one wait
        void* pin = nullptr;
        SAD_RET(pinned(ctx, 4ull * (p + 1 + n) + 64, stream, &pin));
        int32_t* pb = (int32_t*)pin;
        SAD_CUDA(cudaMemcpyAsync(pb, d_bo, 4ull * (p + 1), cudaMemcpyDeviceToHost, stream));
        if (n > 0) SAD_CUDA(cudaMemcpyAsync(pb + p + 1, d_order, 4ull * n, cudaMemcpyDeviceToHost, stream));
        SAD_CUDA(cudaStreamSynchronize(stream));
        memcpy(h_bo.data(), pb, 4ull * (p + 1));
        if (n > 0) memcpy(h_order.data(), pb + p + 1, 4ull * n);
    }
    SAD_CHECK(h_bo[0] == 0 && h_bo[p] == n, SAD_EINVAL,
              "bucket_offsets must start at 0 and end at n = %d", n);
    std::vector<char> seen((size_t)n, 0);
    for (int32_t b = 0; b < p; b++)
        SAD_CHECK(h_bo[b + 1] >= h_bo[b], SAD_EINVAL, "bucket_offsets decreases at %d", b);
    for (int32_t t = 0; t < n; t++) {
        const int32_t i = h_order[t];
        SAD_CHECK(i >= 0 && i < n && !seen[i], SAD_EINVAL,
                  "order is not a permutation of 0..n-1 (entry %d = %d)", t, i);
        seen[i] = 1;
    }
    std::vector<int32_t> srt;
    std::vector<int64_t> score_off;
    plan_buckets(h_bo, h_order, S.h_len, p, &srt, &score_off);
    *total_out = score_off[p];
    SAD_CHECK(mode == SAD_SCORES_PER_BUCKET || mode == SAD_SCORES_PERSISTENT || mode == SAD_SCORES_PERSISTENT_32,
              SAD_EINVAL, "unknown scores mode %d", mode);
    // work items: the packed plan, or one item per query row (longest first for
    // the persistent 32-bit kernel)
    int32_t bias = 0;
    const bool packed = mode == SAD_SCORES_PERSISTENT && packed16_bias(S, h_subst, go, ge, &bias);
    PackedPlan pplan;
    std::vector<GotohItem> items;
    int32_t max_m = 0;
    if (packed) {
        plan_packed(ctx, S, h_bo, h_order, srt, &pplan);
    } else {
        for (int32_t b = 0; b < p; b++) {
            const int32_t lo = h_bo[b], nb = h_bo[b + 1] - lo;
            for (int32_t q = 0; q < nb; q++) {
                items.push_back(GotohItem{b, q, q, nb});
                max_m = std::max(max_m, S.h_len[h_order[lo + srt[lo + q]]]);
            }
        }
        if (mode != SAD_SCORES_PER_BUCKET) {
            std::vector<int64_t> cost(items.size());
            std::vector<int32_t> idx(items.size());
            for (size_t t = 0; t < items.size(); t++) {
                const GotohItem& it = items[t];
                const int32_t lo = h_bo[it.bucket];
                const int64_t mq = S.h_len[h_order[lo + srt[lo + it.q]]];
                int64_t c = 0;
                for (int32_t v = it.v0; v < it.v1; v++) c += mq * S.h_len[h_order[lo + srt[lo + v]]];
                cost[t] = c;
                idx[t] = (int32_t)t;
            }
            std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
            std::vector<GotohItem> sorted(items.size());
            for (size_t t = 0; t < items.size(); t++) sorted[t] = items[idx[t]];
            items.swap(sorted);
        }
    }
    const std::vector<GotohItem>& its = packed ? pplan.all : items;
    // one staging copy: srt, score_off, subst, items, queue heads
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_srt = carve(4ull * (n + 1)), o_so = carve(8ull * (p + 1)),
                 o_sub = carve((size_t)S.alphabet * S.alphabet), o_items = carve(sizeof(GotohItem) * (its.size() + 1)),
                 o_head = carve(4 * (kNumVariants + 1));
    void* plan = nullptr;
    SAD_RET(workspace(ctx, WS_SCORE_PLAN, off, stream, &plan));
    void* pin = nullptr;
    SAD_RET(pinned(ctx, off, stream, &pin));  // earlier copies from it are done: the stream was synchronised above
    char* hp = (char*)pin;
    memcpy(hp + o_srt, srt.data(), 4ull * n);
    memcpy(hp + o_so, score_off.data(), 8ull * (p + 1));
    memcpy(hp + o_sub, h_subst, (size_t)S.alphabet * S.alphabet);
    if (!its.empty()) memcpy(hp + o_items, its.data(), sizeof(GotohItem) * its.size());
    memset(hp + o_head, 0, 4 * (kNumVariants + 1));
    char* dp = (char*)plan;
    SAD_CUDA(cudaMemcpyAsync(dp, hp, off, cudaMemcpyHostToDevice, stream));
    if (d_score_off_out)
        SAD_CUDA(cudaMemcpyAsync(d_score_off_out, dp + o_so, 8ull * (p + 1), cudaMemcpyDeviceToDevice,
                                 stream));
    if (score_off[p] > capacity) {
        set_error("scores need %lld entries, capacity is %lld", (long long)score_off[p],
                  (long long)capacity);
        return SAD_ERANGE;
    }
    GotohLaunch L;
    L.order = d_order;
    L.bucket_off = d_bo;
    L.srt = (const int32_t*)(dp + o_srt);
    L.score_off = (const int64_t*)(dp + o_so);
    L.scores = d_scores;
    L.subst = (const int8_t*)(dp + o_sub);
    L.go = go;
    L.ge = ge;
    L.bias = bias;
    const GotohItem* d_items = (const GotohItem*)(dp + o_items);
    int32_t* d_heads = (int32_t*)(dp + o_head);
    if (packed) return launch_packed(ctx, S, pplan, d_items, d_heads, L, stream);
    if (mode == SAD_SCORES_PER_BUCKET) {
        // one launch per bucket, R from the bucket's median member length
        int64_t first = 0;
        for (int32_t b = 0; b < p; b++) {
            const int32_t lo = h_bo[b], nb = h_bo[b + 1] - lo;
            if (nb == 0) continue;
            int32_t bm = 0;
            for (int32_t q = 0; q < nb; q++) bm = std::max(bm, S.h_len[h_order[lo + q]]);
            const int32_t med = S.h_len[h_order[lo + srt[lo + nb / 2]]];
            L.R = pick_R(med);
            L.G = 32;
            L.max_m = bm;
            L.items = d_items + first;
            L.n_items = nb;
            L.head = nullptr;
            L.persistent = false;
            SAD_RET(gotoh_launch(ctx, S, L, stream));
            first += nb;
        }
        return SAD_OK;
    }
    // persistent 32-bit: one launch over every bucket's rows, longest first
    std::vector<int32_t> all_len(S.h_len.begin(), S.h_len.begin() + n);
    std::sort(all_len.begin(), all_len.end());
    const int32_t med = n ? all_len[n / 2] : 1;
    L.R = pick_R(med);
    L.G = 32;
    L.max_m = max_m;
    L.items = d_items;
    L.n_items = (int32_t)items.size();
    L.head = d_heads;
    L.persistent = true;
    L.persistent_grid = ctx->num_sms * 4;
    return gotoh_launch(ctx, S, L, stream);
}

}  // namespace sad

extern "C" int sad_scores_set_variants(sad_ctx* ctx_in, const int32_t* upper, const int32_t* R,
                                       const int32_t* G, int32_t nbins) {
    using namespace sad;
    clear_error();
    SAD_CHECK(nbins >= 0 && nbins <= ScoreTuning::kMaxBins, SAD_EINVAL, "nbins = %d outside 0..%d", nbins,
              ScoreTuning::kMaxBins);
    SAD_CHECK(nbins == 0 || (upper && R && G), SAD_EINVAL, "a table pointer is NULL");
    for (int32_t b = 0; b < nbins; b++) {
        SAD_CHECK(variant_index(R[b], G[b]) >= 0, SAD_EINVAL,
                  "bin %d: no packed kernel with R = %d rows per lane and G = %d lanes", b, R[b], G[b]);
        SAD_CHECK(b == 0 || upper[b] > upper[b - 1], SAD_EINVAL, "bin bounds must increase");
    }
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->tuning.nbins = nbins;
    for (int32_t b = 0; b < nbins; b++) {
        ctx->tuning.upper[b] = upper[b];
        ctx->tuning.R[b] = R[b];
        ctx->tuning.G[b] = G[b];
    }
    return SAD_OK;
}

namespace sad {
int bucket_pair_scores_locked(sad_ctx* ctx, const sad_seqset* seqs, const int32_t* bucket_offsets,
                              const int32_t* order, int32_t p, const int8_t* subst, int32_t gap_open,
                              int32_t gap_extend, int32_t mode, int64_t* score_offsets, int32_t* scores,
                              int64_t scores_capacity, int32_t mem, cudaStream_t stream);
}  // namespace sad

extern "C" int sad_scores_autotune(sad_ctx* ctx_in, const sad_seqset* seqs, const int32_t* bucket_offsets,
                                   const int32_t* order, int32_t p, const int8_t* subst, int32_t gap_open,
                                   int32_t gap_extend, const int32_t* bin_upper, int32_t nbins, int32_t reps,
                                   int32_t mem, void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mem == SAD_MEM_HOST || mem == SAD_MEM_DEVICE, SAD_EINVAL, "mem = %d", mem);
    SAD_CHECK(seqs && bucket_offsets && subst && bin_upper, SAD_EINVAL, "a required pointer is NULL");
    SAD_CHECK(p >= 1 && nbins >= 1 && nbins <= ScoreTuning::kMaxBins && reps >= 1, SAD_EINVAL,
              "invalid p, nbins or reps");
    for (int32_t b = 1; b < nbins; b++) SAD_CHECK(bin_upper[b] > bin_upper[b - 1], SAD_EINVAL, "bins must increase");
    SAD_CHECK(gap_open <= 0 && gap_extend <= 0, SAD_EINVAL, "gap costs must be <= 0");
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    DevSeqs S;
    SAD_RET(prepare_seqs(ctx, seqs, mem, stream, &S));
    int32_t bias = 0;  // the score calls below derive it again
    SAD_CHECK(packed16_bias(S, subst, gap_open, gap_extend, &bias), SAD_EINVAL,
              "these sequences and costs need the 32-bit kernel; there is nothing to tune");
    const int32_t n = S.n;
    const int32_t* dbo = bucket_offsets;
    const int32_t* dord = order;
    if (mem == SAD_MEM_HOST) {
        void* st = nullptr;
        SAD_RET(workspace(ctx, WS_PART_OUT, 4ull * (p + 1 + n) + 1024, stream, &st));
        SAD_CUDA(cudaMemcpyAsync(st, bucket_offsets, 4ull * (p + 1), cudaMemcpyHostToDevice, stream));
        if (n) SAD_CUDA(cudaMemcpyAsync((int32_t*)st + p + 1, order, 4ull * n, cudaMemcpyHostToDevice, stream));
        dbo = (const int32_t*)st;
        dord = (const int32_t*)st + p + 1;
    }
    int64_t total = 0;
    std::vector<int32_t> hbo((size_t)p + 1), hord((size_t)n);
    SAD_RET(arg_to_host(dbo, 4ull * (p + 1), SAD_MEM_DEVICE, stream, hbo.data()));
    SAD_RET(arg_to_host(dord, 4ull * n, SAD_MEM_DEVICE, stream, hord.data()));
    for (int32_t b = 0; b < p; b++) total += (int64_t)(hbo[b + 1] - hbo[b]) * (hbo[b + 1] - hbo[b] + 1) / 2;
    // cells of every requested bin, then merge consecutive bins until each
    // carries at least 3% of all cells: tiny bins would pick on timing noise
    std::vector<double> bin_cells((size_t)nbins, 0.0);
    {
        std::vector<int32_t> srt;
        std::vector<int64_t> so;
        plan_buckets(hbo, hord, S.h_len, p, &srt, &so);
        for (int32_t b = 0; b < p; b++) {
            const int32_t lo = hbo[b], nb = hbo[b + 1] - lo;
            auto len_at = [&](int32_t pos) { return (double)S.h_len[hord[lo + srt[lo + pos]]]; };
            for (int32_t qp = 0; 2 * qp < nb; qp++) {
                const double m1 = len_at(2 * qp), m2 = 2 * qp + 1 < nb ? len_at(2 * qp + 1) : 0.0;
                const int32_t rows = (int32_t)std::max(m1, m2);
                double sub = 0;
                for (int32_t v = 2 * qp; v < nb; v++) sub += len_at(v);
                int32_t bi = 0;
                while (bi < nbins - 1 && rows > bin_upper[bi]) bi++;
                bin_cells[bi] += (m1 + m2) * sub;
            }
        }
    }
    double all_cells = 0;
    for (double c : bin_cells) all_cells += c;
    std::vector<int32_t> merged;
    {
        double acc = 0;
        for (int32_t b = 0; b < nbins; b++) {
            acc += bin_cells[b];
            if (acc >= 0.03 * all_cells || b == nbins - 1) {
                merged.push_back(bin_upper[b]);
                acc = 0;
            }
        }
    }
    const int32_t nm = (int32_t)merged.size();
    // every timed run is a whole sad_bucket_pair_scores call on the caller's own
    // arguments (sequence staging included), its score launches timed by the
    // tracer; outputs go to buffers of the tuner in the caller's memory space
    std::vector<int64_t> h_so((size_t)p + 1);
    std::vector<int32_t> h_sc((size_t)total + 1);
    void* d_out = nullptr;
    if (mem == SAD_MEM_DEVICE) SAD_CUDA(cudaMalloc(&d_out, 8ull * (p + 1) + 4ull * (total + 1) + 256));
    struct OutFree {
        void* p;
        ~OutFree() {
            if (p) cudaFree(p);
        }
    } out_free{d_out};
    int64_t* so_out = mem == SAD_MEM_DEVICE ? (int64_t*)d_out : h_so.data();
    int32_t* sc_out = mem == SAD_MEM_DEVICE ? (int32_t*)((char*)d_out + round_up(8ll * (p + 1), 256)) : h_sc.data();
    auto score_call = [&]() {
        return bucket_pair_scores_locked(ctx, seqs, bucket_offsets, order, p, subst, gap_open, gap_extend,
                                         SAD_SCORES_PERSISTENT, so_out, sc_out, total, mem, stream);
    };
    // every timed run starts with L2 cleared (a 256 MiB write), as a step's
    // score stage meets it after the k-mer stage (which, like the call's own
    // staging, reads the residues again)
    const size_t flush_bytes = (size_t)256 << 20;
    void* flush = nullptr;
    SAD_CUDA(cudaMalloc(&flush, flush_bytes));
    struct FlushFree {
        void* p;
        ~FlushFree() { cudaFree(p); }
    } flush_free{flush};
    const bool trace_was_on = ctx->trace_on;
    ScoreTuning table = ctx->tuning;
    table.nbins = 0;
    int rc = SAD_OK;
    // per merged bin: every variant that ran, with its time alone
    std::vector<std::vector<std::pair<double, std::pair<int, int>>>> ranked((size_t)nm);
    for (int32_t b = 0; b < nm && rc == SAD_OK; b++) {
        double best_ms = 1e300;
        int best_R = 0, best_G = 0;
        for (int ri = 0; ri < kNumR && rc == SAD_OK; ri++)
            for (int gi = 0; gi < kNumG && rc == SAD_OK; gi++) {
                ScoreTuning& tu = ctx->tuning;
                tu.filter = true;
                tu.lo = b == 0 ? 0 : merged[b - 1];
                tu.hi = merged[b];
                tu.force_R = kPackedR[ri];
                tu.force_G = kPackedG[gi];
                tu.skipped = false;
                trace_reset(ctx, true);
                for (int32_t r = 0; r <= reps && rc == SAD_OK; r++) {
                    if (r == 1) trace_reset(ctx, true);  // the first run warms up
                    if (cudaMemsetAsync(flush, r & 0xff, flush_bytes, stream) != cudaSuccess) rc = SAD_ECUDA;
                    if (rc == SAD_OK) rc = score_call();
                }
                double ms[SAD_NUM_STAGES];
                int32_t cnt[SAD_NUM_STAGES];
                if (rc == SAD_OK) rc = trace_collect(ctx, ms, cnt, SAD_NUM_STAGES);
                if (rc == SAD_OK && !ctx->tuning.skipped && cnt[SAD_STAGE_SCORES_PACKED] > 0) {
                    ranked[b].push_back({ms[SAD_STAGE_SCORES_PACKED], {kPackedR[ri], kPackedG[gi]}});
                    if (ms[SAD_STAGE_SCORES_PACKED] < best_ms) {
                        best_ms = ms[SAD_STAGE_SCORES_PACKED];
                        best_R = kPackedR[ri];
                        best_G = kPackedG[gi];
                    }
                }
            }
        if (best_R > 0) {
            table.upper[table.nbins] = merged[b];
            table.R[table.nbins] = best_R;
            table.G[table.nbins] = best_G;
            table.nbins++;
        }
    }
    table.filter = false;
    // Joint refinement: the bins' variants run side by side on forked streams, so
    // the fastest variant of a bin alone need not be the fastest with the others
    // running (the per-bin table can be 20 % off the best table of the whole
    // stage). Coordinate descent over the bins, largest share of the cells first,
    // every variant that ran in a bin (the four fastest alone when the stage is
    // long) timed as the whole stage: the mean of at least seven runs, each after
    // an L2 clear (some tables run fast in a few runs and slow in most: the mean
    // counts both). It starts from the better of the per-bin table and the
    // least-padding table (A, B, A, B); a change is kept when it gains 0.5 % and
    // again 0.5 % measured beside the current table; two passes, then the result
    // must beat its start in an A, B, A, B comparison.
    const int32_t jreps = std::max(reps, 7);
    auto stage_ms = [&](const ScoreTuning& t, double* out) -> int {
        ctx->tuning = t;
        std::vector<double> runs;
        for (int32_t r = 0; r <= jreps; r++) {
            trace_reset(ctx, true);
            SAD_CUDA(cudaMemsetAsync(flush, r & 0xff, flush_bytes, stream));
            SAD_RET(score_call());
            double ms[SAD_NUM_STAGES];
            int32_t cnt[SAD_NUM_STAGES];
            SAD_RET(trace_collect(ctx, ms, cnt, SAD_NUM_STAGES));
            if (r > 0 && cnt[SAD_STAGE_SCORES_PACKED] > 0) runs.push_back(ms[SAD_STAGE_SCORES_PACKED]);  // run 0 warms up
        }
        if (runs.empty()) {
            *out = 1e300;
            return SAD_OK;
        }
        double sum = 0;
        for (double x : runs) sum += x;
        *out = sum / (double)runs.size();
        return SAD_OK;
    };
    if (rc == SAD_OK && table.nbins > 1) {
        std::vector<int32_t> bin_of((size_t)table.nbins, -1);  // merged bin of each table entry
        for (int32_t e = 0, b = 0; e < table.nbins; e++) {
            while (b < nm && merged[b] != table.upper[e]) b++;
            bin_of[e] = b < nm ? b : -1;
        }
        // the second start: per bin the variant of least padding among those that
        // ran in it (the smallest strip G R that holds the bin's longest rows; then
        // R <= 24; then G nearest 16), the open-ended last bin as timed alone
        ScoreTuning least = table;
        for (int32_t e = 0; e < table.nbins; e++) {
            if (bin_of[e] < 0 || table.upper[e] == INT32_MAX) continue;
            int64_t best_strip = INT64_MAX;
            int best_tie = INT32_MAX;
            for (const auto& c : ranked[bin_of[e]]) {
                const int R = c.second.first, G = c.second.second;
                const int64_t strip = (int64_t)R * G;
                if (strip < table.upper[e]) continue;
                const int tie = (R <= 24 ? 0 : 100) + std::abs(G - 16);
                if (strip < best_strip || (strip == best_strip && tie < best_tie)) {
                    best_strip = strip;
                    best_tie = tie;
                    least.R[e] = R;
                    least.G[e] = G;
                }
            }
        }
        {
            double a1 = 0, b1 = 0, a2 = 0, b2 = 0;
            if (rc == SAD_OK) rc = stage_ms(table, &a1);
            if (rc == SAD_OK) rc = stage_ms(least, &b1);
            if (rc == SAD_OK) rc = stage_ms(table, &a2);
            if (rc == SAD_OK) rc = stage_ms(least, &b2);
            if (rc == SAD_OK && b1 + b2 < a1 + a2) table = least;
        }
        const ScoreTuning start = table;
        // table entries by their bins' cells, largest first
        std::vector<double> mcells((size_t)nm, 0.0);
        for (int32_t b = 0, m = 0; b < nbins && m < nm; b++) {
            mcells[m] += bin_cells[b];
            if (bin_upper[b] == merged[m]) m++;
        }
        std::vector<int32_t> visit;
        for (int32_t e = 0; e < table.nbins; e++)
            if (bin_of[e] >= 0) visit.push_back(e);
        std::stable_sort(visit.begin(), visit.end(),
                         [&](int32_t x, int32_t y) { return mcells[bin_of[x]] > mcells[bin_of[y]]; });
        double best = 0;
        rc = stage_ms(table, &best);
        const bool long_stage = best > 20.0;
        const size_t max_cands = long_stage ? 4 : 64;
        const int passes = long_stage ? 1 : 2;
        for (int pass = 0; pass < passes && rc == SAD_OK; pass++) {
            bool improved = false;
            for (int32_t e : visit) {
                if (rc != SAD_OK) break;
                auto cands = ranked[bin_of[e]];
                std::sort(cands.begin(), cands.end());
                for (size_t c = 0; c < cands.size() && c < max_cands && rc == SAD_OK; c++) {
                    const int R = cands[c].second.first, G = cands[c].second.second;
                    if (R == table.R[e] && G == table.G[e]) continue;
                    ScoreTuning cand = table;
                    cand.R[e] = R;
                    cand.G[e] = G;
                    double t = 0;
                    rc = stage_ms(cand, &t);
                    if (rc == SAD_OK && t < 0.995 * best) {
                        // confirm against the current table, measured again beside it
                        double now = 0, again = 0;
                        rc = stage_ms(table, &now);
                        if (rc == SAD_OK) rc = stage_ms(cand, &again);
                        if (rc == SAD_OK && again < 0.995 * now) {
                            best = again;
                            table = cand;
                            improved = true;
                        } else if (rc == SAD_OK) {
                            best = std::min(best, now);
                        }
                    }
                }
            }
            if (!improved) break;
        }
        // keep the refined table only if it still beats its start, measured A, B, A, B
        double a1 = 0, b1 = 0, a2 = 0, b2 = 0;
        if (rc == SAD_OK) rc = stage_ms(start, &a1);
        if (rc == SAD_OK) rc = stage_ms(table, &b1);
        if (rc == SAD_OK) rc = stage_ms(start, &a2);
        if (rc == SAD_OK) rc = stage_ms(table, &b2);
        if (rc == SAD_OK && b1 + b2 > a1 + a2) table = start;
    }
    ctx->tuning = table;
    trace_reset(ctx, trace_was_on);
    return rc;
}

extern "C" int sad_scores_get_variants(sad_ctx* ctx_in, int32_t* upper, int32_t* R, int32_t* G,
                                       int32_t max_bins, int32_t* nbins) {
    using namespace sad;
    clear_error();
    SAD_CHECK(nbins != nullptr, SAD_EINVAL, "nbins is NULL");
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    *nbins = ctx->tuning.nbins;
    for (int32_t b = 0; b < ctx->tuning.nbins && b < max_bins; b++) {
        upper[b] = ctx->tuning.upper[b];
        R[b] = ctx->tuning.R[b];
        G[b] = ctx->tuning.G[b];
    }
    return SAD_OK;
}

extern "C" int sad_scores_size(const int32_t* bucket_offsets, int32_t p, int32_t mem, int64_t* total) {
    using namespace sad;
    clear_error();
    SAD_CHECK(bucket_offsets && total && p >= 1, SAD_EINVAL, "invalid arguments");
    std::vector<int32_t> bo((size_t)p + 1);
    SAD_RET(arg_to_host(bucket_offsets, 4ull * (p + 1), mem, 0, bo.data()));
    int64_t t = 0;
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = bo[b + 1] - bo[b];
        SAD_CHECK(nb >= 0, SAD_EINVAL, "bucket_offsets decreases at %d", b);
        t += nb * (nb + 1) / 2;
    }
    *total = t;
    return SAD_OK;
}

namespace sad {

// The work of sad_bucket_pair_scores once its arguments are checked and ctx is
// locked: staging of the sequences, the score stage, the copies back (host
// mode) and the status check. The autotuner times candidate tables through it,
// so that it measures exactly what a caller's call runs.
int bucket_pair_scores_locked(sad_ctx* ctx, const sad_seqset* seqs, const int32_t* bucket_offsets,
                              const int32_t* order, int32_t p, const int8_t* subst, int32_t gap_open,
                              int32_t gap_extend, int32_t mode, int64_t* score_offsets, int32_t* scores,
                              int64_t scores_capacity, int32_t mem, cudaStream_t stream) {
    const int32_t A = seqs->alphabet;
    SAD_RET(status_clear(ctx, stream));
    DevSeqs S;
    SAD_RET(prepare_seqs(ctx, seqs, mem, stream, &S));
    const int32_t n = S.n;
    SAD_CHECK(n == 0 || order != nullptr, SAD_EINVAL, "order is NULL");
    // scores must fit int32: |score| <= (max|s| + |go| + |ge|) * (m + n)
    int32_t smax = 0;
    for (int32_t t = 0; t < A * A; t++) smax = std::max(smax, (int32_t)std::abs((int)subst[t]));
    const int64_t bound = ((int64_t)smax + (int64_t)-gap_open + (int64_t)-gap_extend) * 2 *
                          ((int64_t)S.max_len + 1);
    SAD_CHECK(bound < (1ll << 29), SAD_EINVAL, "scores could exceed the 32-bit DP range");
    const int32_t* dbo = bucket_offsets;
    const int32_t* dord = order;
    int64_t* dso = score_offsets;
    int32_t* dsc = scores;
    int64_t total = 0;
    if (mem == SAD_MEM_HOST) {
        void* st = nullptr;
        SAD_RET(workspace(ctx, WS_PART_OUT, 4ull * (p + 1 + n) + 8ull * (p + 1) + 1024, stream, &st));
        int32_t* s32 = (int32_t*)st;
        SAD_CUDA(cudaMemcpyAsync(s32, bucket_offsets, 4ull * (p + 1), cudaMemcpyHostToDevice, stream));
        if (n) SAD_CUDA(cudaMemcpyAsync(s32 + p + 1, order, 4ull * n, cudaMemcpyHostToDevice, stream));
        dbo = s32;
        dord = s32 + p + 1;
        dso = (int64_t*)(((uintptr_t)(s32 + p + 1 + n) + 15) & ~(uintptr_t)15);
        SAD_RET(sad_scores_size(bucket_offsets, p, SAD_MEM_HOST, &total));
        if (total <= scores_capacity) {
            void* so = nullptr;
            SAD_RET(workspace(ctx, WS_SCORE_OUT, 4ull * (total + 1), stream, &so));
            dsc = (int32_t*)so;
        }
    }
    int rc = bucket_scores_device(ctx, S, dbo, dord, p, subst, gap_open, gap_extend, mode, dso, dsc,
                                  scores_capacity, &total, stream);
    if (mem == SAD_MEM_HOST) {
        SAD_CUDA(cudaMemcpyAsync(score_offsets, dso, 8ull * (p + 1), cudaMemcpyDeviceToHost, stream));
        if (rc == SAD_OK && total > 0)
            SAD_CUDA(cudaMemcpyAsync(scores, dsc, 4ull * total, cudaMemcpyDeviceToHost, stream));
    }
    if (rc != SAD_OK) {
        cudaStreamSynchronize(stream);
        return rc;
    }
    SAD_RET(status_check(ctx, stream));
    return SAD_OK;
}

}  // namespace sad

extern "C" int sad_bucket_pair_scores(sad_ctx* ctx_in, const sad_seqset* seqs,
                                      const int32_t* bucket_offsets, const int32_t* order, int32_t p,
                                      const int8_t* subst, int32_t gap_open, int32_t gap_extend,
                                      int32_t mode, int64_t* score_offsets, int32_t* scores,
                                      int64_t scores_capacity, int32_t mem, void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mem == SAD_MEM_HOST || mem == SAD_MEM_DEVICE, SAD_EINVAL, "mem = %d", mem);
    SAD_CHECK(seqs && bucket_offsets && score_offsets && subst, SAD_EINVAL, "a required pointer is NULL");
    SAD_CHECK(p >= 1, SAD_EINVAL, "p = %d < 1", p);
    SAD_CHECK(gap_open <= 0 && gap_extend <= 0, SAD_EINVAL,
              "gap costs must be <= 0 (got open %d, extend %d)", gap_open, gap_extend);
    SAD_CHECK(gap_open >= -(1 << 20) && gap_extend >= -(1 << 20), SAD_EINVAL, "gap costs too large");
    const int32_t A = seqs->alphabet;
    SAD_CHECK(A >= 1 && A <= SAD_MAX_ALPHABET, SAD_EINVAL, "alphabet %d", A);
    for (int32_t x = 0; x < A; x++)
        for (int32_t y = 0; y < A; y++)
            SAD_CHECK(subst[x * A + y] == subst[y * A + x], SAD_EINVAL,
                      "substitution matrix is not symmetric at (%d, %d)", x, y);
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    return bucket_pair_scores_locked(ctx, seqs, bucket_offsets, order, p, subst, gap_open, gap_extend, mode,
                                     score_offsets, scores, scores_capacity, mem, (cudaStream_t)stream_ptr);
}
