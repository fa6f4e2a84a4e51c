// Stage 1 of Sample-Align-D: k-mer counts, all-pairs k-mer similarity, the
// fixed-point D sums, local/global ancestors and the rank keys (Section 2
// "k-mer Rank"; algorithm box: "locally compute k-mer rank", local ancestors
// gathered, global ancestor determined and broadcast).
#include <cmath>
#include <cstring>

#include "kmer_common.cuh"
#include "kmer_stage.cuh"
#include "sad_internal.cuh"

namespace sad {

namespace {

constexpr int kCountThreads = 256;

// ---------------------------------------------------------------------------
// K1: one CTA per sequence. k-mer histogram in shared memory, then
//   C8[i][tau]        = min(count, 255)                       (uint8, stride Vs)
//   planes[i][(t-1)Vs + tau] = e4m3(1.0) if count >= t, t = 1..cap  (optional)
//   sT[i]             = sum_tau min(count, T)
//   excess list of i  = (tau, count - T) for count > T, ascending tau
//   kbits[i / 128]   |= the nonzero 128-byte k-blocks of the plane row (optional)
// T is the residual threshold: cap on the plane path, 255 on the uint8 path.
constexpr int kMaxKBlockWords = (8 * SAD_MAX_KMER_SPACE / 128 + 31) / 32 + 1;

__global__ void __launch_bounds__(kCountThreads)
k_count(const uint8_t* __restrict__ res, const int64_t* __restrict__ pad_off,
        const int32_t* __restrict__ len, int32_t k, int32_t A2, int32_t Vs, ClassMap cm,
        int32_t T, int32_t cap, uint8_t* __restrict__ C8, uint8_t* __restrict__ planes,
        const int64_t* __restrict__ ex_off, int32_t* __restrict__ ex_tau,
        int32_t* __restrict__ ex_val, int32_t* __restrict__ nex, uint32_t* __restrict__ sT,
        uint32_t* __restrict__ kbits, int32_t kbwords) {
    extern __shared__ uint32_t cnt[];  // Vs counters
    __shared__ int32_t warp_tot[kCountThreads / 32];
    __shared__ uint32_t red[kCountThreads / 32];
    __shared__ uint32_t kbm[kMaxKBlockWords];  // this row's nonzero k-blocks
    const int32_t i = blockIdx.x;
    const int32_t L = len[i];
    const uint8_t* x = res + pad_off[i];
    for (int32_t t = threadIdx.x; t < Vs; t += blockDim.x) cnt[t] = 0;
    for (int32_t t = threadIdx.x; t < kbwords; t += blockDim.x) kbm[t] = 0;
    __syncthreads();
    const int32_t nk = L - k + 1;
    for (int32_t pos = threadIdx.x; pos < nk; pos += blockDim.x) {
        uint32_t code = 0;
        for (int32_t t = 0; t < k; t++) code = code * (uint32_t)A2 + cm.c[x[pos + t]];
        atomicAdd(&cnt[code], 1u);
    }
    __syncthreads();
    uint32_t ssum = 0;
    bool heavy = false;
    uint8_t* crow = C8 + (int64_t)i * Vs;
    uint8_t* prow = planes ? planes + (int64_t)i * cap * Vs : nullptr;
    for (int32_t t4 = threadIdx.x * 4; t4 < Vs; t4 += blockDim.x * 4) {
        const uint32_t c0 = cnt[t4], c1 = cnt[t4 + 1], c2 = cnt[t4 + 2], c3 = cnt[t4 + 3];
        const uint32_t T32 = (uint32_t)T;
        ssum += min(c0, T32) + min(c1, T32) + min(c2, T32) + min(c3, T32);
        heavy |= (c0 > T32) | (c1 > T32) | (c2 > T32) | (c3 > T32);
        *(uint32_t*)(crow + t4) =
            min(c0, 255u) | (min(c1, 255u) << 8) | (min(c2, 255u) << 16) | (min(c3, 255u) << 24);
        if (prow) {
            for (int32_t t = 1; t <= cap; t++) {
                const uint32_t tt = (uint32_t)t;
                const uint32_t w = (c0 >= tt ? 0x38u : 0u) | (c1 >= tt ? 0x3800u : 0u) |
                                   (c2 >= tt ? 0x380000u : 0u) | (c3 >= tt ? 0x38000000u : 0u);
                *(uint32_t*)(prow + (int64_t)(t - 1) * Vs + t4) = w;
                if (kbits && w) {
                    const int32_t kb = ((t - 1) * Vs + t4) >> 7;
                    atomicOr(&kbm[kb >> 5], 1u << (kb & 31));
                }
            }
        }
    }
    // block sum of ssum
    for (int o = 16; o > 0; o >>= 1) ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = ssum;
    const int any_heavy = __syncthreads_or(heavy ? 1 : 0);
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int q = 0; q < kCountThreads / 32; q++) s += red[q];
        sT[i] = s;
    }
    if (kbits)
        for (int32_t t = threadIdx.x; t < kbwords; t += blockDim.x)
            if (kbm[t]) atomicOr(&kbits[(int64_t)(i >> 7) * kbwords + t], kbm[t]);
    if (!any_heavy) {
        if (threadIdx.x == 0) nex[i] = 0;
        return;
    }
    // ordered compaction of the counts above T (ascending tau)
    const int64_t eo = ex_off[i];
    int32_t base = 0;
    for (int32_t t0 = 0; t0 < Vs; t0 += blockDim.x) {
        const int32_t tau = t0 + threadIdx.x;
        const bool f = tau < Vs && cnt[tau] > (uint32_t)T;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_tot[w] = __popc(bal);
        __syncthreads();
        int32_t before = 0, total = 0;
        for (int q = 0; q < kCountThreads / 32; q++) {
            const int32_t v = warp_tot[q];
            before += q < w ? v : 0;
            total += v;
        }
        if (f) {
            const int32_t pos = base + before + __popc(bal & ((1u << lane) - 1u));
            ex_tau[eo + pos] = tau;
            ex_val[eo + pos] = (int32_t)cnt[tau] - T;
        }
        base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) nex[i] = base;
}

// Ordered index of the sequences that have an excess list (one CTA).
__global__ void k_heavy_index(int32_t n, const int32_t* __restrict__ nex, int32_t* __restrict__ hidx,
                              int32_t* __restrict__ hlist, int32_t* __restrict__ H) {
    __shared__ int32_t warp_tot[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int32_t base = 0;
    for (int32_t t0 = 0; t0 < n; t0 += blockDim.x) {
        const int32_t i = t0 + threadIdx.x;
        const bool f = i < n && nex[i] > 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_tot[w] = __popc(bal);
        __syncthreads();
        int32_t before = 0, total = 0;
        for (int q = 0; q < nw; q++) {
            before += q < w ? warp_tot[q] : 0;
            total += warp_tot[q];
        }
        if (i < n) {
            const int32_t h = f ? base + before + __popc(bal & ((1u << lane) - 1u)) : -1;
            hidx[i] = h;
            if (f) hlist[h] = i;
        }
        base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *H = base;
}

// Residual numerators R[h1][h2] = sum_tau min(excess_i(tau), excess_j(tau))
// = sum_tau max(0, min(c_i, c_j) - T) for every pair of sequences with
// excess lists (merge of two tau-sorted lists).
// H heavy sequences: *Hp when Hp is given (read on the device, so that the host
// need not wait for it), else Hhost; R is row-major with row length `stride`.
__global__ void k_residual(const int32_t* __restrict__ Hp, int32_t Hhost, int32_t stride,
                           const int32_t* __restrict__ hlist, const int64_t* __restrict__ ex_off,
                           const int32_t* __restrict__ ex_tau, const int32_t* __restrict__ ex_val,
                           const int32_t* __restrict__ nex, int32_t* __restrict__ R) {
    const int64_t H = Hp ? *Hp : Hhost;
    const int64_t npairs = H * (H + 1) / 2;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npairs;
         q += (int64_t)gridDim.x * blockDim.x) {
        // row h1 of the upper triangle starts at h1*H - h1*(h1-1)/2
        double disc = (2.0 * H + 1.0) * (2.0 * H + 1.0) - 8.0 * (double)q;
        int64_t h1 = (int64_t)floor(((2.0 * H + 1.0) - sqrt(disc)) / 2.0);
        if (h1 < 0) h1 = 0;
        if (h1 > H - 1) h1 = H - 1;
        while (h1 > 0 && h1 * H - h1 * (h1 - 1) / 2 > q) h1--;
        while (h1 + 1 < H && (h1 + 1) * H - (h1 + 1) * h1 / 2 <= q) h1++;
        const int64_t h2 = h1 + (q - (h1 * H - h1 * (h1 - 1) / 2));
        const int32_t i = hlist[h1], j = hlist[h2];
        const int32_t* ta = ex_tau + ex_off[i];
        const int32_t* va = ex_val + ex_off[i];
        const int32_t* tb = ex_tau + ex_off[j];
        const int32_t* vb = ex_val + ex_off[j];
        const int32_t na = nex[i], nb = nex[j];
        int32_t x = 0, y = 0, s = 0;
        while (x < na && y < nb) {
            const int32_t a = ta[x], b = tb[y];
            if (a == b) {
                s += min(va[x], vb[y]);
                x++;
                y++;
            } else if (a < b) {
                x++;
            } else {
                y++;
            }
        }
        R[h1 * stride + h2] = s;
        R[h2 * stride + h1] = s;
    }
}

__device__ __forceinline__ uint32_t absdiff4_add(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// ---------------------------------------------------------------------------
// K3a: all-pairs sum_tau min(C_i, C_j) on uint8 count rows (CUDA cores), with
// the fixed-point epilogue fused. One CTA per 64x64 tile of the upper
// triangle; 256 threads, each 4x4 pairs (rows ty+16r, columns tx+16c).
// sum min(x, y) = (sum x + sum y - sum |x - y|) / 2 on the saturated bytes,
// so the inner loop is one vabsdiff4 (four |x-y| plus accumulate) per 4 bytes.
constexpr int kTile = 64;
constexpr int kKC = 64;             // bytes of k per stage
constexpr int kRowB = kKC + 16;     // smem row pitch (bank spread)

// One 64 x 64 tile of sum_tau |x_tau - y_tau| over uint8 count rows of Vs
// bytes (a multiple of kKC): acc[r][c] for the A row ty + 16r and the B row
// tx + 16c. Every thread stages 16 bytes of row lr = tid / 4 of A and of B per
// kKC-byte chunk from ga / gb (its own row pointers, offset by its byte lc;
// va / vb false: a zero row), double-buffered through As / Bs. With kClamp
// every byte is first clamped to T (T4 holds T in each byte), so the sums are
// those of min(count, T).
__device__ __forceinline__ uint4 clamp_bytes(uint4 v, uint32_t T4) {
    return make_uint4(__vminu4(v.x, T4), __vminu4(v.y, T4), __vminu4(v.z, T4), __vminu4(v.w, T4));
}

template <bool kClamp>
__device__ __forceinline__ void sad_tile_64(const uint8_t* __restrict__ ga, const uint8_t* __restrict__ gb,
                                            bool va, bool vb, int32_t Vs, uint32_t T4,
                                            uint8_t (*As)[kTile][kRowB], uint8_t (*Bs)[kTile][kRowB],
                                            uint32_t (&acc)[4][4]) {
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int lr = tid >> 2, lc = (tid & 3) * 16;
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0;
    const int nchunks = Vs / kKC;
    uint4 ra = va ? *(const uint4*)ga : make_uint4(0, 0, 0, 0);
    uint4 rb = vb ? *(const uint4*)gb : make_uint4(0, 0, 0, 0);
    if (kClamp) {
        ra = clamp_bytes(ra, T4);
        rb = clamp_bytes(rb, T4);
    }
    *(uint4*)&As[0][lr][lc] = ra;
    *(uint4*)&Bs[0][lr][lc] = rb;
    __syncthreads();
    for (int ch = 0; ch < nchunks; ch++) {
        const int cur = ch & 1;
        if (ch + 1 < nchunks) {
            ra = va ? *(const uint4*)(ga + (int64_t)(ch + 1) * kKC) : make_uint4(0, 0, 0, 0);
            rb = vb ? *(const uint4*)(gb + (int64_t)(ch + 1) * kKC) : make_uint4(0, 0, 0, 0);
            if (kClamp) {
                ra = clamp_bytes(ra, T4);
                rb = clamp_bytes(rb, T4);
            }
        }
#pragma unroll
        for (int kq = 0; kq < kKC; kq += 16) {
            uint4 a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; r++) a[r] = *(const uint4*)&As[cur][ty + 16 * r][kq];
#pragma unroll
            for (int c = 0; c < 4; c++) b[c] = *(const uint4*)&Bs[cur][tx + 16 * c][kq];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    uint32_t s = acc[r][c];
                    s = absdiff4_add(a[r].x, b[c].x, s);
                    s = absdiff4_add(a[r].y, b[c].y, s);
                    s = absdiff4_add(a[r].z, b[c].z, s);
                    s = absdiff4_add(a[r].w, b[c].w, s);
                    acc[r][c] = s;
                }
        }
        if (ch + 1 < nchunks) {
            *(uint4*)&As[cur ^ 1][lr][lc] = ra;
            *(uint4*)&Bs[cur ^ 1][lr][lc] = rb;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
k_allpairs_u8(int32_t n, int32_t Vs, int32_t ntiles, const uint8_t* __restrict__ C8,
              const uint32_t* __restrict__ sT, SeqTables tab, uint64_t* __restrict__ dloc,
              uint64_t* __restrict__ dcen, int32_t* __restrict__ A) {
    __shared__ __align__(16) uint8_t As[2][kTile][kRowB];
    __shared__ __align__(16) uint8_t Bs[2][kTile][kRowB];
    __shared__ unsigned long long colc[kTile], coll[kTile];
    // tile (ti, tj), ti <= tj, row-major over the upper triangle
    const int64_t idx = blockIdx.x;
    int32_t ti = (int32_t)floor(((2.0 * ntiles + 1.0) -
                                 sqrt((2.0 * ntiles + 1.0) * (2.0 * ntiles + 1.0) - 8.0 * idx)) / 2.0);
    if (ti < 0) ti = 0;
    if (ti > ntiles - 1) ti = ntiles - 1;
    while (ti > 0 && (int64_t)ti * ntiles - (int64_t)ti * (ti - 1) / 2 > idx) ti--;
    while (ti + 1 < ntiles && (int64_t)(ti + 1) * ntiles - (int64_t)(ti + 1) * ti / 2 <= idx) ti++;
    const int32_t tj = ti + (int32_t)(idx - ((int64_t)ti * ntiles - (int64_t)ti * (ti - 1) / 2));
    const int32_t i0 = ti * kTile, j0 = tj * kTile;
    const bool diag = ti == tj;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    if (tid < kTile) {
        colc[tid] = 0;
        coll[tid] = 0;
    }
    // loader: thread -> (row lr, 16-byte chunk lc) of a 64 x 64-byte stage
    const int lr = tid >> 2, lc = (tid & 3) * 16;
    const bool va = i0 + lr < n, vb = j0 + lr < n;
    const uint8_t* ga = C8 + (int64_t)(i0 + lr) * Vs + lc;
    const uint8_t* gb = C8 + (int64_t)(j0 + lr) * Vs + lc;
    uint32_t acc[4][4];
    sad_tile_64<false>(ga, gb, va, vb, Vs, 0u, As, Bs, acc);
    // epilogue: exact numerators, fixed-point terms, row/column sums
    int32_t ci[4], cnk[4], cbl[4], chx[4];
    uint64_t cq[4];
    uint32_t cr[4], cs[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int32_t j = j0 + tx + 16 * c;
        ci[c] = j;
        const bool ok = j < n;
        cnk[c] = ok ? tab.nkb[j] : 0;
        cq[c] = ok ? tab.q32[j] : 0;
        cr[c] = ok ? tab.r32[j] : 0;
        cbl[c] = ok ? tab.blk[j] : -1;
        chx[c] = ok ? tab.hidx[j] : -1;
        cs[c] = ok ? sT[j] : 0;
    }
    uint64_t colsum_c[4] = {0, 0, 0, 0}, colsum_l[4] = {0, 0, 0, 0};
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int32_t i = i0 + ty + 16 * r;
        const bool oki = i < n;
        const int32_t nki = oki ? tab.nkb[i] : 0;
        const uint64_t qi = oki ? tab.q32[i] : 0;
        const uint32_t ri = oki ? tab.r32[i] : 0;
        const int32_t bli = oki ? tab.blk[i] : -2;
        const int32_t hxi = oki ? tab.hidx[i] : -1;
        const uint32_t si = oki ? sT[i] : 0;
        uint64_t rs_c = 0, rs_l = 0;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (!oki || ci[c] >= n) continue;
            const uint32_t a = ((si + cs[c] - acc[r][c]) >> 1) + (uint32_t)residual_at(tab, hxi, chx[c]);
            const uint64_t t = fixed_term(a, nki, qi, ri, cnk[c], cq[c], cr[c]);
            const uint64_t tl = (bli == cbl[c]) ? t : 0;
            rs_c += t;
            rs_l += tl;
            colsum_c[c] += t;
            colsum_l[c] += tl;
            if (A) {
                A[(int64_t)i * n + ci[c]] = (int32_t)a;
                if (!diag) A[(int64_t)ci[c] * n + i] = (int32_t)a;
            }
        }
        // reduce over the 16 tx lanes that share row i
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            rs_c += __shfl_xor_sync(0xffffffffu, rs_c, o);
            rs_l += __shfl_xor_sync(0xffffffffu, rs_l, o);
        }
        if (tx == 0 && oki) {
            atomicAdd((unsigned long long*)&dcen[i], (unsigned long long)rs_c);
            atomicAdd((unsigned long long*)&dloc[i], (unsigned long long)rs_l);
        }
    }
    if (!diag) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (colsum_c[c]) atomicAdd(&colc[tx + 16 * c], (unsigned long long)colsum_c[c]);
            if (colsum_l[c]) atomicAdd(&coll[tx + 16 * c], (unsigned long long)colsum_l[c]);
        }
        __syncthreads();
        if (tid < kTile && j0 + tid < n) {
            if (colc[tid]) atomicAdd((unsigned long long*)&dcen[j0 + tid], colc[tid]);
            if (coll[tid]) atomicAdd((unsigned long long*)&dloc[j0 + tid], coll[tid]);
        }
    }
}

// sum_tau min(x_tau, y_tau, T) over two uint8 count rows, one warp.
__device__ uint32_t warp_minsum(const uint8_t* __restrict__ x, const uint8_t* __restrict__ y,
                                int32_t Vs, uint32_t T) {
    uint32_t s = 0;
    const int lane = threadIdx.x & 31;
    for (int32_t o = lane * 16; o < Vs; o += 32 * 16) {
        const uint4 a = *(const uint4*)(x + o);
        const uint4 b = *(const uint4*)(y + o);
        const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const uint32_t u = (aw[q] >> (8 * t)) & 0xffu, v = (bw[q] >> (8 * t)) & 0xffu;
                s += min(min(u, v), T);
            }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Local ancestor of block b: argmax of dloc over [floor(bN/p), floor((b+1)N/p)),
// lowest index on ties; -1 for an empty block. One CTA per block.
__global__ void k_local_ancestors(int32_t n, int32_t p, const uint64_t* __restrict__ dloc,
                                  int32_t* __restrict__ la) {
    __shared__ unsigned long long bv[32];
    __shared__ int32_t bi[32];
    const int32_t b = blockIdx.x;
    const int64_t lo = (int64_t)b * n / p, hi = (int64_t)(b + 1) * n / p;
    unsigned long long best = 0;
    int32_t besti = -1;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const unsigned long long v = dloc[i];
        if (besti < 0 || v > best) {
            best = v;
            besti = (int32_t)i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int32_t oi = __shfl_xor_sync(0xffffffffu, besti, o);
        if (oi >= 0 && (besti < 0 || ov > best || (ov == best && oi < besti))) {
            best = ov;
            besti = oi;
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        bv[w] = best;
        bi[w] = besti;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < nw; q++)
            if (bi[q] >= 0 && (besti < 0 || bv[q] > best || (bv[q] == best && bi[q] < besti))) {
                best = bv[q];
                besti = bi[q];
            }
        la[b] = besti;
    }
}

// Global-ancestor scores: gsum[b] = sum over non-empty b2 of the fixed-point
// term of (LA_b, LA_b2). One CTA per block; one warp per partner.
__global__ void k_ga_sums(int32_t p, const int32_t* __restrict__ la, const uint8_t* __restrict__ C8,
                          int32_t Vs, uint32_t T, SeqTables tab, uint64_t* __restrict__ gsum) {
    __shared__ unsigned long long acc;
    const int32_t b = blockIdx.x;
    const int32_t x = la[b];
    if (threadIdx.x == 0) acc = 0;
    __syncthreads();
    if (x >= 0) {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int32_t b2 = w; b2 < p; b2 += nw) {
            const int32_t y = la[b2];
            if (y < 0) continue;
            uint32_t a = warp_minsum(C8 + (int64_t)x * Vs, C8 + (int64_t)y * Vs, Vs, T);
            a += (uint32_t)residual_at(tab, tab.hidx[x], tab.hidx[y]);
            if (lane == 0)
                atomicAdd(&acc, (unsigned long long)fixed_term(a, tab.nkb[x], tab.q32[x], tab.r32[x],
                                                               tab.nkb[y], tab.q32[y], tab.r32[y]));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) gsum[b] = acc;
}

// GA = the local ancestor with the largest score (lowest index on ties).
__global__ void k_ga_select(int32_t p, const int32_t* __restrict__ la,
                            const uint64_t* __restrict__ gsum, int32_t* __restrict__ ga) {
    if (threadIdx.x != 0) return;
    int32_t g = -1;
    uint64_t best = 0;
    for (int32_t b = 0; b < p; b++) {
        const int32_t x = la[b];
        if (x < 0) continue;
        if (g < 0 || gsum[b] > best || (gsum[b] == best && x < g)) {
            g = x;
            best = gsum[b];
        }
    }
    *ga = g;
}

// Rank keys against the global ancestor; one warp per sequence.
__global__ void k_key_column(int32_t n, const int32_t* __restrict__ ga_ptr,
                             const uint8_t* __restrict__ C8, int32_t Vs, uint32_t T, SeqTables tab,
                             int32_t* __restrict__ key_a, int32_t* __restrict__ key_b) {
    const int32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const int32_t g = *ga_ptr;
    const int32_t b = min(tab.nkb[i], tab.nkb[g]);
    if (b <= 0) {
        if ((threadIdx.x & 31) == 0) {
            key_a[i] = 0;
            key_b[i] = 1;
        }
        return;
    }
    uint32_t a = warp_minsum(C8 + (int64_t)i * Vs, C8 + (int64_t)g * Vs, Vs, T);
    a += (uint32_t)residual_at(tab, tab.hidx[i], tab.hidx[g]);
    if ((threadIdx.x & 31) == 0) {
        key_a[i] = (int32_t)a;
        key_b[i] = b;
    }
}

// Per-sequence tables of the fixed-point terms: nkb = |x_i| - k + 1, q32 =
// floor(2^32 / nkb), r32 = 2^32 mod nkb, inv = 1/nkb in fp32 (zeros when no
// k-mer fits), and the block of i (largest b with floor(b n / p) <= i).
__global__ void k_seq_tables(int32_t n, int32_t k, int32_t p, const int32_t* __restrict__ len,
                             int32_t* __restrict__ nkb, uint64_t* __restrict__ q32, uint32_t* __restrict__ r32,
                             float* __restrict__ inv, int32_t* __restrict__ blk) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t nk = len[i] - k + 1;
    nkb[i] = nk;
    if (nk >= 1) {
        q32[i] = (1ull << 32) / (uint64_t)nk;
        r32[i] = (uint32_t)((1ull << 32) % (uint64_t)nk);
        inv[i] = 1.0f / (float)nk;
    } else {
        q32[i] = 0;
        r32[i] = 0;
        inv[i] = 0.0f;
    }
    int64_t b = ((int64_t)i * p) / n;
    while (b + 1 < p && (b + 1) * n / p <= i) b++;
    while (b > 0 && b * n / p > i) b--;
    blk[i] = (int32_t)b;
}

// Prefix offsets (one CTA): exoff of the excess lists (nkb / (T+1) entries per
// sequence at most) and loff of the sorted k-mer lists (nkb entries). Thread t
// owns the contiguous segment [t*w, (t+1)*w): it sums its segment, one block
// scan gives every segment's start, and it writes its segment's offsets.
__global__ void __launch_bounds__(1024)
k_seq_offsets(int32_t n, int32_t k, int32_t T, const int32_t* __restrict__ len, int64_t* __restrict__ exoff,
              int64_t* __restrict__ loff) {
    __shared__ long long wex[32], wl[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t seg = (n + (int32_t)blockDim.x - 1) / (int32_t)blockDim.x;
    const int32_t lo = min(n, (int32_t)threadIdx.x * seg), hi = min(n, lo + seg);
    long long ex = 0, l = 0;
    for (int32_t i = lo; i < hi; i++) {
        const int32_t nk = len[i] - k + 1;
        if (nk > 0) {
            ex += nk / (T + 1);
            l += nk;
        }
    }
    // exclusive scan of the segment sums over the block
    long long iex = ex, il = l;
    for (int o = 1; o < 32; o <<= 1) {
        const long long a = __shfl_up_sync(0xffffffffu, iex, o), b = __shfl_up_sync(0xffffffffu, il, o);
        if (lane >= o) {
            iex += a;
            il += b;
        }
    }
    if (lane == 31) {
        wex[w] = iex;
        wl[w] = il;
    }
    __syncthreads();
    long long bex = 0, bl = 0;
    for (int q = 0; q < w; q++) {
        bex += wex[q];
        bl += wl[q];
    }
    long long cex = bex + iex - ex, cl = bl + il - l;  // offsets of my segment's first sequence
    if (threadIdx.x == 0) {
        exoff[0] = 0;
        loff[0] = 0;
    }
    for (int32_t i = lo; i < hi; i++) {
        const int32_t nk = len[i] - k + 1;
        if (nk > 0) {
            cex += nk / (T + 1);
            cl += nk;
        }
        exoff[i + 1] = cex;
        loff[i + 1] = cl;
    }
}

// ---------------------------------------------------------------------------
// Globalized rank (Section 2.3.1: every block's sample set goes to all blocks
// and every sequence is ranked against the s*p samples).

// Position of every sequence in its block ordered by (dloc, index):
// grid (p, chunks of 256 members); sorted[lo + r] = i.
__global__ void k_block_order(int32_t n, int32_t p, const uint64_t* __restrict__ dloc,
                              int32_t* __restrict__ sorted) {
    __shared__ unsigned long long tile[1024];
    const int32_t b = blockIdx.x;
    const int64_t lo = (int64_t)b * n / p, hi = (int64_t)(b + 1) * n / p;
    const int64_t i = lo + (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (lo + (int64_t)blockIdx.y * blockDim.x >= hi) return;  // whole CTA idle (uniform)
    const unsigned long long d = i < hi ? dloc[i] : 0ull;
    int32_t r = 0;
    for (int64_t t0 = lo; t0 < hi; t0 += 1024) {
        const int64_t m = min((int64_t)1024, hi - t0);
        __syncthreads();
        for (int64_t t = threadIdx.x; t < m; t += blockDim.x) tile[t] = dloc[t0 + t];
        __syncthreads();
        for (int64_t t = 0; t < m; t++) {
            const unsigned long long v = tile[t];
            r += (v < d) | ((v == d) & (t0 + t < i));
        }
    }
    if (i < hi) sorted[lo + r] = (int32_t)i;
}

// Sample slot (b, j): the member at 0-based position floor((2j+1) w / (2s)) of
// block b in (dloc, index) order; -1 for an empty block.
__global__ void k_pick_samples(int32_t n, int32_t p, int32_t s, const int32_t* __restrict__ sorted,
                               int32_t* __restrict__ samples) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)p * s) return;
    const int64_t b = t / s, j = t % s;
    const int64_t lo = b * n / p, hi = (b + 1) * n / p, w = hi - lo;
    samples[t] = w > 0 ? sorted[lo + ((2 * j + 1) * w) / (2 * (int64_t)s)] : -1;
}

// G_i = sum over the sample slots of floor(a_i,sigma 2^32 / b_i,sigma): one CTA
// per 64 rows x 64 slots, the numerators from the byte sums clamped to T (plus
// the residual above T), each row's 64 terms summed and added to G_i.
template <bool kClamp>
__global__ void __launch_bounds__(256)
k_sample_sums(int32_t n, int32_t nslots, int32_t Vs, uint32_t T, const uint8_t* __restrict__ C8,
              const uint32_t* __restrict__ sT, SeqTables tab, const int32_t* __restrict__ samples,
              uint64_t* __restrict__ G) {
    __shared__ __align__(16) uint8_t As[2][kTile][kRowB];
    __shared__ __align__(16) uint8_t Bs[2][kTile][kRowB];
    const int32_t i0 = blockIdx.x * kTile, j0 = blockIdx.y * kTile;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int lr = tid >> 2, lc = (tid & 3) * 16;
    const int32_t sl = j0 + lr < nslots ? samples[j0 + lr] : -1;
    const bool va = i0 + lr < n, vb = sl >= 0;
    const uint8_t* ga = C8 + (int64_t)(va ? i0 + lr : 0) * Vs + lc;
    const uint8_t* gb = C8 + (int64_t)(vb ? sl : 0) * Vs + lc;
    uint32_t acc[4][4];
    sad_tile_64<kClamp>(ga, gb, va, vb, Vs, T * 0x01010101u, As, Bs, acc);
    int32_t cnk[4], chx[4];
    uint64_t cq[4];
    uint32_t cr[4], cs[4];
    bool cok[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int32_t j = j0 + tx + 16 * c;
        const int32_t sg = j < nslots ? samples[j] : -1;
        cok[c] = sg >= 0;
        cnk[c] = cok[c] ? tab.nkb[sg] : 0;
        cq[c] = cok[c] ? tab.q32[sg] : 0;
        cr[c] = cok[c] ? tab.r32[sg] : 0;
        chx[c] = cok[c] ? tab.hidx[sg] : -1;
        cs[c] = cok[c] ? sT[sg] : 0;
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int32_t i = i0 + ty + 16 * r;
        const bool oki = i < n;
        const int32_t nki = oki ? tab.nkb[i] : 0;
        const uint64_t qi = oki ? tab.q32[i] : 0;
        const uint32_t ri = oki ? tab.r32[i] : 0;
        const int32_t hxi = oki ? tab.hidx[i] : -1;
        const uint32_t si = oki ? sT[i] : 0;
        uint64_t rs = 0;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (!oki || !cok[c]) continue;
            const uint32_t a = ((si + cs[c] - acc[r][c]) >> 1) + (uint32_t)residual_at(tab, hxi, chx[c]);
            rs += fixed_term(a, nki, qi, ri, cnk[c], cq[c], cr[c]);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
        if (tx == 0 && oki && rs) atomicAdd((unsigned long long*)&G[i], (unsigned long long)rs);
    }
}

}  // namespace

bool uses_sparse_path(const sad_kmer_params* kp) {
    if (kp->cap == SAD_KMER_SPARSE) return true;
    int64_t V = 1;
    for (int t = 0; t < kp->k; t++) {
        V *= kp->kmer_alphabet;
        if (V > SAD_MAX_KMER_SPACE) return true;
    }
    return false;
}

int kmer_rank_device(sad_ctx* ctx, const DevSeqs& S, const sad_kmer_params* kp,
                     const KmerOutDev& out, cudaStream_t stream) {
    const int32_t n = S.n;
    const int32_t k = kp->k, A2 = kp->kmer_alphabet, p = kp->p;
    const bool sparse = uses_sparse_path(kp);
    const int32_t cap = sparse ? 0 : kp->cap;
    int64_t V = 1;
    for (int t = 0; t < k; t++) V = std::min<int64_t>(V * A2, (int64_t)1 << 40);
    const int32_t Vs = sparse ? 0 : (int32_t)round_up(V, 64);
    // counts above T are exact through the residual: the cap of the planes; on the
    // sorted-list path 1 with the byte table (it holds presence only), else 255
    const int32_t T = cap > 0 ? cap : (sparse && sparse_byte_table(ctx, V) ? 1 : 255);
    SAD_CHECK(cap == 0 || S.max_len - k + 1 < 65536, SAD_EINVAL,
              "the threshold-plane path takes sequences of fewer than 65536 k-mers (longest: %d); use cap = 0",
              S.max_len - k + 1);
    SAD_CHECK(!sparse || S.max_len - k + 1 <= SAD_MAX_SPARSE_KMERS, SAD_EINVAL,
              "the sorted-list path takes sequences of at most %d k-mers (longest: %d)", SAD_MAX_SPARSE_KMERS,
              S.max_len - k + 1);
    ClassMap cm;
    memset(&cm, 0, sizeof(cm));
    for (int32_t r = 0; r < S.alphabet; r++) cm.c[r] = kp->class_map ? kp->class_map[r] : (uint8_t)r;

    SAD_CUDA(cudaMemsetAsync(out.dloc, 0, sizeof(uint64_t) * (n > 0 ? n : 1), stream));
    SAD_CUDA(cudaMemsetAsync(out.dcen, 0, sizeof(uint64_t) * (n > 0 ? n : 1), stream));
    if (n == 0) {
        SAD_CUDA(cudaMemsetAsync(out.la, 0xff, sizeof(int32_t) * p, stream));
        SAD_CUDA(cudaMemsetAsync(out.ga, 0xff, sizeof(int32_t), stream));
        if (kp->global_samples > 0 && out.samples)
            SAD_CUDA(cudaMemsetAsync(out.samples, 0xff, 4ull * p * kp->global_samples, stream));
        return SAD_OK;
    }

    // per-sequence tables are computed on the device from the lengths; the host
    // keeps only the totals that size the excess and list workspaces
    int64_t ex_total = 0, list_total = 0;
    for (int32_t i = 0; i < n; i++) {
        const int64_t nk = (int64_t)S.h_len[i] - k + 1;
        if (nk > 0) {
            ex_total += nk / (T + 1);
            list_total += nk;
        }
    }
    // device layout of the misc slot
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_nkb = carve(4ull * n), o_blk = carve(4ull * n), o_q = carve(8ull * n),
                 o_r = carve(4ull * n), o_inv = carve(4ull * n), o_exoff = carve(8ull * (n + 1)),
                 o_loff = carve(8ull * (n + 1)), o_nex = carve(4ull * n), o_nd = carve(4ull * n),
                 o_sT = carve(4ull * n), o_hidx = carve(4ull * n), o_hlist = carve(4ull * n),
                 o_H = carve(16), o_gsum = carve(8ull * p);
    void* misc = nullptr;
    SAD_RET(workspace(ctx, WS_KMER_MISC, off, stream, &misc));
    {
        char* d = (char*)misc;
        TraceScope ts(ctx, SAD_STAGE_COUNT, stream);
        k_seq_tables<<<(n + 255) / 256, 256, 0, stream>>>(n, k, p, S.len, (int32_t*)(d + o_nkb),
                                                          (uint64_t*)(d + o_q), (uint32_t*)(d + o_r),
                                                          (float*)(d + o_inv), (int32_t*)(d + o_blk));
        SAD_LAUNCHED();
        k_seq_offsets<<<1, 1024, 0, stream>>>(n, k, T, S.len, (int64_t*)(d + o_exoff), (int64_t*)(d + o_loff));
        SAD_LAUNCHED();
    }
    char* dm = (char*)misc;
    SeqTables tab;
    tab.nkb = (const int32_t*)(dm + o_nkb);
    tab.q32 = (const uint64_t*)(dm + o_q);
    tab.r32 = (const uint32_t*)(dm + o_r);
    tab.inv = (const float*)(dm + o_inv);
    tab.blk = (const int32_t*)(dm + o_blk);
    tab.hidx = (const int32_t*)(dm + o_hidx);
    tab.R = nullptr;
    tab.H = 0;
    int32_t* d_nex = (int32_t*)(dm + o_nex);
    uint32_t* d_sT = (uint32_t*)(dm + o_sT);
    int32_t* d_hidx = (int32_t*)(dm + o_hidx);
    int32_t* d_hlist = (int32_t*)(dm + o_hlist);
    int32_t* d_H = (int32_t*)(dm + o_H);
    uint64_t* d_gsum = (uint64_t*)(dm + o_gsum);

    // counts (+ planes), or the sorted (code, count) lists
    void* c8 = nullptr;
    const int64_t nrows = round_up(n, 128);
    SAD_RET(workspace(ctx, WS_COUNTS, sparse ? (size_t)(8 * std::max<int64_t>(list_total, 1)) : (size_t)(nrows * Vs),
                      stream, &c8));
    SparseLists L{(const uint2*)c8, (const int64_t*)(dm + o_loff), (const int32_t*)(dm + o_nd)};
    uint8_t* planes = nullptr;
    KBlockMap kbm{nullptr, 0, 0};
    uint32_t* kbm_bits = nullptr;
    if (cap > 0) {
        void* pl = nullptr;
        SAD_RET(workspace(ctx, WS_PLANES, (size_t)(nrows * (int64_t)cap * Vs), stream, &pl));
        planes = (uint8_t*)pl;
        // nonzero k-blocks per 128-row panel, for the tensor-core tiles to skip zero ones
        kbm.npanels = (int32_t)(nrows / 128);
        kbm.kbwords = (int32_t)((((int64_t)cap * Vs + 127) / 128 + 31) / 32);
        void* kb = nullptr;
        SAD_RET(workspace(ctx, WS_KBLOCKS, 4ull * kbm.npanels * kbm.kbwords, stream, &kb));
        kbm_bits = (uint32_t*)kb;
        kbm.bits = kbm_bits;
        SAD_CUDA(cudaMemsetAsync(kb, 0, 4ull * kbm.npanels * kbm.kbwords, stream));
        // padding rows beyond n stay zero for the tensor-core tiles
        if (nrows > n)
            SAD_CUDA(cudaMemsetAsync(planes + (int64_t)n * cap * Vs, 0,
                                     (size_t)((nrows - n) * (int64_t)cap * Vs), stream));
    }
    void* exb = nullptr;
    const int64_t excap = ex_total > 0 ? ex_total : 1;
    SAD_RET(workspace(ctx, WS_EXCESS, (size_t)(8 * excap), stream, &exb));
    int32_t* ex_tau = (int32_t*)exb;
    int32_t* ex_val = ex_tau + excap;
    const size_t smem = sizeof(uint32_t) * Vs;
    int32_t H = 0;
    {
    TraceScope ts(ctx, SAD_STAGE_COUNT, stream);
    if (sparse) {
        SAD_RET(sparse_count(ctx, S, k, A2, cm, T, (const int64_t*)(dm + o_loff), (uint2*)c8,
                             (int32_t*)(dm + o_nd), (const int64_t*)(dm + o_exoff), ex_tau, ex_val, d_nex,
                             stream));
    } else {
        if (smem > 40 * 1024)  // with the static shared memory above the default 48 KiB
            SAD_RET(allow_max_dynamic_smem(ctx, (const void*)k_count));
        k_count<<<n, kCountThreads, smem, stream>>>(S.res, S.pad_off, S.len, k, A2, Vs, cm, T, cap,
                                                   (uint8_t*)c8, planes, (const int64_t*)(dm + o_exoff),
                                                   ex_tau, ex_val, d_nex, d_sT, kbm.bits ? kbm_bits : nullptr,
                                                   kbm.kbwords);
        SAD_LAUNCHED();
    }
    k_heavy_index<<<1, 1024, 0, stream>>>(n, d_nex, d_hidx, d_hlist, d_H);
    SAD_LAUNCHED();
    }
    // Up to 4096 sequences on the dense paths the residual matrix is reserved for
    // every sequence (at most 64 MiB) and k_residual reads H on the device: no wait
    // here (N = 2000: the device idled 23 us for it). Otherwise, and on the
    // sorted-list path, which sizes its hash tables from the distinct k-mer counts,
    // the host reads H (and the counts) back.
    const bool device_H = !sparse && (int64_t)n * n <= (1ll << 24);
    std::vector<int32_t> nd_host;
    int32_t max_nd = 0;
    if (device_H && n > 0) {
        TraceScope ts(ctx, SAD_STAGE_COUNT, stream);
        void* rb = nullptr;
        SAD_RET(workspace(ctx, WS_HEAVY, sizeof(int32_t) * (size_t)n * n, stream, &rb));
        tab.R = (const int32_t*)rb;
        tab.H = n;  // the row length; rows and columns beyond the device's H are never read
        // a small grid: H is usually far below n, and the loop strides over any H
        const int64_t npairs = (int64_t)n * (n + 1) / 2;
        const int grid = (int)std::min<int64_t>((npairs + 255) / 256, (int64_t)ctx->num_sms * 2);
        k_residual<<<grid, 256, 0, stream>>>(d_H, 0, n, d_hlist, (const int64_t*)(dm + o_exoff), ex_tau, ex_val,
                                             d_nex, (int32_t*)rb);
        SAD_LAUNCHED();
    } else {
        SAD_CUDA(cudaMemcpyAsync(&H, d_H, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
        if (sparse) {
            nd_host.resize(n);
            SAD_CUDA(cudaMemcpyAsync(nd_host.data(), dm + o_nd, 4ull * n, cudaMemcpyDeviceToHost, stream));
        }
        SAD_CUDA(cudaStreamSynchronize(stream));
        for (int32_t v : nd_host) max_nd = std::max(max_nd, v);
    }
    if (!device_H && H > 0) {
        TraceScope ts(ctx, SAD_STAGE_COUNT, stream);
        SAD_CHECK((int64_t)H * H <= (1ll << 29), SAD_ENOMEM,
                  "%d sequences have k-mer counts above %d; the residual matrix would need %lld "
                  "entries",
                  H, T, (long long)H * H);
        void* rb = nullptr;
        SAD_RET(workspace(ctx, WS_HEAVY, sizeof(int32_t) * (size_t)H * H, stream, &rb));
        tab.R = (const int32_t*)rb;
        tab.H = H;
        const int64_t npairs = (int64_t)H * (H + 1) / 2;
        const int grid = (int)std::min<int64_t>((npairs + 255) / 256, (int64_t)ctx->num_sms * 16);
        k_residual<<<grid, 256, 0, stream>>>(nullptr, H, H, d_hlist, (const int64_t*)(dm + o_exoff), ex_tau,
                                             ex_val, d_nex, (int32_t*)rb);
        SAD_LAUNCHED();
    }
    // all pairs
    {
    TraceScope ts(ctx, SAD_STAGE_ALLPAIRS, stream);
    if (sparse) {
        SAD_RET(sparse_allpairs(ctx, n, L, tab, nd_host.data(), V, out.dloc, out.dcen, out.A, stream));
    } else if (cap > 0) {
        SAD_RET(allpairs_planes(ctx, n, cap * Vs, planes, kbm, tab, out.dloc, out.dcen, out.A, stream));
    } else {
        const int32_t ntiles = (int32_t)((n + kTile - 1) / kTile);
        const int64_t ntri = (int64_t)ntiles * (ntiles + 1) / 2;
        k_allpairs_u8<<<(unsigned)ntri, 256, 0, stream>>>(n, Vs, ntiles, (const uint8_t*)c8, d_sT,
                                                          tab, out.dloc, out.dcen, out.A);
        SAD_LAUNCHED();
    }
    }
    // ancestors and keys
    {
    TraceScope ts(ctx, SAD_STAGE_RANK, stream);
    k_local_ancestors<<<p, 256, 0, stream>>>(n, p, out.dloc, out.la);
    SAD_LAUNCHED();
    if (sparse) {
        SAD_RET(sparse_ga_sums(ctx, n, p, out.la, L, tab, max_nd, V, d_gsum, stream));
    } else {
        k_ga_sums<<<p, 256, 0, stream>>>(p, out.la, (const uint8_t*)c8, Vs, (uint32_t)T, tab, d_gsum);
        SAD_LAUNCHED();
    }
    k_ga_select<<<1, 32, 0, stream>>>(p, out.la, d_gsum, out.ga);
    SAD_LAUNCHED();
    if (sparse) {
        SAD_RET(sparse_key_column(ctx, n, out.ga, L, tab, max_nd, V, out.key_a, out.key_b, stream));
    } else {
        k_key_column<<<(n + 7) / 8, 256, 0, stream>>>(n, out.ga, (const uint8_t*)c8, Vs, (uint32_t)T,
                                                      tab, out.key_a, out.key_b);
        SAD_LAUNCHED();
    }
    }
    // globalized rank against s samples per block
    const int32_t gs = kp->global_samples;
    if (gs > 0 && out.G && out.samples) {
        TraceScope ts(ctx, SAD_STAGE_GLOBAL, stream);
        void* so = nullptr;
        SAD_RET(workspace(ctx, WS_GLOBAL, 4ull * n, stream, &so));
        int32_t* sorted = (int32_t*)so;
        const int64_t wmax = (n + p - 1) / p + 1;
        k_block_order<<<dim3((unsigned)p, (unsigned)((wmax + 255) / 256)), 256, 0, stream>>>(
            n, p, out.dloc, sorted);
        SAD_LAUNCHED();
        const int64_t nslots = (int64_t)p * gs;
        k_pick_samples<<<(unsigned)((nslots + 255) / 256), 256, 0, stream>>>(n, p, gs, sorted, out.samples);
        SAD_LAUNCHED();
        SAD_CUDA(cudaMemsetAsync(out.G, 0, 8ull * n, stream));
        const dim3 grid((unsigned)((n + kTile - 1) / kTile), (unsigned)((nslots + kTile - 1) / kTile));
        if (sparse)
            SAD_RET(sparse_sample_sums(ctx, n, (int32_t)nslots, out.samples, L, tab, max_nd, V, out.G, stream));
        else if (T < 255)
            k_sample_sums<true><<<grid, 256, 0, stream>>>(n, (int32_t)nslots, Vs, (uint32_t)T,
                                                          (const uint8_t*)c8, d_sT, tab, out.samples, out.G);
        else
            k_sample_sums<false><<<grid, 256, 0, stream>>>(n, (int32_t)nslots, Vs, (uint32_t)T,
                                                           (const uint8_t*)c8, d_sT, tab, out.samples, out.G);
        SAD_LAUNCHED();
    }
    return SAD_OK;
}

int validate_kmer_params(const sad_seqset* s, const sad_kmer_params* kp) {
    SAD_CHECK(kp != nullptr, SAD_EINVAL, "params is NULL");
    SAD_CHECK(kp->k >= 1, SAD_EINVAL, "k = %d < 1", kp->k);
    SAD_CHECK(kp->p >= 1 && kp->p <= 1024, SAD_EINVAL, "p = %d outside 1..1024", kp->p);
    SAD_CHECK(kp->cap >= SAD_KMER_SPARSE && kp->cap <= 8, SAD_EINVAL, "cap = %d outside -1..8", kp->cap);
    SAD_CHECK(kp->global_samples >= 0 && kp->global_samples <= SAD_MAX_GLOBAL_SAMPLES, SAD_EINVAL,
              "global_samples = %d outside 0..%d", kp->global_samples, SAD_MAX_GLOBAL_SAMPLES);
    SAD_CHECK(kp->kmer_alphabet >= 1 && kp->kmer_alphabet <= SAD_MAX_ALPHABET, SAD_EINVAL,
              "kmer_alphabet = %d outside 1..%d", kp->kmer_alphabet, SAD_MAX_ALPHABET);
    const bool sparse = uses_sparse_path(kp);
    SAD_CHECK(kp->cap <= 0 || !sparse, SAD_EINVAL,
              "k-mer space %d^%d exceeds SAD_MAX_KMER_SPACE (%d) of the threshold-plane path",
              kp->kmer_alphabet, kp->k, SAD_MAX_KMER_SPACE);
    int64_t V = 1;
    for (int t = 0; t < kp->k; t++) {
        V *= kp->kmer_alphabet;
        SAD_CHECK(V <= SAD_MAX_SPARSE_KMER_SPACE, SAD_EINVAL,
                  "k-mer space %d^%d exceeds SAD_MAX_SPARSE_KMER_SPACE", kp->kmer_alphabet, kp->k);
    }
    SAD_CHECK(s->alphabet >= 1 && s->alphabet <= SAD_MAX_ALPHABET, SAD_EINVAL,
              "alphabet %d outside 1..%d", s->alphabet, SAD_MAX_ALPHABET);
    if (kp->class_map) {
        for (int32_t r = 0; r < s->alphabet; r++)
            SAD_CHECK(kp->class_map[r] < kp->kmer_alphabet, SAD_EINVAL,
                      "class_map[%d] = %d >= kmer_alphabet %d", r, kp->class_map[r],
                      kp->kmer_alphabet);
    } else {
        SAD_CHECK(s->alphabet <= kp->kmer_alphabet, SAD_EINVAL,
                  "without a class map kmer_alphabet (%d) must be >= alphabet (%d)",
                  kp->kmer_alphabet, s->alphabet);
    }
    return SAD_OK;
}

}  // namespace sad

extern "C" int sad_kmer_rank(sad_ctx* ctx_in, const sad_seqset* seqs, const sad_kmer_params* params,
                             const sad_rank_out* out, int32_t mem, void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mem == SAD_MEM_HOST || mem == SAD_MEM_DEVICE, SAD_EINVAL, "mem = %d", mem);
    SAD_CHECK(out && out->dloc && out->dcen && out->la && out->ga && out->key_a && out->key_b,
              SAD_EINVAL, "an output pointer of sad_rank_out is NULL");
    SAD_CHECK(seqs != nullptr, SAD_EINVAL, "seqs is NULL");
    SAD_RET(validate_kmer_params(seqs, params));
    const int32_t gs = params->global_samples;
    SAD_CHECK(gs == 0 || (out->G && out->sample_idx), SAD_EINVAL,
              "global_samples = %d needs the G and sample_idx outputs", gs);
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    SAD_RET(status_clear(ctx, stream));
    DevSeqs S;
    SAD_RET(prepare_seqs(ctx, seqs, mem, stream, &S));
    const int32_t n = S.n, p = params->p;
    const size_t nslots = (size_t)p * gs;
    KmerOutDev d;
    void* stage = nullptr;
    if (mem == SAD_MEM_DEVICE) {
        d = KmerOutDev{out->dloc, out->dcen, out->la, out->ga, out->key_a, out->key_b, out->A};
        if (gs > 0) {
            d.G = out->G;
            d.samples = out->sample_idx;
        }
    } else {
        const size_t nn = (size_t)(n > 0 ? n : 1);
        const size_t bytes = 8 * nn * 2 + 4 * (size_t)p + 16 + 4 * nn * 2 +
                             (out->A ? 4 * (size_t)n * n : 0) + (gs > 0 ? 8 * nn + 4 * nslots : 0) +
                             10 * 256;
        SAD_RET(workspace(ctx, WS_RANK_OUT, bytes, stream, &stage));
        char* c = (char*)stage;
        size_t o = 0;
        auto take = [&](size_t b) {
            char* r = c + o;
            o = (size_t)round_up((int64_t)(o + b), 256);
            return r;
        };
        d.dloc = (uint64_t*)take(8 * nn);
        d.dcen = (uint64_t*)take(8 * nn);
        d.la = (int32_t*)take(4 * (size_t)p);
        d.ga = (int32_t*)take(16);
        d.key_a = (int32_t*)take(4 * nn);
        d.key_b = (int32_t*)take(4 * nn);
        d.A = out->A ? (int32_t*)take(4 * (size_t)n * n) : nullptr;
        if (gs > 0) {
            d.G = (uint64_t*)take(8 * nn);
            d.samples = (int32_t*)take(4 * nslots);
        }
    }
    SAD_RET(kmer_rank_device(ctx, S, params, d, stream));
    if (mem == SAD_MEM_HOST) {
        SAD_CUDA(cudaMemcpyAsync(out->dloc, d.dloc, 8ull * n, cudaMemcpyDeviceToHost, stream));
        SAD_CUDA(cudaMemcpyAsync(out->dcen, d.dcen, 8ull * n, cudaMemcpyDeviceToHost, stream));
        SAD_CUDA(cudaMemcpyAsync(out->la, d.la, 4ull * p, cudaMemcpyDeviceToHost, stream));
        SAD_CUDA(cudaMemcpyAsync(out->ga, d.ga, 4, cudaMemcpyDeviceToHost, stream));
        SAD_CUDA(cudaMemcpyAsync(out->key_a, d.key_a, 4ull * n, cudaMemcpyDeviceToHost, stream));
        SAD_CUDA(cudaMemcpyAsync(out->key_b, d.key_b, 4ull * n, cudaMemcpyDeviceToHost, stream));
        if (out->A)
            SAD_CUDA(cudaMemcpyAsync(out->A, d.A, 4ull * n * n, cudaMemcpyDeviceToHost, stream));
        if (gs > 0) {
            if (n > 0) SAD_CUDA(cudaMemcpyAsync(out->G, d.G, 8ull * n, cudaMemcpyDeviceToHost, stream));
            SAD_CUDA(cudaMemcpyAsync(out->sample_idx, d.samples, 4 * nslots, cudaMemcpyDeviceToHost, stream));
        }
    }
    SAD_RET(status_check(ctx, stream));
    return SAD_OK;
}
