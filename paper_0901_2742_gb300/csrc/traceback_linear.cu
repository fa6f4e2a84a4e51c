// Alignments in linear space: the optimal global affine-gap alignment of each
// pair, like sad_align_pairs, with memory per pair proportional to the
// sequence length instead of the product of the lengths (the per-processor
// aligner of Section 2.3.3 run on every pair of a bucket, whatever the lengths).
//
// Rows are split at the middle (Hirschberg's divide and conquer, with the
// affine-gap bookkeeping of Myers and Miller): for a block of rows i0..i1 and
// columns j0..j1 a forward pass over the top half gives, for every column j of
// the middle row, the best score of a path ending there (H) and of one ending
// in a vertical gap (V); a pass over the reversed bottom half gives the same for
// paths starting there. The optimal path crosses the middle at the column j
// that maximises Hf + Hr, or Vf + Vr - gap_open when one vertical gap spans the
// cut (its opening would be counted twice). The two halves are then solved
// alone. A vertical gap that continues across a cut opens at no cost at the
// corner of the half it enters or leaves: each block carries the opening cost
// of a vertical gap at its top-left corner (tb) and at its bottom-right corner
// (te), gap_open or 0. Blocks of at most 256 rows are solved directly: the
// wavefront of the alignment kernels with 4 direction bits per cell, kept for
// one block in a per-warp buffer of (columns + 32) x 32 words, and walked back.
//
// One warp aligns one pair (taken from an atomic queue); lane t holds rows
// [8t, 8t + 8) of a 256-row strip. The shorter sequence is taken as the rows.
// Per warp: the four middle-row vectors and a strip boundary row (6 x (L + 2)
// int32) and the direction buffer (128 (L + 32) bytes), L the longest sequence.
#include <algorithm>
#include <cstring>
#include <vector>

#include "sad_internal.cuh"

namespace sad {

namespace {

constexpr int kLR = 8;                  // rows per lane
constexpr int kLG = 32;                 // lanes per pair (one warp)
constexpr int kLStrip = kLR * kLG;      // rows per strip, and the largest base block
constexpr int kLWarps = 4;              // warps per CTA
constexpr int kLStack = 48;             // pending blocks per warp
constexpr int32_t kLNeg = -(1 << 30);

struct LinArgs {
    const uint8_t* res;
    const int64_t* pad_off;
    const int32_t* len;
    const int32_t* pairs;   // (x, y) sequence ids, 2 per pair
    int32_t npairs;
    int32_t* head;          // next pair to take
    const int8_t* subst;
    int32_t alphabet, go, ge;
    int32_t* scores;
    const int64_t* ops_off;
    uint8_t* ops;
    int32_t* ops_len;
    int32_t* vec;           // per warp: Hf, Vf, Hr, Vr, boundary H/F: 6 vlen int32
    uint32_t* dirs;         // per warp: (vlen + 32) x 32 direction words
    int32_t vlen;           // longest sequence + 2
    uint32_t* status;
};

// A pending block: rows (i0, i1], columns (j0, j1], corner opening costs tb, te;
// kind 1 is the two X columns of a vertical gap that spans a cut.
struct Block {
    int32_t i0, i1, j0, j1, tb, te, kind;
};

// Rows and columns of a pass: element t (0-based) of the row sequence is
// x[xs + dx t], of the column sequence y[ys + dy t].
struct Seq2 {
    const uint8_t* x;
    int32_t xs, dx, m;
    const uint8_t* y;
    int32_t ys, dy, n;
};

// One DP pass (no directions) over q.m rows and q.n columns: H(0,0) = 0,
// H(0,j) = go + j ge, V(0,j) = -inf, H(i,0) = V(i,0) = t_open + i ge. Writes the
// last row's H and V for columns 0..n to outH, outV (q.m >= 1).
__device__ void lin_pass(const Seq2& q, const int8_t* __restrict__ sub, int32_t A, int32_t go, int32_t ge,
                         int32_t t_open, int32_t* __restrict__ bnd, int32_t* __restrict__ outH,
                         int32_t* __restrict__ outV, int lane) {
    const int32_t m = q.m, n = q.n;
    const int32_t goe = go + ge;
    const int32_t strips = (m + kLStrip - 1) / kLStrip;
    const int32_t nsteps = n + kLG - 1;
    const int32_t last = m - 1;  // 0-based last row
    const int owner = (last % kLStrip) / kLR, rsel = last % kLR;
    if (lane == 0) {
        outH[0] = t_open + m * ge;
        outV[0] = t_open + m * ge;
    }
    for (int32_t s = 0; s < strips; s++) {
        const int32_t row0 = s * kLStrip + lane * kLR;
        int32_t H[kLR], Hg[kLR], E[kLR];
        uint32_t xr[kLR];
#pragma unroll
        for (int r = 0; r < kLR; r++) {
            H[r] = t_open + (row0 + r + 1) * ge;
            Hg[r] = H[r] + goe;
            E[r] = kLNeg;
            xr[r] = row0 + r < m ? (uint32_t)q.x[q.xs + q.dx * (row0 + r)] * A : 0u;
        }
        int32_t hdiag = row0 == 0 ? 0 : t_open + row0 * ge;
        int32_t hin = 0, fin = kLNeg;
        uint32_t yin = 0;
        const bool last_strip = s == strips - 1;
        for (int32_t tau = 0; tau < nsteps; tau++) {
            if (lane == 0 && tau < n) {
                yin = q.y[q.ys + q.dy * tau];
                if (s == 0) {
                    hin = go + (tau + 1) * ge;
                    fin = kLNeg;
                } else {
                    hin = bnd[2 * (tau + 1)];
                    fin = bnd[2 * (tau + 1) + 1];
                }
            }
            const int32_t j = tau - lane + 1;
            int32_t hout = hin, fout = fin;
            if (j >= 1 && j <= n) {
                int32_t fu = fin, hgu = hin + goe, hd = hdiag;
                int32_t vh = 0, vf = 0;
#pragma unroll
                for (int r = 0; r < kLR; r++) {
                    const int32_t e = max(E[r] + ge, Hg[r]);
                    const int32_t f = max(fu + ge, hgu);
                    const int32_t h = max(hd + sub[xr[r] + yin], max(e, f));
                    hd = H[r];
                    H[r] = h;
                    Hg[r] = h + goe;
                    E[r] = e;
                    fu = f;
                    hgu = Hg[r];
                    if (r == rsel) {
                        vh = h;
                        vf = f;
                    }
                }
                hdiag = hin;
                hout = H[kLR - 1];
                fout = fu;
                if (!last_strip && lane == kLG - 1) {
                    bnd[2 * j] = hout;
                    bnd[2 * j + 1] = fout;
                }
                if (last_strip && lane == owner) {
                    outH[j] = vh;
                    outV[j] = vf;
                }
            }
            hin = __shfl_up_sync(0xffffffffu, hout, 1);
            fin = __shfl_up_sync(0xffffffffu, fout, 1);
            yin = __shfl_up_sync(0xffffffffu, yin, 1);
        }
        __syncwarp();
    }
}

// A block of at most 256 rows (q.m >= 1, q.n >= 1) solved directly: the DP
// with 4 direction bits per cell (bits 0-1 H source: 0 diagonal, 1 E, 2 V; bit
// 2 E extends; bit 3 V extends), the end state chosen by max(H, V - go + te),
// and the walk back. The columns go backwards into out[.. end), with x-codes cx
// (a row residue against a gap) and cy; returns the number of columns (lane 0's
// value) and the block's value in *value.
__device__ int32_t lin_base(const Seq2& q, const int8_t* __restrict__ sub, int32_t A, int32_t go, int32_t ge,
                            int32_t tb, int32_t te, uint32_t* __restrict__ dirs, uint8_t* __restrict__ out,
                            int64_t end, uint8_t cx, uint8_t cy, int lane, int32_t* value) {
    const int32_t m = q.m, n = q.n;
    const int32_t goe = go + ge;
    const int32_t nsteps = n + kLG - 1;
    const int32_t last = m - 1;
    const int owner = last / kLR, rsel = last % kLR;
    const int32_t row0 = lane * kLR;
    int32_t H[kLR], Hg[kLR], E[kLR];
    uint32_t xr[kLR];
#pragma unroll
    for (int r = 0; r < kLR; r++) {
        H[r] = tb + (row0 + r + 1) * ge;
        Hg[r] = H[r] + goe;
        E[r] = kLNeg;
        xr[r] = row0 + r < m ? (uint32_t)q.x[q.xs + q.dx * (row0 + r)] * A : 0u;
    }
    int32_t hdiag = row0 == 0 ? 0 : tb + row0 * ge;
    int32_t hin = 0, fin = kLNeg;
    uint32_t yin = 0;
    int32_t endH = 0, endV = 0;
    for (int32_t tau = 0; tau < nsteps; tau++) {
        if (lane == 0 && tau < n) {
            yin = q.y[q.ys + q.dy * tau];
            hin = go + (tau + 1) * ge;
            fin = kLNeg;
        }
        const int32_t j = tau - lane + 1;
        int32_t hout = hin, fout = fin;
        if (j >= 1 && j <= n) {
            int32_t fu = fin, hgu = hin + goe, hd = hdiag;
            uint32_t bits = 0;
            int32_t vh = 0, vf = 0;
#pragma unroll
            for (int r = 0; r < kLR; r++) {
                const int32_t ex = E[r] + ge, eo = Hg[r];
                const int32_t e = max(ex, eo);
                const int32_t fx = fu + ge, fo = hgu;
                const int32_t f = max(fx, fo);
                const int32_t dg = hd + sub[xr[r] + yin];
                const int32_t h = max(dg, max(e, f));
                const uint32_t src = dg >= max(e, f) ? 0u : (e >= f ? 1u : 2u);
                bits |= (src | ((ex >= eo) ? 4u : 0u) | ((fx >= fo) ? 8u : 0u)) << (4 * r);
                hd = H[r];
                H[r] = h;
                Hg[r] = h + goe;
                E[r] = e;
                fu = f;
                hgu = Hg[r];
                if (r == rsel) {
                    vh = h;
                    vf = f;
                }
            }
            dirs[(int64_t)tau * kLG + lane] = bits;
            hdiag = hin;
            hout = H[kLR - 1];
            fout = fu;
            if (lane == owner && j == n) {
                endH = vh;
                endV = vf;
            }
        }
        hin = __shfl_up_sync(0xffffffffu, hout, 1);
        fin = __shfl_up_sync(0xffffffffu, fout, 1);
        yin = __shfl_up_sync(0xffffffffu, yin, 1);
    }
    endH = __shfl_sync(0xffffffffu, endH, owner);
    endV = __shfl_sync(0xffffffffu, endV, owner);
    __syncwarp();  // the direction words are written
    // the end corner: a vertical gap that ends there pays te instead of go
    const int64_t vend = (int64_t)endV - go + te;
    const bool start_v = vend > (int64_t)endH;
    *value = start_v ? (int32_t)vend : endH;
    int32_t L = 0;
    if (lane == 0) {
        int32_t i = m, j = n, state = start_v ? 2 : 0;  // 0: H, 1: E (gap in x), 2: V (gap in y)
        while (i > 0 && j > 0) {
            const int32_t t = (i - 1) / kLR;
            const uint32_t word = dirs[(int64_t)(j - 1 + t) * kLG + t];
            const uint32_t b = (word >> (4 * ((i - 1) % kLR))) & 0xfu;
            if (state == 0) {
                const uint32_t src = b & 3u;
                if (src == 0) {
                    out[end - 1 - L++] = 'M';
                    i--;
                    j--;
                } else {
                    state = (int)src;
                }
            } else if (state == 1) {
                out[end - 1 - L++] = cy;
                state = (b & 4u) ? 1 : 0;
                j--;
            } else {
                out[end - 1 - L++] = cx;
                state = (b & 8u) ? 2 : 0;
                i--;
            }
        }
        while (i > 0) {
            out[end - 1 - L++] = cx;
            i--;
        }
        while (j > 0) {
            out[end - 1 - L++] = cy;
            j--;
        }
    }
    L = __shfl_sync(0xffffffffu, L, 0);
    __syncwarp();
    return L;
}

__global__ void __launch_bounds__(kLG * kLWarps) k_align_linear(LinArgs a) {
    __shared__ int8_t sub[SAD_MAX_ALPHABET * SAD_MAX_ALPHABET];
    __shared__ Block stack_sh[kLWarps][kLStack];
    for (int t = threadIdx.x; t < a.alphabet * a.alphabet; t += blockDim.x) sub[t] = a.subst[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t slot = (int64_t)blockIdx.x * kLWarps + wid;
    int32_t* vec = a.vec + slot * 6 * (int64_t)a.vlen;
    int32_t *Hf = vec, *Vf = vec + a.vlen, *Hr = vec + 2 * a.vlen, *Vr = vec + 3 * a.vlen, *bnd = vec + 4 * a.vlen;
    uint32_t* dirs = a.dirs + slot * (int64_t)(a.vlen + kLG) * kLG;
    Block* stk = stack_sh[wid];
    const int32_t go = a.go, ge = a.ge, A = a.alphabet;
    for (;;) {
        int32_t pk = 0;
        if (lane == 0) pk = atomicAdd(a.head, 1);
        pk = __shfl_sync(0xffffffffu, pk, 0);
        if (pk >= a.npairs) break;
        const int32_t xs = a.pairs[2 * pk], ys = a.pairs[2 * pk + 1];
        const int32_t mx = a.len[xs], ny = a.len[ys];
        uint8_t* out = a.ops + a.ops_off[pk];
        const int64_t cap = (int64_t)mx + ny;
        // rows: the shorter sequence; columns written for (x, y) as given
        const bool swap = mx > ny;
        Seq2 q;
        q.x = a.res + a.pad_off[swap ? ys : xs];
        q.y = a.res + a.pad_off[swap ? xs : ys];
        const int32_t m = swap ? ny : mx, n = swap ? mx : ny;
        const uint8_t cx = swap ? 'Y' : 'X', cy = swap ? 'X' : 'Y';
        int64_t cursor = 0;
        int32_t score = 0;
        bool first = true;
        int sp = 0;
        bool overflow = false;
        if (lane == 0) stk[0] = Block{0, m, 0, n, go, go, 0};
        sp = 1;
        __syncwarp();
        while (sp > 0) {
            const Block b = stk[sp - 1];
            __syncwarp();
            sp--;
            const int32_t M = b.i1 - b.i0, N = b.j1 - b.j0;
            if (b.kind == 1) {  // the two rows of a vertical gap that spans a cut
                if (lane == 0) {
                    out[cursor] = cx;
                    out[cursor + 1] = cx;
                }
                cursor += 2;
            } else if (M == 0 || N == 0) {
                // one gap run (or nothing)
                const uint8_t c = M == 0 ? cy : cx;
                for (int32_t t = lane; t < M + N; t += 32) out[cursor + t] = c;
                if (first) score = (M + N == 0) ? 0 : go + (M + N) * ge;
                cursor += M + N;
            } else if (M <= kLStrip) {
                q.xs = b.i0;
                q.dx = 1;
                q.m = M;
                q.ys = b.j0;
                q.dy = 1;
                q.n = N;
                int32_t val = 0;
                const int32_t L = lin_base(q, sub, A, go, ge, b.tb, b.te, dirs, out, cap, cx, cy, lane, &val);
                if (first) score = val;
                // move the L columns from the end of the slot to the cursor; chunks go
                // front to back and the source lies behind the destination
                const int64_t src0 = cap - L;
                if (src0 > cursor) {
                    for (int32_t c0 = 0; c0 < L; c0 += 32) {
                        const int32_t c = c0 + lane;
                        const uint8_t v = c < L ? out[src0 + c] : 0;
                        __syncwarp();
                        if (c < L) out[cursor + c] = v;
                        __syncwarp();
                    }
                }
                cursor += L;
            } else {
                const int32_t mid = b.i0 + M / 2;
                // forward over rows (i0, mid], reverse over rows (mid, i1]
                q.xs = b.i0;
                q.dx = 1;
                q.m = mid - b.i0;
                q.ys = b.j0;
                q.dy = 1;
                q.n = N;
                lin_pass(q, sub, A, go, ge, b.tb, bnd, Hf, Vf, lane);
                q.xs = b.i1 - 1;
                q.dx = -1;
                q.m = b.i1 - mid;
                q.ys = b.j1 - 1;
                q.dy = -1;
                lin_pass(q, sub, A, go, ge, b.te, bnd, Hr, Vr, lane);
                __syncwarp();
                // the crossing: the best (value, type, column), ties to type 1 and the smallest column
                long long best = LLONG_MIN;
                int32_t bj = 0, bt = 1;
                for (int32_t j = lane; j <= N; j += 32) {
                    const long long c1 = (long long)Hf[j] + Hr[N - j];
                    const long long c2 = (long long)Vf[j] + Vr[N - j] - go;
                    if (c1 > best) {
                        best = c1;
                        bj = j;
                        bt = 1;
                    }
                    if (c2 > best) {
                        best = c2;
                        bj = j;
                        bt = 2;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int32_t oj = __shfl_xor_sync(0xffffffffu, bj, o);
                    const int32_t ot = __shfl_xor_sync(0xffffffffu, bt, o);
                    if (ob > best || (ob == best && (ot < bt || (ot == bt && oj < bj)))) {
                        best = ob;
                        bj = oj;
                        bt = ot;
                    }
                }
                if (first) score = (int32_t)best;
                if (sp + 3 > kLStack) {
                    overflow = true;
                    break;
                }
                if (lane == 0) {
                    if (bt == 1) {
                        stk[sp] = Block{mid, b.i1, b.j0 + bj, b.j1, go, b.te, 0};
                        stk[sp + 1] = Block{b.i0, mid, b.j0, b.j0 + bj, b.tb, go, 0};
                    } else {
                        stk[sp] = Block{mid + 1, b.i1, b.j0 + bj, b.j1, 0, b.te, 0};
                        stk[sp + 1] = Block{0, 0, 0, 0, 0, 0, 1};
                        stk[sp + 2] = Block{b.i0, mid - 1, b.j0, b.j0 + bj, b.tb, 0, 0};
                    }
                }
                sp += bt == 1 ? 2 : 3;
                __syncwarp();
            }
            first = false;
        }
        if (lane == 0) {
            if (overflow) atomicOr(a.status, STATUS_CAPACITY);
            a.scores[pk] = score;
            a.ops_len[pk] = (int32_t)cursor;
        }
        __syncwarp();
    }
}

}  // namespace

}  // namespace sad

extern "C" int sad_align_pairs_linear(sad_ctx* ctx_in, const sad_seqset* seqs, const int32_t* pairs,
                                      int32_t npairs, const int8_t* subst, int32_t gap_open, int32_t gap_extend,
                                      int32_t* scores, int64_t* ops_offsets, uint8_t* ops, int64_t ops_capacity,
                                      int32_t* ops_len, int32_t mem, void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mem == SAD_MEM_HOST || mem == SAD_MEM_DEVICE, SAD_EINVAL, "mem = %d", mem);
    SAD_CHECK(seqs && subst && ops_offsets, SAD_EINVAL, "a required pointer is NULL");
    SAD_CHECK(npairs >= 0, SAD_EINVAL, "npairs = %d < 0", npairs);
    SAD_CHECK(npairs == 0 || (pairs && scores && ops && ops_len), SAD_EINVAL, "a required pointer is NULL");
    SAD_CHECK(gap_open <= 0 && gap_extend <= 0, SAD_EINVAL, "gap costs must be <= 0");
    SAD_CHECK(gap_open >= -1000 && gap_extend >= -1000, SAD_EINVAL, "gap costs below -1000");
    const int32_t A = seqs->alphabet;
    SAD_CHECK(A >= 1 && A <= SAD_MAX_ALPHABET, SAD_EINVAL, "alphabet %d outside 1..%d", A, SAD_MAX_ALPHABET);
    for (int32_t u = 0; u < A; u++)
        for (int32_t v = 0; v < A; v++)
            SAD_CHECK(subst[u * A + v] == subst[v * A + u], SAD_EINVAL,
                      "substitution matrix is not symmetric at (%d, %d)", u, v);
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    SAD_RET(status_clear(ctx, stream));
    DevSeqs S;
    SAD_RET(prepare_seqs(ctx, seqs, mem, stream, &S));
    std::vector<int32_t> hp((size_t)2 * npairs);
    if (npairs > 0) {
        if (mem == SAD_MEM_HOST) {
            memcpy(hp.data(), pairs, 8ull * npairs);
        } else {
            SAD_CUDA(cudaMemcpyAsync(hp.data(), pairs, 8ull * npairs, cudaMemcpyDeviceToHost, stream));
            SAD_CUDA(cudaStreamSynchronize(stream));
        }
    }
    std::vector<int64_t> hoff((size_t)npairs + 1, 0);
    int32_t max_len = 0;
    for (int32_t k = 0; k < npairs; k++) {
        const int32_t x = hp[2 * k], y = hp[2 * k + 1];
        SAD_CHECK(x >= 0 && x < S.n && y >= 0 && y < S.n, SAD_EINVAL, "pair %d = (%d, %d) outside 0..%d", k, x, y,
                  S.n - 1);
        hoff[k + 1] = hoff[k] + S.h_len[x] + S.h_len[y];
        max_len = std::max({max_len, S.h_len[x], S.h_len[y]});
    }
    const int64_t total = hoff[npairs];
    if (mem == SAD_MEM_HOST) {
        memcpy(ops_offsets, hoff.data(), 8ull * (npairs + 1));
    } else {
        SAD_CUDA(cudaMemcpyAsync(ops_offsets, hoff.data(), 8ull * (npairs + 1), cudaMemcpyHostToDevice, stream));
    }
    SAD_CHECK(total <= ops_capacity, SAD_ERANGE, "the alignments need %lld column bytes, capacity is %lld",
              (long long)total, (long long)ops_capacity);
    if (npairs == 0) {
        SAD_CUDA(cudaStreamSynchronize(stream));
        return SAD_OK;
    }
    int32_t smax = 0;
    for (int32_t t = 0; t < A * A; t++) smax = std::max(smax, (int32_t)std::abs((int)subst[t]));
    // a crossing sum adds two values of a pass: each stays inside +-2^28
    SAD_CHECK(((int64_t)smax - gap_open - gap_extend) * 2 * ((int64_t)max_len + 1) < (1ll << 28), SAD_EINVAL,
              "scores could exceed the 32-bit DP range");
    const int32_t vlen = max_len + 2;
    // persistent warps: about 16 per SM, fewer for few pairs
    const int64_t nwarps = std::min<int64_t>((int64_t)ctx->num_sms * 16, (int64_t)npairs);
    const int64_t grid = (nwarps + kLWarps - 1) / kLWarps;
    const int64_t slots = grid * kLWarps;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_pairs = carve(8ull * npairs), o_off = carve(8ull * (npairs + 1)), o_sub = carve(1024),
                 o_head = carve(16), o_sc = carve(4ull * npairs), o_len = carve(4ull * npairs),
                 o_vec = carve(4ull * 6 * vlen * slots), o_dirs = carve(4ull * (vlen + kLG) * kLG * slots),
                 o_ops = carve(mem == SAD_MEM_HOST ? (size_t)std::max<int64_t>(total, 1) : 0);
    void* w = nullptr;
    SAD_RET(workspace(ctx, WS_TRACE_DIRS, off, stream, &w));
    char* c = (char*)w;
    const cudaMemcpyKind k2 = mem == SAD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    LinArgs la;
    la.res = S.res;
    la.pad_off = S.pad_off;
    la.len = S.len;
    la.pairs = (const int32_t*)(c + o_pairs);
    la.npairs = npairs;
    la.head = (int32_t*)(c + o_head);
    la.subst = (const int8_t*)(c + o_sub);
    la.alphabet = A;
    la.go = gap_open;
    la.ge = gap_extend;
    la.scores = mem == SAD_MEM_HOST ? (int32_t*)(c + o_sc) : scores;
    la.ops_off = (const int64_t*)(c + o_off);
    la.ops = mem == SAD_MEM_HOST ? (uint8_t*)(c + o_ops) : ops;
    la.ops_len = mem == SAD_MEM_HOST ? (int32_t*)(c + o_len) : ops_len;
    la.vec = (int32_t*)(c + o_vec);
    la.dirs = (uint32_t*)(c + o_dirs);
    la.vlen = vlen;
    la.status = ctx->d_status;
    SAD_CUDA(cudaMemcpyAsync((void*)la.pairs, pairs, 8ull * npairs, k2, stream));
    SAD_CUDA(cudaMemcpyAsync((void*)la.ops_off, hoff.data(), 8ull * (npairs + 1), cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync((void*)la.subst, subst, (size_t)A * A, cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemsetAsync(la.head, 0, sizeof(int32_t), stream));
    {
        TraceScope ts(ctx, SAD_STAGE_ALIGN, stream);
        k_align_linear<<<(unsigned)grid, kLG * kLWarps, 0, stream>>>(la);
        SAD_LAUNCHED();
    }
    if (mem == SAD_MEM_HOST) {
        SAD_CUDA(cudaMemcpyAsync(scores, la.scores, 4ull * npairs, cudaMemcpyDeviceToHost, stream));
        SAD_CUDA(cudaMemcpyAsync(ops_len, la.ops_len, 4ull * npairs, cudaMemcpyDeviceToHost, stream));
        if (total > 0) SAD_CUDA(cudaMemcpyAsync(ops, la.ops, (size_t)total, cudaMemcpyDeviceToHost, stream));
    }
    SAD_RET(status_check(ctx, stream));
    return SAD_OK;
}

extern "C" int64_t sad_align_linear_bytes_per_warp(int32_t max_len) {
    using namespace sad;
    if (max_len < 0) return -1;
    const int64_t vlen = (int64_t)max_len + 2;
    return 4 * 6 * vlen + 4 * (vlen + kLG) * kLG;
}
