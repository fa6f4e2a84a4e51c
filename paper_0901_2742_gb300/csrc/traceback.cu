// Alignments, not only scores, of given pairs: the optimal global affine-gap
// alignment of each pair as a string of columns (the per-processor aligner of
// Section 2.3.3 turns the bucket's pair scores into alignments; the paper
// leaves the aligner open, and this is the pairwise step it builds on).
//
// One warp aligns one pair: lane t holds query rows [8t, 8t+8) of the current
// strip of 256 rows and sweeps the subject's columns as a diagonal wavefront
// (H and F of the lane's bottom row move one lane down per step, as in the
// score kernels). Every cell also records where its values came from, 4 bits:
//   bits 0-1  H source: 0 the diagonal (a match column), 1 E, 2 F
//   bit 2     E(i,j) extends E(i,j-1) (else it opens from H(i,j-1))
//   bit 3     F(i,j) extends F(i-1,j) (else it opens from H(i-1,j))
// so a lane step stores exactly one 32-bit word (8 rows x 4 bits), at index
// (strip, step, lane): the 32 lanes of a step write 128 consecutive bytes.
// Lane 0 then walks the bits back from (m, n), and the warp copies the columns
// out in forward order.
#include <algorithm>
#include <cstring>
#include <vector>

#include "sad_internal.cuh"

namespace sad {

namespace {

constexpr int kTrR = 8;          // rows per lane
constexpr int kTrG = 32;         // lanes per pair (one warp)
constexpr int kTrStrip = kTrR * kTrG;
constexpr int kTrWarps = 4;      // warps per CTA
constexpr int32_t kTrNeg = -(1 << 30);

struct TraceArgs {
    const uint8_t* res;
    const int64_t* pad_off;
    const int32_t* len;
    const int32_t* pairs;     // (x, y) sequence ids, 2 per pair
    int32_t pair0, npairs;    // this batch: pairs [pair0, pair0 + npairs)
    const int64_t* dir_off;   // word offset of each batch pair's direction words
    uint32_t* dirs;
    int32_t* bnd;             // per warp slot: H and F of a strip's bottom row
    int64_t bnd_stride;
    const int8_t* subst;
    int32_t alphabet, go, ge;
    int32_t* scores;
    const int64_t* ops_off;
    uint8_t* ops;
    int32_t* ops_len;
};

__device__ __forceinline__ int64_t dir_index(int64_t base, int32_t n, int32_t i, int32_t j) {
    // cell (i, j), 1-based: strip, lane and step of the lane that computed it
    const int32_t s = (i - 1) / kTrStrip;
    const int32_t t = ((i - 1) % kTrStrip) / kTrR;
    const int64_t tau = (int64_t)(j - 1) + t;
    return base + ((int64_t)s * (n + kTrG - 1) + tau) * kTrG + t;
}

__global__ void __launch_bounds__(kTrG * kTrWarps)
k_gotoh_trace(TraceArgs a) {
    __shared__ int8_t sub[SAD_MAX_ALPHABET * SAD_MAX_ALPHABET];
    for (int t = threadIdx.x; t < a.alphabet * a.alphabet; t += blockDim.x) sub[t] = a.subst[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t slot = (int64_t)blockIdx.x * kTrWarps + (threadIdx.x >> 5);
    const int64_t nslots = (int64_t)gridDim.x * kTrWarps;
    int32_t* bnd = a.bnd + slot * a.bnd_stride;
    const int32_t go = a.go, ge = a.ge, goe = go + ge;
    for (int64_t k = slot; k < a.npairs; k += nslots) {
        const int64_t pk = a.pair0 + k;
        const int32_t xs = a.pairs[2 * pk], ys = a.pairs[2 * pk + 1];
        const int32_t m = a.len[xs], n = a.len[ys];
        const uint8_t* x = a.res + a.pad_off[xs];
        const uint8_t* y = a.res + a.pad_off[ys];
        uint8_t* out = a.ops + a.ops_off[pk];
        if (m == 0 || n == 0) {  // one gap run, or nothing
            for (int32_t c = lane; c < m + n; c += 32) out[c] = m == 0 ? 'Y' : 'X';
            if (lane == 0) {
                a.scores[pk] = (m + n == 0) ? 0 : go + (m + n) * ge;
                a.ops_len[pk] = m + n;
            }
            continue;
        }
        const int64_t dbase = a.dir_off[k];
        const int32_t strips = (m + kTrStrip - 1) / kTrStrip;
        const int32_t nsteps = n + kTrG - 1;
        int32_t score = 0;
        for (int32_t s = 0; s < strips; s++) {
            const int32_t row0 = s * kTrStrip + lane * kTrR;  // 0-based residue of my first row
            int32_t H[kTrR], Hg[kTrR], E[kTrR];
            uint32_t xr[kTrR];
#pragma unroll
            for (int r = 0; r < kTrR; r++) {
                H[r] = go + (row0 + r + 1) * ge;
                Hg[r] = H[r] + goe;
                E[r] = kTrNeg;
                xr[r] = row0 + r < m ? (uint32_t)x[row0 + r] * a.alphabet : 0u;
            }
            int32_t hdiag = row0 == 0 ? 0 : go + row0 * ge;  // H(row0, 0)
            int32_t hin = 0, fin = kTrNeg;
            uint32_t yin = 0;
            const bool last_strip = s == strips - 1;
            for (int32_t tau = 0; tau < nsteps; tau++) {
                if (lane == 0 && tau < n) {
                    yin = y[tau];
                    if (s == 0) {
                        hin = go + (tau + 1) * ge;
                        fin = kTrNeg;
                    } else {
                        hin = bnd[2 * (tau + 1)];
                        fin = bnd[2 * (tau + 1) + 1];
                    }
                }
                const int32_t j = tau - lane + 1;
                int32_t hout = hin, fout = fin;
                if (j >= 1 && j <= n) {
                    int32_t fu = fin, hgu = hin + goe, hd = hdiag;
                    uint32_t bits = 0;
#pragma unroll
                    for (int r = 0; r < kTrR; r++) {
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
                    }
                    a.dirs[dbase + ((int64_t)s * nsteps + tau) * kTrG + lane] = bits;
                    hdiag = hin;
                    hout = H[kTrR - 1];
                    fout = fu;
                    if (!last_strip && lane == kTrG - 1) {
                        bnd[2 * j] = hout;
                        bnd[2 * j + 1] = fout;
                    }
                }
                hin = __shfl_up_sync(0xffffffffu, hout, 1);
                fin = __shfl_up_sync(0xffffffffu, fout, 1);
                yin = __shfl_up_sync(0xffffffffu, yin, 1);
            }
            __syncwarp();
            if (last_strip) {
                const int32_t rr = (m - 1) - s * kTrStrip;
                int32_t v = 0;
#pragma unroll
                for (int r = 0; r < kTrR; r++) v = (r == rr % kTrR) ? H[r] : v;
                score = __shfl_sync(0xffffffffu, v, rr / kTrR);
            }
        }
        // traceback by lane 0: columns written backwards from the end of the slot
        const int32_t cap = m + n;
        int32_t L = 0;
        if (lane == 0) {
            int32_t i = m, j = n, state = 0;  // 0: H, 1: E (gap in x), 2: F (gap in y)
            int64_t widx = -1;
            uint32_t word = 0;
            while (i > 0 && j > 0) {
                const int64_t w = dir_index(dbase, n, i, j);
                if (w != widx) {
                    word = a.dirs[w];
                    widx = w;
                }
                const uint32_t b = (word >> (4 * ((i - 1) % kTrR))) & 0xfu;
                if (state == 0) {
                    const uint32_t src = b & 3u;
                    if (src == 0) {
                        out[cap - 1 - L++] = 'M';
                        i--;
                        j--;
                    } else {
                        state = (int)src;
                    }
                } else if (state == 1) {
                    out[cap - 1 - L++] = 'Y';
                    state = (b & 4u) ? 1 : 0;
                    j--;
                } else {
                    out[cap - 1 - L++] = 'X';
                    state = (b & 8u) ? 2 : 0;
                    i--;
                }
            }
            // the border: H(i, 0) and H(0, j) are single gap runs
            while (i > 0) {
                out[cap - 1 - L++] = 'X';
                i--;
            }
            while (j > 0) {
                out[cap - 1 - L++] = 'Y';
                j--;
            }
            a.scores[pk] = score;
            a.ops_len[pk] = L;
        }
        L = __shfl_sync(0xffffffffu, L, 0);
        __syncwarp();
        // move the L columns to the front of the slot, in order; chunks go
        // front to back and the source lies behind the destination
        const int32_t src0 = cap - L;
        if (src0 > 0) {
            for (int32_t c0 = 0; c0 < L; c0 += 32) {
                const int32_t c = c0 + lane;
                const uint8_t v = c < L ? out[src0 + c] : 0;
                __syncwarp();
                if (c < L) out[c] = v;
                __syncwarp();
            }
        }
    }
}

}  // namespace

}  // namespace sad

extern "C" int sad_align_pairs(sad_ctx* ctx_in, const sad_seqset* seqs, const int32_t* pairs, int32_t npairs,
                               const int8_t* subst, int32_t gap_open, int32_t gap_extend, int32_t* scores,
                               int64_t* ops_offsets, uint8_t* ops, int64_t ops_capacity, int32_t* ops_len,
                               int32_t mem, void* stream_ptr) {
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
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    SAD_RET(status_clear(ctx, stream));
    DevSeqs S;
    SAD_RET(prepare_seqs(ctx, seqs, mem, stream, &S));
    // the pairs on the host (layout) and on the device (kernel)
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
    for (int32_t k = 0; k < npairs; k++) {
        const int32_t x = hp[2 * k], y = hp[2 * k + 1];
        SAD_CHECK(x >= 0 && x < S.n && y >= 0 && y < S.n, SAD_EINVAL, "pair %d = (%d, %d) outside 0..%d", k, x, y,
                  S.n - 1);
        hoff[k + 1] = hoff[k] + S.h_len[x] + S.h_len[y];
    }
    const int64_t total = hoff[npairs];
    const cudaMemcpyKind k2 = mem == SAD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
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
    int32_t max_len = 0;
    for (int32_t i = 0; i < S.n; i++) max_len = std::max(max_len, S.h_len[i]);
    SAD_CHECK(((int64_t)smax - gap_open - gap_extend) * 2 * ((int64_t)max_len + 1) < (1ll << 29), SAD_EINVAL,
              "scores could exceed the 32-bit DP range");
    // device buffers: pairs, offsets, subst, per-pair outputs (staged in host mode)
    const int64_t nw = std::min<int64_t>((int64_t)ctx->num_sms * 8 * kTrWarps, (int64_t)npairs);
    const int64_t grid = (nw + kTrWarps - 1) / kTrWarps;
    const int64_t bnd_stride = 2 * ((int64_t)max_len + 1 + 4);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_pairs = carve(8ull * npairs), o_off = carve(8ull * (npairs + 1)), o_sub = carve(1024),
                 o_sc = carve(4ull * npairs), o_len = carve(4ull * npairs), o_doff = carve(8ull * (npairs + 1)),
                 o_bnd = carve(4ull * bnd_stride * grid * kTrWarps),
                 o_ops = carve(mem == SAD_MEM_HOST ? (size_t)std::max<int64_t>(total, 1) : 0);
    void* w = nullptr;
    SAD_RET(workspace(ctx, WS_TRACE, off, stream, &w));
    char* c = (char*)w;
    // batches whose direction words fit the budget
    const int64_t budget_words = (int64_t)1 << 28;  // 1 GiB of direction words at once
    std::vector<int64_t> dwords((size_t)npairs);
    int64_t max_words = 1, sum_words = 0;
    for (int32_t k = 0; k < npairs; k++) {
        const int64_t m = S.h_len[hp[2 * k]], n = S.h_len[hp[2 * k + 1]];
        dwords[k] = (m > 0 && n > 0) ? (int64_t)((m + kTrStrip - 1) / kTrStrip) * (n + kTrG - 1) * kTrG : 0;
        max_words = std::max(max_words, dwords[k]);
        sum_words += dwords[k];
    }
    void* dv = nullptr;
    SAD_RET(workspace(ctx, WS_TRACE_DIRS, 4ull * std::max(max_words, std::min(budget_words, sum_words)), stream,
                      &dv));
    int32_t* d_pairs = (int32_t*)(c + o_pairs);
    int64_t* d_off = (int64_t*)(c + o_off);
    int8_t* d_sub = (int8_t*)(c + o_sub);
    int32_t* d_sc = mem == SAD_MEM_HOST ? (int32_t*)(c + o_sc) : scores;
    int32_t* d_len = mem == SAD_MEM_HOST ? (int32_t*)(c + o_len) : ops_len;
    int64_t* d_doff = (int64_t*)(c + o_doff);
    uint8_t* d_ops = mem == SAD_MEM_HOST ? (uint8_t*)(c + o_ops) : ops;
    SAD_CUDA(cudaMemcpyAsync(d_pairs, pairs, 8ull * npairs, k2, stream));
    SAD_CUDA(cudaMemcpyAsync(d_off, hoff.data(), 8ull * (npairs + 1), cudaMemcpyHostToDevice, stream));
    SAD_CUDA(cudaMemcpyAsync(d_sub, subst, (size_t)A * A, cudaMemcpyHostToDevice, stream));
    std::vector<int64_t> hdoff((size_t)npairs + 1, 0);
    TraceArgs ta;
    ta.res = S.res;
    ta.pad_off = S.pad_off;
    ta.len = S.len;
    ta.pairs = d_pairs;
    ta.dirs = (uint32_t*)dv;
    ta.bnd = (int32_t*)(c + o_bnd);
    ta.bnd_stride = bnd_stride;
    ta.subst = d_sub;
    ta.alphabet = A;
    ta.go = gap_open;
    ta.ge = gap_extend;
    ta.scores = d_sc;
    ta.ops_off = d_off;
    ta.ops = d_ops;
    ta.ops_len = d_len;
    {
        TraceScope ts(ctx, SAD_STAGE_ALIGN, stream);
        for (int32_t k0 = 0; k0 < npairs;) {
            int64_t used = 0;
            int32_t k1 = k0;
            while (k1 < npairs && (k1 == k0 || used + dwords[k1] <= budget_words)) {
                hdoff[k1 - k0] = used;
                used += dwords[k1];
                k1++;
            }
            // the batch's direction offsets, ordered after the previous batch's kernel
            // (a copy from pageable memory has read hdoff when it returns)
            SAD_CUDA(cudaMemcpyAsync(d_doff, hdoff.data(), 8ull * (k1 - k0), cudaMemcpyHostToDevice, stream));
            ta.pair0 = k0;
            ta.npairs = k1 - k0;
            ta.dir_off = d_doff;
            const int64_t g = std::min<int64_t>(grid, ((int64_t)ta.npairs + kTrWarps - 1) / kTrWarps);
            k_gotoh_trace<<<(unsigned)g, kTrG * kTrWarps, 0, stream>>>(ta);
            SAD_LAUNCHED();
            k0 = k1;
        }
    }
    if (mem == SAD_MEM_HOST) {
        SAD_CUDA(cudaMemcpyAsync(scores, d_sc, 4ull * npairs, cudaMemcpyDeviceToHost, stream));
        SAD_CUDA(cudaMemcpyAsync(ops_len, d_len, 4ull * npairs, cudaMemcpyDeviceToHost, stream));
        if (total > 0) SAD_CUDA(cudaMemcpyAsync(ops, d_ops, (size_t)total, cudaMemcpyDeviceToHost, stream));
    }
    SAD_RET(status_check(ctx, stream));
    return SAD_OK;
}
