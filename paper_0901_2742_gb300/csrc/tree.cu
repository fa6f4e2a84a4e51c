// Per-bucket guide trees: the first step of the progressive multiple aligner
// that each processor runs on its bucket (Section 2.3.3 lets it be any
// sequential aligner; progressive aligners build an average-linkage tree from
// the pair scores, then align along it).
//
// Definition (exact integers): inside a bucket of nb members with pair scores
// S (the upper triangle of sad_bucket_pair_scores), the distance of members u
// and v is d_uv = S_uu + S_vv - 2 S_uv. Clusters start as the members (ids
// 0..nb-1); the distance of two clusters is W / (|A| |B|) with W the sum of d
// over their member pairs; the closest pair is merged first (exact rational
// comparison by 128-bit cross-multiplication), ties to the smallest (lower id,
// higher id); merge k creates cluster nb + k, whose W to any cluster C is
// W(A, C) + W(B, C).
//
// GPU mapping: one CTA per bucket (grid-stride over buckets). The pair sums W
// of the live clusters (an nb x nb matrix; a cluster lives in the slot of the
// lower of its two children), the cluster id and the size of every slot sit in
// shared memory when the largest bucket fits, else in a workspace. W is stored
// in 32 bits, with 64-bit cross-products, when the host proves every pair sum
// and product fits (else 64 bits and 128-bit products). A merge is a CTA-wide
// exact argmin over the live pairs (warps take rows, lanes columns; warp
// shuffles, then every warp reduces the per-warp results itself), then the
// merged rows are added into the lower slot: two CTA barriers per merge.
#include <cstring>
#include <vector>

#include "sad_internal.cuh"

namespace sad {

namespace {

// (measured: 128 / 256 / 512 / 1024 threads give 2.05 / 1.30 / 0.97 / 0.88 ms for
// the N = 2000 layout; the scans dominate, not the barriers)
constexpr int kTreeThreads = 1024;

// A candidate merge: pair sum, size product, cluster ids (lo < hi), slots.
struct Cand {
    long long num;
    long long den;
    int32_t lo, hi;
    int32_t si, sj;
};

// a is closer than b: a.num / a.den < b.num / b.den, ties to the smaller (lo, hi)
template <bool kNarrow>
__device__ __forceinline__ bool closer(const Cand& a, const Cand& b) {
    if (b.lo < 0) return a.lo >= 0;
    if (a.lo < 0) return false;
    bool lt, eq;
    if constexpr (kNarrow) {  // |num| < 2^31, den < 2^31: the products fit 63 bits
        const long long x = a.num * b.den, y = b.num * a.den;
        lt = x < y;
        eq = x == y;
    } else {
        const __int128 x = (__int128)a.num * b.den, y = (__int128)b.num * a.den;
        lt = x < y;
        eq = x == y;
    }
    if (!eq) return lt;
    return a.lo != b.lo ? a.lo < b.lo : a.hi < b.hi;
}

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int src) {
    Cand r;
    r.num = __shfl_sync(0xffffffffu, c.num, src);
    r.den = __shfl_sync(0xffffffffu, c.den, src);
    r.lo = __shfl_sync(0xffffffffu, c.lo, src);
    r.hi = __shfl_sync(0xffffffffu, c.hi, src);
    r.si = __shfl_sync(0xffffffffu, c.si, src);
    r.sj = __shfl_sync(0xffffffffu, c.sj, src);
    return r;
}

template <bool kNarrow>
__device__ __forceinline__ Cand warp_min(Cand c, int lane) {
    for (int o = 16; o > 0; o >>= 1) {
        const Cand y = shfl_cand(c, (lane + o) & 31);
        if (closer<kNarrow>(y, c)) c = y;
    }
    return c;
}

// WT: int32_t (kNarrow) or long long. Shared memory (when used): W (nbmax^2 WT),
// cid and sz (nbmax int32 each).
template <typename WT, bool kNarrow>
__global__ void __launch_bounds__(kTreeThreads)
k_guide_trees(int32_t p, int32_t nbmax, bool in_smem, const int32_t* __restrict__ bucket_off,
              const int64_t* __restrict__ score_off, const int32_t* __restrict__ scores,
              const int64_t* __restrict__ w_off, WT* __restrict__ Wall, int32_t* __restrict__ cid_all,
              int32_t* __restrict__ sz_all, const int64_t* __restrict__ merge_off, int32_t* __restrict__ left,
              int32_t* __restrict__ right, long long* __restrict__ num, long long* __restrict__ den) {
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ Cand red[kTreeThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int32_t b = blockIdx.x; b < p; b += gridDim.x) {
        const int32_t nb = bucket_off[b + 1] - bucket_off[b];
        if (nb < 2) continue;
        const int32_t* sc = scores + score_off[b];
        WT* W;
        int32_t *cid, *sz;  // cluster id per slot (-1 once merged away), cluster size
        if (in_smem) {
            W = (WT*)tsm;
            cid = (int32_t*)(tsm + sizeof(WT) * (size_t)nbmax * nbmax);
            sz = cid + nbmax;
        } else {
            W = Wall + w_off[b];
            cid = cid_all + bucket_off[b];
            sz = sz_all + bucket_off[b];
        }
        auto S = [&](int64_t u, int64_t v) {  // u <= v
            return (long long)sc[u * nb - u * (u - 1) / 2 + (v - u)];
        };
        for (int64_t t = threadIdx.x; t < (int64_t)nb * nb; t += blockDim.x) {
            const int64_t u = t / nb, v = t - u * nb;
            W[t] = (WT)(u == v ? 0 : S(u, u) + S(v, v) - 2 * S(min(u, v), max(u, v)));
        }
        for (int32_t u = threadIdx.x; u < nb; u += blockDim.x) {
            cid[u] = u;
            sz[u] = 1;
        }
        __syncthreads();
        for (int32_t k = 0; k < nb - 1; k++) {
            // the closest live pair: warp w takes rows w, w + nw, ..., lanes the columns
            Cand c{0, 1, -1, -1, -1, -1};
            for (int32_t i = warp; i < nb; i += nw) {
                const int32_t ci = cid[i];
                if (ci < 0) continue;
                const long long si = sz[i];
                const WT* Wi = W + (int64_t)i * nb;
                for (int32_t j = i + 1 + lane; j < nb; j += 32) {
                    const int32_t cj = cid[j];
                    if (cj < 0) continue;
                    const Cand x{(long long)Wi[j], si * sz[j], min(ci, cj), max(ci, cj), i, j};
                    if (closer<kNarrow>(x, c)) c = x;
                }
            }
            c = warp_min<kNarrow>(c, lane);
            if (lane == 0) red[warp] = c;
            __syncthreads();
            // every warp reduces the per-warp results (no second barrier)
            c = lane < nw ? red[lane] : Cand{0, 1, -1, -1, -1, -1};
            c = warp_min<kNarrow>(c, lane);
            const int32_t sa = min(c.si, c.sj), sb = max(c.si, c.sj);
            if (threadIdx.x == 0) {
                const int64_t m = merge_off[b] + k;
                left[m] = c.lo;
                right[m] = c.hi;
                num[m] = c.num;
                den[m] = c.den;
                // the new cluster nb + k takes the lower slot; the other slot dies
                cid[sa] = nb + k;
                sz[sa] = sz[sa] + sz[sb];
                cid[sb] = -1;
            }
            for (int32_t x = threadIdx.x; x < nb; x += blockDim.x) {
                if (x == sa || x == sb || cid[x] < 0) continue;
                const WT v = W[(int64_t)sa * nb + x] + W[(int64_t)sb * nb + x];
                W[(int64_t)sa * nb + x] = v;
                W[(int64_t)x * nb + sa] = v;
            }
            __syncthreads();
        }
    }
}

// max |scores[t]| over t < n into *out (zeroed before).
__global__ void k_absmax(const int32_t* __restrict__ x, int64_t n, unsigned int* __restrict__ out) {
    unsigned int m = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = x[t];
        m = max(m, (unsigned int)(v < 0 ? -(int64_t)v : v));
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

}  // namespace

}  // namespace sad

extern "C" int sad_guide_trees(sad_ctx* ctx_in, const int32_t* bucket_offsets, int32_t p,
                               const int64_t* score_offsets, const int32_t* scores, int64_t* merge_offsets,
                               int32_t* left, int32_t* right, int64_t* num, int64_t* den, int32_t mem,
                               void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mem == SAD_MEM_HOST || mem == SAD_MEM_DEVICE, SAD_EINVAL, "mem = %d", mem);
    SAD_CHECK(p >= 1, SAD_EINVAL, "p = %d < 1", p);
    SAD_CHECK(bucket_offsets && score_offsets && merge_offsets, SAD_EINVAL, "a required pointer is NULL");
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    SAD_RET(status_clear(ctx, stream));
    // layout on the host: bucket sizes, merge and workspace offsets
    std::vector<int32_t> bo((size_t)p + 1);
    std::vector<int64_t> so((size_t)p + 1);
    SAD_RET(arg_to_host(bucket_offsets, 4ull * (p + 1), mem, stream, bo.data()));
    SAD_RET(arg_to_host(score_offsets, 8ull * (p + 1), mem, stream, so.data()));
    SAD_CHECK(bo[0] == 0 && so[0] == 0, SAD_EINVAL, "bucket_offsets and score_offsets must start at 0");
    std::vector<int64_t> mo((size_t)p + 1, 0), wo((size_t)p + 1, 0);
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = bo[b + 1] - bo[b];
        SAD_CHECK(nb >= 0, SAD_EINVAL, "bucket_offsets decreases at %d", b);
        SAD_CHECK(so[b + 1] - so[b] == nb * (nb + 1) / 2, SAD_EINVAL,
                  "score_offsets of bucket %d do not hold its %lld pairs u <= v", b, (long long)(nb * (nb + 1) / 2));
        SAD_CHECK(nb <= (1 << 20), SAD_EINVAL, "bucket %d has %lld members (at most 2^20)", b, (long long)nb);
        mo[b + 1] = mo[b] + (nb > 0 ? nb - 1 : 0);
        wo[b + 1] = wo[b] + (nb >= 2 ? nb * nb : 0);
    }
    const int32_t n = bo[p];
    const int64_t M = mo[p], pairs = so[p];
    SAD_CHECK(M == 0 || (left && right && num && den), SAD_EINVAL, "an output pointer is NULL");
    SAD_CHECK(pairs == 0 || scores, SAD_EINVAL, "scores is NULL");
    SAD_CHECK(wo[p] * 8 <= (int64_t)3 << 32, SAD_ENOMEM,
              "the buckets' cluster matrices need %lld bytes (at most 12 GiB)", (long long)(wo[p] * 8));
    // device buffers: tables, W, slots; host-mode inputs and outputs are staged
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_bo = carve(4ull * (p + 1)), o_so = carve(8ull * (p + 1)), o_mo = carve(8ull * (p + 1)),
                 o_wo = carve(8ull * (p + 1)), o_cid = carve(4ull * (n + 1)), o_sz = carve(4ull * (n + 1)),
                 o_sc = carve(mem == SAD_MEM_HOST ? 4ull * (pairs + 1) : 0),
                 o_out = carve(mem == SAD_MEM_HOST ? (4ull * 2 + 8ull * 2) * (M + 1) : 0), o_w = carve(8ull * (wo[p] + 1));
    void* wsp = nullptr;
    SAD_RET(workspace(ctx, WS_TREE, off, stream, &wsp));
    char* w = (char*)wsp;
    void* pin = nullptr;
    const size_t tables = o_cid;  // bucket, score, merge and W offsets
    SAD_RET(pinned(ctx, tables, stream, &pin));
    SAD_CUDA(cudaStreamSynchronize(stream));  // the pinned area may feed an earlier copy
    memcpy((char*)pin + o_bo, bo.data(), 4ull * (p + 1));
    memcpy((char*)pin + o_so, so.data(), 8ull * (p + 1));
    memcpy((char*)pin + o_mo, mo.data(), 8ull * (p + 1));
    memcpy((char*)pin + o_wo, wo.data(), 8ull * (p + 1));
    SAD_CUDA(cudaMemcpyAsync(w, pin, tables, cudaMemcpyHostToDevice, stream));
    const int32_t* d_sc = scores;
    if (mem == SAD_MEM_HOST && pairs > 0) {
        SAD_CUDA(cudaMemcpyAsync(w + o_sc, scores, 4ull * pairs, cudaMemcpyHostToDevice, stream));
        d_sc = (const int32_t*)(w + o_sc);
    }
    int32_t *d_left = left, *d_right = right;
    long long *d_num = (long long*)num, *d_den = (long long*)den;
    if (mem == SAD_MEM_HOST) {
        d_left = (int32_t*)(w + o_out);
        d_right = d_left + (M + 1);
        d_num = (long long*)(w + o_out + 8ull * (M + 1));
        d_den = d_num + (M + 1);
    }
    if (M > 0) {
        // 32-bit pair sums when they provably fit: |d| <= 4 max|S| and a pair sum adds at
        // most floor(nb / 2) ceil(nb / 2) of them; the size products stay below 2^31 too
        int64_t smax = 0;
        if (mem == SAD_MEM_HOST) {
            for (int64_t t = 0; t < pairs; t++) smax = std::max<int64_t>(smax, std::llabs((long long)scores[t]));
        } else {
            unsigned int* d_max = (unsigned int*)(w + o_cid);  // scratch: the slot arrays are written later
            SAD_CUDA(cudaMemsetAsync(d_max, 0, sizeof(unsigned int), stream));
            k_absmax<<<(int)std::min<int64_t>((pairs + 255) / 256, (int64_t)ctx->num_sms * 4), 256, 0, stream>>>(
                d_sc, pairs, d_max);
            SAD_LAUNCHED();
            unsigned int h = 0;
            SAD_CUDA(cudaMemcpyAsync(&h, d_max, sizeof(h), cudaMemcpyDeviceToHost, stream));
            SAD_CUDA(cudaStreamSynchronize(stream));
            smax = h;
        }
        int32_t nbmax = 0;
        for (int32_t b = 0; b < p; b++) nbmax = std::max(nbmax, bo[b + 1] - bo[b]);
        const int64_t half = (int64_t)(nbmax / 2) * ((nbmax + 1) / 2);
        const bool narrow = 4 * smax * half < (1ll << 31) && half < (1ll << 31);
        const size_t wbytes = (narrow ? 4 : 8) * (size_t)nbmax * nbmax;
        const size_t smem = wbytes + 8ull * nbmax;
        const bool in_smem = smem <= ctx->smem_optin - 4096;
        TraceScope ts(ctx, SAD_STAGE_TREE, stream);
        const int grid = std::min<int32_t>(p, ctx->num_sms);
        const size_t dyn = in_smem ? smem : 0;
        if (narrow) {
            SAD_RET(allow_max_dynamic_smem(ctx, (const void*)k_guide_trees<int32_t, true>));
            k_guide_trees<int32_t, true><<<grid, kTreeThreads, dyn, stream>>>(
                p, nbmax, in_smem, (const int32_t*)(w + o_bo), (const int64_t*)(w + o_so), d_sc,
                (const int64_t*)(w + o_wo), (int32_t*)(w + o_w), (int32_t*)(w + o_cid), (int32_t*)(w + o_sz),
                (const int64_t*)(w + o_mo), d_left, d_right, d_num, d_den);
        } else {
            SAD_RET(allow_max_dynamic_smem(ctx, (const void*)k_guide_trees<long long, false>));
            k_guide_trees<long long, false><<<grid, kTreeThreads, dyn, stream>>>(
                p, nbmax, in_smem, (const int32_t*)(w + o_bo), (const int64_t*)(w + o_so), d_sc,
                (const int64_t*)(w + o_wo), (long long*)(w + o_w), (int32_t*)(w + o_cid), (int32_t*)(w + o_sz),
                (const int64_t*)(w + o_mo), d_left, d_right, d_num, d_den);
        }
        SAD_LAUNCHED();
    }
    const cudaMemcpyKind k = mem == SAD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    SAD_CUDA(cudaMemcpyAsync(merge_offsets, w + o_mo, 8ull * (p + 1), k, stream));
    if (mem == SAD_MEM_HOST && M > 0) {
        SAD_CUDA(cudaMemcpyAsync(left, d_left, 4ull * M, k, stream));
        SAD_CUDA(cudaMemcpyAsync(right, d_right, 4ull * M, k, stream));
        SAD_CUDA(cudaMemcpyAsync(num, d_num, 8ull * M, k, stream));
        SAD_CUDA(cudaMemcpyAsync(den, d_den, 8ull * M, k, stream));
    }
    SAD_RET(status_check(ctx, stream));
    return SAD_OK;
}
