// Regular-sampling redistribution by k-mer rank (Section 2.3.2, the sample-sort
// steps of the algorithm box): sort each block by rank, take p-1 evenly spaced
// samples per block, sort the samples, pick p-1 pivots, bucket every sequence.
//
// A rank key (a_i, b_i, i) is packed into one 64-bit integer
//   K_i = floor(a_i 2^32 / b_i) << 31 | i.
// For b <= 2^16 two different fractions differ by at least 2^-32, so the
// fixed-point part orders them exactly and equal fractions tie; the index
// breaks ties. Every comparison below is then a plain 64-bit comparison.
// Integer rank keys G_i (the globalized rank sums, up to about 2^52) are packed
// as the 128-bit integer G_i << 32 | i; the kernels are templated on the key
// type and the two forms share every step.
#include <cuda.h>
#include <cstring>

#include "partition_stage.cuh"
#include "sad_internal.cuh"

namespace sad {

namespace {

constexpr uint32_t STATUS_BAD_KEY = 1u << 3;

using u128 = unsigned __int128;

// sequence index carried in the low bits of a packed key
__device__ __forceinline__ int32_t key_index(uint64_t v) { return (int32_t)(v & 0x7fffffffull); }
__device__ __forceinline__ int32_t key_index(u128 v) { return (int32_t)(uint32_t)v; }

__global__ void k_part_keys(int32_t n, const int32_t* __restrict__ ka, const int32_t* __restrict__ kb,
                            uint64_t* __restrict__ K, uint32_t* __restrict__ status) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = ka[i], b = kb[i];
    if (a < 0 || b < 1 || a > b || b > 65536) {
        atomicOr(status, STATUS_BAD_KEY);
        a = 0;
        b = 1;
    }
    const uint64_t fx = ((uint64_t)a << 32) / (uint64_t)b;
    K[i] = (fx << 31) | (uint64_t)i;
}

// G_i << 32 | i
__global__ void k_part_keys128(int32_t n, const uint64_t* __restrict__ G, u128* __restrict__ K) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    K[i] = ((u128)G[i] << 32) | (u128)(uint32_t)i;
}

// rank of every key inside its block: grid (p, chunks of 256 elements)
template <class KeyT>
__global__ void k_part_block_rank(int32_t n, int32_t p, const KeyT* __restrict__ K,
                                  int32_t* __restrict__ rank) {
    __shared__ KeyT tile[1024];
    const int32_t b = blockIdx.x;
    const int64_t lo = (int64_t)b * n / p, hi = (int64_t)(b + 1) * n / p;
    const int64_t i = lo + (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (lo + (int64_t)blockIdx.y * blockDim.x >= hi) return;  // whole CTA idle (uniform)
    const KeyT key = i < hi ? K[i] : (KeyT)0;
    int32_t r = 0;
    for (int64_t t0 = lo; t0 < hi; t0 += 1024) {
        const int64_t m = min((int64_t)1024, hi - t0);
        __syncthreads();
        for (int64_t t = threadIdx.x; t < m; t += blockDim.x) tile[t] = K[t0 + t];
        __syncthreads();
        for (int64_t t = 0; t < m; t++) r += tile[t] < key;
    }
    if (i < hi) rank[i] = r;
}

// samples: element of rank r in block b is sample j for every j in 1..p-1 with
// floor(j w / p) = r, i.e. j in [ceil(r p / w), ceil((r+1) p / w) - 1]
template <class KeyT>
__global__ void k_part_samples(int32_t n, int32_t p, const KeyT* __restrict__ K,
                               const int32_t* __restrict__ rank, KeyT* __restrict__ Y) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // block of i: largest b with floor(b n / p) <= i
    int64_t b = ((int64_t)i * p) / n;
    while (b + 1 < p && (b + 1) * n / p <= i) b++;
    while (b > 0 && b * n / p > i) b--;
    const int64_t lo = b * n / p, hi = (b + 1) * n / p, w = hi - lo;
    const int64_t r = rank[i];
    int64_t jlo = (r * p + w - 1) / w, jhi = ((r + 1) * p + w - 1) / w - 1;
    if (jlo < 1) jlo = 1;
    if (jhi > p - 1) jhi = p - 1;
    for (int64_t j = jlo; j <= jhi; j++) Y[b * (p - 1) + j - 1] = K[i];
}

// position of every sample in sorted order (equal samples keep their slot order)
template <class KeyT>
__global__ void k_part_sample_rank(int32_t M, const KeyT* __restrict__ Y,
                                   KeyT* __restrict__ Ysorted) {
    __shared__ KeyT tile[1024];
    const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    const KeyT key = s < M ? Y[s] : (KeyT)0;
    int32_t r = 0;
    for (int32_t t0 = 0; t0 < M; t0 += 1024) {
        const int32_t m = min(1024, M - t0);
        __syncthreads();
        for (int32_t t = threadIdx.x; t < m; t += blockDim.x) tile[t] = Y[t0 + t];
        __syncthreads();
        for (int32_t t = 0; t < m; t++) {
            const KeyT v = tile[t];
            r += (v < key) | ((v == key) & (t0 + t < s));
        }
    }
    if (s < M) Ysorted[r] = key;
}

// pivot m = sorted sample at 1-based (m-1) q + max(1, floor(q/2)), q = non-empty blocks
template <class KeyT>
__global__ void k_part_pivots(int32_t n, int32_t p, const KeyT* __restrict__ Ysorted,
                              KeyT* __restrict__ piv, int32_t* __restrict__ pivot_idx) {
    const int32_t m = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (m > p - 1) return;
    const int64_t q = n < p ? n : p;
    if (q == 0) {
        piv[m - 1] = ~(KeyT)0;
        if (pivot_idx) pivot_idx[m - 1] = -1;
        return;
    }
    const int64_t pos1 = (int64_t)(m - 1) * q + (q / 2 > 1 ? q / 2 : 1);
    const KeyT v = Ysorted[pos1 - 1];
    piv[m - 1] = v;
    if (pivot_idx) pivot_idx[m - 1] = key_index(v);
}

// bucket = number of pivots strictly below the key (pivots are sorted)
template <class KeyT>
__global__ void k_part_bucket(int32_t n, int32_t p, const KeyT* __restrict__ K,
                              const KeyT* __restrict__ piv, int32_t* __restrict__ bucket,
                              int32_t* __restrict__ count) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const KeyT key = K[i];
    int32_t lo = 0, hi = p - 1;  // first pivot >= key
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (piv[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    bucket[i] = lo;
    atomicAdd(&count[lo], 1);
}

__global__ void k_part_offsets(int32_t p, const int32_t* __restrict__ count,
                               int32_t* __restrict__ offsets) {
    if (threadIdx.x != 0) return;
    int32_t s = 0;
    offsets[0] = 0;
    for (int32_t b = 0; b < p; b++) {
        s += count[b];
        offsets[b + 1] = s;
    }
}

// one warp per bucket: its members in ascending index (ballot compaction)
__global__ void k_part_scatter(int32_t n, int32_t p, const int32_t* __restrict__ bucket,
                               const int32_t* __restrict__ offsets, int32_t* __restrict__ order) {
    const int32_t b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= p) return;
    const int lane = threadIdx.x & 31;
    int32_t pos = offsets[b];
    for (int32_t t0 = 0; t0 < n; t0 += 32) {
        const int32_t i = t0 + lane;
        const bool f = i < n && bucket[i] == b;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (f) order[pos + __popc(bal & ((1u << lane) - 1u))] = i;
        pos += __popc(bal);
    }
}

}  // namespace

namespace {

// The partition steps on packed keys of type KeyT; fill_keys(K) launches the
// kernel that writes the n keys.
template <class KeyT, class FillKeys>
int partition_run(sad_ctx* ctx, int32_t n, int32_t p, FillKeys fill_keys, int32_t* bucket_offsets,
                  int32_t* order, int32_t* pivot_idx, cudaStream_t stream) {
    const int64_t M = (int64_t)p * (p - 1);
    const size_t kb = sizeof(KeyT);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t oK = carve(kb * (n + 1)), oRank = carve(4ull * (n + 1)), oY = carve(kb * (M + 1)),
                 oYs = carve(kb * (M + 1)), oPiv = carve(kb * p), oBucket = carve(4ull * (n + 1)),
                 oCount = carve(4ull * p);
    void* ws = nullptr;
    SAD_RET(workspace(ctx, WS_PART, off, stream, &ws));
    char* w = (char*)ws;
    KeyT* K = (KeyT*)(w + oK);
    int32_t* rank = (int32_t*)(w + oRank);
    KeyT* Y = (KeyT*)(w + oY);
    KeyT* Ys = (KeyT*)(w + oYs);
    KeyT* piv = (KeyT*)(w + oPiv);
    int32_t* bucket = (int32_t*)(w + oBucket);
    int32_t* count = (int32_t*)(w + oCount);
    SAD_CUDA(cudaMemsetAsync(count, 0, 4ull * p, stream));
    if (n == 0) {
        SAD_CUDA(cudaMemsetAsync(bucket_offsets, 0, 4ull * (p + 1), stream));
        if (pivot_idx && p > 1) SAD_CUDA(cudaMemsetAsync(pivot_idx, 0xff, 4ull * (p - 1), stream));
        return SAD_OK;
    }
    const int nb = (n + 255) / 256;
    TraceScope ts(ctx, SAD_STAGE_PARTITION, stream);
    fill_keys(K);
    SAD_LAUNCHED();
    if (p > 1) {
        const int64_t wmax = (n + p - 1) / p + 1;
        dim3 g((unsigned)p, (unsigned)((wmax + 255) / 256));
        k_part_block_rank<<<g, 256, 0, stream>>>(n, p, (const KeyT*)K, rank);
        SAD_LAUNCHED();
        SAD_CUDA(cudaMemsetAsync(Y, 0xff, kb * M, stream));
        k_part_samples<<<nb, 256, 0, stream>>>(n, p, (const KeyT*)K, rank, Y);
        SAD_LAUNCHED();
        k_part_sample_rank<<<(unsigned)((M + 255) / 256), 256, 0, stream>>>((int32_t)M, (const KeyT*)Y, Ys);
        SAD_LAUNCHED();
        k_part_pivots<<<(p - 1 + 255) / 256, 256, 0, stream>>>(n, p, (const KeyT*)Ys, piv, pivot_idx);
        SAD_LAUNCHED();
    }
    k_part_bucket<<<nb, 256, 0, stream>>>(n, p, (const KeyT*)K, (const KeyT*)piv, bucket, count);
    SAD_LAUNCHED();
    k_part_offsets<<<1, 32, 0, stream>>>(p, count, bucket_offsets);
    SAD_LAUNCHED();
    k_part_scatter<<<(p + 7) / 8, 256, 0, stream>>>(n, p, bucket, bucket_offsets, order);
    SAD_LAUNCHED();
    return SAD_OK;
}

}  // namespace

int partition_device(sad_ctx* ctx, int32_t n, const int32_t* key_a, const int32_t* key_b,
                     int32_t p, int32_t* bucket_offsets, int32_t* order, int32_t* pivot_idx,
                     cudaStream_t stream) {
    uint32_t* status = ctx->d_status;
    return partition_run<uint64_t>(
        ctx, n, p,
        [&](uint64_t* K) {
            k_part_keys<<<(n + 255) / 256, 256, 0, stream>>>(n, key_a, key_b, K, status);
        },
        bucket_offsets, order, pivot_idx, stream);
}

int partition_keys64_device(sad_ctx* ctx, int32_t n, const uint64_t* keys, int32_t p,
                            int32_t* bucket_offsets, int32_t* order, int32_t* pivot_idx,
                            cudaStream_t stream) {
    return partition_run<u128>(
        ctx, n, p,
        [&](u128* K) { k_part_keys128<<<(n + 255) / 256, 256, 0, stream>>>(n, keys, K); },
        bucket_offsets, order, pivot_idx, stream);
}

}  // namespace sad

extern "C" int sad_partition(sad_ctx* ctx_in, int32_t n, const int32_t* key_a,
                             const int32_t* key_b, int32_t p, int32_t* bucket_offsets,
                             int32_t* order, int32_t* pivot_idx, int32_t mem, void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mem == SAD_MEM_HOST || mem == SAD_MEM_DEVICE, SAD_EINVAL, "mem = %d", mem);
    SAD_CHECK(n >= 0, SAD_EINVAL, "n = %d < 0", n);
    SAD_CHECK(p >= 1 && p <= kMaxPartitionP, SAD_EINVAL, "p = %d outside 1..%d", p, kMaxPartitionP);
    SAD_CHECK(bucket_offsets && (n == 0 || (order && key_a && key_b)), SAD_EINVAL,
              "a required pointer is NULL");
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    SAD_RET(status_clear(ctx, stream));
    const int32_t* dka = key_a;
    const int32_t* dkb = key_b;
    int32_t *dbo = bucket_offsets, *dord = order, *dpiv = pivot_idx;
    if (mem == SAD_MEM_HOST) {
        void* st = nullptr;
        const size_t nn = (size_t)n + 1;
        SAD_RET(workspace(ctx, WS_PART_OUT, 4 * (nn * 3 + (size_t)p * 2 + 8) + 1024, stream, &st));
        int32_t* s = (int32_t*)st;
        int32_t* ska = s;
        int32_t* skb = ska + nn;
        dord = skb + nn;
        dbo = dord + nn;
        dpiv = pivot_idx ? dbo + p + 1 : nullptr;
        if (n > 0) {
            SAD_CUDA(cudaMemcpyAsync(ska, key_a, 4ull * n, cudaMemcpyHostToDevice, stream));
            SAD_CUDA(cudaMemcpyAsync(skb, key_b, 4ull * n, cudaMemcpyHostToDevice, stream));
        }
        dka = ska;
        dkb = skb;
    }
    SAD_RET(partition_device(ctx, n, dka, dkb, p, dbo, dord, dpiv, stream));
    if (mem == SAD_MEM_HOST) {
        SAD_CUDA(cudaMemcpyAsync(bucket_offsets, dbo, 4ull * (p + 1), cudaMemcpyDeviceToHost, stream));
        if (n > 0) SAD_CUDA(cudaMemcpyAsync(order, dord, 4ull * n, cudaMemcpyDeviceToHost, stream));
        if (pivot_idx && p > 1)
            SAD_CUDA(cudaMemcpyAsync(pivot_idx, dpiv, 4ull * (p - 1), cudaMemcpyDeviceToHost, stream));
    }
    SAD_RET(status_check(ctx, stream));
    uint32_t s = *ctx->h_status;
    SAD_CHECK(!(s & STATUS_BAD_KEY), SAD_EINVAL,
              "a rank key violates 0 <= key_a <= key_b, 1 <= key_b <= 65536");
    return SAD_OK;
}

extern "C" int sad_partition_keys64(sad_ctx* ctx_in, int32_t n, const uint64_t* keys, int32_t p,
                                    int32_t* bucket_offsets, int32_t* order, int32_t* pivot_idx,
                                    int32_t mem, void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mem == SAD_MEM_HOST || mem == SAD_MEM_DEVICE, SAD_EINVAL, "mem = %d", mem);
    SAD_CHECK(n >= 0, SAD_EINVAL, "n = %d < 0", n);
    SAD_CHECK(p >= 1 && p <= kMaxPartitionP, SAD_EINVAL, "p = %d outside 1..%d", p, kMaxPartitionP);
    SAD_CHECK(bucket_offsets && (n == 0 || (order && keys)), SAD_EINVAL, "a required pointer is NULL");
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    SAD_RET(status_clear(ctx, stream));
    const uint64_t* dkeys = keys;
    int32_t *dbo = bucket_offsets, *dord = order, *dpiv = pivot_idx;
    if (mem == SAD_MEM_HOST) {
        void* st = nullptr;
        const size_t nn = (size_t)n + 1;
        SAD_RET(workspace(ctx, WS_PART_OUT, 8 * nn + 4 * (nn + (size_t)p * 2 + 8) + 1024, stream, &st));
        uint64_t* sk = (uint64_t*)st;
        dord = (int32_t*)(sk + nn);
        dbo = dord + nn;
        dpiv = pivot_idx ? dbo + p + 1 : nullptr;
        if (n > 0) SAD_CUDA(cudaMemcpyAsync(sk, keys, 8ull * n, cudaMemcpyHostToDevice, stream));
        dkeys = sk;
    }
    SAD_RET(partition_keys64_device(ctx, n, dkeys, p, dbo, dord, dpiv, stream));
    if (mem == SAD_MEM_HOST) {
        SAD_CUDA(cudaMemcpyAsync(bucket_offsets, dbo, 4ull * (p + 1), cudaMemcpyDeviceToHost, stream));
        if (n > 0) SAD_CUDA(cudaMemcpyAsync(order, dord, 4ull * n, cudaMemcpyDeviceToHost, stream));
        if (pivot_idx && p > 1)
            SAD_CUDA(cudaMemcpyAsync(pivot_idx, dpiv, 4ull * (p - 1), cudaMemcpyDeviceToHost, stream));
    }
    SAD_RET(status_check(ctx, stream));
    return SAD_OK;
}

namespace sad {

// ---------------------------------------------------------------------------
// Allocation-free variant of the partition for callers that cannot allocate
// device memory. Its scratch is one file-scope device array of fixed size,
// laid out like the workspace of partition_device; the same kernels run on it.
namespace {

constexpr size_t kNaK = 0;
constexpr size_t kNaRank = kNaK + 8ull * SAD_NOALLOC_MAX_N;
constexpr size_t kNaBucket = kNaRank + 4ull * SAD_NOALLOC_MAX_N;
constexpr size_t kNaY = kNaBucket + 4ull * SAD_NOALLOC_MAX_N;
constexpr size_t kNaYs = kNaY + 8ull * SAD_NOALLOC_MAX_P * (SAD_NOALLOC_MAX_P - 1);
constexpr size_t kNaPiv = kNaYs + 8ull * SAD_NOALLOC_MAX_P * (SAD_NOALLOC_MAX_P - 1);
constexpr size_t kNaCount = kNaPiv + 8ull * SAD_NOALLOC_MAX_P;
constexpr size_t kNaStatus = kNaCount + 4ull * SAD_NOALLOC_MAX_P;
constexpr size_t kNaBytes = kNaStatus + 256;

std::mutex g_na_mu;
void* g_na_ptr[64] = {nullptr};
unsigned long long g_na_ctx[64] = {0};  // id of the CUDA context the cached address belongs to

}  // namespace

// Every GPU that loads the library holds this array (about 5 MiB) until exit.
static __device__ __align__(256) unsigned char g_partition_scratch[kNaBytes];

namespace {

// Unique id of the CUDA context current on this thread (driver entry points,
// so that no driver library has to be linked); false when there is none or the
// driver does not offer the calls.
using PFN_ctx_current = CUresult (*)(CUcontext*);
using PFN_ctx_id = CUresult (*)(CUcontext, unsigned long long*);
bool current_ctx_id(unsigned long long* id) {
    static PFN_ctx_current get_current = nullptr;
    static PFN_ctx_id get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (PFN_ctx_current)f;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_ctx_id)f;
        cudaGetLastError();
    });
    CUcontext c = nullptr;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of the scratch array on the current device. The host-side
// name of a __device__ array is only a stand-in, so the address is looked up
// with that device current, once per device, and cached together with the id
// of the context it belongs to: after a device reset the runtime makes a new
// context (and a new copy of the array), and the address is looked up again.
int noalloc_scratch(void** out) {
    int dev = 0;
    SAD_CUDA(cudaGetDevice(&dev));
    SAD_CHECK(dev >= 0 && dev < 64, SAD_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_na_mu);
    unsigned long long id = 0;
    bool known = current_ctx_id(&id);
    if (!g_na_ptr[dev] || !known || id != g_na_ctx[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partition_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            set_error("cudaGetSymbolAddress of the partition scratch failed: %s", cudaGetErrorString(e));
            return SAD_ECUDA;
        }
        known = current_ctx_id(&id);  // the lookup made the context current if none was
        g_na_ptr[dev] = p;
        g_na_ctx[dev] = known ? id : 0;
    }
    *out = g_na_ptr[dev];
    return SAD_OK;
}

}  // namespace

}  // namespace sad

extern "C" int sad_partition_noalloc(int32_t n, const int32_t* key_a, const int32_t* key_b, int32_t p,
                                     int32_t* bucket_offsets, int32_t* order, int32_t* pivot_idx,
                                     void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(n >= 0 && n <= SAD_NOALLOC_MAX_N, SAD_EINVAL,
              "n = %d outside 0..%d: the static scratch of sad_partition_noalloc holds at most %d keys",
              n, SAD_NOALLOC_MAX_N, SAD_NOALLOC_MAX_N);
    SAD_CHECK(p >= 1 && p <= SAD_NOALLOC_MAX_P, SAD_EINVAL,
              "p = %d outside 1..%d: the static scratch of sad_partition_noalloc holds at most %d buckets",
              p, SAD_NOALLOC_MAX_P, SAD_NOALLOC_MAX_P);
    SAD_CHECK(bucket_offsets && (n == 0 || (order && key_a && key_b)), SAD_EINVAL,
              "a required pointer is NULL");
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    void* base = nullptr;
    SAD_RET(noalloc_scratch(&base));
    char* w = (char*)base;
    uint64_t* K = (uint64_t*)(w + kNaK);
    int32_t* rank = (int32_t*)(w + kNaRank);
    int32_t* bucket = (int32_t*)(w + kNaBucket);
    uint64_t* Y = (uint64_t*)(w + kNaY);
    uint64_t* Ys = (uint64_t*)(w + kNaYs);
    uint64_t* piv = (uint64_t*)(w + kNaPiv);
    int32_t* count = (int32_t*)(w + kNaCount);
    uint32_t* status = (uint32_t*)(w + kNaStatus);
    const int64_t M = (int64_t)p * (p - 1);
    // the array keeps the previous call's contents: clear what must start at zero
    SAD_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), stream));
    SAD_CUDA(cudaMemsetAsync(count, 0, 4ull * p, stream));
    if (n == 0) {
        SAD_CUDA(cudaMemsetAsync(bucket_offsets, 0, 4ull * (p + 1), stream));
        if (pivot_idx && p > 1) SAD_CUDA(cudaMemsetAsync(pivot_idx, 0xff, 4ull * (p - 1), stream));
        return SAD_OK;
    }
    const int nb = (n + 255) / 256;
    k_part_keys<<<nb, 256, 0, stream>>>(n, key_a, key_b, K, status);
    SAD_LAUNCHED();
    if (p > 1) {
        const int64_t wmax = (n + p - 1) / p + 1;
        dim3 g((unsigned)p, (unsigned)((wmax + 255) / 256));
        k_part_block_rank<<<g, 256, 0, stream>>>(n, p, K, rank);
        SAD_LAUNCHED();
        SAD_CUDA(cudaMemsetAsync(Y, 0xff, 8ull * M, stream));
        k_part_samples<<<nb, 256, 0, stream>>>(n, p, K, rank, Y);
        SAD_LAUNCHED();
        k_part_sample_rank<<<(unsigned)((M + 255) / 256), 256, 0, stream>>>((int32_t)M, Y, Ys);
        SAD_LAUNCHED();
        k_part_pivots<<<(p - 1 + 255) / 256, 256, 0, stream>>>(n, p, Ys, piv, pivot_idx);
        SAD_LAUNCHED();
    }
    k_part_bucket<<<nb, 256, 0, stream>>>(n, p, K, piv, bucket, count);
    SAD_LAUNCHED();
    k_part_offsets<<<1, 32, 0, stream>>>(p, count, bucket_offsets);
    SAD_LAUNCHED();
    k_part_scatter<<<(p + 7) / 8, 256, 0, stream>>>(n, p, bucket, bucket_offsets, order);
    SAD_LAUNCHED();
    // report bad keys: read the status word into thread-local host memory
    static thread_local uint32_t h_status = 0;
    SAD_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    SAD_CUDA(cudaStreamSynchronize(stream));
    SAD_CHECK(!(h_status & STATUS_BAD_KEY), SAD_EINVAL,
              "a rank key violates 0 <= key_a <= key_b, 1 <= key_b <= 65536");
    return SAD_OK;
}
