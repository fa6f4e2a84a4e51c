// All-pairs k-mer similarity from threshold planes on the 5th-generation
// tensor cores (tcgen05), with the fixed-point D-sum epilogue fused.
//
// min(c, c') = sum_{t>=1} [c >= t][c' >= t]; with planes P_t[i][tau] = [c_i(tau) >= t]
// for t = 1..cap the capped part of a_ij is the dot product of two rows of
// P = [P_1 | ... | P_cap], i.e. one GEMM P P^T. The planes hold 0 or 1.0 in
// e4m3 and the products accumulate in fp32 in tensor memory; every partial sum
// is an integer <= cap * V < 2^24, so the result is exact. (e4m3 rather than
// int8: GB300's int8 tensor rate is far below its fp8 rate.) The part above
// the cap comes from the residual matrix of the sequences whose counts exceed
// it.
//
// Kernel: one CTA per 128 x 128 tile of the upper triangle. Warp 0 streams
// 128 x 128-byte k-blocks of both row panels with TMA (128B swizzle) into a
// ring of shared-memory stages; one thread of warp 1 issues
// tcgen05.mma.kind::f8f6f4 (M = N = 128, K = 32 per instruction) into a TMEM
// accumulator and releases stages with tcgen05.commit; then all four warps
// read the accumulator with tcgen05.ld (warp w owns rows 32w..32w+31) and
// reduce the fixed-point terms into the D sums. Every wait is bounded in time;
// on expiry the kernel sets a status bit, waits (bounded) for its own copies,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "kmer_stage.cuh"

namespace sad {

namespace {

constexpr int kTM = 128;             // tile rows (M) and columns (N)
constexpr int kKB = 128;             // bytes (= e4m3 elements) per k-block
constexpr int kStages = 6;
constexpr int kStageBytes = kTM * kKB;   // one operand panel per stage
constexpr uint32_t kTmemCols = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on any wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of a barrier; false (and the status bit) on timeout.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > kWaitNs) {
            atomicOr(status, STATUS_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int32_t x, int32_t y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                       // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset
    d |= (uint64_t)1 << 46;                       // descriptor version
    d |= (uint64_t)2 << 61;                       // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f8f6f4, A = B = e4m3, D = f32, K-major A and B,
// M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTM >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
          "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
          "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Sum 32 per-lane values over the warp so that lane l ends with the sum of
// everyone's value l (recursive halving: 31 exchanges for 32 sums).
__device__ __forceinline__ uint64_t transpose_reduce32(uint64_t (&x)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int t = 0; t < s; t++) {
            const uint64_t send = upper ? x[t] : x[t + s];
            const uint64_t recv = __shfl_xor_sync(0xffffffffu, send, s);
            x[t] = (upper ? x[t + s] : x[t]) + recv;
        }
    }
    return x[0];
}

struct ColTab {
    int32_t nkb[kTM];
    uint64_t q32[kTM];
    uint32_t r32[kTM];
    int32_t blk[kTM];
    int32_t hidx[kTM];
};

__global__ void __launch_bounds__(128, 1)
k_plane_gemm(const __grid_constant__ CUtensorMap tmap, int32_t n, int32_t kblocks, int32_t ntiles,
             SeqTables tab, uint64_t* __restrict__ dloc, uint64_t* __restrict__ dcen,
             int32_t* __restrict__ A, uint32_t* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kStages];
    __shared__ __align__(8) uint64_t bar_empty[kStages];
    __shared__ __align__(8) uint64_t bar_done;
    __shared__ uint32_t tmem_slot;
    __shared__ int32_t abort_flag;
    __shared__ ColTab ct;
    __shared__ unsigned long long colc[kTM], coll[kTM];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile (ti, tj), ti <= tj, row-major over the upper triangle
    const int64_t idx = blockIdx.x;
    int32_t ti = (int32_t)floor(((2.0 * ntiles + 1.0) -
                                 sqrt((2.0 * ntiles + 1.0) * (2.0 * ntiles + 1.0) - 8.0 * idx)) / 2.0);
    if (ti < 0) ti = 0;
    if (ti > ntiles - 1) ti = ntiles - 1;
    while (ti > 0 && (int64_t)ti * ntiles - (int64_t)ti * (ti - 1) / 2 > idx) ti--;
    while (ti + 1 < ntiles && (int64_t)(ti + 1) * ntiles - (int64_t)(ti + 1) * ti / 2 <= idx) ti++;
    const int32_t tj = ti + (int32_t)(idx - ((int64_t)ti * ntiles - (int64_t)ti * (ti - 1) / 2));
    const int32_t i0 = ti * kTM, j0 = tj * kTM;
    const bool diag = ti == tj;

    // 1024-byte aligned stage ring in dynamic shared memory
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t ring = (raw + 1023u) & ~1023u;
    auto stage_a = [&](int s) { return ring + (uint32_t)(2 * s) * kStageBytes; };
    auto stage_b = [&](int s) { return ring + (uint32_t)(2 * s + 1) * kStageBytes; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_done), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // column tables of this tile
    {
        const int c = threadIdx.x;
        const int32_t j = j0 + c;
        const bool ok = j < n;
        ct.nkb[c] = ok ? tab.nkb[j] : 0;
        ct.q32[c] = ok ? tab.q32[j] : 0;
        ct.r32[c] = ok ? tab.r32[j] : 0;
        ct.blk[c] = ok ? tab.blk[j] : -1;
        ct.hidx[c] = ok ? tab.hidx[j] : -1;
        colc[c] = 0;
        coll[c] = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: TMA k-blocks of the row panels i0.. and j0..
        for (int32_t kb = 0; kb < kblocks; kb++) {
            const int s = kb % kStages;
            if (kb >= kStages && !mbar_wait(smem_u32(&bar_empty[s]), ((kb / kStages) + 1) & 1, status)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (*(volatile int32_t*)&abort_flag) break;
            const uint32_t fb = smem_u32(&bar_full[s]);
            mbar_expect_tx(fb, 2 * kStageBytes);
            tma_load_2d(stage_a(s), &tmap, fb, kb * kKB, i0);
            tma_load_2d(stage_b(s), &tmap, fb, kb * kKB, j0);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        bool ok = true;
        for (int32_t kb = 0; kb < kblocks && ok; kb++) {
            const int s = kb % kStages;
            if (!mbar_wait(smem_u32(&bar_full[s]), (kb / kStages) & 1, status)) {
                atomicExch(&abort_flag, 1);
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int k = 0; k < kKB / 32; k++) {
                const uint64_t da = smem_desc(stage_a(s) + 32u * k);
                const uint64_t db = smem_desc(stage_b(s) + 32u * k);
                mma_f8(tmem, da, db, (kb > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(&bar_empty[s]));
        }
        mma_commit(smem_u32(&bar_done));
    }
    __syncwarp();
    // epilogue: every warp waits for the accumulator
    const bool done_ok = mbar_wait(smem_u32(&bar_done), 0, status);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool valid = done_ok && !*(volatile int32_t*)&abort_flag;

    const int32_t r = warp * 32 + lane;
    const int32_t i = i0 + r;
    const bool oki = i < n;
    const int32_t nki = oki ? tab.nkb[i] : 0;
    const uint64_t qi = oki ? tab.q32[i] : 0;
    const uint32_t ri = oki ? tab.r32[i] : 0;
    const int32_t bli = oki ? tab.blk[i] : -2;
    const int32_t hxi = oki ? tab.hidx[i] : -1;
    uint64_t rs_c = 0, rs_l = 0;
#pragma unroll 1
    for (int c = 0; c < kTM / 32; c++) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(32 * c), v);
        uint64_t cc[32], cl[32];
#pragma unroll
        for (int q = 0; q < 32; q++) {
            const int col = 32 * c + q;
            const int32_t j = j0 + col;
            uint64_t t = 0, tl = 0;
            if (valid && oki && j < n) {
                const uint32_t a = (uint32_t)__uint_as_float(v[q]) +
                                   (uint32_t)residual_at(tab, hxi, ct.hidx[col]);
                t = fixed_term(a, nki, qi, ri, ct.nkb[col], ct.q32[col], ct.r32[col]);
                tl = (bli == ct.blk[col]) ? t : 0;
                if (A) {
                    A[(int64_t)i * n + j] = (int32_t)a;
                    if (!diag) A[(int64_t)j * n + i] = (int32_t)a;
                }
            }
            rs_c += t;
            rs_l += tl;
            cc[q] = t;
            cl[q] = tl;
        }
        if (!diag) {
            const uint64_t sc = transpose_reduce32(cc);
            const uint64_t sl = transpose_reduce32(cl);
            if (sc) atomicAdd(&colc[32 * c + lane], (unsigned long long)sc);
            if (sl) atomicAdd(&coll[32 * c + lane], (unsigned long long)sl);
        }
    }
    if (oki && valid) {
        if (rs_c) atomicAdd((unsigned long long*)&dcen[i], (unsigned long long)rs_c);
        if (rs_l) atomicAdd((unsigned long long*)&dloc[i], (unsigned long long)rs_l);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!diag && valid) {
        const int32_t j = j0 + threadIdx.x;
        if (j < n) {
            if (colc[threadIdx.x]) atomicAdd((unsigned long long*)&dcen[j], colc[threadIdx.x]);
            if (coll[threadIdx.x]) atomicAdd((unsigned long long*)&dloc[j], coll[threadIdx.x]);
        }
    }
    if (warp == 0 && lane == 0 && *(volatile int32_t*)&abort_flag) {
        // let copies already issued land before the CTA exits (bounded)
        for (int s = 0; s < kStages; s++) mbar_wait(smem_u32(&bar_full[s]), 0, status);
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

int get_encoder() {
    std::call_once(g_encode_once, []() {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        cudaGetLastError();
    });
    SAD_CHECK(g_encode != nullptr, SAD_ECUDA, "cuTensorMapEncodeTiled is not available");
    return SAD_OK;
}

}  // namespace

int allpairs_planes(sad_ctx* ctx, int32_t n, int32_t K, const uint8_t* planes, const SeqTables& tab,
                    uint64_t* dloc, uint64_t* dcen, int32_t* A, cudaStream_t stream) {
    if (n == 0) return SAD_OK;
    SAD_CHECK(K % 16 == 0, SAD_EINVAL, "plane row length %d is not a multiple of 16 bytes", K);
    SAD_RET(get_encoder());
    CUtensorMap tmap;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)K};
    const cuuint32_t box[2] = {(cuuint32_t)kKB, (cuuint32_t)kTM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult cr = g_encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)planes, dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    SAD_CHECK(cr == CUDA_SUCCESS, SAD_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    const int32_t ntiles = (n + kTM - 1) / kTM;
    const int64_t ntri = (int64_t)ntiles * (ntiles + 1) / 2;
    const int32_t kblocks = (K + kKB - 1) / kKB;
    const size_t smem = (size_t)2 * kStages * kStageBytes + 1024;
    SAD_RET(allow_max_dynamic_smem(ctx, (const void*)k_plane_gemm));
    k_plane_gemm<<<(unsigned)ntri, 128, smem, stream>>>(tmap, n, kblocks, ntiles, tab, dloc, dcen, A,
                                                        ctx->d_status);
    SAD_LAUNCHED();
    return SAD_OK;
}

}  // namespace sad
