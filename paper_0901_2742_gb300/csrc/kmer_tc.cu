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
// Kernel: persistent CTAs (one per SM) walk a list of 128 x BN tiles (BN = 256
// when there are enough of them, else 128) in an L2-friendly order. Warp 0
// streams 128-byte k-blocks of the row panels with TMA (128B swizzle) into a
// ring of shared-memory stages; one thread of warp 1 issues
// tcgen05.mma.kind::f8f6f4 (M = 128, N = BN, K = 32 per instruction) into one
// of two TMEM accumulators and releases stages with tcgen05.commit; the
// epilogue warps (kEpiParts per TMEM lane quadrant) read the other accumulator
// with tcgen05.ld and reduce the fixed-point D terms while the next tile's
// MMAs run. Every wait is bounded in time; on
// expiry the kernel sets a status bit, waits (bounded) for its own copies,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "kmer_stage.cuh"

namespace sad {

namespace {

constexpr int kTM = 128;             // tile rows (M)
constexpr int kKB = 128;             // bytes (= e4m3 elements) per k-block
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

// Per-column table entry of one tile, staged in shared memory by the epilogue
// warps; all lanes read the same entry (broadcast), one 16-byte load. With
// b = nk of the sequence: 2^32 = q b + r, and rf = r / b in fp32. For b = 1
// the pair (q, r) = (2^32 - 1, 1) keeps the same formula exact; for b <= 0 (no
// k-mer fits, so every numerator of the row is 0) q = r = rf = 0.
struct __align__(16) ColRec {
    int32_t nkb;
    uint32_t q32;
    uint32_t r32;
    float rf;
};

// Less frequently needed per-column fields: block (local D) and excess index.
struct __align__(8) ColAux {
    int32_t blk;
    int32_t hidx;
};

__device__ __forceinline__ ColRec col_rec(const SeqTables& tab, int32_t j, int32_t n) {
    ColRec r{0, 0u, 0u, 0.f};
    if (j < n) {
        const int32_t nk = tab.nkb[j];
        r.nkb = nk;
        if (nk >= 2) {
            r.q32 = (uint32_t)tab.q32[j];  // < 2^31
            r.r32 = tab.r32[j];
            r.rf = (float)r.r32 * tab.inv[j];
        } else if (nk == 1) {
            r.q32 = 0xffffffffu;
            r.r32 = 1u;
            r.rf = 1.0f;
        }
    }
    return r;
}

constexpr float kTwo23 = 8388608.0f;     // 2^23: a float in [2^23, 2^24) has unit spacing
constexpr uint32_t kTwo23Bits = 0x4B000000u;

// floor(a 2^32 / b) for b = min(nk_i, nk_j) < 2^16 and 0 <= a <= b (af = a as
// a float): a 2^32 / b = a q + a r / b, and floor(a r / b) < 2^16 is estimated
// as a * rf rounded to the nearest integer (the estimate is off by far less
// than one half), then corrected by one comparison each way. The rounding and
// the float-to-integer move are one fused multiply-add with 2^23 and one
// integer subtraction, exact below 2^23, so no conversion instruction is used.
__device__ __forceinline__ uint64_t fixed_term_tc(uint32_t a, float af, const ColRec& ri, const ColRec& c) {
    const bool take_i = ri.nkb <= c.nkb;
    const int32_t b = max(take_i ? ri.nkb : c.nkb, 1);
    const uint32_t q = take_i ? ri.q32 : c.q32;
    const uint32_t r = take_i ? ri.r32 : c.r32;
    const float rf = take_i ? ri.rf : c.rf;
    const uint32_t x = a * r;
    uint32_t qq = __float_as_uint(fmaf(af, rf, kTwo23)) - kTwo23Bits;
    const int32_t rem = (int32_t)(x - qq * (uint32_t)b);  // |rem| < 2b < 2^17
    qq = rem < 0 ? qq - 1 : (rem >= b ? qq + 1 : qq);
    return (uint64_t)a * q + qq;
}

// One 32-column chunk of the accumulator for this thread's row i: the exact
// numerators and their fixed-point terms; *sum collects the row sum, cw[u] the
// value that column u contributes to the column reduction. kFull: every pair
// of the tile is valid and off the diagonal (i < j < n). kLoc: only pairs of
// the same block count (the local D sum); tiles without such pairs never run
// this pass, so the all-pairs pass keeps a single 32-entry array live.
template <bool kFull, bool kLoc>
__device__ __forceinline__ void epi_chunk(const uint32_t (&v)[32], int col0, int32_t i, int32_t j0, int32_t n,
                                          bool oki, const ColRec& rowr, int32_t bli, int32_t hxi,
                                          const ColRec* __restrict__ ct, const ColAux* __restrict__ cx,
                                          const SeqTables& tab, int32_t* __restrict__ A, uint64_t& sum,
                                          uint64_t (&cw)[32]) {
#pragma unroll
    for (int u = 0; u < 32; u++) {
        const int col = col0 + u;
        const int32_t j = j0 + col;
        const ColRec c = ct[col];
        float af = __uint_as_float(v[u]);  // an integer below 2^16, exact in fp32
        uint32_t av = __float_as_uint(af + kTwo23) - kTwo23Bits;
        if (hxi >= 0) {
            const int32_t hj = cx[col].hidx;
            if (hj >= 0) {
                av += (uint32_t)tab.R[(int64_t)hxi * tab.H + hj];
                af = __uint_as_float(av | kTwo23Bits) - kTwo23;
            }
        }
        uint64_t tv = fixed_term_tc(av, af, rowr, c);
        bool off_diag = true;
        if (!kFull) {
            const bool use = oki && j < n && i <= j;
            tv = use ? tv : 0;
            off_diag = i != j;  // the diagonal counts once, for its own row
        }
        if (kLoc) {
            tv = bli == cx[col].blk ? tv : 0;
        } else if (A && (kFull || (oki && j < n && i <= j))) {
            A[(int64_t)i * n + j] = (int32_t)av;
            if (i != j) A[(int64_t)j * n + i] = (int32_t)av;
        }
        sum += tv;
        cw[u] = off_diag ? tv : 0;
    }
}

constexpr int kEpiParts = 3;                        // epilogue warps per TMEM lane quadrant
constexpr int kEpiWarps = 4 * kEpiParts;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kGemmThreads = (2 + kEpiWarps) * 32;  // producer, MMA issuer, epilogue

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

template <int BN>
__host__ __device__ constexpr int kStagesFor() {
    return BN == 256 ? 4 : 6;
}

// Instruction descriptor: kind::f8f6f4, A = B = e4m3, D = f32, K-major, M = 128, N = BN.
template <int BN>
__host__ __device__ constexpr uint32_t idesc_for() {
    return (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

template <int BN>
__device__ __forceinline__ void mma_f8n(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc_for<BN>()), "r"(accum));
}

// Persistent all-pairs plane GEMM. Warp 0 streams the k-blocks of every tile
// of this CTA with TMA; warp 1 (one thread) issues the MMAs into one of two
// TMEM accumulators (BN columns each) and hands finished accumulators to the
// epilogue; the epilogue warps read an accumulator (warp w owns rows
// 32(w%4)..+31 and every kEpiParts-th 32-column chunk), release it and reduce
// the fixed-point D terms while the next tile's MMAs run. A tile covers rows i0..i0+127 and columns j0..j0+BN-1; the pair (i, j)
// is taken when i <= j (i < j: both D sums, i = j: its own), so every
// unordered pair is counted exactly once whatever the tile shape.
//
// Zero k-blocks: a k-block adds nothing to a tile when its 128-byte slab is
// zero in every row of the tile's row panel or of its column panel (kbm); the
// producer and the MMA thread both skip such k-blocks by the same test, so they
// stay in step. k-block 0 always runs (it initialises the accumulator). The
// MMA thread adds the k-blocks it ran (x BN) to *work.
template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
k_plane_gemm2(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int32_t n,
              int32_t kblocks, const int2* __restrict__ tiles, int32_t ntiles, SeqTables tab, KBlockMap kbm,
              uint64_t* __restrict__ dloc, uint64_t* __restrict__ dcen, int32_t* __restrict__ A,
              unsigned long long* __restrict__ work, uint32_t* __restrict__ status) {
    constexpr int S = kStagesFor<BN>();
    constexpr uint32_t kA = kTM * kKB, kB = BN * kKB;
    // the nonzero k-blocks of a tile: its row panel's and its column panels' bits, ANDed
    auto tile_bits = [&](int32_t i0, int32_t j0, int32_t w) -> uint32_t {
        if (!kbm.bits) return 0xffffffffu;
        const uint32_t fa = kbm.bits[(int64_t)(i0 >> 7) * kbm.kbwords + w];
        uint32_t fb = 0;
#pragma unroll
        for (int q = 0; q < BN / kTM; q++) {
            const int32_t panel = (j0 >> 7) + q;
            if (panel < kbm.npanels) fb |= kbm.bits[(int64_t)panel * kbm.kbwords + w];
        }
        return fa & fb;
    };
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t empty[S];
    __shared__ __align__(8) uint64_t tfull[2];
    __shared__ __align__(8) uint64_t tempty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int32_t abort_flag;
    __shared__ int32_t epi_stop;
    __shared__ ColRec ct[BN];
    __shared__ ColAux cx[BN];
    __shared__ int32_t tile_loc;  // does this tile touch a block on both axes?
    __shared__ unsigned long long colw_c[4][BN], colw_l[4][BN];  // column sums per lane quadrant
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ring = (smem_u32(smem_raw) + 1023u) & ~1023u;
    auto stA = [&](int s) { return ring + (uint32_t)s * (kA + kB); };
    auto stB = [&](int s) { return ring + (uint32_t)s * (kA + kB) + kA; };
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(smem_u32(&tfull[a]), 1);
            mbar_init(smem_u32(&tempty[a]), kEpiWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"((uint32_t)(2 * BN)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    auto aborted = [&]() { return *(volatile int32_t*)&abort_flag != 0; };
    auto give_up = [&]() { atomicExch(&abort_flag, 1); };

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;  // k-blocks issued so far
            for (int32_t t = blockIdx.x; t < ntiles && !aborted(); t += gridDim.x) {
                const int32_t i0 = tiles[t].x * kTM, j0 = tiles[t].y * BN;
                uint32_t bits = 0;
                for (int32_t kb = 0; kb < kblocks; kb++) {
                    if ((kb & 31) == 0) bits = tile_bits(i0, j0, kb >> 5);
                    if (kb > 0 && !((bits >> (kb & 31)) & 1u)) continue;  // zero in a panel: adds nothing
                    const int s = (int)(g % S);
                    if (g >= (uint32_t)S && !mbar_wait(smem_u32(&empty[s]), ((g / S) + 1) & 1, status)) {
                        give_up();
                        break;
                    }
                    if (aborted()) break;
                    const uint32_t fb = smem_u32(&full[s]);
                    mbar_expect_tx(fb, kA + kB);
                    tma_load_2d(stA(s), &tmA, fb, kb * kKB, i0);
                    tma_load_2d(stB(s), &tmB, fb, kb * kKB, j0);
                    g++;
                }
            }
            // on abort, the last copy issued into every stage lands before the CTA exits (bounded)
            if (aborted())
                for (uint32_t h = (g > (uint32_t)S ? g - S : 0); h < g; h++)
                    mbar_wait(smem_u32(&full[h % S]), (h / S) & 1, status);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t g = 0;
            int32_t lt = 0;
            for (int32_t t = blockIdx.x; t < ntiles && !aborted(); t += gridDim.x, lt++) {
                const int a = lt & 1;
                if (lt >= 2 && !mbar_wait(smem_u32(&tempty[a]), ((lt >> 1) + 1) & 1, status)) {
                    give_up();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(a * BN);
                const int32_t i0 = tiles[t].x * kTM, j0 = tiles[t].y * BN;
                uint32_t bits = 0, ran = 0;
                for (int32_t kb = 0; kb < kblocks; kb++) {
                    if ((kb & 31) == 0) bits = tile_bits(i0, j0, kb >> 5);
                    if (kb > 0 && !((bits >> (kb & 31)) & 1u)) continue;  // the producer skips it too
                    const int s = (int)(g % S);
                    g++;
                    ran++;
                    if (!mbar_wait(smem_u32(&full[s]), ((g - 1) / S) & 1, status)) {
                        give_up();
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (int k = 0; k < kKB / 32; k++)
                        mma_f8n<BN>(acc, smem_desc(stA(s) + 32u * k), smem_desc(stB(s) + 32u * k),
                                    (kb > 0 || k > 0) ? 1u : 0u);
                    mma_commit(smem_u32(&empty[s]));
                }
                mma_commit(smem_u32(&tfull[a]));
                if (work) atomicAdd(work, (unsigned long long)ran * BN);
            }
        }
        __syncwarp();
    } else {
        // epilogue warps: TMEM lane quadrant q = warp % 4 (rows 32q..32q+31) and
        // part h; the kEpiParts warps of a quadrant split the tile's chunks
        const int ew = warp - 2;
        const int q = warp & 3;
        const int h = ew >> 2;            // part: chunks h, h + kEpiParts, ...
        const int et = threadIdx.x - 64;  // 0 .. kEpiThreads - 1
        constexpr int kChunks = BN / 32;  // 32-column chunks of a tile
        int32_t lt = 0;
        for (int32_t t = blockIdx.x; t < ntiles; t += gridDim.x, lt++) {
            const int a = lt & 1;
            const int32_t i0 = tiles[t].x * kTM, j0 = tiles[t].y * BN;
            // one thread samples the abort flag so that all epilogue warps leave together
            if (et == 0) epi_stop = aborted() ? 1 : 0;
            epi_barrier();  // also: the previous tile's tables and column sums are no longer read
            if (epi_stop) break;
            for (int c = et; c < BN; c += kEpiThreads) {
                const int32_t j = j0 + c;
                ct[c] = col_rec(tab, j, n);
                ColAux x{-1, -1};
                if (j < n) {
                    x.blk = tab.blk[j];
                    x.hidx = tab.hidx[j];
                }
                cx[c] = x;
            }
            if (et == 0) {
                // blocks are contiguous index ranges: the tile has same-block pairs
                // only if its row and column block ranges overlap
                const int32_t ilast = min(i0 + kTM, n) - 1, jlast = min(j0 + BN, n) - 1;
                tile_loc = (i0 < n && j0 < n && tab.blk[ilast] >= tab.blk[j0] && tab.blk[jlast] >= tab.blk[i0]) ? 1
                                                                                                          : 0;
            }
            epi_barrier();
            const bool any_loc = tile_loc != 0;
            // this thread's row tables, loaded while the tensor core still runs
            const int32_t i = i0 + 32 * q + lane;
            const bool row_ok = i < n;
            const ColRec rowr = col_rec(tab, row_ok ? i : n, n);
            const int32_t bli = row_ok ? tab.blk[i] : -2;
            const int32_t hxi = row_ok ? tab.hidx[i] : -1;
            const bool ok_wait = mbar_wait(smem_u32(&tfull[a]), (lt >> 1) & 1, status);
            if (!ok_wait) give_up();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const bool valid = ok_wait && !aborted();
            const bool oki = valid && row_ok;
            // every pair valid and off the diagonal: the tile lies right of the
            // diagonal and inside n (uniform over the CTA)
            const bool full = i0 + kTM <= j0 && j0 + BN <= n;
            uint64_t rs_c = 0, rs_l = 0;
#pragma unroll 1
            for (int c = h; c < kChunks; c += kEpiParts) {
                uint32_t v[32];
                tmem_ld32(tmem + (uint32_t)(a * BN) + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * c), v);
                uint64_t cw[32];
                if (full)
                    epi_chunk<true, false>(v, 32 * c, i, j0, n, oki, rowr, bli, hxi, ct, cx, tab, A, rs_c, cw);
                else
                    epi_chunk<false, false>(v, 32 * c, i, j0, n, oki, rowr, bli, hxi, ct, cx, tab, A, rs_c, cw);
                // lane l now sums column 32c + l over this warp's 32 rows
                colw_c[q][32 * c + lane] = transpose_reduce32(cw);
                if (any_loc) {
                    // the local sums: a second pass over the same accumulator columns
                    tmem_ld32(tmem + (uint32_t)(a * BN) + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * c), v);
                    if (full)
                        epi_chunk<true, true>(v, 32 * c, i, j0, n, oki, rowr, bli, hxi, ct, cx, tab, A, rs_l, cw);
                    else
                        epi_chunk<false, true>(v, 32 * c, i, j0, n, oki, rowr, bli, hxi, ct, cx, tab, A, rs_l, cw);
                    colw_l[q][32 * c + lane] = transpose_reduce32(cw);
                } else {
                    colw_l[q][32 * c + lane] = 0ull;
                }
            }
            // the accumulator is read: hand it back to the MMA warp
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty[a]));
            if (oki) {
                if (rs_c) atomicAdd((unsigned long long*)&dcen[i], (unsigned long long)rs_c);
                if (rs_l) atomicAdd((unsigned long long*)&dloc[i], (unsigned long long)rs_l);
            }
            epi_barrier();
            if (valid)
                for (int c = et; c < BN; c += kEpiThreads) {
                    const int32_t j = j0 + c;
                    if (j < n) {
                        const unsigned long long sc = colw_c[0][c] + colw_c[1][c] + colw_c[2][c] + colw_c[3][c];
                        const unsigned long long sl = colw_l[0][c] + colw_l[1][c] + colw_l[2][c] + colw_l[3][c];
                        if (sc) atomicAdd((unsigned long long*)&dcen[j], sc);
                        if (sl) atomicAdd((unsigned long long*)&dloc[j], sl);
                    }
                }
        }
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)(2 * BN)));
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

int allpairs_planes(sad_ctx* ctx, int32_t n, int32_t K, const uint8_t* planes, const KBlockMap& kbm,
                    const SeqTables& tab, uint64_t* dloc, uint64_t* dcen, int32_t* A, cudaStream_t stream) {
    if (n == 0) return SAD_OK;
    SAD_CHECK(K % 16 == 0, SAD_EINVAL, "plane row length %d is not a multiple of 16 bytes", K);
    SAD_RET(get_encoder());
    const int32_t nti = (n + kTM - 1) / kTM;
    // 128 x 256 tiles when there are enough of them to fill the GPU, else 128 x 128
    auto count_tiles = [&](int BN) {
        const int32_t ntj = (n + BN - 1) / BN;
        int64_t c = 0;
        for (int32_t ti = 0; ti < nti; ti++)
            for (int32_t tj = 0; tj < ntj; tj++)
                if ((int64_t)BN * tj + BN - 1 >= (int64_t)kTM * ti) c++;
        return c;
    };
    const int BN = count_tiles(256) >= ctx->num_sms ? 256 : 128;
    const int32_t ntj = (n + BN - 1) / BN;
    // L2-friendly order: groups of 8 row tiles sweep the column tiles together
    std::vector<int2> tiles;
    for (int32_t ib = 0; ib < nti; ib += 8)
        for (int32_t tj = 0; tj < ntj; tj++)
            for (int32_t ti = ib; ti < std::min(nti, ib + 8); ti++)
                if ((int64_t)BN * tj + BN - 1 >= (int64_t)kTM * ti) tiles.push_back(make_int2(ti, tj));
    // tile list, then (256-byte aligned) the work counter of this launch. The list
    // depends on n and the tile shape only: it stays on the device between calls
    // and is uploaded (with one synchronisation) only when it changes.
    const size_t work_off = (size_t)round_up((int64_t)(sizeof(int2) * tiles.size()), 256);
    void* dt = nullptr;
    SAD_RET(workspace(ctx, WS_GEMM_TILES, work_off + 16, stream, &dt));
    unsigned long long* work = (unsigned long long*)((char*)dt + work_off);
    SAD_CUDA(cudaMemsetAsync(work, 0, sizeof(unsigned long long), stream));
    ctx->gemm_work = work;
    const bool same = ctx->gemm_tiles_dev == dt && ctx->gemm_tiles_n == n && ctx->gemm_tiles_bn == BN &&
                      ctx->gemm_tiles_count == (int64_t)tiles.size();
    if (!same) {
        void* pin = nullptr;
        SAD_RET(pinned(ctx, sizeof(int2) * tiles.size(), stream, &pin));
        SAD_CUDA(cudaStreamSynchronize(stream));  // the pinned area may feed an earlier copy
        memcpy(pin, tiles.data(), sizeof(int2) * tiles.size());
        SAD_CUDA(cudaMemcpyAsync(dt, pin, sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, stream));
        SAD_CUDA(cudaStreamSynchronize(stream));  // the pinned area is free again for later copies
        ctx->gemm_tiles_dev = dt;
        ctx->gemm_tiles_n = n;
        ctx->gemm_tiles_bn = BN;
        ctx->gemm_tiles_count = (int64_t)tiles.size();
    }
    CUtensorMap tmA, tmB;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)K};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint32_t boxA[2] = {(cuuint32_t)kKB, (cuuint32_t)kTM};
    const cuuint32_t boxB[2] = {(cuuint32_t)kKB, (cuuint32_t)BN};
    CUresult cr = g_encode(&tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)planes, dims, strides, boxA, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    SAD_CHECK(cr == CUDA_SUCCESS, SAD_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    cr = g_encode(&tmB, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)planes, dims, strides, boxB, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    SAD_CHECK(cr == CUDA_SUCCESS, SAD_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    const int32_t kblocks = (K + kKB - 1) / kKB;
    const int32_t ntiles = (int32_t)tiles.size();
    ctx->gemm_dense_units = (int64_t)ntiles * kblocks * BN;  // k-blocks x BN of every tile
    const int grid = std::min<int32_t>(ntiles, ctx->num_sms);
    TraceScope ts(ctx, SAD_STAGE_PLANE_GEMM, stream);
    if (BN == 256) {
        const size_t smem = (size_t)kStagesFor<256>() * (kTM + 256) * kKB + 1024;
        SAD_RET(allow_max_dynamic_smem(ctx, (const void*)k_plane_gemm2<256>));
        k_plane_gemm2<256><<<grid, kGemmThreads, smem, stream>>>(tmA, tmB, n, kblocks, (const int2*)dt, ntiles, tab,
                                                        kbm, dloc, dcen, A, work, ctx->d_status);
    } else {
        const size_t smem = (size_t)kStagesFor<128>() * (kTM + 128) * kKB + 1024;
        SAD_RET(allow_max_dynamic_smem(ctx, (const void*)k_plane_gemm2<128>));
        k_plane_gemm2<128><<<grid, kGemmThreads, smem, stream>>>(tmA, tmB, n, kblocks, (const int2*)dt, ntiles, tab,
                                                        kbm, dloc, dcen, A, work, ctx->d_status);
    }
    SAD_LAUNCHED();
    return SAD_OK;
}

int plane_gemm_work(sad_ctx* ctx, int64_t* mma_flops, int64_t* dense_flops) {
    unsigned long long units = 0;
    if (ctx->gemm_work) SAD_CUDA(cudaMemcpy(&units, ctx->gemm_work, sizeof(units), cudaMemcpyDeviceToHost));
    // one k-block of one tile column: 2 x 128 rows x 128 bytes of K
    *mma_flops = (int64_t)units * 2 * kTM * kKB;
    *dense_flops = ctx->gemm_dense_units * 2 * kTM * kKB;
    return SAD_OK;
}

}  // namespace sad

extern "C" int sad_kmer_gemm_work(sad_ctx* ctx_in, int64_t* mma_flops, int64_t* dense_flops) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mma_flops && dense_flops, SAD_EINVAL, "an output pointer is NULL");
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    return plane_gemm_work(ctx, mma_flops, dense_flops);
}
