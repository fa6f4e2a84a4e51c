// Register-only throughput probe of the integer pipes that the alignment
// kernels use: the DPX add-max and 3-way max instructions (32-bit and 16x2)
// and plain 32-bit adds, alone and in the instruction mix of one DP row.
//
// The DP roofline of the alignment kernels is derived from unit counts:
// SMs x integer lanes per clock per SM x clock. This probe measures the lanes
// per clock that the DPX instructions actually retire on the GPU at hand, and
// the rows per clock of the packed row mix, so that the derived peak can be
// checked against the hardware instead of being taken on trust.
//
// One CTA per SM (the dynamic shared memory request admits only one), W warps,
// every thread running C independent chains; the CTA's own SM-clock cycles
// (clock64 around the loop, after a barrier on both sides) give the rate per
// SM, so the result does not depend on the clock frequency.
#include <algorithm>
#include <vector>

#include "sad_internal.cuh"

namespace sad {

namespace {

constexpr int kChains = 8;  // independent chains per thread
constexpr int kUnroll = 16;

// One step of every chain. x[] are the chains, k an addend, neg the -inf of
// the row mixes; every operand that varies comes from another chain so that
// nothing can be hoisted out of the loop.
template <int MIX>
__device__ __forceinline__ void probe_step(uint32_t (&x)[kChains], uint32_t (&y)[kChains], uint32_t k,
                                           uint32_t goge, uint32_t neg) {
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        const int c1 = (c + 1) % kChains, c2 = (c + 2) % kChains;
        if (MIX == SAD_PROBE_VIADDMAX_S32) {
            x[c] = (uint32_t)__viaddmax_s32((int)x[c], (int)k, (int)x[c1]);
        } else if (MIX == SAD_PROBE_VIMAX3_S32) {
            x[c] = (uint32_t)__vimax3_s32((int)x[c], (int)x[c1], (int)x[c2]);
        } else if (MIX == SAD_PROBE_VIADDMAX_S16X2) {
            x[c] = __viaddmax_s16x2(x[c], k, x[c1]);
        } else if (MIX == SAD_PROBE_VIMAX3_S16X2) {
            x[c] = __vimax3_s16x2(x[c], x[c1], x[c2]);
        } else if (MIX == SAD_PROBE_IADD) {
            x[c] = x[c] + x[c1];  // every intermediate value is read by the next chain
        }
    }
    if (MIX == SAD_PROBE_ROW_DPX3_ADD2 || MIX == SAD_PROBE_ROW_DPX5 || MIX == SAD_PROBE_ROW_DPX3) {
        // kChains / 2 rows: x[2r] = H (stored as H + go + ge after the row), x[2r+1] = E;
        // y[2r] = F, y[2r+1] = the diagonal H of the row. The row above row r is r - 1.
#pragma unroll
        for (int r = 0; r < kChains / 2; r++) {
            const int up = (r + kChains / 2 - 1) % (kChains / 2);
            uint32_t hd;
            if (MIX == SAD_PROBE_ROW_DPX3_ADD2)
                hd = y[2 * r + 1] + k;  // diagonal H + s
            else if (MIX == SAD_PROBE_ROW_DPX5)
                hd = __viaddmax_s16x2(y[2 * r + 1], k, neg);
            else
                hd = y[2 * r + 1];
            const uint32_t e = __viaddmax_s16x2(x[2 * r + 1], k, x[2 * r]);  // E: extend, or open from H
            const uint32_t f = __viaddmax_s16x2(y[2 * r], k, x[2 * up]);     // F: from the row above
            const uint32_t h = __vimax3_s16x2(hd, e, f);
            y[2 * r + 1] = x[2 * r];  // this column's H is the next column's diagonal
            x[2 * r + 1] = e;
            y[2 * r] = f;
            if (MIX == SAD_PROBE_ROW_DPX3_ADD2)
                x[2 * r] = h + goge;
            else if (MIX == SAD_PROBE_ROW_DPX5)
                x[2 * r] = __viaddmax_s16x2(h, goge, neg);
            else
                x[2 * r] = h;
        }
    }
}

template <int MIX>
__global__ void k_probe_alu(int32_t iters, uint32_t seed, uint32_t k, uint32_t goge, uint32_t neg,
                            uint32_t* __restrict__ sink, long long* __restrict__ cycles) {
    uint32_t x[kChains], y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        x[c] = seed * (uint32_t)(threadIdx.x + 7 * c + 1);
        y[c] = seed ^ (uint32_t)(threadIdx.x * 13 + c);
    }
    __syncthreads();
    const long long t0 = clock64();
#pragma unroll 1
    for (int32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) probe_step<MIX>(x, y, k, goge, neg);
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) acc ^= x[c] ^ y[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int MIX>
int launch_probe(int grid, int threads, size_t smem, int32_t iters, uint32_t* sink, long long* cyc) {
    SAD_CUDA(cudaFuncSetAttribute(k_probe_alu<MIX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // a warm-up launch, then the measured one
    for (int rep = 0; rep < 2; rep++) {
        k_probe_alu<MIX><<<grid, threads, smem>>>(iters, 0x9e3779b9u, 0x00010001u, 0xfff3fff3u, 0u, sink, cyc);
        SAD_LAUNCHED();
    }
    return SAD_OK;
}

}  // namespace

}  // namespace sad

extern "C" int sad_probe_alu(int32_t mix, int32_t warps_per_sm, int32_t iters, double* lanes_per_clk_sm,
                             double* rows_per_clk_sm) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mix >= 0 && mix < SAD_PROBE_NUM_MIXES, SAD_EINVAL, "unknown probe mix %d", mix);
    SAD_CHECK(warps_per_sm >= 1 && warps_per_sm <= 32, SAD_EINVAL, "warps_per_sm %d outside 1..32", warps_per_sm);
    SAD_CHECK(iters >= 1 && iters <= (1 << 20), SAD_EINVAL, "iters %d outside 1..2^20", iters);
    SAD_CHECK(lanes_per_clk_sm && rows_per_clk_sm, SAD_EINVAL, "an output pointer is NULL");
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(nullptr, &ctx));
    const int grid = ctx->num_sms, threads = 32 * warps_per_sm;
    // more than half of the SM's shared memory: one CTA per SM
    const size_t smem = ctx->smem_optin / 2 + 1024;
    uint32_t* sink = nullptr;
    long long* cyc = nullptr;
    SAD_CUDA(cudaMalloc(&sink, sizeof(uint32_t) * (size_t)grid * threads));
    if (cudaMalloc(&cyc, sizeof(long long) * grid) != cudaSuccess) {
        cudaFree(sink);
        cudaGetLastError();
        set_error("cudaMalloc of the probe's cycle counters failed");
        return SAD_ENOMEM;
    }
    int rc = SAD_OK;
    switch (mix) {
        case SAD_PROBE_VIADDMAX_S32: rc = launch_probe<SAD_PROBE_VIADDMAX_S32>(grid, threads, smem, iters, sink, cyc); break;
        case SAD_PROBE_VIMAX3_S32: rc = launch_probe<SAD_PROBE_VIMAX3_S32>(grid, threads, smem, iters, sink, cyc); break;
        case SAD_PROBE_VIADDMAX_S16X2: rc = launch_probe<SAD_PROBE_VIADDMAX_S16X2>(grid, threads, smem, iters, sink, cyc); break;
        case SAD_PROBE_VIMAX3_S16X2: rc = launch_probe<SAD_PROBE_VIMAX3_S16X2>(grid, threads, smem, iters, sink, cyc); break;
        case SAD_PROBE_IADD: rc = launch_probe<SAD_PROBE_IADD>(grid, threads, smem, iters, sink, cyc); break;
        case SAD_PROBE_ROW_DPX3_ADD2: rc = launch_probe<SAD_PROBE_ROW_DPX3_ADD2>(grid, threads, smem, iters, sink, cyc); break;
        case SAD_PROBE_ROW_DPX5: rc = launch_probe<SAD_PROBE_ROW_DPX5>(grid, threads, smem, iters, sink, cyc); break;
        default: rc = launch_probe<SAD_PROBE_ROW_DPX3>(grid, threads, smem, iters, sink, cyc); break;
    }
    std::vector<long long> h(grid);
    if (rc == SAD_OK) {
        cudaError_t e = cudaMemcpy(h.data(), cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error("probe read-back failed: %s", cudaGetErrorString(e));
            rc = SAD_ECUDA;
        }
    }
    cudaFree(sink);
    cudaFree(cyc);
    if (rc != SAD_OK) return rc;
    std::sort(h.begin(), h.end());
    const double cycles = (double)h[grid / 2];  // median CTA (= SM)
    // chain steps per thread, and the probe operations per chain step
    const double steps = (double)iters * kUnroll;
    const bool row = mix == SAD_PROBE_ROW_DPX3_ADD2 || mix == SAD_PROBE_ROW_DPX5 || mix == SAD_PROBE_ROW_DPX3;
    if (row) {
        const double rows = steps * (kChains / 2) * threads;
        *rows_per_clk_sm = rows / cycles;
        const int dpx = mix == SAD_PROBE_ROW_DPX5 ? 5 : 3;
        *lanes_per_clk_sm = rows * dpx / cycles;  // DPX lanes per clock
    } else {
        *rows_per_clk_sm = 0.0;
        *lanes_per_clk_sm = steps * kChains * threads / cycles;
    }
    return SAD_OK;
}
