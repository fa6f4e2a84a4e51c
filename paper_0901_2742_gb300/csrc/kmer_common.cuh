// Device helpers shared by the all-pairs k-mer similarity kernels (CUDA-core
// and tensor-core forms): the per-sequence tables and the exact fixed-point
// epilogue that turns a similarity numerator into the D-sum terms.
#pragma once

#include <cstdint>

namespace sad {

// Per-sequence tables of one k-mer rank call (device arrays of n entries).
struct SeqTables {
    const int32_t* nkb;   // |x_i| - k + 1 (may be <= 0: no k-mer fits)
    const uint64_t* q32;  // floor(2^32 / nkb) for nkb >= 1
    const uint32_t* r32;  // 2^32 mod nkb for nkb >= 1
    const float* inv;     // 1 / nkb rounded to fp32, for nkb >= 1
    const int32_t* blk;   // block of sequence i: largest b with floor(bN/p) <= i
    const int32_t* hidx;  // index among sequences with counts above the threshold, or -1
    const int32_t* R;     // H x H residual numerators of those sequences
    int32_t H;
};

// floor(a * 2^32 / b) with b = min(nkb_i, nkb_j); 0 when b <= 0.
// With 2^32 = q b + r: a 2^32 / b = a q + a r / b, and a r < b^2 < 2^32 for
// b < 2^16, so the remainder part is a 32-bit division.
__device__ __forceinline__ uint64_t fixed_term(uint32_t a, int32_t nki, uint64_t qi, uint32_t ri,
                                               int32_t nkj, uint64_t qj, uint32_t rj) {
    const bool take_i = nki <= nkj;
    const int32_t b = take_i ? nki : nkj;
    if (b <= 0) return 0;
    const uint64_t q = take_i ? qi : qj;
    const uint32_t r = take_i ? ri : rj;
    if (b < 65536) return (uint64_t)a * q + (uint64_t)((a * r) / (uint32_t)b);
    return ((uint64_t)a << 32) / (uint64_t)b;
}

// The same value as fixed_term without an integer division: the quotient
// floor(a r / b) (< b < 2^16) is estimated in fp32 from the reciprocal 1/b,
// whose relative error with the two roundings is below 3 * 2^-24, i.e. below
// 0.02 in absolute terms; one comparison in each direction then makes it exact.
__device__ __forceinline__ uint64_t fixed_term_fast(uint32_t a, int32_t nki, uint64_t qi, uint32_t ri,
                                                    float invi, int32_t nkj, uint64_t qj, uint32_t rj,
                                                    float invj) {
    const bool take_i = nki <= nkj;
    const int32_t b = take_i ? nki : nkj;
    if (b <= 0) return 0;
    if (b >= 65536) return ((uint64_t)a << 32) / (uint64_t)b;
    const uint64_t q = take_i ? qi : qj;
    const uint32_t r = take_i ? ri : rj;
    const float inv = take_i ? invi : invj;
    const uint32_t x = a * r;
    uint32_t qq = __float2uint_rz(__uint2float_rn(x) * inv);
    const int64_t rem = (int64_t)x - (int64_t)qq * b;
    if (rem < 0) qq--;
    else if (rem >= b) qq++;
    return (uint64_t)a * q + qq;
}

__device__ __forceinline__ int32_t residual_at(const SeqTables& t, int32_t hi, int32_t hj) {
    return (hi >= 0 && hj >= 0) ? t.R[(int64_t)hi * t.H + hj] : 0;
}

}  // namespace sad
