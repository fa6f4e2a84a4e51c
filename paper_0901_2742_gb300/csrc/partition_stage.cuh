// Entry point of the partition stage used across translation units.
#pragma once

#include "sad_internal.cuh"

namespace sad {

constexpr int32_t kMaxPartitionP = 1024;

// Partition on device arrays (keys, outputs). Bad keys set a status bit that
// sad_partition turns into SAD_EINVAL.
int partition_device(sad_ctx* ctx, int32_t n, const int32_t* key_a, const int32_t* key_b,
                     int32_t p, int32_t* bucket_offsets, int32_t* order, int32_t* pivot_idx,
                     cudaStream_t stream);

// The same partition on unsigned 64-bit integer keys (ties by index).
int partition_keys64_device(sad_ctx* ctx, int32_t n, const uint64_t* keys, int32_t p,
                            int32_t* bucket_offsets, int32_t* order, int32_t* pivot_idx,
                            cudaStream_t stream);

}  // namespace sad
