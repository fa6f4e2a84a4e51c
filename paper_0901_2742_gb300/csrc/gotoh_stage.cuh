// Entry points of the per-bucket alignment-score stage used across
// translation units.
#pragma once

#include <vector>

#include "sad_internal.cuh"

namespace sad {

// One work item: query row `q` (position in its bucket's length order) against
// the subjects at length-order positions [v0, v1) of the same bucket.
struct GotohItem {
    int32_t bucket;
    int32_t q;
    int32_t v0;
    int32_t v1;
};

struct GotohLaunch {
    const int32_t* order = nullptr;
    const int32_t* bucket_off = nullptr;
    const int32_t* srt = nullptr;
    const int64_t* score_off = nullptr;
    int32_t* scores = nullptr;
    const int8_t* subst = nullptr;
    int32_t go = 0, ge = 0;
    int32_t bias = 0;  // packed form: stored DP value = true value + bias
    int R = 16, G = 32;
    int32_t max_m = 0;
    const GotohItem* items = nullptr;
    int32_t n_items = 0;
    int32_t* head = nullptr;  // persistent queue head (zeroed), or NULL
    bool persistent = false;
    int persistent_grid = 0;
};

void plan_buckets(const std::vector<int32_t>& h_bo, const std::vector<int32_t>& h_order,
                  const std::vector<int32_t>& h_len, int32_t p, std::vector<int32_t>* srt,
                  std::vector<int64_t>* score_off);

int gotoh_launch(sad_ctx* ctx, const DevSeqs& S, const GotohLaunch& L, cudaStream_t stream);

// Scores for a bucket layout already on the device (synchronises `stream`
// once to plan on the host). d_score_off_out (p+1) may be NULL.
int bucket_scores_device(sad_ctx* ctx, const DevSeqs& S, const int32_t* d_bo, const int32_t* d_order,
                         int32_t p, const int8_t* h_subst, int32_t go, int32_t ge, int32_t mode,
                         int64_t* d_score_off_out, int32_t* d_scores, int64_t capacity,
                         int64_t* total_out, cudaStream_t stream);

}  // namespace sad
