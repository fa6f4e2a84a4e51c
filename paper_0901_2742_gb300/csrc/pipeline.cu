// Both stages in one call with every intermediate kept on the device: k-mer
// rank (Section 2), regular-sampling partition (Section 2.3.2) and per-bucket
// alignment scores (algorithm box, "align sequences in each processor").
#include <cstring>

#include "gotoh_stage.cuh"
#include "kmer_stage.cuh"
#include "partition_stage.cuh"
#include "sad_internal.cuh"

extern "C" int sad_pipeline(sad_ctx* ctx_in, const sad_seqset* seqs, const sad_kmer_params* params,
                            const int8_t* subst, int32_t gap_open, int32_t gap_extend, int32_t mode,
                            const sad_rank_out* rank, int32_t* bucket_offsets, int32_t* order,
                            int64_t* score_offsets, int32_t* scores, int64_t scores_capacity,
                            int32_t mem, void* stream_ptr) {
    using namespace sad;
    clear_error();
    SAD_CHECK(mem == SAD_MEM_HOST || mem == SAD_MEM_DEVICE, SAD_EINVAL, "mem = %d", mem);
    SAD_CHECK(seqs && subst && bucket_offsets && score_offsets, SAD_EINVAL,
              "a required pointer is NULL");
    SAD_RET(validate_kmer_params(seqs, params));
    SAD_CHECK(params->p <= kMaxPartitionP, SAD_EINVAL, "p = %d > %d", params->p, kMaxPartitionP);
    SAD_CHECK(gap_open <= 0 && gap_extend <= 0, SAD_EINVAL, "gap costs must be <= 0");
    const int32_t A = seqs->alphabet;
    for (int32_t x = 0; x < A; x++)
        for (int32_t y = 0; y < A; y++)
            SAD_CHECK(subst[x * A + y] == subst[y * A + x], SAD_EINVAL,
                      "substitution matrix is not symmetric at (%d, %d)", x, y);
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    SAD_RET(status_clear(ctx, stream));
    DevSeqs S;
    SAD_RET(prepare_seqs(ctx, seqs, mem, stream, &S));
    const int32_t n = S.n, p = params->p;
    SAD_CHECK(n == 0 || order != nullptr, SAD_EINVAL, "order is NULL");
    int32_t smax = 0;
    for (int32_t t = 0; t < A * A; t++) smax = std::max(smax, (int32_t)std::abs((int)subst[t]));
    const int64_t bound = ((int64_t)smax - gap_open - gap_extend) * 2 * ((int64_t)S.max_len + 1);
    SAD_CHECK(bound < (1ll << 29), SAD_EINVAL, "scores could exceed the 32-bit DP range");
    // intermediates: rank outputs, partition outputs (device)
    const size_t nn = (size_t)(n > 0 ? n : 1);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_dloc = carve(8 * nn), o_dcen = carve(8 * nn), o_la = carve(4ull * p),
                 o_ga = carve(16), o_ka = carve(4 * nn), o_kb = carve(4 * nn),
                 o_bo = carve(4ull * (p + 1)), o_ord = carve(4 * nn), o_so = carve(8ull * (p + 1));
    const int32_t gs = params->global_samples;
    const size_t nslots = (size_t)p * gs;
    const size_t o_G = carve(gs > 0 ? 8 * nn : 0), o_smp = carve(4 * nslots);
    void* w = nullptr;
    SAD_RET(workspace(ctx, WS_PIPE, off, stream, &w));
    char* c = (char*)w;
    KmerOutDev d{(uint64_t*)(c + o_dloc), (uint64_t*)(c + o_dcen), (int32_t*)(c + o_la),
                 (int32_t*)(c + o_ga),     (int32_t*)(c + o_ka),   (int32_t*)(c + o_kb),
                 nullptr};
    int32_t* dbo = (int32_t*)(c + o_bo);
    int32_t* dord = (int32_t*)(c + o_ord);
    int64_t* dso = (int64_t*)(c + o_so);
    if (gs > 0) {
        d.G = (uint64_t*)(c + o_G);
        d.samples = (int32_t*)(c + o_smp);
    }
    // device outputs: the stages write the caller's arrays directly (nothing to copy at the end)
    const bool direct = mem == SAD_MEM_DEVICE;
    if (direct) {
        dbo = bucket_offsets;
        if (n) dord = order;
        dso = score_offsets;
        if (rank) {
            // (arrays of n entries only for n > 0: the stage writes one element of an empty set)
            if (rank->dloc && n) d.dloc = (uint64_t*)rank->dloc;
            if (rank->dcen && n) d.dcen = (uint64_t*)rank->dcen;
            if (rank->la) d.la = rank->la;
            if (rank->ga) d.ga = rank->ga;
            if (rank->key_a && n) d.key_a = rank->key_a;
            if (rank->key_b && n) d.key_b = rank->key_b;
            if (gs > 0 && rank->G && n) d.G = (uint64_t*)rank->G;
            if (gs > 0 && rank->sample_idx) d.samples = rank->sample_idx;
        }
    }
    SAD_RET(kmer_rank_device(ctx, S, params, d, stream));
    if (gs > 0)
        SAD_RET(partition_keys64_device(ctx, n, d.G, p, dbo, dord, nullptr, stream));
    else
        SAD_RET(partition_device(ctx, n, d.key_a, d.key_b, p, dbo, dord, nullptr, stream));
    int32_t* dsc = scores;
    int64_t total = 0;
    if (mem == SAD_MEM_HOST) {
        // the layout is known only after the partition; stage scores on the device
        std::vector<int32_t> hbo((size_t)p + 1);
        SAD_CUDA(cudaMemcpyAsync(hbo.data(), dbo, 4ull * (p + 1), cudaMemcpyDeviceToHost, stream));
        SAD_CUDA(cudaStreamSynchronize(stream));
        for (int32_t b = 0; b < p; b++) {
            const int64_t nb = hbo[b + 1] - hbo[b];
            total += nb * (nb + 1) / 2;
        }
        dsc = nullptr;
        if (total <= scores_capacity) {
            void* so = nullptr;
            SAD_RET(workspace(ctx, WS_SCORE_OUT, 4ull * (total + 1), stream, &so));
            dsc = (int32_t*)so;
        }
    }
    const int rc = bucket_scores_device(ctx, S, dbo, dord, p, subst, gap_open, gap_extend, mode, dso,
                                        dsc, scores_capacity, &total, stream);
    const cudaMemcpyKind k = mem == SAD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (!direct) {
        SAD_CUDA(cudaMemcpyAsync(score_offsets, dso, 8ull * (p + 1), k, stream));
        SAD_CUDA(cudaMemcpyAsync(bucket_offsets, dbo, 4ull * (p + 1), k, stream));
        if (n) SAD_CUDA(cudaMemcpyAsync(order, dord, 4ull * n, k, stream));
    }
    if (rc != SAD_OK) {
        cudaStreamSynchronize(stream);
        return rc;
    }
    if (mem == SAD_MEM_HOST && total > 0)
        SAD_CUDA(cudaMemcpyAsync(scores, dsc, 4ull * total, k, stream));
    if (rank && !direct) {
        if (rank->dloc) SAD_CUDA(cudaMemcpyAsync(rank->dloc, d.dloc, 8ull * n, k, stream));
        if (rank->dcen) SAD_CUDA(cudaMemcpyAsync(rank->dcen, d.dcen, 8ull * n, k, stream));
        if (rank->la) SAD_CUDA(cudaMemcpyAsync(rank->la, d.la, 4ull * p, k, stream));
        if (rank->ga) SAD_CUDA(cudaMemcpyAsync(rank->ga, d.ga, 4, k, stream));
        if (rank->key_a) SAD_CUDA(cudaMemcpyAsync(rank->key_a, d.key_a, 4ull * n, k, stream));
        if (rank->key_b) SAD_CUDA(cudaMemcpyAsync(rank->key_b, d.key_b, 4ull * n, k, stream));
        if (gs > 0 && rank->G) SAD_CUDA(cudaMemcpyAsync(rank->G, d.G, 8ull * n, k, stream));
        if (gs > 0 && rank->sample_idx)
            SAD_CUDA(cudaMemcpyAsync(rank->sample_idx, d.samples, 4 * nslots, k, stream));
    }
    SAD_RET(status_check(ctx, stream));
    return SAD_OK;
}
