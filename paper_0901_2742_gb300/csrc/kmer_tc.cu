// All-pairs k-mer similarity from threshold planes on the tensor cores.
#include "kmer_stage.cuh"

namespace sad {

int allpairs_planes(sad_ctx* ctx, int32_t n, int32_t K, const uint8_t* planes,
                    const SeqTables& tab, uint64_t* dloc, uint64_t* dcen, int32_t* A,
                    cudaStream_t stream) {
    (void)ctx; (void)n; (void)K; (void)planes; (void)tab; (void)dloc; (void)dcen; (void)A;
    (void)stream;
    set_error("the threshold-plane (cap > 0) path is not available in this build");
    return SAD_EINVAL;
}

}  // namespace sad
