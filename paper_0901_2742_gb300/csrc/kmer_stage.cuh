// Entry points of the k-mer rank stage used across translation units.
#pragma once

#include "kmer_common.cuh"
#include "sad_internal.cuh"

namespace sad {

// Device-resident outputs of the k-mer rank stage.
struct KmerOutDev {
    uint64_t* dloc;
    uint64_t* dcen;
    int32_t* la;
    int32_t* ga;
    int32_t* key_a;
    int32_t* key_b;
    int32_t* A;  // nullable
    uint64_t* G = nullptr;        // globalized rank (with kp->global_samples > 0)
    int32_t* samples = nullptr;   // p * global_samples sample slots
};

int validate_kmer_params(const sad_seqset* s, const sad_kmer_params* kp);

// Run the whole stage on a prepared sequence set; every output is a device
// pointer. Synchronises `stream` once (to size the residual matrix).
int kmer_rank_device(sad_ctx* ctx, const DevSeqs& S, const sad_kmer_params* kp,
                     const KmerOutDev& out, cudaStream_t stream);

// All-pairs similarity from e4m3 threshold planes (n rows of K bytes, rows
// padded to a multiple of 128 with zeros) on the tensor cores, with the same
// fixed-point epilogue as the CUDA-core path.
int allpairs_planes(sad_ctx* ctx, int32_t n, int32_t K, const uint8_t* planes,
                    const SeqTables& tab, uint64_t* dloc, uint64_t* dcen, int32_t* A,
                    cudaStream_t stream);

}  // namespace sad
