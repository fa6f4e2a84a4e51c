// Entry points of the k-mer rank stage used across translation units.
#pragma once

#include "kmer_common.cuh"
#include "sad_internal.cuh"

namespace sad {

// Residue -> k-mer letter map, passed by value to the counting kernels.
struct ClassMap {
    uint8_t c[SAD_MAX_ALPHABET];
};

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

// True when the k-mer stage runs on sorted (code, count) lists: cap =
// SAD_KMER_SPARSE, or a k-mer space above SAD_MAX_KMER_SPACE.
bool uses_sparse_path(const sad_kmer_params* kp);

// Run the whole stage on a prepared sequence set; every output is a device
// pointer. Synchronises `stream` once (to size the residual matrix).
int kmer_rank_device(sad_ctx* ctx, const DevSeqs& S, const sad_kmer_params* kp,
                     const KmerOutDev& out, cudaStream_t stream);

// Bitmap of the nonzero 128-byte k-blocks of every 128-row panel of the
// threshold planes: bit kb of word kb / 32 of panel q, kbwords words per panel.
struct KBlockMap {
    const uint32_t* bits;
    int32_t kbwords;
    int32_t npanels;
};

// All-pairs similarity from e4m3 threshold planes (n rows of K bytes, rows
// padded to a multiple of 128 with zeros) on the tensor cores, with the same
// fixed-point epilogue as the CUDA-core path. With a k-block map, a tile skips
// the k-blocks that are zero in its row or column panel (exact: they add 0).
int allpairs_planes(sad_ctx* ctx, int32_t n, int32_t K, const uint8_t* planes, const KBlockMap& kbm,
                    const SeqTables& tab, uint64_t* dloc, uint64_t* dcen, int32_t* A,
                    cudaStream_t stream);

// Tensor-core work of the last plane GEMM of ctx: flops of the MMAs issued
// (k-blocks run) and of every k-block of every tile (host values, read after
// the launch completed; synchronises the device).
int plane_gemm_work(sad_ctx* ctx, int64_t* mma_flops, int64_t* dense_flops);

// ---- sorted-list (sparse) k-mer path ----------------------------------------
// Per sequence i: lists[loff[i] + u], u < nd[i], holds (k-mer code, exact count)
// in ascending code order; loff has room for |x_i| - k + 1 entries.
struct SparseLists {
    const uint2* lists;
    const int64_t* loff;
    const int32_t* nd;
};

// Whether the sorted-list path of this k-mer space uses the byte table (one
// byte per k-mer code in shared memory; counts above 1 then go to the residual)
// instead of the hash table (counts above 255 to the residual).
bool sparse_byte_table(const sad_ctx* ctx, int64_t V);

// Sort every sequence's k-mer codes and run-length encode them; counts above T
// also go to the excess lists (ascending code) used by the residual matrix.
int sparse_count(sad_ctx* ctx, const DevSeqs& S, int32_t k, int32_t A2, const ClassMap& cm, int32_t T,
                 const int64_t* loff, uint2* lists, int32_t* nd, const int64_t* ex_off, int32_t* ex_tau,
                 int32_t* ex_val, int32_t* nex, cudaStream_t stream);

// The rows x columns hash-table kernel in four uses. V bounds the distinct
// k-mers of a row set; h_nd is a host copy of every sequence's distinct k-mer
// count and max_nd the largest of them:
// all pairs i <= j with the fused fixed-point D sums (and a_ij into A when not NULL),
int sparse_allpairs(sad_ctx* ctx, int32_t n, const SparseLists& L, const SeqTables& tab,
                    const int32_t* h_nd, int64_t V, uint64_t* dloc, uint64_t* dcen, int32_t* A,
                    cudaStream_t stream);
// G_j += sum over the sample slots of the fixed-point terms (globalized rank),
int sparse_sample_sums(sad_ctx* ctx, int32_t n, int32_t nslots, const int32_t* samples, const SparseLists& L,
                       const SeqTables& tab, int32_t max_nd, int64_t V, uint64_t* G, cudaStream_t stream);
// the global-ancestor sums over the local ancestors (gsum[b], b < p),
int sparse_ga_sums(sad_ctx* ctx, int32_t n, int32_t p, const int32_t* la, const SparseLists& L,
                   const SeqTables& tab, int32_t max_nd, int64_t V, uint64_t* gsum, cudaStream_t stream);
// and the rank keys of every sequence against the global ancestor.
int sparse_key_column(sad_ctx* ctx, int32_t n, const int32_t* ga, const SparseLists& L, const SeqTables& tab,
                      int32_t max_nd, int64_t V, int32_t* key_a, int32_t* key_b, cudaStream_t stream);

}  // namespace sad
