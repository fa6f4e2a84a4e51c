// Internal runtime shared by the CUDA translation units of libsad: error
// reporting, the per-device context with its cached workspaces, host/device
// staging and the device-resident copy of a sequence set.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <vector>

#include "sad.h"

namespace sad {

void set_error(const char* fmt, ...);
void clear_error();

#define SAD_CUDA(expr)                                                                      \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            ::sad::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, \
                             __LINE__);                                                     \
            return SAD_ECUDA;                                                               \
        }                                                                                   \
    } while (0)

// After a kernel launch: count it and surface launch errors.
void note_launch();
#define SAD_LAUNCHED()                      \
    do {                                    \
        ::sad::note_launch();               \
        SAD_CUDA(cudaGetLastError());       \
    } while (0)

#define SAD_CHECK(cond, code, ...)            \
    do {                                      \
        if (!(cond)) {                        \
            ::sad::set_error(__VA_ARGS__);    \
            return (code);                    \
        }                                     \
    } while (0)

#define SAD_RET(expr)              \
    do {                           \
        int _rc = (expr);          \
        if (_rc != SAD_OK) return _rc; \
    } while (0)

// Bits of the device status word (set by kernels with atomicOr).
enum : uint32_t {
    STATUS_BAD_RESIDUE = 1u << 0,   // a residue code >= alphabet
    STATUS_TIMEOUT = 1u << 1,       // a bounded wait gave up
    STATUS_CAPACITY = 1u << 2,      // an internal capacity was exceeded
    STATUS_BAD_INPUT = 1u << 3,     // an input array holds a value out of range
};

// Workspace slots; each slot is a grow-only device buffer owned by a context.
enum Slot : int {
    WS_RES_STAGE = 0,  // host-mode residue staging
    WS_OFFS,           // int64 offsets copy
    WS_RES_PAD,        // 16-byte aligned residues
    WS_SEQ_META,       // padded offsets, lengths
    WS_COUNTS,         // uint8 counts
    WS_PLANES,         // threshold planes
    WS_EXCESS,         // excess lists
    WS_HEAVY,          // heavy index/list, residual matrix
    WS_KMER_MISC,      // per-sequence aux arrays
    WS_RANK_OUT,       // staging of rank outputs (host mode)
    WS_PART,           // partition scratch
    WS_PART_OUT,       // staging of partition outputs
    WS_SCORE_PLAN,     // Gotoh work items and per-bucket tables
    WS_SCORE_SCRATCH,  // strip-boundary scratch of the Gotoh kernels
    WS_SCORE_OUT,      // staging of scores (host mode)
    WS_SCORE_ITEMS,    // packed-kernel work items and queue heads
    WS_SCORE_SCRATCH_LONG,  // strip boundaries of queries too long to pack
    WS_PIPE,           // pipeline intermediates
    WS_GEMM_TILES,     // tile list of the plane GEMM
    WS_GLOBAL,         // block order of the globalized rank
    WS_TRACE,          // alignment (traceback) call: pairs, offsets, outputs
    WS_TRACE_DIRS,     // traceback direction words
    WS_KBLOCKS,        // per 128-row panel of the planes: bitmap of nonzero 128-byte k-blocks
    WS_TREE,           // guide trees: tables, cluster matrices, staging
    WS_PROG,           // progressive alignment: call tables and staged outputs
    WS_PROG_LEVEL,     // progressive alignment: one batch of merges (jobs, scores, directions)
    WS_NUM_SLOTS
};

struct Buffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// Variant table of the packed alignment kernel: query pairs with at most
// upper[b] rows use R[b] rows per lane and G[b] lanes per subject.
struct ScoreTuning {
    static constexpr int kMaxBins = 16;
    int nbins = 0;
    int32_t upper[kMaxBins] = {};
    int32_t R[kMaxBins] = {};
    int32_t G[kMaxBins] = {};
    // autotuning in progress: only query pairs with lo < rows <= hi are
    // scored, all with variant (force_R, force_G)
    bool filter = false;
    bool skipped = false;  // set when a pair of the bin did not fit the forced variant
    int32_t lo = 0, hi = 0, force_R = 0, force_G = 0;
};

struct TraceStage {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    double ms = 0;
    int32_t count = 0;
};

// One traced interval: stage and its start and end in ms after the first
// traced interval's start.
struct TraceSpan {
    int32_t stage;
    double t0, t1;
};

}  // namespace sad

struct sad_ctx {
    int device = 0;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    size_t smem_optin = 0;
    sad::Buffer ws[sad::WS_NUM_SLOTS];
    uint32_t* d_status = nullptr;     // device status word
    uint32_t* h_status = nullptr;     // pinned mirror
    void* h_pinned = nullptr;         // small pinned staging area
    size_t h_pinned_bytes = 0;
    std::mutex mu;
    sad::ScoreTuning tuning;
    cudaGraphExec_t score_graph = nullptr;  // last batched score launch set, replayed while unchanged
    std::vector<char> score_graph_sig;
    bool aux_ready = false;
    cudaStream_t aux[8] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[8] = {};
    bool trace_on = false;
    sad::TraceStage trace[SAD_NUM_STAGES];
    cudaEvent_t trace_origin = nullptr;      // begin event of the first interval since the last read
    std::vector<sad::TraceSpan> timeline;    // intervals of the last read, by start time
    std::vector<cudaEvent_t> event_pool;
    unsigned long long* gemm_work = nullptr;  // device: k-blocks x BN the last plane GEMM ran
    int64_t gemm_dense_units = 0;             // k-blocks x BN of all its tiles
    void* gemm_tiles_dev = nullptr;           // tile list on the device, for (n, BN, count) below
    int32_t gemm_tiles_n = -1, gemm_tiles_bn = 0;
    int64_t gemm_tiles_count = 0;
    std::vector<sad::Buffer> prog_chunks;     // progressive alignment: profile and column-map arena
    int32_t prog_columns = 0;                 // progressive DP columns per lane step: 0 chosen per batch, 1, 2
    int64_t prog_spin_limit = 0;              // progressive strip hand-off wait bound in polls: 0 = the default
};

namespace sad {

// Resolve ctx (NULL -> default context of the current device) and make its
// device current.
int resolve_ctx(sad_ctx* in, sad_ctx** out);

// Grow-only workspace of a slot; synchronises `stream` before freeing an old
// buffer. Returns SAD_OK and the pointer, or SAD_ENOMEM.
int workspace(sad_ctx* ctx, Slot slot, size_t bytes, cudaStream_t stream, void** out);

// Allow kernel `fn` the device's maximum dynamic shared memory. The attribute
// is process-wide per kernel, so it is raised once (under a lock) and never
// lowered: concurrent callers with different needs cannot race on it.
int allow_max_dynamic_smem(sad_ctx* ctx, const void* fn);

// Pinned host scratch of at least `bytes` (grow-only).
int pinned(sad_ctx* ctx, size_t bytes, cudaStream_t stream, void** out);

// Device status word helpers: clear before a stage, read (synchronising
// `stream`) after it and turn set bits into an error code.
int status_clear(sad_ctx* ctx, cudaStream_t stream);
int status_check(sad_ctx* ctx, cudaStream_t stream);

// Copy `bytes` from an argument buffer in `mem` space into device memory of a
// workspace slot (host mode), or return the device pointer itself.
int arg_to_device(sad_ctx* ctx, Slot slot, const void* arg, size_t bytes, int32_t mem,
                  cudaStream_t stream, const void** dev);

// Read a small argument array in `mem` space into host memory.
int arg_to_host(const void* arg, size_t bytes, int32_t mem, cudaStream_t stream, void* host);

// Device-resident sequence set: every sequence starts on a 16-byte boundary
// and is followed by at least 16 bytes of zero padding.
struct DevSeqs {
    int32_t n = 0;
    int32_t alphabet = 0;
    const uint8_t* res = nullptr;   // padded residues
    const int64_t* pad_off = nullptr;  // n+1 padded starts
    const int32_t* len = nullptr;   // n lengths
    std::vector<int64_t> h_off;     // host copy of the caller's offsets
    std::vector<int32_t> h_len;     // host lengths
    int32_t max_len = 0;
};

// Validate a sequence set and build its device-resident copy (residue codes
// are checked on the device; a bad code sets STATUS_BAD_RESIDUE).
int prepare_seqs(sad_ctx* ctx, const sad_seqset* s, int32_t mem, cudaStream_t stream,
                 DevSeqs* out);

constexpr int kAuxStreams = 8;  // forked streams for concurrent kernel variants

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Tracer internals (the caller holds ctx->mu): clear and switch on/off; wait
// for the recorded events and report per-stage milliseconds and counts.
int trace_reset(sad_ctx* ctx, bool on);
int trace_collect(sad_ctx* ctx, double* ms, int32_t* counts, int32_t nstages);

// Records CUDA events around a stage on `stream` when the context traces.
class TraceScope {
  public:
    TraceScope(sad_ctx* ctx, int stage, cudaStream_t stream);
    ~TraceScope();

  private:
    sad_ctx* ctx_;
    int stage_;
    cudaStream_t stream_;
    cudaEvent_t end_ = nullptr;
};

}  // namespace sad
