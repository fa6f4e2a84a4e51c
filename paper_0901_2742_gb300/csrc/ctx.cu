// Context, workspaces, error reporting and sequence staging for libsad.
#include <cstdarg>
#include <atomic>
#include <algorithm>
#include <cstring>

#include "sad_internal.cuh"

namespace sad {

namespace {
thread_local char g_err[1024] = "";
std::atomic<uint64_t> g_launches{0};
std::mutex g_default_mu;
sad_ctx* g_default[64] = {nullptr};
}  // namespace

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static cudaEvent_t take_event(sad_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

TraceScope::TraceScope(sad_ctx* ctx, int stage, cudaStream_t stream)
    : ctx_(ctx), stage_(stage), stream_(stream) {
    if (!ctx_ || !ctx_->trace_on) return;
    cudaEvent_t b = take_event(ctx_);
    end_ = take_event(ctx_);
    if (!b || !end_) return;
    cudaEventRecord(b, stream_);
    if (!ctx_->trace_origin) ctx_->trace_origin = b;
    ctx_->trace[stage_].pending.push_back({b, end_});
}

TraceScope::~TraceScope() {
    if (end_) cudaEventRecord(end_, stream_);
}

static int ctx_init(int32_t device, sad_ctx* c) {
    int ndev = 0;
    SAD_CUDA(cudaGetDeviceCount(&ndev));
    SAD_CHECK(device >= 0 && device < ndev, SAD_EINVAL, "device %d out of range (%d devices)",
              device, ndev);
    SAD_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    SAD_CUDA(cudaGetDeviceProperties(&prop, device));
    SAD_CHECK(prop.major == 10 && prop.minor == 3, SAD_ECUDA,
              "libsad is built for sm_103 (GB300); device %d is sm_%d%d", device, prop.major,
              prop.minor);
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    c->cc_major = prop.major;
    c->cc_minor = prop.minor;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    SAD_CUDA(cudaMalloc(&c->d_status, sizeof(uint32_t)));
    SAD_CUDA(cudaMemset(c->d_status, 0, sizeof(uint32_t)));
    SAD_CUDA(cudaMallocHost(&c->h_status, sizeof(uint32_t)));
    return SAD_OK;
}

int resolve_ctx(sad_ctx* in, sad_ctx** out) {
    if (in) {
        SAD_CUDA(cudaSetDevice(in->device));
        *out = in;
        return SAD_OK;
    }
    int dev = 0;
    SAD_CUDA(cudaGetDevice(&dev));
    SAD_CHECK(dev >= 0 && dev < 64, SAD_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_default_mu);
    if (!g_default[dev]) {
        sad_ctx* c = new sad_ctx();
        int rc = ctx_init(dev, c);
        if (rc != SAD_OK) {
            delete c;
            return rc;
        }
        g_default[dev] = c;
    }
    *out = g_default[dev];
    return SAD_OK;
}

int workspace(sad_ctx* ctx, Slot slot, size_t bytes, cudaStream_t stream, void** out) {
    Buffer& b = ctx->ws[slot];
    if (bytes == 0) bytes = 16;
    if (b.bytes < bytes) {
        if (b.ptr) {
            SAD_CUDA(cudaStreamSynchronize(stream));
            SAD_CUDA(cudaFree(b.ptr));
            b.ptr = nullptr;
            b.bytes = 0;
        }
        size_t want = bytes + bytes / 8;  // some headroom against repeated growth
        cudaError_t e = cudaMalloc(&b.ptr, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.ptr = nullptr;
            set_error("cudaMalloc of %zu bytes for workspace slot %d failed: %s", want, (int)slot,
                      cudaGetErrorString(e));
            return SAD_ENOMEM;
        }
        b.bytes = want;
    }
    *out = b.ptr;
    return SAD_OK;
}

int allow_max_dynamic_smem(sad_ctx* ctx, const void* fn) {
    static std::mutex mu;
    static std::vector<std::pair<int, const void*>> done;
    std::lock_guard<std::mutex> lock(mu);
    for (auto& d : done)
        if (d.first == ctx->device && d.second == fn) return SAD_OK;
    cudaFuncAttributes attr;
    SAD_CUDA(cudaFuncGetAttributes(&attr, fn));
    const int dyn = (int)ctx->smem_optin - (int)attr.sharedSizeBytes;  // room left by static smem
    SAD_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    done.push_back({ctx->device, fn});
    return SAD_OK;
}

int pinned(sad_ctx* ctx, size_t bytes, cudaStream_t stream, void** out) {
    if (ctx->h_pinned_bytes < bytes) {
        if (ctx->h_pinned) {
            SAD_CUDA(cudaStreamSynchronize(stream));
            SAD_CUDA(cudaFreeHost(ctx->h_pinned));
            ctx->h_pinned = nullptr;
            ctx->h_pinned_bytes = 0;
        }
        size_t want = bytes + bytes / 8 + 4096;
        cudaError_t e = cudaMallocHost(&ctx->h_pinned, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMallocHost of %zu bytes failed: %s", want, cudaGetErrorString(e));
            return SAD_ENOMEM;
        }
        ctx->h_pinned_bytes = want;
    }
    *out = ctx->h_pinned;
    return SAD_OK;
}

int status_clear(sad_ctx* ctx, cudaStream_t stream) {
    SAD_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), stream));
    return SAD_OK;
}

int status_check(sad_ctx* ctx, cudaStream_t stream) {
    SAD_CUDA(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, stream));
    SAD_CUDA(cudaStreamSynchronize(stream));
    SAD_CUDA(cudaGetLastError());
    uint32_t s = *ctx->h_status;
    SAD_CHECK(!(s & STATUS_BAD_RESIDUE), SAD_EINVAL, "a residue code is >= the alphabet size");
    SAD_CHECK(!(s & STATUS_TIMEOUT), SAD_ETIMEOUT, "a bounded device-side wait gave up");
    SAD_CHECK(!(s & STATUS_CAPACITY), SAD_ECUDA, "an internal device capacity was exceeded");
    SAD_CHECK(!(s & STATUS_BAD_INPUT), SAD_EINVAL, "an input array holds a value out of range");
    return SAD_OK;
}

int arg_to_device(sad_ctx* ctx, Slot slot, const void* arg, size_t bytes, int32_t mem,
                  cudaStream_t stream, const void** dev) {
    if (mem == SAD_MEM_DEVICE) {
        *dev = arg;
        return SAD_OK;
    }
    void* d = nullptr;
    SAD_RET(workspace(ctx, slot, bytes, stream, &d));
    if (bytes) SAD_CUDA(cudaMemcpyAsync(d, arg, bytes, cudaMemcpyHostToDevice, stream));
    *dev = d;
    return SAD_OK;
}

int arg_to_host(const void* arg, size_t bytes, int32_t mem, cudaStream_t stream, void* host) {
    if (!bytes) return SAD_OK;
    if (mem == SAD_MEM_HOST) {
        memcpy(host, arg, bytes);
        return SAD_OK;
    }
    SAD_CUDA(cudaMemcpyAsync(host, arg, bytes, cudaMemcpyDeviceToHost, stream));
    SAD_CUDA(cudaStreamSynchronize(stream));
    return SAD_OK;
}

// One CTA per sequence: copy into the 16-byte aligned layout, zero the
// padding, and flag any residue code >= alphabet.
__global__ void k_gather_pad(const uint8_t* __restrict__ src, const int64_t* __restrict__ off,
                             const int64_t* __restrict__ pad_off, int32_t alphabet,
                             uint8_t* __restrict__ dst, uint32_t* __restrict__ status) {
    const int32_t i = blockIdx.x;
    const int64_t s0 = off[i], len = off[i + 1] - off[i];
    const int64_t d0 = pad_off[i], dlen = pad_off[i + 1] - pad_off[i];
    bool bad = false;
    for (int64_t t = threadIdx.x; t < dlen; t += blockDim.x) {
        uint8_t v = 0;
        if (t < len) {
            v = src[s0 + t];
            if (v >= alphabet) {
                bad = true;
                v = 0;
            }
        }
        dst[d0 + t] = v;
    }
    if (bad) atomicOr(status, STATUS_BAD_RESIDUE);
}

int prepare_seqs(sad_ctx* ctx, const sad_seqset* s, int32_t mem, cudaStream_t stream,
                 DevSeqs* out) {
    SAD_CHECK(s != nullptr, SAD_EINVAL, "seqs is NULL");
    SAD_CHECK(s->n >= 0, SAD_EINVAL, "n = %d < 0", s->n);
    SAD_CHECK(s->alphabet >= 1 && s->alphabet <= SAD_MAX_ALPHABET, SAD_EINVAL,
              "alphabet %d outside 1..%d", s->alphabet, SAD_MAX_ALPHABET);
    SAD_CHECK(s->offsets != nullptr, SAD_EINVAL, "offsets is NULL");
    const int32_t n = s->n;
    out->n = n;
    out->alphabet = s->alphabet;
    out->h_off.resize((size_t)n + 1);
    SAD_RET(arg_to_host(s->offsets, sizeof(int64_t) * (n + 1), mem, stream, out->h_off.data()));
    SAD_CHECK(out->h_off[0] == 0, SAD_EINVAL, "offsets[0] = %lld, must be 0",
              (long long)out->h_off[0]);
    out->h_len.resize(n);
    std::vector<int64_t> pad((size_t)n + 1);
    pad[0] = 0;
    int32_t mx = 0;
    for (int32_t i = 0; i < n; i++) {
        int64_t L = out->h_off[i + 1] - out->h_off[i];
        SAD_CHECK(L >= 0 && L <= (1 << 24), SAD_EINVAL,
                  "sequence %d has length %lld (offsets must be nondecreasing, length <= 2^24)", i,
                  (long long)L);
        out->h_len[i] = (int32_t)L;
        mx = L > mx ? (int32_t)L : mx;
        pad[i + 1] = pad[i] + round_up(L, 16) + 16;
    }
    out->max_len = mx;
    const int64_t total = out->h_off[n];
    SAD_CHECK(n == 0 || s->residues != nullptr || total == 0, SAD_EINVAL, "residues is NULL");
    // device metadata: padded offsets (n+1 int64) then lengths (n int32)
    void* meta = nullptr;
    size_t meta_bytes = sizeof(int64_t) * (n + 1) + sizeof(int32_t) * (n + 4);
    SAD_RET(workspace(ctx, WS_SEQ_META, meta_bytes, stream, &meta));
    int64_t* d_pad = (int64_t*)meta;
    int32_t* d_len = (int32_t*)(d_pad + n + 1);
    void* pin = nullptr;
    SAD_RET(pinned(ctx, meta_bytes, stream, &pin));
    // the pinned area may still feed a previous copy (with device offsets the
    // stream was synchronised just above, reading them)
    if (mem == SAD_MEM_HOST) SAD_CUDA(cudaStreamSynchronize(stream));
    memcpy(pin, pad.data(), sizeof(int64_t) * (n + 1));
    memcpy((char*)pin + sizeof(int64_t) * (n + 1), out->h_len.data(), sizeof(int32_t) * n);
    SAD_CUDA(cudaMemcpyAsync(meta, pin, sizeof(int64_t) * (n + 1) + sizeof(int32_t) * n,
                             cudaMemcpyHostToDevice, stream));
    void* dres = nullptr;
    SAD_RET(workspace(ctx, WS_RES_PAD, (size_t)pad[n] + 64, stream, &dres));
    if (n > 0) {
        const void* src = nullptr;
        SAD_RET(arg_to_device(ctx, WS_RES_STAGE, s->residues, (size_t)total, mem, stream, &src));
        const void* doff = nullptr;
        SAD_RET(arg_to_device(ctx, WS_OFFS, s->offsets, sizeof(int64_t) * (n + 1), mem, stream,
                              &doff));
        TraceScope ts(ctx, SAD_STAGE_PREPARE, stream);
        k_gather_pad<<<n, 128, 0, stream>>>((const uint8_t*)src, (const int64_t*)doff, d_pad,
                                            s->alphabet, (uint8_t*)dres, ctx->d_status);
        SAD_LAUNCHED();
    }
    out->res = (const uint8_t*)dres;
    out->pad_off = d_pad;
    out->len = d_len;
    return SAD_OK;
}


int trace_reset(sad_ctx* ctx, bool on) {
    for (auto& st : ctx->trace) {
        for (auto& pr : st.pending) {
            cudaEventSynchronize(pr.second);
            ctx->event_pool.push_back(pr.first);
            ctx->event_pool.push_back(pr.second);
        }
        st.pending.clear();
        st.ms = 0;
        st.count = 0;
    }
    ctx->trace_origin = nullptr;
    ctx->timeline.clear();
    ctx->trace_on = on;
    return SAD_OK;
}

int trace_collect(sad_ctx* ctx, double* ms, int32_t* counts, int32_t nstages) {
    // every interval's times first (the origin is one of the begin events), then
    // the events go back to the pool
    ctx->timeline.clear();
    for (int s = 0; s < SAD_NUM_STAGES; s++) {
        auto& st = ctx->trace[s];
        for (auto& pr : st.pending) {
            SAD_CUDA(cudaEventSynchronize(pr.second));
            float t = 0, a = 0, b = 0;
            SAD_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second));
            SAD_CUDA(cudaEventElapsedTime(&a, ctx->trace_origin, pr.first));
            SAD_CUDA(cudaEventElapsedTime(&b, ctx->trace_origin, pr.second));
            ctx->timeline.push_back(TraceSpan{s, a, b});
            st.ms += t;
            st.count++;
        }
    }
    std::stable_sort(ctx->timeline.begin(), ctx->timeline.end(),
                     [](const TraceSpan& x, const TraceSpan& y) { return x.t0 < y.t0; });
    for (int s = 0; s < SAD_NUM_STAGES; s++) {
        auto& st = ctx->trace[s];
        for (auto& pr : st.pending) {
            ctx->event_pool.push_back(pr.first);
            ctx->event_pool.push_back(pr.second);
        }
        st.pending.clear();
        if (s < nstages) {
            ms[s] = st.ms;
            counts[s] = st.count;
        }
        st.ms = 0;
        st.count = 0;
    }
    ctx->trace_origin = nullptr;
    for (int s = SAD_NUM_STAGES; s < nstages; s++) {
        ms[s] = 0;
        counts[s] = 0;
    }
    return SAD_OK;
}

}  // namespace sad

extern "C" {

int sad_ctx_create(int32_t device, sad_ctx** out) {
    sad::clear_error();
    SAD_CHECK(out != nullptr, SAD_EINVAL, "out is NULL");
    sad_ctx* c = new sad_ctx();
    int rc = sad::ctx_init(device, c);
    if (rc != SAD_OK) {
        delete c;
        return rc;
    }
    *out = c;
    return SAD_OK;
}

int sad_ctx_destroy(sad_ctx* ctx) {
    sad::clear_error();
    if (!ctx) return SAD_OK;
    SAD_CUDA(cudaSetDevice(ctx->device));
    SAD_CUDA(cudaDeviceSynchronize());
    for (auto& b : ctx->ws)
        if (b.ptr) cudaFree(b.ptr);
    for (auto& b : ctx->prog_chunks)
        if (b.ptr) cudaFree(b.ptr);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->score_graph) cudaGraphExecDestroy(ctx->score_graph);
    if (ctx->aux_ready) {
        for (int v = 0; v < sad::kAuxStreams; v++) {
            cudaStreamDestroy(ctx->aux[v]);
            cudaEventDestroy(ctx->ev_join[v]);
        }
        cudaEventDestroy(ctx->ev_fork);
    }
    for (auto& st : ctx->trace)
        for (auto& pr : st.pending) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    delete ctx;
    return SAD_OK;
}

const char* sad_last_error(void) { return sad::g_err; }

uint64_t sad_launch_count(void) { return sad::g_launches.load(); }

int sad_trace_enable(sad_ctx* ctx_in, int32_t on) {
    sad::clear_error();
    sad_ctx* ctx = nullptr;
    SAD_RET(sad::resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    sad::trace_reset(ctx, on != 0);
    return SAD_OK;
}

int sad_trace_read(sad_ctx* ctx_in, double* ms, int32_t* counts, int32_t nstages) {
    sad::clear_error();
    SAD_CHECK(ms && counts && nstages >= 0, SAD_EINVAL, "invalid arguments");
    sad_ctx* ctx = nullptr;
    SAD_RET(sad::resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    return sad::trace_collect(ctx, ms, counts, nstages);
}

int sad_trace_timeline(sad_ctx* ctx_in, int32_t* stage, double* t0_ms, double* t1_ms, int32_t max_entries,
                       int32_t* n_entries) {
    using namespace sad;
    clear_error();
    SAD_CHECK(n_entries != nullptr, SAD_EINVAL, "n_entries is NULL");
    SAD_CHECK(max_entries >= 0 && (max_entries == 0 || (stage && t0_ms && t1_ms)), SAD_EINVAL,
              "an output pointer is NULL");
    sad_ctx* ctx = nullptr;
    SAD_RET(resolve_ctx(ctx_in, &ctx));
    std::lock_guard<std::mutex> lock(ctx->mu);
    const int32_t n = (int32_t)ctx->timeline.size();
    for (int32_t t = 0; t < n && t < max_entries; t++) {
        stage[t] = ctx->timeline[t].stage;
        t0_ms[t] = ctx->timeline[t].t0;
        t1_ms[t] = ctx->timeline[t].t1;
    }
    *n_entries = n;
    return SAD_OK;
}

const char* sad_version(void) { return "sad-gb300 0.1 (sm_103a)"; }

}  // extern "C"
