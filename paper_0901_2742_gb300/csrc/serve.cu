// Serving loop: a stream of partition-and-score jobs of different sizes,
// admitted by device memory and run concurrently on one GPU.
//
// The server owns `slots` workers; each worker has its own context (cached
// workspaces) and stream. A job waits in a FIFO queue until a worker is free
// and its device-memory estimate fits in what the running jobs leave of the
// budget; the first queued job that fits is taken, so a small job can pass a
// large one that does not fit yet. Jobs on different workers run at the same
// time, their kernels overlapping on the device; every result is bit-identical
// to the same job run alone (all arithmetic is exact integer arithmetic and
// no job reads another's memory). A job larger than the whole budget is
// refused at submission. A job with bad input fails alone with its own error
// code. Cancellation takes effect before the job starts or between its stages.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gotoh_stage.cuh"
#include "kmer_stage.cuh"
#include "partition_stage.cuh"
#include "sad_internal.cuh"

namespace sad {
namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t id = 0;
    std::vector<uint8_t> res;
    std::vector<int64_t> offs;
    int32_t n = 0, alphabet = 0;
    sad_kmer_params kp{};
    std::vector<uint8_t> class_map;
    std::vector<int8_t> subst;
    int32_t go = 0, ge = 0;
    int64_t est = 0;
    int state = SAD_JOB_QUEUED;
    int rc = SAD_OK;
    std::string err;
    std::atomic<bool> cancel{false};
    std::vector<int32_t> bucket_offsets, order, scores;
    std::vector<int64_t> score_offsets;
    Clock::time_point t_submit, t_start, t_done;
    // device interval: events on the worker's stream before the job's first and
    // after its last device operation
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool timed = false;
    ~Job() {
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

}  // namespace
}  // namespace sad

struct sad_server {
    sad_server_config cfg{};
    int64_t budget = 0;
    int64_t reserved = 0;
    std::vector<std::thread> workers;
    std::vector<sad_ctx*> slot_ctx;
    std::vector<cudaStream_t> slot_stream;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<sad::Job>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<sad::Job>> jobs;
    uint64_t next_id = 1;
    bool stopping = false;
    int32_t running = 0;
    int64_t n_done = 0, n_failed = 0, n_cancelled = 0;
    std::vector<double> latencies_ms;
    sad::Clock::time_point t_first_submit, t_last_done;
    bool any_submit = false;
    cudaEvent_t origin = nullptr;  // recorded at creation: zero of the jobs' device intervals
};

namespace sad {
namespace {

int64_t kmer_space(const sad_kmer_params& kp) {
    int64_t V = 1;
    for (int t = 0; t < kp.k; t++) V *= kp.kmer_alphabet;
    return V;
}

// Conservative device bytes of one job: staged and padded residues, counts and
// planes, excess lists, per-sequence tables, partition scratch, and the scores
// of buckets within the regular-sampling bound (each < 2N/p + p members).
int64_t estimate_job_bytes(int32_t n, int64_t total, const sad_kmer_params& kp) {
    const bool sparse = uses_sparse_path(&kp);
    const int64_t Vs = sparse ? 0 : round_up(kmer_space(kp), 64);
    const int64_t rows = round_up(std::max<int32_t>(n, 1), 128);
    const int64_t p = kp.p;
    const int64_t w = 2 * ((int64_t)n + p - 1) / p + p;
    const int64_t score_ints = std::min<int64_t>((int64_t)n * (n + 1) / 2, p * w * (w + 1) / 2);
    int64_t b = 2 * total + 48ll * n + 64 * 1024;         // residues (raw + padded), tables
    b += sparse ? 8 * total : rows * Vs * (1 + kp.cap);     // sorted lists, or counts and planes
    b += 8 * total;                                         // excess lists (upper bound)
    b += 48ll * n + 40 * p * p;                             // partition (up to 16-byte keys)
    b += 12ll * n + 4 * p * kp.global_samples;              // globalized rank
    b += 4 * score_ints + 16ll * n;                         // scores, plan
    b += 8ll * 1024 * 1024;                                 // residual matrix and kernel scratch headroom
    return b;
}

void run_job(sad_server* s, int slot, Job* job) {
    sad_ctx* ctx = s->slot_ctx[slot];
    cudaStream_t stream = s->slot_stream[slot];
    auto fail = [&](int rc) {
        job->rc = rc;
        job->err = sad_last_error();
    };
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaSetDevice failed");
        return fail(SAD_ECUDA);
    }
    clear_error();
    if (cudaEventCreate(&job->ev0) != cudaSuccess || cudaEventCreate(&job->ev1) != cudaSuccess ||
        cudaEventRecord(job->ev0, stream) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaEventCreate/Record failed");
        return fail(SAD_ECUDA);
    }
    int rc = status_clear(ctx, stream);
    if (rc != SAD_OK) return fail(rc);
    sad_seqset ss{job->res.data(), job->offs.data(), job->n, job->alphabet};
    DevSeqs S;
    rc = prepare_seqs(ctx, &ss, SAD_MEM_HOST, stream, &S);
    if (rc != SAD_OK) return fail(rc);
    const int32_t n = job->n, p = job->kp.p;
    const size_t nn = (size_t)std::max<int32_t>(n, 1);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_dloc = carve(8 * nn), o_dcen = carve(8 * nn), o_la = carve(4ull * p), o_ga = carve(16),
                 o_ka = carve(4 * nn), o_kb = carve(4 * nn), o_bo = carve(4ull * (p + 1)),
                 o_ord = carve(4 * nn), o_so = carve(8ull * (p + 1));
    const int32_t gs = job->kp.global_samples;
    const size_t o_G = carve(gs > 0 ? 8 * nn : 0), o_smp = carve(4ull * p * gs);
    void* w = nullptr;
    rc = workspace(ctx, WS_PIPE, off, stream, &w);
    if (rc != SAD_OK) return fail(rc);
    char* c = (char*)w;
    KmerOutDev d{(uint64_t*)(c + o_dloc), (uint64_t*)(c + o_dcen), (int32_t*)(c + o_la), (int32_t*)(c + o_ga),
                 (int32_t*)(c + o_ka),     (int32_t*)(c + o_kb),   nullptr};
    int32_t* dbo = (int32_t*)(c + o_bo);
    int32_t* dord = (int32_t*)(c + o_ord);
    int64_t* dso = (int64_t*)(c + o_so);
    if (gs > 0) {
        d.G = (uint64_t*)(c + o_G);
        d.samples = (int32_t*)(c + o_smp);
    }
    sad_kmer_params kp = job->kp;
    kp.class_map = job->class_map.empty() ? nullptr : job->class_map.data();
    rc = kmer_rank_device(ctx, S, &kp, d, stream);
    if (rc != SAD_OK) return fail(rc);
    if (job->cancel.load()) return fail(SAD_ECANCELED);
    rc = gs > 0 ? partition_keys64_device(ctx, n, d.G, p, dbo, dord, nullptr, stream)
                : partition_device(ctx, n, d.key_a, d.key_b, p, dbo, dord, nullptr, stream);
    if (rc != SAD_OK) return fail(rc);
    job->bucket_offsets.assign((size_t)p + 1, 0);
    if (cudaMemcpyAsync(job->bucket_offsets.data(), dbo, 4ull * (p + 1), cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        set_error("copy of the bucket layout failed");
        return fail(SAD_ECUDA);
    }
    if (job->cancel.load()) return fail(SAD_ECANCELED);
    int64_t total = 0;
    for (int32_t b = 0; b < p; b++) {
        const int64_t nb = job->bucket_offsets[b + 1] - job->bucket_offsets[b];
        total += nb * (nb + 1) / 2;
    }
    void* sw = nullptr;
    rc = workspace(ctx, WS_SCORE_OUT, 4ull * (total + 1), stream, &sw);
    if (rc != SAD_OK) return fail(rc);
    rc = bucket_scores_device(ctx, S, dbo, dord, p, job->subst.data(), job->go, job->ge, SAD_SCORES_PERSISTENT,
                              dso, (int32_t*)sw, total, &total, stream);
    if (rc != SAD_OK) return fail(rc);
    job->order.assign(nn, 0);
    job->score_offsets.assign((size_t)p + 1, 0);
    job->scores.assign((size_t)std::max<int64_t>(total, 1), 0);
    bool ok = cudaMemcpyAsync(job->order.data(), dord, 4ull * n, cudaMemcpyDeviceToHost, stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(job->score_offsets.data(), dso, 8ull * (p + 1), cudaMemcpyDeviceToHost,
                               stream) == cudaSuccess;
    ok = ok && (total == 0 || cudaMemcpyAsync(job->scores.data(), sw, 4ull * total, cudaMemcpyDeviceToHost,
                                              stream) == cudaSuccess);
    if (!ok) {
        cudaGetLastError();
        set_error("copy of the job results failed");
        return fail(SAD_ECUDA);
    }
    job->scores.resize((size_t)total);
    job->order.resize((size_t)n);
    job->timed = cudaEventRecord(job->ev1, stream) == cudaSuccess;
    cudaGetLastError();
    rc = status_check(ctx, stream);
    if (rc != SAD_OK) return fail(rc);
    job->rc = SAD_OK;
}

void worker_main(sad_server* s, int slot) {
    for (;;) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            for (;;) {
                if (s->stopping) return;
                // the first queued job that fits in the budget left
                auto it = std::find_if(s->queue.begin(), s->queue.end(), [&](const std::shared_ptr<Job>& j) {
                    return s->reserved + j->est <= s->budget;
                });
                if (it != s->queue.end()) {
                    job = *it;
                    s->queue.erase(it);
                    break;
                }
                s->cv_work.wait(lock);
            }
            s->reserved += job->est;
            s->running++;
            job->state = SAD_JOB_RUNNING;
            job->t_start = Clock::now();
        }
        if (job->cancel.load()) {
            job->rc = SAD_ECANCELED;
        } else {
            run_job(s, slot, job.get());
        }
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->reserved -= job->est;
            s->running--;
            job->t_done = Clock::now();
            s->t_last_done = job->t_done;
            if (job->rc == SAD_OK) {
                job->state = SAD_JOB_DONE;
                s->n_done++;
                s->latencies_ms.push_back(
                    std::chrono::duration<double, std::milli>(job->t_done - job->t_submit).count());
            } else if (job->rc == SAD_ECANCELED) {
                job->state = SAD_JOB_CANCELLED;
                s->n_cancelled++;
            } else {
                job->state = SAD_JOB_FAILED;
                s->n_failed++;
            }
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (v[hi] - v[lo]) * (pos - lo);
}

}  // namespace
}  // namespace sad

extern "C" {

int sad_server_create(const sad_server_config* cfg, sad_server** out) {
    using namespace sad;
    clear_error();
    SAD_CHECK(cfg && out, SAD_EINVAL, "NULL argument");
    SAD_CHECK(cfg->slots >= 1 && cfg->slots <= 64, SAD_EINVAL, "slots = %d outside 1..64", cfg->slots);
    SAD_CHECK(cfg->queue_capacity >= 1, SAD_EINVAL, "queue_capacity = %d < 1", cfg->queue_capacity);
    SAD_CHECK(cfg->hbm_budget >= 0, SAD_EINVAL, "hbm_budget < 0");
    SAD_CUDA(cudaSetDevice(cfg->device));
    auto* s = new sad_server();
    s->cfg = *cfg;
    if (cfg->hbm_budget > 0) {
        s->budget = cfg->hbm_budget;
    } else {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            set_error("cudaMemGetInfo failed");
            return SAD_ECUDA;
        }
        s->budget = (int64_t)(0.9 * (double)fr);
    }
    for (int i = 0; i < cfg->slots; i++) {
        sad_ctx* c = nullptr;
        int rc = sad_ctx_create(cfg->device, &c);
        cudaStream_t st = nullptr;
        if (rc == SAD_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            rc = SAD_ECUDA;
        }
        if (rc != SAD_OK) {
            for (size_t q = 0; q < s->slot_ctx.size(); q++) {
                cudaStreamDestroy(s->slot_stream[q]);
                sad_ctx_destroy(s->slot_ctx[q]);
            }
            if (c) sad_ctx_destroy(c);
            delete s;
            return rc;
        }
        s->slot_ctx.push_back(c);
        s->slot_stream.push_back(st);
    }
    if (cudaEventCreate(&s->origin) != cudaSuccess || cudaEventRecord(s->origin, s->slot_stream[0]) != cudaSuccess ||
        cudaEventSynchronize(s->origin) != cudaSuccess) {
        cudaGetLastError();
        if (s->origin) cudaEventDestroy(s->origin);
        for (size_t q = 0; q < s->slot_ctx.size(); q++) {
            cudaStreamDestroy(s->slot_stream[q]);
            sad_ctx_destroy(s->slot_ctx[q]);
        }
        delete s;
        set_error("cudaEventCreate/Record of the server origin failed");
        return SAD_ECUDA;
    }
    for (int i = 0; i < cfg->slots; i++) s->workers.emplace_back(worker_main, s, i);
    *out = s;
    return SAD_OK;
}

int sad_server_submit(sad_server* s, const sad_job* job, uint64_t* job_id) {
    using namespace sad;
    clear_error();
    SAD_CHECK(s && job && job_id, SAD_EINVAL, "NULL argument");
    SAD_CHECK(job->n >= 0, SAD_EINVAL, "n = %d < 0", job->n);
    SAD_CHECK(job->offsets && (job->n == 0 || job->residues), SAD_EINVAL, "sequence pointers are NULL");
    SAD_CHECK(job->subst, SAD_EINVAL, "subst is NULL");
    sad_seqset ss{job->residues, job->offsets, job->n, job->alphabet};
    SAD_RET(validate_kmer_params(&ss, &job->kmer));
    SAD_CHECK(job->kmer.p <= kMaxPartitionP, SAD_EINVAL, "p = %d > %d", job->kmer.p, kMaxPartitionP);
    SAD_CHECK(job->gap_open <= 0 && job->gap_extend <= 0, SAD_EINVAL, "gap costs must be <= 0");
    const int32_t A = job->alphabet;
    for (int32_t x = 0; x < A; x++)
        for (int32_t y = 0; y < A; y++)
            SAD_CHECK(job->subst[x * A + y] == job->subst[y * A + x], SAD_EINVAL,
                      "substitution matrix is not symmetric at (%d, %d)", x, y);
    SAD_CHECK(job->offsets[0] == 0, SAD_EINVAL, "offsets[0] must be 0");
    for (int32_t i = 0; i < job->n; i++)
        SAD_CHECK(job->offsets[i + 1] >= job->offsets[i], SAD_EINVAL, "offsets decrease at %d", i);
    auto j = std::make_shared<Job>();
    const int64_t total = job->offsets[job->n];
    j->res.assign(job->residues, job->residues + total);
    j->offs.assign(job->offsets, job->offsets + job->n + 1);
    j->n = job->n;
    j->alphabet = A;
    j->kp = job->kmer;
    if (job->kmer.class_map) j->class_map.assign(job->kmer.class_map, job->kmer.class_map + A);
    j->subst.assign(job->subst, job->subst + (size_t)A * A);
    j->go = job->gap_open;
    j->ge = job->gap_extend;
    j->est = estimate_job_bytes(job->n, total, job->kmer);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        SAD_CHECK(j->est <= s->budget, SAD_ENOMEM,
                  "job needs about %lld bytes of device memory, more than the server budget %lld",
                  (long long)j->est, (long long)s->budget);
        SAD_CHECK((int32_t)s->queue.size() < s->cfg.queue_capacity, SAD_EBUSY, "the queue is full (%d jobs)",
                  s->cfg.queue_capacity);
        j->id = s->next_id++;
        j->t_submit = Clock::now();
        if (!s->any_submit) {
            s->any_submit = true;
            s->t_first_submit = j->t_submit;
        }
        s->jobs[j->id] = j;
        s->queue.push_back(j);
        *job_id = j->id;
    }
    s->cv_work.notify_one();
    return SAD_OK;
}

int sad_server_poll(sad_server* s, uint64_t job_id, int32_t* state) {
    using namespace sad;
    clear_error();
    SAD_CHECK(s && state, SAD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    SAD_CHECK(it != s->jobs.end(), SAD_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    *state = it->second->state;
    if (it->second->state == SAD_JOB_FAILED) {
        set_error("%s", it->second->err.c_str());
        return it->second->rc;
    }
    return SAD_OK;
}

int sad_server_wait(sad_server* s, uint64_t job_id, int64_t timeout_ms) {
    using namespace sad;
    clear_error();
    SAD_CHECK(s, SAD_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    SAD_CHECK(it != s->jobs.end(), SAD_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    std::shared_ptr<Job> j = it->second;
    auto finished = [&] {
        return j->state == SAD_JOB_DONE || j->state == SAD_JOB_FAILED || j->state == SAD_JOB_CANCELLED;
    };
    if (timeout_ms < 0) {
        s->cv_done.wait(lock, finished);
    } else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), finished)) {
        set_error("job %llu still %s after %lld ms", (unsigned long long)job_id,
                  j->state == SAD_JOB_QUEUED ? "queued" : "running", (long long)timeout_ms);
        return SAD_EBUSY;
    }
    if (j->state == SAD_JOB_CANCELLED) {
        set_error("job %llu was cancelled", (unsigned long long)job_id);
        return SAD_ECANCELED;
    }
    if (j->state == SAD_JOB_FAILED) {
        set_error("%s", j->err.c_str());
        return j->rc;
    }
    return SAD_OK;
}

int sad_server_result(sad_server* s, uint64_t job_id, int32_t* bucket_offsets, int32_t* order,
                      int64_t* score_offsets, int32_t* scores, int64_t capacity, int64_t* n_scores,
                      double* latency_ms) {
    using namespace sad;
    clear_error();
    SAD_CHECK(s && n_scores, SAD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    SAD_CHECK(it != s->jobs.end(), SAD_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    Job* j = it->second.get();
    SAD_CHECK(j->state == SAD_JOB_DONE, SAD_EBUSY, "job %llu has no result (state %d)",
              (unsigned long long)job_id, j->state);
    *n_scores = (int64_t)j->scores.size();
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
    SAD_CHECK(capacity >= (int64_t)j->scores.size(), SAD_ERANGE, "scores need %lld entries, capacity %lld",
              (long long)j->scores.size(), (long long)capacity);
    const int32_t p = j->kp.p;
    if (bucket_offsets) memcpy(bucket_offsets, j->bucket_offsets.data(), 4ull * (p + 1));
    if (order) memcpy(order, j->order.data(), 4ull * j->n);
    if (score_offsets) memcpy(score_offsets, j->score_offsets.data(), 8ull * (p + 1));
    if (scores && !j->scores.empty()) memcpy(scores, j->scores.data(), 4ull * j->scores.size());
    return SAD_OK;
}

int sad_server_release(sad_server* s, uint64_t job_id) {
    using namespace sad;
    clear_error();
    SAD_CHECK(s, SAD_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    SAD_CHECK(it != s->jobs.end(), SAD_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    const int st = it->second->state;
    SAD_CHECK(st == SAD_JOB_DONE || st == SAD_JOB_FAILED || st == SAD_JOB_CANCELLED, SAD_EBUSY,
              "job %llu is still queued or running", (unsigned long long)job_id);
    s->jobs.erase(it);
    return SAD_OK;
}

int sad_server_cancel(sad_server* s, uint64_t job_id) {
    using namespace sad;
    clear_error();
    SAD_CHECK(s, SAD_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    SAD_CHECK(it != s->jobs.end(), SAD_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    std::shared_ptr<Job> j = it->second;
    j->cancel.store(true);
    auto q = std::find(s->queue.begin(), s->queue.end(), j);
    if (q != s->queue.end()) {
        s->queue.erase(q);
        j->state = SAD_JOB_CANCELLED;
        j->rc = SAD_ECANCELED;
        j->t_done = Clock::now();
        s->n_cancelled++;
        s->cv_done.notify_all();
    }
    return SAD_OK;
}

int sad_server_job_span(sad_server* s, uint64_t job_id, double* t0_ms, double* t1_ms) {
    using namespace sad;
    clear_error();
    SAD_CHECK(s && t0_ms && t1_ms, SAD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    SAD_CHECK(it != s->jobs.end(), SAD_ENOTFOUND, "unknown job %llu", (unsigned long long)job_id);
    Job* j = it->second.get();
    SAD_CHECK(j->state == SAD_JOB_DONE && j->timed, SAD_EBUSY, "job %llu has no device interval (state %d)",
              (unsigned long long)job_id, j->state);
    float a = 0, b = 0;
    SAD_CUDA(cudaEventElapsedTime(&a, s->origin, j->ev0));
    SAD_CUDA(cudaEventElapsedTime(&b, s->origin, j->ev1));
    *t0_ms = a;
    *t1_ms = b;
    return SAD_OK;
}

int sad_server_get_stats(sad_server* s, sad_server_stats* out) {
    using namespace sad;
    clear_error();
    SAD_CHECK(s && out, SAD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    out->done = s->n_done;
    out->failed = s->n_failed;
    out->cancelled = s->n_cancelled;
    out->queued = (int64_t)s->queue.size();
    out->running = s->running;
    out->p50_ms = percentile(s->latencies_ms, 0.50);
    out->p99_ms = percentile(s->latencies_ms, 0.99);
    out->mean_ms = 0;
    for (double v : s->latencies_ms) out->mean_ms += v;
    if (!s->latencies_ms.empty()) out->mean_ms /= (double)s->latencies_ms.size();
    const double span = s->any_submit && s->n_done
                            ? std::chrono::duration<double>(s->t_last_done - s->t_first_submit).count()
                            : 0.0;
    out->jobs_per_s = span > 0 ? (double)s->n_done / span : 0.0;
    out->budget_bytes = s->budget;
    out->reserved_bytes = s->reserved;
    return SAD_OK;
}

int sad_server_destroy(sad_server* s) {
    using namespace sad;
    clear_error();
    if (!s) return SAD_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
        for (auto& j : s->queue) {
            j->state = SAD_JOB_CANCELLED;
            j->rc = SAD_ECANCELED;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    s->queue.clear();
    s->jobs.clear();  // the jobs' events go before their streams
    for (size_t q = 0; q < s->slot_ctx.size(); q++) {
        cudaStreamDestroy(s->slot_stream[q]);
        sad_ctx_destroy(s->slot_ctx[q]);
    }
    if (s->origin) cudaEventDestroy(s->origin);
    delete s;
    return SAD_OK;
}

}  // extern "C"
