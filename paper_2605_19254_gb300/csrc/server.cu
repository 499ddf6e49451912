// Serving loop for exact products: continuous batching over the grouped launch.
//
// Jobs (C = A B, operands on the device) are queued on submit.  Each step
//  1. retires the batches whose completion event has fired,
//  2. admits queued jobs in arrival order while their workspace fits what is
//     left of the HBM budget (a job that does not fit waits, later ones that
//     do may pass it), at most max_batch per step,
//  3. runs the admitted jobs as one smf_rns_matmul_grouped call (one launch
//     per phase over all of them) on one of two server streams, with its
//     workspace from the stream-ordered allocator, freed on that stream after
//     the call, so batches on the two streams overlap on the device.
// Jobs that arrive while batches run are admitted by the next step that finds
// room.  Every job keeps its submit, start and finish times (host clock).
#include <chrono>
#include <deque>
#include <vector>

#include "smf_internal.h"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Job {
    smf_bigmat A, B, C;
    size_t bytes = 0;  // workspace of the job alone (admission estimate)
    int state = SMF_JOB_QUEUED;
    int status = SMF_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
};

struct Batch {
    std::vector<int64_t> jobs;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;
};

}  // namespace

struct smf_server {
    smf_ctx* ctx = nullptr;
    size_t budget = 0, in_use = 0;
    int max_batch = 0;
    cudaStream_t streams[2] = {nullptr, nullptr};
    int next_stream = 0;
    std::vector<Job> jobs;        // indexed by job id
    std::deque<int64_t> queue;    // waiting job ids, arrival order
    std::vector<Batch> running;
};

extern "C" {

int smf_server_admit(size_t budget_left, int n, const size_t* bytes, int max_batch, int* admit) {
    if (n < 0 || max_batch < 0 || (n > 0 && (!bytes || !admit))) return -1;
    int taken = 0;
    size_t left = budget_left;
    for (int i = 0; i < n; i++) {
        admit[i] = 0;
        if (taken < max_batch && bytes[i] <= left) {
            admit[i] = 1;
            left -= bytes[i];
            taken++;
        }
    }
    return taken;
}

int smf_server_create(smf_ctx* ctx, size_t budget_bytes, int max_batch, smf_server** out) {
    if (!ctx || !out || budget_bytes == 0 || max_batch < 1) return SMF_E_INVALID;
    *out = nullptr;
    smf_server* s = new smf_server();
    s->ctx = ctx;
    s->budget = budget_bytes;
    s->max_batch = max_batch;
    cudaSetDevice(ctx->device);
    for (int i = 0; i < 2; i++) {
        if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < i; j++) cudaStreamDestroy(s->streams[j]);
            delete s;
            return SMF_E_CUDA;
        }
    }
    *out = s;
    return SMF_OK;
}

int smf_server_submit(smf_server* s, const smf_bigmat* A, const smf_bigmat* B, smf_bigmat* C, int64_t* job) {
    if (!s || !A || !B || !C || !job) return SMF_E_INVALID;
    size_t bytes = 0;
    const int st = smf_rns_matmul_grouped_workspace(s->ctx, 1, A, B, C, &bytes);
    if (st) return st;
    if (bytes > s->budget) return SMF_E_NOMEM;
    Job j;
    j.A = *A;
    j.B = *B;
    j.C = *C;
    j.bytes = bytes;
    j.t_submit = now_s();
    *job = (int64_t)s->jobs.size();
    s->jobs.push_back(j);
    s->queue.push_back(*job);
    return SMF_OK;
}

// Retire finished batches; then admit and launch one batch.  *launched gets
// the number of jobs started (0 when nothing was waiting or nothing fitted).
int smf_server_step(smf_server* s, int* launched) {
    if (!s) return SMF_E_INVALID;
    if (launched) *launched = 0;
    cudaSetDevice(s->ctx->device);
    // 1. retire
    for (size_t b = 0; b < s->running.size();) {
        Batch& bt = s->running[b];
        const cudaError_t q = cudaEventQuery(bt.done);
        if (q == cudaErrorNotReady) {
            b++;
            continue;
        }
        const double t = now_s();
        for (int64_t id : bt.jobs) {
            Job& j = s->jobs[id];
            j.state = q == cudaSuccess ? SMF_JOB_DONE : SMF_JOB_FAILED;
            if (q != cudaSuccess) j.status = SMF_E_CUDA;
            j.t_done = t;
        }
        if (q != cudaSuccess) cudaGetLastError();
        cudaEventDestroy(bt.done);
        s->in_use -= bt.bytes;
        s->running.erase(s->running.begin() + (long)b);
    }
    if (s->queue.empty()) return SMF_OK;
    // 2. admit by the jobs' own estimates
    std::vector<int64_t> ids(s->queue.begin(), s->queue.end());
    std::vector<size_t> est(ids.size());
    for (size_t i = 0; i < ids.size(); i++) est[i] = s->jobs[ids[i]].bytes;
    std::vector<int> admit(ids.size());
    const size_t left = s->budget - s->in_use;
    if (smf_server_admit(left, (int)ids.size(), est.data(), s->max_batch, admit.data()) <= 0) return SMF_OK;
    std::vector<int64_t> take;
    for (size_t i = 0; i < ids.size(); i++)
        if (admit[i]) take.push_back(ids[i]);
    // the batch's exact workspace (its basis covers the largest bound in it);
    // hand jobs back from the end until it fits
    std::vector<smf_bigmat> As, Bs, Cs;
    size_t bytes = 0;
    for (;;) {
        As.clear();
        Bs.clear();
        Cs.clear();
        for (int64_t id : take) {
            As.push_back(s->jobs[id].A);
            Bs.push_back(s->jobs[id].B);
            Cs.push_back(s->jobs[id].C);
        }
        const int st = smf_rns_matmul_grouped_workspace(s->ctx, (int)take.size(), As.data(), Bs.data(), Cs.data(),
                                                        &bytes);
        if (st) return st;
        if (bytes <= left || take.size() == 1) break;
        take.pop_back();
    }
    if (bytes > left) return SMF_OK;  // the first admitted job alone no longer fits: wait
    // 3. launch
    cudaStream_t st = s->streams[s->next_stream];
    s->next_stream ^= 1;
    void* ws = nullptr;
    if (bytes > 0 && cudaMallocAsync(&ws, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return SMF_OK;  // the pool cannot grow right now: the jobs stay queued
    }
    Batch bt;
    bt.jobs = take;
    bt.bytes = bytes;
    const double t = now_s();
    int rc = smf_rns_matmul_grouped(s->ctx, (int)take.size(), As.data(), Bs.data(), Cs.data(), ws, bytes, st);
    if (ws) cudaFreeAsync(ws, st);
    if (rc == SMF_OK && cudaEventCreateWithFlags(&bt.done, cudaEventDisableTiming) != cudaSuccess) rc = SMF_E_CUDA;
    if (rc == SMF_OK && cudaEventRecord(bt.done, st) != cudaSuccess) rc = SMF_E_CUDA;
    // the launched jobs leave the queue
    std::deque<int64_t> rest;
    for (int64_t id : s->queue) {
        bool in = false;
        for (int64_t k : take) in = in || k == id;
        if (!in) rest.push_back(id);
    }
    s->queue.swap(rest);
    for (int64_t id : take) {
        Job& j = s->jobs[id];
        j.t_start = t;
        j.state = rc == SMF_OK ? SMF_JOB_RUNNING : SMF_JOB_FAILED;
        j.status = rc;
        if (rc != SMF_OK) j.t_done = t;
    }
    if (rc != SMF_OK) {
        if (bt.done) cudaEventDestroy(bt.done);
        return rc;
    }
    s->in_use += bytes;
    s->running.push_back(bt);
    if (launched) *launched = (int)take.size();
    return SMF_OK;
}

int smf_server_job(const smf_server* s, int64_t job, int* state, int* status, double times[3]) {
    if (!s || job < 0 || job >= (int64_t)s->jobs.size()) return SMF_E_INVALID;
    const Job& j = s->jobs[job];
    if (state) *state = j.state;
    if (status) *status = j.status;
    if (times) {
        times[0] = j.t_submit;
        times[1] = j.t_start;
        times[2] = j.t_done;
    }
    return SMF_OK;
}

int smf_server_stats(const smf_server* s, int* queued, int* running_batches, size_t* bytes_in_use) {
    if (!s) return SMF_E_INVALID;
    if (queued) *queued = (int)s->queue.size();
    if (running_batches) *running_batches = (int)s->running.size();
    if (bytes_in_use) *bytes_in_use = s->in_use;
    return SMF_OK;
}

int smf_server_drain(smf_server* s) {
    if (!s) return SMF_E_INVALID;
    for (;;) {
        int n = 0;
        const int rc = smf_server_step(s, &n);
        if (rc) return rc;
        if (s->queue.empty() && s->running.empty()) return SMF_OK;
        if (n == 0 && s->running.empty()) return SMF_E_NOMEM;  // queued jobs, nothing running, nothing launched
        if (n == 0) cudaEventSynchronize(s->running.front().done);
    }
}

int smf_server_destroy(smf_server* s) {
    if (!s) return SMF_OK;
    cudaSetDevice(s->ctx->device);
    for (Batch& b : s->running) {
        cudaEventSynchronize(b.done);
        cudaEventDestroy(b.done);
    }
    for (cudaStream_t st : s->streams)
        if (st) cudaStreamDestroy(st);
    delete s;
    return SMF_OK;
}

}  // extern "C"
