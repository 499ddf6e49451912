// Serving Smith-form jobs (the Smith form of Sections 1-2 as a request
// stream): continuous batching of smf_smith_form calls on one GPU.
//
// A server owns `workers` host threads, each with its own context (same device
// and form) and its own non-blocking CUDA stream.  Submitted jobs wait in a
// queue; a free worker takes the first queued job whose estimated device
// footprint fits what is left of the server's budget (a job that does not fit
// waits, later jobs that fit may pass it), so jobs that arrive while others run
// start as workers and memory free up, and their device work overlaps on the
// GPU.  Each job's state (its matrix's digit planes, A^-1 mod p, the lifting
// residuals, the eliminations' matrices) stays on the device for its whole run;
// the driver's scratch is allocated in stream order, so one job's frees never
// stall another job's kernels.  Each job records submit, start and finish
// times on a monotonic host clock.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "smf_internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct SmithJob {
    int64_t n = 0;
    int32_t bits = 0;
    uint64_t seed = 0;
    std::vector<int64_t> A;        // the matrix, copied at submit (row-major n x n)
    size_t bytes = 0;              // estimated device footprint
    int state = SMF_JOB_QUEUED;
    int status = SMF_OK;
    double t[3] = {0, 0, 0};       // submit, start, finish
    std::vector<uint32_t> limbs;   // the invariant factors, as smf_smith_form returns them
    std::vector<int64_t> offsets;
    std::string msg;               // the worker context's last error, for a failed job
};

}  // namespace

struct smf_smith_server {
    int device = 0;
    smf_form form = SMF_FORM_INT8LIMB;
    size_t budget = 0;
    clk::time_point epoch;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;         // job ids in arrival order
    std::deque<SmithJob> jobs;         // stable addresses: workers hold references while jobs are added
    size_t in_use = 0;
    int running = 0;
    bool stop = false;
    std::vector<std::thread> threads;
    std::vector<smf_ctx*> ctxs;
    std::vector<cudaStream_t> streams;
    std::string err;
};

namespace {

double now_s(const smf_smith_server* S) {
    return std::chrono::duration<double>(clk::now() - S->epoch).count();
}

// Device bytes of one smf_smith_form call on an n x n matrix: A as words and
// as digit planes, A^-1 mod p and the Gauss-Jordan scratch (n x 2n words and
// panels), the lifting's residuals and digit planes, and the eliminations'
// matrices (four 32-bit lanes for the determinants): about 64 n^2 bytes, plus a
// fixed part for the small buffers and the bases.
size_t smith_footprint(int64_t n) { return (size_t)64 * n * n + ((size_t)64 << 20); }

// The first queued job that fits what is left of the budget (-1: none).
int64_t admit_one(smf_smith_server* S) {
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        SmithJob& j = S->jobs[*it];
        if (!S->budget || S->in_use + j.bytes <= S->budget) {
            const int64_t id = *it;
            S->queue.erase(it);
            return id;
        }
    }
    return -1;
}

void worker(smf_smith_server* S, int w) {
    smf_ctx* ctx = S->ctxs[w];
    cudaStream_t st = S->streams[w];
    cudaSetDevice(S->device);
    for (;;) {
        int64_t id = -1;
        SmithJob* jp = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || (id = admit_one(S)) >= 0; });
            if (id < 0) return;  // stopping, nothing admitted
            jp = &S->jobs[id];   // the deque keeps this address while jobs are added
            jp->state = SMF_JOB_RUNNING;
            jp->t[1] = now_s(S);
            S->in_use += jp->bytes;
            S->running++;
        }
        SmithJob& j = *jp;  // the job's fields are this worker's until it is marked done
        smf_bigmat A{j.n, j.n, j.n, 1, j.bits, j.A.data(), 0, 0};
        std::vector<int64_t> offsets(j.n + 1);
        int64_t cap = j.n + (int64_t)(j.n * (j.bits + 16)) / 32 + 64;
        std::vector<uint32_t> limbs(cap);
        int rc = smf_smith_form(ctx, &A, j.seed, limbs.data(), cap, offsets.data(), nullptr, nullptr, st);
        if (rc == SMF_E_NOMEM && offsets[j.n] > cap) {
            cap = offsets[j.n];
            limbs.assign(cap, 0);
            rc = smf_smith_form(ctx, &A, j.seed, limbs.data(), cap, offsets.data(), nullptr, nullptr, st);
        }
        if (rc == SMF_OK) limbs.resize(offsets[j.n]);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            j.status = rc;
            if (rc != SMF_OK) j.msg = smf_last_error(ctx);
            j.limbs = std::move(limbs);
            j.offsets = std::move(offsets);
            j.A.clear();
            j.A.shrink_to_fit();
            j.t[2] = now_s(S);
            j.state = rc == SMF_OK ? SMF_JOB_DONE : SMF_JOB_FAILED;
            S->in_use -= j.bytes;
            S->running--;
        }
        S->cv_work.notify_all();  // memory freed: another worker may admit a waiting job
        S->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

int smf_smith_server_create(int device, smf_form form, size_t budget_bytes, int workers, smf_smith_server** out) {
    if (!out || workers < 1 || workers > 64) return SMF_E_INVALID;
    auto* S = new smf_smith_server();
    S->device = device;
    S->form = form;
    S->budget = budget_bytes;
    S->epoch = clk::now();
    int dev0 = 0;
    cudaGetDevice(&dev0);
    for (int w = 0; w < workers; w++) {
        smf_ctx* c = nullptr;
        int rc = smf_create(&c, device, form, 0);
        cudaStream_t st = nullptr;
        if (rc == SMF_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            smf_destroy(c);
            rc = SMF_E_CUDA;
        }
        if (rc != SMF_OK) {
            for (size_t i = 0; i < S->ctxs.size(); i++) {
                cudaStreamDestroy(S->streams[i]);
                smf_destroy(S->ctxs[i]);
            }
            cudaSetDevice(dev0);
            delete S;
            return rc;
        }
        S->ctxs.push_back(c);
        S->streams.push_back(st);
    }
    cudaSetDevice(dev0);
    for (int w = 0; w < workers; w++) S->threads.emplace_back(worker, S, w);
    *out = S;
    return SMF_OK;
}

int smf_smith_server_submit(smf_smith_server* S, const smf_bigmat* A, uint64_t seed, int64_t* job) {
    if (!S || !A || !job) return SMF_E_INVALID;
    if (A->rows != A->cols || A->rows < 1 || A->words != 1 || A->ld < A->cols || !A->data || A->on_device ||
        A->bits < 1)
        return SMF_E_INVALID;  // host matrices with a declared entry bound
    SmithJob j;
    j.n = A->rows;
    j.bits = A->bits;
    j.seed = seed;
    j.bytes = smith_footprint(j.n);
    if (S->budget && j.bytes > S->budget) return SMF_E_NOMEM;
    j.A.resize((size_t)j.n * j.n);
    for (int64_t r = 0; r < j.n; r++)
        std::copy((const int64_t*)A->data + r * A->ld, (const int64_t*)A->data + r * A->ld + j.n,
                  j.A.begin() + r * j.n);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        j.t[0] = now_s(S);
        *job = (int64_t)S->jobs.size();
        S->jobs.push_back(std::move(j));
        S->queue.push_back(*job);
    }
    S->cv_work.notify_one();
    return SMF_OK;
}

int smf_smith_server_job(smf_smith_server* S, int64_t job, int* state, int* status, double times[3]) {
    if (!S) return SMF_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (job < 0 || job >= (int64_t)S->jobs.size()) return SMF_E_INVALID;
    const SmithJob& j = S->jobs[job];
    if (state) *state = j.state;
    if (status) *status = j.status;
    if (times)
        for (int i = 0; i < 3; i++) times[i] = j.t[i];
    return SMF_OK;
}

int smf_smith_server_result(smf_smith_server* S, int64_t job, uint32_t* limbs, int64_t cap, int64_t* offsets) {
    if (!S || !offsets || cap < 0 || (cap > 0 && !limbs)) return SMF_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (job < 0 || job >= (int64_t)S->jobs.size()) return SMF_E_INVALID;
    const SmithJob& j = S->jobs[job];
    if (j.state != SMF_JOB_DONE) return j.state == SMF_JOB_FAILED ? j.status : SMF_E_INVALID;
    std::copy(j.offsets.begin(), j.offsets.end(), offsets);
    if ((int64_t)j.limbs.size() > cap) return SMF_E_NOMEM;
    std::copy(j.limbs.begin(), j.limbs.end(), limbs);
    return SMF_OK;
}

int smf_smith_server_message(smf_smith_server* S, int64_t job, char* buf, int64_t cap) {
    if (!S || !buf || cap < 1) return SMF_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (job < 0 || job >= (int64_t)S->jobs.size()) return SMF_E_INVALID;
    const std::string& m = S->jobs[job].msg;
    const size_t k = std::min(m.size(), (size_t)(cap - 1));
    std::copy(m.begin(), m.begin() + k, buf);
    buf[k] = 0;
    return SMF_OK;
}

int smf_smith_server_stats(smf_smith_server* S, int* queued, int* running, size_t* bytes_in_use) {
    if (!S) return SMF_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = (int)S->queue.size();
    if (running) *running = S->running;
    if (bytes_in_use) *bytes_in_use = S->in_use;
    return SMF_OK;
}

int smf_smith_server_drain(smf_smith_server* S) {
    if (!S) return SMF_E_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->queue.empty() && S->running == 0; });
    return SMF_OK;
}

int smf_smith_server_destroy(smf_smith_server* S) {
    if (!S) return SMF_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->queue.clear();  // jobs not started are dropped
    }
    S->cv_work.notify_all();
    for (auto& t : S->threads) t.join();
    for (size_t i = 0; i < S->ctxs.size(); i++) {
        cudaStreamDestroy(S->streams[i]);
        smf_destroy(S->ctxs[i]);
    }
    delete S;
    return SMF_OK;
}

}  // extern "C"
