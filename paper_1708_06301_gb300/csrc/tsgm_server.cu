// Serving loop: many camera streams, each sending frames (left/right images and the pose from its
// own odometry) at its own rate; the per-stream state of the method (previous disparity and
// variance maps, Sec. 2.2's D^{k-1}, P^{k-1}) stays on the device between frames.
//
// Continuous batching: a scheduler thread admits a frame as soon as its stream has no frame in
// flight and an execution slot of its image size is free, so frames that arrive while others
// are on the GPU start on their own CUDA stream and overlap with them. Slots (a context with its
// scratch and a CUDA stream) are created per image size as far as the HBM budget allows, at least
// one per size. A slot runs the time step on the stream's own state buffers, so admitting a
// stream moves no maps.

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "tsgm_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    int stream = 0;
    std::vector<uint8_t> left, right;
    float R[9], t[3], K[9];
    float baseline = 0.0f;
    bool has_pose = false;
    float* outD = nullptr;
    float* outP = nullptr;
    Clock::time_point t_submit;
    double latency_ms = 0.0;
    tsgm_status status = TSGM_OK;
    bool done = false;
};

struct SrvStream {
    int W = 0, H = 0, D = 0;
    int cls = 0;  // slot class (image size)
    float* stateD = nullptr;
    float* stateP = nullptr;
    int has_prev = 0;
    bool busy = false;
};

struct Slot {
    tsgm_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    uint8_t* pin_l = nullptr;
    uint8_t* pin_r = nullptr;
    float* pin_D = nullptr;
    float* pin_P = nullptr;
    cudaEvent_t done = nullptr;
    std::shared_ptr<Req> req;
    int cls = 0;
};

}  // namespace

struct tsgm_server {
    std::vector<SrvStream> streams;
    std::vector<Slot> slots;
    std::vector<tsgm_params> cls_params;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> pending;
    std::map<uint64_t, std::shared_ptr<Req>> tickets;
    std::vector<double> latencies;
    uint64_t next_ticket = 1;
    uint64_t completed = 0;
    uint64_t max_in_flight = 0;
    bool stop = false;
    std::thread worker;
    std::string err;
    int device = 0;
};

namespace {

// Enqueue one frame of r on slot s (called by the worker with the lock held).
tsgm_status launch_on(tsgm_server* S, Slot& s, const std::shared_ptr<Req>& r) {
    SrvStream& ss = S->streams[r->stream];
    tsgm_ctx* ctx = s.ctx;
    const size_t n = (size_t)ss.W * ss.H;
    std::memcpy(s.pin_l, r->left.data(), n);
    std::memcpy(s.pin_r, r->right.data(), n);
    cudaError_t e = cudaMemcpyAsync(ctx->d_left, s.pin_l, n, cudaMemcpyHostToDevice, s.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_right, s.pin_r, n, cudaMemcpyHostToDevice, s.st);
    if (e != cudaSuccess) return TSGM_ERR_CUDA;
    // run the step on this stream's own state
    float* keepD = ctx->stateD;
    float* keepP = ctx->stateP;
    ctx->stateD = ss.stateD;
    ctx->stateP = ss.stateP;
    ctx->has_prev = ss.has_prev;
    const tsgm_status st = tsgm_frame(ctx, ctx->d_left, ctx->d_right, r->has_pose ? r->R : nullptr,
                                      r->has_pose ? r->t : nullptr, r->K, r->baseline, ctx->d_outD,
                                      ctx->d_outP);
    ctx->stateD = keepD;
    ctx->stateP = keepP;
    if (st != TSGM_OK) return st;
    ss.has_prev = 1;
    e = cudaMemcpyAsync(s.pin_D, ctx->d_outD, n * sizeof(float), cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s.pin_P, ctx->d_outP, n * sizeof(float), cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess) e = cudaEventRecord(s.done, s.st);
    return e == cudaSuccess ? TSGM_OK : TSGM_ERR_CUDA;
}

void finish(tsgm_server* S, Slot& s, tsgm_status st) {
    std::shared_ptr<Req> r = s.req;
    SrvStream& ss = S->streams[r->stream];
    if (st == TSGM_OK) {
        const size_t n = (size_t)ss.W * ss.H;
        std::memcpy(r->outD, s.pin_D, n * sizeof(float));
        std::memcpy(r->outP, s.pin_P, n * sizeof(float));
    }
    r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
    r->status = st;
    r->done = true;
    S->latencies.push_back(r->latency_ms);
    ++S->completed;
    ss.busy = false;
    s.req.reset();
}

void worker_loop(tsgm_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool progress = false;
        // completions
        for (Slot& s : S->slots) {
            if (!s.req) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            finish(S, s, q == cudaSuccess ? TSGM_OK : TSGM_ERR_CUDA);
            progress = true;
        }
        if (progress) S->cv_done.notify_all();
        // admissions, oldest request first; a stream's frames stay in order
        for (auto it = S->pending.begin(); it != S->pending.end();) {
            std::shared_ptr<Req> r = *it;
            SrvStream& ss = S->streams[r->stream];
            if (ss.busy) {
                ++it;
                continue;
            }
            Slot* free_slot = nullptr;
            for (Slot& s : S->slots)
                if (!s.req && s.cls == ss.cls) {
                    free_slot = &s;
                    break;
                }
            if (!free_slot) {
                ++it;
                continue;
            }
            free_slot->req = r;
            ss.busy = true;
            const tsgm_status st = launch_on(S, *free_slot, r);
            if (st != TSGM_OK) finish(S, *free_slot, st);
            it = S->pending.erase(it);
            progress = true;
        }
        uint64_t in_flight = 0;
        for (Slot& s : S->slots) in_flight += s.req ? 1 : 0;
        S->max_in_flight = std::max<uint64_t>(S->max_in_flight, in_flight);
        if (S->stop && S->pending.empty() && in_flight == 0) break;
        if (!progress) {
            // nothing new: wait for a submission or poll the GPU again shortly
            S->cv_work.wait_for(lk, std::chrono::microseconds(in_flight ? 50 : 2000));
        }
    }
}

}  // namespace

extern "C" {

tsgm_status tsgm_server_create(const tsgm_params* streams, int32_t n_streams,
                               uint64_t hbm_budget_bytes, tsgm_server** out) {
    if (!out) return TSGM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!streams || n_streams < 1) return TSGM_ERR_INVALID_ARG;
    tsgm_server* S = new (std::nothrow) tsgm_server();
    if (!S) return TSGM_ERR_OUT_OF_MEMORY;
    cudaGetDevice(&S->device);
    // slot classes: one per distinct (width, height, d_max) with the first stream's parameters
    std::map<std::tuple<int, int, int>, int> cls_of;
    std::vector<int> cls_count;
    for (int i = 0; i < n_streams; ++i) {
        const tsgm_params& p = streams[i];
        auto key = std::make_tuple(p.width, p.height, p.d_max);
        if (!cls_of.count(key)) {
            cls_of[key] = (int)S->cls_params.size();
            tsgm_params q = p;
            q.flags &= ~(uint32_t)TSGM_FLAG_KEEP_INTERNALS;
            S->cls_params.push_back(q);
            cls_count.push_back(0);
        }
        const int c = cls_of[key];
        ++cls_count[c];
        SrvStream ss;
        ss.W = p.width;
        ss.H = p.height;
        ss.D = p.d_max + 1;
        ss.cls = c;
        const size_t n = (size_t)p.width * p.height;
        if (cudaMalloc((void**)&ss.stateD, n * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&ss.stateP, n * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            S->streams.push_back(ss);
            tsgm_server_destroy(S);
            return TSGM_ERR_OUT_OF_MEMORY;
        }
        S->streams.push_back(ss);
    }
    // bytes of one slot of each class: measured from the free memory a context takes
    auto make_slot = [&](int c) -> bool {
        Slot s;
        s.cls = c;
        const tsgm_params& p = S->cls_params[c];
        const size_t n = (size_t)p.width * p.height;
        if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess) return false;
        if (tsgm_create(&p, s.st, &s.ctx) != TSGM_OK) {
            cudaStreamDestroy(s.st);
            return false;
        }
        if (cudaMallocHost((void**)&s.pin_l, n) != cudaSuccess ||
            cudaMallocHost((void**)&s.pin_r, n) != cudaSuccess ||
            cudaMallocHost((void**)&s.pin_D, n * sizeof(float)) != cudaSuccess ||
            cudaMallocHost((void**)&s.pin_P, n * sizeof(float)) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
            S->slots.push_back(s);
            return false;
        }
        S->slots.push_back(s);
        return true;
    };
    uint64_t used = 0;
    bool ok = true;
    std::vector<uint64_t> cls_bytes(S->cls_params.size(), 0);
    for (size_t c = 0; c < S->cls_params.size() && ok; ++c) {
        size_t f0 = 0, f1 = 0, total = 0;
        cudaMemGetInfo(&f0, &total);
        ok = make_slot((int)c);
        cudaMemGetInfo(&f1, &total);
        cls_bytes[c] = f0 > f1 ? (uint64_t)(f0 - f1) : 1;
        used += cls_bytes[c];
    }
    // more slots, round-robin over the classes in proportion to their streams, within budget
    bool grew = true;
    while (ok && grew) {
        grew = false;
        for (size_t c = 0; c < S->cls_params.size(); ++c) {
            int have = 0;
            for (const Slot& s : S->slots) have += s.cls == (int)c;
            if (have >= cls_count[c]) continue;  // never more slots than streams of the class
            if (used + cls_bytes[c] > hbm_budget_bytes) continue;
            if (!make_slot((int)c)) {
                ok = false;
                break;
            }
            used += cls_bytes[c];
            grew = true;
        }
    }
    if (!ok) {
        cudaGetLastError();
        tsgm_server_destroy(S);
        return TSGM_ERR_OUT_OF_MEMORY;
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return TSGM_OK;
}

void tsgm_server_destroy(tsgm_server* S) {
    if (!S) return;
    if (S->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv_work.notify_all();
        S->worker.join();
    }
    for (Slot& s : S->slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        if (s.ctx) tsgm_destroy(s.ctx);
        if (s.st) cudaStreamDestroy(s.st);
        if (s.pin_l) cudaFreeHost(s.pin_l);
        if (s.pin_r) cudaFreeHost(s.pin_r);
        if (s.pin_D) cudaFreeHost(s.pin_D);
        if (s.pin_P) cudaFreeHost(s.pin_P);
        if (s.done) cudaEventDestroy(s.done);
    }
    for (SrvStream& ss : S->streams) {
        if (ss.stateD) cudaFree(ss.stateD);
        if (ss.stateP) cudaFree(ss.stateP);
    }
    delete S;
}

tsgm_status tsgm_server_submit(tsgm_server* S, int32_t stream, const uint8_t* left_host,
                               const uint8_t* right_host, const float R[9], const float t[3],
                               const float K[9], float baseline, float* D_host, float* P_host,
                               uint64_t* ticket) {
    if (!S || !left_host || !right_host || !K || !D_host || !P_host || !ticket)
        return TSGM_ERR_INVALID_ARG;
    if (stream < 0 || stream >= (int32_t)S->streams.size()) return TSGM_ERR_INVALID_ARG;
    auto r = std::make_shared<Req>();
    const SrvStream& ss = S->streams[stream];
    const size_t n = (size_t)ss.W * ss.H;
    r->stream = stream;
    r->left.assign(left_host, left_host + n);
    r->right.assign(right_host, right_host + n);
    r->has_pose = R && t;
    if (r->has_pose) {
        std::memcpy(r->R, R, sizeof(r->R));
        std::memcpy(r->t, t, sizeof(r->t));
    }
    std::memcpy(r->K, K, sizeof(r->K));
    r->baseline = baseline;
    r->outD = D_host;
    r->outP = P_host;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->ticket = S->next_ticket++;
        S->tickets[r->ticket] = r;
        S->pending.push_back(r);
        *ticket = r->ticket;
    }
    S->cv_work.notify_all();
    return TSGM_OK;
}

tsgm_status tsgm_server_wait(tsgm_server* S, uint64_t ticket, double* latency_ms) {
    if (!S) return TSGM_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return TSGM_ERR_INVALID_ARG;
    std::shared_ptr<Req> r = it->second;
    S->cv_done.wait(lk, [&] { return r->done; });
    if (latency_ms) *latency_ms = r->latency_ms;
    S->tickets.erase(it);
    return r->status;
}

tsgm_status tsgm_server_stats(tsgm_server* S, double* p50_ms, double* p99_ms, uint64_t* completed,
                              int32_t* n_slots, uint64_t* max_in_flight) {
    if (!S) return TSGM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> v = S->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
        return v[k];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (completed) *completed = S->completed;
    if (n_slots) *n_slots = (int32_t)S->slots.size();
    if (max_in_flight) *max_in_flight = S->max_in_flight;
    return TSGM_OK;
}

}  // extern "C"
