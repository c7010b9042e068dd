// Serving loop: many camera streams, each sending frames (left/right images and the pose from its
// own odometry) at its own rate; the per-stream state of the method (previous disparity and
// variance maps, Sec. 2.2's D^{k-1}, P^{k-1}) stays on the device between frames.
//
// Continuous batching on the batched time step: one batch (tsgm_batch) holds every stream's
// state, scratch and a shared volume pool sized by the HBM budget. A scheduler thread runs ticks:
// each tick takes the oldest waiting frame of every stream that has one, copies their images in,
// runs ONE replay of the batched time-step graph over those streams (the others sit the tick
// out) and copies the results out. Frames that arrive while a tick runs go into the next one.
// A stream whose windows do not fit the pool cells left in a tick is refused by the step with
// its state untouched and its frame stays first in line (refused streams are served first next
// tick), so the budget bounds memory without dropping frames.
//
// Ticks are pipelined: images and results live in two device buffers per stream used in turn,
// so a tick's results go back to pinned memory on a copy stream while the next tick computes,
// and helper threads copy them into the callers' arrays meanwhile; the scheduler only waits for
// a tick's compute (to learn which streams the pool refused) before it starts the next.

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
#include <vector>

#include "tsgm_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kPinnedInputs = 3;  // pinned image buffers per stream (frames waiting at once)
constexpr int kCopyThreads = 4;

struct Req {
    uint64_t ticket = 0;
    int stream = 0;
    uint8_t* img = nullptr;     // left then right, pinned (from the stream's free list) or heap
    bool img_pinned = false;
    std::vector<uint8_t> heap;  // images when no pinned buffer was free
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
    int W = 0, H = 0;
    size_t n = 0;
    std::deque<std::shared_ptr<Req>> queue;  // waiting frames, in submission order
    std::vector<uint8_t*> free_img;           // pinned image buffers not in use
    std::vector<uint8_t*> all_img;
    bool ran = false;                         // a frame of this stream has run (it has a state)
    uint8_t* d_img[2] = {nullptr, nullptr};   // device left, right of even / odd ticks
    float* d_out[2] = {nullptr, nullptr};     // device D, P of even / odd ticks
    float* pin_out[2] = {nullptr, nullptr};   // pinned D, P of even / odd ticks
};

struct CopyTask {
    std::shared_ptr<Req> r;
    const float* src = nullptr;  // pinned D then P
    size_t n = 0;
    int parity = 0;
    cudaEvent_t ready = nullptr;  // the copy into src has finished
};

}  // namespace

struct tsgm_server {
    tsgm_batch* batch = nullptr;
    std::vector<SrvStream> streams;
    cudaStream_t st = nullptr;      // the batch's steps
    cudaStream_t s_in = nullptr;    // images in
    cudaStream_t s_out = nullptr;   // results out
    cudaEvent_t e_in[2] = {nullptr, nullptr}, e_done[2] = {nullptr, nullptr},
                e_out[2] = {nullptr, nullptr};
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_copy;
    std::map<uint64_t, std::shared_ptr<Req>> tickets;
    std::vector<double> latencies;
    uint64_t next_ticket = 1;
    uint64_t completed = 0;
    uint64_t max_in_flight = 0;
    int32_t slots = 0;
    bool stop = false;
    std::thread worker;
    std::vector<std::thread> copiers;
    std::deque<CopyTask> copy_q;
    int copies_pending[2] = {0, 0};
    bool copy_stop = false;
    int device = 0;  // the CUDA device of the server (its threads work on it)
};

namespace {

// Complete a request (lock held).
void finish_locked(tsgm_server* S, const std::shared_ptr<Req>& r, tsgm_status st) {
    r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
    r->status = st;
    r->done = true;
    S->latencies.push_back(r->latency_ms);
    ++S->completed;
    SrvStream& ss = S->streams[r->stream];
    if (r->img_pinned) ss.free_img.push_back(r->img);
    r->img = nullptr;
    r->img_pinned = false;
    r->heap.clear();
    r->heap.shrink_to_fit();
}

void copier_loop(tsgm_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_copy.wait(lk, [&] { return S->copy_stop || !S->copy_q.empty(); });
        if (S->copy_q.empty()) return;  // stop requested and nothing left
        CopyTask t = S->copy_q.front();
        S->copy_q.pop_front();
        lk.unlock();
        const bool ok = cudaEventSynchronize(t.ready) == cudaSuccess;
        if (ok) {
            std::memcpy(t.r->outD, t.src, t.n * sizeof(float));
            std::memcpy(t.r->outP, t.src + t.n, t.n * sizeof(float));
        }
        lk.lock();
        finish_locked(S, t.r, ok ? TSGM_OK : TSGM_ERR_CUDA);
        --S->copies_pending[t.parity];
        S->cv_done.notify_all();
        S->cv_copy.notify_all();
    }
}

bool any_waiting(const tsgm_server* S) {
    for (const SrvStream& ss : S->streams)
        if (!ss.queue.empty()) return true;
    return false;
}

void worker_loop(tsgm_server* S) {
    const int ns = (int)S->streams.size();
    std::vector<const uint8_t*> L(ns), Rimg(ns);
    std::vector<float*> Dp(ns), Pp(ns);
    std::vector<float> Rm(9 * ns), tv(3 * ns), Km(9 * ns), bl(ns);
    std::vector<std::shared_ptr<Req>> tick(ns);
    std::vector<int32_t> status(ns);
    static const float kEye[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    int parity = 0;
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_work.wait(lk, [&] { return S->stop || any_waiting(S); });
        if (!any_waiting(S)) break;  // stop requested and every frame is done
        // the oldest waiting frame of every stream; frames that cannot run are refused alone
        int n_tick = 0;
        for (int i = 0; i < ns; ++i) {
            SrvStream& ss = S->streams[i];
            tick[i].reset();
            while (!ss.queue.empty()) {
                std::shared_ptr<Req> r = ss.queue.front();
                float H[16];
                const bool ok = !ss.ran || (r->has_pose && tsgm_build_H(r->R, r->t, r->K,
                                                                       r->baseline, H) == TSGM_OK);
                if (ok) {
                    tick[i] = r;
                    ++n_tick;
                    break;
                }
                ss.queue.pop_front();
                finish_locked(S, r, TSGM_ERR_INVALID_ARG);
                S->cv_done.notify_all();
            }
        }
        if (n_tick == 0) continue;
        // the pinned result buffers of this parity were handed to the copiers two ticks ago
        S->cv_copy.wait(lk, [&] { return S->copies_pending[parity] == 0; });
        lk.unlock();
        // images in (on the input stream), then the step after them and after the copy out of
        // the results this tick's buffers held two ticks ago
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < ns; ++i) {
            SrvStream& ss = S->streams[i];
            const std::shared_ptr<Req>& r = tick[i];
            L[i] = Rimg[i] = nullptr;
            Dp[i] = Pp[i] = nullptr;
            if (!r) continue;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(ss.d_img[parity], r->img, 2 * ss.n, cudaMemcpyHostToDevice,
                                    S->s_in);
            L[i] = ss.d_img[parity];
            Rimg[i] = ss.d_img[parity] + ss.n;
            Dp[i] = ss.d_out[parity];
            Pp[i] = ss.d_out[parity] + ss.n;
            // a stream without a state does not read its pose: identity, valid intrinsics
            const bool warp = ss.ran;
            std::memcpy(&Rm[9 * i], warp ? r->R : kEye, 9 * sizeof(float));
            for (int k = 0; k < 3; ++k) tv[3 * i + k] = warp ? r->t[k] : 0.0f;
            std::memcpy(&Km[9 * i], warp ? r->K : kEye, 9 * sizeof(float));
            bl[i] = warp ? r->baseline : 1.0f;
        }
        if (e == cudaSuccess) e = cudaEventRecord(S->e_in[parity], S->s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(S->st, S->e_in[parity], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(S->st, S->e_out[parity], 0);
        tsgm_status fst = e == cudaSuccess ? TSGM_OK : TSGM_ERR_CUDA;
        if (fst == TSGM_OK)
            fst = tsgm_batch_frame(S->batch, L.data(), Rimg.data(), Rm.data(), tv.data(), Km.data(),
                                   bl.data(), Dp.data(), Pp.data());
        if (fst == TSGM_OK &&
            (cudaEventRecord(S->e_done[parity], S->st) != cudaSuccess ||
             cudaEventSynchronize(S->e_done[parity]) != cudaSuccess))
            fst = TSGM_ERR_CUDA;
        if (fst == TSGM_OK) fst = tsgm_batch_stream_status(S->batch, status.data());
        // results of the streams that ran back to pinned memory, beside the next tick
        if (fst == TSGM_OK && cudaStreamWaitEvent(S->s_out, S->e_done[parity], 0) != cudaSuccess)
            fst = TSGM_ERR_CUDA;
        for (int i = 0; i < ns && fst == TSGM_OK; ++i) {
            if (!tick[i] || status[i] != 0) continue;
            SrvStream& ss = S->streams[i];
            if (cudaMemcpyAsync(ss.pin_out[parity], ss.d_out[parity], 2 * ss.n * sizeof(float),
                                cudaMemcpyDeviceToHost, S->s_out) != cudaSuccess)
                fst = TSGM_ERR_CUDA;
        }
        if (fst == TSGM_OK && cudaEventRecord(S->e_out[parity], S->s_out) != cudaSuccess)
            fst = TSGM_ERR_CUDA;
        lk.lock();
        int ran = 0;
        for (int i = 0; i < ns; ++i) {
            if (!tick[i]) continue;
            SrvStream& ss = S->streams[i];
            if (fst != TSGM_OK) {  // the whole tick failed: its frames fail
                ss.queue.pop_front();
                finish_locked(S, tick[i], fst);
                continue;
            }
            if (status[i] != 0) continue;  // refused by the pool: first in line next tick
            ss.queue.pop_front();
            ss.ran = true;
            ++ran;
            S->copy_q.push_back(CopyTask{tick[i], ss.pin_out[parity], ss.n, parity, S->e_out[parity]});
            ++S->copies_pending[parity];
        }
        S->max_in_flight = std::max<uint64_t>(S->max_in_flight, (uint64_t)ran);
        S->cv_copy.notify_all();
        S->cv_done.notify_all();
        parity ^= 1;
    }
}

void release(tsgm_server* S) {
    for (cudaStream_t q : {S->st, S->s_in, S->s_out})
        if (q) cudaStreamSynchronize(q);
    if (S->batch) tsgm_batch_destroy(S->batch);
    for (SrvStream& ss : S->streams) {
        for (uint8_t* p : ss.all_img) cudaFreeHost(p);
        for (int b = 0; b < 2; ++b) {
            if (ss.pin_out[b]) cudaFreeHost(ss.pin_out[b]);
            if (ss.d_img[b]) cudaFree(ss.d_img[b]);
            if (ss.d_out[b]) cudaFree(ss.d_out[b]);
        }
    }
    for (int b = 0; b < 2; ++b)
        for (cudaEvent_t ev : {S->e_in[b], S->e_done[b], S->e_out[b]})
            if (ev) cudaEventDestroy(ev);
    for (cudaStream_t q : {S->st, S->s_in, S->s_out})
        if (q) cudaStreamDestroy(q);
    delete S;
}

}  // namespace

extern "C" {

tsgm_status tsgm_server_create(const tsgm_params* streams, int32_t n_streams,
                               uint64_t hbm_budget_bytes, tsgm_server** out) {
    if (!out) return TSGM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!streams || n_streams < 1) return TSGM_ERR_INVALID_ARG;
    // one batched time step serves every stream: one prediction and window rule for all
    for (int i = 0; i < n_streams; ++i) {
        const tsgm_params& p = streams[i];
        if (p.flags & (TSGM_FLAG_EDGE_REJECT | TSGM_FLAG_PRED_LR_CHECK | TSGM_FLAG_SAD_CHECK))
            return TSGM_ERR_UNIMPLEMENTED;
        if (((p.flags ^ streams[0].flags) & ~(uint32_t)TSGM_FLAG_KEEP_INTERNALS) ||
            p.gamma_f != streams[0].gamma_f || p.sigma_mult != streams[0].sigma_mult ||
            !(p.q >= 0.0f && p.q <= 3.0e38f) || !(p.sigma_mult >= 0.0f && p.sigma_mult <= 3.0e38f))
            return TSGM_ERR_INVALID_ARG;
    }
    tsgm_server* S = new (std::nothrow) tsgm_server();
    if (!S) return TSGM_ERR_OUT_OF_MEMORY;
    cudaGetDevice(&S->device);
    std::vector<tsgm_params> prm(streams, streams + n_streams);
    for (tsgm_params& p : prm) p.flags &= ~(uint32_t)TSGM_FLAG_KEEP_INTERNALS;
    size_t f0 = 0, f1 = 0, total = 0;
    cudaMemGetInfo(&f0, &total);
    bool ok = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&S->s_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&S->s_out, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaEventCreateWithFlags(&S->e_in[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&S->e_done[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&S->e_out[b], cudaEventDisableTiming) == cudaSuccess &&
             // recorded once, so that the first ticks' waits on them are satisfied
             cudaEventRecord(S->e_out[b], S->s_out) == cudaSuccess;
    S->streams.resize((size_t)n_streams);
    for (int i = 0; i < n_streams && ok; ++i) {
        SrvStream& ss = S->streams[i];
        ss.W = prm[i].width;
        ss.H = prm[i].height;
        ss.n = (size_t)ss.W * ss.H;
        for (int b = 0; b < 2 && ok; ++b)
            ok = cudaMalloc((void**)&ss.d_img[b], 2 * ss.n) == cudaSuccess &&
                 cudaMalloc((void**)&ss.d_out[b], 2 * ss.n * sizeof(float)) == cudaSuccess &&
                 cudaMallocHost((void**)&ss.pin_out[b], 2 * ss.n * sizeof(float)) == cudaSuccess;
        for (int k = 0; k < kPinnedInputs && ok; ++k) {
            uint8_t* p = nullptr;
            ok = cudaMallocHost((void**)&p, 2 * ss.n) == cudaSuccess;
            if (ok) {
                ss.all_img.push_back(p);
                ss.free_img.push_back(p);
            }
        }
    }
    tsgm_status st = TSGM_OK;
    if (ok) {
        cudaMemGetInfo(&f1, &total);
        const uint64_t used = f0 > f1 ? (uint64_t)(f0 - f1) : 0;
        const uint64_t left = hbm_budget_bytes > used ? hbm_budget_bytes - used : 1;
        st = tsgm::batch_create(prm.data(), n_streams, 0, left, S->st, &S->batch);
        ok = st == TSGM_OK;
    }
    if (ok) {
        // streams whose full-range step fits the pool at once (in stream order)
        uint64_t pool = 0, largest = 0, used = 0;
        tsgm_batch_pool(S->batch, &pool, &largest);
        for (int i = 0; i < n_streams; ++i) {
            const uint64_t need =
                ((uint64_t)prm[i].width * prm[i].height * (uint64_t)((prm[i].d_max + 4) & ~3) + 255) &
                ~255ull;
            if (need <= pool - used) {
                used += need;
                ++S->slots;
            }
        }
    }
    if (!ok) {
        cudaGetLastError();
        release(S);
        return st == TSGM_ERR_INVALID_ARG ? TSGM_ERR_INVALID_ARG : TSGM_ERR_OUT_OF_MEMORY;
    }
    for (int k = 0; k < kCopyThreads; ++k) S->copiers.emplace_back(copier_loop, S);
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
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->copy_stop = true;
    }
    S->cv_copy.notify_all();
    for (std::thread& t : S->copiers)
        if (t.joinable()) t.join();
    release(S);
}

tsgm_status tsgm_server_submit(tsgm_server* S, int32_t stream, const uint8_t* left_host,
                               const uint8_t* right_host, const float R[9], const float t[3],
                               const float K[9], float baseline, float* D_host, float* P_host,
                               uint64_t* ticket) {
    if (!S || !left_host || !right_host || !K || !D_host || !P_host || !ticket)
        return TSGM_ERR_INVALID_ARG;
    if (stream < 0 || stream >= (int32_t)S->streams.size()) return TSGM_ERR_INVALID_ARG;
    auto r = std::make_shared<Req>();
    SrvStream& ss = S->streams[stream];
    const size_t n = ss.n;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!ss.free_img.empty()) {
            r->img = ss.free_img.back();
            ss.free_img.pop_back();
            r->img_pinned = true;
        }
    }
    if (!r->img) {
        r->heap.resize(2 * n);
        r->img = r->heap.data();
    }
    std::memcpy(r->img, left_host, n);
    std::memcpy(r->img + n, right_host, n);
    r->stream = stream;
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
        ss.queue.push_back(r);
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
    S->tickets.erase(ticket);
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
    if (n_slots) *n_slots = S->slots;
    if (max_in_flight) *max_in_flight = S->max_in_flight;
    return TSGM_OK;
}

}  // extern "C"
