// Host side of the tsgm C ABI: context lifetime, argument checks, stage orchestration on the
// context's CUDA stream, stage timing with CUDA events, inspection copies.

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "tsgm_internal.cuh"

using namespace tsgm;

namespace {

constexpr size_t kEventPool = 8192;  // events kept for stage timing (two per record)

tsgm_status fail(tsgm_ctx* c, tsgm_status s, const char* msg) {
    if (c) c->err = msg;
    return s;
}

tsgm_status cuda_fail(tsgm_ctx* c, cudaError_t e, const char* where) {
    if (c) {
        char buf[256];
        std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
        c->err = buf;
    }
    return TSGM_ERR_CUDA;
}

#define TSGM_CK(expr, where)                                     \
    do {                                                         \
        cudaError_t e_ = (expr);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

// launch one of this library's kernels and count it
#define TSGM_LAUNCH(expr, where)                                 \
    do {                                                         \
        ++ctx->launches;                                         \
        TSGM_CK(expr, where);                                    \
    } while (0)

#define TSGM_TRY(expr)                    \
    do {                                  \
        tsgm_status s_ = (expr);          \
        if (s_ != TSGM_OK) return s_;     \
    } while (0)

tsgm_status check_params(const tsgm_params* p, std::string& why) {
    char buf[200];
    if (p->width < 1 || p->height < 1 || (int64_t)p->width * p->height >= (1ll << 31)) {
        why = "width/height out of range";
        return TSGM_ERR_INVALID_ARG;
    }
    if (p->width > 13000) {
        why = "width must be <= 13000 (per-column state of one row is kept in shared memory)";
        return TSGM_ERR_INVALID_ARG;
    }
    if (p->d_max < 0 || p->d_max + 1 > TSGM_MAX_LABELS) {
        why = "d_max must be in [0, 255]";
        return TSGM_ERR_INVALID_ARG;
    }
    if (p->census_w < 1 || p->census_h < 1 || !(p->census_w & 1) || !(p->census_h & 1) ||
        p->census_w > 15 || p->census_h > 15 ||
        p->census_w * p->census_h - 1 > TSGM_MAX_CENSUS_BITS || p->census_w * p->census_h < 3) {
        why = "census window must be odd, at most 15 x 15 and have 2..64 bits";
        return TSGM_ERR_INVALID_ARG;
    }
    if (p->n_paths != 4 && p->n_paths != 8) {
        why = "n_paths must be 4 or 8";
        return TSGM_ERR_INVALID_ARG;
    }
    const int Bc = p->census_w * p->census_h - 1;
    if (p->P1 < 0 || p->P2 < p->P1 || Bc + p->P2 > 255) {
        std::snprintf(buf, sizeof(buf),
                      "need 0 <= P1 <= P2 and census bits + P2 <= 255 (got P1=%d, P2=%d)", p->P1, p->P2);
        why = buf;
        return TSGM_ERR_INVALID_ARG;
    }
    const uint64_t cells = (uint64_t)p->width * p->height * (uint64_t)(p->d_max + 4);
    if (cells + 64 >= (1ull << 32)) {
        why = "width * height * (d_max + 1) must stay below 2^32 cells";
        return TSGM_ERR_INVALID_ARG;
    }
    if (!(p->edge_thr >= 0.0f) || !std::isfinite(p->edge_thr)) {
        why = "edge_thr must be finite and >= 0";
        return TSGM_ERR_INVALID_ARG;
    }
    if (!(p->pred_lr_tol >= 0.0f) || !std::isfinite(p->pred_lr_tol)) {
        why = "pred_lr_tol must be finite and >= 0";
        return TSGM_ERR_INVALID_ARG;
    }
    if (p->sad_w < 1 || p->sad_w > 31 || p->sad_w % 2 == 0 || p->sad_h < 1 || p->sad_h > 31 ||
        p->sad_h % 2 == 0) {
        why = "sad_w and sad_h must be odd, 1 .. 31";
        return TSGM_ERR_INVALID_ARG;
    }
    if (!(p->sad_thr >= 0.0f) || !std::isfinite(p->sad_thr)) {
        why = "sad_thr must be finite and >= 0";
        return TSGM_ERR_INVALID_ARG;
    }
    if (!(p->gamma_f >= 0.0f) || !std::isfinite(p->gamma_f)) {
        why = "gamma_f must be finite and >= 0";
        return TSGM_ERR_INVALID_ARG;
    }
    if (!(p->sigma_mult >= 0.0f) || !(p->q >= 0.0f) || !(p->S_max >= 0.0f) || !(p->r_min >= 0.0f) ||
        p->lr_tol < 0 || !std::isfinite(p->sigma_mult) || !std::isfinite(p->q) ||
        !std::isfinite(p->S_max) || !std::isfinite(p->r_min)) {
        why = "sigma_mult, q, S_max, r_min must be finite and >= 0, lr_tol >= 0";
        return TSGM_ERR_INVALID_ARG;
    }
    return TSGM_OK;
}

// ----- stage timing ---------------------------------------------------------------------------
void timing_resolve(tsgm_ctx* c) {
    for (const tsgm_ctx::EventRec& r : c->ev_recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->ms[r.stage] += ms;
            c->cnt[r.stage] += 1;
        }
    }
    c->ev_recs.clear();
    c->ev_used = 0;
}

void stage_begin(tsgm_ctx* c, int s, cudaStream_t st) {
    if (!c->prof || c->ev_pool.size() < 2) return;
    if (c->ev_used + 2 > c->ev_pool.size()) timing_resolve(c);
    tsgm_ctx::EventRec r;
    r.stage = s;
    r.a = c->ev_pool[c->ev_used++];
    r.b = c->ev_pool[c->ev_used++];
    cudaEventRecord(r.a, st);
    c->ev_recs.push_back(r);
}
void stage_begin(tsgm_ctx* c, int s) { stage_begin(c, s, c->stream); }

void stage_end(tsgm_ctx* c, int s, cudaStream_t st) {
    if (!c->prof || c->ev_recs.empty()) return;
    tsgm_ctx::EventRec& r = c->ev_recs.back();
    if (r.stage == s) cudaEventRecord(r.b, st);
}
void stage_end(tsgm_ctx* c, int s) { stage_end(c, s, c->stream); }

template <typename T>
cudaError_t alloc(T** p, size_t count) {
    return cudaMalloc((void**)p, count * sizeof(T) + 64);
}

void free_all(tsgm_ctx* c) {
    void* bufs[] = {c->censusL, c->censusR, c->keys,   c->predD,  c->predP,   c->Dz,
                    c->rz,      c->stateD,  c->stateP, c->lo,     c->hi,      c->dstar,
                    c->dright,  c->lrvalid, c->off,    c->rowsum, c->C,       c->S,
                    c->rowcells, c->cells,  c->desc,  c->Lvol,  c->adj_partials,
                    c->wq,      c->gkeys,   c->wds,
                    c->d_left,  c->d_right, c->d_outD, c->d_outP,
                    c->d_left1, c->d_right1, c->d_outD1, c->d_outP1};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
    for (cudaGraphExec_t& x : c->fexec) {
        if (x) cudaGraphExecDestroy(x);
        x = nullptr;
    }
    for (int k = 0; k < 2; ++k) {
        if (c->ev_slot_in[k]) cudaEventDestroy(c->ev_slot_in[k]);
        if (c->ev_slot_used[k]) cudaEventDestroy(c->ev_slot_used[k]);
        if (c->ev_slot_out[k]) cudaEventDestroy(c->ev_slot_out[k]);
        c->ev_slot_in[k] = c->ev_slot_used[k] = c->ev_slot_out[k] = nullptr;
    }
    if (c->s_h2d) cudaStreamDestroy(c->s_h2d);
    if (c->s_d2h) cudaStreamDestroy(c->s_d2h);
    c->s_h2d = c->s_d2h = nullptr;
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->aux) cudaStreamDestroy(c->aux);
    c->ev_fork = c->ev_join = nullptr;
    c->aux = nullptr;
}

// H = Gamma T Gamma^{-1} (Eq. 1-4) in binary64; x, y relative to the principal point.
void build_H64(const float R[9], const float t[3], double f, double b, double H[16]) {
    const double G[4][4] = {{f, 0, 0, 0}, {0, f, 0, 0}, {0, 0, 0, f * b}, {0, 0, 1, 0}};
    const double Gi[4][4] = {
        {1.0 / f, 0, 0, 0}, {0, 1.0 / f, 0, 0}, {0, 0, 0, 1}, {0, 0, 1.0 / (f * b), 0}};
    const double T[4][4] = {{(double)R[0], (double)R[1], (double)R[2], (double)t[0]},
                            {(double)R[3], (double)R[4], (double)R[5], (double)t[1]},
                            {(double)R[6], (double)R[7], (double)R[8], (double)t[2]},
                            {0, 0, 0, 1}};
    double TG[4][4];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += T[r][k] * Gi[k][c];
            TG[r][c] = s;
        }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += G[r][k] * TG[k][c];
            H[r * 4 + c] = s;
        }
}

// ----- stages -----------------------------------------------------------------------------------
tsgm_status warp_stage(tsgm_ctx* ctx, const float* prevD, const float* prevP, const float R[9],
                       const float t[3], const float K[9], float baseline, float* predD,
                       float* predP) {
    float H32[16];
    if (tsgm_build_H(R, t, K, baseline, H32) != TSGM_OK)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "invalid pose or calibration (f, baseline > 0, finite R, t)");
    stage_begin(ctx, TSGM_STAGE_WARP);
    TSGM_CK(cudaMemsetAsync(ctx->keys, 0xFF, sizeof(unsigned long long) * ctx->n, ctx->stream),
            "memset z-buffer");
    TSGM_LAUNCH(launch_warp_scatter(prevD, prevP, H32, K[2], K[5], ctx->W, ctx->H, ctx->keys, ctx->stream),
            "warp scatter");
    TSGM_LAUNCH(launch_warp_gather(ctx->keys, prevD, prevP, ctx->prm.q, ctx->n, predD, predP, ctx->stream),
            "warp gather");
    stage_end(ctx, TSGM_STAGE_WARP);
    return TSGM_OK;
}

// Sec. 2.2 / Fig. 3(d): the prediction's left-right check, in place.
tsgm_status pred_lr_stage(tsgm_ctx* ctx, float* D, float* P) {
    stage_begin(ctx, TSGM_STAGE_WARP);
    TSGM_LAUNCH(launch_pred_lr(D, P, ctx->W, ctx->H, ctx->prm.pred_lr_tol, ctx->stream),
                "prediction left-right check");
    stage_end(ctx, TSGM_STAGE_WARP);
    return TSGM_OK;
}

// Sec. 2.4: SAD check of an updated map, in place on (D, P) and (D2, P2) when given.
tsgm_status sad_stage(tsgm_ctx* ctx, const uint8_t* left, const uint8_t* right, float* D, float* P,
                      float* D2, float* P2) {
    const tsgm_params& p = ctx->prm;
    const float lim = p.sad_thr * (float)(p.sad_w * p.sad_h);
    stage_begin(ctx, TSGM_STAGE_KALMAN);
    TSGM_LAUNCH(launch_sad_check(left, right, ctx->W, ctx->H, p.sad_w, p.sad_h, lim, D, P, D2, P2,
                                 ctx->stream),
                "SAD check");
    stage_end(ctx, TSGM_STAGE_KALMAN);
    return TSGM_OK;
}

// Sec. 2.2 edge rejection, in place on (D, P) through the D_z/r_z scratch.
tsgm_status edge_reject_stage(tsgm_ctx* ctx, float* D, float* P) {
    stage_begin(ctx, TSGM_STAGE_WARP);
    TSGM_LAUNCH(launch_edge_reject(D, P, ctx->W, ctx->H, ctx->prm.edge_thr, ctx->Dz, ctx->rz,
                                   ctx->stream),
                "edge reject");
    const size_t bytes = sizeof(float) * (size_t)ctx->n;
    TSGM_CK(cudaMemcpyAsync(D, ctx->Dz, bytes, cudaMemcpyDeviceToDevice, ctx->stream), "copy");
    TSGM_CK(cudaMemcpyAsync(P, ctx->rz, bytes, cudaMemcpyDeviceToDevice, ctx->stream), "copy");
    stage_end(ctx, TSGM_STAGE_WARP);
    return TSGM_OK;
}

// Eq. 7-8, in place on (D, P): horizontal pass into the D_z/r_z scratch, vertical pass back.
tsgm_status fill_gaps_stage(tsgm_ctx* ctx, float* D, float* P) {
    stage_begin(ctx, TSGM_STAGE_WARP);
    TSGM_LAUNCH(launch_fill_gaps(D, P, ctx->W, ctx->H, ctx->prm.gamma_f, 0, ctx->Dz, ctx->rz, ctx->stream),
                "fill gaps");
    TSGM_LAUNCH(launch_fill_gaps(ctx->Dz, ctx->rz, ctx->W, ctx->H, ctx->prm.gamma_f, 1, D, P, ctx->stream),
                "fill gaps");
    stage_end(ctx, TSGM_STAGE_WARP);
    return TSGM_OK;
}

tsgm_status windows_stage(tsgm_ctx* ctx, const float* pD, const float* pP, int16_t* lo,
                          int16_t* hi) {
    stage_begin(ctx, TSGM_STAGE_WINDOWS);
    TSGM_LAUNCH(launch_windows(pD, pP, ctx->W, ctx->H, ctx->D, ctx->prm.sigma_mult, lo, hi, ctx->rowsum,
                               ctx->rowcells, ctx->wq, ctx->stream),
                "windows");
    TSGM_LAUNCH(launch_offsets(lo, hi, ctx->rowsum, ctx->rowcells, ctx->W, ctx->H, ctx->off, ctx->desc,
                               ctx->cells, ctx->wq, ctx->stream),
                "offsets");
    stage_end(ctx, TSGM_STAGE_WINDOWS);
    return TSGM_OK;
}

// The census of both images on the context's second stream, forked from its stream here; the cost
// (match_stages) joins it. The census reads only the images, so it runs beside the prediction and
// window stages enqueued in between.
tsgm_status census_fork(tsgm_ctx* ctx, const uint8_t* left, const uint8_t* right) {
    const tsgm_params& p = ctx->prm;
    TSGM_CK(cudaEventRecord(ctx->ev_fork, ctx->stream), "census fork");
    TSGM_CK(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0), "census fork");
    stage_begin(ctx, TSGM_STAGE_CENSUS, ctx->aux);
    TSGM_LAUNCH(launch_census(left, right, ctx->W, ctx->H, p.census_w, p.census_h, ctx->censusL,
                              ctx->censusR, ctx->aux),
                "census");
    stage_end(ctx, TSGM_STAGE_CENSUS, ctx->aux);
    TSGM_CK(cudaEventRecord(ctx->ev_join, ctx->aux), "census join");
    return TSGM_OK;
}

// Matching on windows whose offsets are already in ctx->off and census codes forked by
// census_fork.
tsgm_status match_stages(tsgm_ctx* ctx, const int16_t* lo, const int16_t* hi, float* Dz,
                         float* rz, bool full) {
    const tsgm_params& p = ctx->prm;
    TSGM_CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0), "census join");
    stage_begin(ctx, TSGM_STAGE_COST);
    TSGM_LAUNCH(launch_cost(ctx->censusL, ctx->censusR, ctx->desc, ctx->W, ctx->H, ctx->Bc, ctx->C,
                            ctx->stream),
                "cost");
    stage_end(ctx, TSGM_STAGE_COST);
    stage_begin(ctx, TSGM_STAGE_SGM);
    TSGM_LAUNCH(launch_sgm(ctx->C, ctx->desc, ctx->W, ctx->H, ctx->D, p.n_paths, p.P1, p.P2, ctx->Lvol,
                           ctx->max_cells, ctx->wq, full, ctx->stream),
                "sgm");
    if (ctx->D <= 128 && !full) ++ctx->launches;  // launch_sgm enqueues both lane-group forms
    stage_end(ctx, TSGM_STAGE_SGM);
    const bool keep = (p.flags & TSGM_FLAG_KEEP_INTERNALS) != 0;
    const float s_thr = p.S_max * (float)p.n_paths;
    stage_begin(ctx, TSGM_STAGE_SELECT);
    if (full) {
        TSGM_LAUNCH(launch_select_full(ctx->Lvol, ctx->max_cells, p.n_paths, ctx->W, ctx->H, ctx->D,
                                       ctx->Bc, p.P2, s_thr, p.r_min, p.lr_tol, Dz, rz,
                                       keep ? ctx->S : nullptr, keep ? ctx->dstar : nullptr,
                                       keep ? ctx->dright : nullptr, keep ? ctx->lrvalid : nullptr,
                                       ctx->stream),
                    "select");
    } else {
        TSGM_LAUNCH(launch_select(ctx->Lvol, ctx->max_cells, p.n_paths, ctx->desc, ctx->W, ctx->H, ctx->D,
                                  s_thr, p.r_min, p.lr_tol, Dz, rz, keep ? ctx->S : nullptr,
                                  keep ? ctx->dstar : nullptr, keep ? ctx->dright : nullptr,
                                  keep ? ctx->lrvalid : nullptr, ctx->wq, ctx->gkeys, ctx->wds,
                                  ctx->stream),
                    "select");
        ++ctx->launches;  // launch_select enqueues two kernels (wide windows, then the rows)
    }
    stage_end(ctx, TSGM_STAGE_SELECT);
    return TSGM_OK;
}

}  // namespace

extern "C" {

void tsgm_default_params(tsgm_params* p, int32_t width, int32_t height) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->width = width;
    p->height = height;
    p->d_max = 127;
    p->census_w = 9;
    p->census_h = 7;
    p->n_paths = 8;
    p->P1 = 8;
    p->P2 = 32;
    p->sigma_mult = 3.0f;
    p->q = 0.25f;
    p->S_max = 10.0f;
    p->r_min = 0.5f;
    p->lr_tol = 1;
    p->flags = 0;
    p->gamma_f = 1.0f;
    p->edge_thr = 1.0f;
    p->pred_lr_tol = 1.0f;
    p->sad_w = 5;
    p->sad_h = 5;
    p->sad_thr = 30.0f;
}

tsgm_status tsgm_create(const tsgm_params* p, void* cuda_stream, tsgm_ctx** out) {
    if (!out) return TSGM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p) return TSGM_ERR_INVALID_ARG;
    std::string why;
    if (check_params(p, why) != TSGM_OK) {
        std::fprintf(stderr, "tsgm_create: %s\n", why.c_str());
        return TSGM_ERR_INVALID_ARG;
    }
    tsgm_ctx* ctx = new (std::nothrow) tsgm_ctx();
    if (!ctx) return TSGM_ERR_OUT_OF_MEMORY;
    ctx->prm = *p;
    ctx->W = p->width;
    ctx->H = p->height;
    ctx->D = p->d_max + 1;
    ctx->n = p->width * p->height;
    ctx->Bc = p->census_w * p->census_h - 1;
    // storage of the ragged volumes: every pixel's block is its window rounded up to 4 cells
    ctx->max_cells = (uint64_t)ctx->n * (uint64_t)((ctx->D + 3) & ~3);
    ctx->stream = (cudaStream_t)cuda_stream;  // NULL: the legacy default stream
    const size_t n = (size_t)ctx->n;
    bool ok = true;
    ok = ok && cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && alloc(&ctx->censusL, n) == cudaSuccess;
    ok = ok && alloc(&ctx->censusR, n) == cudaSuccess;
    ok = ok && alloc(&ctx->keys, n) == cudaSuccess;
    ok = ok && alloc(&ctx->predD, n) == cudaSuccess;
    ok = ok && alloc(&ctx->predP, n) == cudaSuccess;
    ok = ok && alloc(&ctx->Dz, n) == cudaSuccess;
    ok = ok && alloc(&ctx->rz, n) == cudaSuccess;
    ok = ok && alloc(&ctx->stateD, n) == cudaSuccess;
    ok = ok && alloc(&ctx->stateP, n) == cudaSuccess;
    ok = ok && alloc(&ctx->lo, n) == cudaSuccess;
    ok = ok && alloc(&ctx->hi, n) == cudaSuccess;
    ok = ok && alloc(&ctx->dstar, n) == cudaSuccess;
    ok = ok && alloc(&ctx->dright, n) == cudaSuccess;
    ok = ok && alloc(&ctx->lrvalid, n) == cudaSuccess;
    ok = ok && alloc(&ctx->off, n + 1) == cudaSuccess;
    ok = ok && alloc(&ctx->rowsum, (size_t)ctx->H) == cudaSuccess;
    ok = ok && alloc(&ctx->rowcells, 2 * (size_t)ctx->H) == cudaSuccess;
    ok = ok && alloc(&ctx->cells, 2) == cudaSuccess;
    ok = ok && alloc(&ctx->wq, n + 1) == cudaSuccess;
    ok = ok && alloc(&ctx->gkeys, n) == cudaSuccess;
    ok = ok && alloc(&ctx->wds, n) == cudaSuccess;
    // no key yet (the selection keeps this state between images); complete before any stream
    ok = ok && cudaMemset(ctx->gkeys, 0xFF, n * sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(nullptr) == cudaSuccess;
    ok = ok && alloc(&ctx->desc, n) == cudaSuccess;
    ok = ok && alloc(&ctx->C, (size_t)ctx->max_cells + 64) == cudaSuccess;
    ok = ok && alloc(&ctx->S, (size_t)ctx->max_cells + 64) == cudaSuccess;
    ok = ok && alloc(&ctx->Lvol, (size_t)ctx->max_cells * (size_t)p->n_paths + 64) == cudaSuccess;
    ok = ok && alloc(&ctx->adj_partials, (size_t)kAdjointBlocks * 6) == cudaSuccess;
    ok = ok && alloc(&ctx->d_left, n) == cudaSuccess;
    ok = ok && alloc(&ctx->d_right, n) == cudaSuccess;
    ok = ok && alloc(&ctx->d_outD, n) == cudaSuccess;
    ok = ok && alloc(&ctx->d_outP, n) == cudaSuccess;
    ok = ok && alloc(&ctx->d_left1, n) == cudaSuccess;
    ok = ok && alloc(&ctx->d_right1, n) == cudaSuccess;
    ok = ok && alloc(&ctx->d_outD1, n) == cudaSuccess;
    ok = ok && alloc(&ctx->d_outP1, n) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&ctx->s_h2d, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&ctx->s_d2h, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 2; ++k) {
        ok = ok && cudaEventCreateWithFlags(&ctx->ev_slot_in[k], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&ctx->ev_slot_used[k], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&ctx->ev_slot_out[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        free_all(ctx);
        delete ctx;
        return TSGM_ERR_OUT_OF_MEMORY;
    }
    *out = ctx;
    return TSGM_OK;
}

void tsgm_destroy(tsgm_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
}

const char* tsgm_last_error(const tsgm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

tsgm_status tsgm_set_stream(tsgm_ctx* ctx, void* cuda_stream) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return TSGM_OK;
}

tsgm_status tsgm_build_H(const float R[9], const float t[3], const float K[9], float baseline,
                         float H_out[16]) {
    if (!R || !t || !K || !H_out) return TSGM_ERR_INVALID_ARG;
    const double f = (double)K[0];
    if (!(f > 0.0) || !(baseline > 0.0f) || !std::isfinite(f) || !std::isfinite(baseline))
        return TSGM_ERR_INVALID_ARG;
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(R[k])) return TSGM_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(t[k])) return TSGM_ERR_INVALID_ARG;
    double H[16];
    build_H64(R, t, f, (double)baseline, H);
    for (int k = 0; k < 16; ++k) H_out[k] = (float)H[k];
    return TSGM_OK;
}

tsgm_status tsgm_warp_predict(tsgm_ctx* ctx, const float* prev_D, const float* prev_P,
                              const float R[9], const float t[3], const float K[9], float baseline,
                              float* pred_D, float* pred_P) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!prev_D || !prev_P || !R || !t || !K || !pred_D || !pred_P)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_warp_predict: null pointer");
    if (pred_D == prev_D || pred_P == prev_P || pred_D == prev_P || pred_P == prev_D)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_warp_predict: outputs alias inputs");
    return warp_stage(ctx, prev_D, prev_P, R, t, K, baseline, pred_D, pred_P);
}

tsgm_status tsgm_fill_gaps(tsgm_ctx* ctx, float* pred_D, float* pred_P) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!pred_D || !pred_P) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_fill_gaps: null pointer");
    if (pred_D == ctx->Dz || pred_P == ctx->rz || pred_D == ctx->rz || pred_P == ctx->Dz)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_fill_gaps: maps alias the context scratch");
    return fill_gaps_stage(ctx, pred_D, pred_P);
}

tsgm_status tsgm_edge_reject(tsgm_ctx* ctx, float* pred_D, float* pred_P) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!pred_D || !pred_P) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_edge_reject: null pointer");
    if (pred_D == ctx->Dz || pred_P == ctx->rz || pred_D == ctx->rz || pred_P == ctx->Dz)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_edge_reject: maps alias the context scratch");
    return edge_reject_stage(ctx, pred_D, pred_P);
}

tsgm_status tsgm_pred_lr_check(tsgm_ctx* ctx, float* pred_D, float* pred_P) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!pred_D || !pred_P) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_pred_lr_check: null pointer");
    if (pred_D == pred_P) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_pred_lr_check: maps alias");
    return pred_lr_stage(ctx, pred_D, pred_P);
}

tsgm_status tsgm_sad_check(tsgm_ctx* ctx, const uint8_t* left, const uint8_t* right, float* D,
                           float* P) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!left || !right || !D || !P) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_sad_check: null pointer");
    if (D == P) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_sad_check: maps alias");
    return sad_stage(ctx, left, right, D, P, nullptr, nullptr);
}

tsgm_status tsgm_windows(tsgm_ctx* ctx, const float* pred_D, const float* pred_P, int16_t* d_lo,
                         int16_t* d_hi, uint64_t* n_cells_host) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!pred_D || !pred_P || !d_lo || !d_hi)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_windows: null pointer");
    TSGM_TRY(windows_stage(ctx, pred_D, pred_P, d_lo, d_hi));
    if (n_cells_host) return tsgm_cells(ctx, n_cells_host);
    return TSGM_OK;
}

tsgm_status tsgm_match(tsgm_ctx* ctx, const uint8_t* left, const uint8_t* right,
                       const int16_t* d_lo, const int16_t* d_hi, float* D_z, float* r_z) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!left || !right || !d_lo || !d_hi || !D_z || !r_z)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_match: null pointer");
    TSGM_TRY(census_fork(ctx, left, right));
    // the caller's windows are copied, clamped into [0, d_max], into the context's buffers
    stage_begin(ctx, TSGM_STAGE_OFFSETS);
    TSGM_LAUNCH(launch_sanitize(d_lo, d_hi, ctx->W, ctx->H, ctx->D, ctx->lo, ctx->hi, ctx->rowsum,
                                ctx->rowcells, ctx->wq, ctx->stream),
                "windows copy");
    TSGM_LAUNCH(launch_offsets(ctx->lo, ctx->hi, ctx->rowsum, ctx->rowcells, ctx->W, ctx->H, ctx->off,
                               ctx->desc, ctx->cells, ctx->wq, ctx->stream),
                "offsets");
    stage_end(ctx, TSGM_STAGE_OFFSETS);
    return match_stages(ctx, ctx->lo, ctx->hi, D_z, r_z, false);
}

tsgm_status tsgm_kalman_update(tsgm_ctx* ctx, const float* pred_D, const float* pred_P,
                               const float* D_z, const float* r_z, float* D, float* P) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!pred_D || !pred_P || !D_z || !r_z || !D || !P)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_kalman_update: null pointer");
    stage_begin(ctx, TSGM_STAGE_KALMAN);
    TSGM_LAUNCH(launch_kalman(pred_D, pred_P, D_z, r_z, ctx->n, D, P, nullptr, nullptr, ctx->stream),
            "kalman");
    stage_end(ctx, TSGM_STAGE_KALMAN);
    return TSGM_OK;
}

}  // extern "C"

namespace {

// Every stage of one time step, enqueued on the context's streams (the census on the second).
tsgm_status frame_enqueue(tsgm_ctx* ctx, const uint8_t* left, const uint8_t* right,
                          const float R[9], const float t[3], const float K[9], float baseline,
                          float* D, float* P) {
    TSGM_TRY(census_fork(ctx, left, right));
    if (ctx->has_prev) {
        TSGM_TRY(warp_stage(ctx, ctx->stateD, ctx->stateP, R, t, K, baseline, ctx->predD, ctx->predP));
        if (ctx->prm.flags & TSGM_FLAG_EDGE_REJECT) TSGM_TRY(edge_reject_stage(ctx, ctx->predD, ctx->predP));
        if (ctx->prm.flags & TSGM_FLAG_FILL_GAPS) TSGM_TRY(fill_gaps_stage(ctx, ctx->predD, ctx->predP));
        if (ctx->prm.flags & TSGM_FLAG_PRED_LR_CHECK) TSGM_TRY(pred_lr_stage(ctx, ctx->predD, ctx->predP));
    } else {
        TSGM_LAUNCH(launch_fill(ctx->predD, -1.0f, ctx->n, ctx->stream), "fill");
        TSGM_LAUNCH(launch_fill(ctx->predP, -1.0f, ctx->n, ctx->stream), "fill");
    }
    if (ctx->prm.flags & TSGM_FLAG_FULL_RANGE) {
        // windows from an empty prediction: the whole range everywhere
        TSGM_LAUNCH(launch_fill(ctx->Dz, -1.0f, ctx->n, ctx->stream), "fill");
        TSGM_TRY(windows_stage(ctx, ctx->Dz, ctx->Dz, ctx->lo, ctx->hi));
    } else {
        TSGM_TRY(windows_stage(ctx, ctx->predD, ctx->predP, ctx->lo, ctx->hi));
    }
    // every window is the whole range on a first frame and in the full-range mode
    const bool full = !ctx->has_prev || (ctx->prm.flags & TSGM_FLAG_FULL_RANGE) != 0;
    TSGM_TRY(match_stages(ctx, ctx->lo, ctx->hi, ctx->Dz, ctx->rz, full));
    stage_begin(ctx, TSGM_STAGE_KALMAN);
    TSGM_LAUNCH(launch_kalman(ctx->predD, ctx->predP, ctx->Dz, ctx->rz, ctx->n, D, P, ctx->stateD,
                          ctx->stateP, ctx->stream),
            "kalman");
    stage_end(ctx, TSGM_STAGE_KALMAN);
    if (ctx->prm.flags & TSGM_FLAG_SAD_CHECK)
        TSGM_TRY(sad_stage(ctx, left, right, D, P, ctx->stateD, ctx->stateP));
    ctx->has_prev = 1;
    return TSGM_OK;
}

// The step as a CUDA graph: captured from the context's stream, then either used to update in
// place the instantiated graph of the last step of its kind (a first frame, or a frame with a
// previous state: the same kernels, new pointers and pose) or instantiated anew, and launched. A step of ~20 small kernels
// runs with shorter gaps between them this way. Not for the legacy default streams (they cannot
// be captured) nor while stage timing is on; a capture that fails leaves the context on the
// direct path for good. Returns false when the step was not run (the caller runs it directly).
bool frame_graph(tsgm_ctx* ctx, const uint8_t* left, const uint8_t* right, const float R[9],
                 const float t[3], const float K[9], float baseline, float* D, float* P,
                 tsgm_status* st) {
    if (ctx->graph_off || ctx->prof || ctx->stream == nullptr || ctx->stream == cudaStreamLegacy ||
        ctx->stream == cudaStreamPerThread)
        return false;
    // the caller may be capturing the stream itself: then the kernels go into its capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;
    }
    if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        ctx->graph_off = true;
        return false;
    }
    const int had_prev = ctx->has_prev;
    const uint64_t launches = ctx->launches;
    const tsgm_status s = frame_enqueue(ctx, left, right, R, t, K, baseline, D, P);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
    if (s != TSGM_OK || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        ctx->has_prev = had_prev;
        ctx->launches = launches;
        if (s != TSGM_OK) {  // an argument or launch error: nothing ran, report it
            *st = s;
            return true;
        }
        ctx->graph_off = true;  // the capture itself failed: run this step directly
        return false;
    }
    bool ok = true;
    cudaGraphExec_t& ex = ctx->fexec[had_prev ? 1 : 0];
    if (ex) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(ex, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(ex);
            ex = nullptr;
        }
    }
    if (!ex) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    if (ok) ok = cudaGraphLaunch(ex, ctx->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (ex) cudaGraphExecDestroy(ex);
        ex = nullptr;
        ctx->graph_off = true;
        ctx->has_prev = had_prev;
        ctx->launches = launches;
        return false;
    }
    *st = TSGM_OK;
    return true;
}

}  // namespace

extern "C" {

tsgm_status tsgm_frame(tsgm_ctx* ctx, const uint8_t* left, const uint8_t* right, const float R[9],
                       const float t[3], const float K[9], float baseline, float* D, float* P) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!left || !right || !K || !D || !P)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_frame: null pointer");
    if (D == P) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_frame: D and P alias");
    if (ctx->has_prev && (!R || !t))
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_frame: pose required after the first frame");
    tsgm_status st = TSGM_OK;
    if (frame_graph(ctx, left, right, R, t, K, baseline, D, P, &st)) return st;
    return frame_enqueue(ctx, left, right, R, t, K, baseline, D, P);
}

tsgm_status tsgm_frame_host(tsgm_ctx* ctx, const uint8_t* left_host, const uint8_t* right_host,
                            const float R[9], const float t[3], const float K[9], float baseline,
                            float* D_host, float* P_host) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!left_host || !right_host || !D_host || !P_host)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_frame_host: null pointer");
    const size_t n = (size_t)ctx->n;
    // copies still pending from tsgm_frame_host_async use the same staging
    TSGM_CK(cudaStreamSynchronize(ctx->s_h2d), "synchronize");
    TSGM_CK(cudaStreamSynchronize(ctx->s_d2h), "synchronize");
    TSGM_CK(cudaMemcpyAsync(ctx->d_left, left_host, n, cudaMemcpyHostToDevice, ctx->stream), "h2d left");
    TSGM_CK(cudaMemcpyAsync(ctx->d_right, right_host, n, cudaMemcpyHostToDevice, ctx->stream), "h2d right");
    TSGM_TRY(tsgm_frame(ctx, ctx->d_left, ctx->d_right, R, t, K, baseline, ctx->d_outD, ctx->d_outP));
    TSGM_CK(cudaMemcpyAsync(D_host, ctx->d_outD, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream), "d2h D");
    TSGM_CK(cudaMemcpyAsync(P_host, ctx->d_outP, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream), "d2h P");
    TSGM_CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    return TSGM_OK;
}

tsgm_status tsgm_frame_host_async(tsgm_ctx* ctx, const uint8_t* left_host,
                                  const uint8_t* right_host, const float R[9], const float t[3],
                                  const float K[9], float baseline, float* D_host, float* P_host) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!left_host || !right_host || !D_host || !P_host)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_frame_host_async: null pointer");
    if (D_host == P_host) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_frame_host_async: D and P alias");
    if (ctx->has_prev && (!R || !t))
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_frame_host_async: pose required after the first frame");
    const size_t n = (size_t)ctx->n;
    const int s = ctx->hslot;
    ctx->hslot ^= 1;
    uint8_t* const dl = s ? ctx->d_left1 : ctx->d_left;
    uint8_t* const dr = s ? ctx->d_right1 : ctx->d_right;
    float* const dD = s ? ctx->d_outD1 : ctx->d_outD;
    float* const dP = s ? ctx->d_outP1 : ctx->d_outP;
    // inputs: once the frame that used this slot two calls ago is done with it
    TSGM_CK(cudaStreamWaitEvent(ctx->s_h2d, ctx->ev_slot_used[s], 0), "wait");
    TSGM_CK(cudaMemcpyAsync(dl, left_host, n, cudaMemcpyHostToDevice, ctx->s_h2d), "h2d left");
    TSGM_CK(cudaMemcpyAsync(dr, right_host, n, cudaMemcpyHostToDevice, ctx->s_h2d), "h2d right");
    TSGM_CK(cudaEventRecord(ctx->ev_slot_in[s], ctx->s_h2d), "record");
    // the step: after its inputs, and after the slot's outputs of two calls ago were copied out
    TSGM_CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_slot_in[s], 0), "wait");
    TSGM_CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_slot_out[s], 0), "wait");
    TSGM_TRY(tsgm_frame(ctx, dl, dr, R, t, K, baseline, dD, dP));
    TSGM_CK(cudaEventRecord(ctx->ev_slot_used[s], ctx->stream), "record");
    // outputs: after the step, beside the next one
    TSGM_CK(cudaStreamWaitEvent(ctx->s_d2h, ctx->ev_slot_used[s], 0), "wait");
    TSGM_CK(cudaMemcpyAsync(D_host, dD, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->s_d2h), "d2h D");
    TSGM_CK(cudaMemcpyAsync(P_host, dP, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->s_d2h), "d2h P");
    TSGM_CK(cudaEventRecord(ctx->ev_slot_out[s], ctx->s_d2h), "record");
    return TSGM_OK;
}

tsgm_status tsgm_wait(tsgm_ctx* ctx) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    TSGM_CK(cudaStreamSynchronize(ctx->s_d2h), "synchronize");
    TSGM_CK(cudaStreamSynchronize(ctx->s_h2d), "synchronize");
    TSGM_CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    return TSGM_OK;
}

tsgm_status tsgm_reset(tsgm_ctx* ctx) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    ctx->has_prev = 0;
    return TSGM_OK;
}

tsgm_status tsgm_state_export(tsgm_ctx* ctx, float* D_host, float* P_host, int32_t* has_prev) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!D_host || !P_host || !has_prev)
        return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_state_export: null pointer");
    const size_t bytes = (size_t)ctx->n * sizeof(float);
    TSGM_CK(cudaMemcpyAsync(D_host, ctx->stateD, bytes, cudaMemcpyDeviceToHost, ctx->stream), "d2h state");
    TSGM_CK(cudaMemcpyAsync(P_host, ctx->stateP, bytes, cudaMemcpyDeviceToHost, ctx->stream), "d2h state");
    TSGM_CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    *has_prev = ctx->has_prev;
    return TSGM_OK;
}

tsgm_status tsgm_state_import(tsgm_ctx* ctx, const float* D_host, const float* P_host,
                              int32_t has_prev) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!has_prev) {
        ctx->has_prev = 0;
        return TSGM_OK;
    }
    if (!D_host || !P_host) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_state_import: null pointer");
    const size_t bytes = (size_t)ctx->n * sizeof(float);
    TSGM_CK(cudaMemcpyAsync(ctx->stateD, D_host, bytes, cudaMemcpyHostToDevice, ctx->stream), "h2d state");
    TSGM_CK(cudaMemcpyAsync(ctx->stateP, P_host, bytes, cudaMemcpyHostToDevice, ctx->stream), "h2d state");
    TSGM_CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    ctx->has_prev = 1;
    return TSGM_OK;
}

tsgm_status tsgm_census(tsgm_ctx* ctx, const uint8_t* img, uint64_t* codes) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!img || !codes) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_census: null pointer");
    TSGM_LAUNCH(launch_census(img, nullptr, ctx->W, ctx->H, ctx->prm.census_w, ctx->prm.census_h, codes,
                          nullptr, ctx->stream),
            "census");
    return TSGM_OK;
}

tsgm_status tsgm_inspect(tsgm_ctx* ctx, tsgm_buffer which, void* dst, uint64_t count) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!dst) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_inspect: null pointer");
    const uint64_t n = (uint64_t)ctx->n;
    const void* src = nullptr;
    uint64_t cap = 0, esz = 0;
    switch (which) {
        case TSGM_BUF_CENSUS_L: src = ctx->censusL; cap = n; esz = 8; break;
        case TSGM_BUF_CENSUS_R: src = ctx->censusR; cap = n; esz = 8; break;
        case TSGM_BUF_OFFSETS: src = ctx->off; cap = n + 1; esz = 4; break;
        case TSGM_BUF_COST: src = ctx->C; cap = ctx->max_cells; esz = 1; break;
        case TSGM_BUF_S: src = ctx->S; cap = ctx->max_cells; esz = 2; break;
        case TSGM_BUF_DSTAR: src = ctx->dstar; cap = n; esz = 2; break;
        case TSGM_BUF_DRIGHT: src = ctx->dright; cap = n; esz = 2; break;
        case TSGM_BUF_LR_VALID: src = ctx->lrvalid; cap = n; esz = 1; break;
        case TSGM_BUF_ZKEYS: src = ctx->keys; cap = n; esz = 8; break;
        case TSGM_BUF_WINDOWS_LO: src = ctx->lo; cap = n; esz = 2; break;
        case TSGM_BUF_WINDOWS_HI: src = ctx->hi; cap = n; esz = 2; break;
        case TSGM_BUF_PRED_D: src = ctx->predD; cap = n; esz = 4; break;
        case TSGM_BUF_PRED_P: src = ctx->predP; cap = n; esz = 4; break;
        case TSGM_BUF_COUNTS: src = ctx->cells; cap = 2; esz = 4; break;
        default: return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_inspect: unknown buffer");
    }
    if (count > cap) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_inspect: count exceeds buffer");
    if (count == 0) return TSGM_OK;
    TSGM_CK(cudaMemcpyAsync(dst, src, count * esz, cudaMemcpyDeviceToDevice, ctx->stream), "inspect copy");
    return TSGM_OK;
}

tsgm_status tsgm_cells(tsgm_ctx* ctx, uint64_t* n_cells) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!n_cells) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_cells: null pointer");
    uint32_t v = 0;
    TSGM_CK(cudaMemcpyAsync(&v, ctx->cells, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream),
            "read cell count");
    TSGM_CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    *n_cells = v;
    return TSGM_OK;
}

tsgm_status tsgm_launches(tsgm_ctx* ctx, uint64_t* n) {
    if (!ctx || !n) return TSGM_ERR_INVALID_ARG;
    *n = ctx->launches;
    return TSGM_OK;
}

tsgm_status tsgm_profile(tsgm_ctx* ctx, int32_t enable) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (enable && ctx->ev_pool.empty()) {
        ctx->ev_pool.resize(kEventPool);
        for (size_t k = 0; k < kEventPool; ++k) {
            if (cudaEventCreate(&ctx->ev_pool[k]) != cudaSuccess) {
                ctx->ev_pool.resize(k);
                return fail(ctx, TSGM_ERR_CUDA, "event creation failed");
            }
        }
    }
    if (!enable) timing_resolve(ctx);
    ctx->ev_recs.clear();
    ctx->ev_used = 0;
    for (int s = 0; s < TSGM_N_STAGES; ++s) {
        ctx->ms[s] = 0.0;
        ctx->cnt[s] = 0;
    }
    ctx->prof = enable != 0;
    return TSGM_OK;
}

tsgm_status tsgm_stage_times(tsgm_ctx* ctx, double ms[TSGM_N_STAGES], int64_t count[TSGM_N_STAGES]) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!ms || !count) return fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_stage_times: null pointer");
    timing_resolve(ctx);
    for (int s = 0; s < TSGM_N_STAGES; ++s) {
        ms[s] = ctx->ms[s];
        count[s] = ctx->cnt[s];
    }
    return TSGM_OK;
}

}  // extern "C"
