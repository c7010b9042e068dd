// Internal declarations shared by the tsgm CUDA sources (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "tsgm.h"

namespace tsgm {

constexpr int kInf = 0x3FFF;          // +inf for path costs held in 32-bit registers
constexpr uint64_t kEmptyKey = ~0ull; // empty z-buffer slot
constexpr int kAdjointBlocks = 152 * 4;  // blocks of the adjoint reduction (one partial each)

// Per-call device views of the inputs of the matching stages.
struct MatchBufs {
    const uint8_t* left;
    const uint8_t* right;
    const int16_t* lo;
    const int16_t* hi;
    float* Dz;
    float* rz;
};

// Launchers (defined in tsgm_predict.cu / tsgm_match.cu). Each enqueues on `st` and returns the
// launch status (cudaGetLastError).
cudaError_t launch_warp_scatter(const float* Dprev, const float* Pprev, const float* H, float cx,
                                float cy, int W, int Hh, unsigned long long* keys, cudaStream_t st);
cudaError_t launch_warp_gather(const unsigned long long* keys, const float* Dprev,
                               const float* Pprev, float q, int n, float* Dpred, float* Ppred,
                               cudaStream_t st);
cudaError_t launch_windows(const float* Dp, const float* Pp, int W, int Hh, int D, float k,
                           int16_t* lo, int16_t* hi, uint32_t* rowsum, uint32_t* rowcells,
                           uint32_t* wq, cudaStream_t st);
cudaError_t launch_sanitize(const int16_t* lo_in, const int16_t* hi_in, int W, int Hh, int D,
                            int16_t* lo, int16_t* hi, uint32_t* rowsum, uint32_t* rowcells,
                            uint32_t* wq, cudaStream_t st);
// wq: the queue of wide pixels (see select_split), cleared by launch_windows / launch_sanitize
cudaError_t launch_offsets(const int16_t* lo, const int16_t* hi, const uint32_t* rowsum,
                           const uint32_t* rowcells, int W, int Hh, uint32_t* off, uint2* desc,
                           uint32_t* cells_total, uint32_t* wq, cudaStream_t st);
cudaError_t launch_fill(float* a, float v, int n, cudaStream_t st);
// left-right check of a prediction, in place, one block per row
cudaError_t launch_pred_lr(float* D, float* P, int W, int Hh, float tol, cudaStream_t st);
// SAD check of an updated map, in place on (D, P) and, when given, on (D2, P2)
cudaError_t launch_sad_check(const uint8_t* left, const uint8_t* right, int W, int Hh, int sw,
                             int sh, float lim, float* D, float* P, float* D2, float* P2,
                             cudaStream_t st);
cudaError_t launch_edge_reject(const float* Din, const float* Pin, int W, int Hh, float thr,
                               float* Dout, float* Pout, cudaStream_t st);
cudaError_t launch_fill_gaps(const float* Din, const float* Pin, int W, int Hh, float gamma_f,
                             int vertical, float* Dout, float* Pout, cudaStream_t st);
cudaError_t launch_kalman(const float* Dp, const float* Pp, const float* Dz, const float* rz, int n,
                          float* D, float* P, float* D2, float* P2, cudaStream_t st);

cudaError_t launch_census(const uint8_t* imgA, const uint8_t* imgB, int W, int Hh, int cw, int ch,
                          uint64_t* outA, uint64_t* outB, cudaStream_t st);
cudaError_t launch_cost(const uint64_t* cl, const uint64_t* cr, const uint2* desc, int W, int Hh,
                        int Bc, uint8_t* C, cudaStream_t st);
// wq: the queue of wide pixels written by launch_offsets (its count picks the lane groups);
// full: every window is [0, D - 1] (one launch of the full-range kernel, desc and wq unread)
cudaError_t launch_sgm(const uint8_t* C, const uint2* desc, int W, int Hh, int D, int n_paths,
                       int P1, int P2, uint8_t* Lvol, uint64_t vol_stride, const uint32_t* wq,
                       bool full, cudaStream_t st);
// every window [0, D - 1]: one kernel, desc and the wide queue unread (Bc: census bits)
cudaError_t launch_select_full(const uint8_t* Lvol, uint64_t vol_stride, int n_paths, int W, int Hh,
                               int D, int Bc, int P2, float s_thr, float r_min, int lr_tol,
                               float* Dz, float* rz, uint16_t* S, int16_t* dstar, int16_t* dright,
                               uint8_t* valid, cudaStream_t st);
cudaError_t launch_select(const uint8_t* Lvol, uint64_t vol_stride, int n_paths, const uint2* desc,
                          int W, int Hh, int D, float s_thr, float r_min, int lr_tol, float* Dz,
                          float* rz, uint16_t* S, int16_t* dstar, int16_t* dright, uint8_t* valid,
                          const uint32_t* wq, uint32_t* gkeys, int16_t* wds, cudaStream_t st);

// A batch (tsgm_batch_create) whose volume pool is sized by an HBM budget instead of labels per
// pixel: whatever the budget leaves after the per-stream buffers, at least the largest stream at
// full range and at most every stream at full range (hbm_budget_bytes = 0: as tsgm_batch_create).
tsgm_status batch_create(const tsgm_params* streams, int32_t n_streams, int32_t max_labels,
                         uint64_t hbm_budget_bytes, void* cuda_stream, tsgm_batch** out);

}  // namespace tsgm

// The opaque context of the public ABI.
struct tsgm_ctx {
    tsgm_params prm;
    int W = 0, H = 0, D = 0, n = 0, Bc = 0;
    uint64_t max_cells = 0;
    cudaStream_t stream = nullptr;
    // second stream: the census of both images runs there beside the prediction and the windows
    // (forked from `stream` by ev_fork, joined before the cost by ev_join)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // device scratch, all sized at create time
    uint64_t* censusL = nullptr;
    uint64_t* censusR = nullptr;
    unsigned long long* keys = nullptr;
    float* predD = nullptr;
    float* predP = nullptr;
    float* Dz = nullptr;
    float* rz = nullptr;
    float* stateD = nullptr;
    float* stateP = nullptr;
    int16_t* lo = nullptr;
    int16_t* hi = nullptr;
    int16_t* dstar = nullptr;
    int16_t* dright = nullptr;
    uint8_t* lrvalid = nullptr;
    uint32_t* off = nullptr;       // block start of each pixel (+ storage size at [n])
    uint2* desc = nullptr;         // {off, lo | w << 16} per pixel
    uint32_t* rowsum = nullptr;    // storage cells per row
    uint32_t* rowcells = nullptr;  // true window cells per row, then (at + H) wide pixels per row
    uint32_t* cells = nullptr;     // [0] true window cells of the image, [1] pixels wider than 32
    uint32_t* wq = nullptr;        // queue of the wide pixels of the selection (n + 1 words)
    uint32_t* gkeys = nullptr;     // right-view keys of the wide pixels (all ones between images)
    int16_t* wds = nullptr;        // winners of the wide pixels
    uint8_t* C = nullptr;          // ragged matching cost
    uint16_t* S = nullptr;         // aggregated cost, written only with TSGM_FLAG_KEEP_INTERNALS
    uint8_t* Lvol = nullptr;       // one ragged uint8 volume of path costs per SGM direction
    double* adj_partials = nullptr;  // per-block partial sums of the adjoint (6 per block)
    // staging for tsgm_frame_host
    uint8_t* d_left = nullptr;
    uint8_t* d_right = nullptr;
    float* d_outD = nullptr;
    float* d_outP = nullptr;
    // tsgm_frame_host_async: two staging slots (slot 0 is the buffers above), used in turn; input
    // copies on s_h2d, output copies on s_d2h; per slot: inputs copied (ev_slot_in), frame done with
    // the slot (ev_slot_used), outputs copied out (ev_slot_out)
    uint8_t* d_left1 = nullptr;
    uint8_t* d_right1 = nullptr;
    float* d_outD1 = nullptr;
    float* d_outP1 = nullptr;
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_slot_in[2] = {nullptr, nullptr};
    cudaEvent_t ev_slot_used[2] = {nullptr, nullptr};
    cudaEvent_t ev_slot_out[2] = {nullptr, nullptr};
    int hslot = 0;

    int has_prev = 0;
    // the time step as a graph (tsgm_frame): [0] a full-range step, [1] a reduced one
    cudaGraphExec_t fexec[2] = {nullptr, nullptr};
    bool graph_off = false;           // tsgm_frame launches its kernels directly
    uint64_t launches = 0;  // kernels enqueued by this context (for launch accounting)
    std::string err;

    // stage timing: a ring of event pairs resolved lazily by tsgm_stage_times
    struct EventRec {
        int stage;
        cudaEvent_t a, b;
    };
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<EventRec> ev_recs;
    size_t ev_used = 0;
    double ms[TSGM_N_STAGES] = {};
    int64_t cnt[TSGM_N_STAGES] = {};
};
