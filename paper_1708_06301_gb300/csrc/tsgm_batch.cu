// Batched processing of many camera streams of different sizes and disparity ranges: the
// matching of caller windows (tsgm_batch_match, Sec. 2.3-2.4 applied to every stream) and the
// whole time step (tsgm_batch_frame, Sec. 2: prediction, gap filling, windows, matching, update,
// with every stream's state kept on the device). Every stage is one launch over the work units
// of all streams (pixels, rows, census tiles, path lines); the path aggregation is a persistent
// kernel whose warps pull path lines from one global queue, ordered direction-major so that the
// long horizontal chains of every stream start first and large and small streams balance; each
// form of the step is captured once in a CUDA graph and replayed. A stream can sit a step out
// (tsgm_batch_frame with no images for it): its blocks return at once and its state stays. The
// launch shape of the aggregation and the grid of the cost kernel are chosen by an autotuner
// that times the candidates on the caller's data.

#include <algorithm>
#include <cfloat>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tsgm_kernels.cuh"
#include "tsgm_predict.cuh"
#include "tsgm_sgm.cuh"

namespace {

using namespace tsgm;
using namespace tsgm::dev;

constexpr int kMaxStreams = 128;

// Device-side view of one stream.
struct BStream {
    int W, H, D, n;
    // per-call inputs and outputs, rewritten before every replay
    const uint8_t* left;
    const uint8_t* right;
    const int16_t* lo_in;
    const int16_t* hi_in;
    float* Dz;
    float* rz;
    // scratch owned by the batch
    int16_t* lo;
    int16_t* hi;
    uint64_t* censusL;
    uint64_t* censusR;
    uint2* desc;
    uint32_t* off;
    uint32_t* rowsum;
    uint32_t* rowcells;  // true cells per row, then (at + H) pixels wider than kNarrowMax per row
    uint32_t* cells;     // [0] true cells, [1] pixels wider than kNarrowMax
    uint32_t* status;  // 0 ok, 1: the windows did not fit the free part of the volume pool
    uint8_t* C;         // the batch's volume pool (shared by all streams; each step a stream's
    uint8_t* Lvol;      // volumes start at its reserved base cell)
    uint64_t capacity;  // cells of the pool per volume (C and each direction of Lvol)
    int active;         // 0: the stream sits this step out
    // time-step form: the previous state, the prediction and its scratch, the matched maps
    WarpParams wp;
    float q;
    unsigned long long* keys;  // z-buffer, all empty between steps (the gather empties them)
    float* stateD;
    float* stateP;
    float* predD;
    float* predP;
    float* tmpD;
    float* tmpP;
    float* Dm;  // matched disparity and variance (the form's own D_z, r_z)
    float* rm;
    float* outD;  // caller outputs of this step
    float* outP;
};

struct BTable {
    int ns;
    int row_base[kMaxStreams + 1];   // prefix of image rows
    int tile_base[kMaxStreams + 1];  // prefix of census tiles (one image)
    int px_base[kMaxStreams + 1];    // prefix of pixels
    int tiles_x[kMaxStreams];
    int pblk_base[kMaxStreams + 1];  // prefix of 256-pixel blocks
    // groups of path lines (the lines one warp walks together), direction-major: slot s holds the
    // lines of direction code s; items of stream i in slot s are [slot_base[s][i],
    // slot_base[s][i+1]); slot_base[s][ns] == slot_base[s+1][0]
    int slot_base[8][kMaxStreams + 1];
    int total_items;
    // volume pool: every step each active stream reserves the cells of its windows, in order of
    // how many steps in a row it has been refused (then stream order); device arrays
    uint64_t* base;     // first pool cell of the stream's volumes this step
    uint32_t* age;      // consecutive steps the stream was refused for lack of pool cells
    int* has_prev;      // time-step form: the stream holds a state from an earlier step
};

__device__ __forceinline__ int find_stream(const int* base, int ns, int item) {
    int lo = 0, hi = ns - 1;  // largest i with base[i] <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) kb_sanitize(const BStream* __restrict__ st,
                                                   const BTable* __restrict__ tb) {
    const int s = find_stream(tb->row_base, tb->ns, blockIdx.x);
    const BStream& b = st[s];
    if (!b.active) return;
    sanitize_row(b.lo_in, b.hi_in, b.W, b.D, blockIdx.x - tb->row_base[s], b.lo, b.hi, b.rowsum,
                 b.rowcells, b.rowcells + b.H);
}

__global__ void __launch_bounds__(512) kb_offsets(const BStream* __restrict__ st,
                                                  const BTable* __restrict__ tb) {
    const int s = find_stream(tb->row_base, tb->ns, blockIdx.x);
    const BStream& b = st[s];
    if (!b.active || *b.status != 0u) return;
    const int y = blockIdx.x - tb->row_base[s];
    offsets_row(b.lo, b.hi, b.rowsum, b.rowcells, b.rowcells + b.H, b.W, b.H, y, b.off, b.desc,
                b.cells, nullptr);
}

// Reservation of the volume pool, one block of kMaxStreams threads: each active stream needs the
// padded cells of its windows (the sum of its row totals), rounded up to 256 so that every
// stream's volumes stay 256-byte aligned; the streams are served longest-refused first (then in
// stream order), each taking the next free cells if they suffice and being refused otherwise
// (status 1: the step skips the stream).
__global__ void __launch_bounds__(kMaxStreams) kb_reserve(const BStream* __restrict__ st,
                                                          const BTable* __restrict__ tb) {
    __shared__ uint64_t need[kMaxStreams];
    __shared__ int order[kMaxStreams];
    __shared__ int n_active;
    const int ns = tb->ns, i = threadIdx.x;
    if (i == 0) n_active = 0;
    __syncthreads();
    const bool act = i < ns && st[i].active;
    if (act) {
        const BStream& b = st[i];
        uint64_t c = 0;
        for (int y = 0; y < b.H; ++y) c += b.rowsum[y];
        need[i] = (c + 255) & ~255ull;
        atomicAdd(&n_active, 1);
        const uint32_t a = tb->age[i];
        int r = 0;
        for (int j = 0; j < ns; ++j) {
            if (j == i || !st[j].active) continue;
            const uint32_t aj = tb->age[j];
            r += (aj > a || (aj == a && j < i)) ? 1 : 0;
        }
        order[r] = i;
    }
    __syncthreads();
    if (i == 0) {
        const uint64_t cap = st[0].capacity;
        uint64_t used = 0;
        for (int r = 0; r < n_active; ++r) {
            const int k = order[r];
            const bool fit = need[k] <= cap - used;
            *st[k].status = fit ? 0u : 1u;
            tb->base[k] = fit ? used : 0;
            tb->age[k] = fit ? 0u : tb->age[k] + 1u;
            if (fit) used += need[k];
        }
    }
}

template <int CW, int CH>
__global__ void __launch_bounds__(kCtW* kCtH) kb_census(const BStream* __restrict__ st,
                                                         const BTable* __restrict__ tb, int cw,
                                                         int ch) {
    const int s = find_stream(tb->tile_base, tb->ns, blockIdx.x);
    const BStream& b = st[s];
    if (!b.active) return;
    const int t = blockIdx.x - tb->tile_base[s];
    const int tx = t % tb->tiles_x[s], ty = t / tb->tiles_x[s];
    census_tile<CW, CH>(blockIdx.z ? b.right : b.left, b.W, b.H, cw, ch, tx * kCtW, ty * kCtH,
                        blockIdx.z ? b.censusR : b.censusL);
}

__global__ void __launch_bounds__(256) kb_cost(const BStream* __restrict__ st,
                                               const BTable* __restrict__ tb, int Bc) {
    const int ngroups = (gridDim.x * blockDim.x) / kCostLanes;
    const int sub = threadIdx.x % kCostLanes;
    const int total = tb->px_base[tb->ns];
    for (int gi = (blockIdx.x * blockDim.x + threadIdx.x) / kCostLanes; gi < total; gi += ngroups) {
        const int s = find_stream(tb->px_base, tb->ns, gi);
        const BStream& b = st[s];
        if (!b.active || *b.status != 0u) continue;
        cost_pixels(b.censusL, b.censusR, b.desc, b.W, b.n, Bc, b.C + tb->base[s],
                    gi - tb->px_base[s], sub, b.n);
    }
}

// persistent path aggregation: warps take items from a global counter until none is left; an item
// is what a warp walks together, NG = 32 / GL lines of one direction of one stream (see
// sgm_group_lines), every stream's horizontal lines (the longest chains) first. Lines are walked
// whole: the streams' lines fill the GPU many times over, so cutting them into segments would
// only add the segments' second walks (measured: 18.7 -> 18.2 ms a step without them)
template <int LPLW, int GL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, GL == 8 ? 24 / WARPS : 1) kb_sgm(const BStream* __restrict__ st,
                                                     const BTable* __restrict__ tb, int n_slots,
                                                     int P1, int P2, int* __restrict__ counter) {
    constexpr int NG = 32 / GL;
    extern __shared__ uint32_t sgm_smem32[];
    uint32_t* wsm = sgm_smem32 + (threadIdx.x >> 5) * grp_words_ng<LPLW, NG>();
    const int lane = threadIdx.x & 31;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= tb->total_items) return;
        int slot = 0;
        while (slot + 1 < n_slots && item >= tb->slot_base[slot + 1][0]) ++slot;
        const int s = find_stream(tb->slot_base[slot], tb->ns, item);
        const BStream& b = st[s];
        if (!b.active || *b.status != 0u) continue;
        const int code = slot;
        const int nlines = code <= 1 ? b.H : (code <= 3 ? b.W : b.W + b.H - 1);
        const uint64_t base = tb->base[s];
        sgm_group_lines<LPLW, GL>(b.C + base, b.desc, b.W, b.H, P1, P2, code,
                                  (item - tb->slot_base[slot][s]) * NG, nlines, 1,
                                  b.Lvol + (size_t)code * b.capacity + base, wsm);
    }
}

template <int NPATHS>
__global__ void __launch_bounds__(kSelThreads, 2) kb_select(const BStream* __restrict__ st,
                                                         const BTable* __restrict__ tb, int DP,
                                                         float s_thr, float r_min, int lr_tol) {
    extern __shared__ uint32_t sel_smem[];
    __shared__ int n_wide;
    const int s = find_stream(tb->row_base, tb->ns, blockIdx.x);
    const BStream& b = st[s];
    const int y = blockIdx.x - tb->row_base[s];
    if (!b.active) return;
    if (*b.status != 0u) {
        for (int x = threadIdx.x; x < b.W; x += blockDim.x) {
            b.Dz[y * b.W + x] = -1.0f;
            b.rz[y * b.W + x] = -1.0f;
        }
        return;
    }
    select_row<NPATHS>(b.Lvol + tb->base[s], b.capacity, b.desc, b.W, y, DP, s_thr, r_min, lr_tol, b.Dz, b.rz,
                       nullptr, nullptr, nullptr, nullptr, sel_smem, n_wide);
}

// ---- time-step form: one launch per stage over the pixels (256 per block) or rows of every
// active stream

// block b's stream and first pixel, or -1 when the stream sits the step out
__device__ __forceinline__ int px_block(const BStream* __restrict__ st, const BTable* __restrict__ tb,
                                        int& s) {
    s = find_stream(tb->pblk_base, tb->ns, blockIdx.x);
    return st[s].active ? ((int)blockIdx.x - tb->pblk_base[s]) * 256 : -1;
}

// Prediction, scatter (Eq. 3, z-buffer): streams with a previous state only.
__global__ void __launch_bounds__(256) kb_scatter(const BStream* __restrict__ st,
                                                  const BTable* __restrict__ tb) {
    int s;
    const int p0 = px_block(st, tb, s);
    const BStream& b = st[s];
    const int i = p0 + threadIdx.x;
    if (p0 < 0 || !tb->has_prev[s] || i >= b.n) return;
    warp_scatter_px(i, b.W, b.H, b.stateD, b.stateP, b.wp, b.keys);
}

// Prediction, gather and variance (Eq. 5-6); empties the z-buffer for the next step. Without a
// previous state: no prediction.
__global__ void __launch_bounds__(256) kb_gather(const BStream* __restrict__ st,
                                                 const BTable* __restrict__ tb) {
    int s;
    const int p0 = px_block(st, tb, s);
    const BStream& b = st[s];
    const int i = p0 + threadIdx.x;
    if (p0 < 0 || i >= b.n) return;
    if (tb->has_prev[s]) {
        const unsigned long long key = b.keys[i];
        b.keys[i] = kEmptyKey;
        warp_gather_px(i, key, b.stateD, b.stateP, b.q, b.predD, b.predP);
    } else {
        b.predD[i] = -1.0f;
        b.predP[i] = -1.0f;
    }
}

// Gap filling of the prediction (Eq. 7-8): the horizontal pass into the scratch maps, then the
// vertical one back into the prediction.
__global__ void __launch_bounds__(256) kb_fill_gaps(const BStream* __restrict__ st,
                                                    const BTable* __restrict__ tb, float gamma_f,
                                                    int vertical) {
    int s;
    const int p0 = px_block(st, tb, s);
    const BStream& b = st[s];
    const int i = p0 + threadIdx.x;
    if (p0 < 0 || !tb->has_prev[s] || i >= b.n) return;
    if (vertical)
        fill_gaps_px(i, b.W, b.H, b.tmpD, b.tmpP, gamma_f, 1, b.predD, b.predP);
    else
        fill_gaps_px(i, b.W, b.H, b.predD, b.predP, gamma_f, 0, b.tmpD, b.tmpP);
}

// Windows (Sec. 2.3), one block per row; full: every window the whole range.
__global__ void __launch_bounds__(256) kb_windows(const BStream* __restrict__ st,
                                                  const BTable* __restrict__ tb, float k,
                                                  int full) {
    const int s = find_stream(tb->row_base, tb->ns, blockIdx.x);
    const BStream& b = st[s];
    if (!b.active) return;
    const int y = blockIdx.x - tb->row_base[s];
    windows_row(b.predD, b.predP, b.W, b.D, k, y, b.lo, b.hi, b.rowsum, b.rowcells,
                b.rowcells + b.H, full != 0);
}

// Kalman update (Eq. 10-12) into the caller's maps and the stream's state. A stream refused by
// the pool keeps its state and its outputs as they were (its frame runs again in a later step).
__global__ void __launch_bounds__(256) kb_kalman(const BStream* __restrict__ st,
                                                 const BTable* __restrict__ tb) {
    int s;
    const int p0 = px_block(st, tb, s);
    const BStream& b = st[s];
    const int i = p0 + threadIdx.x;
    if (p0 < 0 || *b.status != 0u || i >= b.n) return;
    kalman_px(i, b.predD, b.predP, b.Dm, b.rm, b.outD, b.outP, b.stateD, b.stateP);
    if (i == 0) tb->has_prev[s] = 1;
}

struct SgmShape {
    int warps;   // warps per block
    int blocks;  // blocks per SM
};
const SgmShape kShapes[] = {{4, 4}, {4, 8}, {8, 2}, {8, 4}, {8, 6}, {16, 2}, {16, 3}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

using SgmKernel = void (*)(const BStream*, const BTable*, int, int, int, int*);

int lplw_for(int maxD) { return maxD <= 64 ? 2 : (maxD <= 128 ? 4 : 8); }

template <int LPLW, int GL>
SgmKernel sgm_kernel_lg(int warps) {
    return warps == 4 ? kb_sgm<LPLW, GL, 4> : (warps == 8 ? kb_sgm<LPLW, GL, 8> : kb_sgm<LPLW, GL, 16>);
}

template <int LPLW>
SgmKernel sgm_kernel_l(int gl, int warps) {
    if constexpr (LPLW == 8) return sgm_kernel_lg<LPLW, 8>(warps);  // see the 256-label rule
    else return gl == 4 ? sgm_kernel_lg<LPLW, 4>(warps) : sgm_kernel_lg<LPLW, 8>(warps);
}

SgmKernel sgm_kernel(int maxD, int gl, int warps) {
    switch (lplw_for(maxD)) {
        case 2: return sgm_kernel_l<2>(gl, warps);
        case 4: return sgm_kernel_l<4>(gl, warps);
        default: return sgm_kernel_l<8>(gl, warps);
    }
}

template <int LPLW>
int sgm_words(int gl) { return gl == 4 ? grp_words_ng<LPLW, 8>() : grp_words_ng<LPLW, 4>(); }

size_t sgm_smem_bytes(int maxD, int gl, int warps) {
    const int L = lplw_for(maxD);
    const int words = L == 2 ? sgm_words<2>(gl) : (L == 4 ? sgm_words<4>(gl) : sgm_words<8>(gl));
    return (size_t)warps * words * sizeof(uint32_t);
}

}  // namespace

struct tsgm_batch {
    tsgm_params prm;  // common parameters (width/height/d_max of stream 0)
    int ns = 0;
    std::vector<int> W, H, D;
    int maxW = 0, maxD = 0, sms = 152;
    cudaStream_t user = nullptr;
    cudaStream_t exec = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<void*> allocs;
    BStream* h_streams = nullptr;  // pinned host copy of the stream table
    BStream* d_streams = nullptr;
    BTable* h_table = nullptr;
    BTable* d_table = nullptr;
    int* d_counter = nullptr;
    cudaGraphExec_t fgraph = nullptr;  // the time-step form
    uint64_t pool_cells = 0;             // cells of the volume pool (per volume)
    uint32_t* d_status = nullptr;        // the streams' statuses (device), one array
    uint32_t* h_status = nullptr;        // pinned copy
    uint64_t full_need = 0, max_need = 0;  // cells of every stream / of the largest one at full range
    std::vector<uint8_t> seen;           // stream was active in a time step since create / reset
    std::string step_err;  // why the time-step form cannot run on these streams ("" if it can)
    int shape = 3;  // index into kShapes
    int cost_blocks = 8;  // blocks per SM of the cost kernel
    int gl = 8;     // lanes per path line in the aggregation (4: windows up to 16 labels in one step)
    bool shape_ok[kNumShapes] = {};  // the shape's shared memory fits a block
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev_sgm_a = nullptr, ev_sgm_b = nullptr;  // around the aggregation (profiled steps)
    uint64_t launches = 0;
    std::string err;
};

namespace {

tsgm_status bfail(tsgm_batch* b, tsgm_status s, const std::string& msg) {
    if (b) b->err = msg;
    return s;
}

tsgm_status bcuda(tsgm_batch* b, cudaError_t e, const char* where) {
    return bfail(b, TSGM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
bool balloc(tsgm_batch* b, T** p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) + 64) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    b->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return true;
}

// enqueue every stage of one batched step on b->exec (used for capture and for tuning)
cudaError_t enqueue_step(tsgm_batch* b, int shape, bool timed = false) {
    const tsgm_params& p = b->prm;
    cudaStream_t st = b->exec;
    const BTable& t = *b->h_table;
    cudaError_t e = cudaMemcpyAsync(b->d_streams, b->h_streams, sizeof(BStream) * b->ns,
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const int rows = t.row_base[b->ns];
    kb_sanitize<<<rows, 256, 0, st>>>(b->d_streams, b->d_table);
    kb_reserve<<<1, kMaxStreams, 0, st>>>(b->d_streams, b->d_table);
    kb_offsets<<<rows, 512, 0, st>>>(b->d_streams, b->d_table);
    {
        const dim3 cg(t.tile_base[b->ns], 1, 2), cb(kCtW, kCtH);
        if (p.census_w == 9 && p.census_h == 7)
            kb_census<9, 7><<<cg, cb, 0, st>>>(b->d_streams, b->d_table, p.census_w, p.census_h);
        else if (p.census_w == 5 && p.census_h == 5)
            kb_census<5, 5><<<cg, cb, 0, st>>>(b->d_streams, b->d_table, p.census_w, p.census_h);
        else
            kb_census<0, 0><<<cg, cb, 0, st>>>(b->d_streams, b->d_table, p.census_w, p.census_h);
    }
    kb_cost<<<b->sms * b->cost_blocks, 256, 0, st>>>(b->d_streams, b->d_table,
                                                     p.census_w * p.census_h - 1);
    if ((e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st)) != cudaSuccess) return e;
    if (timed && (e = cudaEventRecord(b->ev_sgm_a, st)) != cudaSuccess) return e;
    const SgmShape sh = kShapes[shape];
    const int grid = b->sms * sh.blocks;
    sgm_kernel(b->maxD, b->gl, sh.warps)<<<grid, sh.warps * 32,
                                           sgm_smem_bytes(b->maxD, b->gl, sh.warps), st>>>(
        b->d_streams, b->d_table, p.n_paths, p.P1, p.P2, b->d_counter);
    if (timed && (e = cudaEventRecord(b->ev_sgm_b, st)) != cudaSuccess) return e;
    const int DP = 256;
    const size_t sel_smem = (size_t)((4 * b->maxW + 1) & ~1) * 4 + (size_t)(kSelThreads / 32) * DP * 2;
    const float s_thr = p.S_max * (float)p.n_paths;
    if (p.n_paths == 8)
        kb_select<8><<<rows, kSelThreads, sel_smem, st>>>(b->d_streams, b->d_table, DP, s_thr,
                                                          p.r_min, p.lr_tol);
    else
        kb_select<4><<<rows, kSelThreads, sel_smem, st>>>(b->d_streams, b->d_table, DP, s_thr,
                                                          p.r_min, p.lr_tol);
    return cudaGetLastError();
}

tsgm_status capture(tsgm_batch* b) {
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->exec, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "begin capture");
    cudaError_t e2 = enqueue_step(b, b->shape);
    e = cudaStreamEndCapture(b->exec, &g);
    if (e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, e2, "capture step");
    }
    if (e != cudaSuccess) return bcuda(b, e, "end capture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(b, e, "instantiate graph");
    return TSGM_OK;
}

// enqueue every stage of one time step of all streams (Sec. 2) on b->exec: prediction (warp,
// gap filling), windows, census, cost, aggregation, selection, Kalman update
cudaError_t enqueue_frame_step(tsgm_batch* b, int shape) {
    const tsgm_params& p = b->prm;
    cudaStream_t st = b->exec;
    const BTable& t = *b->h_table;
    cudaError_t e = cudaMemcpyAsync(b->d_streams, b->h_streams, sizeof(BStream) * b->ns,
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const int rows = t.row_base[b->ns];
    const int pblocks = t.pblk_base[b->ns];
    kb_scatter<<<pblocks, 256, 0, st>>>(b->d_streams, b->d_table);
    kb_gather<<<pblocks, 256, 0, st>>>(b->d_streams, b->d_table);
    if (p.flags & TSGM_FLAG_FILL_GAPS) {
        kb_fill_gaps<<<pblocks, 256, 0, st>>>(b->d_streams, b->d_table, p.gamma_f, 0);
        kb_fill_gaps<<<pblocks, 256, 0, st>>>(b->d_streams, b->d_table, p.gamma_f, 1);
    }
    kb_windows<<<rows, 256, 0, st>>>(b->d_streams, b->d_table, p.sigma_mult,
                                     (p.flags & TSGM_FLAG_FULL_RANGE) ? 1 : 0);
    kb_reserve<<<1, kMaxStreams, 0, st>>>(b->d_streams, b->d_table);
    kb_offsets<<<rows, 512, 0, st>>>(b->d_streams, b->d_table);
    {
        const dim3 cg(t.tile_base[b->ns], 1, 2), cb(kCtW, kCtH);
        if (p.census_w == 9 && p.census_h == 7)
            kb_census<9, 7><<<cg, cb, 0, st>>>(b->d_streams, b->d_table, p.census_w, p.census_h);
        else if (p.census_w == 5 && p.census_h == 5)
            kb_census<5, 5><<<cg, cb, 0, st>>>(b->d_streams, b->d_table, p.census_w, p.census_h);
        else
            kb_census<0, 0><<<cg, cb, 0, st>>>(b->d_streams, b->d_table, p.census_w, p.census_h);
    }
    kb_cost<<<b->sms * b->cost_blocks, 256, 0, st>>>(b->d_streams, b->d_table,
                                                     p.census_w * p.census_h - 1);
    if ((e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st)) != cudaSuccess) return e;
    const SgmShape sh = kShapes[shape];
    sgm_kernel(b->maxD, b->gl, sh.warps)<<<b->sms * sh.blocks, sh.warps * 32,
                                           sgm_smem_bytes(b->maxD, b->gl, sh.warps), st>>>(
        b->d_streams, b->d_table, p.n_paths, p.P1, p.P2, b->d_counter);
    const int DP = 256;
    const size_t sel_smem = (size_t)((4 * b->maxW + 1) & ~1) * 4 + (size_t)(kSelThreads / 32) * DP * 2;
    const float s_thr = p.S_max * (float)p.n_paths;
    if (p.n_paths == 8)
        kb_select<8><<<rows, kSelThreads, sel_smem, st>>>(b->d_streams, b->d_table, DP, s_thr,
                                                          p.r_min, p.lr_tol);
    else
        kb_select<4><<<rows, kSelThreads, sel_smem, st>>>(b->d_streams, b->d_table, DP, s_thr,
                                                          p.r_min, p.lr_tol);
    kb_kalman<<<pblocks, 256, 0, st>>>(b->d_streams, b->d_table);
    return cudaGetLastError();
}

// kernels of one time step (the census counts as one: both images in one launch)
int frame_kernels(const tsgm_batch* b) {
    return 10 + ((b->prm.flags & TSGM_FLAG_FILL_GAPS) ? 2 : 0);
}

tsgm_status capture_frame(tsgm_batch* b) {
    if (b->fgraph) {
        cudaGraphExecDestroy(b->fgraph);
        b->fgraph = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->exec, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "begin capture");
    cudaError_t e2 = enqueue_frame_step(b, b->shape);
    e = cudaStreamEndCapture(b->exec, &g);
    if (e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, e2, "capture time step");
    }
    if (e != cudaSuccess) return bcuda(b, e, "end capture");
    e = cudaGraphInstantiate(&b->fgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(b, e, "instantiate graph");
    return TSGM_OK;
}

tsgm_status set_io(tsgm_batch* b, const uint8_t* const* left, const uint8_t* const* right,
                   const int16_t* const* d_lo, const int16_t* const* d_hi, float* const* D_z,
                   float* const* r_z) {
    if (!left || !right || !d_lo || !d_hi || !D_z || !r_z)
        return bfail(b, TSGM_ERR_INVALID_ARG, "tsgm_batch_match: null pointer array");
    for (int i = 0; i < b->ns; ++i) {
        if (!left[i] || !right[i] || !d_lo[i] || !d_hi[i] || !D_z[i] || !r_z[i])
            return bfail(b, TSGM_ERR_INVALID_ARG, "tsgm_batch_match: null pointer for stream " +
                                                      std::to_string(i));
        BStream& s = b->h_streams[i];
        s.left = left[i];
        s.right = right[i];
        s.lo_in = d_lo[i];
        s.hi_in = d_hi[i];
        s.Dz = D_z[i];
        s.rz = r_z[i];
        s.active = 1;
    }
    return TSGM_OK;
}

}  // namespace

namespace tsgm {

tsgm_status batch_create(const tsgm_params* streams, int32_t n_streams, int32_t max_labels,
                         uint64_t hbm_budget_bytes, void* cuda_stream, tsgm_batch** out) {
    if (!out) return TSGM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!streams || n_streams < 1 || n_streams > kMaxStreams) return TSGM_ERR_INVALID_ARG;
    const tsgm_params& p0 = streams[0];
    for (int i = 0; i < n_streams; ++i) {
        const tsgm_params& p = streams[i];
        if (p.census_w != p0.census_w || p.census_h != p0.census_h || p.n_paths != p0.n_paths ||
            p.P1 != p0.P1 || p.P2 != p0.P2 || p.S_max != p0.S_max || p.r_min != p0.r_min ||
            p.lr_tol != p0.lr_tol)
            return TSGM_ERR_INVALID_ARG;  // matching parameters must be shared by the batch
        if (p.width < 1 || p.height < 1 || p.width > 13000 || p.d_max < 0 || p.d_max > 255)
            return TSGM_ERR_INVALID_ARG;
        if (p.census_w * p.census_h - 1 + p.P2 > 255 || p.P1 < 0 || p.P2 < p.P1)
            return TSGM_ERR_INVALID_ARG;
        if (p.census_w < 1 || p.census_h < 1 || !(p.census_w & 1) || !(p.census_h & 1) ||
            p.census_w > 15 || p.census_h > 15 || p.census_w * p.census_h - 1 > 64 ||
            (p.n_paths != 4 && p.n_paths != 8))
            return TSGM_ERR_INVALID_ARG;
        // a stream's cell offsets are 32-bit
        if ((uint64_t)p.width * p.height * (uint64_t)((p.d_max + 4) & ~3) > 0xFFFFFF00ull)
            return TSGM_ERR_INVALID_ARG;
    }
    size_t free0 = 0, total0 = 0;
    cudaMemGetInfo(&free0, &total0);
    tsgm_batch* b = new (std::nothrow) tsgm_batch();
    if (!b) return TSGM_ERR_OUT_OF_MEMORY;
    b->prm = p0;
    // the time-step form runs one prediction and window rule over all streams
    for (int i = 0; i < n_streams && b->step_err.empty(); ++i) {
        const tsgm_params& p = streams[i];
        if (p.flags != p0.flags || p.gamma_f != p0.gamma_f || p.sigma_mult != p0.sigma_mult)
            b->step_err = "tsgm_batch_frame: flags, gamma_f and sigma_mult differ across streams";
        else if (!(p.q >= 0.0f && p.q <= FLT_MAX) || !(p.sigma_mult >= 0.0f && p.sigma_mult <= FLT_MAX))
            b->step_err = "tsgm_batch_frame: q and sigma_mult must be finite and >= 0";
    }
    b->ns = n_streams;
    b->user = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    bool ok = cudaStreamCreateWithFlags(&b->exec, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreate(&b->ev_sgm_a) == cudaSuccess && cudaEventCreate(&b->ev_sgm_b) == cudaSuccess &&
              cudaMallocHost((void**)&b->h_streams, sizeof(BStream) * n_streams) == cudaSuccess &&
              cudaMallocHost((void**)&b->h_table, sizeof(BTable)) == cudaSuccess;
    ok = ok && balloc(b, &b->d_streams, n_streams) && balloc(b, &b->d_table, 1) &&
         balloc(b, &b->d_counter, 1);
    if (ok) {
        std::memset(b->h_streams, 0, sizeof(BStream) * n_streams);
        std::memset(b->h_table, 0, sizeof(BTable));
        BTable& t = *b->h_table;
        t.ns = n_streams;
        uint64_t full_need = 0, max_need = 0;
        // the streams' step statuses side by side (read back with one copy)
        ok = balloc(b, &b->d_status, (size_t)n_streams) &&
             cudaMallocHost((void**)&b->h_status, sizeof(uint32_t) * n_streams) == cudaSuccess;
        for (int i = 0; i < n_streams && ok; ++i) {
            const tsgm_params& p = streams[i];
            BStream& s = b->h_streams[i];
            s.W = p.width;
            s.H = p.height;
            s.D = p.d_max + 1;
            s.n = p.width * p.height;
            const int lab = (max_labels > 0 && max_labels < s.D) ? max_labels : s.D;
            const uint64_t full_i = ((uint64_t)s.n * (uint64_t)((s.D + 3) & ~3) + 255) & ~255ull;
            b->pool_cells += ((uint64_t)s.n * (uint64_t)((lab + 3) & ~3) + 255) & ~255ull;
            full_need += full_i;
            max_need = std::max<uint64_t>(max_need, full_i);
            b->W.push_back(s.W);
            b->H.push_back(s.H);
            b->D.push_back(s.D);
            b->maxW = std::max(b->maxW, s.W);
            b->maxD = std::max(b->maxD, s.D);
            const size_t n = (size_t)s.n;
            s.status = b->d_status + i;
            ok = balloc(b, &s.lo, n) && balloc(b, &s.hi, n) && balloc(b, &s.censusL, n) &&
                 balloc(b, &s.censusR, n) && balloc(b, &s.desc, n) && balloc(b, &s.off, n + 1) &&
                 balloc(b, &s.rowsum, (size_t)s.H) && balloc(b, &s.rowcells, 2 * (size_t)s.H) &&
                 balloc(b, &s.cells, 2) &&
                 // time-step form: z-buffer, state, prediction and its scratch, matched maps
                 balloc(b, &s.keys, n) && balloc(b, &s.stateD, n) && balloc(b, &s.stateP, n) &&
                 balloc(b, &s.predD, n) && balloc(b, &s.predP, n) && balloc(b, &s.tmpD, n) &&
                 balloc(b, &s.tmpP, n) && balloc(b, &s.Dm, n) && balloc(b, &s.rm, n) &&
                 cudaMemset(s.keys, 0xFF, n * sizeof(unsigned long long)) == cudaSuccess;
            s.q = p.q;
            t.row_base[i + 1] = t.row_base[i] + s.H;
            t.tiles_x[i] = (s.W + kCtW - 1) / kCtW;
            t.tile_base[i + 1] = t.tile_base[i] + t.tiles_x[i] * ((s.H + kCtH - 1) / kCtH);
            t.px_base[i + 1] = t.px_base[i] + s.n;
            t.pblk_base[i + 1] = t.pblk_base[i] + (s.n + 255) / 256;
        }
        // lines per warp: windows of up to 16 labels fit the 4-lane groups (8 lines per warp),
        // wider ones (up to 32 in one step) the 8-lane groups
        // (256 labels: always the 8-lane groups, as in the single-image aggregation)
        b->gl = (max_labels > 0 && max_labels <= 16 && b->maxD <= 128) ? 4 : 8;
        const int NG = 32 / b->gl;
        // direction-major line order: every stream's horizontal lines first
        int item = 0;
        for (int slot = 0; slot < p0.n_paths; ++slot) {
            for (int i = 0; i < n_streams; ++i) {
                t.slot_base[slot][i] = item;
                const BStream& s = b->h_streams[i];
                const int code = slot;
                const int nl = code <= 1 ? s.H : (code <= 3 ? s.W : s.W + s.H - 1);
                item += (nl + NG - 1) / NG;
            }
            t.slot_base[slot][n_streams] = item;
        }
        t.total_items = item;
        // the volume pool: with a budget, what the budget leaves after everything above (at
        // least one full-range stream, at most all streams at full range)
        b->full_need = full_need;
        b->max_need = max_need;
        if (ok && hbm_budget_bytes > 0) {
            size_t f1 = 0, t1 = 0;
            cudaMemGetInfo(&f1, &t1);
            const uint64_t used = free0 > f1 ? (uint64_t)(free0 - f1) : 0;
            const uint64_t left = hbm_budget_bytes > used ? hbm_budget_bytes - used : 0;
            b->pool_cells = (left / (uint64_t)(1 + p0.n_paths)) & ~255ull;
            b->pool_cells = std::min(std::max(b->pool_cells, max_need), full_need);
        }
        uint8_t* pool_C = nullptr;
        uint8_t* pool_L = nullptr;
        ok = ok && balloc(b, &pool_C, (size_t)b->pool_cells + 64) &&
             balloc(b, &pool_L, (size_t)b->pool_cells * p0.n_paths + 64) &&
             balloc(b, &t.base, (size_t)n_streams) && balloc(b, &t.age, (size_t)n_streams) &&
             balloc(b, &t.has_prev, (size_t)n_streams) &&
             cudaMemset(t.age, 0, sizeof(uint32_t) * n_streams) == cudaSuccess &&
             cudaMemset(t.has_prev, 0, sizeof(int) * n_streams) == cudaSuccess &&
             cudaMemset(t.base, 0, sizeof(uint64_t) * n_streams) == cudaSuccess;
        for (int i = 0; i < n_streams && ok; ++i) {
            BStream& s = b->h_streams[i];
            s.C = pool_C;
            s.Lvol = pool_L;
            s.capacity = b->pool_cells;
            ok = cudaMemset(s.status, 0, sizeof(uint32_t)) == cudaSuccess;
        }
        b->seen.assign((size_t)n_streams, 0);
        ok = ok && cudaMemcpy(b->d_table, b->h_table, sizeof(BTable), cudaMemcpyHostToDevice) == cudaSuccess;
        int smem_max = 48 * 1024;
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        int first_ok = -1;
        for (int k = 0; ok && k < kNumShapes; ++k) {
            const size_t sm = sgm_smem_bytes(b->maxD, b->gl, kShapes[k].warps);
            if (sm > (size_t)smem_max) continue;  // does not fit: never launched
            if (sm > 48 * 1024)
                ok = cudaFuncSetAttribute(sgm_kernel(b->maxD, b->gl, kShapes[k].warps),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm) == cudaSuccess;
            b->shape_ok[k] = ok;
            if (ok && first_ok < 0) first_ok = k;
        }
        if (first_ok < 0) ok = false;
        if (ok && !b->shape_ok[b->shape]) b->shape = first_ok;
        const size_t sel_smem = (size_t)((4 * b->maxW + 1) & ~1) * 4 + (size_t)(kSelThreads / 32) * 256 * 2;
        if (ok && sel_smem > 48 * 1024) {
            ok = cudaFuncSetAttribute(kb_select<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sel_smem) == cudaSuccess &&
                 cudaFuncSetAttribute(kb_select<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sel_smem) == cudaSuccess;
        }
    }
    if (!ok) {
        cudaGetLastError();
        tsgm_batch_destroy(b);
        return TSGM_ERR_OUT_OF_MEMORY;
    }
    *out = b;
    return TSGM_OK;
}

}  // namespace tsgm

extern "C" {

tsgm_status tsgm_batch_create(const tsgm_params* streams, int32_t n_streams, int32_t max_labels,
                              void* cuda_stream, tsgm_batch** out) {
    return tsgm::batch_create(streams, n_streams, max_labels, 0, cuda_stream, out);
}

void tsgm_batch_destroy(tsgm_batch* b) {
    if (!b) return;
    if (b->exec) cudaStreamSynchronize(b->exec);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->fgraph) cudaGraphExecDestroy(b->fgraph);
    for (void* q : b->allocs) cudaFree(q);
    if (b->h_streams) cudaFreeHost(b->h_streams);
    if (b->h_table) cudaFreeHost(b->h_table);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->ev_sgm_a) cudaEventDestroy(b->ev_sgm_a);
    if (b->ev_sgm_b) cudaEventDestroy(b->ev_sgm_b);
    if (b->exec) cudaStreamDestroy(b->exec);
    delete b;
}

const char* tsgm_batch_last_error(const tsgm_batch* b) { return b ? b->err.c_str() : "null batch"; }

tsgm_status tsgm_batch_match(tsgm_batch* b, const uint8_t* const* left,
                             const uint8_t* const* right, const int16_t* const* d_lo,
                             const int16_t* const* d_hi, float* const* D_z, float* const* r_z) {
    if (!b) return TSGM_ERR_INVALID_ARG;
    // the graph reads the pinned table when it runs: wait for the previous replay before
    // rewriting it
    cudaError_t e = cudaEventSynchronize(b->ev_out);
    if (e != cudaSuccess) return bcuda(b, e, "previous batch step");
    tsgm_status s = set_io(b, left, right, d_lo, d_hi, D_z, r_z);
    if (s != TSGM_OK) return s;
    if (!b->graph && (s = capture(b)) != TSGM_OK) return s;
    if ((e = cudaEventRecord(b->ev_in, b->user)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->exec, b->ev_in, 0)) != cudaSuccess ||
        (e = cudaGraphLaunch(b->graph, b->exec)) != cudaSuccess ||
        (e = cudaEventRecord(b->ev_out, b->exec)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->user, b->ev_out, 0)) != cudaSuccess)
        return bcuda(b, e, "batch step");
    b->launches += 7;
    return TSGM_OK;
}

tsgm_status tsgm_batch_autotune(tsgm_batch* b, const uint8_t* const* left,
                                const uint8_t* const* right, const int16_t* const* d_lo,
                                const int16_t* const* d_hi, float* const* D_z, float* const* r_z,
                                int32_t reps, double* best_ms, int32_t* best_shape) {
    if (!b) return TSGM_ERR_INVALID_ARG;
    tsgm_status s = set_io(b, left, right, d_lo, d_hi, D_z, r_z);
    if (s != TSGM_OK) return s;
    if (reps < 1) reps = 3;
    cudaError_t e = cudaEventSynchronize(b->ev_out);
    if (e != cudaSuccess) return bcuda(b, e, "previous batch step");
    cudaEvent_t a = nullptr, z = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&z);
    double best = 1e30;
    int best_i = b->shape;
    for (int i = 0; i < kNumShapes; ++i) {
        if (!b->shape_ok[i]) continue;
        e = enqueue_step(b, i);  // warm-up
        if (e != cudaSuccess) break;
        cudaEventRecord(a, b->exec);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue_step(b, i);
        cudaEventRecord(z, b->exec);
        if (e == cudaSuccess) e = cudaEventSynchronize(z);
        float ms = 0.0f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, z);
        if (e == cudaSuccess && ms / reps < best) {
            best = ms / reps;
            best_i = i;
        }
    }
    b->shape = best_i;
    // then the cost kernel's grid (blocks per SM), with the chosen aggregation shape
    int best_c = b->cost_blocks;
    for (int cb : {2, 4, 8, 16}) {
        if (e != cudaSuccess) break;
        b->cost_blocks = cb;
        e = enqueue_step(b, best_i);  // warm-up
        if (e != cudaSuccess) break;
        cudaEventRecord(a, b->exec);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue_step(b, best_i);
        cudaEventRecord(z, b->exec);
        if (e == cudaSuccess) e = cudaEventSynchronize(z);
        float ms = 0.0f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, z);
        if (e == cudaSuccess && ms / reps < best) {
            best = ms / reps;
            best_c = cb;
        }
    }
    b->cost_blocks = best_c;
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    if (e != cudaSuccess) return bcuda(b, e, "autotune");
    if (b->fgraph) {  // the time-step form is captured again with the new shape when next used
        cudaGraphExecDestroy(b->fgraph);
        b->fgraph = nullptr;
    }
    if ((s = capture(b)) != TSGM_OK) return s;
    if (best_ms) *best_ms = best;
    if (best_shape) *best_shape = best_i;
    return TSGM_OK;
}

tsgm_status tsgm_batch_cells(tsgm_batch* b, uint64_t* cells, int32_t* overflowed) {
    if (!b || !cells) return TSGM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(b->exec);
    if (e != cudaSuccess) return bcuda(b, e, "synchronize");
    uint64_t tot = 0;
    int32_t over = 0;
    for (int i = 0; i < b->ns; ++i) {
        if (!b->h_streams[i].active) continue;  // sat the last step out
        uint32_t c = 0, st = 0;
        if (cudaMemcpy(&st, b->h_streams[i].status, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            (st == 0u &&
             cudaMemcpy(&c, b->h_streams[i].cells, 4, cudaMemcpyDeviceToHost) != cudaSuccess))
            return bfail(b, TSGM_ERR_CUDA, "tsgm_batch_cells: copy");
        tot += c;
        over += st != 0u;
    }
    *cells = tot;
    if (overflowed) *overflowed = over;
    return TSGM_OK;
}

tsgm_status tsgm_batch_stream_status(tsgm_batch* b, int32_t* status) {
    if (!b || !status) return TSGM_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(b->h_status, b->d_status, sizeof(uint32_t) * b->ns,
                                    cudaMemcpyDeviceToHost, b->exec);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->exec);
    if (e != cudaSuccess) return bcuda(b, e, "tsgm_batch_stream_status");
    for (int i = 0; i < b->ns; ++i)
        status[i] = !b->h_streams[i].active ? 1 : (b->h_status[i] ? 2 : 0);
    return TSGM_OK;
}

tsgm_status tsgm_batch_pool(tsgm_batch* b, uint64_t* pool_cells, uint64_t* largest_full_range) {
    if (!b || !pool_cells) return TSGM_ERR_INVALID_ARG;
    *pool_cells = b->pool_cells;
    if (largest_full_range) *largest_full_range = b->max_need;
    return TSGM_OK;
}

tsgm_status tsgm_batch_profile(tsgm_batch* b, const uint8_t* const* left,
                               const uint8_t* const* right, const int16_t* const* d_lo,
                               const int16_t* const* d_hi, float* const* D_z, float* const* r_z,
                               float* sgm_ms, float* step_ms) {
    if (!b || !sgm_ms || !step_ms) return TSGM_ERR_INVALID_ARG;
    tsgm_status s = set_io(b, left, right, d_lo, d_hi, D_z, r_z);
    if (s != TSGM_OK) return s;
    cudaError_t e = cudaEventSynchronize(b->ev_out);
    cudaEvent_t a = nullptr, z = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&z);
    if (e == cudaSuccess) e = cudaEventRecord(a, b->exec);
    if (e == cudaSuccess) e = enqueue_step(b, b->shape, true);
    if (e == cudaSuccess) e = cudaEventRecord(z, b->exec);
    if (e == cudaSuccess) e = cudaEventSynchronize(z);
    if (e == cudaSuccess) e = cudaEventElapsedTime(sgm_ms, b->ev_sgm_a, b->ev_sgm_b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(step_ms, a, z);
    if (a) cudaEventDestroy(a);
    if (z) cudaEventDestroy(z);
    if (e != cudaSuccess) return bcuda(b, e, "tsgm_batch_profile");
    b->launches += 7;
    return TSGM_OK;
}

tsgm_status tsgm_batch_frame(tsgm_batch* b, const uint8_t* const* left,
                             const uint8_t* const* right, const float* R, const float* t,
                             const float* K, const float* baseline, float* const* D,
                             float* const* P) {
    if (!b) return TSGM_ERR_INVALID_ARG;
    const tsgm_params& p = b->prm;
    if (!b->step_err.empty()) return bfail(b, TSGM_ERR_INVALID_ARG, b->step_err);
    if (b->pool_cells < b->max_need)
        return bfail(b, TSGM_ERR_INVALID_ARG,
                     "tsgm_batch_frame: the volume pool cannot hold the largest stream at full "
                     "range (a first frame); create the batch with max_labels = 0");
    if (p.flags & (TSGM_FLAG_EDGE_REJECT | TSGM_FLAG_PRED_LR_CHECK | TSGM_FLAG_SAD_CHECK))
        return bfail(b, TSGM_ERR_UNIMPLEMENTED,
                     "tsgm_batch_frame: edge rejection and the consistency checks of the "
                     "prediction and update are not in the batched step");
    if (!left || !right || !K || !baseline || !D || !P)
        return bfail(b, TSGM_ERR_INVALID_ARG, "tsgm_batch_frame: null pointer array");
    // every argument is checked before anything is changed or enqueued
    std::vector<WarpParams> wps((size_t)b->ns);
    for (int i = 0; i < b->ns; ++i) {
        if (!left[i] && !right[i]) continue;  // this stream sits the step out
        if (!left[i] || !right[i] || !D[i] || !P[i])
            return bfail(b, TSGM_ERR_INVALID_ARG,
                         "tsgm_batch_frame: null pointer for stream " + std::to_string(i));
        if (D[i] == P[i])
            return bfail(b, TSGM_ERR_INVALID_ARG,
                         "tsgm_batch_frame: D and P alias for stream " + std::to_string(i));
        const float* Ki = K + 9 * i;
        wps[i].cx = Ki[2];
        wps[i].cy = Ki[5];
        if (b->seen[i]) {
            if (!R || !t)
                return bfail(b, TSGM_ERR_INVALID_ARG,
                             "tsgm_batch_frame: poses required after a stream's first frame");
            if (tsgm_build_H(R + 9 * i, t + 3 * i, Ki, baseline[i], wps[i].h) != TSGM_OK)
                return bfail(b, TSGM_ERR_INVALID_ARG,
                             "tsgm_batch_frame: invalid pose or calibration for stream " +
                                 std::to_string(i));
        }
    }
    cudaError_t e = cudaEventSynchronize(b->ev_out);
    if (e != cudaSuccess) return bcuda(b, e, "previous batch step");
    for (int i = 0; i < b->ns; ++i) {
        BStream& hs = b->h_streams[i];
        hs.active = left[i] ? 1 : 0;
        if (!hs.active) continue;
        hs.left = left[i];
        hs.right = right[i];
        hs.outD = D[i];
        hs.outP = P[i];
        hs.Dz = hs.Dm;
        hs.rz = hs.rm;
        hs.wp = wps[i];
    }
    tsgm_status s;
    if (!b->fgraph && (s = capture_frame(b)) != TSGM_OK) return s;
    if ((e = cudaEventRecord(b->ev_in, b->user)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->exec, b->ev_in, 0)) != cudaSuccess ||
        (e = cudaGraphLaunch(b->fgraph, b->exec)) != cudaSuccess ||
        (e = cudaEventRecord(b->ev_out, b->exec)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->user, b->ev_out, 0)) != cudaSuccess)
        return bcuda(b, e, "batch time step");
    b->launches += frame_kernels(b);
    for (int i = 0; i < b->ns; ++i)
        if (b->h_streams[i].active) b->seen[i] = 1;
    return TSGM_OK;
}

tsgm_status tsgm_batch_reset(tsgm_batch* b) {
    if (!b) return TSGM_ERR_INVALID_ARG;
    cudaError_t e = cudaEventSynchronize(b->ev_out);
    if (e != cudaSuccess) return bcuda(b, e, "previous batch step");
    e = cudaMemsetAsync(b->h_table->has_prev, 0, sizeof(int) * b->ns, b->exec);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->exec);
    if (e != cudaSuccess) return bcuda(b, e, "tsgm_batch_reset");
    std::fill(b->seen.begin(), b->seen.end(), 0);
    return TSGM_OK;
}

tsgm_status tsgm_batch_launches(tsgm_batch* b, uint64_t* n) {
    if (!b || !n) return TSGM_ERR_INVALID_ARG;
    *n = b->launches;
    return TSGM_OK;
}

}  // extern "C"
