/*
 * tsgm — temporal SGM in an ego-motion-reduced disparity search space, GB300 (sm_103a).
 *
 * C ABI of the data-parallel hot path of Fucek, Markovic, Cvisic, Petrovic, "Dense Disparity
 * Estimation in Ego-motion Reduced Search Space" (arXiv 1708.06301):
 *   disparity prediction  (Sec. 2.2, Eq. 3, 5, 6)  -> tsgm_warp_predict
 *   reduced search space  (Sec. 2.3)               -> tsgm_windows
 *   stereo matching       (Sec. 2.3, 2.4, Eq. 9)   -> tsgm_match
 *   disparity update      (Sec. 2.4, Eq. 10-12)    -> tsgm_kalman_update
 *   one whole time step   (Sec. 2, steps 2-4)      -> tsgm_frame / tsgm_frame_host
 *
 * Conventions (all calls):
 *   - Image and map pointers are DEVICE pointers (except tsgm_frame_host, tsgm_build_H and the
 *     state export/import), caller-owned, dense row-major with pitch = width; pixel index
 *     i = y * width + x. uint8 images; float32 disparity (px) and variance (px^2) maps.
 *   - An invalid disparity or variance is -1.0f. A map value is valid iff it is finite and >= 0.
 *   - A disparity window is [d_lo, d_hi] inclusive, int16, inside [0, d_max].
 *   - Calls are asynchronous on the context's CUDA stream unless stated otherwise; outputs are
 *     ready when that stream reaches the point of the call. Inputs must stay valid until then.
 *   - Every call returns a tsgm_status; on failure tsgm_last_error() gives a message. No call
 *     throws across the ABI. A context is not thread-safe: one host thread at a time.
 *   - The context owns every scratch buffer, allocated once in tsgm_create for the maximum
 *     problem (width x height pixels x (d_max + 1) labels); no call allocates device memory
 *     afterwards (tsgm_frame_host uses pinned staging allocated at create time too).
 *   - Pose convention (Eq. 2): M^k = R M^{k-1} + t maps previous-frame camera coordinates to
 *     current ones; R row-major 3x3, t in metres; forward motion by s gives t = (0, 0, -s).
 *     K is the row-major 3x3 intrinsic matrix; f = K[0], cx = K[2], cy = K[5].
 */
#ifndef TSGM_H
#define TSGM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSGM_MAX_LABELS 256   /* d_max + 1 <= 256 */
#define TSGM_MAX_CENSUS_BITS 64

typedef struct tsgm_ctx tsgm_ctx;

typedef enum {
    TSGM_OK = 0,
    TSGM_ERR_INVALID_ARG = 1,   /* null pointer, bad size or parameter; nothing was launched */
    TSGM_ERR_OUT_OF_MEMORY = 2, /* tsgm_create could not allocate its buffers */
    TSGM_ERR_CUDA = 3,          /* a CUDA call failed; message in tsgm_last_error */
    TSGM_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    TSGM_ERR_STATE = 5,         /* call not valid in the current state (e.g. no previous frame) */
    TSGM_ERR_UNIMPLEMENTED = 6
} tsgm_status;

/* Flags for tsgm_params.flags */
#define TSGM_FLAG_KEEP_INTERNALS 1u  /* also write d*, right-view disparities and the LR mask of
                                        the last tsgm_match into context buffers (tsgm_inspect) */
#define TSGM_FLAG_FULL_RANGE 2u      /* tsgm_frame ignores the prediction when choosing windows:
                                        plain full-range SGM every frame (still Kalman-updated) */
#define TSGM_FLAG_FILL_GAPS 4u       /* tsgm_frame fills one-pixel gaps of the prediction
                                        (Sec. 2.2, Eq. 7-8) before choosing the windows */
#define TSGM_FLAG_EDGE_REJECT 8u     /* tsgm_frame rejects predicted pixels next to a disparity
                                        discontinuity (Sec. 2.2, disparity refinement), before
                                        the gap filling */
#define TSGM_FLAG_PRED_LR_CHECK 16u  /* tsgm_frame checks the prediction against the right view's
                                        prediction (Sec. 2.2, Fig. 3(d)), after the gap filling */
#define TSGM_FLAG_SAD_CHECK 32u      /* tsgm_frame rejects pixels of the updated map whose left /
                                        right patch SAD is high (Sec. 2.4), after the update */

typedef struct {
    int32_t width, height;       /* image size, 1 <= width <= 13000, 1 <= height */
    int32_t d_max;               /* labels are 0..d_max; d_max + 1 <= TSGM_MAX_LABELS */
    int32_t census_w, census_h;  /* odd census window; census_w * census_h - 1 <= 64 */
    int32_t n_paths;             /* SGM paths: 4 (->, <-, down, up) or 8 (+ 4 diagonals) */
    int32_t P1, P2;              /* SGM penalties, 0 <= P1 <= P2, census bits + P2 <= 255 */
    float sigma_mult;            /* window half-width in standard deviations (Sec. 2.3: 3) */
    float q;                     /* ego-motion variance in disparity space, px^2 (Eq. 5) */
    float S_max;                 /* matching-variance threshold per path (Eq. 9, Sec. 2.3) */
    float r_min;                 /* floor of the matching variance r, px^2 */
    int32_t lr_tol;              /* left-right check tolerance in px (Sec. 2.4) */
    uint32_t flags;              /* TSGM_FLAG_* */
    float gamma_f;               /* similarity threshold of the gap filling (Eq. 8), px */
    float edge_thr;              /* discontinuity threshold of the edge rejection, px */
    float pred_lr_tol;           /* similarity threshold of the prediction's left-right check, px */
    int32_t sad_w, sad_h;        /* SAD check patch, odd sizes 1 .. 31 */
    float sad_thr;               /* SAD check: mean absolute difference per patch pixel, grey levels */
} tsgm_params;

/* Fill *p with the defaults: d_max 127, census 9x7, 8 paths, P1 8, P2 32, sigma_mult 3,
 * q 0.25, S_max 10, r_min 0.5, lr_tol 1, flags 0, gamma_f 1, edge_thr 1, pred_lr_tol 1,
 * SAD patch 5x5, sad_thr 30. */
void tsgm_default_params(tsgm_params* p, int32_t width, int32_t height);

/* Create a context. `cuda_stream` is the cudaStream_t every call of the context is enqueued on
 * (NULL: the legacy default stream). Allocates all device scratch for the given size. Errors:
 * INVALID_ARG (bad parameters), OUT_OF_MEMORY, CUDA. On failure *out is set to NULL. */
tsgm_status tsgm_create(const tsgm_params* p, void* cuda_stream, tsgm_ctx** out);

/* Release all resources. Synchronises the context stream first. NULL is ignored. */
void tsgm_destroy(tsgm_ctx* ctx);

/* Message of the last failed call on this context (static storage owned by the context). */
const char* tsgm_last_error(const tsgm_ctx* ctx);

/* Use another CUDA stream for subsequent calls (NULL: the legacy default stream). */
tsgm_status tsgm_set_stream(tsgm_ctx* ctx, void* cuda_stream);

/* Host-side: the disparity-space homography H = Gamma T Gamma^{-1} (Sec. 2.1, Eq. 1-4) in
 * binary64, returned as row-major 4x4 rounded to binary32. x, y are measured from the
 * principal point. Errors: INVALID_ARG for null pointers, f <= 0 or baseline <= 0. */
tsgm_status tsgm_build_H(const float R[9], const float t[3], const float K[9], float baseline,
                         float H_out[16]);

/* Disparity prediction (Sec. 2.2): warp prev_D by the pose in disparity space (Eq. 3, with the
 * homogeneous divide), resolve collisions by keeping the highest predicted disparity (ties: the
 * lowest source index), predict the variance p = Phi^2 p + q with Phi = d'/d (Eq. 5-6).
 * Sources with an invalid d or p, or d <= 0, are skipped; unreached targets are invalid.
 * prev_D, prev_P: width*height floats (inputs); pred_D, pred_P: width*height floats (outputs,
 * must not alias the inputs). The z-buffer keys stay in the context (tsgm_inspect). */
tsgm_status tsgm_warp_predict(tsgm_ctx* ctx, const float* prev_D, const float* prev_P,
                              const float R[9], const float t[3], const float K[9],
                              float baseline, float* pred_D, float* pred_P);

/* Gap filling of a prediction (Sec. 2.2, Eq. 7-8), in place: an invalid pixel whose two
 * horizontal neighbours are valid with |d_l - d_r| < gamma_f takes their mean disparity and mean
 * variance; then the same with the vertical neighbours on the horizontally filled map. Each pass
 * reads the map as it was before the pass. Uses the context's D_z/r_z buffers as scratch. */
tsgm_status tsgm_fill_gaps(tsgm_ctx* ctx, float* pred_D, float* pred_P);

/* Edge rejection of a prediction (Sec. 2.2, disparity refinement), in place: a valid pixel whose
 * 8-neighbourhood (inside the image) holds a valid prediction differing by at least edge_thr
 * becomes invalid (-1 in both maps); invalid neighbours do not count. The pass reads the map as it
 * was before it. Uses the context's D_z/r_z buffers as scratch. */
tsgm_status tsgm_edge_reject(tsgm_ctx* ctx, float* pred_D, float* pred_P);

/* Left-right consistency check of a prediction (Sec. 2.2, Sec. 3 and Fig. 3(d); the paper leaves
 * the right view's propagation open: here it is formed from the left prediction). In place on
 * the device maps pred_D, pred_P (W x H, row-major, -1 = invalid). Every valid pixel (x, y, d)
 * lands on the right view's pixel x - round(d) of its row, round(d) = floor(d + 1/2) in binary32,
 * and the right view keeps the largest disparity landing on each pixel; a valid pixel stays valid
 * when its landing pixel is inside the image and holds a disparity within pred_lr_tol of its own,
 * else it becomes -1 in both maps (seen by one camera only, or hidden behind a nearer surface). */
tsgm_status tsgm_pred_lr_check(tsgm_ctx* ctx, float* pred_D, float* pred_P);

/* SAD check (Sec. 2.4, disparity consistency check) on an updated map, in place on the device
 * maps D, P with the device images left, right (uint8, W x H): the sum of absolute differences
 * between the sad_w x sad_h patch of the left image around (x, y) and the right image's patch
 * around (x - round(d), y), coordinates clamped into the image; a valid pixel whose SAD is above
 * sad_thr * sad_w * sad_h (binary32) becomes -1 in both maps, so that the next image searches it
 * over the whole range. */
tsgm_status tsgm_sad_check(tsgm_ctx* ctx, const uint8_t* left, const uint8_t* right, float* D,
                           float* P);

/* Reduced search space (Sec. 2.3): d_lo = max(0, floor(d - k sqrt(p))), d_hi = min(d_max,
 * ceil(d + k sqrt(p))) with k = sigma_mult, binary32; the whole range [0, d_max] where the
 * prediction is invalid or the interval misses [0, d_max]. Also builds the ragged-volume
 * offsets in the context. If n_cells_host is not NULL the call synchronises the stream and
 * writes the number of (pixel, disparity) cells, sum of the window lengths. */
tsgm_status tsgm_windows(tsgm_ctx* ctx, const float* pred_D, const float* pred_P,
                         int16_t* d_lo, int16_t* d_hi, uint64_t* n_cells_host);

/* Stereo matching restricted to the windows (Sec. 2.3-2.4): census transform of both images,
 * Hamming cost per window cell (x - d < 0 costs all census bits), SGM path aggregation with
 * penalties P1/P2 over n_paths directions where a neighbour's disparities outside its own
 * window do not exist, winner-takes-all (lowest d on ties), parabolic sub-pixel refinement,
 * matching variance r = n_l + n_r (Eq. 9, aggregated-cost reading, floored at r_min), and the
 * left-right check. left, right: uint8 images; d_lo, d_hi: windows, copied into the context
 * and clamped there to 0 <= d_lo <= d_hi <= d_max (the clamped copy is what is matched and what
 * tsgm_inspect shows); D_z, r_z: float outputs, -1 where the left-right check fails. */
tsgm_status tsgm_match(tsgm_ctx* ctx, const uint8_t* left, const uint8_t* right,
                       const int16_t* d_lo, const int16_t* d_hi, float* D_z, float* r_z);

/* Pixel-wise Kalman update (Sec. 2.4, Eq. 10-12): K = p/(p+r), d = d_p + K (d_z - d_p),
 * p' = (1 - K) p, binary32. Only a measurement: (d_z, r); only a prediction: (d_p, p);
 * neither: (-1, -1). Outputs may alias the prediction inputs. */
tsgm_status tsgm_kalman_update(tsgm_ctx* ctx, const float* pred_D, const float* pred_P,
                               const float* D_z, const float* r_z, float* D, float* P);

/* One time step (Sec. 2): predict from the context's previous state with the pose, choose the
 * windows, match, update; the result is written to D, P (device) and kept as the next
 * frame's previous state, except where the matched disparity was rejected (left-right check):
 * there D, P carry the prediction, but the state keeps no value, so that the next frame
 * searches the whole range at that pixel (Sec. 2.4, disparity consistency check). The first
 * call after create/reset has no prediction and searches the whole range (Sec. 3); its R, t
 * may be NULL. Such a frame, and every frame with TSGM_FLAG_FULL_RANGE, is aggregated and
 * selected by kernels for full windows (the same results as the windowed ones on windows
 * [0, d_max]). On a context created with a non-default CUDA stream, while stage timing is off
 * and the caller is not capturing that stream, the step's ~20 kernels are launched as one CUDA
 * graph (captured each call; the instantiated graph of the last call of the same kind, a first
 * frame or a later one, is updated in place), which shortens the gaps between them; the results
 * are the same either way. An argument error found while enqueueing (an invalid pose) then
 * leaves nothing enqueued. */
tsgm_status tsgm_frame(tsgm_ctx* ctx, const uint8_t* left, const uint8_t* right,
                       const float R[9], const float t[3], const float K[9], float baseline,
                       float* D, float* P);

/* tsgm_frame with HOST buffers: copies left/right (width*height bytes each) to the device,
 * runs the step and copies D, P (width*height floats each) back. Pinned host memory gives
 * asynchronous copies; the call synchronises the stream before returning. */
tsgm_status tsgm_frame_host(tsgm_ctx* ctx, const uint8_t* left_host, const uint8_t* right_host,
                            const float R[9], const float t[3], const float K[9],
                            float baseline, float* D_host, float* P_host);

/* tsgm_frame_host without waiting: the input copies, the step and the output copies are
 * enqueued and the call returns. The copies run on two transfer streams of the context and the
 * context has two device staging slots, used in turn, so that one frame's copies overlap the
 * computation of the frames before and after it. left_host/right_host must not change, and
 * D_host/P_host must not be read, until tsgm_wait returns; host buffers must be pinned
 * (page-locked). Frames complete in call order. */
tsgm_status tsgm_frame_host_async(tsgm_ctx* ctx, const uint8_t* left_host,
                                  const uint8_t* right_host, const float R[9], const float t[3],
                                  const float K[9], float baseline, float* D_host, float* P_host);

/* Wait for every frame and copy enqueued on the context. */
tsgm_status tsgm_wait(tsgm_ctx* ctx);

/* Forget the previous frame: the next tsgm_frame searches the whole range. */
tsgm_status tsgm_reset(tsgm_ctx* ctx);

/* Checkpoint of the per-stream state (previous D, P and whether it exists) through host
 * buffers of width*height floats: the last frame's D, P without the pixels whose match was
 * rejected (see tsgm_frame). Export synchronises the stream. */
tsgm_status tsgm_state_export(tsgm_ctx* ctx, float* D_host, float* P_host, int32_t* has_prev);
tsgm_status tsgm_state_import(tsgm_ctx* ctx, const float* D_host, const float* P_host,
                              int32_t has_prev);

/* Census transform of one image (the matching cost's first stage): for every pixel p, bit b
 * (LSB first) is [I(q) < I(p)] for the b-th neighbour q of the census window in row-major
 * order without the centre, coordinates clamped to the border. codes: width*height uint64. */
tsgm_status tsgm_census(tsgm_ctx* ctx, const uint8_t* img, uint64_t* codes);

/* Internal buffers of the last call, for inspection and tests. */
typedef enum {
    TSGM_BUF_CENSUS_L = 0,  /* uint64 [n]     census of the left image (last match)     */
    TSGM_BUF_CENSUS_R = 1,  /* uint64 [n]     census of the right image                 */
    TSGM_BUF_OFFSETS = 2,   /* uint32 [n + 1] start of each pixel's block in the ragged volume:
                               exclusive scan of the window lengths rounded up to a multiple
                               of 4; [n] is the storage size. Pixel i's cell j (disparity
                               d_lo + j) is at offsets[i] + j.                              */
    TSGM_BUF_COST = 3,      /* uint8  [storage] ragged matching cost                     */
    TSGM_BUF_S = 4,         /* uint16 [storage] aggregated cost S = sum of path costs    */
    TSGM_BUF_DSTAR = 5,     /* int16  [n]     winner-takes-all disparity (KEEP_INTERNALS) */
    TSGM_BUF_DRIGHT = 6,    /* int16  [n]     right-view disparity, -1 none (KEEP_INTERNALS) */
    TSGM_BUF_LR_VALID = 7,  /* uint8  [n]     1 where the left-right check passed (KEEP_INTERNALS) */
    TSGM_BUF_ZKEYS = 8,     /* uint64 [n]     z-buffer keys of the last warp: high 32 bits =
                                              ~bits(d'), low 32 = source index; ~0 = empty */
    TSGM_BUF_WINDOWS_LO = 9,  /* int16 [n]    windows of the last tsgm_frame              */
    TSGM_BUF_WINDOWS_HI = 10,
    TSGM_BUF_PRED_D = 11,   /* float [n]      prediction of the last tsgm_frame            */
    TSGM_BUF_PRED_P = 12,
    TSGM_BUF_COUNTS = 13    /* uint32 [2]     of the last match: [0] true window cells, [1] pixels
                                              whose window is wider than 32 labels          */
} tsgm_buffer;

/* Copy an internal buffer (device to device, on the context stream) into dst. `count` is the
 * number of elements to copy; for the cell buffers the storage size is offsets[n].
 * INVALID_ARG if count exceeds the buffer. */
tsgm_status tsgm_inspect(tsgm_ctx* ctx, tsgm_buffer which, void* dst, uint64_t count);

/* Number of (pixel, disparity) cells of the windows of the last match/windows call: the sum of
 * the window lengths (synchronises the stream). */
tsgm_status tsgm_cells(tsgm_ctx* ctx, uint64_t* n_cells);

/* Number of kernels this context has enqueued since create (CUDA library copies such as the
 * z-buffer memset are not counted). */
tsgm_status tsgm_launches(tsgm_ctx* ctx, uint64_t* n);

/* Stage timing with CUDA events on the context's streams. When enabled, each call records events
 * around its stages; tsgm_stage_times returns the accumulated milliseconds per stage since the
 * last enable (synchronises) and the number of times each was recorded. The events add a little
 * time to the calls that record them. Stage ids: */
#define TSGM_STAGE_WARP 0      /* scatter + gather, and the prediction's refinements (edge
                                  rejection, gap filling, left-right check) */
#define TSGM_STAGE_WINDOWS 1   /* windows + offsets */
#define TSGM_STAGE_CENSUS 2    /* on the context's second stream, beside the stages before the cost */
#define TSGM_STAGE_COST 3
#define TSGM_STAGE_SGM 4       /* path aggregation */
#define TSGM_STAGE_SELECT 5    /* WTA, sub-pixel, r, LR check (both selection kernels) */
#define TSGM_STAGE_KALMAN 6    /* the update, and the SAD check of the updated map */
#define TSGM_STAGE_OFFSETS 7   /* offsets of caller windows in tsgm_match */
#define TSGM_N_STAGES 8
tsgm_status tsgm_profile(tsgm_ctx* ctx, int32_t enable);
tsgm_status tsgm_stage_times(tsgm_ctx* ctx, double ms[TSGM_N_STAGES], int64_t count[TSGM_N_STAGES]);

/* Adjoint of the float stages (training/fitting form): prediction (Sec. 2.2, Eq. 3, 5, 6) then
 * the Kalman update (Sec. 2.4, Eq. 10-12) as a function of the pose, q and a measurement-variance
 * scale s_r (r = s_r * r_z).
 *   pose6 = (w0, w1, w2, t0, t1, t2): R = exp([w]x) (Rodrigues, binary64 then rounded to
 *   binary32 for the warp), t in metres, convention of Eq. 2.
 * tsgm_adjoint_forward writes D, P (device, width*height floats) and keeps the z-buffer winners
 * in the context. tsgm_adjoint_backward must follow it with the same inputs: given the upstream
 * gradients grad_D, grad_P (device), it recomputes every quantity except the winners (target
 * pixels are roundings, piecewise constant in the pose) and writes dL/d(w0, w1, w2, t0, t1, t2,
 * q, s_r) to the host array grad_out[8] (binary64; synchronises the stream). dL/dt0 and dL/dt1
 * are 0: with the winners fixed, lateral translation does not change any predicted depth. */
tsgm_status tsgm_adjoint_forward(tsgm_ctx* ctx, const float* prev_D, const float* prev_P,
                                 const double pose6[6], const float K[9], float baseline, float q,
                                 float r_scale, const float* D_z, const float* r_z, float* D,
                                 float* P);
tsgm_status tsgm_adjoint_backward(tsgm_ctx* ctx, const float* prev_D, const float* prev_P,
                                  const double pose6[6], const float K[9], float baseline, float q,
                                  float r_scale, const float* D_z, const float* r_z,
                                  const float* grad_D, const float* grad_P, double grad_out[8]);

/* ---------------------------------------------------------------------------------------------
 * Batched matching over many camera streams of different sizes and disparity ranges (the
 * tsgm_match step of every stream, Sec. 2.3-2.4). One call runs one CUDA graph: every stage is a
 * single launch over the work of all streams, and the path aggregation is a persistent kernel
 * whose warps take path lines of any stream from one queue.
 * ------------------------------------------------------------------------------------------- */
typedef struct tsgm_batch tsgm_batch;

/* streams[i] gives width, height and d_max of stream i (n_streams <= 128, W x H x (d_max + 1)
 * below 2^32); the matching parameters (census window, paths, P1, P2, S_max, r_min, lr_tol) must
 * be equal across streams. The ragged cost and path volumes of all streams live in one pool of
 * sum_i W_i x H_i x L_i cells per volume, L_i = max_labels (or d_max + 1 if smaller or if
 * max_labels is 0) rounded up to 4. Every step each stream that runs reserves the padded cells of
 * its windows from the pool, streams refused at the previous step first, then in stream order;
 * a stream that does not fit the cells left is refused for this step (tsgm_batch_stream_status):
 * tsgm_batch_match writes -1 to its outputs, tsgm_batch_frame leaves its outputs and state as
 * they were. With max_labels = 0 every stream always fits. The batch works on its own CUDA
 * stream, ordered after and before `cuda_stream` (NULL: legacy default stream) with events.
 * Errors: INVALID_ARG, OUT_OF_MEMORY. */
tsgm_status tsgm_batch_create(const tsgm_params* streams, int32_t n_streams, int32_t max_labels,
                              void* cuda_stream, tsgm_batch** out);
void tsgm_batch_destroy(tsgm_batch* b);
const char* tsgm_batch_last_error(const tsgm_batch* b);

/* One step: host arrays of n_streams device pointers (images, windows, outputs as in
 * tsgm_match). The first call captures the graph; later calls update the pointer table and
 * replay it. A call waits until the previous step of this batch has finished on the GPU. */
tsgm_status tsgm_batch_match(tsgm_batch* b, const uint8_t* const* left,
                             const uint8_t* const* right, const int16_t* const* d_lo,
                             const int16_t* const* d_hi, float* const* D_z, float* const* r_z);

/* Time every candidate launch shape of the path aggregation (warps per block x blocks per SM)
 * on these inputs, `reps` steps each, keep the fastest; then, with that shape, every candidate
 * grid of the cost kernel (2, 4, 8 or 16 blocks per SM); re-capture the graph (both step forms
 * use the result). Outputs the best mean step time (ms) and the chosen aggregation shape index.
 * Synchronises. */
tsgm_status tsgm_batch_autotune(tsgm_batch* b, const uint8_t* const* left,
                                const uint8_t* const* right, const int16_t* const* d_lo,
                                const int16_t* const* d_hi, float* const* D_z, float* const* r_z,
                                int32_t reps, double* best_ms, int32_t* best_shape);

/* Total window cells of the last step over the streams that ran it, and how many streams were
 * refused for lack of pool cells. Synchronises. */
tsgm_status tsgm_batch_cells(tsgm_batch* b, uint64_t* cells, int32_t* overflowed);

/* One step run with direct launches instead of the graph, timed with CUDA events on the batch's
 * stream: device time of the path aggregation kernel and of the whole step (ms). Synchronises. */
tsgm_status tsgm_batch_profile(tsgm_batch* b, const uint8_t* const* left,
                               const uint8_t* const* right, const int16_t* const* d_lo,
                               const int16_t* const* d_hi, float* const* D_z, float* const* r_z,
                               float* sgm_ms, float* step_ms);

/* One time step of every stream (Sec. 2, the per-frame loop of tsgm_frame run for all streams at
 * once): pose warp of the stream's previous state with the z-buffer (Eq. 3-6), gap filling
 * (Eq. 7-8, with TSGM_FLAG_FILL_GAPS), the +-k sigma windows (Sec. 2.3; the whole range with
 * TSGM_FLAG_FULL_RANGE), census, cost, aggregation, selection with the left-right check
 * (Sec. 2.4, Eq. 9) and the Kalman update (Eq. 10-12). The previous state of each stream stays
 * on the device inside the batch, so stream i's outputs equal those of a tsgm_frame context fed
 * the same frames. The whole step is one CUDA graph (captured by the first call, replayed after).
 *   left, right : host arrays of n_streams device pointers to W_i x H_i u8 images; a stream whose
 *                 left and right are both NULL sits the step out (its state is kept)
 *   R, t        : host arrays, n_streams x 9 and n_streams x 3 floats, the motion from the
 *                 stream's previous frame to this one (Eq. 1-4); unread for a stream's first
 *                 frame and for streams sitting out; may be NULL when no stream needs them
 *   K, baseline : host arrays, n_streams x 9 floats (row-major intrinsics) and n_streams floats
 *   D, P        : host arrays of n_streams device pointers to W_i x H_i f32 outputs (updated
 *                 disparity and variance; -1 where neither a prediction nor a match exists)
 * A stream refused by the volume pool (see tsgm_batch_create) keeps its state and outputs; the
 * caller runs that frame again in a later step. R and t are required for every stream that was
 * active in an earlier step since create or reset (they are unread while the stream holds no
 * state yet, e.g. when its first frame was refused).
 * Stream parameters: flags, gamma_f and sigma_mult must be equal across streams and q finite
 * >= 0, and the pool must hold the largest stream at full range (max_labels = 0 does);
 * TSGM_FLAG_EDGE_REJECT, _PRED_LR_CHECK and _SAD_CHECK are not in the batched step
 * (UNIMPLEMENTED); TSGM_FLAG_KEEP_INTERNALS is ignored. All arguments are checked before
 * anything is enqueued: INVALID_ARG (null pointer of an active stream, D[i] == P[i], invalid
 * pose or calibration, poses missing) leaves every stream's state as it was. Ordered on the
 * batch's CUDA stream like tsgm_batch_match; a call waits for the previous step to finish. */
tsgm_status tsgm_batch_frame(tsgm_batch* b, const uint8_t* const* left,
                             const uint8_t* const* right, const float* R, const float* t,
                             const float* K, const float* baseline, float* const* D,
                             float* const* P);

/* Forget every stream's previous state: the next tsgm_batch_frame is a first frame for all. */
tsgm_status tsgm_batch_reset(tsgm_batch* b);

/* Per stream, what the last step did with it: 0 ran, 1 sat the step out (tsgm_batch_frame with
 * no images for it), 2 refused for lack of pool cells. status: host array of n_streams.
 * Synchronises. */
tsgm_status tsgm_batch_stream_status(tsgm_batch* b, int32_t* status);

/* Cells of the volume pool (per volume) and the cells of the largest stream at full range. */
tsgm_status tsgm_batch_pool(tsgm_batch* b, uint64_t* pool_cells, uint64_t* largest_full_range);

/* Kernels launched by this batch (graph steps count their kernels). */
tsgm_status tsgm_batch_launches(tsgm_batch* b, uint64_t* n);

/* ---------------------------------------------------------------------------------------------
 * Serving: many camera streams each sending frames at their own rate. The per-stream state
 * (previous D, P) stays on the device. A scheduler thread runs ticks of the batched time step
 * (tsgm_batch_frame): each tick takes the oldest waiting frame of every stream that has one and
 * runs them all in one graph replay; frames arriving meanwhile go into the next tick (continuous
 * batching). The ragged volumes of all streams share one pool sized by the HBM budget (at least
 * the largest stream at full range); a stream that does not fit the cells left in a tick keeps
 * its state and its frame runs in a later tick, so the budget bounds memory and drops nothing.
 * ------------------------------------------------------------------------------------------- */
typedef struct tsgm_server tsgm_server;

/* streams[i]: parameters of camera stream i (frames of a stream must have its size); the
 * matching parameters, flags, gamma_f and sigma_mult must be equal across streams (INVALID_ARG)
 * and TSGM_FLAG_EDGE_REJECT, _PRED_LR_CHECK and _SAD_CHECK are not served (UNIMPLEMENTED).
 * hbm_budget_bytes bounds the device memory of the server (state, scratch, pool). */
tsgm_status tsgm_server_create(const tsgm_params* streams, int32_t n_streams,
                               uint64_t hbm_budget_bytes, tsgm_server** out);
/* Finishes every submitted frame, then releases everything. */
void tsgm_server_destroy(tsgm_server* s);
/* Queue one frame of `stream` (host images of its size, copied at once; pose as in tsgm_frame,
 * NULL for the stream's first frame). D_host, P_host receive the result and must stay valid until
 * tsgm_server_wait returns for the ticket. Frames of one stream run in submission order. */
tsgm_status tsgm_server_submit(tsgm_server* s, int32_t stream, const uint8_t* left_host,
                               const uint8_t* right_host, const float R[9], const float t[3],
                               const float K[9], float baseline, float* D_host, float* P_host,
                               uint64_t* ticket);
/* Block until the ticket's frame is done; returns its status and its latency (submit to result). */
tsgm_status tsgm_server_wait(tsgm_server* s, uint64_t ticket, double* latency_ms);
/* Latency percentiles over all finished frames, their number, the number of streams whose
 * full-range step the pool holds at once (n_slots) and the most frames run in one tick. */
tsgm_status tsgm_server_stats(tsgm_server* s, double* p50_ms, double* p99_ms, uint64_t* completed,
                              int32_t* n_slots, uint64_t* max_in_flight);

/* Disparity prediction that allocates nothing (the paper has no counterpart: this is a
 * deployment variant of tsgm_warp_predict).
 *
 * Some callers cannot allocate device memory: a process whose GPU memory is owned by another
 * framework's caching allocator, where a cudaMalloc outside it can fail once the pool holds the
 * free memory, or a real-time loop that must not call cudaMalloc because it can block on the
 * device. This call does what tsgm_warp_predict does, without a context: its z-buffer is a
 * fixed array of TSGM_NOALLOC_MAX_PIXELS 64-bit keys (16 MiB) in the library's device memory,
 * held by every GPU that loads the library until the process exits. It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   prev_D, prev_P, pred_D, pred_P: device maps of width*height floats, as in tsgm_warp_predict;
 *   q: variance added to every predicted pixel, finite and >= 0; cuda_stream: stream to enqueue
 *   on (NULL: the legacy default stream); errbuf: optional buffer of errbuf_len bytes for a
 *   message.
 * Returns INVALID_ARG (nothing launched) for null pointers, outputs that alias inputs, a q that
 * is negative, infinite or NaN, a bad pose or calibration, or width * height >
 * TSGM_NOALLOC_MAX_PIXELS; CUDA if a launch fails.
 * The first call on a device looks up the array's device address on that device (a one-time
 * set-up); make that first call before any stream capture. The address is kept for the life of
 * the device's context: do not use this call across a cudaDeviceReset. Every call shares the
 * one array and resets the keys it uses, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. */
#define TSGM_NOALLOC_MAX_PIXELS 2097152
tsgm_status tsgm_warp_predict_noalloc(const float* prev_D, const float* prev_P, int32_t width,
                                      int32_t height, const float R[9], const float t[3],
                                      const float K[9], float baseline, float q, float* pred_D,
                                      float* pred_P, void* cuda_stream, char* errbuf,
                                      size_t errbuf_len);

#ifdef __cplusplus
}
#endif
#endif /* TSGM_H */
