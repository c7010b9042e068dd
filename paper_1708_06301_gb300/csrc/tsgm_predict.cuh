// Device-side bodies of the prediction, window and update stages (Sec. 2.2-2.4), one pixel or
// one image row each, shared by the single-image kernels (tsgm_predict.cu) and the batched ones
// (tsgm_batch.cu).
//
// Every float operation that can decide an integer later (target pixel, z-buffer order, window
// bounds, the Kalman output warped by the next frame) uses explicit round-to-nearest intrinsics
// in a fixed order, so no FMA contraction or reassociation changes a result.
#pragma once

#include <cfloat>

#include "tsgm_kernels.cuh"

namespace tsgm {
namespace dev {

// The disparity-space homography H (Eq. 4, row-major 4 x 4) and the principal point.
struct WarpParams {
    float h[16];
    float cx, cy;
};

// Warp scatter of source pixel i (Eq. 3 + homogeneous divide; z-buffer of Sec. 2.2 "disparity
// refinement"): the key packs ~bits(d') (bits of a positive float grow with its value, so the
// complement makes atomicMin keep the largest d') above the source index (equal d' -> lowest
// index).
__device__ __forceinline__ void warp_scatter_px(int i, int W, int Hh,
                                                const float* __restrict__ Dprev,
                                                const float* __restrict__ Pprev,
                                                const WarpParams& wp,
                                                unsigned long long* __restrict__ keys) {
    const float d = Dprev[i];
    const float p = Pprev[i];
    if (!(d > 0.0f && d <= FLT_MAX && valid_value(p))) return;
    const int v = i / W;
    const int u = i - v * W;
    const float xt = __fsub_rn((float)u, wp.cx);
    const float yt = __fsub_rn((float)v, wp.cy);
    float w[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float* h = wp.h + 4 * r;
        float s = __fadd_rn(__fmul_rn(h[0], xt), __fmul_rn(h[1], yt));
        s = __fadd_rn(s, __fmul_rn(h[2], d));
        w[r] = __fadd_rn(s, h[3]);
    }
    if (!(w[3] > 0.0f)) return;
    const float xp = __fdiv_rn(w[0], w[3]);
    const float yp = __fdiv_rn(w[1], w[3]);
    const float dp = __fdiv_rn(w[2], w[3]);
    if (!(dp > 0.0f && dp <= FLT_MAX)) return;
    const float fx = floorf(__fadd_rn(__fadd_rn(xp, wp.cx), 0.5f));
    const float fy = floorf(__fadd_rn(__fadd_rn(yp, wp.cy), 0.5f));
    if (!(fx >= 0.0f && fx <= (float)(W - 1) && fy >= 0.0f && fy <= (float)(Hh - 1))) return;
    const int tgt = (int)fy * W + (int)fx;
    const unsigned long long key =
        ((unsigned long long)(~__float_as_uint(dp)) << 32) | (unsigned long long)(unsigned)i;
    atomicMin(keys + tgt, key);
}

// Warp gather + variance prediction of target pixel i (Eq. 5-6): p' = (d'/d)^2 p + q; an empty
// key is no prediction.
__device__ __forceinline__ void warp_gather_px(int i, unsigned long long key,
                                               const float* __restrict__ Dprev,
                                               const float* __restrict__ Pprev, float q,
                                               float* __restrict__ Dpred,
                                               float* __restrict__ Ppred) {
    float dp = -1.0f, pp = -1.0f;
    if (key != kEmptyKey) {
        const unsigned src = (unsigned)(key & 0xFFFFFFFFull);
        dp = __uint_as_float(~(unsigned)(key >> 32));
        const float phi = __fdiv_rn(dp, Dprev[src]);
        const float phi2 = __fmul_rn(phi, phi);
        pp = __fadd_rn(__fmul_rn(phi2, Pprev[src]), q);
    }
    Dpred[i] = dp;
    Ppred[i] = pp;
}

// Windows of image row y (Sec. 2.3), one block: [floor(d - k sqrt(p)), ceil(d + k sqrt(p))]
// clipped to [0, D-1]; the whole range without a valid prediction or when the interval misses
// the range (or everywhere, with full); writes the row's totals (storage cells, true cells,
// windows wider than kNarrowMax).
__device__ __forceinline__ void windows_row(const float* __restrict__ Dp,
                                            const float* __restrict__ Pp, int W, int D, float k,
                                            int y, int16_t* __restrict__ lo,
                                            int16_t* __restrict__ hi,
                                            uint32_t* __restrict__ rowsum,
                                            uint32_t* __restrict__ rowcells,
                                            uint32_t* __restrict__ rowwide, bool full = false) {
    __shared__ uint32_t sh[33];
    uint32_t acc = 0, acc_true = 0, acc_wide = 0;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int i = y * W + x;
        const float d = full ? -1.0f : Dp[i], p = full ? -1.0f : Pp[i];
        int a = 0, b = D - 1;
        if (valid_value(d) && valid_value(p)) {
            const float s = __fsqrt_rn(p);
            const float r = __fmul_rn(k, s);
            const float lo_f = floorf(__fsub_rn(d, r));
            const float hi_f = ceilf(__fadd_rn(d, r));
            if (lo_f <= (float)(D - 1) && hi_f >= 0.0f) {
                a = lo_f < 0.0f ? 0 : (int)lo_f;
                b = hi_f > (float)(D - 1) ? D - 1 : (int)hi_f;
            }
        }
        lo[i] = (int16_t)a;
        hi[i] = (int16_t)b;
        acc_true += (uint32_t)(b - a + 1);
        acc += block_cells(b - a + 1);
        acc_wide += (b - a + 1 > kNarrowMax) ? 1u : 0u;
    }
    row_totals(acc, acc_true, acc_wide, y, sh, rowsum, rowcells, rowwide);
}

// Kalman update of pixel i (Eq. 10-12); with D2, the state for the next frame, which keeps only
// measured pixels: where the match was rejected the true minimum may lie outside the window, so
// the next frame searches the whole range there (Sec. 2.4, disparity consistency check).
__device__ __forceinline__ void kalman_px(int i, const float* __restrict__ Dp,
                                          const float* __restrict__ Pp,
                                          const float* __restrict__ Dz,
                                          const float* __restrict__ rz, float* D, float* P,
                                          float* D2, float* P2) {
    const float dp = Dp[i], pp = Pp[i], dz = Dz[i], r = rz[i];
    const bool pv = valid_value(dp) && valid_value(pp);
    const bool mv = valid_value(dz) && valid_value(r);
    float d, p;
    if (pv && mv) {
        const float K = __fdiv_rn(pp, __fadd_rn(pp, r));
        d = __fadd_rn(dp, __fmul_rn(K, __fsub_rn(dz, dp)));
        p = __fmul_rn(__fsub_rn(1.0f, K), pp);
    } else if (mv) {
        d = dz;
        p = r;
    } else if (pv) {
        d = dp;
        p = pp;
    } else {
        d = -1.0f;
        p = -1.0f;
    }
    D[i] = d;
    P[i] = p;
    if (D2) {
        D2[i] = mv ? d : -1.0f;
        P2[i] = mv ? p : -1.0f;
    }
}

// Gap filling of pixel i (Eq. 7-8), one pass: horizontal (vertical == 0) or vertical
// neighbours, reading the input maps and writing the output maps (distinct buffers).
__device__ __forceinline__ void fill_gaps_px(int i, int W, int Hh, const float* __restrict__ Din,
                                             const float* __restrict__ Pin, float gamma_f,
                                             int vertical, float* __restrict__ Dout,
                                             float* __restrict__ Pout) {
    float d = Din[i], p = Pin[i];
    if (!(valid_value(d) && valid_value(p))) {
        const int y = i / W, x = i - y * W;
        const bool inner = vertical ? (y > 0 && y < Hh - 1) : (x > 0 && x < W - 1);
        if (inner) {
            const int a = vertical ? i - W : i - 1;
            const int b = vertical ? i + W : i + 1;
            const float da = Din[a], db = Din[b], pa = Pin[a], pb = Pin[b];
            if (valid_value(da) && valid_value(pa) && valid_value(db) && valid_value(pb) &&
                fabsf(__fsub_rn(da, db)) < gamma_f) {
                d = __fmul_rn(__fadd_rn(da, db), 0.5f);
                p = __fmul_rn(__fadd_rn(pa, pb), 0.5f);
            }
        }
    }
    Dout[i] = d;
    Pout[i] = p;
}

}  // namespace dev
}  // namespace tsgm
