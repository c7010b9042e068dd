// Adjoint of the float stages of one time step: the disparity-space warp with its variance
// prediction (Sec. 2.2, Eq. 3, 5, 6) followed by the pixel-wise Kalman update (Sec. 2.4,
// Eq. 10-12), differentiated with respect to the 6-DoF pose, the prediction variance q and a
// scale s_r of the measurement variance (r = s_r r_z).
//
// The z-buffer winners of the forward pass are kept (the target pixel is a rounding of the
// warped position, piecewise constant in the pose, so it has no derivative); everything else is
// recomputed in the backward pass from the inputs. With the winner of target t being source s
// (disparity d, variance p, centred coordinates x~, y~):
//   w3 = H30 x~ + H31 y~ + H32 d + H33,  d' = d / w3,  p' = (d'/d)^2 p + q,
// and only w3 depends on the pose (H30 = R20/f, H31 = R21/f, H32 = t2/(f b), H33 = R22), so the
// pose gradient flows through dL/dR[2][0..2] and dL/dt2; the host maps dL/dR to the rotation
// vector with the exact derivative of the Rodrigues formula.

#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "tsgm_internal.cuh"

namespace {

constexpr int kAdjThreads = 256;
constexpr int kAdjBlocks = tsgm::kAdjointBlocks;  // partial sums per block, summed on the host

__device__ __forceinline__ bool valid_value(float v) { return v >= 0.0f && v <= FLT_MAX; }

// Kalman update with the measurement variance scaled by s_r (same order of operations as the
// plain update, r = s_r * r_z first).
__global__ void __launch_bounds__(256) k_kalman_scaled(const float* __restrict__ Dp,
                                                       const float* __restrict__ Pp,
                                                       const float* __restrict__ Dz,
                                                       const float* __restrict__ rz, float s_r,
                                                       int n, float* __restrict__ D,
                                                       float* __restrict__ P) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float dp = Dp[i], pp = Pp[i], dz = Dz[i];
        const float r = __fmul_rn(s_r, rz[i]);
        const bool pv = valid_value(dp) && valid_value(pp);
        const bool mv = valid_value(dz) && valid_value(rz[i]);
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
    }
}

struct AdjParams {
    float h30, h31, h32, h33;
    float cx, cy;
    double inv_f, inv_fb;
    float q, s_r;
};

// Per target pixel: the local derivatives of (D, P) chained with the upstream gradients, summed
// in binary64 per block: out[block * 6 + {dR20, dR21, dR22, dt2, dq, ds_r}].
__global__ void __launch_bounds__(kAdjThreads) k_adjoint(
    const unsigned long long* __restrict__ keys, const float* __restrict__ Dprev,
    const float* __restrict__ Pprev, const float* __restrict__ Dz, const float* __restrict__ rz,
    const float* __restrict__ gD, const float* __restrict__ gP, int W, int n, AdjParams a,
    double* __restrict__ out) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double gd = gD[i], gp = gP[i];
        const float dz = Dz[i], rzi = rz[i];
        const bool mv = valid_value(dz) && valid_value(rzi);
        const unsigned long long key = keys[i];
        if (key == tsgm::kEmptyKey) {
            if (mv) acc[5] += gp * (double)rzi;  // P = s_r r_z
            continue;
        }
        const int s = (int)(unsigned)(key & 0xFFFFFFFFull);
        const int v = s / W;
        const int u = s - v * W;
        const double d = Dprev[s], p = Pprev[s];
        const double xt = (double)((float)u - a.cx), yt = (double)((float)v - a.cy);
        const double w3 = (double)a.h30 * xt + (double)a.h31 * yt + (double)a.h32 * d + (double)a.h33;
        const double dp = d / w3;                        // d'
        const double pp = p * (dp / d) * (dp / d) + a.q;  // p'
        double dL_ddp, dL_dpp, dL_dr = 0.0;
        if (mv) {
            const double r = (double)a.s_r * (double)rzi;
            const double den = pp + r;
            const double K = pp / den;
            dL_ddp = gd * (1.0 - K);
            dL_dpp = gd * ((double)dz - dp) * r / (den * den) + gp * (r * r) / (den * den);
            dL_dr = -gd * ((double)dz - dp) * pp / (den * den) + gp * (pp * pp) / (den * den);
        } else {
            dL_ddp = gd;
            dL_dpp = gp;
        }
        // p' depends on d' as well: dp'/dd' = 2 p d' / d^2
        const double dL_ddp_tot = dL_ddp + dL_dpp * 2.0 * p * dp / (d * d);
        const double dL_dw3 = dL_ddp_tot * (-dp / w3);
        acc[0] += dL_dw3 * xt * a.inv_f;
        acc[1] += dL_dw3 * yt * a.inv_f;
        acc[2] += dL_dw3;
        acc[3] += dL_dw3 * d * a.inv_fb;
        acc[4] += dL_dpp;
        acc[5] += dL_dr * (double)rzi;
    }
    // block reduction
    __shared__ double sh[kAdjThreads / 32][6];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        double x = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double x = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) x += sh[w][threadIdx.x];
        out[blockIdx.x * 6 + threadIdx.x] = x;
    }
}

// R = exp([w]x) (Rodrigues) in binary64, row-major.
void rodrigues(const double w[3], double R[9]) {
    const double th = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double k[3] = {0, 0, 0};
    if (th > 0) {
        k[0] = w[0] / th;
        k[1] = w[1] / th;
        k[2] = w[2] / th;
    }
    const double c = std::cos(th), s = std::sin(th), C = 1.0 - c;
    R[0] = c + k[0] * k[0] * C;
    R[1] = k[0] * k[1] * C - k[2] * s;
    R[2] = k[0] * k[2] * C + k[1] * s;
    R[3] = k[1] * k[0] * C + k[2] * s;
    R[4] = c + k[1] * k[1] * C;
    R[5] = k[1] * k[2] * C - k[0] * s;
    R[6] = k[2] * k[0] * C - k[1] * s;
    R[7] = k[2] * k[1] * C + k[0] * s;
    R[8] = c + k[2] * k[2] * C;
}

// dR/dw_i for R = exp([w]x): (w_i [w]x + [w x (I - R) e_i]x) R / |w|^2, and [e_i]x at w = 0.
void rodrigues_jacobian(const double w[3], const double R[9], double dR[3][9]) {
    const double n2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    auto skew = [](const double a[3], double S[9]) {
        S[0] = 0; S[1] = -a[2]; S[2] = a[1];
        S[3] = a[2]; S[4] = 0; S[5] = -a[0];
        S[6] = -a[1]; S[7] = a[0]; S[8] = 0;
    };
    for (int i = 0; i < 3; ++i) {
        double S[9];
        if (n2 < 1e-24) {
            double e[3] = {0, 0, 0};
            e[i] = 1.0;
            skew(e, dR[i]);
            continue;
        }
        // v = w x ((I - R) e_i)
        double col[3] = {-R[0 * 3 + i], -R[1 * 3 + i], -R[2 * 3 + i]};
        col[i] += 1.0;
        const double v[3] = {w[1] * col[2] - w[2] * col[1], w[2] * col[0] - w[0] * col[2],
                             w[0] * col[1] - w[1] * col[0]};
        double Sw[9], Sv[9];
        skew(w, Sw);
        skew(v, Sv);
        for (int k = 0; k < 9; ++k) S[k] = (w[i] * Sw[k] + Sv[k]) / n2;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double x = 0.0;
                for (int m = 0; m < 3; ++m) x += S[r * 3 + m] * R[m * 3 + c];
                dR[i][r * 3 + c] = x;
            }
    }
}

tsgm_status adj_fail(tsgm_ctx* c, tsgm_status s, const char* msg) {
    if (c) c->err = msg;
    return s;
}

tsgm_status adj_cuda(tsgm_ctx* c, cudaError_t e, const char* where) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    if (c) c->err = buf;
    return TSGM_ERR_CUDA;
}

bool pose_R_t(const double pose6[6], float R32[9], float t32[3], double R64[9]) {
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(pose6[k])) return false;
    rodrigues(pose6, R64);
    for (int k = 0; k < 9; ++k) R32[k] = (float)R64[k];
    for (int k = 0; k < 3; ++k) t32[k] = (float)pose6[3 + k];
    return true;
}

}  // namespace

extern "C" {

tsgm_status tsgm_adjoint_forward(tsgm_ctx* ctx, const float* prev_D, const float* prev_P,
                                 const double pose6[6], const float K[9], float baseline, float q,
                                 float r_scale, const float* D_z, const float* r_z, float* D,
                                 float* P) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!prev_D || !prev_P || !pose6 || !K || !D_z || !r_z || !D || !P)
        return adj_fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_adjoint_forward: null pointer");
    if (!(q >= 0.0f) || !(r_scale >= 0.0f))
        return adj_fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_adjoint_forward: q and r_scale must be >= 0");
    float R32[9], t32[3], H32[16];
    double R64[9];
    if (!pose_R_t(pose6, R32, t32, R64) || tsgm_build_H(R32, t32, K, baseline, H32) != TSGM_OK)
        return adj_fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_adjoint_forward: invalid pose or calibration");
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemsetAsync(ctx->keys, 0xFF, sizeof(unsigned long long) * ctx->n, st);
    if (e == cudaSuccess)
        e = tsgm::launch_warp_scatter(prev_D, prev_P, H32, K[2], K[5], ctx->W, ctx->H, ctx->keys, st);
    if (e == cudaSuccess)
        e = tsgm::launch_warp_gather(ctx->keys, prev_D, prev_P, q, ctx->n, ctx->predD, ctx->predP, st);
    if (e == cudaSuccess) {
        int blocks = (ctx->n + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        k_kalman_scaled<<<blocks, 256, 0, st>>>(ctx->predD, ctx->predP, D_z, r_z, r_scale, ctx->n,
                                                 D, P);
        e = cudaGetLastError();
        ctx->launches += 3;
    }
    if (e != cudaSuccess) return adj_cuda(ctx, e, "tsgm_adjoint_forward");
    return TSGM_OK;
}

tsgm_status tsgm_adjoint_backward(tsgm_ctx* ctx, const float* prev_D, const float* prev_P,
                                  const double pose6[6], const float K[9], float baseline, float q,
                                  float r_scale, const float* D_z, const float* r_z,
                                  const float* grad_D, const float* grad_P, double grad_out[8]) {
    if (!ctx) return TSGM_ERR_INVALID_ARG;
    if (!prev_D || !prev_P || !pose6 || !K || !D_z || !r_z || !grad_D || !grad_P || !grad_out)
        return adj_fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_adjoint_backward: null pointer");
    float R32[9], t32[3], H32[16];
    double R64[9];
    if (!pose_R_t(pose6, R32, t32, R64) || tsgm_build_H(R32, t32, K, baseline, H32) != TSGM_OK)
        return adj_fail(ctx, TSGM_ERR_INVALID_ARG, "tsgm_adjoint_backward: invalid pose or calibration");
    AdjParams a;
    a.h30 = H32[12];
    a.h31 = H32[13];
    a.h32 = H32[14];
    a.h33 = H32[15];
    a.cx = K[2];
    a.cy = K[5];
    a.inv_f = 1.0 / (double)K[0];
    a.inv_fb = 1.0 / ((double)K[0] * (double)baseline);
    a.q = q;
    a.s_r = r_scale;
    cudaStream_t st = ctx->stream;
    k_adjoint<<<kAdjBlocks, kAdjThreads, 0, st>>>(ctx->keys, prev_D, prev_P, D_z, r_z, grad_D, grad_P,
                                                  ctx->W, ctx->n, a, ctx->adj_partials);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    static thread_local double host_part[kAdjBlocks * 6];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_part, ctx->adj_partials, sizeof(double) * kAdjBlocks * 6,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return adj_cuda(ctx, e, "tsgm_adjoint_backward");
    double g[6] = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < kAdjBlocks; ++b)
        for (int k = 0; k < 6; ++k) g[k] += host_part[b * 6 + k];
    // H is built from the binary32 R; dL/dR[2][j] maps to the rotation vector through dR/dw
    double dR[3][9];
    rodrigues_jacobian(pose6, R64, dR);
    for (int i = 0; i < 3; ++i) grad_out[i] = g[0] * dR[i][6] + g[1] * dR[i][7] + g[2] * dR[i][8];
    grad_out[3] = 0.0;  // lateral translation moves pixels but not their depth
    grad_out[4] = 0.0;
    grad_out[5] = g[3];
    grad_out[6] = g[4];
    grad_out[7] = g[5];
    return TSGM_OK;
}

}  // extern "C"
