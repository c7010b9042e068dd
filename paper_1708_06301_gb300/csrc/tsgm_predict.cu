// Disparity prediction (Sec. 2.2), reduced windows (Sec. 2.3) and the pixel-wise Kalman update
// (Sec. 2.4) as elementwise / per-row kernels.
//
// Every float operation that can decide an integer later (target pixel, z-buffer order, window
// bounds, the Kalman output warped by the next frame) uses explicit round-to-nearest intrinsics
// in a fixed order, so no FMA contraction or reassociation changes a result.

#include <cfloat>

#include "tsgm_kernels.cuh"
#include "tsgm_predict.cuh"

namespace tsgm {
namespace {

using namespace dev;

// ---------------------------------------------------------------------------------------------
// Warp scatter (Eq. 3 + homogeneous divide; z-buffer of Sec. 2.2 "disparity refinement").
// One thread per source pixel; the key packs ~bits(d') (bits of a positive float grow with its
// value, so the complement makes atomicMin keep the largest d') above the source index (equal
// d' -> lowest index).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_warp_scatter(const float* __restrict__ Dprev,
                                                      const float* __restrict__ Pprev,
                                                      WarpParams wp, int W, int Hh,
                                                      unsigned long long* __restrict__ keys) {
    const int n = W * Hh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        warp_scatter_px(i, W, Hh, Dprev, Pprev, wp, keys);
}

// Warp gather + variance prediction (Eq. 5-6): p' = (d'/d)^2 p + q.
__global__ void __launch_bounds__(256) k_warp_gather(const unsigned long long* __restrict__ keys,
                                                     const float* __restrict__ Dprev,
                                                     const float* __restrict__ Pprev, float q,
                                                     int n, float* __restrict__ Dpred,
                                                     float* __restrict__ Ppred) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        warp_gather_px(i, keys[i], Dprev, Pprev, q, Dpred, Ppred);
}

// ---------------------------------------------------------------------------------------------
// Windows (Sec. 2.3): [floor(d - k sqrt(p)), ceil(d + k sqrt(p))] clipped to [0, D-1]; the
// whole range without a valid prediction or when the interval misses the range. One block per
// row; also writes the row's total window length.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_windows(const float* __restrict__ Dp,
                                                 const float* __restrict__ Pp, int W, int D,
                                                 float k, int16_t* __restrict__ lo,
                                                 int16_t* __restrict__ hi,
                                                 uint32_t* __restrict__ rowsum,
                                                 uint32_t* __restrict__ rowcells,
                                                 uint32_t* __restrict__ rowwide,
                                                 uint32_t* __restrict__ wq) {
    const int y = blockIdx.x;
    if (y == 0 && threadIdx.x == 0) wq[0] = 0u;  // the offsets pass queues this image's wide pixels
    windows_row(Dp, Pp, W, D, k, y, lo, hi, rowsum, rowcells, rowwide);
}

// Caller-supplied windows, clamped copies and row totals (see sanitize_row).
__global__ void __launch_bounds__(256) k_sanitize_rowsum(const int16_t* __restrict__ lo_in,
                                                         const int16_t* __restrict__ hi_in, int W,
                                                         int D, int16_t* __restrict__ lo,
                                                         int16_t* __restrict__ hi,
                                                         uint32_t* __restrict__ rowsum,
                                                         uint32_t* __restrict__ rowcells,
                                                         uint32_t* __restrict__ wq) {
    if (blockIdx.x == 0 && threadIdx.x == 0) wq[0] = 0u;  // see k_windows
    sanitize_row(lo_in, hi_in, W, D, blockIdx.x, lo, hi, rowsum, rowcells, rowcells + gridDim.x);
}

// Block starts and descriptors of the ragged volume, one block per row (see offsets_row).
__global__ void __launch_bounds__(512) k_offsets(const int16_t* __restrict__ lo,
                                                 const int16_t* __restrict__ hi,
                                                 const uint32_t* __restrict__ rowsum,
                                                 const uint32_t* __restrict__ rowcells, int W,
                                                 int Hh, uint32_t* __restrict__ off,
                                                 uint2* __restrict__ desc,
                                                 uint32_t* __restrict__ cells_total,
                                                 uint32_t* __restrict__ wq) {
    offsets_row(lo, hi, rowsum, rowcells, rowcells + Hh, W, Hh, blockIdx.x, off, desc, cells_total,
                wq);
}

// ---------------------------------------------------------------------------------------------
// Kalman update (Eq. 10-12). Optional second output (the context's state for the next frame).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_kalman(const float* __restrict__ Dp,
                                                const float* __restrict__ Pp,
                                                const float* __restrict__ Dz,
                                                const float* __restrict__ rz, int n,
                                                float* D, float* P, float* D2, float* P2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        kalman_px(i, Dp, Pp, Dz, rz, D, P, D2, P2);
}

// Gap filling (Eq. 7-8), one pass: horizontal (vertical == 0) or vertical neighbours, reading
// the input maps and writing the output maps (distinct buffers).
__global__ void __launch_bounds__(256) k_fill_gaps(const float* __restrict__ Din,
                                                   const float* __restrict__ Pin, int W, int Hh,
                                                   float gamma_f, int vertical,
                                                   float* __restrict__ Dout,
                                                   float* __restrict__ Pout) {
    const int n = W * Hh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        fill_gaps_px(i, W, Hh, Din, Pin, gamma_f, vertical, Dout, Pout);
}

__global__ void __launch_bounds__(256) k_fill(float* __restrict__ a, float v, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = v;
}

int grid_for(int n, int threads) {
    int g = (n + threads - 1) / threads;
    const int cap = 152 * 16;  // grid-stride beyond 16 blocks per SM
    return g < 1 ? 1 : (g > cap ? cap : g);
}

// ---------------------------------------------------------------------------------------------
// Edge rejection (Sec. 2.2, disparity refinement): a valid predicted pixel with a valid
// 8-neighbour whose disparity differs by at least thr becomes invalid; one thread per pixel,
// out of place.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_edge_reject(const float* __restrict__ Din,
                                                     const float* __restrict__ Pin, int W, int Hh,
                                                     float thr, float* __restrict__ Dout,
                                                     float* __restrict__ Pout) {
    const int n = W * Hh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float d = Din[i], p = Pin[i];
        bool edge = false;
        if (valid_value(d) && valid_value(p)) {
            const int y = i / W, x = i - y * W;
            for (int dy = -1; dy <= 1; ++dy) {
                const int yn = y + dy;
                if (yn < 0 || yn >= Hh) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xn = x + dx;
                    if ((dx == 0 && dy == 0) || xn < 0 || xn >= W) continue;
                    const int j = yn * W + xn;
                    const float dn = Din[j], pn = Pin[j];
                    if (valid_value(dn) && valid_value(pn) && !(fabsf(__fsub_rn(d, dn)) < thr))
                        edge = true;
                }
            }
        }
        Dout[i] = edge ? -1.0f : d;
        Pout[i] = edge ? -1.0f : p;
    }
}

// ---------------------------------------------------------------------------------------------
// Left-right check of the prediction (Sec. 2.2, Fig. 3(d)), one block per row, in place: the
// right view's prediction of the row in shared memory (every valid pixel lands on x - round(d),
// round(d) = floor(d + 1/2) in binary32, and the right pixel keeps the largest disparity, by an
// atomic maximum on the bit patterns of non-negative floats), then a pixel stays valid where its
// landing pixel lies in the image and holds a disparity within tol of its own.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int right_col(int x, float d) {
    const float rf = floorf(__fadd_rn(d, 0.5f));
    return rf > (float)x ? -1 : x - (int)rf;
}

__global__ void __launch_bounds__(512) k_pred_lr(float* __restrict__ D, float* __restrict__ P,
                                                 int W, float tol) {
    extern __shared__ unsigned int rbits[];  // W right pixels (0 = +0.0f, below any landing)
    float* const d = D + (size_t)blockIdx.x * W;
    float* const p = P + (size_t)blockIdx.x * W;
    for (int x = threadIdx.x; x < W; x += blockDim.x) rbits[x] = 0u;
    __syncthreads();
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const float dv = d[x];
        if (!(valid_value(dv) && valid_value(p[x]))) continue;
        const int r = right_col(x, dv);
        if (r >= 0) atomicMax(rbits + r, __float_as_uint(dv));
    }
    __syncthreads();
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const float dv = d[x];
        if (!(valid_value(dv) && valid_value(p[x]))) continue;
        const int r = right_col(x, dv);
        if (!(r >= 0 && fabsf(__fsub_rn(dv, __uint_as_float(rbits[r]))) <= tol)) {
            d[x] = -1.0f;
            p[x] = -1.0f;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// SAD check of an updated map (Sec. 2.4), one thread per pixel, in place: the left patch around
// (x, y) against the right patch around (x - round(d), y), coordinates clamped into the image; a
// valid pixel whose SAD is above lim is rejected in (D, P) and, when given, in (D2, P2).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sad_check(const uint8_t* __restrict__ L,
                                                   const uint8_t* __restrict__ R, int W, int Hh,
                                                   int sw, int sh, float lim,
                                                   float* __restrict__ D, float* __restrict__ P,
                                                   float* __restrict__ D2, float* __restrict__ P2) {
    const int n = W * Hh;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float dv = D[i];
    if (!(valid_value(dv) && valid_value(P[i]))) return;
    const int y = i / W, x = i - y * W;
    const float rf = floorf(__fadd_rn(dv, 0.5f));
    const int dx = rf > (float)(2 * W) ? 2 * W : (int)rf;  // beyond the image either way
    const int hw = sw / 2, hh = sh / 2;
    int sad = 0;
    for (int v = -hh; v <= hh; ++v) {
        const int yy = min(max(y + v, 0), Hh - 1);
        const uint8_t* const lrow = L + (size_t)yy * W;
        const uint8_t* const rrow = R + (size_t)yy * W;
        for (int u = -hw; u <= hw; ++u) {
            const int xl = min(max(x + u, 0), W - 1);
            const int xr = min(max(x - dx + u, 0), W - 1);
            sad += abs((int)__ldg(lrow + xl) - (int)__ldg(rrow + xr));
        }
    }
    if ((float)sad > lim) {
        D[i] = -1.0f;
        P[i] = -1.0f;
        if (D2) {
            D2[i] = -1.0f;
            P2[i] = -1.0f;
        }
    }
}

}  // namespace

cudaError_t launch_warp_scatter(const float* Dprev, const float* Pprev, const float* H, float cx,
                                float cy, int W, int Hh, unsigned long long* keys,
                                cudaStream_t st) {
    WarpParams wp;
    for (int i = 0; i < 16; ++i) wp.h[i] = H[i];
    wp.cx = cx;
    wp.cy = cy;
    k_warp_scatter<<<grid_for(W * Hh, 256), 256, 0, st>>>(Dprev, Pprev, wp, W, Hh, keys);
    return cudaGetLastError();
}

cudaError_t launch_warp_gather(const unsigned long long* keys, const float* Dprev,
                               const float* Pprev, float q, int n, float* Dpred, float* Ppred,
                               cudaStream_t st) {
    k_warp_gather<<<grid_for(n, 256), 256, 0, st>>>(keys, Dprev, Pprev, q, n, Dpred, Ppred);
    return cudaGetLastError();
}

cudaError_t launch_pred_lr(float* D, float* P, int W, int Hh, float tol, cudaStream_t st) {
    const size_t smem = (size_t)W * sizeof(unsigned int);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_pred_lr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_pred_lr<<<Hh, 512, smem, st>>>(D, P, W, tol);
    return cudaGetLastError();
}

cudaError_t launch_sad_check(const uint8_t* left, const uint8_t* right, int W, int Hh, int sw,
                             int sh, float lim, float* D, float* P, float* D2, float* P2,
                             cudaStream_t st) {
    const int n = W * Hh;
    k_sad_check<<<(n + 255) / 256, 256, 0, st>>>(left, right, W, Hh, sw, sh, lim, D, P, D2, P2);
    return cudaGetLastError();
}

cudaError_t launch_windows(const float* Dp, const float* Pp, int W, int Hh, int D, float k,
                           int16_t* lo, int16_t* hi, uint32_t* rowsum, uint32_t* rowcells,
                           uint32_t* wq, cudaStream_t st) {
    k_windows<<<Hh, 256, 0, st>>>(Dp, Pp, W, D, k, lo, hi, rowsum, rowcells, rowcells + Hh, wq);
    return cudaGetLastError();
}

cudaError_t launch_sanitize(const int16_t* lo_in, const int16_t* hi_in, int W, int Hh, int D,
                            int16_t* lo, int16_t* hi, uint32_t* rowsum, uint32_t* rowcells,
                            uint32_t* wq, cudaStream_t st) {
    k_sanitize_rowsum<<<Hh, 256, 0, st>>>(lo_in, hi_in, W, D, lo, hi, rowsum, rowcells, wq);
    return cudaGetLastError();
}

cudaError_t launch_offsets(const int16_t* lo, const int16_t* hi, const uint32_t* rowsum,
                           const uint32_t* rowcells, int W, int Hh, uint32_t* off, uint2* desc,
                           uint32_t* cells_total, uint32_t* wq, cudaStream_t st) {
    k_offsets<<<Hh, 512, 0, st>>>(lo, hi, rowsum, rowcells, W, Hh, off, desc, cells_total, wq);
    return cudaGetLastError();
}

cudaError_t launch_edge_reject(const float* Din, const float* Pin, int W, int Hh, float thr,
                               float* Dout, float* Pout, cudaStream_t st) {
    const int n = W * Hh;
    int blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_edge_reject<<<blocks, 256, 0, st>>>(Din, Pin, W, Hh, thr, Dout, Pout);
    return cudaGetLastError();
}

cudaError_t launch_fill_gaps(const float* Din, const float* Pin, int W, int Hh, float gamma_f,
                             int vertical, float* Dout, float* Pout, cudaStream_t st) {
    k_fill_gaps<<<grid_for(W * Hh, 256), 256, 0, st>>>(Din, Pin, W, Hh, gamma_f, vertical, Dout, Pout);
    return cudaGetLastError();
}

cudaError_t launch_fill(float* a, float v, int n, cudaStream_t st) {
    k_fill<<<grid_for(n, 256), 256, 0, st>>>(a, v, n);
    return cudaGetLastError();
}

cudaError_t launch_kalman(const float* Dp, const float* Pp, const float* Dz, const float* rz, int n,
                          float* D, float* P, float* D2, float* P2, cudaStream_t st) {
    k_kalman<<<grid_for(n, 256), 256, 0, st>>>(Dp, Pp, Dz, rz, n, D, P, D2, P2);
    return cudaGetLastError();
}

}  // namespace tsgm
