// Device-side bodies of the matching and ragged-offset kernels, shared by the single-image
// kernels (tsgm_match.cu, tsgm_predict.cu) and the batched ones (tsgm_batch.cu). Each function
// does the work of one unit (a census tile, a group of pixels, a path line, an image row) of one
// image; the kernels only decide which unit and which image.
#pragma once

#include <cfloat>

#include "tsgm_internal.cuh"

namespace tsgm {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool valid_value(float v) { return v >= 0.0f && v <= FLT_MAX; }

// Storage of one pixel's window in the ragged volumes: rounded up to a multiple of 4 cells so that
// every block starts 4-byte aligned in the uint8 volumes (32-bit loads and stores of 4 labels).
__device__ __forceinline__ uint32_t block_cells(int w) { return (uint32_t)((w + 3) & ~3); }

// ---------------------------------------------------------------------------------------------
// Block-wide helpers (blockDim.x a multiple of 32, at most 1024)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* sh /* >= 32 words */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    uint32_t t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0u;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[0] = t;
    }
    __syncthreads();
    const uint32_t r = sh[0];
    __syncthreads();
    return r;
}

// Exclusive scan across the block; returns this thread's exclusive prefix and the block total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = (lane < nw) ? sh[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += u;
        }
        if (lane < nw) sh[lane] = ti - t;  // exclusive prefix of warp totals
        if (lane == nw - 1) sh[32] = ti;   // block total
    }
    __syncthreads();
    const uint32_t r = sh[wid] + inc - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// Caller-supplied windows: copy them clamped into [0, D-1] with lo <= hi (so that every later
// kernel stays inside the ragged volume whatever the input) and write the row's total length.
__device__ __forceinline__ void sanitize_row(const int16_t* __restrict__ lo_in,
                                             const int16_t* __restrict__ hi_in, int W, int D, int y,
                                             int16_t* __restrict__ lo, int16_t* __restrict__ hi,
                                             uint32_t* __restrict__ rowsum,
                                             uint32_t* __restrict__ rowcells) {
    __shared__ uint32_t sh[33];
    uint32_t acc = 0, acc_true = 0;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int i = y * W + x;
        const int a = min(max((int)lo_in[i], 0), D - 1);
        const int b = min(max((int)hi_in[i], a), D - 1);
        lo[i] = (int16_t)a;
        hi[i] = (int16_t)b;
        acc_true += (uint32_t)(b - a + 1);
        acc += block_cells(b - a + 1);
    }
    const uint32_t t = block_sum(acc, sh);
    const uint32_t tt = block_sum(acc_true, sh);
    if (threadIdx.x == 0) {
        rowsum[y] = t;
        rowcells[y] = tt;
    }
}

// Offsets of the ragged volume: pixel i's block starts at off[i] = sum of the (4-aligned) block
// sizes of the pixels before it (row-major); off[n] = storage size. One block per row: base =
// sum of earlier row totals, then a block scan. Also writes the per-pixel descriptor
// {off, lo | w << 16} used by the matching kernels, and (last row) the number of true cells.
__device__ __forceinline__ void offsets_row(const int16_t* __restrict__ lo,
                                            const int16_t* __restrict__ hi,
                                            const uint32_t* __restrict__ rowsum,
                                            const uint32_t* __restrict__ rowcells, int W, int Hh,
                                            int y, uint32_t* __restrict__ off,
                                            uint2* __restrict__ desc,
                                            uint32_t* __restrict__ cells_total) {
    __shared__ uint32_t sh[33];
    uint32_t part = 0;
    for (int r = threadIdx.x; r < y; r += blockDim.x) part += rowsum[r];
    uint32_t base = block_sum(part, sh);
    for (int x0 = 0; x0 < W; x0 += blockDim.x) {
        const int x = x0 + threadIdx.x;
        const int i = y * W + x;
        int a = 0, w = 0;
        if (x < W) {
            a = lo[i];
            w = hi[i] - a + 1;
        }
        const uint32_t bw = (x < W) ? block_cells(w) : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(bw, sh, &tot);
        if (x < W) {
            off[i] = base + ex;
            desc[i] = make_uint2(base + ex, (uint32_t)a | ((uint32_t)w << 16));
        }
        base += tot;
    }
    if (y == Hh - 1) {
        uint32_t c = 0;
        for (int r = threadIdx.x; r < Hh; r += blockDim.x) c += rowcells[r];
        c = block_sum(c, sh);
        if (threadIdx.x == 0) {
            off[(size_t)W * Hh] = base;
            *cells_total = c;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Census transform on a shared-memory tile (32 x 8 outputs per block, border-clamped halo).
// bit b (LSB first) = [I(q) < I(p)], q over the window in row-major order without the centre.
// ---------------------------------------------------------------------------------------------
constexpr int kCtW = 32, kCtH = 8, kCmax = 15;

// one 32 x 8 tile whose top-left output pixel is (bx, by); block of kCtW x kCtH threads
__device__ __forceinline__ void census_tile(const uint8_t* __restrict__ img, int W, int Hh, int cw,
                                            int ch, int bx, int by, uint64_t* __restrict__ out) {
    __shared__ uint8_t tile[kCtH + kCmax][kCtW + kCmax];
    const int rx = cw / 2, ry = ch / 2;
    const int tw = kCtW + 2 * rx, th = kCtH + 2 * ry;
    for (int t = threadIdx.y * kCtW + threadIdx.x; t < tw * th; t += kCtW * kCtH) {
        const int ty = t / tw, tx = t - ty * tw;
        const int gx = min(max(bx + tx - rx, 0), W - 1);
        const int gy = min(max(by + ty - ry, 0), Hh - 1);
        tile[ty][tx] = img[gy * W + gx];
    }
    __syncthreads();
    const int x = bx + threadIdx.x, y = by + threadIdx.y;
    if (x >= W || y >= Hh) return;
    const int cx = threadIdx.x + rx, cy = threadIdx.y + ry;
    const uint8_t c = tile[cy][cx];
    uint64_t code = 0;
    int bit = 0;
    for (int dy = -ry; dy <= ry; ++dy)
        for (int dx = -rx; dx <= rx; ++dx) {
            if (dx == 0 && dy == 0) continue;
            code |= (uint64_t)(tile[cy + dy][cx + dx] < c) << bit;
            ++bit;
        }
    out[y * W + x] = code;
}

// pixels g, g + ngroups, ... of one image, each walked by a group of 8 lanes (lane `sub`)
__device__ __forceinline__ void cost_pixels(const uint64_t* __restrict__ cl,
                                            const uint64_t* __restrict__ cr,
                                            const uint2* __restrict__ desc, int W, int n, int Bc,
                                            uint8_t* __restrict__ C, int g, int sub, int ngroups) {
    for (int i = g; i < n; i += ngroups) {
        const int y = i / W;
        const int x = i - y * W;
        const uint2 dsc = desc[i];
        const uint32_t o = dsc.x;
        const int a = (int)(dsc.y & 0xFFFFu);
        const int w = (int)(dsc.y >> 16);
        const uint64_t c0 = cl[i];
        const uint64_t* row = cr + (size_t)y * W;
        for (int j = sub; j < w; j += 8) {
            const int xr = x - (a + j);
            const int c = xr >= 0 ? __popcll(c0 ^ row[xr]) : Bc;
            C[o + j] = (uint8_t)c;
        }
    }
}

struct SgmLines {
    int start[9];  // prefix sums of line counts per slot
    int code[8];   // direction code per slot
    int nslots;
};

constexpr int kSgmWarps = 8;
constexpr uint32_t kInf2 = ((uint32_t)kInf << 16) | (uint32_t)kInf;

__device__ __forceinline__ void dir_of(int code, int& dx, int& dy) {
    dx = (code == 0 || code == 4 || code == 7) ? 1 : ((code == 1 || code == 5 || code == 6) ? -1 : 0);
    dy = (code == 2 || code == 4 || code == 6) ? 1 : ((code == 3 || code == 5 || code == 7) ? -1 : 0);
}

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// packed pair of 16-bit labels (e, e+1) kept only where inside [lo, hi], +inf elsewhere
__device__ __forceinline__ uint32_t mask_pair(uint32_t v, int e, int lo, int hi) {
    const uint32_t l = (e >= lo && e <= hi) ? (v & 0xFFFFu) : (uint32_t)kInf;
    const uint32_t h = (e + 1 >= lo && e + 1 <= hi) ? (v >> 16) : (uint32_t)kInf;
    return l | (h << 16);
}

// One path line: direction `code`, line index `l` of that direction; Lv is the direction's
// volume, buf0 this warp's two shared buffers of 32*LPL labels.
template <int LPL>
__device__ __forceinline__ void sgm_line(const uint8_t* __restrict__ C,
                                         const uint2* __restrict__ desc, int W, int Hh, int D,
                                         int P1, int P2, int code, int l, uint8_t* __restrict__ Lv,
                                         uint32_t* const buf0) {
    constexpr int NP = LPL / 2;       // packed pairs per lane in the dense representation
    constexpr int DP = 32 * LPL;      // labels covered by the dense representation (>= D)
    const int lane = threadIdx.x & 31;
    int dx, dy;
    dir_of(code, dx, dy);
    int x0, y0;
    if (dy == 0) {
        x0 = dx > 0 ? 0 : W - 1;
        y0 = l;
    } else if (dx == 0) {
        x0 = l;
        y0 = dy > 0 ? 0 : Hh - 1;
    } else if (l < Hh) {
        x0 = dx > 0 ? 0 : W - 1;
        y0 = l;
    } else {
        const int k = l - Hh;
        x0 = dx > 0 ? k + 1 : k;
        y0 = dy > 0 ? 0 : Hh - 1;
    }
    const int nx = dx > 0 ? W - x0 : (dx < 0 ? x0 + 1 : 0x7fffffff);
    const int ny = dy > 0 ? Hh - y0 : (dy < 0 ? y0 + 1 : 0x7fffffff);
    const int len = min(nx, ny);
    const int step = dy * W + dx;
    const int i0 = y0 * W + x0;

    constexpr int kBufPairs = DP / 2;  // two buffers of DP uint16 labels, viewed as pairs

    // dense-label masks: lanes' pairs beyond D hold +inf and contribute nothing
    uint32_t keep[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int e = LPL * lane + 2 * k;
        keep[k] = (e < D ? 0xFFFFu : 0u) | (e + 1 < D ? 0xFFFF0000u : 0u);
    }
    const uint32_t P1P1 = ((uint32_t)P1 << 16) | (uint32_t)P1;
    const uint32_t P2P2 = ((uint32_t)P2 << 16) | (uint32_t)P2;

    int qlo = 0, qw = 0, m = 0;
    int loc = 0;  // where the predecessor lives: 0 narrow registers, 1 dense registers, 2 smem
    int qb = 0;   // smem buffer holding the predecessor when loc == 2
    int Nreg = kInf;
    uint32_t Dreg[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) Dreg[k] = kInf2;

    // Descriptors of the line: block `blk` of 32 pixels (one per lane) in dc0, the next in dc1.
    int blk = 0;
    uint2 dc0 = lane < len ? __ldg(desc + (i0 + lane * step)) : make_uint2(0u, 0u);
    uint2 dc1 = 32 + lane < len ? __ldg(desc + (i0 + (32 + lane) * step)) : make_uint2(0u, 0u);
    // descriptor of pixel kk of the line; kk never decreases and advances by at most one
    auto fetch = [&](int kk, uint32_t& o_, uint32_t& lw_) {
        if ((kk >> 5) != blk) {
            dc0 = dc1;
            ++blk;
            const int t = ((blk + 1) << 5) + lane;
            dc1 = t < len ? __ldg(desc + (i0 + t * step)) : make_uint2(0u, 0u);
        }
        o_ = __shfl_sync(kFull, dc0.x, kk & 31);
        lw_ = __shfl_sync(kFull, dc0.y, kk & 31);
    };
    // write the predecessor into smem buffer 0 if it is held in registers
    auto spill = [&]() {
        if (loc != 2) __syncwarp();  // earlier reads of buffer 0 are done before it is rewritten
        if (loc == 0) {
            if (lane < qw) reinterpret_cast<uint16_t*>(buf0)[qlo + lane] = (uint16_t)Nreg;
        } else if (loc == 1) {
#pragma unroll
            for (int k2 = 0; k2 < NP; ++k2) buf0[(LPL * lane) / 2 + k2] = Dreg[k2];
        }
        if (loc != 2) {
            qb = 0;
            loc = 2;
            __syncwarp();
        }
    };
    auto emit_narrow = [&](uint32_t o, int L, int w) {
        if (lane < w) Lv[o + lane] = (uint8_t)L;
    };
    auto load_dense_cost = [&](uint32_t o, uint32_t (&c2)[NP]) {
        const uint16_t* C16 = reinterpret_cast<const uint16_t*>(C + o);
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
            const int e = LPL * lane + 2 * k2;
            const uint32_t b = (e < D) ? (uint32_t)__ldg(C16 + (e >> 1)) : 0u;
            c2[k2] = __byte_perm(b, 0u, 0x4140);  // bytes (c0, c1) -> u16x2
        }
    };
    // one dense step from the predecessor values Lq (labels LPL*lane + ..), result in Dreg
    auto dense_step = [&](const uint32_t (&Lq)[NP], const uint32_t (&c2)[NP]) -> int {
        uint32_t left_in = __shfl_up_sync(kFull, Lq[NP - 1], 1);
        uint32_t right_in = __shfl_down_sync(kFull, Lq[0], 1);
        if (lane == 0) left_in = kInf2;
        if (lane == 31) right_in = kInf2;
        const uint32_t mm = ((uint32_t)m << 16) | (uint32_t)m;
        const uint32_t mP2 = mm + P2P2;
        uint32_t pmin = kInf2;
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
            const uint32_t prev = (k2 == 0) ? left_in : Lq[k2 - 1];
            const uint32_t next = (k2 == NP - 1) ? right_in : Lq[k2 + 1];
            const uint32_t lm1 = __byte_perm(prev, Lq[k2], 0x5432);  // (d-1) values
            const uint32_t lp1 = __byte_perm(Lq[k2], next, 0x5432);  // (d+1) values
            uint32_t t = vmin2(lm1, lp1) + P1P1;
            t = vmin2(vmin2(t, Lq[k2]), mP2);
            const uint32_t Lnew = (c2[k2] + t) - mm;
            Dreg[k2] = (Lnew & keep[k2]) | (kInf2 & ~keep[k2]);
            pmin = vmin2(pmin, Dreg[k2]);
        }
        return (int)min(pmin & 0xFFFFu, pmin >> 16);
    };
    // dense store: the low byte of every 16-bit label, four labels per 32-bit store when the
    // lane's labels start 4-aligned (LPL a multiple of 4), otherwise two per 16-bit store
    auto emit_dense = [&](uint32_t o) {
        if constexpr (LPL % 4 == 0) {
#pragma unroll
            for (int k4 = 0; k4 < NP / 2; ++k4) {
                const int e = LPL * lane + 4 * k4;
                if (e < D)
                    *reinterpret_cast<uint32_t*>(Lv + o + e) =
                        __byte_perm(Dreg[2 * k4], Dreg[2 * k4 + 1], 0x6420);
            }
        } else {
#pragma unroll
            for (int k2 = 0; k2 < NP; ++k2) {
                const int e = LPL * lane + 2 * k2;
                if (e < D)
                    *reinterpret_cast<uint16_t*>(Lv + o + e) =
                        (uint16_t)__byte_perm(Dreg[k2], 0u, 0x0020);
            }
        }
    };

    uint32_t o, lw;
    fetch(0, o, lw);
    int k = 0;
    while (k < len) {
        int lo = (int)(lw & 0xFFFFu);
        int w = (int)(lw >> 16);
        if (w <= 32) {
            // ------------------------------------------------------------ narrow run
            int c = lane < w ? (int)__ldg(C + o + lane) : 0;
            int L;
            if (k == 0) {
                L = c;
            } else {
                spill();
                const uint16_t* src16 = reinterpret_cast<const uint16_t*>(buf0 + qb * kBufPairs);
                const int d = lo + lane;
                const int qhi = qlo + qw - 1;
                const int vc = (d >= qlo && d <= qhi) ? (int)src16[d] : kInf;
                const int vl = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src16[d - 1] : kInf;
                const int vr = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src16[d + 1] : kInf;
                L = c + min(min(min(vl, vr) + P1, vc), m + P2) - m;
            }
            for (;;) {
                // look one pixel ahead: its descriptor and (if narrow) its costs
                const bool more = k + 1 < len;
                uint32_t o_n = 0, lw_n = 0;
                int c_n = 0;
                if (more) {
                    fetch(k + 1, o_n, lw_n);
                    const int w_n = (int)(lw_n >> 16);
                    c_n = (w_n <= 32 && lane < w_n) ? (int)__ldg(C + o_n + lane) : 0;
                }
                L = lane < w ? L : kInf;
                emit_narrow(o, L, w);
                m = (int)__reduce_min_sync(kFull, (unsigned)L);
                Nreg = L;
                qlo = lo;
                qw = w;
                loc = 0;
                ++k;
                if (!more) break;
                o = o_n;
                lw = lw_n;
                lo = (int)(lw & 0xFFFFu);
                w = (int)(lw >> 16);
                if (w > 32) break;
                const int s_ = lane + (lo - qlo);
                int vc = __shfl_sync(kFull, Nreg, s_ & 31);
                int vl = __shfl_sync(kFull, Nreg, (s_ - 1) & 31);
                int vr = __shfl_sync(kFull, Nreg, (s_ + 1) & 31);
                vc = ((unsigned)s_ < (unsigned)qw) ? vc : kInf;
                vl = ((unsigned)(s_ - 1) < (unsigned)qw) ? vl : kInf;
                vr = ((unsigned)(s_ + 1) < (unsigned)qw) ? vr : kInf;
                L = c_n + min(min(min(vl, vr) + P1, vc), m + P2) - m;
            }
        } else if (w == D) {
            // ------------------------------------------------------------ full-range run
            uint32_t c2[NP];
            load_dense_cost(o, c2);
            int lmin;
            if (k == 0) {
                uint32_t pmin = kInf2;
#pragma unroll
                for (int k2 = 0; k2 < NP; ++k2) {
                    Dreg[k2] = (c2[k2] & keep[k2]) | (kInf2 & ~keep[k2]);
                    pmin = vmin2(pmin, Dreg[k2]);
                }
                lmin = (int)min(pmin & 0xFFFFu, pmin >> 16);
            } else {
                spill();
                const uint32_t* srcp = buf0 + qb * kBufPairs;
                const int qhi = qlo + qw - 1;
                uint32_t Lq[NP];
#pragma unroll
                for (int k2 = 0; k2 < NP; ++k2)
                    Lq[k2] = mask_pair(srcp[(LPL * lane) / 2 + k2], LPL * lane + 2 * k2, qlo, qhi);
                lmin = dense_step(Lq, c2);
            }
            for (;;) {
                const bool more = k + 1 < len;
                uint32_t o_n = 0, lw_n = 0;
                if (more) {
                    fetch(k + 1, o_n, lw_n);
                    if ((int)(lw_n >> 16) == D) load_dense_cost(o_n, c2);
                }
                emit_dense(o);
                m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
                qlo = 0;
                qw = D;
                loc = 1;
                ++k;
                if (!more) break;
                o = o_n;
                lw = lw_n;
                if ((int)(lw >> 16) != D) break;
                uint32_t Lq[NP];
#pragma unroll
                for (int k2 = 0; k2 < NP; ++k2) Lq[k2] = Dreg[k2];
                lmin = dense_step(Lq, c2);
            }
        } else {
            // ------------------------------------------------------------ general window
            if (k > 0) spill();
            __syncwarp();
            const uint16_t* src16 = reinterpret_cast<const uint16_t*>(buf0 + qb * kBufPairs);
            uint16_t* dst16 = reinterpret_cast<uint16_t*>(buf0 + (qb ^ 1) * kBufPairs);
            const int qhi = qlo + qw - 1;
            int lmin = kInf;
            for (int j0 = 0; j0 < w; j0 += 32) {
                const int j = j0 + lane;
                const bool act = j < w;
                const int d = lo + j;
                const int c = act ? (int)__ldg(C + o + j) : 0;
                int L;
                if (k == 0) {
                    L = c;
                } else {
                    const int vc = (d >= qlo && d <= qhi) ? (int)src16[d] : kInf;
                    const int vl = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src16[d - 1] : kInf;
                    const int vr = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src16[d + 1] : kInf;
                    L = c + min(min(min(vl, vr) + P1, vc), m + P2) - m;
                }
                L = act ? L : kInf;
                if (act) dst16[d] = (uint16_t)L;
                lmin = min(lmin, L);
                if (act) Lv[o + j] = (uint8_t)L;
            }
            m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
            qb ^= 1;
            loc = 2;
            qlo = lo;
            qw = w;
            __syncwarp();
            if (++k < len) fetch(k, o, lw);
        }
    }
}

constexpr int kSelThreads = 512;
constexpr int kSelNarrow = 16;

__device__ __forceinline__ int count_side(const uint16_t* __restrict__ s, int start, int dirn,
                                          int lo_idx, int hi_idx, int s0, float thr, int lane) {
    int carry = 0, count = 0;
    for (int t0 = 0;; t0 += 32) {
        const int jj = start + dirn * (t0 + lane);
        const bool in = jj >= lo_idx && jj <= hi_idx;
        int v = in ? (int)s[jj] - s0 : (1 << 20);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += u;
        }
        const unsigned ok = __ballot_sync(kFull, (float)(carry + v) < thr);
        const int c = __popc(ok);
        count += c;
        const int tot = __shfl_sync(kFull, v, 31);
        if (c < 32) break;
        carry += tot;
    }
    return count;
}

// sum of the path volumes for labels j .. j+3 of the block at o: two u16x2 words
template <int NPATHS>
__device__ __forceinline__ void sum_paths(const uint8_t* __restrict__ Lvol, uint64_t stride,
                                          uint32_t o, int j, uint32_t& p0, uint32_t& p1) {
    uint32_t v[NPATHS];
#pragma unroll
    for (int r = 0; r < NPATHS; ++r)
        v[r] = __ldg(reinterpret_cast<const uint32_t*>(Lvol + r * stride + o + j));
    p0 = 0u;
    p1 = 0u;
#pragma unroll
    for (int r = 0; r < NPATHS; ++r) {
        p0 += __byte_perm(v[r], 0u, 0x4140);
        p1 += __byte_perm(v[r], 0u, 0x4342);
    }
}

// One image row y of one image; a whole block works on it. `smem` holds the per-column state of
// the row followed by the per-warp scratch; `n_wide` is a block-shared counter.
template <int NPATHS>
__device__ __forceinline__ void select_row(
    const uint8_t* __restrict__ Lvol, uint64_t vol_stride, const uint2* __restrict__ desc, int W,
    int y, int DP, float s_thr, float r_min, int lr_tol, float* __restrict__ Dz,
    float* __restrict__ rz, uint16_t* __restrict__ S_out, int16_t* __restrict__ dstar_out,
    int16_t* __restrict__ dright_out, uint8_t* __restrict__ valid_out, uint32_t* sel_smem,
    int& n_wide) {
    uint32_t* drk = sel_smem;                    // W keys
    float* dzs = (float*)(drk + W);              // W
    float* rzs = dzs + W;                        // W
    int16_t* ds = (int16_t*)(rzs + W);           // W
    int16_t* wideq = ds + W;                     // W queued wide pixels
    // per-warp scratch of DP labels, 8-byte aligned for the 4-label stores
    uint16_t* scr_all = (uint16_t*)(sel_smem + ((3 * W + W + 1) & ~1));
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int x = threadIdx.x; x < W; x += blockDim.x) drk[x] = 0xFFFFFFFFu;
    if (threadIdx.x == 0) n_wide = 0;
    __syncthreads();

    // ---- narrow windows: one thread per pixel
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int i = y * W + x;
        const uint2 dsc = desc[i];
        const uint32_t o = dsc.x;
        const int a = (int)(dsc.y & 0xFFFFu);
        const int w = (int)(dsc.y >> 16);
        if (w > kSelNarrow) {
            wideq[atomicAdd(&n_wide, 1)] = (int16_t)x;
            continue;
        }
        uint32_t sp[kSelNarrow / 2];  // S as u16x2 pairs
#pragma unroll
        for (int q = 0; q < kSelNarrow / 4; ++q) {
            if (4 * q < w) {
                sum_paths<NPATHS>(Lvol, vol_stride, o, 4 * q, sp[2 * q], sp[2 * q + 1]);
                if (S_out) *reinterpret_cast<uint2*>(S_out + o + 4 * q) = make_uint2(sp[2 * q], sp[2 * q + 1]);
            } else {
                sp[2 * q] = 0xFFFFFFFFu;
                sp[2 * q + 1] = 0xFFFFFFFFu;
            }
        }
        int sv[kSelNarrow];
#pragma unroll
        for (int j = 0; j < kSelNarrow; ++j)
            sv[j] = (j < w) ? (int)((j & 1) ? (sp[j >> 1] >> 16) : (sp[j >> 1] & 0xFFFFu)) : 0x7FFFFFFF;
        int js = 0, s0 = sv[0];
#pragma unroll
        for (int j = 1; j < kSelNarrow; ++j)
            if (sv[j] < s0) {
                s0 = sv[j];
                js = j;
            }
        int sm = 0, spv = 0;
#pragma unroll
        for (int j = 0; j < kSelNarrow; ++j) {
            if (j == js - 1) sm = sv[j];
            if (j == js + 1) spv = sv[j];
            if (j < w) {
                const int xr = x - (a + j);
                if (xr >= 0) atomicMin(drk + xr, ((uint32_t)sv[j] << 9) | (uint32_t)(a + j));
            }
        }
        float delta = 0.0f;
        if (js >= 1 && js + 1 < w) {
            const int den = 2 * (sm - 2 * s0 + spv);
            if (den > 0) delta = __fdiv_rn((float)(sm - spv), (float)den);
        }
        // counts: running sums outwards from d*; walking labels in order of distance keeps the
        // sums growing, so every label whose sum is below the threshold is in the counted run
        int nl = 0, nr = 0, acc = 0;
#pragma unroll
        for (int j = kSelNarrow - 1; j >= 0; --j) {
            if (j < js) {
                acc += sv[j] - s0;
                nl += ((float)acc < s_thr) ? 1 : 0;
            }
        }
        acc = 0;
#pragma unroll
        for (int j = 0; j < kSelNarrow; ++j) {
            if (j > js && j < w) {
                acc += sv[j] - s0;
                nr += ((float)acc < s_thr) ? 1 : 0;
            }
        }
        float r = (float)(nl + nr);
        if (r < r_min) r = r_min;
        ds[x] = (int16_t)(a + js);
        dzs[x] = __fadd_rn((float)(a + js), delta);
        rzs[x] = r;
    }
    __syncthreads();

    // ---- wide windows: one warp per pixel
    uint16_t* scr = scr_all + wid * DP;
    const int nwide = n_wide;
    for (int q = wid; q < nwide; q += nw) {
        const int x = wideq[q];
        const int i = y * W + x;
        const uint2 dsc = desc[i];
        const uint32_t o = dsc.x;
        const int a = (int)(dsc.y & 0xFFFFu);
        const int w = (int)(dsc.y >> 16);
        unsigned best = 0xFFFFFFFFu;
        for (int j = 4 * lane; j < w; j += 128) {
            uint32_t p0, p1;
            sum_paths<NPATHS>(Lvol, vol_stride, o, j, p0, p1);
            *reinterpret_cast<uint2*>(scr + j) = make_uint2(p0, p1);
            if (S_out) *reinterpret_cast<uint2*>(S_out + o + j) = make_uint2(p0, p1);
            const unsigned sv[4] = {p0 & 0xFFFFu, p0 >> 16, p1 & 0xFFFFu, p1 >> 16};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (j + t < w) {
                    best = min(best, (sv[t] << 16) | (unsigned)(j + t));
                    const int xr = x - (a + j + t);
                    if (xr >= 0) atomicMin(drk + xr, (sv[t] << 9) | (unsigned)(a + j + t));
                }
            }
        }
        __syncwarp();
        best = __reduce_min_sync(kFull, best);
        const int js = (int)(best & 0xFFFFu);
        const int s0 = (int)(best >> 16);
        float delta = 0.0f;
        if (js >= 1 && js + 1 < w) {
            const int smv = scr[js - 1], spv = scr[js + 1];
            const int den = 2 * (smv - 2 * s0 + spv);
            if (den > 0) delta = __fdiv_rn((float)(smv - spv), (float)den);
        }
        const int nl = count_side(scr, js - 1, -1, 0, w - 1, s0, s_thr, lane);
        const int nr = count_side(scr, js + 1, +1, 0, w - 1, s0, s_thr, lane);
        float r = (float)(nl + nr);
        if (r < r_min) r = r_min;
        if (lane == 0) {
            ds[x] = (int16_t)(a + js);
            dzs[x] = __fadd_rn((float)(a + js), delta);
            rzs[x] = r;
        }
        __syncwarp();
    }
    __syncthreads();
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int i = y * W + x;
        const int d = ds[x];
        const int xr = x - d;
        bool ok = false;
        if (xr >= 0) {
            const uint32_t kk = drk[xr];
            ok = kk != 0xFFFFFFFFu && abs(d - (int)(kk & 0x1FFu)) <= lr_tol;
        }
        Dz[i] = ok ? dzs[x] : -1.0f;
        rz[i] = ok ? rzs[x] : -1.0f;
        if (dstar_out) {
            dstar_out[i] = (int16_t)d;
            const uint32_t kx = drk[x];
            dright_out[i] = kx == 0xFFFFFFFFu ? (int16_t)-1 : (int16_t)(kx & 0x1FFu);
            valid_out[i] = ok ? 1 : 0;
        }
    }
}

}  // namespace dev
}  // namespace tsgm
