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

// Windows wider than this many labels leave the narrow representation of the path aggregation
// (one label per lane); their count per row is kept with the row totals (rowwide).
constexpr int kNarrowMax = 32;

// Windows of at most this many labels are selected by one thread; wider ones by a warp.
constexpr int kSelNarrow = 16;

// Queue of the pixels wider than kSelNarrow: wq[0] their number, wq[1 ..] their indices. They are selected apart from their rows (select_wide) unless more than
// a quarter of the image is wide, when every row takes its own (one decision for the whole image,
// from wq[0], by both selection kernels).
__host__ __device__ __forceinline__ bool select_split(uint32_t n_wide, int n) {
    return 4ull * n_wide <= (unsigned long long)n;
}

// Row statistics written next to the windows: storage cells, true cells, pixels wider than
// kNarrowMax (rowwide).
__device__ __forceinline__ void row_totals(uint32_t acc, uint32_t acc_true, uint32_t acc_wide,
                                           int y, uint32_t* sh, uint32_t* __restrict__ rowsum,
                                           uint32_t* __restrict__ rowcells,
                                           uint32_t* __restrict__ rowwide) {
    const uint32_t t = block_sum(acc, sh);
    const uint32_t tt = block_sum(acc_true, sh);
    const uint32_t tw = block_sum(acc_wide, sh);
    if (threadIdx.x == 0) {
        rowsum[y] = t;
        rowcells[y] = tt;
        rowwide[y] = tw;
    }
}

// Caller-supplied windows: copy them clamped into [0, D-1] with lo <= hi (so that every later
// kernel stays inside the ragged volume whatever the input) and write the row's totals.
__device__ __forceinline__ void sanitize_row(const int16_t* __restrict__ lo_in,
                                             const int16_t* __restrict__ hi_in, int W, int D, int y,
                                             int16_t* __restrict__ lo, int16_t* __restrict__ hi,
                                             uint32_t* __restrict__ rowsum,
                                             uint32_t* __restrict__ rowcells,
                                             uint32_t* __restrict__ rowwide) {
    __shared__ uint32_t sh[33];
    uint32_t acc = 0, acc_true = 0, acc_wide = 0;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int i = y * W + x;
        const int a = min(max((int)lo_in[i], 0), D - 1);
        const int b = min(max((int)hi_in[i], a), D - 1);
        lo[i] = (int16_t)a;
        hi[i] = (int16_t)b;
        acc_true += (uint32_t)(b - a + 1);
        acc += block_cells(b - a + 1);
        acc_wide += (b - a + 1 > kNarrowMax) ? 1u : 0u;
    }
    row_totals(acc, acc_true, acc_wide, y, sh, rowsum, rowcells, rowwide);
}

// Offsets of the ragged volume: pixel i's block starts at off[i] = sum of the (4-aligned) block
// sizes of the pixels before it (row-major); off[n] = storage size. One block per row: base =
// sum of earlier row totals, then a block scan. Also writes the per-pixel descriptor
// {off, lo | w << 16} used by the matching kernels, and (last row) the number of true cells in
// cells_total[0] and the number of pixels wider than kNarrowMax in cells_total[1].
__device__ __forceinline__ void offsets_row(const int16_t* __restrict__ lo,
                                            const int16_t* __restrict__ hi,
                                            const uint32_t* __restrict__ rowsum,
                                            const uint32_t* __restrict__ rowcells,
                                            const uint32_t* __restrict__ rowwide, int W, int Hh,
                                            int y, uint32_t* __restrict__ off,
                                            uint2* __restrict__ desc,
                                            uint32_t* __restrict__ cells_total,
                                            uint32_t* __restrict__ wq) {
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
        if (wq) {
            // the wide pixels of this chunk of the row into the queue: places within the block by
            // a shared counter, one global atomic per chunk
            __shared__ uint32_t wcnt, wbase;
            if (threadIdx.x == 0) wcnt = 0u;
            __syncthreads();
            const unsigned bal = __ballot_sync(kFull, x < W && w > kSelNarrow);
            const int lane = threadIdx.x & 31;
            uint32_t at = 0;
            if (lane == 0 && bal) at = atomicAdd(&wcnt, (uint32_t)__popc(bal));
            at = __shfl_sync(kFull, at, 0);
            __syncthreads();
            if (threadIdx.x == 0) wbase = wcnt ? atomicAdd(wq, wcnt) : 0u;
            __syncthreads();
            if ((bal >> lane) & 1u)
                wq[1 + wbase + at + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)i;
        }
        base += tot;
    }
    if (y == Hh - 1) {
        uint32_t c = 0, wd = 0;
        for (int r = threadIdx.x; r < Hh; r += blockDim.x) {
            c += rowcells[r];
            wd += rowwide[r];
        }
        c = block_sum(c, sh);
        wd = block_sum(wd, sh);
        if (threadIdx.x == 0) {
            off[(size_t)W * Hh] = base;
            cells_total[0] = c;
            cells_total[1] = wd;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Census transform on a shared-memory tile (32 x 8 outputs per block, border-clamped halo).
// bit b (LSB first) = [I(q) < I(p)], q over the window in row-major order without the centre.
// ---------------------------------------------------------------------------------------------
constexpr int kCtW = 32, kCtH = 8, kCmax = 15;

// one 32 x 8 tile whose top-left output pixel is (bx, by); block of kCtW x kCtH threads.
// CW x CH > 0: the window size is a compile-time constant and the comparisons unroll into
// constant bit positions; 0 x 0: any size given at run time (cw, ch).
template <int CW, int CH>
__device__ __forceinline__ void census_tile(const uint8_t* __restrict__ img, int W, int Hh, int cw,
                                            int ch, int bx, int by, uint64_t* __restrict__ out) {
    __shared__ uint8_t tile[kCtH + kCmax][kCtW + kCmax];
    if constexpr (CW > 0) {
        cw = CW;
        ch = CH;
    }
    const int rx = cw / 2, ry = ch / 2;
    const int tw = kCtW + 2 * rx, th = kCtH + 2 * ry;
    for (int ty = threadIdx.y; ty < th; ty += kCtH) {
        const int gy = min(max(by + ty - ry, 0), Hh - 1);
        for (int tx = threadIdx.x; tx < tw; tx += kCtW) {
            const int gx = min(max(bx + tx - rx, 0), W - 1);
            tile[ty][tx] = img[gy * W + gx];
        }
    }
    __syncthreads();
    const int x = bx + threadIdx.x, y = by + threadIdx.y;
    if (x >= W || y >= Hh) return;
    const int cx = threadIdx.x + rx, cy = threadIdx.y + ry;
    const uint8_t c = tile[cy][cx];
    uint64_t code = 0;
    if constexpr (CW > 0) {
        constexpr int RX = CW / 2, RY = CH / 2;
#pragma unroll
        for (int dy = -RY; dy <= RY; ++dy)
#pragma unroll
            for (int dx = -RX; dx <= RX; ++dx) {
                if (dx == 0 && dy == 0) continue;
                const int bit = (dy + RY) * CW + (dx + RX) - ((dy > 0 || (dy == 0 && dx > 0)) ? 1 : 0);
                code |= (uint64_t)(tile[cy + dy][cx + dx] < c) << bit;
            }
    } else {
        int bit = 0;
        for (int dy = -ry; dy <= ry; ++dy)
            for (int dx = -rx; dx <= rx; ++dx) {
                if (dx == 0 && dy == 0) continue;
                code |= (uint64_t)(tile[cy + dy][cx + dx] < c) << bit;
                ++bit;
            }
    }
    out[y * W + x] = code;
}

// pixels g, g + ngroups, ... of one image, each walked by a group of kCostLanes = 4 lanes (lane
// `sub` takes cells 4 sub .. 4 sub + 3 of every 16, one 32-bit store; a pixel's block is a multiple of 4
// cells, so the last word's cells past the window are padding); the row and column advance by the
// stride's quotient and remainder (no division per pixel), and the next pixel's descriptor and
// left code are loaded while the current one's cells are computed
constexpr int kCostLanes = 4;  // lanes per pixel of the cost computation

__device__ __forceinline__ void cost_pixels(const uint64_t* __restrict__ cl,
                                            const uint64_t* __restrict__ cr,
                                            const uint2* __restrict__ desc, int W, int n, int Bc,
                                            uint8_t* __restrict__ C, int g, int sub, int ngroups) {
    const int dy = g + ngroups < n ? ngroups / W : 0, dx = ngroups - dy * W;  // one pixel: unused
    int y = g / W, x = g - y * W;
    uint2 dnext = g < n ? desc[g] : make_uint2(0u, 0u);
    uint64_t cnext = g < n ? cl[g] : 0ull;
    for (int i = g; i < n; i += ngroups) {
        const uint2 dsc = dnext;
        const uint64_t c0 = cnext;
        if (i + ngroups < n) {
            dnext = desc[i + ngroups];
            cnext = cl[i + ngroups];
        }
        const uint32_t o = dsc.x;
        const int a = (int)(dsc.y & 0xFFFFu);
        const int w = (int)(dsc.y >> 16);
        const uint64_t* row = cr + (size_t)y * W;
        for (int j = 4 * sub; j < w; j += 4 * kCostLanes) {
            const int xr = x - (a + j);  // cells j .. j + 3 match columns xr .. xr - 3
            uint32_t word = 0u;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = xr - q >= 0 ? __popcll(c0 ^ row[xr - q]) : Bc;
                word |= (uint32_t)c << (8 * q);
            }
            *reinterpret_cast<uint32_t*>(C + o + j) = word;
        }
        y += dy;
        x += dx;
        if (x >= W) {
            x -= W;
            ++y;
        }
    }
}

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

// Start pixel, step and length of line l of direction `code` in a W x Hh image.
__device__ __forceinline__ void line_geometry(int code, int l, int W, int Hh, int& i0, int& step,
                                              int& len) {
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
    len = min(nx, ny);
    step = dy * W + dx;
    i0 = y0 * W + x0;
}

// Asynchronous copies global -> shared complete by commit groups (not by the issuing thread's
// registers, so that many copies can be in flight per warp).
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kSelThreads = 512;

// The Eq. 9 threshold as an integer. A running sum n of in-window labels is below 2^20 (at most
// 256 labels of S <= 8 x 255), and for such n, (float)n < thr exactly when n < count_limit(thr):
// the least integer not below thr, capped at 2^20 (none for thr <= 0 or NaN). count_side's
// out-of-window sentinel (2^20) is then never counted, whatever thr.
__device__ __forceinline__ int count_limit(float thr) {
    return thr > 0.0f ? (thr >= 1048576.0f ? 1048576 : (int)ceilf(thr)) : 0;
}

__device__ __forceinline__ int count_side(const uint16_t* __restrict__ s, int start, int dirn,
                                          int lo_idx, int hi_idx, int s0, int lim, int lane) {
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
        const unsigned ok = __ballot_sync(kFull, carry + v < lim);
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

// One window wider than kSelNarrow by a whole warp (Eq. 9 and the right-view keys): v holds this
// lane's words of the NPATHS path-cost volumes (labels 4 lane + 128 c .. + 3 of chunk c). The
// aggregated costs go to the warp's scratch scr (and to S_out when given), the right-view key of
// every label to keymin(xr, key); returns the winner, its sub-pixel disparity and the matching
// variance.
template <int NPATHS, int NCH, class KeyMin>
__device__ __forceinline__ void select_wide(const uint32_t (&v)[NCH * NPATHS], uint2 dsc, int x,
                                            float s_thr, float r_min, uint16_t* scr,
                                            uint16_t* __restrict__ S_out, const KeyMin& keymin,
                                            int& dstar, float& dz, float& rr) {
    const int lane = threadIdx.x & 31;
    const uint32_t o = dsc.x;
    const int a = (int)(dsc.y & 0xFFFFu);
    const int w = (int)(dsc.y >> 16);
    unsigned best = 0xFFFFFFFFu;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const int j = 4 * lane + 128 * c;
        if (j < w) {
            uint32_t p0 = 0u, p1 = 0u;
#pragma unroll
            for (int r = 0; r < NPATHS; ++r) {
                p0 += __byte_perm(v[c * NPATHS + r], 0u, 0x4140);
                p1 += __byte_perm(v[c * NPATHS + r], 0u, 0x4342);
            }
            *reinterpret_cast<uint2*>(scr + j) = make_uint2(p0, p1);
            if (S_out) *reinterpret_cast<uint2*>(S_out + o + j) = make_uint2(p0, p1);
            const unsigned sv[4] = {p0 & 0xFFFFu, p0 >> 16, p1 & 0xFFFFu, p1 >> 16};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (j + t < w) {
                    best = min(best, (sv[t] << 16) | (unsigned)(j + t));
                    const int xr = x - (a + j + t);
                    if (xr >= 0) keymin(xr, (sv[t] << 9) | (unsigned)(a + j + t));
                }
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
    const int lim = count_limit(s_thr);
    const int nl = count_side(scr, js - 1, -1, 0, w - 1, s0, lim, lane);
    const int nr = count_side(scr, js + 1, +1, 0, w - 1, s0, lim, lane);
    float r = (float)(nl + nr);
    if (r < r_min) r = r_min;
    dstar = a + js;
    dz = __fadd_rn((float)(a + js), delta);
    rr = r;
    __syncwarp();  // the scratch is free for the next pixel
}

// The path costs of a wide window (see select_wide) into this lane's words v.
template <int NPATHS, int NCH>
__device__ __forceinline__ void load_wide_costs(const uint8_t* __restrict__ Lvol, uint64_t stride,
                                                uint2 dsc, uint32_t (&v)[NCH * NPATHS]) {
    const int lane = threadIdx.x & 31;
    const int w = (int)(dsc.y >> 16);
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const int j = 4 * lane + 128 * c;
#pragma unroll
        for (int r = 0; r < NPATHS; ++r)
            v[c * NPATHS + r] =
                j < w ? __ldg(reinterpret_cast<const uint32_t*>(Lvol + r * stride + dsc.x + j)) : 0u;
    }
}

// Full-range selection (every window [0, D - 1], pixel i's block of rD cells at cell i rD): lane
// j's cost words of pixel i, labels LPL j .. LPL j + LPL - 1 of each of the NPATHS volumes (words
// past D read as 0).
template <int NPATHS, int LPL>
__device__ __forceinline__ void load_full_costs(const uint8_t* __restrict__ Lvol, uint64_t stride,
                                                size_t o, int D, uint32_t (&v)[NPATHS * (LPL >= 4 ? LPL / 4 : 1)]) {
    constexpr int NW = LPL >= 4 ? LPL / 4 : 1;
    const int base = LPL * (int)(threadIdx.x & 31);
#pragma unroll
    for (int r = 0; r < NPATHS; ++r) {
        const uint8_t* const src = Lvol + r * stride + o + base;
        if constexpr (LPL == 2) {
            v[r] = base < D ? (uint32_t)__ldg(reinterpret_cast<const uint16_t*>(src)) : 0u;
        } else {
#pragma unroll
            for (int g = 0; g < NW; ++g)
                v[r * NW + g] = base + 4 * g < D ? __ldg(reinterpret_cast<const uint32_t*>(src) + g) : 0u;
        }
    }
}

// One full-range pixel by a whole warp (Eq. 9 and the right-view keys), v from load_full_costs:
// the sums S(d) of the path costs (with `bytesum`, when every path cost is below 128, two volumes'
// words are added bytewise first), every label's right-view key to keymin(xr, S << 9 | d) for
// xr = x - d >= 0, and the winner d* (least S, then least d; the same keys order both), its
// sub-pixel offset and the matching variance, as select_wide. scr: this warp's D labels of
// scratch.
template <int NPATHS, int LPL, class KeyMin>
__device__ __forceinline__ void select_full_px(const uint32_t (&v)[NPATHS * (LPL >= 4 ? LPL / 4 : 1)],
                                               int D, bool bytesum, int x, size_t o, float s_thr,
                                               float r_min, uint16_t* scr,
                                               uint16_t* __restrict__ S_out, const KeyMin& keymin,
                                               int& dstar, float& dz, float& rr) {
    constexpr int NW = LPL >= 4 ? LPL / 4 : 1;
    constexpr int NP = LPL / 2;
    const int lane = threadIdx.x & 31;
    const int base = LPL * lane;
    // S as packed pairs (labels base + 2k, base + 2k + 1)
    uint32_t S[NP];
#pragma unroll
    for (int g = 0; g < NW; ++g) {
        uint32_t p0 = 0u, p1 = 0u;
        if (bytesum && NPATHS % 2 == 0) {
#pragma unroll
            for (int r = 0; r < NPATHS; r += 2) {
                const uint32_t b = v[r * NW + g] + v[(r + 1) * NW + g];  // bytes < 256: no carry
                p0 += __byte_perm(b, 0u, 0x4140);
                p1 += __byte_perm(b, 0u, 0x4342);
            }
        } else {
#pragma unroll
            for (int r = 0; r < NPATHS; ++r) {
                p0 += __byte_perm(v[r * NW + g], 0u, 0x4140);
                p1 += __byte_perm(v[r * NW + g], 0u, 0x4342);
            }
        }
        S[2 * g] = p0;
        if (2 * g + 1 < NP) S[2 * g + 1] = p1;
    }
    if constexpr (LPL == 2) {
        if (base < D) {
            *reinterpret_cast<uint32_t*>(scr + base) = S[0];
            if (S_out) *reinterpret_cast<uint32_t*>(S_out + o + base) = S[0];
        }
    } else {
#pragma unroll
        for (int g = 0; g < NW; ++g) {
            if (base + 4 * g < D) {
                *reinterpret_cast<uint2*>(scr + base + 4 * g) = make_uint2(S[2 * g], S[2 * g + 1]);
                if (S_out) *reinterpret_cast<uint2*>(S_out + o + base + 4 * g) = make_uint2(S[2 * g], S[2 * g + 1]);
            }
        }
    }
    unsigned best = 0xFFFFFFFFu;
    const bool all_xr = x >= D - 1;  // every label's right-view column inside the image
#pragma unroll
    for (int t = 0; t < LPL; ++t) {
        const int d = base + t;
        if (d < D) {
            const unsigned sv = (t & 1) ? (S[t >> 1] >> 16) : (S[t >> 1] & 0xFFFFu);
            const unsigned key = (sv << 9) | (unsigned)d;
            best = min(best, key);
            if (all_xr || x - d >= 0) keymin(x - d, key);
        }
    }
    __syncwarp();
    best = __reduce_min_sync(kFull, best);
    const int js = (int)(best & 0x1FFu);
    const int s0 = (int)(best >> 9);
    float delta = 0.0f;
    if (js >= 1 && js + 1 < D) {
        const int smv = scr[js - 1], spv = scr[js + 1];
        const int den = 2 * (smv - 2 * s0 + spv);
        if (den > 0) delta = __fdiv_rn((float)(smv - spv), (float)den);
    }
    const int lim = count_limit(s_thr);
    const int nl = count_side(scr, js - 1, -1, 0, D - 1, s0, lim, lane);
    const int nr = count_side(scr, js + 1, +1, 0, D - 1, s0, lim, lane);
    float r = (float)(nl + nr);
    if (r < r_min) r = r_min;
    dstar = js;
    dz = __fadd_rn((float)js, delta);
    rr = r;
    __syncwarp();  // the scratch is free for the next pixel
}

// One window of at most NL (a multiple of 4, <= kSelNarrow) labels by one thread: its aggregated
// costs (to S_out when given), every label's right-view key to keymin(xr, key), the winner's index
// js in the window, its sub-pixel offset delta and the matching variance r (Eq. 9).
template <int NPATHS, int NL, class KeyMin>
__device__ __forceinline__ void select_narrow(const uint8_t* __restrict__ Lvol, uint64_t vol_stride,
                                              uint32_t o, int a, int w, int x, float s_thr,
                                              float r_min, uint16_t* __restrict__ S_out,
                                              const KeyMin& keymin, int& js_out, float& delta_out,
                                              float& r_out) {
    uint32_t sp[NL / 2];  // S as u16x2 pairs
#pragma unroll
    for (int q = 0; q < NL / 4; ++q) {
        if (4 * q < w) {
            sum_paths<NPATHS>(Lvol, vol_stride, o, 4 * q, sp[2 * q], sp[2 * q + 1]);
            if (S_out) *reinterpret_cast<uint2*>(S_out + o + 4 * q) = make_uint2(sp[2 * q], sp[2 * q + 1]);
        } else {
            sp[2 * q] = 0xFFFFFFFFu;
            sp[2 * q + 1] = 0xFFFFFFFFu;
        }
    }
    int sv[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j)
        sv[j] = (j < w) ? (int)((j & 1) ? (sp[j >> 1] >> 16) : (sp[j >> 1] & 0xFFFFu)) : 0x7FFFFFFF;
    int js = 0, s0 = sv[0];
#pragma unroll
    for (int j = 1; j < NL; ++j)
        if (sv[j] < s0) {
            s0 = sv[j];
            js = j;
        }
    int sm = 0, spv = 0;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
        if (j == js - 1) sm = sv[j];
        if (j == js + 1) spv = sv[j];
        if (j < w) {
            const int xr = x - (a + j);
            if (xr >= 0) keymin(xr, ((uint32_t)sv[j] << 9) | (uint32_t)(a + j));
        }
    }
    float delta = 0.0f;
    if (js >= 1 && js + 1 < w) {
        const int den = 2 * (sm - 2 * s0 + spv);
        if (den > 0) delta = __fdiv_rn((float)(sm - spv), (float)den);
    }
    // counts: running sums outwards from d*; walking labels in order of distance keeps the
    // sums growing, so every label whose sum is below the threshold is in the counted run
    const int lim = count_limit(s_thr);
    int nl = 0, nr = 0, acc = 0;
#pragma unroll
    for (int j = NL - 1; j >= 0; --j) {
        if (j < js) {
            acc += sv[j] - s0;
            nl += acc < lim ? 1 : 0;
        }
    }
    acc = 0;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
        if (j > js && j < w) {
            acc += sv[j] - s0;
            nr += acc < lim ? 1 : 0;
        }
    }
    float r = (float)(nl + nr);
    if (r < r_min) r = r_min;
    js_out = js;
    delta_out = delta;
    r_out = r;
}

// Selection of the pixels [x0, x1) of image row y (Eq. 9 and the left-right check), by one block.
// The right-view keys of the row (per column xr, the (S << 9 | d) minimum over the pixels
// x = xr + d whose window holds d) are reached through `part`: keymin(xr, key) (an atomic minimum
// from one of this block's pixels), key(xr) (the row's final key, after sync()), own_keys(),
// nkeys and key_base() (this block's key array and the column of its first key) and sync()
// (every block working on the row). Narrow windows: one thread each. Wide ones: when the image
// is split (select_split over the queue wq), already selected by select_wide, whose winners are
// in wds and whose keys this block merges from gkeys_row (and resets for the next image);
// otherwise queued in the block and taken one warp each. `smem` holds this block's keys and the
// per-pixel state of its pixels, then the per-warp scratch; `n_wide` is block-shared.
template <int NPATHS, int NCH, class Part>
__device__ __forceinline__ void select_part(
    const uint8_t* __restrict__ Lvol, uint64_t vol_stride, const uint2* __restrict__ desc, int W,
    int y, int x0, int x1, int DP, float s_thr, float r_min, int lr_tol, float* __restrict__ Dz,
    float* __restrict__ rz, uint16_t* __restrict__ S_out, int16_t* __restrict__ dstar_out,
    int16_t* __restrict__ dright_out, uint8_t* __restrict__ valid_out, uint32_t* sel_smem,
    int& n_wide, Part& part, int n, const uint32_t* __restrict__ wq,
    uint32_t* __restrict__ gkeys_row, const int16_t* __restrict__ wds) {
    // split: the wide pixels were selected apart (select_wide over the queue wq); their winners
    // are in wds, their keys in gkeys_row (merged here and reset for the next image)
    const bool split = wq != nullptr && select_split(wq[0], n);
    const int npx = x1 - x0;
    uint32_t* drk = part.own_keys();              // nkeys keys (may alias sel_smem)
    float* dzs = (float*)(sel_smem + part.nkeys); // npx
    float* rzs = dzs + npx;                       // npx
    int16_t* ds = (int16_t*)(rzs + npx);          // npx
    int16_t* wideq = ds + npx;                    // npx queued wide pixels
    // per-warp scratch of DP labels, 8-byte aligned for the 4-label stores
    uint16_t* scr_all = (uint16_t*)(sel_smem + ((part.nkeys + 3 * npx + 1) & ~1));
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = threadIdx.x; t < part.nkeys; t += blockDim.x) drk[t] = 0xFFFFFFFFu;
    if (threadIdx.x == 0) n_wide = 0;
    __syncthreads();  // keymin touches only this block's keys until the row's barrier below

    // ---- narrow windows: one thread per pixel, the labels unrolled to the widest narrow window
    // of the warp's pixels (8, 12 or 16)
    for (int xb = x0 + (threadIdx.x & ~31); xb < x1; xb += blockDim.x) {
        const int x = xb + lane;
        const bool in = x < x1;
        const int i = y * W + x;
        const uint2 dsc = in ? desc[i] : make_uint2(0u, 0u);
        const uint32_t o = dsc.x;
        const int a = (int)(dsc.y & 0xFFFFu);
        const int w = (int)(dsc.y >> 16);
        if (in && w > kSelNarrow) {
            if (split)
                ds[x - x0] = -1;
            else
                wideq[atomicAdd(&n_wide, 1)] = (int16_t)(x - x0);
        }
        const bool narrow = in && w <= kSelNarrow;
        const int wmax = (int)__reduce_max_sync(kFull, narrow ? (unsigned)w : 0u);
        if (!narrow) continue;
        auto km = [&](int xr, uint32_t k) { part.keymin(xr, k); };
        int js;
        float delta, r;
        if (wmax <= 8)
            select_narrow<NPATHS, 8>(Lvol, vol_stride, o, a, w, x, s_thr, r_min, S_out, km, js, delta, r);
        else if (wmax <= 12)
            select_narrow<NPATHS, 12>(Lvol, vol_stride, o, a, w, x, s_thr, r_min, S_out, km, js, delta, r);
        else
            select_narrow<NPATHS, 16>(Lvol, vol_stride, o, a, w, x, s_thr, r_min, S_out, km, js, delta, r);
        ds[x - x0] = (int16_t)(a + js);
        dzs[x - x0] = __fadd_rn((float)(a + js), delta);
        rzs[x - x0] = r;
    }
    __syncthreads();

    // ---- wide windows: one warp per pixel, the path costs of the next two pixels loaded during
    // this one (NCH chunks of 128 labels cover the widest window)
    uint16_t* scr = scr_all + wid * DP;
    const int nwide = n_wide;
    auto load_wide = [&](int q, uint32_t (&v)[NCH * NPATHS], uint2& dsc) {
        if (q >= nwide) return;
        dsc = desc[y * W + x0 + wideq[q]];
        load_wide_costs<NPATHS, NCH>(Lvol, vol_stride, dsc, v);
    };
    uint32_t vcur[NCH * NPATHS], vnext[NCH * NPATHS], vnext2[NCH * NPATHS];
    uint2 dcur = make_uint2(0u, 0u), dnext = make_uint2(0u, 0u), dnext2 = make_uint2(0u, 0u);
    load_wide(wid, vcur, dcur);
    load_wide(wid + nw, vnext, dnext);
    for (int q = wid; q < nwide; q += nw) {
        load_wide(q + 2 * nw, vnext2, dnext2);
        const int x = x0 + wideq[q];
        int dsr;
        float dzr, rr;
        select_wide<NPATHS, NCH>(vcur, dcur, x, s_thr, r_min, scr, S_out,
                                 [&](int xr, uint32_t k) { part.keymin(xr, k); }, dsr, dzr, rr);
        if (lane == 0) {
            ds[x - x0] = (int16_t)dsr;
            dzs[x - x0] = dzr;
            rzs[x - x0] = rr;
        }
#pragma unroll
        for (int t = 0; t < NCH * NPATHS; ++t) {
            vcur[t] = vnext[t];
            vnext[t] = vnext2[t];
        }
        dcur = dnext;
        dnext = dnext2;
    }
    // the kernel that selected the wide pixels apart (k_select_wide) may still be running when
    // this one was launched as its programmatic dependent: wait for its grid and its writes
    // (winners, outputs, keys) before reading them; without such a launch this returns at once
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (split) {
        __syncthreads();  // this block's key atomics are done
        const int kb = part.key_base();
        for (int t = threadIdx.x; t < part.nkeys; t += blockDim.x) {
            const int xr = kb + t;
            if (xr >= 0 && xr < W) drk[t] = min(drk[t], gkeys_row[xr]);
        }
    }
    part.sync();  // every key of the row is final
    for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
        const int i = y * W + x;
        int d = ds[x - x0];
        const bool wide_px = split && d < 0;
        if (wide_px) d = wds[i];
        const int xr = x - d;
        bool ok = false;
        if (xr >= 0) {
            const uint32_t kk = part.key(xr);
            ok = kk != 0xFFFFFFFFu && abs(d - (int)(kk & 0x1FFu)) <= lr_tol;
        }
        if (wide_px) {
            if (!ok) {
                Dz[i] = -1.0f;
                rz[i] = -1.0f;
            }
        } else {
            Dz[i] = ok ? dzs[x - x0] : -1.0f;
            rz[i] = ok ? rzs[x - x0] : -1.0f;
        }
        if (split) gkeys_row[x] = 0xFFFFFFFFu;
        if (dstar_out) {
            dstar_out[i] = (int16_t)d;
            const uint32_t kx = part.key(x);
            dright_out[i] = kx == 0xFFFFFFFFu ? (int16_t)-1 : (int16_t)(kx & 0x1FFu);
            valid_out[i] = ok ? 1 : 0;
        }
    }
    part.sync();  // no block leaves while another may still read its keys
}

// One whole row per block: the keys in this block's shared memory.
struct RowPart {
    uint32_t* keys;
    int nkeys;
    __device__ uint32_t* own_keys() const { return keys; }
    __device__ void keymin(int xr, uint32_t k) const { atomicMin(keys + xr, k); }
    __device__ uint32_t key(int xr) const { return keys[xr]; }
    __device__ void sync() const { __syncthreads(); }
    __device__ int key_base() const { return 0; }
};

template <int NPATHS>
__device__ __forceinline__ void select_row(
    const uint8_t* __restrict__ Lvol, uint64_t vol_stride, const uint2* __restrict__ desc, int W,
    int y, int DP, float s_thr, float r_min, int lr_tol, float* __restrict__ Dz,
    float* __restrict__ rz, uint16_t* __restrict__ S_out, int16_t* __restrict__ dstar_out,
    int16_t* __restrict__ dright_out, uint8_t* __restrict__ valid_out, uint32_t* sel_smem,
    int& n_wide, int n = 0, const uint32_t* __restrict__ wq = nullptr,
    uint32_t* __restrict__ gkeys_row = nullptr, const int16_t* __restrict__ wds = nullptr) {
    RowPart part{sel_smem, W};
    select_part<NPATHS, 2>(Lvol, vol_stride, desc, W, y, 0, W, DP, s_thr, r_min, lr_tol, Dz, rz,
                           S_out, dstar_out, dright_out, valid_out, sel_smem, n_wide, part, n, wq,
                           gkeys_row, wds);
}

}  // namespace dev
}  // namespace tsgm
