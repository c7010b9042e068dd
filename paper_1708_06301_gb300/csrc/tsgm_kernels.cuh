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

// 4-byte asynchronous copy global -> shared (completion tracked by commit groups, not by the
// issuing thread's registers, so that many copies can be in flight per warp).
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared memory of sgm_line, in 32-bit words, for labels up to DP = 32 * LPL: two label buffers
// (2 x DP uint16) and a ring of kRingW cost slots of DP bytes.
constexpr int kRingW = 8, kPrefW = 6;  // ring slots and prefetch distance of sgm_line
// narrow walker: predecessor rows of 32 labels with kInf pads on both sides (see sgm_line_narrow)
constexpr int kRowPad = 3, kRowLen = 32 + 2 * kRowPad;
template <int LPL>
__host__ __device__ constexpr int sgm_warp_words() { return (32 * LPL) * (1 + kRingW / 4); }

// One path line walked by a whole warp: direction `code`, line index `l` of that direction; Lv is
// the direction's volume, wsm this warp's shared memory (sgm_warp_words).
//
// Three representations of the predecessor's path costs: narrow (w <= 32, lane j <-> label lo + j,
// neighbours by three shuffles at the window offset), dense (w == D, LPL labels per lane packed as
// 16-bit pairs, min.u16x2 arithmetic, neighbours by two shuffles) and shared memory (absolute
// label index), which also carries every change between the first two. The costs of the pixels
// 1 .. kPrefW ahead are in flight into a ring of shared-memory slots (cp.async), so a step never
// waits for memory; descriptors come 32 pixels at a time, two blocks ahead.
template <int LPL>
__device__ __forceinline__ void sgm_line(const uint8_t* __restrict__ C,
                                         const uint2* __restrict__ desc, int W, int Hh, int D,
                                         int P1, int P2, int code, int l, uint8_t* __restrict__ Lv,
                                         uint32_t* const wsm) {
    static_assert(LPL == 2 || LPL == 4 || LPL == 8, "labels per lane");
    constexpr int NP = LPL / 2;        // packed pairs per lane in the dense form
    constexpr int DP = 32 * LPL;       // labels covered by the dense form (>= D)
    constexpr int kBufPairs = DP / 2;  // two buffers of DP uint16 labels, as pairs
    constexpr int R = kRingW, PF = kPrefW;
    uint32_t* const buf0 = wsm;
    uint8_t* const ring = reinterpret_cast<uint8_t*>(wsm + DP);
    const int lane = threadIdx.x & 31;
    int i0, step, len;
    line_geometry(code, l, W, Hh, i0, step, len);

    // dense-label masks: lanes' pairs beyond D hold +inf and contribute nothing
    uint32_t keep[NP];
#pragma unroll
    for (int k2 = 0; k2 < NP; ++k2) {
        const int e = LPL * lane + 2 * k2;
        keep[k2] = (e < D ? 0xFFFFu : 0u) | (e + 1 < D ? 0xFFFF0000u : 0u);
    }
    const bool dense_lane = LPL * lane < D;
    const uint32_t P1P1 = ((uint32_t)P1 << 16) | (uint32_t)P1;
    const uint32_t P2P2 = ((uint32_t)P2 << 16) | (uint32_t)P2;

    int qlo = 0, qw = 0, m = 0;
    int loc = 0;  // where the predecessor lives: 0 narrow registers, 1 dense registers, 2 smem
    int qb = 0;   // smem buffer holding the predecessor when loc == 2
    int Nreg = kInf;
    uint32_t Dreg[NP];
#pragma unroll
    for (int k2 = 0; k2 < NP; ++k2) Dreg[k2] = kInf2;

    // descriptors in blocks of 32 pixels (one per lane): dc0 block blk, dc1 the next, dc2 the one
    // after (in flight)
    auto ldesc = [&](int kk) -> uint2 {
        return kk < len ? __ldg(desc + (i0 + kk * step)) : make_uint2(0u, 0u);
    };
    uint2 dc0 = ldesc(lane), dc1 = ldesc(32 + lane), dc2 = ldesc(64 + lane);
    int blk = 0;
    auto desc_at = [&](int kk, uint32_t& o_, uint32_t& lw_) {  // kk in block blk or blk + 1
        const bool first = (kk >> 5) == blk;
        o_ = __shfl_sync(kFull, first ? dc0.x : dc1.x, kk & 31);
        lw_ = __shfl_sync(kFull, first ? dc0.y : dc1.y, kk & 31);
    };
    // start the copy of pixel kk's costs (its whole window, whole 4-byte words) into its slot
    auto issue = [&](int kk) {
        uint32_t o_, lw_;
        desc_at(kk, o_, lw_);
        const int w_ = kk < len ? (int)(lw_ >> 16) : 0;
        uint8_t* slot = ring + (kk & (R - 1)) * DP;
#pragma unroll
        for (int t = 0; t < (DP + 127) / 128; ++t) {
            const int j = lane + 32 * t;
            if (4 * j < w_) cp_async4(slot + 4 * j, C + o_ + 4 * j);
        }
        cp_async_commit();
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
        if (!dense_lane) return;
        if constexpr (LPL % 4 == 0) {
#pragma unroll
            for (int k4 = 0; k4 < NP / 2; ++k4)
                if (LPL * lane + 4 * k4 < D)
                    *reinterpret_cast<uint32_t*>(Lv + o + LPL * lane + 4 * k4) =
                        __byte_perm(Dreg[2 * k4], Dreg[2 * k4 + 1], 0x6420);
        } else {
            *reinterpret_cast<uint16_t*>(Lv + o + LPL * lane) =
                (uint16_t)__byte_perm(Dreg[0], 0u, 0x0020);
        }
    };

    // Software pipeline: at the top of step k the descriptor of pixel k and (narrow pixels) this
    // lane's cost byte are in registers, prepared during step k - 1. A step first starts the
    // neighbour shuffles of the narrow recurrence (the head of the dependent chain), then, while
    // they are in flight, starts the copy of pixel k + PF, waits for pixel k + 1's copy and reads
    // its descriptor and cost byte, and only then finishes pixel k. Runs of narrow pixels take a
    // tight loop of their own.
    for (int u = 0; u < PF; ++u) issue(u);
    cp_async_wait<PF - 1>();
    __syncwarp();
    uint32_t o, lw;
    desc_at(0, o, lw);
    int c = (lane < (int)(lw >> 16)) ? (int)ring[lane] : 0;
    // prepare pixel k + 1 (its copy landed, descriptor and cost byte in registers)
    auto prepare_next = [&](int k, uint32_t& o_n, uint32_t& lw_n, int& c_n) {
        issue(k + PF);  // into the slot of pixel k + PF - R, read two steps ago
        cp_async_wait<PF - 1>();  // pixel k + 1's copy has landed ...
        __syncwarp();             // ... for every lane's part of it
        if (((k + 1) & 31) == 0) {
            dc0 = dc1;
            dc1 = dc2;
            ++blk;
            dc2 = ldesc(((blk + 2) << 5) + lane);
        }
        desc_at(k + 1, o_n, lw_n);
        c_n = (lane < (int)(lw_n >> 16)) ? (int)ring[((k + 1) & (R - 1)) * DP + lane] : 0;
    };
    int k = 0;
    while (k < len) {
        // ---------------------------------------------------------------- narrow runs
        // consecutive narrow pixels after a narrow one: a tight loop without dispatch, unrolled so
        // that consecutive steps use different registers (a store or copy still reading its
        // operands does not hold up the next step)
        if (k > 0 && loc == 0) {
#pragma unroll 4
            while (k < len && (int)(lw >> 16) <= 32) {
                const int lo = (int)(lw & 0xFFFFu);
                const int w = (int)(lw >> 16);
                const int s_ = lane + (lo - qlo);
                int vc = __shfl_sync(kFull, Nreg, s_ & 31);
                int vl = __shfl_sync(kFull, Nreg, (s_ - 1) & 31);
                int vr = __shfl_sync(kFull, Nreg, (s_ + 1) & 31);
                uint32_t o_n, lw_n;
                int c_n;
                prepare_next(k, o_n, lw_n, c_n);
                vc = ((unsigned)s_ < (unsigned)qw) ? vc : kInf;
                vl = ((unsigned)(s_ - 1) < (unsigned)qw) ? vl : kInf;
                vr = ((unsigned)(s_ + 1) < (unsigned)qw) ? vr : kInf;
                int L = c + min(min(min(vl, vr) + P1, vc), m + P2) - m;
                L = lane < w ? L : kInf;
                if (lane < w) Lv[o + lane] = (uint8_t)L;
                m = (int)__reduce_min_sync(kFull, (unsigned)L);
                Nreg = L;
                qlo = lo;
                qw = w;
                o = o_n;
                lw = lw_n;
                c = c_n;
                ++k;
            }
            if (k >= len) break;
        }
        // ---------------------------------------------------------------- full-range runs
        // consecutive full-range pixels after a full-range one: the same, for the dense form
        if (k > 0 && loc == 1) {
#pragma unroll 2
            while (k < len && (int)(lw >> 16) == D) {
                uint32_t o_n, lw_n;
                int c_n;
                prepare_next(k, o_n, lw_n, c_n);
                const uint8_t* cs = ring + (k & (R - 1)) * DP;
                uint32_t c2[NP];
                if constexpr (LPL == 2) {
                    c2[0] = __byte_perm(*reinterpret_cast<const uint16_t*>(cs + 2 * lane), 0u,
                                        0x4140);
                } else {
#pragma unroll
                    for (int r = 0; r < LPL / 4; ++r) {
                        const uint32_t wd =
                            *reinterpret_cast<const uint32_t*>(cs + LPL * lane + 4 * r);
                        c2[2 * r] = __byte_perm(wd, 0u, 0x4140);
                        c2[2 * r + 1] = __byte_perm(wd, 0u, 0x4342);
                    }
                }
                uint32_t Lq[NP];
#pragma unroll
                for (int k2 = 0; k2 < NP; ++k2) Lq[k2] = Dreg[k2];
                const int lmin = dense_step(Lq, c2);
                emit_dense(o);
                m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
                o = o_n;
                lw = lw_n;
                c = c_n;
                ++k;
            }
            qlo = 0;
            qw = D;
            if (k >= len) break;
        }
        // ---------------------------------------------------------------- any other step
        const int lo = (int)(lw & 0xFFFFu);
        const int w = (int)(lw >> 16);
        const int s_ = lane + (lo - qlo);
        int vc = __shfl_sync(kFull, Nreg, s_ & 31);
        int vl = __shfl_sync(kFull, Nreg, (s_ - 1) & 31);
        int vr = __shfl_sync(kFull, Nreg, (s_ + 1) & 31);
        uint32_t o_n, lw_n;
        int c_n;
        prepare_next(k, o_n, lw_n, c_n);
        const uint8_t* cs = ring + (k & (R - 1)) * DP;
        if (w <= 32) {
            // ------------------------------------------------------------ narrow step
            int L;
            if (k == 0) {
                L = c;
            } else if (loc == 0) {
                vc = ((unsigned)s_ < (unsigned)qw) ? vc : kInf;
                vl = ((unsigned)(s_ - 1) < (unsigned)qw) ? vl : kInf;
                vr = ((unsigned)(s_ + 1) < (unsigned)qw) ? vr : kInf;
                L = c + min(min(min(vl, vr) + P1, vc), m + P2) - m;
            } else {
                spill();
                const uint16_t* src16 = reinterpret_cast<const uint16_t*>(buf0 + qb * kBufPairs);
                const int d = lo + lane;
                const int qhi = qlo + qw - 1;
                const int uc = (d >= qlo && d <= qhi) ? (int)src16[d] : kInf;
                const int ul = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src16[d - 1] : kInf;
                const int ur = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src16[d + 1] : kInf;
                L = c + min(min(min(ul, ur) + P1, uc), m + P2) - m;
            }
            L = lane < w ? L : kInf;
            if (lane < w) Lv[o + lane] = (uint8_t)L;
            m = (int)__reduce_min_sync(kFull, (unsigned)L);
            Nreg = L;
            loc = 0;
        } else if (w == D) {
            // ------------------------------------------------------------ full-range step
            uint32_t c2[NP];
            if constexpr (LPL == 2) {
                c2[0] = __byte_perm(*reinterpret_cast<const uint16_t*>(cs + 2 * lane), 0u, 0x4140);
            } else {
#pragma unroll
                for (int r = 0; r < LPL / 4; ++r) {
                    const uint32_t wd = *reinterpret_cast<const uint32_t*>(cs + LPL * lane + 4 * r);
                    c2[2 * r] = __byte_perm(wd, 0u, 0x4140);
                    c2[2 * r + 1] = __byte_perm(wd, 0u, 0x4342);
                }
            }
            int lmin;
            if (k == 0) {
                uint32_t pmin = kInf2;
#pragma unroll
                for (int k2 = 0; k2 < NP; ++k2) {
                    Dreg[k2] = (c2[k2] & keep[k2]) | (kInf2 & ~keep[k2]);
                    pmin = vmin2(pmin, Dreg[k2]);
                }
                lmin = (int)min(pmin & 0xFFFFu, pmin >> 16);
            } else if (loc == 1) {
                uint32_t Lq[NP];
#pragma unroll
                for (int k2 = 0; k2 < NP; ++k2) Lq[k2] = Dreg[k2];
                lmin = dense_step(Lq, c2);
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
            emit_dense(o);
            m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
            loc = 1;
        } else {
            // ------------------------------------------------------------ other widths (smem)
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
                const int c = act ? (int)cs[j] : 0;
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
                if (act) {
                    dst16[d] = (uint16_t)L;
                    Lv[o + j] = (uint8_t)L;
                }
                lmin = min(lmin, L);
            }
            m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
            qb ^= 1;
            loc = 2;
            __syncwarp();
        }
        qlo = lo;
        qw = w;
        o = o_n;
        lw = lw_n;
        c = c_n;
        ++k;
    }
    cp_async_wait<0>();  // the copies past the line end (empty groups) are retired
    __syncwarp();
}

// ---------------------------------------------------------------------------------------------
// One path line of narrow windows walked by a whole warp (lane j <-> label lo + j, as the narrow
// representation of sgm_line), with the prefetch done 32 pixels at a time: at the start of each
// block of 32 pixels every lane fetches the descriptor of one pixel two blocks ahead and copies
// the costs of one pixel of the next block into its 32-byte slot (cp.async), so that a step is
// the recurrence alone: two shuffles for its descriptor, one shared load for its cost, three
// shuffles for the predecessor, the min chain, one store and one reduction. Windows wider than 32
// take a slow step (costs read straight from global memory, predecessor through the label
// buffers). For lines with few such pixels.
// ---------------------------------------------------------------------------------------------
template <int LPL, bool kPure>
__device__ __forceinline__ void sgm_line_narrow(const uint8_t* __restrict__ C,
                                                const uint2* __restrict__ desc, int W, int Hh,
                                                int D, int P1, int P2, int code, int l,
                                                uint8_t* __restrict__ Lv, uint32_t* const wsm) {
    constexpr int DP = 32 * LPL;
    uint16_t* const buf16 = reinterpret_cast<uint16_t*>(wsm);       // 2 x DP labels
    uint8_t* const cblk = reinterpret_cast<uint8_t*>(wsm + DP);     // 2 blocks x 32 x 32 bytes
    // two rows (ping-pong by step parity) holding the path costs of a narrow pixel, label
    // qlo + j at position kRowPad + j, kInf in the pads and past its window
    int* const rows = reinterpret_cast<int*>(wsm + DP + 2 * 32 * 32 / 4);
    const int lane = threadIdx.x & 31;
    for (int t = lane; t < 2 * kRowLen; t += 32) rows[t] = kInf;
    int i0, step, len;
    line_geometry(code, l, W, Hh, i0, step, len);
    (void)D;

    auto ldesc = [&](int kk) -> uint2 {
        return kk < len ? __ldg(desc + (i0 + kk * step)) : make_uint2(0u, 0u);
    };
    // this lane copies the costs of its pixel of block b (narrow windows only) into its slot
    auto copy_block = [&](int b, uint2 d) {
        const int w_ = (int)(d.y >> 16);
        if (w_ <= 32) {
            uint8_t* dst = cblk + (b & 1) * 1024 + lane * 32;
            const uint8_t* src = C + d.x;
            for (int i = 0; 4 * i < w_; ++i) cp_async4(dst + 4 * i, src + 4 * i);
        }
        cp_async_commit();
    };

    const int nblk = (len + 31) >> 5;
    uint2 dA = ldesc(lane), dB = ldesc(32 + lane);
    copy_block(0, dA);
    int qlo = 0, qw = 0, m = 0, Nreg = kInf, qb = 0;
    bool in_regs = true;  // predecessor in Nreg (else in label buffer qb, absolute index)

    for (int b = 0; b < nblk; ++b) {
        __syncwarp();  // reads of the buffer about to be refilled are done
        copy_block(b + 1, dB);
        const uint2 dC = ldesc(((b + 2) << 5) + lane);
        cp_async_wait<1>();  // this block's copies have landed ...
        __syncwarp();        // ... for every lane
        const uint8_t* cb = cblk + (b & 1) * 1024;
        const int kend = min(32, len - (b << 5));
        // pixels of this block whose window is narrow (past the line's end: w = 0, narrow)
        const uint32_t nmask = kPure ? ~0u : __ballot_sync(kFull, (int)(dA.y >> 16) <= 32);
        // a narrow step after a narrow one: straight-line code (the first pixel is a select, not
        // a branch), so that the steps of a group of four interleave
        // the predecessor's labels d - 1 .. d + 1 come from its padded row: the offset clamped to
        // [-2, 33] reads only pads when out of range, so no range checks are needed
        auto fast_step = [&](int u) {
            const int k = (b << 5) + u;
            const uint32_t o = __shfl_sync(kFull, dA.x, u);
            const uint32_t lw = __shfl_sync(kFull, dA.y, u);
            const int lo = (int)(lw & 0xFFFFu);
            const int w = (int)(lw >> 16);
            const int c = lane < w ? (int)cb[u * 32 + lane] : 0;
            const int* prow = rows + ((k + 1) & 1) * kRowLen;
            const int sc = min(max(lane + (lo - qlo), -2), 33) + kRowPad;
            const int vl = prow[sc - 1], vc = prow[sc], vr = prow[sc + 1];
            int L = c + min(min(min(vl, vr) + P1, vc), m + P2) - m;
            L = k == 0 ? c : L;
            L = lane < w ? L : kInf;
            rows[(k & 1) * kRowLen + kRowPad + lane] = L;
            if (lane < w) Lv[o + lane] = (uint8_t)L;
            m = (int)__reduce_min_sync(kFull, (unsigned)L);
            __syncwarp();  // this row is complete for the next step
            Nreg = L;
            qlo = lo;
            qw = w;
        };
        // any step (wide windows, or a narrow one after a wide one)
        auto slow_step = [&](int u) {
            const int k = (b << 5) + u;
            const uint32_t o = __shfl_sync(kFull, dA.x, u);
            const uint32_t lw = __shfl_sync(kFull, dA.y, u);
            const int lo = (int)(lw & 0xFFFFu);
            const int w = (int)(lw >> 16);
            if (w <= 32) {
                const int c = lane < w ? (int)cb[u * 32 + lane] : 0;
                int L;
                if (k == 0) {
                    L = c;
                } else if (in_regs) {
                    const int s_ = lane + (lo - qlo);
                    int vc = __shfl_sync(kFull, Nreg, s_ & 31);
                    int vl = __shfl_sync(kFull, Nreg, (s_ - 1) & 31);
                    int vr = __shfl_sync(kFull, Nreg, (s_ + 1) & 31);
                    vc = ((unsigned)s_ < (unsigned)qw) ? vc : kInf;
                    vl = ((unsigned)(s_ - 1) < (unsigned)qw) ? vl : kInf;
                    vr = ((unsigned)(s_ + 1) < (unsigned)qw) ? vr : kInf;
                    L = c + min(min(min(vl, vr) + P1, vc), m + P2) - m;
                } else {
                    const uint16_t* src16 = buf16 + qb * DP;
                    const int d = lo + lane, qhi = qlo + qw - 1;
                    const int uc = (d >= qlo && d <= qhi) ? (int)src16[d] : kInf;
                    const int ul = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src16[d - 1] : kInf;
                    const int ur = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src16[d + 1] : kInf;
                    L = c + min(min(min(ul, ur) + P1, uc), m + P2) - m;
                }
                L = lane < w ? L : kInf;
                rows[(k & 1) * kRowLen + kRowPad + lane] = L;
                if (lane < w) Lv[o + lane] = (uint8_t)L;
                m = (int)__reduce_min_sync(kFull, (unsigned)L);
                __syncwarp();  // this row is complete for the next step
                Nreg = L;
                in_regs = true;
            } else {
                // ---------------------------------------------------- slow step: wide window
                if (k > 0 && in_regs) {
                    __syncwarp();  // earlier reads of buffer qb are done
                    if (lane < qw) buf16[qb * DP + qlo + lane] = (uint16_t)Nreg;
                    __syncwarp();
                }
                const uint16_t* src16 = buf16 + qb * DP;
                uint16_t* dst16 = buf16 + (qb ^ 1) * DP;
                const int qhi = qlo + qw - 1;
                int lmin = kInf;
                // every cost load first (one memory round trip), then the labels
                int cv[LPL];
#pragma unroll
                for (int r = 0; r < LPL; ++r)
                    cv[r] = 32 * r + lane < w ? (int)__ldg(C + o + 32 * r + lane) : 0;
#pragma unroll
                for (int r = 0; r < LPL; ++r) {
                    const int j0 = 32 * r;
                    if (j0 >= w) break;
                    const int j = j0 + lane;
                    const bool act = j < w;
                    const int d = lo + j;
                    const int c = cv[r];
                    int L;
                    if (k == 0) {
                        L = c;
                    } else {
                        const int uc = (d >= qlo && d <= qhi) ? (int)src16[d] : kInf;
                        const int ul = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src16[d - 1] : kInf;
                        const int ur = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src16[d + 1] : kInf;
                        L = c + min(min(min(ul, ur) + P1, uc), m + P2) - m;
                    }
                    L = act ? L : kInf;
                    if (act) {
                        dst16[d] = (uint16_t)L;
                        Lv[o + j] = (uint8_t)L;
                    }
                    lmin = min(lmin, L);
                }
                m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
                qb ^= 1;
                in_regs = false;
                __syncwarp();
            }
            qlo = lo;
            qw = w;
        };
        for (int u0 = 0; u0 < kend; u0 += 4) {
            if ((kPure || in_regs) && u0 + 4 <= kend && ((nmask >> u0) & 15u) == 15u) {
                fast_step(u0);
                fast_step(u0 + 1);
                fast_step(u0 + 2);
                fast_step(u0 + 3);
            } else {
                for (int u = u0; u < u0 + 4 && u < kend; ++u) {
                    if (kPure)
                        fast_step(u);
                    else
                        slow_step(u);
                }
            }
        }
        dA = dB;
        dB = dC;
    }
    cp_async_wait<0>();
    __syncwarp();
}

// ---------------------------------------------------------------------------------------------
// One path line of narrow and full-range windows (the image-border lines of a reduced frame),
// walked by a whole warp: the narrow walker's block copies, padded rows and straight-line groups
// for narrow pixels, and the dense form of sgm_line (LPL labels per lane packed as uint16 pairs)
// for full-range pixels, whose costs are copied by each lane (its own words) two groups of four
// pixels ahead into a ring of kRingM slots, with straight-line groups of four full-range steps.
// Changes of representation and other widths (slow step, costs read from global memory) go
// through the two label buffers.
// ---------------------------------------------------------------------------------------------
constexpr int kRingM = 16;  // full-range cost slots of the mixed walker (3 groups in flight)
template <int LPL>
__host__ __device__ constexpr int sgm_mixed_words() {
    return 32 * LPL + 2 * 32 * 32 / 4 + 2 * kRowLen + kRingM * (32 * LPL > 128 ? 32 * LPL : 128) / 4;
}

template <int LPL>
__device__ __forceinline__ void sgm_line_mixed(const uint8_t* __restrict__ C,
                                               const uint2* __restrict__ desc, int W, int Hh,
                                               int D, int P1, int P2, int code, int l,
                                               uint8_t* __restrict__ Lv, uint32_t* const wsm) {
    constexpr int NP = LPL / 2;
    constexpr int DP = 32 * LPL;
    constexpr int kBufPairs = DP / 2;
    constexpr int SL = DP > 128 ? DP : 128;  // dense slot bytes
    uint32_t* const buf0 = wsm;                                          // 2 x DP labels
    uint16_t* const buf16 = reinterpret_cast<uint16_t*>(wsm);
    uint8_t* const cblk = reinterpret_cast<uint8_t*>(wsm + DP);          // 2 x 32 x 32 bytes
    int* const rows = reinterpret_cast<int*>(wsm + DP + 2 * 32 * 32 / 4);  // 2 padded rows
    uint8_t* const dring = reinterpret_cast<uint8_t*>(wsm + DP + 2 * 32 * 32 / 4 + 2 * kRowLen);
    const int lane = threadIdx.x & 31;
    int i0, step, len;
    line_geometry(code, l, W, Hh, i0, step, len);
    for (int t = lane; t < 2 * kRowLen; t += 32) rows[t] = kInf;

    uint32_t keep[NP];
#pragma unroll
    for (int k2 = 0; k2 < NP; ++k2) {
        const int e = LPL * lane + 2 * k2;
        keep[k2] = (e < D ? 0xFFFFu : 0u) | (e + 1 < D ? 0xFFFF0000u : 0u);
    }
    const bool dense_lane = LPL * lane < D;
    const uint32_t P1P1 = ((uint32_t)P1 << 16) | (uint32_t)P1;
    const uint32_t P2P2 = ((uint32_t)P2 << 16) | (uint32_t)P2;

    auto ldesc = [&](int kk) -> uint2 {
        return kk < len ? __ldg(desc + (i0 + kk * step)) : make_uint2(0u, 0u);
    };
    auto copy_block = [&](int b, uint2 d) {  // this lane's pixel of block b, narrow windows only
        const int w_ = (int)(d.y >> 16);
        if (w_ <= 32) {
            uint8_t* dst = cblk + (b & 1) * 1024 + lane * 32;
            const uint8_t* src = C + d.x;
            for (int t = 0; 4 * t < w_; ++t) cp_async4(dst + 4 * t, src + 4 * t);
        }
    };
    auto copy_dense = [&](int kk, uint32_t o_) {  // this lane's cost words of a full-range pixel
        uint8_t* slot = dring + (kk & (kRingM - 1)) * SL;
        if constexpr (LPL == 2) {
            if (4 * (lane >> 1) < D) cp_async4(slot + 4 * lane, C + o_ + 4 * (lane >> 1));
        } else {
#pragma unroll
            for (int r = 0; r < LPL / 4; ++r)
                if (LPL * lane + 4 * r < D) cp_async4(slot + LPL * lane + 4 * r, C + o_ + LPL * lane + 4 * r);
        }
    };
    auto dense_costs = [&](int kk, uint32_t (&c2)[NP]) {
        const uint8_t* cs = dring + (kk & (kRingM - 1)) * SL;
        if constexpr (LPL == 2) {
            const uint32_t wd = *reinterpret_cast<const uint32_t*>(cs + 4 * lane);
            c2[0] = __byte_perm(wd, 0u, (lane & 1) ? 0x4342 : 0x4140);
        } else {
#pragma unroll
            for (int r = 0; r < LPL / 4; ++r) {
                const uint32_t wd = *reinterpret_cast<const uint32_t*>(cs + LPL * lane + 4 * r);
                c2[2 * r] = __byte_perm(wd, 0u, 0x4140);
                c2[2 * r + 1] = __byte_perm(wd, 0u, 0x4342);
            }
        }
    };

    int qlo = 0, qw = 0, m = 0, Nreg = kInf, qb = 0;
    int loc = 0;  // predecessor: 0 narrow (Nreg and its padded row), 1 dense (Dreg), 2 label buffer qb
    uint32_t Dreg[NP];
#pragma unroll
    for (int k2 = 0; k2 < NP; ++k2) Dreg[k2] = kInf2;

    auto spill = [&]() {  // the predecessor into label buffer 0 if it is in registers
        if (loc == 2) return;
        __syncwarp();
        if (loc == 0) {
            if (lane < qw) buf16[qlo + lane] = (uint16_t)Nreg;
        } else {
#pragma unroll
            for (int k2 = 0; k2 < NP; ++k2) buf0[(LPL * lane) / 2 + k2] = Dreg[k2];
        }
        qb = 0;
        loc = 2;
        __syncwarp();
    };
    auto dense_update = [&](const uint32_t (&Lq)[NP], const uint32_t (&c2)[NP]) -> int {
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
            const uint32_t lm1 = __byte_perm(prev, Lq[k2], 0x5432);
            const uint32_t lp1 = __byte_perm(Lq[k2], next, 0x5432);
            uint32_t t = vmin2(lm1, lp1) + P1P1;
            t = vmin2(vmin2(t, Lq[k2]), mP2);
            const uint32_t Lnew = (c2[k2] + t) - mm;
            Dreg[k2] = (Lnew & keep[k2]) | (kInf2 & ~keep[k2]);
            pmin = vmin2(pmin, Dreg[k2]);
        }
        return (int)min(pmin & 0xFFFFu, pmin >> 16);
    };
    auto emit_dense = [&](uint32_t o) {
        if (!dense_lane) return;
        if constexpr (LPL % 4 == 0) {
#pragma unroll
            for (int k4 = 0; k4 < NP / 2; ++k4)
                if (LPL * lane + 4 * k4 < D)
                    *reinterpret_cast<uint32_t*>(Lv + o + LPL * lane + 4 * k4) =
                        __byte_perm(Dreg[2 * k4], Dreg[2 * k4 + 1], 0x6420);
        } else {
            *reinterpret_cast<uint16_t*>(Lv + o + LPL * lane) =
                (uint16_t)__byte_perm(Dreg[0], 0u, 0x0020);
        }
    };

    const int nblk = (len + 31) >> 5;
    uint2 dA = ldesc(lane), dB = ldesc(32 + lane);
    uint32_t dmA = __ballot_sync(kFull, (int)(dA.y >> 16) == D);
    uint32_t dmB = __ballot_sync(kFull, (int)(dB.y >> 16) == D);
    copy_block(0, dA);
    // groups 0 and 1 (pixels 0 .. 7, all in block 0)
    for (int g = 0; g < 2; ++g) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int p = 4 * g + t;
            if (p < len && ((dmA >> p) & 1u)) copy_dense(p, __shfl_sync(kFull, dA.x, p));
        }
        cp_async_commit();
    }

    for (int b = 0; b < nblk; ++b) {
        const uint8_t* cb = cblk + (b & 1) * 1024;
        const int kend = min(32, len - (b << 5));
        const uint32_t nmask = __ballot_sync(kFull, (int)(dA.y >> 16) <= 32);
        uint2 dC = make_uint2(0u, 0u);
        uint32_t dmC = 0u;
        for (int u0 = 0; u0 < kend; u0 += 4) {
            // copies: at the block's first group the next block's narrow costs (its descriptors
            // two blocks ahead too), at every group the full-range pixels two groups ahead
            __syncwarp();  // reads of the slots about to be refilled are done
            if (u0 == 0) {
                copy_block(b + 1, dB);
                dC = ldesc(((b + 2) << 5) + lane);
                dmC = __ballot_sync(kFull, (int)(dC.y >> 16) == D);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int u = u0 + 8 + t;  // pixel (b << 5) + u, in this block or the next
                const int p = (b << 5) + u;
                const bool nxt = u >= 32;
                const uint32_t dm = nxt ? dmB : dmA;
                if (p < len && ((dm >> (u & 31)) & 1u))
                    copy_dense(p, __shfl_sync(kFull, nxt ? dB.x : dA.x, u & 31));
            }
            cp_async_commit();
            cp_async_wait<2>();  // this group's full-range copies (and this block's) have landed
            __syncwarp();
            const bool full4 = u0 + 4 <= kend;
            // ---------------------------------------------------------------- group kinds
            if (full4 && loc == 0 && ((nmask >> u0) & 15u) == 15u) {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int u = u0 + t;
                    const int k = (b << 5) + u;
                    const uint32_t o = __shfl_sync(kFull, dA.x, u);
                    const uint32_t lw = __shfl_sync(kFull, dA.y, u);
                    const int lo = (int)(lw & 0xFFFFu);
                    const int w = (int)(lw >> 16);
                    const int c = lane < w ? (int)cb[u * 32 + lane] : 0;
                    const int* prow = rows + ((k + 1) & 1) * kRowLen;
                    const int sc = min(max(lane + (lo - qlo), -2), 33) + kRowPad;
                    const int vl = prow[sc - 1], vc = prow[sc], vr = prow[sc + 1];
                    int L = c + min(min(min(vl, vr) + P1, vc), m + P2) - m;
                    L = k == 0 ? c : L;
                    L = lane < w ? L : kInf;
                    rows[(k & 1) * kRowLen + kRowPad + lane] = L;
                    if (lane < w) Lv[o + lane] = (uint8_t)L;
                    m = (int)__reduce_min_sync(kFull, (unsigned)L);
                    __syncwarp();
                    Nreg = L;
                    qlo = lo;
                    qw = w;
                }
                continue;
            }
            if (full4 && loc == 1 && ((dmA >> u0) & 15u) == 15u) {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int u = u0 + t;
                    const int k = (b << 5) + u;
                    const uint32_t o = __shfl_sync(kFull, dA.x, u);
                    uint32_t c2[NP];
                    dense_costs(k, c2);
                    uint32_t Lq[NP];
#pragma unroll
                    for (int k2 = 0; k2 < NP; ++k2) Lq[k2] = Dreg[k2];
                    const int lmin = dense_update(Lq, c2);
                    emit_dense(o);
                    m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
                }
                continue;  // qlo = 0, qw = D already
            }
            // ---------------------------------------------------------------- any steps
            for (int u = u0; u < u0 + 4 && u < kend; ++u) {
                const int k = (b << 5) + u;
                const uint32_t o = __shfl_sync(kFull, dA.x, u);
                const uint32_t lw = __shfl_sync(kFull, dA.y, u);
                const int lo = (int)(lw & 0xFFFFu);
                const int w = (int)(lw >> 16);
                if (w <= 32) {
                    const int c = lane < w ? (int)cb[u * 32 + lane] : 0;
                    int L;
                    if (k == 0) {
                        L = c;
                    } else if (loc == 0) {
                        const int* prow = rows + ((k + 1) & 1) * kRowLen;
                        const int sc = min(max(lane + (lo - qlo), -2), 33) + kRowPad;
                        L = c + min(min(min(prow[sc - 1], prow[sc + 1]) + P1, prow[sc]), m + P2) - m;
                    } else {
                        spill();
                        const uint16_t* src16 = buf16 + qb * DP;
                        const int d = lo + lane, qhi = qlo + qw - 1;
                        const int uc = (d >= qlo && d <= qhi) ? (int)src16[d] : kInf;
                        const int ul = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src16[d - 1] : kInf;
                        const int ur = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src16[d + 1] : kInf;
                        L = c + min(min(min(ul, ur) + P1, uc), m + P2) - m;
                    }
                    L = lane < w ? L : kInf;
                    rows[(k & 1) * kRowLen + kRowPad + lane] = L;
                    if (lane < w) Lv[o + lane] = (uint8_t)L;
                    m = (int)__reduce_min_sync(kFull, (unsigned)L);
                    __syncwarp();
                    Nreg = L;
                    loc = 0;
                } else if (w == D) {
                    uint32_t c2[NP];
                    dense_costs(k, c2);
                    int lmin;
                    if (k == 0) {
                        uint32_t pmin = kInf2;
#pragma unroll
                        for (int k2 = 0; k2 < NP; ++k2) {
                            Dreg[k2] = (c2[k2] & keep[k2]) | (kInf2 & ~keep[k2]);
                            pmin = vmin2(pmin, Dreg[k2]);
                        }
                        lmin = (int)min(pmin & 0xFFFFu, pmin >> 16);
                    } else if (loc == 1) {
                        uint32_t Lq[NP];
#pragma unroll
                        for (int k2 = 0; k2 < NP; ++k2) Lq[k2] = Dreg[k2];
                        lmin = dense_update(Lq, c2);
                    } else {
                        spill();
                        const uint32_t* srcp = buf0 + qb * kBufPairs;
                        const int qhi = qlo + qw - 1;
                        uint32_t Lq[NP];
#pragma unroll
                        for (int k2 = 0; k2 < NP; ++k2)
                            Lq[k2] = mask_pair(srcp[(LPL * lane) / 2 + k2], LPL * lane + 2 * k2, qlo, qhi);
                        lmin = dense_update(Lq, c2);
                    }
                    emit_dense(o);
                    m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
                    loc = 1;
                } else {
                    // ---------------------------------------------------- other widths
                    if (k > 0) spill();
                    __syncwarp();
                    const uint16_t* src16 = buf16 + qb * DP;
                    uint16_t* dst16 = buf16 + (qb ^ 1) * DP;
                    const int qhi = qlo + qw - 1;
                    int lmin = kInf;
                    // every cost load first (one memory round trip), then the labels
                    int cv[LPL];
#pragma unroll
                    for (int r = 0; r < LPL; ++r)
                        cv[r] = 32 * r + lane < w ? (int)__ldg(C + o + 32 * r + lane) : 0;
#pragma unroll
                    for (int r = 0; r < LPL; ++r) {
                        const int j0 = 32 * r;
                        if (j0 >= w) break;
                        const int j = j0 + lane;
                        const bool act = j < w;
                        const int d = lo + j;
                        const int c = cv[r];
                        int L;
                        if (k == 0) {
                            L = c;
                        } else {
                            const int uc = (d >= qlo && d <= qhi) ? (int)src16[d] : kInf;
                            const int ul = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src16[d - 1] : kInf;
                            const int ur = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src16[d + 1] : kInf;
                            L = c + min(min(min(ul, ur) + P1, uc), m + P2) - m;
                        }
                        L = act ? L : kInf;
                        if (act) {
                            dst16[d] = (uint16_t)L;
                            Lv[o + j] = (uint8_t)L;
                        }
                        lmin = min(lmin, L);
                    }
                    m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
                    qb ^= 1;
                    loc = 2;
                    __syncwarp();
                }
                qlo = lo;
                qw = w;
            }
        }
        dA = dB;
        dB = dC;
        dmA = dmB;
        dmB = dmC;
    }
    cp_async_wait<0>();
    __syncwarp();
}

// ---------------------------------------------------------------------------------------------
// Pairs of lines. Directions come in opposite pairs (codes 2s and 2s + 1) that walk the same
// geometric lines from their two ends; one warp walks both lines of a pair step by step, the two
// independent recurrences interleaved (a lone recurrence leaves the warp waiting on its own
// dependent chain most of the time).
// ---------------------------------------------------------------------------------------------

// Line index, in direction codeB (the opposite of the direction of line lA of codeA), of the same
// geometric line.
__device__ __forceinline__ int partner_line(int codeA, int lA, int codeB, int W, int Hh) {
    int dx, dy;
    dir_of(codeA, dx, dy);
    if (dx == 0 || dy == 0) return lA;
    int i0, step, len;
    line_geometry(codeA, lA, W, Hh, i0, step, len);
    const int e = i0 + (len - 1) * step;  // codeB starts where line lA ends
    const int xs = e % W, ys = e / W;
    int dxB, dyB;
    dir_of(codeB, dxB, dyB);
    if (xs == (dxB > 0 ? 0 : W - 1)) return ys;
    return Hh + (dxB > 0 ? xs - 1 : xs);
}

// Smem words of one warp of the aggregation kernels: the largest of the narrow walker (label
// buffers and two cost blocks), the general walker and the paired full-range walker (two rings).
constexpr int kRingP = 8, kPrefP = 6;  // ring slots and prefetch distance of the full-range pair
template <int LPL>
__host__ __device__ constexpr int sgm_narrow_words() {
    return 32 * LPL + 2 * 32 * 32 / 4 + 2 * kRowLen;
}
// (the narrow walker's layout: DP words of label buffers, 2 x 32 x 32 cost bytes, two padded rows)
template <int LPL>
__host__ __device__ constexpr int sgm_dense_slot() { return 32 * LPL > 128 ? 32 * LPL : 128; }
template <int LPL>
__host__ __device__ constexpr int sgm_pair_words0() {
    return sgm_narrow_words<LPL>() > 2 * kRingP * sgm_dense_slot<LPL>() / 4
               ? (sgm_narrow_words<LPL>() > sgm_warp_words<LPL>() ? sgm_narrow_words<LPL>()
                                                                   : sgm_warp_words<LPL>())
               : (2 * kRingP * sgm_dense_slot<LPL>() / 4 > sgm_warp_words<LPL>()
                      ? 2 * kRingP * sgm_dense_slot<LPL>() / 4
                      : sgm_warp_words<LPL>());
}

template <int LPL>
__host__ __device__ constexpr int sgm_pair_words() {
    return sgm_pair_words0<LPL>() > sgm_mixed_words<LPL>() ? sgm_pair_words0<LPL>()
                                                           : sgm_mixed_words<LPL>();
}

// Two lines whose windows are all the full range (the dense form of sgm_line, interleaved). Each
// lane copies its own cost bytes of the pixel kPrefP ahead into its own part of a ring slot, so
// no warp synchronisation is needed per step.
template <int LPL>
__device__ __forceinline__ void sgm_pair_dense(const uint8_t* __restrict__ C,
                                               const uint2* __restrict__ desc, int W, int Hh,
                                               int D, int P1, int P2, const int (&code)[2],
                                               const int (&l)[2], uint8_t* const (&Lv)[2],
                                               uint32_t* const wsm) {
    constexpr int NP = LPL / 2;
    constexpr int SL = sgm_dense_slot<LPL>();  // ring slot bytes
    constexpr int R = kRingP, PF = kPrefP;
    const int lane = threadIdx.x & 31;
    int i0[2], step[2], len = 0;
#pragma unroll
    for (int i = 0; i < 2; ++i) line_geometry(code[i], l[i], W, Hh, i0[i], step[i], len);
    uint32_t keep[NP];
#pragma unroll
    for (int k2 = 0; k2 < NP; ++k2) {
        const int e = LPL * lane + 2 * k2;
        keep[k2] = (e < D ? 0xFFFFu : 0u) | (e + 1 < D ? 0xFFFF0000u : 0u);
    }
    const bool dense_lane = LPL * lane < D;
    const uint32_t P1P1 = ((uint32_t)P1 << 16) | (uint32_t)P1;
    const uint32_t P2P2 = ((uint32_t)P2 << 16) | (uint32_t)P2;
    auto ldesc = [&](int i, int kk) -> uint32_t {
        return kk < len ? __ldg(&desc[i0[i] + kk * step[i]].x) : 0u;
    };
    auto ring = [&](int i) { return reinterpret_cast<uint8_t*>(wsm) + i * R * SL; };
    // this lane's cost words of pixel kk of line i, from offset o_, into its part of the slot
    auto issue = [&](int i, int kk, uint32_t o_) {
        if (kk >= len) return;
        uint8_t* slot = ring(i) + (kk & (R - 1)) * SL;
        if constexpr (LPL == 2) {
            if (4 * (lane >> 1) < D) cp_async4(slot + 4 * lane, C + o_ + 4 * (lane >> 1));
        } else {
#pragma unroll
            for (int r = 0; r < LPL / 4; ++r)
                if (LPL * lane + 4 * r < D)
                    cp_async4(slot + LPL * lane + 4 * r, C + o_ + LPL * lane + 4 * r);
        }
    };
    uint32_t dc0[2], dc1[2], dc2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        dc0[i] = ldesc(i, lane);
        dc1[i] = ldesc(i, 32 + lane);
        dc2[i] = ldesc(i, 64 + lane);
    }
    int blk = 0;
    auto off_at = [&](int i, int kk) -> uint32_t {  // kk in block blk or blk + 1
        const bool first = (kk >> 5) == blk;
        return __shfl_sync(kFull, first ? dc0[i] : dc1[i], kk & 31);
    };
    for (int u = 0; u < PF; ++u) {
#pragma unroll
        for (int i = 0; i < 2; ++i) issue(i, u, off_at(i, u));
        cp_async_commit();
    }
    uint32_t Dreg[2][NP];
    int m[2] = {0, 0};
#pragma unroll 2
    for (int k = 0; k < len; ++k) {
        if (k > 0 && (k & 31) == 0) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                dc0[i] = dc1[i];
                dc1[i] = dc2[i];
                dc2[i] = ldesc(i, ((blk + 3) << 5) + lane);
            }
            ++blk;
        }
        uint32_t o[2], on[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            o[i] = off_at(i, k);
            on[i] = off_at(i, k + PF);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) issue(i, k + PF, on[i]);
        cp_async_commit();
        cp_async_wait<PF>();  // pixel k's copies (this lane's part) have landed
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const uint8_t* cs = ring(i) + (k & (R - 1)) * SL;
            uint32_t c2[NP];
            if constexpr (LPL == 2) {
                const uint32_t wd = *reinterpret_cast<const uint32_t*>(cs + 4 * lane);
                c2[0] = __byte_perm(wd, 0u, (lane & 1) ? 0x4342 : 0x4140);
            } else {
#pragma unroll
                for (int r = 0; r < LPL / 4; ++r) {
                    const uint32_t wd = *reinterpret_cast<const uint32_t*>(cs + LPL * lane + 4 * r);
                    c2[2 * r] = __byte_perm(wd, 0u, 0x4140);
                    c2[2 * r + 1] = __byte_perm(wd, 0u, 0x4342);
                }
            }
            uint32_t pmin = kInf2;
            if (k == 0) {
#pragma unroll
                for (int k2 = 0; k2 < NP; ++k2) {
                    Dreg[i][k2] = (c2[k2] & keep[k2]) | (kInf2 & ~keep[k2]);
                    pmin = vmin2(pmin, Dreg[i][k2]);
                }
            } else {
                uint32_t left_in = __shfl_up_sync(kFull, Dreg[i][NP - 1], 1);
                uint32_t right_in = __shfl_down_sync(kFull, Dreg[i][0], 1);
                if (lane == 0) left_in = kInf2;
                if (lane == 31) right_in = kInf2;
                const uint32_t mm = ((uint32_t)m[i] << 16) | (uint32_t)m[i];
                const uint32_t mP2 = mm + P2P2;
                uint32_t Lq[NP];
#pragma unroll
                for (int k2 = 0; k2 < NP; ++k2) Lq[k2] = Dreg[i][k2];
#pragma unroll
                for (int k2 = 0; k2 < NP; ++k2) {
                    const uint32_t prev = (k2 == 0) ? left_in : Lq[k2 - 1];
                    const uint32_t next = (k2 == NP - 1) ? right_in : Lq[k2 + 1];
                    const uint32_t lm1 = __byte_perm(prev, Lq[k2], 0x5432);
                    const uint32_t lp1 = __byte_perm(Lq[k2], next, 0x5432);
                    uint32_t t = vmin2(lm1, lp1) + P1P1;
                    t = vmin2(vmin2(t, Lq[k2]), mP2);
                    const uint32_t Lnew = (c2[k2] + t) - mm;
                    Dreg[i][k2] = (Lnew & keep[k2]) | (kInf2 & ~keep[k2]);
                    pmin = vmin2(pmin, Dreg[i][k2]);
                }
            }
            if (dense_lane) {
                if constexpr (LPL % 4 == 0) {
#pragma unroll
                    for (int k4 = 0; k4 < NP / 2; ++k4)
                        if (LPL * lane + 4 * k4 < D)
                            *reinterpret_cast<uint32_t*>(Lv[i] + o[i] + LPL * lane + 4 * k4) =
                                __byte_perm(Dreg[i][2 * k4], Dreg[i][2 * k4 + 1], 0x6420);
                } else {
                    *reinterpret_cast<uint16_t*>(Lv[i] + o[i] + LPL * lane) =
                        (uint16_t)__byte_perm(Dreg[i][0], 0u, 0x0020);
                }
            }
            m[i] = (int)__reduce_min_sync(kFull, min(pmin & 0xFFFFu, pmin >> 16));
        }
    }
    cp_async_wait<0>();
    __syncwarp();
}

// One pair of lines of one image: scan the windows of the (common) geometric line once. Lines
// whose windows are all the full range are walked together by one twin with the paired full-range
// walker (two interleaved recurrences per warp); other lines are walked one per twin, line A by
// twin 0 and line B by twin 1: with the branch-free narrow walker when no window is wider than 32
// labels; the general walker when more than one pixel in 8 has a window of 33 .. D - 1 labels;
// the narrow walker when at most one pixel in 8 is wide and the wide ones are scattered (runs
// shorter than 8 on average); else the mixed walker (narrow and full-range runs at full speed).
// twin < 0: this warp walks the whole pair alone. dense_twin: which twin walks an
// all-full-range pair (the launch alternates it so that the walking warps of a block fall on all
// four SM sub-partitions). The choice changes the work, never the result.
template <int LPL>
__device__ __forceinline__ void sgm_pair(const uint8_t* __restrict__ C,
                                         const uint2* __restrict__ desc, int W, int Hh, int D,
                                         int P1, int P2, int codeA, int lA, uint8_t* __restrict__ LvA,
                                         uint8_t* __restrict__ LvB, uint32_t* const wsm, int twin,
                                         int dense_twin = 0) {
    const int lane = threadIdx.x & 31;
    const int codeB = codeA + 1;
    const int lB = partner_line(codeA, lA, codeB, W, Hh);
    int i0, step, len;
    line_geometry(codeA, lA, W, Hh, i0, step, len);
    int wide = 0, full = 0, runs = 0;
    bool carry = false;  // whether the last pixel of the previous 32 was wide
    for (int k0 = 0; k0 < len; k0 += 32) {
        const int kk = k0 + lane;
        const int w_ = kk < len ? (int)(__ldg(&desc[i0 + kk * step].y) >> 16) : 0;
        const bool wd = w_ > 32;
        const bool up = __shfl_up_sync(kFull, wd, 1) != 0;  // every lane takes part
        const bool before = lane == 0 ? carry : up;
        wide += wd ? 1 : 0;
        full += w_ == D ? 1 : 0;
        runs += (wd && !before) ? 1 : 0;  // a run of wide windows starts here
        carry = __shfl_sync(kFull, wd, 31) != 0;
    }
    wide = (int)__reduce_add_sync(kFull, (unsigned)wide);
    full = (int)__reduce_add_sync(kFull, (unsigned)full);
    runs = (int)__reduce_add_sync(kFull, (unsigned)runs);
    const int other = wide - (D > 32 ? full : 0);  // windows of 33 .. D - 1 labels
    if (full == len && D > 32) {
        if (twin >= 0 && twin != dense_twin) return;
        const int code[2] = {codeA, codeB};
        const int l[2] = {lA, lB};
        uint8_t* const Lv[2] = {LvA, LvB};
        sgm_pair_dense<LPL>(C, desc, W, Hh, D, P1, P2, code, l, Lv, wsm);
        return;
    }
    for (int t = 0; t < 2; ++t) {
        if (twin >= 0 && twin != t) continue;
        const int code = t ? codeB : codeA;
        const int li = t ? lB : lA;
        uint8_t* const Lv = t ? LvB : LvA;
        if (wide == 0)
            sgm_line_narrow<LPL, true>(C, desc, W, Hh, D, P1, P2, code, li, Lv, wsm);
        else if (other * 8 > len)
            sgm_line<LPL>(C, desc, W, Hh, D, P1, P2, code, li, Lv, wsm);
        else if (runs * 8 > wide && wide * 8 <= len)  // few wide windows, scattered
            sgm_line_narrow<LPL, false>(C, desc, W, Hh, D, P1, P2, code, li, Lv, wsm);
        else
            sgm_line_mixed<LPL>(C, desc, W, Hh, D, P1, P2, code, li, Lv, wsm);
    }
}

constexpr int kSelThreads = 512;

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
    const int nl = count_side(scr, js - 1, -1, 0, w - 1, s0, s_thr, lane);
    const int nr = count_side(scr, js + 1, +1, 0, w - 1, s0, s_thr, lane);
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
    int nl = 0, nr = 0, acc = 0;
#pragma unroll
    for (int j = NL - 1; j >= 0; --j) {
        if (j < js) {
            acc += sv[j] - s0;
            nl += ((float)acc < s_thr) ? 1 : 0;
        }
    }
    acc = 0;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
        if (j > js && j < w) {
            acc += sv[j] - s0;
            nr += ((float)acc < s_thr) ? 1 : 0;
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

    // ---- wide windows: one warp per pixel, the next pixel's path costs loaded during this one
    // (NCH chunks of 128 labels cover the widest window)
    uint16_t* scr = scr_all + wid * DP;
    const int nwide = n_wide;
    auto load_wide = [&](int q, uint32_t (&v)[NCH * NPATHS], uint2& dsc) {
        if (q >= nwide) return;
        dsc = desc[y * W + x0 + wideq[q]];
        load_wide_costs<NPATHS, NCH>(Lvol, vol_stride, dsc, v);
    };
    uint32_t vcur[NCH * NPATHS], vnext[NCH * NPATHS];
    uint2 dcur = make_uint2(0u, 0u), dnext = make_uint2(0u, 0u);
    load_wide(wid, vcur, dcur);
    for (int q = wid; q < nwide; q += nw) {
        load_wide(q + nw, vnext, dnext);
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
        for (int t = 0; t < NCH * NPATHS; ++t) vcur[t] = vnext[t];
        dcur = dnext;
    }
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
