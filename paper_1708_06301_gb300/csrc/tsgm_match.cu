// Stereo matching restricted to per-pixel disparity windows (Sec. 2.3-2.4):
//   census transform -> ragged Hamming cost -> SGM path aggregation -> WTA / sub-pixel /
//   matching variance (Eq. 9) -> left-right check.
//
// Ragged volume: the cells of pixel i are off[i] .. off[i+1]-1, cell j <-> disparity lo[i] + j.
// C is uint8 (Hamming distance), S is uint16 (sum of the path costs, accumulated with packed
// 32-bit reductions: two neighbouring cells per word, no carry since S <= P (Bc + P2) < 2^16).

#include <cfloat>

#include "tsgm_internal.cuh"

namespace tsgm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------------------------
// Census transform on a shared-memory tile (32 x 8 outputs per block, border-clamped halo).
// bit b (LSB first) = [I(q) < I(p)], q over the window in row-major order without the centre.
// ---------------------------------------------------------------------------------------------
constexpr int kCtW = 32, kCtH = 8, kCmax = 15;

__global__ void __launch_bounds__(kCtW* kCtH) k_census(const uint8_t* __restrict__ imgA,
                                                        const uint8_t* __restrict__ imgB, int W,
                                                        int Hh, int cw, int ch,
                                                        uint64_t* __restrict__ outA,
                                                        uint64_t* __restrict__ outB) {
    __shared__ uint8_t tile[kCtH + kCmax][kCtW + kCmax];
    const uint8_t* img = blockIdx.z ? imgB : imgA;
    uint64_t* out = blockIdx.z ? outB : outA;
    const int rx = cw / 2, ry = ch / 2;
    const int bx = blockIdx.x * kCtW, by = blockIdx.y * kCtH;
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

// ---------------------------------------------------------------------------------------------
// Ragged cost: C(p, d) = popcount(cL(x,y) ^ cR(x-d,y)), x - d < 0 -> Bc. Groups of 8 lanes walk
// one pixel's window; the same pass zeroes S for the aggregation that follows.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cost(const uint64_t* __restrict__ cl,
                                              const uint64_t* __restrict__ cr,
                                              const int16_t* __restrict__ lo,
                                              const int16_t* __restrict__ hi,
                                              const uint32_t* __restrict__ off, int W, int n,
                                              int Bc, uint8_t* __restrict__ C,
                                              uint16_t* __restrict__ S) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    const int ngroups = (gridDim.x * blockDim.x) >> 3;
    for (int i = g; i < n; i += ngroups) {
        const int y = i / W;
        const int x = i - y * W;
        const int a = lo[i];
        const int w = hi[i] - a + 1;
        const uint32_t o = off[i];
        const uint64_t c0 = cl[i];
        const uint64_t* row = cr + (size_t)y * W;
        for (int j = sub; j < w; j += 8) {
            const int xr = x - (a + j);
            const int c = xr >= 0 ? __popcll(c0 ^ row[xr]) : Bc;
            C[o + j] = (uint8_t)c;
            S[o + j] = 0;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// SGM path aggregation. One warp walks one path line (all lines of all directions in one
// launch, horizontal ones first since they are the longest). Along direction r with
// predecessor q:
//   L(p,d) = C(p,d) + min(L(q,d), L(q,d-1)+P1, L(q,d+1)+P1, m+P2) - m,  m = min_k L(q,k)
// where L(q,.) outside q's window is +inf and the first pixel of a line has L = C.
// Narrow windows (<= 32 labels) keep L in a register, lane j <-> label lo + j, and fetch the
// predecessor's values with shuffles by the window offset. Wider windows go through a
// per-warp shared-memory buffer indexed by absolute disparity. Each lane adds its L to S with
// a packed 32-bit reduction covering two neighbouring cells.
// Direction codes: 0 (+1,0) 1 (-1,0) 2 (0,+1) 3 (0,-1) 4 (+1,+1) 5 (-1,-1) 6 (-1,+1) 7 (+1,-1)
// ---------------------------------------------------------------------------------------------
struct SgmLines {
    int start[9];   // prefix sums of line counts per slot
    int code[8];    // direction code per slot
    int nslots;
};

constexpr int kSgmWarps = 8;

__device__ __forceinline__ void dir_of(int code, int& dx, int& dy) {
    // 0 (+1,0) 1 (-1,0) 2 (0,+1) 3 (0,-1) 4 (+1,+1) 5 (-1,-1) 6 (-1,+1) 7 (+1,-1)
    dx = (code == 0 || code == 4 || code == 7) ? 1 : ((code == 1 || code == 5 || code == 6) ? -1 : 0);
    dy = (code == 2 || code == 4 || code == 6) ? 1 : ((code == 3 || code == 5 || code == 7) ? -1 : 0);
}

// Adds L (this lane's cell g = o + j, active if `act`) to S with packed pairs. Cells at even g
// carry their right neighbour (next lane, same chunk); a cell at odd g is sent alone (high
// half) only by the first lane of a chunk, otherwise the previous lane already covered it.
__device__ __forceinline__ void emit_pair(uint32_t* S32, uint32_t g, int L, bool act,
                                          bool next_act, int lane) {
    const int Ln = __shfl_down_sync(kFull, L, 1);
    if (!act) return;
    if ((g & 1u) == 0u) {
        const uint32_t v = (uint32_t)L | ((next_act && lane < 31) ? ((uint32_t)Ln << 16) : 0u);
        atomicAdd(S32 + (g >> 1), v);
    } else if (lane == 0) {
        atomicAdd(S32 + (g >> 1), (uint32_t)L << 16);
    }
}

__global__ void __launch_bounds__(kSgmWarps * 32) k_sgm(const uint8_t* __restrict__ C,
                                                        const int16_t* __restrict__ lo_,
                                                        const int16_t* __restrict__ hi_,
                                                        const uint32_t* __restrict__ off,
                                                        int W, int Hh, int D, int P1, int P2,
                                                        SgmLines lines, uint32_t* S32) {
    extern __shared__ uint16_t sgm_smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * kSgmWarps + wib;
    if (gw >= lines.start[lines.nslots]) return;
    int slot = 0;
    while (gw >= lines.start[slot + 1]) ++slot;
    const int l = gw - lines.start[slot];
    int dx, dy;
    dir_of(lines.code[slot], dx, dy);
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

    uint16_t* buf0 = sgm_smem + wib * 2 * D;
    uint16_t* buf1 = buf0 + D;

    int qlo = 0, qw = 0, m = 0;
    int Lreg = kInf;
    bool q_in_reg = true;
    int qb = 0;

    int i = y0 * W + x0;
    // software pipeline: window of the current pixel loaded one step ahead
    int lo = __ldg(lo_ + i);
    int w = __ldg(hi_ + i) - lo + 1;
    uint32_t o = __ldg(off + i);
    for (int k = 0; k < len; ++k) {
        int lo_n = 0, w_n = 0;
        uint32_t o_n = 0;
        if (k + 1 < len) {
            const int in = i + step;
            lo_n = __ldg(lo_ + in);
            w_n = __ldg(hi_ + in) - lo_n + 1;
            o_n = __ldg(off + in);
        }
        int lmin = kInf;
        if (w <= 32 && (k == 0 || q_in_reg)) {
            const bool act = lane < w;
            const int c = act ? (int)__ldg(C + o + lane) : 0;
            int L;
            if (k == 0) {
                L = c;
            } else {
                const int s = lane + (lo - qlo);
                int vc = __shfl_sync(kFull, Lreg, s & 31);
                int vl = __shfl_sync(kFull, Lreg, (s - 1) & 31);
                int vr = __shfl_sync(kFull, Lreg, (s + 1) & 31);
                vc = ((unsigned)s < (unsigned)qw) ? vc : kInf;
                vl = ((unsigned)(s - 1) < (unsigned)qw) ? vl : kInf;
                vr = ((unsigned)(s + 1) < (unsigned)qw) ? vr : kInf;
                const int t = min(min(min(vl, vr) + P1, vc), m + P2);
                L = c + t - m;
            }
            L = act ? L : kInf;
            emit_pair(S32, o + lane, L, act, lane + 1 < w, lane);
            Lreg = L;
            lmin = L;
            q_in_reg = true;
        } else {
            if (k > 0 && q_in_reg) {
                if (lane < qw) buf0[qlo + lane] = (uint16_t)Lreg;
                qb = 0;
                __syncwarp();
            }
            const uint16_t* src = qb ? buf1 : buf0;
            uint16_t* dst = qb ? buf0 : buf1;
            const int qhi = qlo + qw - 1;
            if (w <= 32) {
                // narrow pixel after a wide one: read shared memory, keep the result in a register
                const bool act = lane < w;
                const int d = lo + lane;
                const int c = act ? (int)__ldg(C + o + lane) : 0;
                const int vc = (d >= qlo && d <= qhi) ? (int)src[d] : kInf;
                const int vl = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src[d - 1] : kInf;
                const int vr = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src[d + 1] : kInf;
                const int t = min(min(min(vl, vr) + P1, vc), m + P2);
                int L = act ? c + t - m : kInf;
                emit_pair(S32, o + lane, L, act, lane + 1 < w, lane);
                Lreg = L;
                lmin = L;
                q_in_reg = true;
            } else {
                for (int j0 = 0; j0 < w; j0 += 32) {
                    const int j = j0 + lane;
                    const bool act = j < w;
                    const int d = lo + j;
                    const int c = act ? (int)__ldg(C + o + j) : 0;
                    int L;
                    if (k == 0) {
                        L = c;
                    } else {
                        const int vc = (d >= qlo && d <= qhi) ? (int)src[d] : kInf;
                        const int vl = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src[d - 1] : kInf;
                        const int vr = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src[d + 1] : kInf;
                        const int t = min(min(min(vl, vr) + P1, vc), m + P2);
                        L = c + t - m;
                    }
                    L = act ? L : kInf;
                    if (act) dst[d] = (uint16_t)L;
                    lmin = min(lmin, L);
                    emit_pair(S32, o + j, L, act, j + 1 < w, lane);
                }
                q_in_reg = false;
                qb ^= 1;
            }
        }
        m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
        qlo = lo;
        qw = w;
        __syncwarp();
        i += step;
        lo = lo_n;
        w = w_n;
        o = o_n;
    }
}

// ---------------------------------------------------------------------------------------------
// Selection + left-right check. One block per image row; one warp per pixel at a time.
//  * d* = argmin S (lowest d on ties), packed key (S << 16 | j) reduced over the warp;
//  * sub-pixel parabola when d*-1 and d*+1 are in the window;
//  * r = n_l + n_r (Eq. 9): prefix sums of S(d) - S(d*) walking away from d*, counted while
//    below s_thr (the rise is >= 0, so the counted labels form a run next to d*);
//  * right-view disparity D_R(xr) = argmin over cells with x - d = xr of (S, d), built in shared
//    memory with atomicMin on (S << 9 | d); after the row, |d* - D_R(x - d*)| <= tol passes.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int count_side(const uint16_t* __restrict__ s, int start, int dirn,
                                          int lo_idx, int hi_idx, int s0, float thr, int lane) {
    // labels start, start+dirn, ... inside [lo_idx, hi_idx]; returns how many are counted
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

__global__ void __launch_bounds__(1024) k_select(const uint16_t* __restrict__ S,
                                                 const int16_t* __restrict__ lo_,
                                                 const int16_t* __restrict__ hi_,
                                                 const uint32_t* __restrict__ off, int W,
                                                 float s_thr, float r_min, int lr_tol,
                                                 float* __restrict__ Dz, float* __restrict__ rz,
                                                 int16_t* __restrict__ dstar_out,
                                                 int16_t* __restrict__ dright_out,
                                                 uint8_t* __restrict__ valid_out) {
    extern __shared__ uint32_t sel_smem[];
    uint32_t* drk = sel_smem;                      // W keys
    float* dzs = (float*)(drk + W);                // W
    float* rzs = dzs + W;                          // W
    int16_t* ds = (int16_t*)(rzs + W);             // W
    const int y = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int x = threadIdx.x; x < W; x += blockDim.x) drk[x] = 0xFFFFFFFFu;
    __syncthreads();
    for (int x = wid; x < W; x += nw) {
        const int i = y * W + x;
        const int a = lo_[i];
        const int w = hi_[i] - a + 1;
        const uint16_t* s = S + off[i];
        unsigned best = 0xFFFFFFFFu;
        for (int j = lane; j < w; j += 32) {
            const unsigned sv = s[j];
            best = min(best, (sv << 16) | (unsigned)j);
            const int xr = x - (a + j);
            if (xr >= 0) atomicMin(drk + xr, (sv << 9) | (unsigned)(a + j));
        }
        best = __reduce_min_sync(kFull, best);
        const int js = (int)(best & 0xFFFFu);
        const int s0 = (int)(best >> 16);
        float delta = 0.0f;
        if (js >= 1 && js + 1 < w) {
            const int sm = s[js - 1], sp = s[js + 1];
            const int den = 2 * (sm - 2 * s0 + sp);
            if (den > 0) delta = __fdiv_rn((float)(sm - sp), (float)den);
        }
        const int nl = count_side(s, js - 1, -1, 0, w - 1, s0, s_thr, lane);
        const int nr = count_side(s, js + 1, +1, 0, w - 1, s0, s_thr, lane);
        float r = (float)(nl + nr);
        if (r < r_min) r = r_min;
        if (lane == 0) {
            ds[x] = (int16_t)(a + js);
            dzs[x] = __fadd_rn((float)(a + js), delta);
            rzs[x] = r;
        }
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

}  // namespace

cudaError_t launch_census(const uint8_t* imgA, const uint8_t* imgB, int W, int Hh, int cw, int ch,
                          uint64_t* outA, uint64_t* outB, cudaStream_t st) {
    dim3 blk(kCtW, kCtH);
    dim3 grd((W + kCtW - 1) / kCtW, (Hh + kCtH - 1) / kCtH, imgB ? 2 : 1);
    k_census<<<grd, blk, 0, st>>>(imgA, imgB, W, Hh, cw, ch, outA, outB);
    return cudaGetLastError();
}

cudaError_t launch_cost(const uint64_t* cl, const uint64_t* cr, const int16_t* lo,
                        const int16_t* hi, const uint32_t* off, int W, int Hh, int Bc, uint8_t* C,
                        uint16_t* S, cudaStream_t st) {
    const int n = W * Hh;
    int blocks = (n * 8 + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_cost<<<blocks, 256, 0, st>>>(cl, cr, lo, hi, off, W, n, Bc, C, S);
    return cudaGetLastError();
}

cudaError_t launch_sgm(const uint8_t* C, const int16_t* lo, const int16_t* hi, const uint32_t* off,
                       int W, int Hh, int D, int n_paths, int P1, int P2, uint16_t* S,
                       cudaStream_t st) {
    // slots ordered longest lines first: horizontal, vertical, then diagonals
    static const int order8[8] = {0, 1, 2, 3, 4, 5, 6, 7};
    SgmLines L;
    L.nslots = n_paths;
    L.start[0] = 0;
    for (int s = 0; s < n_paths; ++s) {
        const int code = order8[s];
        L.code[s] = code;
        const int cnt = code <= 1 ? Hh : (code <= 3 ? W : W + Hh - 1);
        L.start[s + 1] = L.start[s] + cnt;
    }
    const int nlines = L.start[n_paths];
    const int blocks = (nlines + kSgmWarps - 1) / kSgmWarps;
    const size_t smem = (size_t)kSgmWarps * 2 * D * sizeof(uint16_t);
    k_sgm<<<blocks, kSgmWarps * 32, smem, st>>>(C, lo, hi, off, W, Hh, D, P1, P2, L,
                                                 reinterpret_cast<uint32_t*>(S));
    return cudaGetLastError();
}

cudaError_t launch_select(const uint16_t* S, const int16_t* lo, const int16_t* hi,
                          const uint32_t* off, int W, int Hh, float s_thr, float r_min, int lr_tol,
                          float* Dz, float* rz, int16_t* dstar, int16_t* dright, uint8_t* valid,
                          cudaStream_t st) {
    const size_t smem = (size_t)W * (4 + 4 + 4 + 2);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = 1024;
    k_select<<<Hh, threads, smem, st>>>(S, lo, hi, off, W, s_thr, r_min, lr_tol, Dz, rz, dstar,
                                        dright, valid);
    return cudaGetLastError();
}

}  // namespace tsgm
