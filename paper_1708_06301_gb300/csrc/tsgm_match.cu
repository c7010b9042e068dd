// Stereo matching restricted to per-pixel disparity windows (Sec. 2.3-2.4):
//   census transform -> ragged Hamming cost -> SGM path aggregation -> WTA / sub-pixel /
//   matching variance (Eq. 9) -> left-right check.
//
// Ragged volume: pixel i owns cells off[i] .. off[i] + w_i - 1, cell j <-> disparity lo[i] + j,
// in a block of w_i rounded up to even (so every block starts 4-byte aligned in the uint16
// aggregate). C is uint8 (Hamming distance); S is uint16, the sum of the path costs, built with
// packed 32-bit reductions of two neighbouring cells (no carry: S <= P (Bc + P2) <= 2040).
// Each pixel's {off, lo | w << 16} descriptor is read once per pixel.

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
// one pixel's window; the same pass zeroes the pixel's S block for the aggregation.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cost(const uint64_t* __restrict__ cl,
                                              const uint64_t* __restrict__ cr,
                                              const uint2* __restrict__ desc, int W, int n,
                                              int Bc, uint8_t* __restrict__ C,
                                              uint16_t* __restrict__ S) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    const int ngroups = (gridDim.x * blockDim.x) >> 3;
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
        uint32_t* S32 = reinterpret_cast<uint32_t*>(S + o);
        for (int j = sub; 2 * j < w; j += 8) S32[j] = 0u;
    }
}

// ---------------------------------------------------------------------------------------------
// SGM path aggregation. One warp walks one path line; all lines of all directions are in one
// launch, horizontal ones first since they are the longest chains. Along direction r with
// predecessor q:
//   L(p,d) = C(p,d) + min(L(q,d), L(q,d-1)+P1, L(q,d+1)+P1, m+P2) - m,  m = min_k L(q,k)
// where L(q,.) outside q's window is +inf and the first pixel of a line has L = C.
// Three step kinds, by the window of the current pixel p:
//   N  (w <= 32): lane j <-> label lo + j, one register; the predecessor's values come by
//      shuffles at the window offset (from registers) or from shared memory;
//   F  (w == D > 32): dense labels, lane j <-> labels LPL*j .. LPL*j+LPL-1 packed two per
//      32-bit register and updated with min.u16x2; the predecessor comes from the dense
//      registers (full-range run) or from shared memory;
//   G  (otherwise): per-warp shared-memory buffer indexed by absolute disparity.
// Whenever the representation changes, the predecessor is written to shared memory first.
// Every lane adds its L to S with packed 32-bit reductions of aligned cell pairs.
// Direction codes: 0 (+1,0) 1 (-1,0) 2 (0,+1) 3 (0,-1) 4 (+1,+1) 5 (-1,-1) 6 (-1,+1) 7 (+1,-1)
// ---------------------------------------------------------------------------------------------
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

template <int LPL>
__global__ void __launch_bounds__(kSgmWarps * 32) k_sgm(const uint8_t* __restrict__ C,
                                                        const uint2* __restrict__ desc, int W,
                                                        int Hh, int D, int P1, int P2,
                                                        SgmLines lines, uint32_t* S32) {
    constexpr int NP = LPL / 2;       // packed pairs per lane in the dense representation
    constexpr int DP = 32 * LPL;      // labels covered by the dense representation (>= D)
    extern __shared__ uint32_t sgm_smem32[];
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
    const int i0 = y0 * W + x0;

    // two shared-memory buffers of DP labels (uint16) per warp, viewed as uint32 pairs
    uint32_t* const buf0 = sgm_smem32 + wib * DP;  // DP/2 pairs per buffer
    constexpr int kBufPairs = DP / 2;

    // dense-label masks: lanes' pairs beyond D hold +inf and contribute nothing
    uint32_t keep[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int e = LPL * lane + 2 * k;
        keep[k] = (e < D ? 0xFFFFu : 0u) | (e + 1 < D ? 0xFFFF0000u : 0u);
    }

    const uint32_t P1P1 = ((uint32_t)P1 << 16) | (uint32_t)P1;
    int qlo = 0, qw = 0, m = 0;
    int loc = 0;  // where the predecessor lives: 0 narrow registers, 1 dense registers, 2 smem
    int qb = 0;   // smem buffer holding the predecessor when loc == 2
    int Nreg = kInf;
    uint32_t Dreg[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) Dreg[k] = kInf2;

    // Descriptors of the line, 32 pixels per lane-wide load, two blocks kept (current, next),
    // and the costs of the next pixel loaded one step ahead (they do not depend on L).
    uint2 dc0 = lane < len ? __ldg(desc + (i0 + lane * step)) : make_uint2(0u, 0u);
    uint2 dc1 = 32 + lane < len ? __ldg(desc + (i0 + (32 + lane) * step)) : make_uint2(0u, 0u);
    uint32_t o_n = __shfl_sync(kFull, dc0.x, 0);
    uint32_t lw_n = __shfl_sync(kFull, dc0.y, 0);
    int cN_n = 0;
    uint32_t cD_n[NP];
    auto prefetch = [&](uint32_t o, uint32_t lw) {
        const int w = (int)(lw >> 16);
        cN_n = (lane < w) ? (int)__ldg(C + o + lane) : 0;
        const uint16_t* C16 = reinterpret_cast<const uint16_t*>(C + o);
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) {
            const int e = LPL * lane + 2 * k2;
            const uint32_t b = (w == D && w > 32 && e < D) ? (uint32_t)__ldg(C16 + (e >> 1)) : 0u;
            cD_n[k2] = __byte_perm(b, 0u, 0x4140);  // bytes (c0, c1) -> u16x2
        }
    };
    prefetch(o_n, lw_n);

    for (int k = 0; k < len; ++k) {
        const uint32_t o = o_n;
        const int lo = (int)(lw_n & 0xFFFFu);
        const int w = (int)(lw_n >> 16);
        const int cN = cN_n;
        uint32_t c2[NP];
#pragma unroll
        for (int k2 = 0; k2 < NP; ++k2) c2[k2] = cD_n[k2];
        const bool first = (k == 0);

        // next pixel: descriptor and costs
        const int kn = k + 1;
        if ((kn & 31) == 0) {
            dc0 = dc1;
            const int kk = kn + 32 + lane;
            dc1 = kk < len ? __ldg(desc + (i0 + kk * step)) : make_uint2(0u, 0u);
        }
        if (kn < len) {
            o_n = __shfl_sync(kFull, dc0.x, kn & 31);
            lw_n = __shfl_sync(kFull, dc0.y, kn & 31);
            prefetch(o_n, lw_n);
        }

        // make the predecessor available in the representation this step reads
        const bool p_narrow = w <= 32;
        const bool p_full = !p_narrow && w == D;
        if (!first) {
            const bool need_smem = (p_narrow && loc != 0) || (p_full && loc != 1) ||
                                   (!p_narrow && !p_full);
            if (need_smem && loc != 2) {
                if (loc == 0) {
                    if (lane < qw) reinterpret_cast<uint16_t*>(buf0)[qlo + lane] = (uint16_t)Nreg;
                } else {
#pragma unroll
                    for (int k2 = 0; k2 < NP; ++k2) buf0[(LPL * lane) / 2 + k2] = Dreg[k2];
                }
                qb = 0;
                loc = 2;
                __syncwarp();
            }
        }
        const uint32_t* srcp = buf0 + qb * kBufPairs;
        const uint16_t* src16 = reinterpret_cast<const uint16_t*>(srcp);
        int lmin;
        if (p_narrow) {
            const bool act = lane < w;
            int L;
            if (first) {
                L = cN;
            } else {
                int vc, vl, vr;
                if (loc == 0) {
                    const int s = lane + (lo - qlo);
                    vc = __shfl_sync(kFull, Nreg, s & 31);
                    vl = __shfl_sync(kFull, Nreg, (s - 1) & 31);
                    vr = __shfl_sync(kFull, Nreg, (s + 1) & 31);
                    vc = ((unsigned)s < (unsigned)qw) ? vc : kInf;
                    vl = ((unsigned)(s - 1) < (unsigned)qw) ? vl : kInf;
                    vr = ((unsigned)(s + 1) < (unsigned)qw) ? vr : kInf;
                } else {
                    const int d = lo + lane;
                    const int qhi = qlo + qw - 1;
                    vc = (d >= qlo && d <= qhi) ? (int)src16[d] : kInf;
                    vl = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src16[d - 1] : kInf;
                    vr = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src16[d + 1] : kInf;
                }
                const int t = min(min(min(vl, vr) + P1, vc), m + P2);
                L = cN + t - m;
            }
            L = act ? L : kInf;
            const int Ln = __shfl_down_sync(kFull, L, 1);
            if (act && !(lane & 1))
                atomicAdd(S32 + ((o + lane) >> 1),
                          (uint32_t)L | ((lane + 1 < w) ? ((uint32_t)Ln << 16) : 0u));
            Nreg = L;
            lmin = L;
            loc = 0;
        } else if (p_full) {
            uint32_t Lq[NP];
            if (!first) {
                if (loc == 1) {
#pragma unroll
                    for (int k2 = 0; k2 < NP; ++k2) Lq[k2] = Dreg[k2];
                } else {
                    const int qhi = qlo + qw - 1;
#pragma unroll
                    for (int k2 = 0; k2 < NP; ++k2)
                        Lq[k2] = mask_pair(srcp[(LPL * lane) / 2 + k2], LPL * lane + 2 * k2, qlo, qhi);
                }
            }
            uint32_t pmin = kInf2;
            if (first) {
#pragma unroll
                for (int k2 = 0; k2 < NP; ++k2) {
                    Dreg[k2] = (c2[k2] & keep[k2]) | (kInf2 & ~keep[k2]);
                    pmin = vmin2(pmin, Dreg[k2]);
                }
            } else {
                uint32_t left_in = __shfl_up_sync(kFull, Lq[NP - 1], 1);
                uint32_t right_in = __shfl_down_sync(kFull, Lq[0], 1);
                if (lane == 0) left_in = kInf2;
                if (lane == 31) right_in = kInf2;
                const uint32_t mm = ((uint32_t)m << 16) | (uint32_t)m;
                const uint32_t mP2 = mm + (((uint32_t)P2 << 16) | (uint32_t)P2);
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
            }
            // packed reductions: the lane's pairs are 4-byte aligned (even block start, LPL even)
#pragma unroll
            for (int k2 = 0; k2 < NP; ++k2) {
                const int e = LPL * lane + 2 * k2;
                if (e < D) atomicAdd(S32 + ((o + e) >> 1), Dreg[k2] & keep[k2]);
            }
            lmin = (int)min(pmin & 0xFFFFu, pmin >> 16);
            loc = 1;
        } else {
            // general window: shared memory indexed by absolute disparity
            uint16_t* dst16 = reinterpret_cast<uint16_t*>(buf0 + (qb ^ 1) * kBufPairs);
            const int qhi = qlo + qw - 1;
            lmin = kInf;
            for (int j0 = 0; j0 < w; j0 += 32) {
                const int j = j0 + lane;
                const bool act = j < w;
                const int d = lo + j;
                const int c = (j0 == 0) ? cN : (act ? (int)__ldg(C + o + j) : 0);
                int L;
                if (first) {
                    L = c;
                } else {
                    const int vc = (d >= qlo && d <= qhi) ? (int)src16[d] : kInf;
                    const int vl = (d - 1 >= qlo && d - 1 <= qhi) ? (int)src16[d - 1] : kInf;
                    const int vr = (d + 1 >= qlo && d + 1 <= qhi) ? (int)src16[d + 1] : kInf;
                    const int t = min(min(min(vl, vr) + P1, vc), m + P2);
                    L = c + t - m;
                }
                L = act ? L : kInf;
                if (act) dst16[d] = (uint16_t)L;
                lmin = min(lmin, L);
                const int Ln = __shfl_down_sync(kFull, L, 1);
                if (act && !(j & 1))
                    atomicAdd(S32 + ((o + j) >> 1),
                              (uint32_t)L | ((j + 1 < w) ? ((uint32_t)Ln << 16) : 0u));
            }
            qb ^= 1;
            loc = 2;
        }
        m = (int)__reduce_min_sync(kFull, (unsigned)lmin);
        qlo = lo;
        qw = w;
        __syncwarp();
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
                                                 const uint2* __restrict__ desc, int W,
                                                 float s_thr, float r_min, int lr_tol,
                                                 float* __restrict__ Dz, float* __restrict__ rz,
                                                 int16_t* __restrict__ dstar_out,
                                                 int16_t* __restrict__ dright_out,
                                                 uint8_t* __restrict__ valid_out) {
    extern __shared__ uint32_t sel_smem[];
    uint32_t* drk = sel_smem;            // W keys
    float* dzs = (float*)(drk + W);      // W
    float* rzs = dzs + W;                // W
    int16_t* ds = (int16_t*)(rzs + W);   // W
    const int y = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int x = threadIdx.x; x < W; x += blockDim.x) drk[x] = 0xFFFFFFFFu;
    __syncthreads();
    for (int x = wid; x < W; x += nw) {
        const int i = y * W + x;
        const uint2 dsc = desc[i];
        const int a = (int)(dsc.y & 0xFFFFu);
        const int w = (int)(dsc.y >> 16);
        const uint16_t* s = S + dsc.x;
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

cudaError_t launch_cost(const uint64_t* cl, const uint64_t* cr, const uint2* desc, int W, int Hh,
                        int Bc, uint8_t* C, uint16_t* S, cudaStream_t st) {
    const int n = W * Hh;
    int blocks = (n * 8 + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_cost<<<blocks, 256, 0, st>>>(cl, cr, desc, W, n, Bc, C, S);
    return cudaGetLastError();
}

template <int LPL>
static cudaError_t launch_sgm_t(const uint8_t* C, const uint2* desc, int W, int Hh, int D,
                                int P1, int P2, const SgmLines& L, uint32_t* S32, cudaStream_t st) {
    const int nlines = L.start[L.nslots];
    const int blocks = (nlines + kSgmWarps - 1) / kSgmWarps;
    const size_t smem = (size_t)kSgmWarps * 2 * (32 * LPL) * sizeof(uint16_t);  // 2 buffers/warp
    k_sgm<LPL><<<blocks, kSgmWarps * 32, smem, st>>>(C, desc, W, Hh, D, P1, P2, L, S32);
    return cudaGetLastError();
}

cudaError_t launch_sgm(const uint8_t* C, const uint2* desc, int W, int Hh, int D, int n_paths,
                       int P1, int P2, uint16_t* S, cudaStream_t st) {
    // slots ordered longest lines first: horizontal, vertical, then diagonals
    SgmLines L;
    L.nslots = n_paths;
    L.start[0] = 0;
    for (int s = 0; s < n_paths; ++s) {
        const int code = s;
        L.code[s] = code;
        const int cnt = code <= 1 ? Hh : (code <= 3 ? W : W + Hh - 1);
        L.start[s + 1] = L.start[s] + cnt;
    }
    uint32_t* S32 = reinterpret_cast<uint32_t*>(S);
    if (D <= 64) return launch_sgm_t<2>(C, desc, W, Hh, D, P1, P2, L, S32, st);
    if (D <= 128) return launch_sgm_t<4>(C, desc, W, Hh, D, P1, P2, L, S32, st);
    if (D <= 192) return launch_sgm_t<6>(C, desc, W, Hh, D, P1, P2, L, S32, st);
    return launch_sgm_t<8>(C, desc, W, Hh, D, P1, P2, L, S32, st);
}

cudaError_t launch_select(const uint16_t* S, const uint2* desc, int W, int Hh, float s_thr,
                          float r_min, int lr_tol, float* Dz, float* rz, int16_t* dstar,
                          int16_t* dright, uint8_t* valid, cudaStream_t st) {
    const size_t smem = (size_t)W * (4 + 4 + 4 + 2);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_select<<<Hh, 1024, smem, st>>>(S, desc, W, s_thr, r_min, lr_tol, Dz, rz, dstar, dright,
                                     valid);
    return cudaGetLastError();
}

}  // namespace tsgm
