// Stereo matching restricted to per-pixel disparity windows (Sec. 2.3-2.4):
//   census transform -> ragged Hamming cost -> SGM path aggregation -> WTA / sub-pixel /
//   matching variance (Eq. 9) -> left-right check.
//
// Ragged volumes: pixel i owns cells off[i] .. off[i] + w_i - 1 (cell j <-> disparity lo[i] + j)
// of a block of w_i rounded up to a multiple of 4 cells, so blocks start 4-byte aligned. C is the
// uint8 Hamming cost; each SGM direction r writes its path cost L_r (<= census bits + P2 <= 255)
// to its own uint8 volume with plain stores, and the selection kernel forms S = sum_r L_r.
// Each pixel's {off, lo | w << 16} descriptor is read once per pixel.

#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>

#include "tsgm_kernels.cuh"
#include "tsgm_sgm.cuh"

namespace tsgm {
namespace {

using namespace dev;

template <int CW, int CH>
__global__ void __launch_bounds__(kCtW* kCtH) k_census(const uint8_t* __restrict__ imgA,
                                                        const uint8_t* __restrict__ imgB, int W,
                                                        int Hh, int cw, int ch,
                                                        uint64_t* __restrict__ outA,
                                                        uint64_t* __restrict__ outB) {
    census_tile<CW, CH>(blockIdx.z ? imgB : imgA, W, Hh, cw, ch, blockIdx.x * kCtW,
                        blockIdx.y * kCtH, blockIdx.z ? outB : outA);
}

__global__ void __launch_bounds__(256) k_cost(const uint64_t* __restrict__ cl,
                                              const uint64_t* __restrict__ cr,
                                              const uint2* __restrict__ desc, int W, int n,
                                              int Bc, uint8_t* __restrict__ C) {
    cost_pixels(cl, cr, desc, W, n, Bc, C, (blockIdx.x * blockDim.x + threadIdx.x) / kCostLanes,
                threadIdx.x % kCostLanes, (gridDim.x * blockDim.x) / kCostLanes);
}

// Path aggregation of one image: all lines of all directions in one launch, NG groups of lanes
// per warp, each on a line of one direction or on a segment of a long horizontal line (see
// sgm_group_lines; horizontal lines first: they are the longest chains).
// The lines' groups are 4 lanes wide (windows of up to 16 labels in straight-line code, 8 lines
// per warp) unless more than one pixel in 16 has a wider window (wq[0], the count of windows
// wider than kSelNarrow = 16 labels, written by the offsets pass) or D > 128: then 8 lanes (up to
// 32 labels, 4 lines per warp). Each form is its own kernel (so that each gets its own register
// allocation: the 8-lane form needs fewer registers, and a full-range frame's 3000 warps then
// fit on the GPU at once); both are launched, and the one that is not the frame's form returns
// at once.
constexpr int kGrpWarps = 4;

template <int LPLW, int GL>
__global__ void __launch_bounds__(kGrpWarps * 32, GL == 8 ? (LPLW == 8 ? 6 : 8) : 5) k_sgm(
    const uint8_t* __restrict__ C, const uint2* __restrict__ desc, int W, int Hh, int P1, int P2,
    GrpLines lines, uint8_t* __restrict__ Lvol, uint64_t vol_stride,
    const uint32_t* __restrict__ wq, int n) {
    extern __shared__ uint32_t sgm_smem32[];
    constexpr int NG = 32 / GL;
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * kGrpWarps + wib;
    uint32_t* const wsm = sgm_smem32 + wib * grp_words_ng<LPLW, NG>();
    // 256 labels: always the 8-lane groups (the 4-lane form's dense step would hold 64 labels
    // of costs per lane)
    const bool eight = LPLW == 8 || 16ull * wq[0] > (unsigned long long)n;
    if (eight != (GL == 8)) return;
    int code, first, nlines, seg;
    if (!grp_warp_lines(lines, NG, gw, code, first, nlines, seg)) return;
    uint8_t* const Lv = Lvol + (size_t)code * vol_stride;
    sgm_group_lines<LPLW, GL>(C, desc, W, Hh, P1, P2, code, first, nlines, seg, Lv, wsm);
}

// Path aggregation of an image whose windows are all the full range (every block rD = D rounded
// up to 4 cells, pixel i's at cell i rD): one warp per line (sgm_full_line), lines in the same
// direction-major order, no descriptors read.
constexpr int kFullWarps = 8;

// Warp gw's line: direction codes 0 .. n_paths - 1 in turn (horizontal, vertical, diagonal).
__device__ __forceinline__ bool full_warp_line(int n_paths, int W, int Hh, int gw, int& code,
                                               int& line) {
    int base = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (c < n_paths) {
            const int cnt = c <= 1 ? Hh : (c <= 3 ? W : W + Hh - 1);
            if (gw < base + cnt) {
                code = c;
                line = gw - base;
                return true;
            }
            base += cnt;
        }
    }
    return false;
}

template <int LPLW, bool V16, bool EXACT>
__global__ void __launch_bounds__(kFullWarps * 32, LPLW == 8 ? (EXACT ? 6 : 5) : (EXACT ? 8 : 6)) k_sgm_full(
    const uint8_t* __restrict__ C, int W, int Hh, int D, int P1, int P2, int n_paths,
    uint8_t* __restrict__ Lvol, uint64_t vol_stride) {
    __shared__ __align__(16) uint32_t ring[kFullWarps * kFullRing * 8 * LPLW];
    const int gw = blockIdx.x * kFullWarps + (threadIdx.x >> 5);
    int code = 0, line = 0;
    if (!full_warp_line(n_paths, W, Hh, gw, code, line)) return;
    sgm_full_line<LPLW, V16, EXACT>(C, W, Hh, D, (D + 3) & ~3, P1, P2, code, line,
                                    Lvol + (size_t)code * vol_stride,
                                    ring + (threadIdx.x >> 5) * kFullRing * 8 * LPLW);
}

template <int LPLW>
static void launch_sgm_full_t(const uint8_t* C, int W, int Hh, int D, int P1, int P2, int n_paths,
                              int nwarps, uint8_t* Lvol, uint64_t vol_stride, cudaStream_t st) {
    const int blocks = (nwarps + kFullWarps - 1) / kFullWarps;
    const int rD = (D + 3) & ~3;
    if (D == 32 * LPLW)
        k_sgm_full<LPLW, true, true><<<blocks, kFullWarps * 32, 0, st>>>(C, W, Hh, D, P1, P2, n_paths, Lvol, vol_stride);
    else if (rD == 32 * LPLW)
        k_sgm_full<LPLW, true, false><<<blocks, kFullWarps * 32, 0, st>>>(C, W, Hh, D, P1, P2, n_paths, Lvol, vol_stride);
    else
        k_sgm_full<LPLW, false, false><<<blocks, kFullWarps * 32, 0, st>>>(C, W, Hh, D, P1, P2, n_paths, Lvol, vol_stride);
}

// Selection of one image: a cluster of kSelCluster blocks per row, each block a quarter of the
// row's pixels (seg columns from x0). Every block keeps the right-view keys its own pixels can
// reach, columns x0 - (D - 1) .. x0 + seg - 1, with atomics in its own shared memory (merging the
// keys of the wide windows that k_select_wide took); after the cluster barrier the key of column
// xr is the minimum over the (at most few) blocks whose pixels reach it, read through distributed
// shared memory.
constexpr int kSelCluster = 4;
constexpr int kSelThreadsCl = 256;
// k_select's blocks: a thread per pixel of the block's quarter row (rounded up to whole warps), at
// most this many (then a thread takes several)
constexpr int kSelThreadsMax = 512;

struct ClusterPart {
    uint32_t* keys;
    int nkeys;   // seg + D - 1
    int seg, D, W, base;  // base: the column of keys[0] (x0 - (D - 1))
    __device__ uint32_t* own_keys() const { return keys; }
    __device__ void keymin(int xr, uint32_t k) const { atomicMin(keys + (xr - base), k); }
    __device__ uint32_t key(int xr) const {
        // pixels x = xr + d (d < D) lie in the blocks from xr's block to (xr + D - 1)'s
        const int b0 = xr / seg, b1 = min(W - 1, xr + D - 1) / seg;
        uint32_t k = 0xFFFFFFFFu;
        for (int b = b0; b <= b1; ++b)
            k = min(k, cooperative_groups::this_cluster().map_shared_rank(keys, b)[xr - (b * seg - (D - 1))]);
        return k;
    }
    __device__ void sync() const { cooperative_groups::this_cluster().sync(); }
    __device__ int key_base() const { return base; }
};

template <int NPATHS, int NCH>
__global__ void __cluster_dims__(kSelCluster, 1, 1) __launch_bounds__(kSelThreadsMax) k_select(
    const uint8_t* __restrict__ Lvol, uint64_t vol_stride, const uint2* __restrict__ desc, int W,
    int DP, int DPim, float s_thr, float r_min, int lr_tol, float* __restrict__ Dz,
    float* __restrict__ rz, uint16_t* __restrict__ S_out, int16_t* __restrict__ dstar_out,
    int16_t* __restrict__ dright_out, uint8_t* __restrict__ valid_out, int n,
    const uint32_t* __restrict__ wq, uint32_t* __restrict__ gkeys, const int16_t* __restrict__ wds) {
    extern __shared__ uint32_t sel_smem[];
    __shared__ int n_wide;
    const int rank = (int)cooperative_groups::this_cluster().block_rank();
    const int y = blockIdx.x / kSelCluster;
    const int seg = (W + kSelCluster - 1) / kSelCluster;
    const int x0 = min(W, rank * seg), x1 = min(W, x0 + seg);
    const int D = DPim;
    ClusterPart part{sel_smem, seg + D - 1, seg, D, W, rank * seg - (D - 1)};
    select_part<NPATHS, NCH>(Lvol, vol_stride, desc, W, y, x0, x1, DP, s_thr, r_min, lr_tol, Dz, rz,
                             S_out, dstar_out, dright_out, valid_out, sel_smem, n_wide, part, n, wq,
                             gkeys + (size_t)y * W, wds);
}

// Selection of an image whose windows are all the full range: a cluster of kSelCluster blocks per
// row as k_select (the right-view keys of a block's pixels in its shared memory, merged across the
// cluster), every pixel by one warp (select_full_px), the path costs of a warp's next pixel loaded
// during the current one. bytesum: census bits + P2 < 128 (every path cost below 128).
template <int NPATHS, int LPL>
__global__ void __cluster_dims__(kSelCluster, 1, 1) __launch_bounds__(kSelThreadsCl) k_select_full(
    const uint8_t* __restrict__ Lvol, uint64_t vol_stride, int W, int D, int bytesum, float s_thr,
    float r_min, int lr_tol, float* __restrict__ Dz, float* __restrict__ rz,
    uint16_t* __restrict__ S_out, int16_t* __restrict__ dstar_out,
    int16_t* __restrict__ dright_out, uint8_t* __restrict__ valid_out) {
    constexpr int NW = LPL >= 4 ? LPL / 4 : 1;
    extern __shared__ uint32_t sel_smem[];
    const int rank = (int)cooperative_groups::this_cluster().block_rank();
    const int y = blockIdx.x / kSelCluster;
    const int seg = (W + kSelCluster - 1) / kSelCluster;
    const int x0 = min(W, rank * seg), x1 = min(W, x0 + seg);
    const int npx = x1 - x0;
    const int rD = (D + 3) & ~3;
    ClusterPart part{sel_smem, seg + D - 1, seg, D, W, rank * seg - (D - 1)};
    uint32_t* const drk = part.own_keys();
    float* const dzs = reinterpret_cast<float*>(sel_smem + part.nkeys);
    float* const rzs = dzs + seg;
    int16_t* const ds = reinterpret_cast<int16_t*>(rzs + seg);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint16_t* const scr = reinterpret_cast<uint16_t*>(sel_smem + ((part.nkeys + 3 * seg + 1) & ~1)) +
                          wid * ((D + 7) & ~7);
    for (int t = threadIdx.x; t < part.nkeys; t += blockDim.x) drk[t] = 0xFFFFFFFFu;
    __syncthreads();

    auto px = [&](const uint32_t (&v)[NPATHS * NW], int q) {
        const int x = x0 + q;
        const size_t o = (size_t)(y * W + x) * rD;
        int dsr;
        float dzr, rr;
        select_full_px<NPATHS, LPL>(v, D, bytesum != 0, x, o, s_thr, r_min, scr, S_out,
                                    [&](int xr, uint32_t k) { part.keymin(xr, k); }, dsr, dzr, rr);
        if (lane == 0) {
            ds[q] = (int16_t)dsr;
            dzs[q] = dzr;
            rzs[q] = rr;
        }
    };
    // two register sets in turn: the next pixel's costs load during the current one
    uint32_t va[NPATHS * NW], vb[NPATHS * NW];
    auto load = [&](uint32_t (&v)[NPATHS * NW], int q) {
        load_full_costs<NPATHS, LPL>(Lvol, vol_stride, (size_t)(y * W + x0 + q) * rD, D, v);
    };
    if (wid < npx) load(va, wid);
    for (int q = wid; q < npx; q += 2 * nw) {
        if (q + nw < npx) load(vb, q + nw);
        px(va, q);
        if (q + nw >= npx) break;
        if (q + 2 * nw < npx) load(va, q + 2 * nw);
        px(vb, q + nw);
    }
    part.sync();  // every key of the row is final
    for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
        const int i = y * W + x;
        const int d = ds[x - x0];
        const int xr = x - d;
        bool ok = false;
        if (xr >= 0) {
            const uint32_t kk = part.key(xr);
            ok = kk != 0xFFFFFFFFu && abs(d - (int)(kk & 0x1FFu)) <= lr_tol;
        }
        Dz[i] = ok ? dzs[x - x0] : -1.0f;
        rz[i] = ok ? rzs[x - x0] : -1.0f;
        if (dstar_out) {
            dstar_out[i] = (int16_t)d;
            const uint32_t kx = part.key(x);
            dright_out[i] = kx == 0xFFFFFFFFu ? (int16_t)-1 : (int16_t)(kx & 0x1FFu);
            valid_out[i] = ok ? 1 : 0;
        }
    }
    part.sync();  // no block leaves while another may still read its keys
}

// The wide windows of the queue wq (see select_split), one warp per pixel (pixel t of the queue by
// warp t mod the launch's warps, the next one's path costs loaded during the current one): winner,
// sub-pixel disparity and matching variance into wds, Dz and rz (the row's selection clears Dz and
// rz where the left-right check fails), right-view keys into gkeys (atomic minimum per column).
template <int NPATHS, int NCH>
__global__ void __launch_bounds__(256) k_select_wide(const uint8_t* __restrict__ Lvol,
                                                     uint64_t vol_stride,
                                                     const uint2* __restrict__ desc, int W, int n,
                                                     float s_thr, float r_min,
                                                     float* __restrict__ Dz, float* __restrict__ rz,
                                                     uint16_t* __restrict__ S_out,
                                                     int16_t* __restrict__ wds,
                                                     uint32_t* __restrict__ gkeys,
                                                     const uint32_t* __restrict__ wq) {
    __shared__ __align__(16) uint16_t scr_all[8][NCH * 128];
    // k_select, launched next with programmatic serialisation, may start its narrow pixels now:
    // it waits for this grid (griddepcontrol.wait) before it reads what this kernel writes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int count = (int)wq[0];
    if (!select_split((uint32_t)count, n)) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nwarps = gridDim.x * 8;
    uint16_t* const scr = scr_all[wid];
    // the path costs of the next two pixels are loaded during the current one
    uint32_t vcur[NCH * NPATHS], vnext[NCH * NPATHS], vnext2[NCH * NPATHS];
    uint2 dcur = make_uint2(0u, 0u), dnext = make_uint2(0u, 0u), dnext2 = make_uint2(0u, 0u);
    int t = blockIdx.x * 8 + wid;
    int icur = 0, inext = 0, inext2 = 0;
    if (t < count) {
        icur = (int)wq[1 + t];
        dcur = desc[icur];
        load_wide_costs<NPATHS, NCH>(Lvol, vol_stride, dcur, vcur);
    }
    if (t + nwarps < count) {
        inext = (int)wq[1 + t + nwarps];
        dnext = desc[inext];
        load_wide_costs<NPATHS, NCH>(Lvol, vol_stride, dnext, vnext);
    }
    for (; t < count; t += nwarps) {
        if (t + 2 * nwarps < count) {
            inext2 = (int)wq[1 + t + 2 * nwarps];
            dnext2 = desc[inext2];
            load_wide_costs<NPATHS, NCH>(Lvol, vol_stride, dnext2, vnext2);
        }
        const int y = icur / W, x = icur - y * W;
        uint32_t* const grow = gkeys + (size_t)y * W;
        int dsr;
        float dzr, rr;
        select_wide<NPATHS, NCH>(vcur, dcur, x, s_thr, r_min, scr, S_out,
                                 [&](int xr, uint32_t k) { atomicMin(grow + xr, k); }, dsr, dzr, rr);
        if (lane == 0) {
            wds[icur] = (int16_t)dsr;
            Dz[icur] = dzr;
            rz[icur] = rr;
        }
#pragma unroll
        for (int q = 0; q < NCH * NPATHS; ++q) {
            vcur[q] = vnext[q];
            vnext[q] = vnext2[q];
        }
        dcur = dnext;
        dnext = dnext2;
        icur = inext;
        inext = inext2;
    }
}

}  // namespace

cudaError_t launch_census(const uint8_t* imgA, const uint8_t* imgB, int W, int Hh, int cw, int ch,
                          uint64_t* outA, uint64_t* outB, cudaStream_t st) {
    dim3 blk(kCtW, kCtH);
    dim3 grd((W + kCtW - 1) / kCtW, (Hh + kCtH - 1) / kCtH, imgB ? 2 : 1);
    if (cw == 9 && ch == 7)
        k_census<9, 7><<<grd, blk, 0, st>>>(imgA, imgB, W, Hh, cw, ch, outA, outB);
    else if (cw == 5 && ch == 5)
        k_census<5, 5><<<grd, blk, 0, st>>>(imgA, imgB, W, Hh, cw, ch, outA, outB);
    else
        k_census<0, 0><<<grd, blk, 0, st>>>(imgA, imgB, W, Hh, cw, ch, outA, outB);
    return cudaGetLastError();
}

cudaError_t launch_cost(const uint64_t* cl, const uint64_t* cr, const uint2* desc, int W, int Hh,
                        int Bc, uint8_t* C, cudaStream_t st) {
    // a group of lanes per pixel: blocks retire as their pixels' windows are done, so that the
    // few wide windows of a reduced frame spread over the launch instead of lengthening the
    // loops of a fixed grid
    const int n = W * Hh;
    const int blocks = (int)(((size_t)n * kCostLanes + 255) / 256);
    k_cost<<<blocks, 256, 0, st>>>(cl, cr, desc, W, n, Bc, C);
    return cudaGetLastError();
}

template <int LPLW, int GL>
static cudaError_t launch_sgm_form(const uint8_t* C, const uint2* desc, int W, int Hh, int P1,
                                   int P2, const GrpLines& L, uint8_t* Lvol, uint64_t vol_stride,
                                   const uint32_t* wq, cudaStream_t st) {
    constexpr int NG = 32 / GL;
    int nwarps = 0;
    for (int s = 0; s < L.nslots; ++s) {
        const int per = NG / grp_slot_seg(L, s, NG);
        nwarps += (L.count[s] + per - 1) / per;
    }
    const size_t smem = (size_t)kGrpWarps * grp_words_ng<LPLW, NG>() * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_sgm<LPLW, GL>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_sgm<LPLW, GL><<<(nwarps + kGrpWarps - 1) / kGrpWarps, kGrpWarps * 32, smem, st>>>(
        C, desc, W, Hh, P1, P2, L, Lvol, vol_stride, wq, W * Hh);
    return cudaGetLastError();
}

// both forms for D <= 128 (the 8-lane one first: on a full-range frame it does the work), the
// 8-lane form alone beyond
template <int LPLW>
static cudaError_t launch_sgm_t(const uint8_t* C, const uint2* desc, int W, int Hh, int P1, int P2,
                                const GrpLines& L, uint8_t* Lvol, uint64_t vol_stride,
                                const uint32_t* wq, cudaStream_t st) {
    cudaError_t e = launch_sgm_form<LPLW, 8>(C, desc, W, Hh, P1, P2, L, Lvol, vol_stride, wq, st);
    if constexpr (LPLW < 8) {
        if (e == cudaSuccess)
            e = launch_sgm_form<LPLW, 4>(C, desc, W, Hh, P1, P2, L, Lvol, vol_stride, wq, st);
    }
    return e;
}

cudaError_t launch_sgm(const uint8_t* C, const uint2* desc, int W, int Hh, int D, int n_paths,
                       int P1, int P2, uint8_t* Lvol, uint64_t vol_stride, const uint32_t* wq,
                       bool full, cudaStream_t st) {
    // direction codes: horizontal (0, 1), vertical (2, 3), then the diagonals
    GrpLines L;
    L.nslots = n_paths;
    for (int code = 0; code < n_paths; ++code) {
        L.code[code] = code;
        L.count[code] = code <= 1 ? Hh : (code <= 3 ? W : W + Hh - 1);
        // long lines in segments
        L.seg[code] = grp_seg(code <= 1 ? W : (code <= 3 ? Hh : (W < Hh ? W : Hh)));
    }
    if (full) {
        int nwarps = 0;
        for (int code = 0; code < n_paths; ++code) nwarps += L.count[code];
        if (D <= 64)
            launch_sgm_full_t<2>(C, W, Hh, D, P1, P2, n_paths, nwarps, Lvol, vol_stride, st);
        else if (D <= 128)
            launch_sgm_full_t<4>(C, W, Hh, D, P1, P2, n_paths, nwarps, Lvol, vol_stride, st);
        else
            launch_sgm_full_t<8>(C, W, Hh, D, P1, P2, n_paths, nwarps, Lvol, vol_stride, st);
        return cudaGetLastError();
    }
    if (D <= 64) return launch_sgm_t<2>(C, desc, W, Hh, P1, P2, L, Lvol, vol_stride, wq, st);
    if (D <= 128) return launch_sgm_t<4>(C, desc, W, Hh, P1, P2, L, Lvol, vol_stride, wq, st);
    return launch_sgm_t<8>(C, desc, W, Hh, P1, P2, L, Lvol, vol_stride, wq, st);
}

template <int NPATHS, int LPL>
static cudaError_t launch_select_full_t(const uint8_t* Lvol, uint64_t vol_stride, int W, int Hh,
                                        int D, int bytesum, float s_thr, float r_min, int lr_tol,
                                        float* Dz, float* rz, uint16_t* S, int16_t* dstar,
                                        int16_t* dright, uint8_t* valid, cudaStream_t st) {
    const int seg = (W + kSelCluster - 1) / kSelCluster;
    const size_t smem = (size_t)((seg + D - 1 + 3 * seg + 1) & ~1) * 4 +
                        (size_t)(kSelThreadsCl / 32) * ((D + 7) & ~7) * sizeof(uint16_t);
    auto kern = k_select_full<NPATHS, LPL>;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<Hh * kSelCluster, kSelThreadsCl, smem, st>>>(Lvol, vol_stride, W, D, bytesum, s_thr, r_min,
                                                        lr_tol, Dz, rz, S, dstar, dright, valid);
    return cudaGetLastError();
}

template <int NPATHS>
static cudaError_t launch_select_full_p(const uint8_t* Lvol, uint64_t vol_stride, int W, int Hh,
                                        int D, int bytesum, float s_thr, float r_min, int lr_tol,
                                        float* Dz, float* rz, uint16_t* S, int16_t* dstar,
                                        int16_t* dright, uint8_t* valid, cudaStream_t st) {
    if (D <= 64)
        return launch_select_full_t<NPATHS, 2>(Lvol, vol_stride, W, Hh, D, bytesum, s_thr, r_min,
                                               lr_tol, Dz, rz, S, dstar, dright, valid, st);
    if (D <= 128)
        return launch_select_full_t<NPATHS, 4>(Lvol, vol_stride, W, Hh, D, bytesum, s_thr, r_min,
                                               lr_tol, Dz, rz, S, dstar, dright, valid, st);
    return launch_select_full_t<NPATHS, 8>(Lvol, vol_stride, W, Hh, D, bytesum, s_thr, r_min,
                                           lr_tol, Dz, rz, S, dstar, dright, valid, st);
}

cudaError_t launch_select_full(const uint8_t* Lvol, uint64_t vol_stride, int n_paths, int W, int Hh,
                               int D, int Bc, int P2, float s_thr, float r_min, int lr_tol,
                               float* Dz, float* rz, uint16_t* S, int16_t* dstar, int16_t* dright,
                               uint8_t* valid, cudaStream_t st) {
    const int bytesum = Bc + P2 < 128 ? 1 : 0;
    return n_paths == 8
               ? launch_select_full_p<8>(Lvol, vol_stride, W, Hh, D, bytesum, s_thr, r_min, lr_tol,
                                         Dz, rz, S, dstar, dright, valid, st)
               : launch_select_full_p<4>(Lvol, vol_stride, W, Hh, D, bytesum, s_thr, r_min, lr_tol,
                                         Dz, rz, S, dstar, dright, valid, st);
}

cudaError_t launch_select(const uint8_t* Lvol, uint64_t vol_stride, int n_paths, const uint2* desc,
                          int W, int Hh, int D, float s_thr, float r_min, int lr_tol, float* Dz,
                          float* rz, uint16_t* S, int16_t* dstar, int16_t* dright, uint8_t* valid,
                          const uint32_t* wq, uint32_t* gkeys, int16_t* wds, cudaStream_t st) {
    // per-warp scratch for the wide windows: up to 256 labels
    const int DP = 256;
    const int n = W * Hh;
    const int seg = (W + kSelCluster - 1) / kSelCluster;
    const int threads = std::min(kSelThreadsMax, std::max(64, (seg + 31) & ~31));
    const size_t smem = (size_t)((seg + D - 1 + 3 * seg + 1) & ~1) * 4 +
                        (size_t)(threads / 32) * DP * sizeof(uint16_t);
    auto wide = n_paths == 8 ? (D <= 128 ? k_select_wide<8, 1> : k_select_wide<8, 2>)
                             : (D <= 128 ? k_select_wide<4, 1> : k_select_wide<4, 2>);
    wide<<<152 * 8, 256, 0, st>>>(Lvol, vol_stride, desc, W, n, s_thr, r_min, Dz, rz, S, wds,
                                  gkeys, wq);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto kern = n_paths == 8 ? (D <= 128 ? k_select<8, 1> : k_select<8, 2>)
                             : (D <= 128 ? k_select<4, 1> : k_select<4, 2>);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // programmatic dependent launch: the row clusters select their narrow pixels while
    // k_select_wide still runs, and wait for it before they merge its keys and winners
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(Hh * kSelCluster));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, Lvol, vol_stride, desc, W, DP, D, s_thr, r_min, lr_tol, Dz, rz,
                           S, dstar, dright, valid, n, wq, gkeys, wds);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace tsgm
