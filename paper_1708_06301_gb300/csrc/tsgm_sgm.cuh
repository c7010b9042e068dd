// SGM path aggregation restricted to per-pixel disparity windows (Sec. 2.3), several path lines
// per warp in lockstep.
//
// Recurrence of one path direction r (Hirschmueller's, on windows): for pixel p with predecessor
// q = p - r along the line,
//   L(p, d) = C(p, d) + min(L(q, d), L(q, d - 1) + P1, L(q, d + 1) + P1, m(q) + P2) - m(q),
//   m(q) = min over q's window of L(q, .),
// where L(q, .) outside q's window is +inf (so a window that does not overlap its predecessor's
// keeps only the m + P2 term) and the first pixel of a line has L = C.
//
// Work split. A warp walks NG = 32 / GL lines of one direction at once, one group of GL lanes per
// line, all groups taking their k-th step together. In a group, lane j holds labels lo + 4j ..
// lo + 4j + 3 of the current window as two packed 16-bit pairs (min.u16x2 arithmetic), so a
// window of up to 4 GL labels is one step of straight-line code; m is a GL-lane shuffle
// reduction. A window wider than 4 GL labels is taken by the whole warp (LPLW labels per lane,
// m by redux.sync), one such group after the other.
//
// State. Each line keeps its last L as a row of 16-bit labels in shared memory, indexed relative
// to the window's lo, with +inf padding on both sides; two rows per line, used in turn. A step
// reads the predecessor's labels d - 1 .. d + 1 at the offset lo - lo(q), clamped into the padding
// (so that no range test is needed): this makes every change of window, narrow or wide, one code
// path. The costs of the step PF ahead are in flight into a ring of shared-memory slots
// (cp.async, issued by the group's own lanes), and the window descriptors come in blocks of 32
// steps per line (cp.async), two blocks in the ring.
//
// Each direction writes its path costs L (<= census bits + P2 <= 255) as bytes into its own
// ragged volume; the selection sums the directions.
#pragma once

#include "tsgm_kernels.cuh"

namespace tsgm {
namespace dev {

constexpr int kGPadL = 16, kGPadR = 16;  // +inf labels before and after a state row
constexpr int kGSlots = 8, kGPref = 6;   // cost ring slots per line and prefetch distance (steps)
constexpr int kGBlk = 32;                // steps per descriptor block
constexpr int kGSkew = 16;               // bytes between the cost rings of two lines (bank skew)

// labels of the wide (whole-warp) form: LPLW per lane, >= D
template <int LPLW>
__host__ __device__ constexpr int grp_dp() { return 32 * LPLW; }
// 16-bit entries of one state row
template <int LPLW>
__host__ __device__ constexpr int grp_row() { return kGPadL + grp_dp<LPLW>() + kGPadR; }
// shared memory of one warp in 32-bit words, for NG lines: state rows (2 per line), cost ring,
// descriptor ring
template <int LPLW, int NG>
__host__ __device__ constexpr int grp_words_ng() {
    return NG * (grp_row<LPLW>() + 32) + NG * (kGSlots * grp_dp<LPLW>() + kGSkew) / 4 +
           2 * kGBlk * NG * 2;
}

// Word offset of line g's two state rows (ROW / 2 words each, inside the line's ROW + 32 words).
// The start bank is chosen so that the NG lines' lanes, which read and write their rows at a
// stride of two words (lane j: entries 4j ..), fall on distinct banks when their windows move
// alike: half of the lines on even banks, half on odd, 2 GL banks apart.
template <int LPLW, int NG>
__device__ __forceinline__ int grp_row_base(int g) {
    constexpr int GL = 32 / NG, STR = grp_row<LPLW>() + 32;
    const int bank = 2 * GL * (g % (NG / 2)) + g / (NG / 2);
    return g * STR + ((bank - g * STR) & 31);
}
// the most any lane-group width needs (4 lanes per line: 8 lines)
template <int LPLW>
__host__ __device__ constexpr int grp_words() { return grp_words_ng<LPLW, 8>(); }

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

// mask of a packed label pair: both kept, the low one kept, none (rem labels left in the window)
__device__ __forceinline__ uint32_t pair_keep(int rem) {
    return rem >= 2 ? 0xFFFFFFFFu : (rem == 1 ? 0x0000FFFFu : 0u);
}

// Pair `np` (labels 2np, 2np + 1 of this lane's LPL) from the predecessor's packed words A[np],
// A[np + 1] (A[i] = entries e + 2i, e + 2i + 1 where e is the predecessor entry of label d - 1):
// min(L(d), L(d - 1) + P1, L(d + 1) + P1, m + P2) as a packed pair.
__device__ __forceinline__ uint32_t grp_t(uint32_t a0, uint32_t a1, uint32_t P1x2, uint32_t mP2) {
    const uint32_t t = vmin2(vmin2(a0, a1) + P1x2, __byte_perm(a0, a1, 0x5432));
    return vmin2(t, mP2);
}

// NG lines of direction `code`, lines first_line .. first_line + NG - 1 (those < nlines), one
// group of GL lanes each. Lv: the direction's volume; wsm: this warp's shared memory.
template <int LPLW, int GL>
__device__ __forceinline__ void sgm_group_lines(const uint8_t* __restrict__ C,
                                                const uint2* __restrict__ desc, int W, int Hh,
                                                int P1, int P2, int code, int first_line,
                                                int nlines, uint8_t* __restrict__ Lv,
                                                uint32_t* const wsm) {
    static_assert(GL == 4 || GL == 8, "lanes per line");
    static_assert(LPLW == 2 || LPLW == 4 || LPLW == 8, "labels per lane of the wide form");
    constexpr int NG = 32 / GL;
    constexpr int CAPN = 4 * GL;          // labels of the narrow form
    constexpr int DP = grp_dp<LPLW>();    // labels of the wide form
    constexpr int ROW = grp_row<LPLW>();  // entries of a state row
    constexpr int PF = kGPref, NS = kGSlots;
    constexpr int PER = kGBlk / GL;       // descriptors each lane loads per block
    static_assert(CAPN + 16 <= DP + kGPadR, "narrow padding inside the row");
    const int lane = threadIdx.x & 31;
    const int g = lane / GL, j = lane % GL;

    // state rows: line g's two rows start at word grp_row_base(g) (bank-skewed, 4-byte aligned)
    auto row_of = [&](int gi, int which) -> uint16_t* {
        return reinterpret_cast<uint16_t*>(wsm + grp_row_base<LPLW, NG>(gi) + which * (ROW / 2));
    };
    constexpr int RS = NS * DP + kGSkew;  // bytes of one line's cost ring
    uint8_t* const ring = reinterpret_cast<uint8_t*>(wsm + NG * (ROW + 32));  // [NG][RS]
    uint2* const dring = reinterpret_cast<uint2*>(ring + NG * RS);       // [2][kGBlk][NG]

    const int l = first_line + g;
    int i0 = 0, stp = 0, len = 0;
    if (l < nlines) line_geometry(code, l, W, Hh, i0, stp, len);
    const int maxlen = (int)__reduce_max_sync(kFull, (unsigned)len);
    if (maxlen == 0) return;

    for (int t = lane; t < NG * (ROW + 32); t += 32) wsm[t] = kInf2;

    auto dslot = [&](int s) -> uint2* {
        return dring + (((s >> 5) & 1) * kGBlk + (s & 31)) * NG + g;
    };
    auto load_block = [&](int b) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int s = b * kGBlk + j * PER + q;
            if (s < len) cp_async8(dslot(s), desc + (i0 + s * stp));
        }
    };
    // the costs of step s (its whole window, whole 4-byte words) into the line's ring slot; one
    // commit group per call
    auto issue = [&](int s) {
        if (s < len) {
            const uint2 ds = *dslot(s);
            const int nw = ((int)(ds.y >> 16) + 3) >> 2;
            uint8_t* const slot = ring + g * RS + (s % NS) * DP;
            for (int t = j; t < nw; t += GL) cp_async4(slot + 4 * t, C + ds.x + 4 * t);
        }
        cp_async_commit();
    };

    load_block(0);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    load_block(1);
    for (int s = 0; s < PF; ++s) issue(s);

    const uint32_t P1x2 = ((uint32_t)P1 << 16) | (uint32_t)P1;
    const uint32_t P2x2 = ((uint32_t)P2 << 16) | (uint32_t)P2;
    // predecessor of the first step: all +inf, m = 0 and no P2 term, so that L = C
    int lo_old = 0, cap_old = 0;
    uint32_t mm2 = 0u, mP2 = 0u;
    int cur = 0;

    for (int k = 0; k < maxlen; ++k) {
        if (k > 0 && (k & 31) == 0) load_block((k >> 5) + 1);
        issue(k + PF);
        cp_async_wait<PF>();  // this lane's copies of step k (and older) have landed
        __syncwarp();         // ... and every lane's
        const bool act = k < len;
        const uint2 ds = act ? *dslot(k) : make_uint2(0u, 0u);
        const int lo = (int)(ds.y & 0xFFFFu), w = (int)(ds.y >> 16);
        const bool wide = w > CAPN;

        // ---- narrow step of this lane's line (computed everywhere, stored where it applies) ----
        {
            const uint16_t* const rold = row_of(g, cur);
            uint16_t* const rnew = row_of(g, cur ^ 1);
            const int e = min(max(lo - lo_old + 4 * j - 1, -6), cap_old);
            const int b = kGPadL + e;
            const uint32_t* r32 = reinterpret_cast<const uint32_t*>(rold) + (b >> 1);
            const uint32_t sel = (b & 1) ? 0x5432u : 0x3210u;
            const uint32_t w0 = r32[0], w1 = r32[1], w2 = r32[2], w3 = r32[3];
            const uint32_t A0 = __byte_perm(w0, w1, sel), A1 = __byte_perm(w1, w2, sel),
                           A2 = __byte_perm(w2, w3, sel);
            const uint32_t cw =
                *reinterpret_cast<const uint32_t*>(ring + g * RS + (k % NS) * DP + 4 * j);
            const int rem = w - 4 * j;
            const uint32_t k0 = pair_keep(rem), k1 = pair_keep(rem - 2);
            uint32_t L0 = (__byte_perm(cw, 0u, 0x4140) + grp_t(A0, A1, P1x2, mP2)) - mm2;
            uint32_t L1 = (__byte_perm(cw, 0u, 0x4342) + grp_t(A1, A2, P1x2, mP2)) - mm2;
            L0 = (L0 & k0) | (kInf2 & ~k0);
            L1 = (L1 & k1) | (kInf2 & ~k1);
            const uint32_t pm = vmin2(L0, L1);
            int m = (int)min(pm & 0xFFFFu, pm >> 16);
#pragma unroll
            for (int s = 1; s < GL; s <<= 1) m = min(m, __shfl_xor_sync(kFull, m, s));
            if (act && !wide) {
                uint32_t* const rw = reinterpret_cast<uint32_t*>(rnew + kGPadL);
                rw[2 * j] = L0;
                rw[2 * j + 1] = L1;
                if (j < 4) {
                    rw[CAPN / 2 + 2 * j] = kInf2;
                    rw[CAPN / 2 + 2 * j + 1] = kInf2;
                }
                if (rem > 0)
                    *reinterpret_cast<uint32_t*>(Lv + ds.x + 4 * j) = __byte_perm(L0, L1, 0x6420);
                lo_old = lo;
                cap_old = CAPN;
                mm2 = (uint32_t)m * 0x10001u;
                mP2 = mm2 + P2x2;
            }
        }

        // ---- wide windows: the whole warp, one line after the other ----
        unsigned wb = __ballot_sync(kFull, act && wide && j == 0);
        while (wb) {
            const int gg = (__ffs(wb) - 1) / GL;
            wb &= wb - 1;
            const int src = gg * GL;
            const int lo_g = __shfl_sync(kFull, lo, src), w_g = __shfl_sync(kFull, w, src);
            const uint32_t o_g = __shfl_sync(kFull, ds.x, src);
            const int lo_old_g = __shfl_sync(kFull, lo_old, src);
            const int cap_old_g = __shfl_sync(kFull, cap_old, src);
            const uint32_t mm2_g = __shfl_sync(kFull, mm2, src);
            const uint32_t mP2_g = __shfl_sync(kFull, mP2, src);
            const uint16_t* const rold = row_of(gg, cur);
            uint16_t* const rnew = row_of(gg, cur ^ 1);
            constexpr int NPW = LPLW / 2;  // packed pairs per lane
            const int e = min(max(lo_g - lo_old_g + LPLW * lane - 1, -(LPLW + 2)), cap_old_g);
            const int b = kGPadL + e;
            const uint32_t* r32 = reinterpret_cast<const uint32_t*>(rold) + (b >> 1);
            const uint32_t sel = (b & 1) ? 0x5432u : 0x3210u;
            uint32_t wv[NPW + 2], A[NPW + 1];
#pragma unroll
            for (int i = 0; i < NPW + 2; ++i) wv[i] = r32[i];
#pragma unroll
            for (int i = 0; i < NPW + 1; ++i) A[i] = __byte_perm(wv[i], wv[i + 1], sel);
            const uint8_t* const cs = ring + gg * RS + (k % NS) * DP + LPLW * lane;
            uint32_t cpk[NPW];
            if constexpr (LPLW == 2) {
                cpk[0] = __byte_perm((uint32_t)*reinterpret_cast<const uint16_t*>(cs), 0u, 0x4140);
            } else {
#pragma unroll
                for (int q = 0; q < LPLW / 4; ++q) {
                    const uint32_t c4 = reinterpret_cast<const uint32_t*>(cs)[q];
                    cpk[2 * q] = __byte_perm(c4, 0u, 0x4140);
                    cpk[2 * q + 1] = __byte_perm(c4, 0u, 0x4342);
                }
            }
            const int rem = w_g - LPLW * lane;
            uint32_t Lw[NPW];
            uint32_t pm = kInf2;
#pragma unroll
            for (int i = 0; i < NPW; ++i) {
                const uint32_t kp = pair_keep(rem - 2 * i);
                const uint32_t v = (cpk[i] + grp_t(A[i], A[i + 1], P1x2, mP2_g)) - mm2_g;
                Lw[i] = (v & kp) | (kInf2 & ~kp);
                pm = vmin2(pm, Lw[i]);
            }
            const int mg = (int)__reduce_min_sync(kFull, min(pm & 0xFFFFu, pm >> 16));
            uint16_t* const dst = rnew + kGPadL + LPLW * lane;
            if constexpr (LPLW == 2) {
                *reinterpret_cast<uint32_t*>(dst) = Lw[0];
                if (rem > 0)
                    *reinterpret_cast<uint16_t*>(Lv + o_g + 2 * lane) =
                        (uint16_t)__byte_perm(Lw[0], 0u, 0x0020);
            } else {
#pragma unroll
                for (int q = 0; q < LPLW / 4; ++q) {
                    reinterpret_cast<uint32_t*>(dst)[2 * q] = Lw[2 * q];
                    reinterpret_cast<uint32_t*>(dst)[2 * q + 1] = Lw[2 * q + 1];
                    if (rem > 4 * q)
                        *reinterpret_cast<uint32_t*>(Lv + o_g + LPLW * lane + 4 * q) =
                            __byte_perm(Lw[2 * q], Lw[2 * q + 1], 0x6420);
                }
            }
            if (g == gg) {
                lo_old = lo_g;
                cap_old = DP;
                mm2 = (uint32_t)mg * 0x10001u;
                mP2 = mm2 + P2x2;
            }
        }
        cur ^= 1;
    }
    cp_async_wait<0>();
    __syncwarp();
}

// Lines of one image for the grouped walker: direction codes in launch order (horizontal pairs
// first: the longest chains) and their line counts.
struct GrpLines {
    int code[8];
    int count[8];
    int nslots;
};

// Map warp gw of the launch to (direction code, first line, line count) for NG lines per warp;
// false when gw is past the last line.
__device__ __forceinline__ bool grp_warp_lines(const GrpLines& L, int NG, int gw, int& code,
                                               int& first, int& nlines) {
    int base = 0;
    for (int s = 0; s < L.nslots; ++s) {
        const int nw = (L.count[s] + NG - 1) / NG;
        if (gw < base + nw) {
            code = L.code[s];
            first = (gw - base) * NG;
            nlines = L.count[s];
            return true;
        }
        base += nw;
    }
    return false;
}

}  // namespace dev
}  // namespace tsgm
