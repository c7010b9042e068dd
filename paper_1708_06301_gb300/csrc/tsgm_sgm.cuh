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
// Long lines in segments. A line's steps form one dependent chain, and the longest lines bound
// the launch. A line can be cut into S segments walked at once by S groups: segment 0 starts at
// the line's start; every other one starts as if a line began there (L = C), which is a guess.
// The recursion forgets its start fast (a window that shares no label with its predecessor's,
// or P2 capping every difference, makes L independent of what came before), so the guess and
// the true state agree after a few steps. The guess is then checked exactly: each later segment
// is walked again from the true end state of the segment before it, and before its steps 16, 32
// and kGFix its state is compared with the state the first walk had at the same pixel (three
// checkpoints; the first two only for windows of the narrow form). Equal states give equal
// values from there on, so the walk stops at the first check that agrees and the first walk's
// later values stand; a difference at the last check makes the walk go on to the segment's end
// (and the next segment is walked again from that end, and so on), so the result is the
// sequential recurrence's in every case. Lines of different lengths in one warp check at their
// own steps.
//
// State. Each line keeps its last L as a row of 16-bit labels in shared memory, indexed relative
// to the window's lo, with +inf padding on both sides; two rows per line, used in turn. A step
// reads the predecessor's labels d - 1 .. d + 1 at the offset lo - lo(q), clamped into the padding
// (so that no range test is needed): this makes every change of window, narrow or wide, one code
// path. The window descriptors come in blocks of kGBlk steps per line (cp.async into a small
// shared-memory ring, two blocks deep); the costs of the next step are loaded into registers
// during the current one (two register sets, used in turn), in the form the next step takes:
// each lane its own word (narrow), the lanes' share of one wide window (whole warp), or each
// lane its share of its own line's wide window (dense).
//
// Each direction writes its path costs L (<= census bits + P2 <= 255) as bytes into its own
// ragged volume; the selection sums the directions.
#pragma once

#include "tsgm_kernels.cuh"

namespace tsgm {
namespace dev {

constexpr int kGPadL = 16, kGPadR = 16;  // +inf labels before and after a state row
constexpr int kGBlk = 8;                 // steps per descriptor block (4 blocks in the ring)
constexpr int kGFix = 64;                // steps a segment is walked again before the check

// labels of the wide (whole-warp) form: LPLW per lane, >= D
template <int LPLW>
__host__ __device__ constexpr int grp_dp() { return 32 * LPLW; }
// 16-bit entries of one state row
template <int LPLW>
__host__ __device__ constexpr int grp_row() { return kGPadL + grp_dp<LPLW>() + kGPadR; }
// shared memory of one warp in 32-bit words, for NG lines: state rows (2 per line), checkpoints
// (one wide state and two narrow states, 4 (32 / NG) labels, per line), descriptor ring (4 blocks)
template <int LPLW, int NG>
__host__ __device__ constexpr int grp_words_ng() {
    return NG * (grp_row<LPLW>() + 32) + NG * grp_dp<LPLW>() / 2 + 2 * 4 * 32 / 2 +
           4 * kGBlk * NG * 2;
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

// NG / S lines of direction `code`, lines first_line .. (those < nlines), S segments each (S
// divides NG; the caller keeps every line at least 16 S steps long when S > 1), one group of GL
// lanes per segment: group g walks segment g % S of line first_line + g / S. Lv: the direction's
// volume; wsm: this warp's shared memory (grp_words_ng<LPLW, NG>).
template <int LPLW, int GL>
__device__ __forceinline__ void sgm_group_lines(const uint8_t* __restrict__ C,
                                                const uint2* __restrict__ desc, int W, int Hh,
                                                int P1, int P2, int code, int first_line,
                                                int nlines, int S, uint8_t* __restrict__ Lv,
                                                uint32_t* const wsm) {
    static_assert(GL == 4 || GL == 8, "lanes per line");
    static_assert(LPLW == 2 || LPLW == 4 || LPLW == 8, "labels per lane of the wide form");
    constexpr int NG = 32 / GL;
    constexpr int CAPN = 4 * GL;          // labels of the narrow form
    constexpr int DP = grp_dp<LPLW>();    // labels of the wide form
    constexpr int ROW = grp_row<LPLW>();  // entries of a state row
    constexpr int CKW = DP / 2;           // words of a checkpoint
    constexpr int PER = kGBlk / GL;       // descriptors each lane loads per block
    constexpr int LPD = DP / GL;          // labels per lane of the dense step
    constexpr int NWD = LPD / 4;          // its cost words
    constexpr int NWC = LPLW >= 4 ? LPLW / 4 : 1;  // cost words per lane of the whole-warp step
    static_assert(CAPN + 16 <= DP + kGPadR, "narrow padding inside the row");
    static_assert(4 * kGBlk == 32 && PER >= 1, "the descriptor ring index is a mask");
    const int lane = threadIdx.x & 31;
    const int g = lane / GL, j = lane % GL;
    const unsigned gmask = ((1u << GL) - 1u) << (g * GL);

    // shared memory of this group, by word index into wsm: two state rows (bank-skewed),
    // checkpoint, descriptor ring column (entry s at word dcol + 2 NG (s & 31))
    const int rowA = grp_row_base<LPLW, NG>(g);
    const int rowB = rowA + ROW / 2;
    uint32_t* const ckpt = wsm + NG * (ROW + 32) + g * CKW;  // the last check's (any window)
    uint32_t* const ckn0 = wsm + NG * (ROW + 32) + NG * CKW + g * (CAPN / 2);  // the narrow ones
    uint32_t* const ckn1 = ckn0 + NG * (CAPN / 2);
    const int dcol0 = NG * (ROW + 32) + NG * CKW + 2 * NG * (CAPN / 2);  // the ring
    const int dcol = dcol0 + 2 * g;
    uint2* const dcol_g = reinterpret_cast<uint2*>(wsm + dcol);

    const int li = first_line + g / S, sg = g % S;
    int i0 = 0, stp = 0, llen = 0;
    if (li < nlines) line_geometry(code, li, W, Hh, i0, stp, llen);
    // segment 0 is the shortest, so that every later one ends at the same step; a line too short
    // to cut (a diagonal near a corner) is walked whole by its first group
    int slen = llen, p0 = i0;
    if (S > 1 && llen > 0) {
        if (llen >= 16 * S) {
            const int Lseg = (llen + S - 1) / S, len0 = llen - (S - 1) * Lseg;
            slen = sg == 0 ? len0 : Lseg;
            p0 = i0 + (sg == 0 ? 0 : len0 + (sg - 1) * Lseg) * stp;
        } else if (sg > 0) {
            slen = 0;
        }
    }
    const int maxslen = (int)__reduce_max_sync(kFull, (unsigned)slen);
    if (maxslen == 0) return;
    // the steps before which a later segment's state is saved (first walk) or compared (again);
    // the last (kc2) may coincide with the others in a short segment, and then wins
    const bool later = S > 1 && sg > 0 && slen > 0;
    const int kc0 = later ? min(16, slen) : -1, kc2 = later ? min(kGFix, slen) : -1;
    static_assert(kGFix <= 64, "check steps 16 .. kGFix as bits k - 1 of one word");
    // the steps at which some group of the warp checks (bit k - 1), so that a step tests a
    // register instead of voting
    uint64_t cbits =
        later ? (1ull << (kc0 - 1)) | (1ull << (min(32, slen) - 1)) | (1ull << (kc2 - 1)) : 0ull;
    cbits = ((uint64_t)__reduce_or_sync(kFull, (unsigned)(cbits >> 32)) << 32) |
            (uint64_t)__reduce_or_sync(kFull, (unsigned)cbits);

    for (int t = lane; t < NG * (ROW + 32); t += 32) wsm[t] = kInf2;
    // every ring entry holds a valid descriptor at all times (an empty window until written), so
    // that the descriptor reads and the cost loads they address need no guard
    for (int t = lane; t < 4 * kGBlk * NG * 2; t += 32) wsm[dcol0 + t] = 0u;
    __syncwarp();  // before any lane's copies land in the ring

    auto load_block = [&](int b) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int s = b * kGBlk + j * PER + q;
            if (s < slen) cp_async8(dcol_g + (s & 31) * NG, desc + (p0 + s * stp));
        }
        cp_async_commit();
    };
    // (entries past the walk hold stale but valid descriptors; what they feed is not stored)
    auto dread = [&](int s) -> uint2 {
        return *reinterpret_cast<const uint2*>(wsm + dcol + 2 * NG * (s & 31));
    };

    const uint32_t P1x2 = ((uint32_t)P1 << 16) | (uint32_t)P1;
    // predecessor of a first step: all +inf, m = 0 and no P2 term, so that L = C
    int lo_old = 0, w_old = 0, cap_old = 0;  // the state's window and its row's labels
    int mm = 0, mP = 0;                      // m and m + P2 of the state
    int prow = rowA;                         // the predecessor of the next step (word index)
    int nrow = rowB;                         // the row the next step writes
    // the windows of the three checkpoints, lo << 16 | w (w = 0xFFFF: a state too wide to save)
    int ckw2 = 0, ckw0 = 0, ckw1 = 0;
    bool walker = slen > 0;  // this group walks in the current pass

    // costs of a step, in the form the step takes (two sets, used in turn)
    uint32_t cn[2], cw[2][NWC], cd[2][NWD];
    // load the costs of a step whose descriptor is dsc (this lane's group) and whose wide vote is
    // wb (lanes GL g of the wide groups) into set q
    // (every load is unconditional, from the cost word itself or, past the window, from C[0]:
    // the value is masked later, and no instruction waits on a load in the step that issues it)
    auto fetch = [&](int q, uint2 dsc, unsigned wb) {
        const int w_ = (int)(dsc.y >> 16);
        const uint32_t* const C32 = reinterpret_cast<const uint32_t*>(C);
        const int nwide = __popc(wb);
        if (nwide >= 2) {
#pragma unroll
            for (int i = 0; i < NWD; ++i) {
                const int t = LPD * j + 4 * i;
                cd[q][i] = __ldg(C32 + (t < w_ ? (dsc.x + t) >> 2 : 0u));
            }
        } else {
            cn[q] = __ldg(C32 + (4 * j < w_ ? (dsc.x >> 2) + j : 0u));
            if (nwide == 1) {
                const int src = __ffs(wb) - 1;
                const unsigned o_g = __shfl_sync(kFull, dsc.x, src);
                const int w_g = (int)(__shfl_sync(kFull, dsc.y, src) >> 16);
                if constexpr (LPLW == 2) {
                    const uint16_t* const C16 = reinterpret_cast<const uint16_t*>(C);
                    cw[q][0] = (uint32_t)__ldg(C16 + (2 * lane < w_g ? (o_g >> 1) + lane : 0u));
                } else {
#pragma unroll
                    for (int i = 0; i < NWC; ++i) {
                        const int t = LPLW * lane + 4 * i;
                        cw[q][i] = __ldg(C32 + (t < w_g ? (o_g + t) >> 2 : 0u));
                    }
                }
            }
        }
    };

    // narrow step of this group's line: lane j's labels lo + 4j .. lo + 4j + 3 as two packed
    // 16-bit pairs (computed everywhere; stored and taken as the new state where `keep`)
    auto narrow = [&](uint2 ds, uint32_t cwd, bool keep) {
        const int lo = (int)(ds.y & 0xFFFFu), w = (int)(ds.y >> 16);
        const int e = min(max(lo - lo_old + 4 * j - 1, -6), cap_old);
        const int ea = kGPadL + e;  // entry e of the predecessor row
        const uint32_t* const r32 = wsm + prow + (ea >> 1);
        const uint32_t sh = (uint32_t)(ea & 1) << 4;
        const uint32_t w0 = r32[0], w1 = r32[1], w2 = r32[2], w3 = r32[3];
        // predecessor entries e .. e + 5 as three pairs
        const uint32_t q0 = __funnelshift_r(w0, w1, sh), q1 = __funnelshift_r(w1, w2, sh),
                       q2 = __funnelshift_r(w2, w3, sh);
        const uint32_t mm2 = (uint32_t)mm * 0x10001u, mP2 = (uint32_t)mP * 0x10001u;
        const int rem = w - 4 * j;
        const uint32_t k0 = pair_keep(rem), k1 = pair_keep(rem - 2);
        const uint32_t v0 = (__byte_perm(cwd, 0u, 0x4140) + grp_t(q0, q1, P1x2, mP2)) - mm2;
        const uint32_t v1 = (__byte_perm(cwd, 0u, 0x4342) + grp_t(q1, q2, P1x2, mP2)) - mm2;
        const uint32_t pk0 = (v0 & k0) | (kInf2 & ~k0), pk1 = (v1 & k1) | (kInf2 & ~k1);
        const uint32_t pm = vmin2(pk0, pk1);
        int m = (int)min(pm & 0xFFFFu, pm >> 16);
#pragma unroll
        for (int t = 1; t < GL; t <<= 1) m = min(m, __shfl_xor_sync(kFull, m, t));
        if (keep) {
            uint32_t* const rw = wsm + nrow + kGPadL / 2 + 2 * j;
            rw[0] = pk0;
            rw[1] = pk1;
            if (GL == 4 || j < 4) {
                rw[CAPN / 2] = kInf2;
                rw[CAPN / 2 + 1] = kInf2;
            }
            if (rem > 0) *reinterpret_cast<uint32_t*>(Lv + ds.x + 4 * j) = __byte_perm(pk0, pk1, 0x6420);
            lo_old = lo;
            w_old = w;
            cap_old = CAPN;
            mm = m;
            mP = m + P2;
        }
    };

    for (int pass = 0;; ++pass) {
        load_block(0);
        cp_async_wait<0>();
        __syncwarp();
        load_block(1);
        bool stop = false;     // the walk of this pass ended at a check (the states agreed)
        bool changed = false;  // this pass changed the segment's end state
        // the step the warp's walk ends at: every segment's end in the first walk; in a walk
        // again the end of the segments still walking, updated at every check
        int kend = pass == 0 ? maxslen : (int)__reduce_max_sync(kFull, walker ? (unsigned)slen : 0u);
        // the pipeline: step k's descriptor (dcur) and wide vote (wcur) are known one step ahead,
        // its costs were loaded during step k - 1
        uint2 dcur = dread(0);
        unsigned wcur = __ballot_sync(kFull, walker && (int)(dcur.y >> 16) > CAPN && j == 0);
        fetch(0, dcur, wcur);

        // one step; q: the cost set of this step (the next step's costs go to the other set)
        auto step = [&](int k, int q) -> bool {
            if (k >= 1 && k <= 64 && ((cbits >> (k - 1)) & 1ull)) {
                const bool at = walker && !stop && (k == kc0 || k == min(32, slen) || k == kc2);
                // a check: save the state (first walk) or compare with it; the state is L over
                // the window (lo, w), entries past w are +inf in every row. The rows of the last
                // step were written by other lanes: synchronise first.
                __syncwarp();
                const int ci = k == kc2 ? 2 : (k == min(32, slen) ? 1 : 0);
                uint32_t* const ck = ci == 2 ? ckpt : (ci == 1 ? ckn1 : ckn0);
                const int cap = ci == 2 ? DP : CAPN;  // a wider state is never equal here
                const int cwin = ci == 2 ? ckw2 : (ci == 1 ? ckw1 : ckw0);
                const bool fits = w_old <= cap;
                bool eq = cwin == ((lo_old << 16) | w_old) && fits;
                const uint32_t* const pr = wsm + prow;
                if (at && fits) {
                    for (int t = j; t < (w_old + 1) / 2; t += GL) {
                        const uint32_t v = pr[kGPadL / 2 + t];
                        if (pass == 0) ck[t] = v;
                        else eq = eq && ck[t] == v;
                    }
                }
                const bool same = (__ballot_sync(kFull, !eq) & gmask) == 0u;
                // the first walk saves; a walk again stops where the states agree, and where
                // they differ goes on and rewrites the values after this step: they now follow
                // this state, so it becomes the reference of the next comparison
                const bool save = at && (pass == 0 || !same);
                if (at && pass > 0) {
                    stop = same;
                    changed = !same && ci == 2;
                    if (!same && fits)
                        for (int t = j; t < (w_old + 1) / 2; t += GL) ck[t] = pr[kGPadL / 2 + t];
                }
                if (save) {
                    const int nwin = (lo_old << 16) | (fits ? w_old : 0xFFFF);
                    if (ci == 2) ckw2 = nwin;
                    else if (ci == 1) ckw1 = nwin;
                    else ckw0 = nwin;
                }
                if (pass > 0) kend = (int)__reduce_max_sync(kFull, (walker && !stop) ? (unsigned)slen : 0u);
            }
            if (k >= kend) return false;
            const bool go = walker && !stop && k < slen;
            const uint2 ds = dcur;
            // voted a step ahead (a line whose walk stops at this step's check may still be in
            // it: its wide step then recomputes the values it already holds, which is harmless)
            const unsigned wb0 = wcur;
            // descriptor blocks: block b + 1 (requested at step 8 (b - 1)) is complete at step
            // 8 b, when block b + 2 is requested; the next step's descriptor is in block b or b + 1
            if ((k & (kGBlk - 1)) == 0) {
                cp_async_wait<0>();
                __syncwarp();
                load_block(k / kGBlk + 2);
            } else {
                __syncwarp();  // the rows of the last step are visible
            }
            // the next step's descriptor now; its wide vote and cost loads after this step's
            // work, so that neither waits in front of it
            const bool nxt = walker && !stop && k + 1 < slen;
            dcur = dread(k + 1);

            if (wb0 == 0u) {
                narrow(ds, cn[q], go);
            } else if (__popc(wb0) >= 2) {
                // ---- dense step: every group its own window with its own lanes, LPD labels per
                // lane, in chunks of 8 (several wide windows at once: the full-range band at the
                // image border, a full-range frame)
                const int lo = (int)(ds.y & 0xFFFFu), w = (int)(ds.y >> 16);
                const uint32_t mm2 = (uint32_t)mm * 0x10001u, mP2 = (uint32_t)mP * 0x10001u;
                const uint32_t* const pr = wsm + prow;
                uint32_t* const nr = wsm + nrow;
                uint32_t pm = kInf2;
#pragma unroll
                for (int c = 0; c < LPD / 8; ++c) {
                    const int base = LPD * j + 8 * c;  // first label of the chunk, from lo
                    const int e = min(max(lo - lo_old + base - 1, -10), cap_old);
                    const int b = kGPadL + e;
                    const uint32_t* r32 = pr + (b >> 1);
                    const uint32_t sel = (b & 1) ? 0x5432u : 0x3210u;
                    uint32_t wv[6], A[5];
#pragma unroll
                    for (int i = 0; i < 6; ++i) wv[i] = r32[i];
#pragma unroll
                    for (int i = 0; i < 5; ++i) A[i] = __byte_perm(wv[i], wv[i + 1], sel);
                    const uint32_t c4a = cd[q][2 * c], c4b = cd[q][2 * c + 1];
                    const uint32_t cp[4] = {__byte_perm(c4a, 0u, 0x4140), __byte_perm(c4a, 0u, 0x4342),
                                            __byte_perm(c4b, 0u, 0x4140), __byte_perm(c4b, 0u, 0x4342)};
                    const int rem = w - base;
                    uint32_t Lc[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint32_t kp = pair_keep(rem - 2 * i);
                        const uint32_t v = (cp[i] + grp_t(A[i], A[i + 1], P1x2, mP2)) - mm2;
                        Lc[i] = (v & kp) | (kInf2 & ~kp);
                        pm = vmin2(pm, Lc[i]);
                    }
                    if (go) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) nr[kGPadL / 2 + base / 2 + i] = Lc[i];
                        if (rem > 0)
                            *reinterpret_cast<uint32_t*>(Lv + ds.x + base) = __byte_perm(Lc[0], Lc[1], 0x6420);
                        if (rem > 4)
                            *reinterpret_cast<uint32_t*>(Lv + ds.x + base + 4) =
                                __byte_perm(Lc[2], Lc[3], 0x6420);
                    }
                }
                int m = (int)min(pm & 0xFFFFu, pm >> 16);
#pragma unroll
                for (int t = 1; t < GL; t <<= 1) m = min(m, __shfl_xor_sync(kFull, m, t));
                if (go) {
                    lo_old = lo;
                    w_old = w;
                    cap_old = DP;
                    mm = m;
                    mP = m + P2;
                }
            } else {
                // ---- one wide window: the other lines' narrow steps, then the whole warp ----
                const int w = (int)(ds.y >> 16);
                narrow(ds, cn[q], go && w <= CAPN);
                const int src = __ffs(wb0) - 1;
                const int gg = src / GL;
                const int lo_g = (int)(__shfl_sync(kFull, ds.y, src) & 0xFFFFu);
                const int w_g = (int)(__shfl_sync(kFull, ds.y, src) >> 16);
                const uint32_t o_g = __shfl_sync(kFull, ds.x, src);
                const int lo_old_g = __shfl_sync(kFull, lo_old, src);
                const int cap_old_g = __shfl_sync(kFull, cap_old, src);
                const uint32_t mm2_g = (uint32_t)__shfl_sync(kFull, mm, src) * 0x10001u;
                const uint32_t mP2_g = (uint32_t)__shfl_sync(kFull, mP, src) * 0x10001u;
                const uint32_t* const rold = wsm + __shfl_sync(kFull, prow, src);
                uint32_t* const rnew = wsm + __shfl_sync(kFull, nrow, src);
                constexpr int NPW = LPLW / 2;  // packed pairs per lane
                const int e2 = min(max(lo_g - lo_old_g + LPLW * lane - 1, -(LPLW + 2)), cap_old_g);
                const int b2 = kGPadL + e2;
                const uint32_t* q32 = rold + (b2 >> 1);
                const uint32_t sel2 = (b2 & 1) ? 0x5432u : 0x3210u;
                uint32_t wv[NPW + 2], A[NPW + 1];
#pragma unroll
                for (int i = 0; i < NPW + 2; ++i) wv[i] = q32[i];
#pragma unroll
                for (int i = 0; i < NPW + 1; ++i) A[i] = __byte_perm(wv[i], wv[i + 1], sel2);
                uint32_t cpk[NPW];
                if constexpr (LPLW == 2) {
                    cpk[0] = __byte_perm(cw[q][0], 0u, 0x4140);
                } else {
#pragma unroll
                    for (int i = 0; i < NWC; ++i) {
                        cpk[2 * i] = __byte_perm(cw[q][i], 0u, 0x4140);
                        cpk[2 * i + 1] = __byte_perm(cw[q][i], 0u, 0x4342);
                    }
                }
                const int rem2 = w_g - LPLW * lane;
                uint32_t Lw[NPW];
                uint32_t pw2 = kInf2;
#pragma unroll
                for (int i = 0; i < NPW; ++i) {
                    const uint32_t kp = pair_keep(rem2 - 2 * i);
                    const uint32_t v = (cpk[i] + grp_t(A[i], A[i + 1], P1x2, mP2_g)) - mm2_g;
                    Lw[i] = (v & kp) | (kInf2 & ~kp);
                    pw2 = vmin2(pw2, Lw[i]);
                }
                const int mg = (int)__reduce_min_sync(kFull, min(pw2 & 0xFFFFu, pw2 >> 16));
                uint32_t* const dst = rnew + kGPadL / 2 + LPLW * lane / 2;
#pragma unroll
                for (int i = 0; i < NPW; ++i) dst[i] = Lw[i];
                if constexpr (LPLW == 2) {
                    if (rem2 > 0)
                        *reinterpret_cast<uint16_t*>(Lv + o_g + 2 * lane) =
                            (uint16_t)__byte_perm(Lw[0], 0u, 0x0020);
                } else {
#pragma unroll
                    for (int i = 0; i < NWC; ++i)
                        if (rem2 > 4 * i)
                            *reinterpret_cast<uint32_t*>(Lv + o_g + LPLW * lane + 4 * i) =
                                __byte_perm(Lw[2 * i], Lw[2 * i + 1], 0x6420);
                }
                if (g == gg) {
                    lo_old = lo_g;
                    w_old = w_g;
                    cap_old = DP;
                    mm = mg;
                    mP = mg + P2;
                }
            }
            wcur = __ballot_sync(kFull, nxt && (int)(dcur.y >> 16) > CAPN && j == 0);
            fetch(q ^ 1, dcur, wcur);
            if (go) {
                const int t = nrow;
                nrow = (prow == rowA || prow == rowB) ? prow : (nrow == rowA ? rowB : rowA);
                prow = t;
            }
            return true;
        };
        for (int k = 0;; k += 2) {
            if (!step(k, 0)) break;
            if (!step(k + 1, 1)) break;
        }
        cp_async_wait<0>();
        __syncwarp();
        // the next pass: the later segments (first walk done), then every segment whose
        // predecessor's end state changed in this pass, from that end state
        const int src = (sg > 0 ? g - 1 : g) * GL;
        const bool pchanged = __shfl_sync(kFull, (int)changed, src) != 0;
        const int plo = __shfl_sync(kFull, lo_old, src), pcap = __shfl_sync(kFull, cap_old, src);
        const int pwid = __shfl_sync(kFull, w_old, src);
        const int pmm = __shfl_sync(kFull, mm, src), pmP = __shfl_sync(kFull, mP, src);
        const int pprow = __shfl_sync(kFull, prow, src);
        walker = sg > 0 && slen > 0 && (pass == 0 || pchanged);
        if (!__any_sync(kFull, walker)) break;
        if (walker) {
            lo_old = plo;
            w_old = pwid;
            cap_old = pcap;
            mm = pmm;
            mP = pmP;
            // the first step reads the predecessor's row and writes the row of this group that
            // does not hold its end state: the next segment, walking again in the same pass, may
            // read that end state in this same step
            nrow = prow == rowA ? rowB : rowA;
            prow = pprow;
        }
    }
}

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

// Cost ring of the full-range walker: kFullRing steps of one pixel's cost slice each (32 LPLW
// bytes, the slice's layout in the volume), copied in blocks of kFullBlk steps, kFullAhead blocks
// ahead of the walk (the block a copy overwrites was read in the iteration before).
constexpr int kFullBlk = 4;
constexpr int kFullRing = 16;
constexpr int kFullAhead = 3;
static_assert(kFullRing == (kFullAhead + 1) * kFullBlk, "ring of the blocks in flight + the one read");

// One path line whose windows are all the full range [0, D - 1] (a first frame, or the
// full-range mode: known before the launch), one warp, lane j holding labels LPLW j .. LPLW j +
// LPLW - 1 of the state in registers as packed 16-bit pairs: the neighbours d - 1 and d + 1 across
// lanes come by shuffle, m by redux.sync (on the lane minimum held in both halves, so that the
// result is m in both halves). Labels from D on are +inf. Same recurrence and first step (L = C)
// as sgm_group_lines.
// The costs of a step (pixel i's block of rD = D rounded up to 4 cells, at cell i rD) reach the
// ring by cp.async, kFullAhead blocks of kFullBlk steps ahead, so that a long line is not bound
// by the load latency: with V16 (rD = 32 LPLW, a multiple of 16 bytes) in 16-byte pieces of the
// block's slices spread over the lanes, else each lane copies the 4-byte words of its labels.
// EXACT: D = 32 LPLW (no label of any lane past the range). ring: this warp's kFullRing * 8 * LPLW
// words of shared memory.
template <int LPLW, bool V16, bool EXACT>
__device__ __forceinline__ void sgm_full_line(const uint8_t* __restrict__ C, int W, int Hh, int D,
                                              int rD, int P1, int P2, int code, int line,
                                              uint8_t* __restrict__ Lv, uint32_t* const ring) {
    static_assert(LPLW == 2 || LPLW == 4 || LPLW == 8, "labels per lane");
    constexpr int NP = LPLW / 2;          // packed pairs per lane
    constexpr int SLOT = 32 * LPLW;       // bytes of a ring slot
    constexpr int NCH = kFullBlk * SLOT / 16;  // 16-byte pieces of a block
    const int lane = threadIdx.x & 31;
    int i0 = 0, stp = 0, len = 0;
    line_geometry(code, line, W, Hh, i0, stp, len);
    const int base = LPLW * lane;  // this lane's first label
    uint32_t kp[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) kp[k] = EXACT ? 0xFFFFFFFFu : pair_keep(D - (base + 2 * k));
    const uint32_t P1x2 = ((uint32_t)P1 << 16) | (uint32_t)P1;
    const uint32_t P2x2 = ((uint32_t)P2 << 16) | (uint32_t)P2;
    uint8_t* const ring8 = reinterpret_cast<uint8_t*>(ring);

    // copies of block b (steps kFullBlk b ..) into ring slots (kFullBlk b ..) mod kFullRing
    auto issue = [&](int b) {
        if constexpr (V16) {
#pragma unroll
            for (int r = 0; r < (NCH + 31) / 32; ++r) {
                const int c = lane + 32 * r;
                const int q = c / (SLOT / 16), o = 16 * (c % (SLOT / 16));
                const int s = kFullBlk * b + q;
                if ((NCH % 32 == 0 || c < NCH) && s < len)
                    cp_async16(ring8 + (s & (kFullRing - 1)) * SLOT + o,
                               C + (size_t)(i0 + s * stp) * rD + o);
            }
        } else {
            // the 4-byte words of this lane's labels (one word of two lanes when LPLW = 2)
            const int wb = LPLW == 2 ? 4 * (lane >> 1) : base;
            const bool owner = LPLW != 2 || (lane & 1) == 0;
#pragma unroll
            for (int q = 0; q < kFullBlk; ++q) {
                const int s = kFullBlk * b + q;
                if (s < len && owner) {
#pragma unroll
                    for (int g = 0; g < (LPLW == 8 ? 2 : 1); ++g)
                        if (wb + 4 * g < D)
                            cp_async4(ring8 + (s & (kFullRing - 1)) * SLOT + wb + 4 * g,
                                      C + (size_t)(i0 + s * stp) * rD + wb + 4 * g);
                }
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int b = 0; b < kFullAhead; ++b) issue(b);

    uint32_t P[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) P[k] = kInf2;
    uint32_t mm2 = 0u, mP2 = 0u;  // a first step: no predecessor, L = C
    const bool live = EXACT || base < D;
    // step s: costs from ring slot s mod kFullRing, result to pixel i0 + s stp
    auto step = [&](int s) {
        const uint8_t* const sl = ring8 + (s & (kFullRing - 1)) * SLOT + base;
        uint32_t cp[NP];
        if constexpr (LPLW == 2) {
            cp[0] = __byte_perm((uint32_t)*reinterpret_cast<const uint16_t*>(sl), 0u, 0x4140);
        } else {
#pragma unroll
            for (int g = 0; g < LPLW / 4; ++g) {
                const uint32_t w = reinterpret_cast<const uint32_t*>(sl)[g];
                cp[2 * g] = __byte_perm(w, 0u, 0x4140);
                cp[2 * g + 1] = __byte_perm(w, 0u, 0x4342);
            }
        }
        uint32_t up = __shfl_up_sync(kFull, P[NP - 1], 1);
        uint32_t dn = __shfl_down_sync(kFull, P[0], 1);
        if (lane == 0) up = kInf2;
        if (lane == 31) dn = kInf2;
        // X[k]: the pair (label base + 2k - 1, base + 2k) of the predecessor
        uint32_t X[NP + 1];
        X[0] = __byte_perm(up, P[0], 0x5432);
#pragma unroll
        for (int k = 1; k < NP; ++k) X[k] = __byte_perm(P[k - 1], P[k], 0x5432);
        X[NP] = __byte_perm(P[NP - 1], dn, 0x5432);
        uint32_t pm = 0u;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            // as grp_t, with the pair (L(d), L(d + 1)) taken from P[k] itself
            const uint32_t t = vmin2(vmin2(vmin2(X[k], X[k + 1]) + P1x2, P[k]), mP2);
            const uint32_t v = (cp[k] + t) - mm2;
            P[k] = EXACT ? v : (v & kp[k]) | (kInf2 & ~kp[k]);
            pm = k == 0 ? P[0] : vmin2(pm, P[k]);
        }
        // the lane's minimum in both halves, then the warp's: m in both halves
        mm2 = __reduce_min_sync(kFull, vmin2(pm, __byte_perm(pm, 0u, 0x1032)));
        mP2 = mm2 + P2x2;
        if (live) {
            uint8_t* const dst = Lv + (size_t)(unsigned)(i0 + s * stp) * (unsigned)rD + base;
            if constexpr (LPLW == 2) {
                *reinterpret_cast<uint16_t*>(dst) = (uint16_t)__byte_perm(P[0], 0u, 0x0020);
            } else {
#pragma unroll
                for (int g = 0; g < LPLW / 4; ++g)
                    if (EXACT || base + 4 * g < D)
                        reinterpret_cast<uint32_t*>(dst)[g] = __byte_perm(P[2 * g], P[2 * g + 1], 0x6420);
            }
        }
    };
    const int nfull = len / kFullBlk;
    for (int b = 0; b < nfull; ++b) {
        cp_async_wait<kFullAhead - 1>();  // block b (the oldest in flight) has landed
        __syncwarp();                     // ... for every lane (pieces copied by other lanes)
        issue(b + kFullAhead);
#pragma unroll
        for (int q = 0; q < kFullBlk; ++q) step(kFullBlk * b + q);
    }
    if (nfull * kFullBlk < len) {
        cp_async_wait<kFullAhead - 1>();
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kFullBlk; ++q)
            if (kFullBlk * nfull + q < len) step(kFullBlk * nfull + q);
    }
    cp_async_wait<0>();
}

// Lines of one image for the grouped walker: direction codes in launch order (horizontal pairs
// first: the longest chains) and their line counts.
struct GrpLines {
    int code[8];
    int count[8];
    int seg[8];  // segments per line (a power of two; the kernel takes at most its groups)
    int nslots;
};

// Segments per line for lines of up to `len` steps: as many (a power of two, at most 8) as keep
// every segment at least kGSegMin steps long, so that the longest chain of the launch, a segment
// plus its second walk, is short.
constexpr int kGSegMin = 64;
__host__ __device__ __forceinline__ int grp_seg(int len) {
    int S = 1;
    while (S < 8 && len >= 2 * S * kGSegMin) S *= 2;
    return S;
}

// Segments per line of slot s for NG groups per warp: at most NG; with 8-lane groups (NG = 4,
// the form of images with many wide windows, e.g. a full-range frame) only the horizontal lines
// are cut, so that the launch stays one wave of warps.
__host__ __device__ __forceinline__ int grp_slot_seg(const GrpLines& L, int s, int NG) {
    const int S = L.seg[s] < NG ? L.seg[s] : NG;
    return (NG == 4 && L.code[s] > 1) ? 1 : S;
}

// Map warp gw of the launch to (direction code, first line, line count, segments) for NG groups
// per warp (NG / seg lines); false when gw is past the last line.
__device__ __forceinline__ bool grp_warp_lines(const GrpLines& L, int NG, int gw, int& code,
                                               int& first, int& nlines, int& seg) {
    int base = 0;
    for (int s = 0; s < L.nslots; ++s) {
        const int per = NG / grp_slot_seg(L, s, NG);
        const int nw = (L.count[s] + per - 1) / per;
        if (gw < base + nw) {
            code = L.code[s];
            first = (gw - base) * per;
            nlines = L.count[s];
            seg = grp_slot_seg(L, s, NG);
            return true;
        }
        base += nw;
    }
    return false;
}

}  // namespace dev
}  // namespace tsgm
