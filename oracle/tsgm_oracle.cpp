// Plain, slow, obviously-correct CPU oracle of the ego-motion-reduced SGM hot path
// (Fucek, Markovic, Cvisic, Petrovic, "Dense Disparity Estimation in Ego-motion Reduced
// Search Space", arXiv 1708.06301).
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls this file; only
// the tests, the smoke check and the benchmark's CPU-baseline leg do. It shares no code, header,
// table or constant generator with the CUDA library.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fPIC -shared (no SIMD intrinsics, no -ffast-math).
//
// Precision: the paper fixes none. Every float quantity whose value later decides an integer
// (warp target pixel, z-buffer order, window bounds, and the Kalman output that the next frame
// warps) is computed in IEEE binary32 with the operation order written below and no contraction,
// which is the precision of the GPU kernels; the disparity-space homography is built in binary64
// and rounded to binary32 once. Each such function is pinned by the tests against a binary64
// closed form or a geometric construction within a stated bound.
//
// Conventions shared with the rest of the project (they are readings of the paper, not code):
//   * maps are dense row-major W x H, pixel index i = y*W + x;
//   * an invalid disparity or variance is stored as -1.0f;
//   * a window is [lo, hi] (inclusive, int16) inside [0, D-1]; the ragged volume stores the
//     cells of pixel i at off[i] .. off[i+1]-1, cell j <-> disparity lo[i] + j.
//
// Parity status: every function below is pinned by a `-m "not gpu"` test (tests/test_oracle_pins.py),
// and tests/test_oracle_mutants.py checks that a planted mistake in any of them fails a pin.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cfloat>
#include <vector>
#include <algorithm>

extern "C" {

// ------------------------------------------------------------------------------------------
// Eq. 1-4 (Sec. 2.1, "Disparity space"): H = Gamma T Gamma^{-1}.
// Gamma maps homogeneous Euclidean M = (X,Y,Z,1) to disparity space (fX, fY, fb, Z) ~ (x,y,d,1).
// T = [R t; 0 1] maps previous-frame camera coordinates to current ones (Eq. 2, M^k = T M^{k-1}).
// x, y are measured from the principal point. Inputs R (row-major 3x3), t, f, b; output H
// row-major 4x4 in binary64.
// ------------------------------------------------------------------------------------------
void oracle_build_H(const double* R, const double* t, double f, double b, double* H) {
    double G[4][4] = {{f, 0, 0, 0}, {0, f, 0, 0}, {0, 0, 0, f * b}, {0, 0, 1, 0}};
    // Gamma^{-1}: (a0,a1,a2,a3) -> (a0/f, a1/f, a3, a2/(f b)), written out from Eq. 1
    double Gi[4][4] = {{1.0 / f, 0, 0, 0}, {0, 1.0 / f, 0, 0}, {0, 0, 0, 1}, {0, 0, 1.0 / (f * b), 0}};
    double T[4][4] = {{R[0], R[1], R[2], t[0]},
                      {R[3], R[4], R[5], t[1]},
                      {R[6], R[7], R[8], t[2]},
                      {0, 0, 0, 1}};
    double TG[4][4];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += T[r][k] * Gi[k][c];
            TG[r][c] = s;
        }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += G[r][k] * TG[k][c];
            H[r * 4 + c] = s;
        }
}

static inline bool finite_nonneg(float v) { return v >= 0.0f && v <= FLT_MAX; }

// ------------------------------------------------------------------------------------------
// Sec. 2.2: forward warp of the previous map (Eq. 3 with the homogeneous divide), occlusion
// resolution "keep the highest predicted disparity" (Sec. 2.2, disparity refinement), and the
// variance prediction p = Phi^2 p + q with Phi = d^{k|k-1} / d^{k-1} (Eq. 5-6).
//
// A source pixel (u,v) takes part iff d > 0 and p >= 0 (both finite). With x~ = u - cx,
// y~ = v - cy the transformed point is w = H (x~, y~, d, 1); it is kept iff w3 > 0 and
// d' = w2/w3 > 0, and it lands on target (round(x'+cx), round(y'+cy)) with round(v) =
// floor(v + 0.5), x' = w0/w3, y' = w1/w3, if that pixel is inside the image. Among the sources
// that land on one target the largest d' wins; equal d' go to the lowest source index.
// Targets that nothing reaches are invalid (-1, -1). `winner` receives the source index (or -1).
// ------------------------------------------------------------------------------------------
void oracle_warp_predict(int W, int Hh, const float* Dprev, const float* Pprev, const float* Hm,
                         float cx, float cy, float q, float* Dpred, float* Ppred, int32_t* winner) {
    const int n = W * Hh;
    std::vector<float> best(n, -1.0f);
    std::vector<int32_t> src(n, -1);
    for (int v = 0; v < Hh; ++v) {
        for (int u = 0; u < W; ++u) {
            const int i = v * W + u;
            const float d = Dprev[i], p = Pprev[i];
            if (!(d > 0.0f && d <= FLT_MAX && finite_nonneg(p))) continue;
            const float xt = (float)u - cx;
            const float yt = (float)v - cy;
            float w[4];
            for (int r = 0; r < 4; ++r) {
                const float* h = Hm + 4 * r;
                float a = h[0] * xt;
                float b = h[1] * yt;
                float s = a + b;
                float c = h[2] * d;
                s = s + c;
                s = s + h[3];
                w[r] = s;
            }
            if (!(w[3] > 0.0f)) continue;
            const float xp = w[0] / w[3];
            const float yp = w[1] / w[3];
            const float dp = w[2] / w[3];
            if (!(dp > 0.0f && dp <= FLT_MAX)) continue;
            const float fx = std::floor((xp + cx) + 0.5f);
            const float fy = std::floor((yp + cy) + 0.5f);
            if (!(fx >= 0.0f && fx <= (float)(W - 1) && fy >= 0.0f && fy <= (float)(Hh - 1))) continue;
            const int tgt = (int)fy * W + (int)fx;
            if (dp > best[tgt]) {  // strict: the lowest source index keeps a tie
                best[tgt] = dp;
                src[tgt] = i;
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        if (src[i] < 0) {
            Dpred[i] = -1.0f;
            Ppred[i] = -1.0f;
        } else {
            const float dp = best[i];
            const float phi = dp / Dprev[src[i]];
            const float phi2 = phi * phi;
            const float pp = phi2 * Pprev[src[i]];
            Dpred[i] = dp;
            Ppred[i] = pp + q;
        }
        if (winner) winner[i] = src[i];
    }
}

// ------------------------------------------------------------------------------------------
// Sec. 2.2, Eq. 7-8: filling the gaps that forward motion leaves in the prediction ("zooming").
// An invalid predicted pixel whose two horizontal neighbours are valid and similar,
// |d_{i-1} - d_{i+1}| < gamma_f (f_s of Eq. 8), takes their mean (Eq. 7); then the same with the
// vertical neighbours on the horizontally filled map. Each pass reads the map as it was before
// that pass (a pixel filled in a pass does not serve as a neighbour in the same pass). The variance
// of a filled pixel is the mean of its two neighbours' variances. In place on D, P.
// ------------------------------------------------------------------------------------------
void oracle_fill_gaps(int W, int Hh, float gamma_f, float* D, float* P) {
    const int n = W * Hh;
    std::vector<float> d0(D, D + n), p0(P, P + n);
    for (int pass = 0; pass < 2; ++pass) {
        for (int y = 0; y < Hh; ++y)
            for (int x = 0; x < W; ++x) {
                const int i = y * W + x;
                if (finite_nonneg(d0[i]) && finite_nonneg(p0[i])) continue;
                int a, b;
                if (pass == 0) {
                    if (x == 0 || x == W - 1) continue;
                    a = i - 1;
                    b = i + 1;
                } else {
                    if (y == 0 || y == Hh - 1) continue;
                    a = i - W;
                    b = i + W;
                }
                if (!(finite_nonneg(d0[a]) && finite_nonneg(p0[a]) && finite_nonneg(d0[b]) &&
                      finite_nonneg(p0[b])))
                    continue;
                const float diff = std::fabs(d0[a] - d0[b]);
                if (!(diff < gamma_f)) continue;
                const float ds = d0[a] + d0[b];
                const float ps = p0[a] + p0[b];
                D[i] = ds * 0.5f;
                P[i] = ps * 0.5f;
            }
        std::copy(D, D + n, d0.begin());
        std::copy(P, P + n, p0.begin());
    }
}

// ------------------------------------------------------------------------------------------
// Sec. 2.2, disparity refinement: predicted pixels near a disparity discontinuity are rejected.
// Reading (the paper gives neither the neighbourhood nor the threshold): a valid predicted pixel
// becomes invalid (-1, -1) when one of its 8 neighbours inside the image holds a valid
// prediction whose disparity differs by at least edge_thr (the negation of the similarity of
// Eq. 8); invalid neighbours are holes, not edges. Reads the map as it was before the pass.
// ------------------------------------------------------------------------------------------
void oracle_edge_reject(int W, int Hh, float edge_thr, float* D, float* P) {
    const int n = W * Hh;
    std::vector<float> d0(D, D + n), p0(P, P + n);
    for (int y = 0; y < Hh; ++y)
        for (int x = 0; x < W; ++x) {
            const int i = y * W + x;
            if (!(finite_nonneg(d0[i]) && finite_nonneg(p0[i]))) continue;
            bool edge = false;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    const int xn = x + dx, yn = y + dy;
                    if (xn < 0 || xn >= W || yn < 0 || yn >= Hh) continue;
                    const int j = yn * W + xn;
                    if (!(finite_nonneg(d0[j]) && finite_nonneg(p0[j]))) continue;
                    if (!(std::fabs(d0[i] - d0[j]) < edge_thr)) edge = true;
                }
            if (edge) {
                D[i] = -1.0f;
                P[i] = -1.0f;
            }
        }
}

// ------------------------------------------------------------------------------------------
// Sec. 2.2 and Sec. 3 (Fig. 3(d)): left-right consistency check of the prediction. The right
// view's prediction is formed from the left one: a valid predicted pixel (x, y, d) lands on the
// right view's pixel x_r = x - round(d) of its row, round(d) = floor(d + 1/2) in binary32, and the
// right view keeps the largest disparity landing on each pixel (the nearest surface). A left pixel
// stays valid when x_r lies inside the image and the right prediction there differs from d by at
// most tol; otherwise D and P become -1 (seen by one camera only, or hidden in the right view
// behind a nearer surface). In place.
// ------------------------------------------------------------------------------------------
static inline int right_column(int x, float d) {
    const float rf = std::floor(d + 0.5f);
    return rf > (float)x ? -1 : x - (int)rf;
}

void oracle_pred_lr_check(int W, int Hh, float tol, float* D, float* P) {
    std::vector<float> R(W);
    for (int y = 0; y < Hh; ++y) {
        float* d = D + (size_t)y * W;
        float* p = P + (size_t)y * W;
        for (int x = 0; x < W; ++x) R[x] = -1.0f;
        for (int x = 0; x < W; ++x) {
            if (!(finite_nonneg(d[x]) && finite_nonneg(p[x]))) continue;
            const int r = right_column(x, d[x]);
            if (r >= 0 && d[x] > R[r]) R[r] = d[x];
        }
        for (int x = 0; x < W; ++x) {
            if (!(finite_nonneg(d[x]) && finite_nonneg(p[x]))) continue;
            const int r = right_column(x, d[x]);
            if (!(r >= 0 && std::fabs(d[x] - R[r]) <= tol)) {
                d[x] = -1.0f;
                p[x] = -1.0f;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Sec. 2.4 (disparity consistency check), the SAD check on the left and right images: the sum of
// absolute differences between the sw x sh patch of the left image around (x, y) and the right
// image's patch around (x - round(d), y), every coordinate clamped into the image. A pixel whose
// SAD exceeds sad_thr times the patch area (binary32) is rejected (D = P = -1), so that the next
// image searches it over the whole range. Applied to the updated map, in place.
// ------------------------------------------------------------------------------------------
void oracle_sad_check(int W, int Hh, int sw, int sh, float sad_thr, const uint8_t* L,
                      const uint8_t* R, float* D, float* P) {
    const float lim = sad_thr * (float)(sw * sh);
    const int hw = sw / 2, hh = sh / 2;
    auto clampi = [](int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); };
    for (int y = 0; y < Hh; ++y)
        for (int x = 0; x < W; ++x) {
            const int i = y * W + x;
            if (!(finite_nonneg(D[i]) && finite_nonneg(P[i]))) continue;
            const float rf = std::floor(D[i] + 0.5f);
            const int dx = rf > (float)(2 * W) ? 2 * W : (int)rf;  // beyond the image either way
            int sad = 0;
            for (int v = -hh; v <= hh; ++v)
                for (int u = -hw; u <= hw; ++u) {
                    const int yy = clampi(y + v, 0, Hh - 1);
                    const int xl = clampi(x + u, 0, W - 1);
                    const int xr = clampi(x - dx + u, 0, W - 1);
                    sad += std::abs((int)L[yy * W + xl] - (int)R[yy * W + xr]);
                }
            if ((float)sad > lim) {
                D[i] = -1.0f;
                P[i] = -1.0f;
            }
        }
}

// ------------------------------------------------------------------------------------------
// Sec. 2.3: reduced search interval [d - 3 sqrt(p), d + 3 sqrt(p)] (multiplier k = sigma_mult),
// rounded outwards to integers and clipped to [0, D-1]. A pixel without a valid prediction
// (d < 0, p < 0, NaN or inf), or whose interval misses [0, D-1], is searched over the whole
// range (Sec. 2.4, consistency check; Sec. 3, first frame). Writes lo, hi and the exclusive
// prefix sum off[0..n] of the window lengths; returns the number of cells off[n].
// ------------------------------------------------------------------------------------------
int64_t oracle_windows(int W, int Hh, int D, float sigma_mult, const float* Dp, const float* Pp,
                       int16_t* lo, int16_t* hi, uint32_t* off) {
    const int n = W * Hh;
    uint64_t acc = 0;
    for (int i = 0; i < n; ++i) {
        int a = 0, b = D - 1;
        const float d = Dp[i], p = Pp[i];
        if (finite_nonneg(d) && finite_nonneg(p)) {
            const float s = std::sqrt(p);
            const float r = sigma_mult * s;
            const float lo_f = std::floor(d - r);
            const float hi_f = std::ceil(d + r);
            if (lo_f <= (float)(D - 1) && hi_f >= 0.0f) {
                a = lo_f < 0.0f ? 0 : (int)lo_f;
                b = hi_f > (float)(D - 1) ? D - 1 : (int)hi_f;
            }
        }
        lo[i] = (int16_t)a;
        hi[i] = (int16_t)b;
        off[i] = (uint32_t)acc;
        acc += (uint64_t)(b - a + 1);
    }
    off[n] = (uint32_t)acc;
    return (int64_t)acc;
}

// ------------------------------------------------------------------------------------------
// Matching cost (Sec. 2.3 uses SGM on a matching cost it does not name; census + Hamming):
// census code of p: for every q of the cw x ch window except the centre, in row-major order,
// bit b (LSB first) = [I(q) < I(p)]; coordinates outside the image are clamped to the border.
// ------------------------------------------------------------------------------------------
void oracle_census(int W, int Hh, int cw, int ch, const uint8_t* img, uint64_t* codes) {
    const int rx = cw / 2, ry = ch / 2;
    for (int y = 0; y < Hh; ++y)
        for (int x = 0; x < W; ++x) {
            const uint8_t c = img[y * W + x];
            uint64_t code = 0;
            int bit = 0;
            for (int dy = -ry; dy <= ry; ++dy)
                for (int dx = -rx; dx <= rx; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    int qx = std::min(std::max(x + dx, 0), W - 1);
                    int qy = std::min(std::max(y + dy, 0), Hh - 1);
                    if (img[qy * W + qx] < c) code |= (uint64_t)1 << bit;
                    ++bit;
                }
            codes[y * W + x] = code;
        }
}

static inline int popcount64(uint64_t v) {
    int c = 0;
    while (v) {
        v &= v - 1;
        ++c;
    }
    return c;
}

// C(p,d) = Hamming(cL(x,y), cR(x-d,y)) for d in the window of p; x-d < 0 costs Bc (all bits).
void oracle_cost(int W, int Hh, int Bc, const uint64_t* cl, const uint64_t* cr, const int16_t* lo,
                 const int16_t* hi, const uint32_t* off, uint8_t* C) {
    for (int y = 0; y < Hh; ++y)
        for (int x = 0; x < W; ++x) {
            const int i = y * W + x;
            for (int d = lo[i]; d <= hi[i]; ++d) {
                int c = Bc;
                if (x - d >= 0) c = popcount64(cl[i] ^ cr[y * W + x - d]);
                C[off[i] + (d - lo[i])] = (uint8_t)c;
            }
        }
}

// ------------------------------------------------------------------------------------------
// SGM path aggregation (Sec. 2.3, eight paths, each minimising a 1-D energy that penalises
// disparity changes; Hirschmueller 2008 recursion) restricted to each pixel's window.
// Along direction r, with predecessor q = p - r:
//   L(p,d) = C(p,d) + min( L(q,d), L(q,d-1)+P1, L(q,d+1)+P1, m + P2 ) - m,  m = min_k L(q,k)
// where L(q,.) outside q's window does not exist (treated as +inf) and m runs over q's window.
// The first pixel of a path (q outside the image) has L(p,d) = C(p,d).
// Direction codes: 0 (+1,0)  1 (-1,0)  2 (0,+1)  3 (0,-1)  4 (+1,+1)  5 (-1,-1)  6 (-1,+1)  7 (+1,-1)
// ------------------------------------------------------------------------------------------
static const int kDir[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {-1, 1}, {1, -1}};

void oracle_sgm_path(int W, int Hh, int dir, int P1, int P2, const uint8_t* C, const int16_t* lo,
                     const int16_t* hi, const uint32_t* off, uint16_t* L) {
    const int dx = kDir[dir][0], dy = kDir[dir][1];
    // visit pixels so that every predecessor is done first: rows in the direction of dy,
    // columns in the direction of dx (for dy == 0 the row order is irrelevant).
    const int y0 = dy >= 0 ? 0 : Hh - 1, y1 = dy >= 0 ? Hh : -1, sy = dy >= 0 ? 1 : -1;
    const int x0 = dx >= 0 ? 0 : W - 1, x1 = dx >= 0 ? W : -1, sx = dx >= 0 ? 1 : -1;
    for (int y = y0; y != y1; y += sy)
        for (int x = x0; x != x1; x += sx) {
            const int i = y * W + x;
            const int qx = x - dx, qy = y - dy;
            const bool first = qx < 0 || qx >= W || qy < 0 || qy >= Hh;
            const int j = first ? -1 : qy * W + qx;
            int m = 1 << 30;
            if (!first)
                for (int k = lo[j]; k <= hi[j]; ++k) m = std::min(m, (int)L[off[j] + (k - lo[j])]);
            for (int d = lo[i]; d <= hi[i]; ++d) {
                const int c = C[off[i] + (d - lo[i])];
                if (first) {
                    L[off[i] + (d - lo[i])] = (uint16_t)c;
                    continue;
                }
                int best = m + P2;
                if (d >= lo[j] && d <= hi[j]) best = std::min(best, (int)L[off[j] + (d - lo[j])]);
                if (d - 1 >= lo[j] && d - 1 <= hi[j]) best = std::min(best, (int)L[off[j] + (d - 1 - lo[j])] + P1);
                if (d + 1 >= lo[j] && d + 1 <= hi[j]) best = std::min(best, (int)L[off[j] + (d + 1 - lo[j])] + P1);
                L[off[i] + (d - lo[i])] = (uint16_t)(c + best - m);
            }
        }
}

// S(p,d) = sum over the first n_paths directions of L_r(p,d) (4 paths: 0-3, 8 paths: 0-7).
void oracle_sgm(int W, int Hh, int n_paths, int P1, int P2, const uint8_t* C, const int16_t* lo,
                const int16_t* hi, const uint32_t* off, uint16_t* S) {
    const int n = W * Hh;
    const uint32_t cells = off[n];
    std::vector<uint16_t> L(cells);
    std::memset(S, 0, sizeof(uint16_t) * cells);
    for (int r = 0; r < n_paths; ++r) {
        oracle_sgm_path(W, Hh, r, P1, P2, C, lo, hi, off, L.data());
        for (uint32_t k = 0; k < cells; ++k) S[k] = (uint16_t)(S[k] + L[k]);
    }
}

// ------------------------------------------------------------------------------------------
// Disparity selection and matching variance.
//  * winner-takes-all d* = argmin_{d in window} S(p,d), lowest d on ties;
//  * sub-pixel offset from the parabola through S(d*-1), S(d*), S(d*+1) when both neighbours
//    are inside the window: delta = (S- - S+) / (2 (S- - 2 S0 + S+)), else 0; Dz = d* + delta;
//  * matching variance r = n_l + n_r (Sec. 2.3 "Matching uncertainty", Eq. 9): walking away
//    from d* on each side, a neighbour is counted while the running sum of its cost rise
//    S(d) - S(d*) stays below the threshold s_thr (the paper's S_max, here on the aggregated
//    cost); the walk stops at the window edge. r is floored at r_min.
// ------------------------------------------------------------------------------------------
void oracle_select(int W, int Hh, const uint16_t* S, const int16_t* lo, const int16_t* hi,
                   const uint32_t* off, float s_thr, float r_min, int32_t* dstar, float* Dz,
                   float* rz) {
    const int n = W * Hh;
    for (int i = 0; i < n; ++i) {
        const uint16_t* s = S + off[i];
        const int a = lo[i], b = hi[i];
        int best = a;
        for (int d = a + 1; d <= b; ++d)
            if (s[d - a] < s[best - a]) best = d;
        float delta = 0.0f;
        if (best - 1 >= a && best + 1 <= b) {
            const int sm = s[best - 1 - a], s0 = s[best - a], sp = s[best + 1 - a];
            const int den = 2 * (sm - 2 * s0 + sp);
            if (den > 0) delta = (float)(sm - sp) / (float)den;
        }
        int nl = 0, nr = 0;
        int run = 0;
        for (int d = best - 1; d >= a; --d) {
            run += s[d - a] - s[best - a];
            if ((float)run < s_thr) ++nl; else break;
        }
        run = 0;
        for (int d = best + 1; d <= b; ++d) {
            run += s[d - a] - s[best - a];
            if ((float)run < s_thr) ++nr; else break;
        }
        float r = (float)(nl + nr);
        if (r < r_min) r = r_min;
        dstar[i] = best;
        Dz[i] = (float)best + delta;
        rz[i] = r;
    }
}

// ------------------------------------------------------------------------------------------
// Left-right consistency check (Sec. 2.4, "Disparity consistency check"). The right-view
// disparity of column xr is D_R(xr) = argmin over d with xr + d < W and d inside the window of
// the left pixel (xr + d, y) of S(xr + d, d), d < D, lowest d on ties (-1 if no candidate). A left
// pixel passes iff x - d* >= 0 and |d* - D_R(x - d*)| <= tol. Failing pixels get Dz = rz = -1.
// `dright` (W x H) and `valid` (W x H) are outputs for inspection.
// ------------------------------------------------------------------------------------------
void oracle_lr_check(int W, int Hh, int D, const uint16_t* S, const int16_t* lo, const int16_t* hi,
                     const uint32_t* off, const int32_t* dstar, int tol, int32_t* dright,
                     uint8_t* valid, float* Dz, float* rz) {
    for (int y = 0; y < Hh; ++y) {
        for (int xr = 0; xr < W; ++xr) {
            int bd = -1, bs = 1 << 30;
            for (int x = xr; x < W && x - xr < D; ++x) {
                const int d = x - xr;
                const int i = y * W + x;
                if (d < lo[i] || d > hi[i]) continue;
                const int s = S[off[i] + (d - lo[i])];
                if (s < bs) {  // increasing d, strict: lowest d keeps a tie
                    bs = s;
                    bd = d;
                }
            }
            dright[y * W + xr] = bd;
        }
        for (int x = 0; x < W; ++x) {
            const int i = y * W + x;
            const int d = dstar[i];
            bool ok = false;
            if (x - d >= 0) {
                const int dr = dright[y * W + x - d];
                ok = dr >= 0 && std::abs(d - dr) <= tol;
            }
            valid[i] = ok ? 1 : 0;
            if (!ok) {
                Dz[i] = -1.0f;
                rz[i] = -1.0f;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Pixel-wise Kalman update (Sec. 2.4, Eq. 10-12): K = p/(p+r); d = d_p + K (d_z - d_p);
// p' = (1-K) p. A pixel with only a measurement takes (d_z, r); with only a prediction it keeps
// (d_p, p); with neither it is invalid (-1, -1). Valid means finite and >= 0.
// ------------------------------------------------------------------------------------------
void oracle_kalman(int n, const float* Dp, const float* Pp, const float* Dz, const float* rz,
                   float* D, float* P) {
    for (int i = 0; i < n; ++i) {
        const bool pv = finite_nonneg(Dp[i]) && finite_nonneg(Pp[i]);
        const bool mv = finite_nonneg(Dz[i]) && finite_nonneg(rz[i]);
        if (pv && mv) {
            const float s = Pp[i] + rz[i];
            const float K = Pp[i] / s;
            const float innov = Dz[i] - Dp[i];
            const float corr = K * innov;
            D[i] = Dp[i] + corr;
            const float omk = 1.0f - K;
            P[i] = omk * Pp[i];
        } else if (mv) {
            D[i] = Dz[i];
            P[i] = rz[i];
        } else if (pv) {
            D[i] = Dp[i];
            P[i] = Pp[i];
        } else {
            D[i] = -1.0f;
            P[i] = -1.0f;
        }
    }
}

}  // extern "C"
