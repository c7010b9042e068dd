"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks one oracle function against something other than itself: a geometric
construction, a closed form, a hand-worked case, a textbook formulation written independently
here, or brute force on tiny inputs. They are chosen so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1708_06301_gb300 import synth

F, B = 721.0, 0.54


# ----------------------------------------------------------------------------------------------
# Eq. 1-4: disparity-space homography
# ----------------------------------------------------------------------------------------------

def _geometric_transfer(R, t, f, b, x, y, d):
    """Back-project (x, y, d) to Euclidean space, apply M' = R M + t (Eq. 2), project again."""
    Z = f * b / d
    M = np.array([x * Z / f, y * Z / f, Z])
    Mp = R @ M + t
    return f * Mp[0] / Mp[2], f * Mp[1] / Mp[2], f * b / Mp[2]


@pytest.mark.parametrize("seed", range(6))
def test_H_matches_geometric_transfer(seed):
    R, t = synth.random_pose(100 + seed, max_t=1.5, max_rot_deg=3.0)
    R = R.astype(np.float64)
    t = t.astype(np.float64)
    H64, H32 = oracle.build_H(R, t, F, B)
    rs = synth.Stream(seed, 1)
    for _ in range(50):
        x, y, d = rs.uniform(-600, 600), rs.uniform(-180, 180), rs.uniform(1, 127)
        w = H64 @ np.array([x, y, d, 1.0])
        got = w[:3] / w[3]  # Eq. 3: divide by the fourth component
        exp = _geometric_transfer(R, t, F, B, x, y, d)
        np.testing.assert_allclose(got, exp, rtol=1e-10, atol=1e-9)
    assert np.array_equal(H32, H64.astype(np.float32))


def test_H_identity_pose_is_identity():
    H64, _ = oracle.build_H(np.eye(3), np.zeros(3), F, B)
    np.testing.assert_allclose(H64, np.eye(4), atol=1e-15)


# ----------------------------------------------------------------------------------------------
# Sec. 2.2: warp, z-buffer, variance prediction (Eq. 3, 5, 6)
# ----------------------------------------------------------------------------------------------

def _cxcy(W, H):
    return np.float32((W - 1) / 2.0), np.float32((H - 1) / 2.0)


def test_warp_identity_pose_leaves_maps_unchanged():
    W, H = 57, 23
    D, P = synth.random_maps(7, W, H, invalid_frac=0.2)
    _, H32 = oracle.build_H(np.eye(3), np.zeros(3), F, B)
    cx, cy = _cxcy(W, H)
    q = 0.25
    Dp, Pp, win = oracle.warp_predict(D, P, H32, cx, cy, q)
    valid = D > 0
    assert np.array_equal(Dp[valid], D[valid])  # bit-exact
    assert np.array_equal(Pp[valid], (P[valid] + np.float32(q)).astype(np.float32))  # Phi = 1
    assert np.all(Dp[~valid] == -1) and np.all(Pp[~valid] == -1)
    idx = np.arange(W * H).reshape(H, W)
    assert np.array_equal(win[valid], idx[valid])


def test_warp_lateral_shift_and_zbuffer_bruteforce():
    """t = (3b/8, 0, 0): points at d = 8 move 3 px right, d = 16 move 6 px (x' = x + d t_x / b),
    disparity unchanged. Collisions are resolved by brute force: highest d, then lowest index."""
    W, H = 40, 9
    rs = synth.uniform01(3, np.arange(W * H)).reshape(H, W)
    D = np.where(rs < 0.5, 8.0, 16.0).astype(np.float32)
    D[rs > 0.9] = -1.0
    P = (0.1 + synth.uniform01(4, np.arange(W * H)).reshape(H, W)).astype(np.float32)
    P[D < 0] = -1.0
    t = np.array([3 * B / 8, 0, 0], dtype=np.float32)
    _, H32 = oracle.build_H(np.eye(3), t.astype(np.float64), F, B)
    cx, cy = _cxcy(W, H)
    Dp, Pp, win = oracle.warp_predict(D, P, H32, cx, cy, 0.5)
    # brute force
    expD = np.full((H, W), -1.0, np.float32)
    expW = np.full((H, W), -1, np.int64)
    for v in range(H):
        cands = {}
        for u in range(W):
            if D[v, u] <= 0:
                continue
            tu = u + (3 if D[v, u] == 8 else 6)
            if tu < W:
                cands.setdefault(tu, []).append((D[v, u], v * W + u))
        for tu, lst in cands.items():
            best = max(d for d, _ in lst)
            src = min(i for d, i in lst if d == best)
            expD[v, tu] = best
            expW[v, tu] = src
    assert np.array_equal(Dp, expD)
    assert np.array_equal(win, expW)
    ok = expW >= 0
    assert np.array_equal(Pp[ok], (P.reshape(-1)[expW[ok]] + np.float32(0.5)).astype(np.float32))


def test_warp_forward_motion_fronto_parallel_wall():
    """A wall at Z = 20 m seen after moving forward s: every prediction is f b/(Z - s) and
    Phi = Z/(Z - s), so p' = Phi^2 p + q (Eq. 5-6); checked in binary64 within 1e-6 rel."""
    W, H, Z, s, q = 64, 32, 20.0, 1.3, 0.25
    D = np.full((H, W), F * B / Z, np.float32)
    P = (0.1 + 3.9 * synth.uniform01(9, np.arange(W * H)).reshape(H, W)).astype(np.float32)
    _, H32 = oracle.build_H(np.eye(3), np.array([0, 0, -s]), F, B)
    cx, cy = _cxcy(W, H)
    Dp, Pp, win = oracle.warp_predict(D, P, H32, cx, cy, q)
    hit = win >= 0
    assert hit.mean() > 0.5  # zooming in leaves gaps (Sec. 2.2) but most pixels are reached
    np.testing.assert_allclose(Dp[hit], F * B / (Z - s), rtol=1e-6)
    phi = (Dp[hit].astype(np.float64)) / D.reshape(-1)[win[hit]].astype(np.float64)
    exp = phi ** 2 * P.reshape(-1)[win[hit]].astype(np.float64) + q
    np.testing.assert_allclose(Pp[hit], exp, rtol=1e-6)
    np.testing.assert_allclose(phi, Z / (Z - s), rtol=1e-6)
    # zooming: sources spread outwards from the principal point, so the image centre is reached
    assert hit[H // 2, W // 2]
    # each winner lands (x~ Z/(Z-s), y~ Z/(Z-s)) from the principal point; the target pixel is
    # the nearest one (round to nearest, not truncation)
    src = win[hit]
    su, sv = src % W, src // W
    x_land = (su - float(cx)) * Z / (Z - s) + float(cx)
    y_land = (sv - float(cy)) * Z / (Z - s) + float(cy)
    tv, tu = np.nonzero(hit)
    assert np.all(np.abs(x_land - tu) <= 0.5 + 1e-4)
    assert np.all(np.abs(y_land - tv) <= 0.5 + 1e-4)


def test_wrappers_reject_inputs_that_do_not_match_their_sizes():
    """The C functions trust the sizes they are given; the wrappers refuse a map of another shape
    (it would be read past its end) and a ragged layout that is not the scan of its windows."""
    D = np.ones((4, 6), np.float32)
    H = np.eye(4, dtype=np.float32)
    with pytest.raises(ValueError):
        oracle.warp_predict(D, np.ones((4, 1), np.float32), H, 2.5, 1.5, 0.0)
    with pytest.raises(ValueError):
        oracle.kalman(D, D, D, D[:, :5])
    with pytest.raises(ValueError):
        oracle.fill_gaps(D, D.T, 1.0)
    lo = np.zeros((4, 6), np.int16)
    hi = np.full((4, 6), 3, np.int16)
    off = oracle.offsets(lo, hi)
    with pytest.raises(ValueError):
        oracle.sgm(np.zeros(int(off[-1]) - 1, np.uint8), lo, hi, off, 4, 8, 32)
    bad = off.copy()
    bad[3] += 1
    with pytest.raises(ValueError):
        oracle.sgm(np.zeros(int(off[-1]), np.uint8), lo, hi, bad, 4, 8, 32)
    with pytest.raises(ValueError):
        oracle.sgm(np.zeros(int(off[-1]), np.uint8), hi, lo, off, 4, 8, 32)


def test_warp_zbuffer_tie_goes_to_lowest_source():
    """Moving backwards from a fronto-parallel wall shrinks the image: several sources with the
    same predicted disparity land on one target; the lowest source index must win. Landing
    pixels come from the geometric construction (binary64), keeping only sources that land at
    least 1e-3 px away from a rounding boundary."""
    W, H, Z, s = 48, 24, 10.0, 4.0
    D = np.full((H, W), F * B / Z, np.float32)
    P = np.ones((H, W), np.float32)
    _, H32 = oracle.build_H(np.eye(3), np.array([0, 0, +s]), F, B)
    cx, cy = _cxcy(W, H)
    _, _, win = oracle.warp_predict(D, P, H32, cx, cy, 0.0)
    uu, vv = np.meshgrid(np.arange(W), np.arange(H))
    xl = (uu - float(cx)) * Z / (Z + s) + float(cx) + 0.5
    yl = (vv - float(cy)) * Z / (Z + s) + float(cy) + 0.5
    sure = (np.abs(xl - np.round(xl)) > 1e-3) & (np.abs(yl - np.round(yl)) > 1e-3)
    tx, ty = np.floor(xl).astype(int), np.floor(yl).astype(int)
    idx = vv * W + uu
    n_ties = 0
    for t in set(zip(ty[sure].tolist(), tx[sure].tolist())):
        srcs = idx[(ty == t[0]) & (tx == t[1])]
        if np.all(sure.reshape(-1)[srcs]):
            assert win[t] == srcs.min()
            n_ties += len(srcs) > 1
    assert n_ties > 20


def test_warp_ground_plane_against_renderer():
    """Forward translation over a ground plane: the predicted disparity at every reached pixel
    is the ground-plane disparity of a point landing within half a pixel of that row, and agrees
    with the next frame's rendered ground truth up to the plane's disparity slope b/h per row."""
    W, H, h, s = 160, 80, 1.65, 0.8
    cam = synth.Camera(W, H, F, B)
    scene = synth.Scene(ground_y=h, far_z=1e7, boxes=np.zeros((0, 4)), tex_seed=1)
    _, Z0 = synth.render(scene, cam, np.eye(3), np.zeros(3))
    _, Z1 = synth.render(scene, cam, np.eye(3), np.array([0, 0, s]))
    D0 = (F * B / Z0).astype(np.float32)
    D1 = (F * B / Z1).astype(np.float32)
    ground = np.broadcast_to(np.arange(H)[:, None] > cam.cy + 2, (H, W))
    D0 = np.where(ground, D0, -1.0).astype(np.float32)
    P0 = np.where(ground, 1.0, -1.0).astype(np.float32)
    _, H32 = oracle.build_H(np.eye(3), np.array([0, 0, -s]), F, B)
    Dp, Pp, win = oracle.warp_predict(D0, P0, H32, np.float32(cam.cx), np.float32(cam.cy), 0.0)
    hit = win >= 0
    assert hit.sum() > 0.3 * ground.sum()
    rows = np.nonzero(hit)[0]
    y_land = cam.cy + h * Dp[hit].astype(np.float64) / B  # ground plane: d = b (y - cy) / h
    assert np.all(np.abs(y_land - rows) <= 0.5 + 1e-3)
    assert np.all(np.abs(Dp[hit] - D1[hit]) <= 0.5 * B / h + 1e-3)
    # each winner's predicted disparity is its source point seen s metres closer: f b / (Z - s)
    # (the plane maps onto itself either way, so this is what tells forward from backward)
    Zsrc = F * B / D0.reshape(-1)[win[hit]].astype(np.float64)
    np.testing.assert_allclose(Dp[hit], F * B / (Zsrc - s), rtol=2e-5)


# ----------------------------------------------------------------------------------------------
# Sec. 2.3: reduced window
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("d,p,D,exp", [
    (10.0, 1.0, 64, (7, 13)),        # 10 -+ 3
    (10.5, 0.25, 64, (9, 12)),       # 10.5 -+ 1.5
    (10.2, 0.25, 64, (8, 12)),       # [8.7, 11.7] rounded outwards
    (2.0, 4.0, 64, (0, 8)),          # clipped at 0
    (62.0, 4.0, 64, (56, 63)),       # clipped at D-1
    (10.0, 0.0, 64, (10, 10)),       # zero variance: one label
    (-1.0, -1.0, 64, (0, 63)),       # no prediction: whole range
    (10.0, float("nan"), 64, (0, 63)),
    (10.0, float("inf"), 64, (0, 63)),
    (100.0, 1.0, 64, (0, 63)),       # interval entirely above the range: whole range
    (0.0, 0.01, 64, (0, 1)),
    (63.0, 0.0, 64, (63, 63)),       # the top label alone is inside the range
    (0.0, 0.0, 64, (0, 0)),          # the bottom label alone
    (64.0, 0.0, 64, (0, 63)),        # one label above the range: a miss, whole range
])
def test_window_hand_cases(d, p, D, exp):
    lo, hi, off, n = oracle.windows(np.array([[d]], np.float32), np.array([[p]], np.float32), D, 3.0)
    assert (int(lo[0, 0]), int(hi[0, 0])) == exp
    assert n == exp[1] - exp[0] + 1 and off[0] == 0 and off[1] == n


def test_window_offsets_are_exclusive_scan():
    W, H = 33, 7
    D, P = synth.random_maps(5, W, H, d_range=(0, 70), p_range=(0, 9), invalid_frac=0.3)
    lo, hi, off, n = oracle.windows(D, P, 64, 3.0)
    w = (hi.astype(np.int64) - lo + 1).reshape(-1)
    assert np.all(w >= 1) and np.all(lo >= 0) and np.all(hi <= 63)
    assert n == w.sum() and off[0] == 0
    assert np.array_equal(off[1:].astype(np.int64), np.cumsum(w))
    # an invalid prediction searches the whole range
    assert np.all(lo[D < 0] == 0) and np.all(hi[D < 0] == 63)


# ----------------------------------------------------------------------------------------------
# Census + Hamming cost
# ----------------------------------------------------------------------------------------------

def test_census_hand_example():
    img = np.array([[1, 2, 3], [4, 5, 6], [7, 8, 9]], np.uint8)
    c = oracle.census(img, 3, 3)
    # centre 5: neighbours in row-major order 1,2,3,4,6,7,8,9 -> bits 0..3 set
    assert c[1, 1] == 0b00001111
    # corner (0,0) value 1 with border clamp: nothing is smaller
    assert c[0, 0] == 0
    # corner (2,2) value 9, window clamped to the border: the 8 neighbours in row-major order
    # read 5, 6, 6, 8, 9, 8, 9, 9 -> bits 0, 1, 2, 3 and 5 are set
    exp = 0
    bit = 0
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dx == 0 and dy == 0:
                continue
            qy, qx = min(max(2 + dy, 0), 2), min(max(2 + dx, 0), 2)
            if img[qy, qx] < 9:
                exp |= 1 << bit
            bit += 1
    assert c[2, 2] == exp == 0b00101111


def test_census_bruteforce_and_constant():
    img, _ = synth.random_images(11, 13, 9)
    for cw, ch in ((5, 5), (9, 7), (3, 3)):
        c = oracle.census(img, cw, ch)
        H, W = img.shape
        for y in range(H):
            for x in range(W):
                bits = []
                for dy in range(-(ch // 2), ch // 2 + 1):
                    for dx in range(-(cw // 2), cw // 2 + 1):
                        if dx or dy:
                            q = img[min(max(y + dy, 0), H - 1), min(max(x + dx, 0), W - 1)]
                            bits.append(int(q < img[y, x]))
                assert int(c[y, x]) == sum(b << i for i, b in enumerate(bits))
    assert not oracle.census(np.full((8, 8), 77, np.uint8), 9, 7).any()


def _popcount(v):
    return bin(int(v)).count("1")


def test_border_cost_is_the_census_bit_count():
    """B_c, the cost of a disparity that leaves the image, is the largest Hamming distance two
    census codes can have: the bit count of a local maximum's code (every neighbour darker)."""
    for cw, ch in ((3, 3), (5, 5), (9, 7)):
        img = np.zeros((ch + 2, cw + 2), np.uint8)
        img[ch // 2 + 1, cw // 2 + 1] = 200
        code = oracle.census(img, cw, ch)[ch // 2 + 1, cw // 2 + 1]
        assert oracle.Params(8, 8, census_w=cw, census_h=ch).Bc == _popcount(code)


def test_cost_hamming_and_border():
    a, b = synth.random_images(12, 21, 6)
    D = 8
    cl, cr = oracle.census(a, 9, 7), oracle.census(b, 9, 7)
    lo = np.zeros((6, 21), np.int16)
    hi = np.full((6, 21), D - 1, np.int16)
    off = oracle.offsets(lo, hi)
    C = oracle.cost(cl, cr, lo, hi, off, 62)
    for y in range(6):
        for x in range(21):
            for d in range(D):
                exp = 62 if x - d < 0 else _popcount(int(cl[y, x]) ^ int(cr[y, x - d]))
                assert C[off[y * 21 + x] + d] == exp
    # identical images: zero cost at d = 0
    C0 = oracle.cost(cl, cl, lo, hi, off, 62)
    assert np.all(C0[off[:-1]] == 0)


# ----------------------------------------------------------------------------------------------
# SGM aggregation (Sec. 2.3)
# ----------------------------------------------------------------------------------------------

DIRS = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (-1, 1), (1, -1)]


def _textbook_sgm_dense(Cd, n_paths, P1, P2):
    """Full-range SGM on a dense (H, W, D) volume, written independently of the oracle:
    vectorised over d, each path swept with numpy."""
    H, W, D = Cd.shape
    Cd = Cd.astype(np.int64)
    S = np.zeros_like(Cd)
    for dx, dy in DIRS[:n_paths]:
        L = np.zeros_like(Cd)
        ys = range(H) if dy >= 0 else range(H - 1, -1, -1)
        xs = list(range(W)) if dx >= 0 else list(range(W - 1, -1, -1))
        for y in ys:
            for x in xs:
                qx, qy = x - dx, y - dy
                if not (0 <= qx < W and 0 <= qy < H):
                    L[y, x] = Cd[y, x]
                    continue
                Lq = L[qy, qx]
                m = Lq.min()
                up = np.concatenate([[np.iinfo(np.int64).max // 4], Lq[:-1]]) + P1
                dn = np.concatenate([Lq[1:], [np.iinfo(np.int64).max // 4]]) + P1
                L[y, x] = Cd[y, x] + np.minimum(np.minimum(Lq, up), np.minimum(dn, m + P2)) - m
        S += L
    return S


@pytest.mark.parametrize("n_paths", [4, 8])
def test_sgm_full_windows_equal_textbook(n_paths):
    H, W, D = 11, 17, 12
    a, b = synth.random_images(21, W, H)
    cl, cr = oracle.census(a, 5, 5), oracle.census(b, 5, 5)
    lo = np.zeros((H, W), np.int16)
    hi = np.full((H, W), D - 1, np.int16)
    off = oracle.offsets(lo, hi)
    C = oracle.cost(cl, cr, lo, hi, off, 24)
    S = oracle.sgm(C, lo, hi, off, n_paths, 8, 32)
    S_tb = _textbook_sgm_dense(C.reshape(H, W, D), n_paths, 8, 32)
    assert np.array_equal(S.reshape(H, W, D).astype(np.int64), S_tb)


def _pen(a, b, P1, P2):
    return 0 if a == b else (P1 if abs(a - b) == 1 else P2)


def _line(W, H, dx, dy, start):
    x, y = start
    pts = []
    while 0 <= x < W and 0 <= y < H:
        pts.append((x, y))
        x, y = x + dx, y + dy
    return pts


def _line_starts(W, H, dx, dy):
    return [(x, y) for y in range(H) for x in range(W)
            if not (0 <= x - dx < W and 0 <= y - dy < H)]


@pytest.mark.parametrize("direction", range(8))
def test_sgm_path_equals_bruteforce_min_energy(direction):
    """Each path is exact 1-D dynamic programming: the normalised L_r equals the minimum, over
    every labelling of the path prefix inside the windows, of data cost plus P1/P2 penalties,
    up to a per-pixel constant."""
    H, W, D, P1, P2 = 4, 6, 4, 3, 7
    rs = synth.uniform01(31, direction, np.arange(W * H * D)).reshape(H, W, D)
    Cd = np.floor(rs * 20).astype(np.uint8)
    lo_l = np.floor(synth.uniform01(32, direction, np.arange(W * H)) * D).astype(np.int64)
    hi_l = lo_l + np.floor(synth.uniform01(33, direction, np.arange(W * H)) * (D - lo_l)).astype(np.int64)
    lo = lo_l.astype(np.int16).reshape(H, W)
    hi = hi_l.astype(np.int16).reshape(H, W)
    off = oracle.offsets(lo, hi)
    C = np.concatenate([Cd[i // W, i % W, lo_l[i]:hi_l[i] + 1] for i in range(W * H)])
    L = oracle.sgm_path(C, lo, hi, off, direction, P1, P2).astype(np.int64)
    dx, dy = DIRS[direction]
    checked = 0
    for st in _line_starts(W, H, dx, dy):
        pts = _line(W, H, dx, dy, st)
        for k in range(len(pts)):
            prefix = pts[:k + 1]
            doms = [range(lo[y, x], hi[y, x] + 1) for x, y in prefix]
            best = {}
            for lab in itertools.product(*doms):
                e = sum(int(Cd[y, x, l]) for (x, y), l in zip(prefix, lab))
                e += sum(_pen(lab[i - 1], lab[i], P1, P2) for i in range(1, len(lab)))
                best[lab[-1]] = min(best.get(lab[-1], 1 << 60), e)
            x, y = prefix[-1]
            i = y * W + x
            Lp = {d: L[off[i] + d - lo[y, x]] for d in range(lo[y, x], hi[y, x] + 1)}
            eb = min(best.values())
            lb = min(Lp.values())
            assert {d: v - eb for d, v in best.items()} == {d: v - lb for d, v in Lp.items()}
            checked += 1
    assert checked == W * H


def test_sgm_bound_and_reduced_equals_restricted_dense():
    """S <= P (Bc + P2); and shrinking windows never changes costs inside a window
    (the ragged cost is the dense cost restricted to the window)."""
    H, W, D = 9, 23, 16
    a, b = synth.random_images(41, W, H)
    cl, cr = oracle.census(a, 9, 7), oracle.census(b, 9, 7)
    lo, hi = synth.random_windows(42, W, H, D, 1, 9, full_frac=0.2)
    off = oracle.offsets(lo, hi)
    C = oracle.cost(cl, cr, lo, hi, off, 62)
    S = oracle.sgm(C, lo, hi, off, 8, 8, 32)
    assert S.max() <= 8 * (62 + 32)
    lof = np.zeros_like(lo)
    hif = np.full_like(hi, D - 1)
    offf = oracle.offsets(lof, hif)
    Cf = oracle.cost(cl, cr, lof, hif, offf, 62).reshape(H, W, D)
    for i in range(W * H):
        y, x = divmod(i, W)
        assert np.array_equal(C[off[i]:off[i + 1]], Cf[y, x, lo[y, x]:hi[y, x] + 1])


# ----------------------------------------------------------------------------------------------
# WTA, sub-pixel, matching variance (Eq. 9)
# ----------------------------------------------------------------------------------------------

def _select_one(s, lo=0, s_thr=8.0, r_min=0.0):
    s = np.asarray(s, np.uint16)
    loa = np.array([[lo]], np.int16)
    hia = np.array([[lo + len(s) - 1]], np.int16)
    off = np.array([0, len(s)], np.uint32)
    d, Dz, rz = oracle.select(s, loa, hia, off, s_thr, r_min)
    return int(d[0, 0]), float(Dz[0, 0]), float(rz[0, 0])


def test_select_parabola_vertex_exact():
    # S(d) = (2d - 21)^2 = 4 (d - 10.5)^2: tie at 10/11 -> d* = 10, vertex 10.5
    s = [(2 * d - 21) ** 2 for d in range(20)]
    assert _select_one(s)[:2] == (10, 10.5)
    # S(d) = 3 (4d - 29)^2 = 48 (d - 7.25)^2: vertex 7.25
    s = [3 * (4 * d - 29) ** 2 for d in range(16)]
    assert _select_one(s)[:2] == (7, 7.25)
    # same curve in a window starting at 5: disparities are absolute
    assert _select_one(s[5:12], lo=5)[:2] == (7, 7.25)
    # minimum on the window edge: no sub-pixel step
    assert _select_one([4, 9, 12], lo=3)[:2] == (3, 3.0)
    # minimum one label inside either edge: both neighbours exist, the parabola applies
    # (delta = (4 - 3) / (2 (4 - 2 + 3)) = 0.1 and its mirror image)
    assert _select_one([4, 1, 3])[:2] == (1, float(np.float32(1) + np.float32(1) / np.float32(10)))
    assert _select_one([3, 1, 4])[:2] == (1, float(np.float32(1) + np.float32(-1) / np.float32(10)))


def test_select_matching_variance_hand_cases():
    # S = [10, 5, 3, 4, 9, 20], d* = 2; left: +2 (count), +7 -> 9 >= 8 stop; right: +1, +6 -> 7
    # (count both), +17 stop  ->  r = 1 + 2 = 3
    # sub-pixel delta = (5 - 4) / (2 (5 - 6 + 4)) = 1/6, rounded to binary32
    exp_dz = float(np.float32(2) + np.float32(1) / np.float32(6))
    assert _select_one([10, 5, 3, 4, 9, 20], s_thr=8.0) == (2, exp_dz, 3.0)
    # flat bottom: equal neighbours count while the sum stays below the threshold (the case the
    # paper's extension of the slope measure is made for)
    d, _, r = _select_one([50, 3, 3, 3, 3, 50], s_thr=8.0)
    assert d == 1 and r == 3.0
    # a running sum equal to the threshold is not below it: S = [20, 8, 0, 8, 20], thr 8 -> r = 0
    assert _select_one([20, 8, 0, 8, 20], s_thr=8.0)[2] == 0.0
    assert _select_one([20, 7, 0, 8, 20], s_thr=8.0)[2] == 1.0
    # r floored at r_min
    assert _select_one([9, 0, 9], s_thr=8.0, r_min=0.5)[2] == 0.5
    # a threshold between integers: a running sum of 7 is below 7.5 but not below 7.0
    assert _select_one([20, 7, 0, 1, 20], s_thr=7.5)[2] == 2.0
    assert _select_one([20, 7, 0, 1, 20], s_thr=7.0)[2] == 1.0
    # a threshold above every running sum: the count stops at the window's edges, every other
    # label of the window counted (here 2 + 2), in a window that starts at 40 as well
    assert _select_one([5, 3, 0, 4, 9], s_thr=1.0e9)[2] == 4.0
    assert _select_one([5, 3, 0, 4, 9], lo=40, s_thr=3.0e7)[2] == 4.0


def test_select_argmin_bruteforce():
    H, W, D = 5, 7, 10
    lo, hi = synth.random_windows(51, W, H, D, 1, 10)
    off = oracle.offsets(lo, hi)
    S = np.floor(synth.uniform01(52, np.arange(off[-1])) * 30).astype(np.uint16)
    d, _, _ = oracle.select(S, lo, hi, off, 40.0, 0.5)
    for i in range(W * H):
        y, x = divmod(i, W)
        assert d[y, x] == lo[y, x] + int(np.argmin(S[off[i]:off[i + 1]]))


def test_matching_variance_threshold_is_per_path():
    """Eq. 9's threshold S_max is read as per path: on the aggregated cost of n paths it is
    n * S_max. On a 1 x 1 image every path is its own first pixel, so each path cost is the
    matching cost and S = n C; the count must then equal Eq. 9 evaluated on C with S_max. Equal
    left and right pixels give C = (0, B_c, B_c, ...) (a disparity > 0 leaves the image), so with
    B_c = 24 < S_max = 30 < 2 B_c one neighbour of d* = 0 is counted."""
    for n_paths in (4, 8):
        prm = oracle.Params(1, 1, d_max=7, n_paths=n_paths, S_max=30.0, r_min=0.0)
        tr = oracle.Tracker(prm)
        img = np.array([[90]], np.uint8)
        D, P = tr.frame(img, img, None, None, np.eye(3), 0.5)
        assert D[0, 0] == 0.0 and P[0, 0] == 1.0


# ----------------------------------------------------------------------------------------------
# Left-right check (Sec. 2.4)
# ----------------------------------------------------------------------------------------------

def test_lr_check_bruteforce():
    H, W, D = 4, 19, 8
    lo, hi = synth.random_windows(61, W, H, D, 1, 8, full_frac=0.3)
    off = oracle.offsets(lo, hi)
    S = np.floor(synth.uniform01(62, np.arange(off[-1])) * 25).astype(np.uint16)
    dstar, Dz, rz = oracle.select(S, lo, hi, off, 40.0, 0.5)
    dright, valid, Dzm, rzm = oracle.lr_check(S, lo, hi, off, dstar, D, 1, Dz, rz)
    for y in range(H):
        for xr in range(W):
            cands = []
            for x in range(W):
                d = x - xr
                i = y * W + x
                if 0 <= d < D and lo[y, x] <= d <= hi[y, x]:
                    cands.append((int(S[off[i] + d - lo[y, x]]), d))
            exp = min(cands)[1] if cands else -1
            assert dright[y, xr] == exp
        for x in range(W):
            d = dstar[y, x]
            ok = x - d >= 0 and dright[y, x - d] >= 0 and abs(d - dright[y, x - d]) <= 1
            assert valid[y, x] == ok
            if ok:
                assert Dzm[y, x] == Dz[y, x] and rzm[y, x] == rz[y, x]
            else:
                assert Dzm[y, x] == -1 and rzm[y, x] == -1


def test_lr_check_consistent_pair_passes():
    """A left view whose costs are minimal exactly on a constant disparity passes everywhere it
    has a right correspondence, and fails where x - d* < 0 (no right pixel)."""
    H, W, D, d0 = 2, 16, 6, 3
    lo = np.zeros((H, W), np.int16)
    hi = np.full((H, W), D - 1, np.int16)
    off = oracle.offsets(lo, hi)
    S = np.array([[0 if d == d0 else 10 + d for d in range(D)] for _ in range(W * H)],
                 np.uint16).reshape(-1)
    dstar, Dz, rz = oracle.select(S, lo, hi, off, 8.0, 0.5)
    _, valid, _, _ = oracle.lr_check(S, lo, hi, off, dstar, D, 1, Dz, rz)
    assert np.all(valid[:, d0:] == 1) and np.all(valid[:, :d0] == 0)


# ----------------------------------------------------------------------------------------------
# Kalman update (Eq. 10-12)
# ----------------------------------------------------------------------------------------------

def test_kalman_information_form():
    n = 5000
    dp = (1 + 126 * synth.uniform01(71, np.arange(n))).astype(np.float32)
    pp = (0.1 + 3.9 * synth.uniform01(72, np.arange(n))).astype(np.float32)
    dz = (1 + 126 * synth.uniform01(73, np.arange(n))).astype(np.float32)
    rz = (0.5 + 4 * synth.uniform01(74, np.arange(n))).astype(np.float32)
    D, P = oracle.kalman(dp, pp, dz, rz)
    p64, r64 = pp.astype(np.float64), rz.astype(np.float64)
    expD = (r64 * dp + p64 * dz) / (p64 + r64)     # information-form fusion
    expP = p64 * r64 / (p64 + r64)
    np.testing.assert_allclose(D, expD, rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(P, expP, rtol=1e-6)


def test_kalman_limits_and_missing_sides():
    dp = np.array([10, 10, 10, -1, 10, -1], np.float32)
    pp = np.array([1, 1e30, 1, -1, 2, -1], np.float32)
    dz = np.array([12, 12, -1, 12, 12, -1], np.float32)
    rz = np.array([0, 1, -1, 3, 2, -1], np.float32)
    D, P = oracle.kalman(dp, pp, dz, rz)
    assert D[0] == 12 and P[0] == 0          # r -> 0: take the measurement
    assert abs(D[1] - 12) < 1e-5             # p -> inf: take the measurement
    assert D[2] == 10 and P[2] == 1          # no measurement: keep the prediction
    assert D[3] == 12 and P[3] == 3          # no prediction: take the measurement
    assert D[4] == 11 and P[4] == 1          # equal variances: midpoint, half variance
    assert D[5] == -1 and P[5] == -1
    # validity needs both the value and its variance: a prediction with an invalid or infinite
    # variance is no prediction (the p -> inf limit takes the measurement and its variance),
    # a measurement with an invalid variance is no measurement
    dp = np.array([10, 10, 10], np.float32)
    pp = np.array([np.inf, -1, 1], np.float32)
    dz = np.array([12, 12, 12], np.float32)
    rz = np.array([2, 2, -1], np.float32)
    D, P = oracle.kalman(dp, pp, dz, rz)
    assert D[0] == 12 and P[0] == 2
    assert D[1] == 12 and P[1] == 2
    assert D[2] == 10 and P[2] == 1


# ----------------------------------------------------------------------------------------------
# Whole pipeline properties
# ----------------------------------------------------------------------------------------------

def test_tracker_prediction_adds_the_ego_motion_variance():
    """With an identity pose the warp moves nothing and Phi = 1 (Eq. 5), so the tracker's raw
    prediction of frame 2 is frame 1's map, with its variance raised by q (Eq. 6)."""
    seq = synth.small_pair(1)
    prm = oracle.Params(320, 96, q=0.75)
    tr = oracle.Tracker(prm)
    D1, P1 = tr.frame(seq.left[0], seq.right[0], seq.R[0], seq.t[0], seq.K, B)
    o = tr.frame(seq.left[0], seq.right[0], np.eye(3), np.zeros(3), seq.K, B, keep=True)
    v = (D1 > 0) & (P1 >= 0)
    assert v.mean() > 0.5
    assert np.array_equal(o["Dpred_raw"][v], D1[v])
    assert np.array_equal(o["Ppred_raw"][v], (P1[v] + np.float32(0.75)).astype(np.float32))
    assert np.all(o["Dpred_raw"][~v] == -1)


def test_tracker_rejected_measurement_is_searched_in_full_next_frame():
    """Sec. 2.4 (disparity consistency check): the true minimum may lie outside a reduced window,
    so where the matched disparity was rejected the next frame searches the whole range. The
    updated map itself still carries the prediction there (Sec. 3: it combines the matched and
    the predicted map). With identity poses every pixel predicts only itself, so the pixels
    rejected in frame 2 are exactly the ones without a prediction in frame 3."""
    seq = synth.small_pair(1)
    prm = oracle.Params(320, 96)
    tr = oracle.Tracker(prm)
    I3, z3 = np.eye(3, dtype=np.float32), np.zeros(3, np.float32)
    tr.frame(seq.left[0], seq.right[0], seq.R[0], seq.t[0], seq.K, B)
    noise, _ = synth.random_images(5, 320, 96)
    # frame 2: an unrelated right view, so that many matches fail the left-right check
    o2 = tr.frame(seq.left[0], noise, I3, z3, seq.K, B, keep=True)
    pv = o2["Dpred"] >= 0
    rej = pv & (o2["Dz"] < 0)
    acc = pv & (o2["Dz"] >= 0)
    assert rej.sum() > 1000 and acc.sum() > 100
    assert np.array_equal(o2["D"][rej], o2["Dpred"][rej])
    assert np.array_equal(o2["P"][rej], o2["Ppred"][rej])
    assert np.all(o2["D_state"][rej] == -1) and np.all(o2["P_state"][rej] == -1)
    assert np.array_equal(o2["D_state"][acc], o2["D"][acc])
    o3 = tr.frame(seq.left[0], seq.right[0], I3, z3, seq.K, B, keep=True)
    assert np.all(o3["Dpred_raw"][rej] == -1)
    assert np.all(o3["lo"][rej] == 0) and np.all(o3["hi"][rej] == prm.D - 1)
    w3 = o3["hi"].astype(np.int64) - o3["lo"] + 1
    assert np.all(w3[acc] < prm.D)


def test_tracker_full_range_option():
    """full_range searches [0, D-1] everywhere and keeps the prediction and the update: frame 2
    equals the Kalman update (Eq. 10-12) of the warped prediction with a full-range match."""
    seq = synth.small_pair(1)
    prm = oracle.Params(320, 96, full_range=True)
    tr = oracle.Tracker(prm)
    tr.frame(seq.left[0], seq.right[0], seq.R[0], seq.t[0], seq.K, B)
    o = tr.frame(seq.left[1], seq.right[1], seq.R[1], seq.t[1], seq.K, B, keep=True)
    assert np.all(o["lo"] == 0) and np.all(o["hi"] == 63) and o["n_cells"] == 320 * 96 * 64
    assert (o["Dpred"] >= 0).mean() > 0.5
    lo, hi = np.zeros((96, 320), np.int16), np.full((96, 320), 63, np.int16)
    Dz, rz = oracle.match(seq.left[1], seq.right[1], lo, hi, prm)
    D, P = oracle.kalman(o["Dpred"], o["Ppred"], Dz, rz)
    assert np.array_equal(o["D"], D) and np.array_equal(o["P"], P)


def test_pipeline_small_pair_reduced_vs_full():
    """Frame 2 of the 320x96 pair: the reduced search considers a fraction of the cells and is at
    least as accurate (bad-3px over ground truth) as full-range SGM on the same frame."""
    seq = synth.small_pair(1)
    prm = oracle.Params(320, 96)
    tr = oracle.Tracker(prm)
    tr.frame(seq.left[0], seq.right[0], seq.R[0], seq.t[0], seq.K, B)
    o = tr.frame(seq.left[1], seq.right[1], seq.R[1], seq.t[1], seq.K, B, keep=True)
    assert o["n_cells"] < 0.5 * 320 * 96 * 64
    lo = np.zeros((96, 320), np.int16)
    hi = np.full((96, 320), 63, np.int16)
    Dz_full, _ = oracle.match(seq.left[1], seq.right[1], lo, hi, prm)
    gt = seq.gt_disp[1]

    def bad(d):
        return float(np.mean((d < 0) | (np.abs(d - gt) > 3)))

    assert bad(o["D"]) <= bad(Dz_full)


# ----------------------------------------------------------------------------------------------
# Sec. 2.2, Eq. 7-8: gap filling
# ----------------------------------------------------------------------------------------------

def test_fill_gaps_hand_cases():
    I = -1.0
    D = np.array([[5, I, 5.5, I, 9, I, I, 3],
                  [1, 1, 1, 1, 1, 1, 1, 1],
                  [2, 2, 2, I, 2, 2, 2, 2]], np.float32)
    P = np.where(D >= 0, 1.0, -1.0).astype(np.float32)
    P[0, 0], P[0, 2] = 2.0, 4.0
    Df, Pf = oracle.fill_gaps(D, P, 1.0)
    assert Df[0, 1] == 5.25 and Pf[0, 1] == 3.0        # similar neighbours: mean (Eq. 7)
    assert Df[0, 3] == -1                              # |5.5 - 9| >= gamma_f (Eq. 8): invalid
    assert Df[0, 5] == -1 and Df[0, 6] == -1           # two-pixel gap: no immediate pair
    assert Df[2, 3] == 2.0 and Pf[2, 3] == 1.0
    # vertical pass
    D2 = np.array([[4, 4, 4], [I, I, I], [4.5, 9, 4.2]], np.float32)
    P2 = np.where(D2 >= 0, 1.0, -1.0).astype(np.float32)
    Df2, _ = oracle.fill_gaps(D2, P2, 1.0)
    assert Df2[1, 0] == 4.25
    assert Df2[1, 1] == -1                             # |4 - 9| >= gamma_f
    assert Df2[1, 2] == np.float32((np.float32(4) + np.float32(4.2)) * np.float32(0.5))
    # similarity is strict (Eq. 8): neighbours exactly gamma_f apart do not fill the gap
    E = np.array([[5, I, 6]], np.float32)
    EP = np.where(E >= 0, 1.0, -1.0).astype(np.float32)
    assert oracle.fill_gaps(E, EP, 1.0)[0][0, 1] == -1
    assert oracle.fill_gaps(E, EP, 1.5)[0][0, 1] == 5.5


def test_fill_gaps_horizontal_pass_comes_first():
    """(1, 1) has dissimilar horizontal neighbours (0 and 20) and an invalid upper neighbour that
    only the horizontal pass fills: it is filled iff the horizontal pass runs before the vertical
    one (Sec. 2.2 describes the horizontal filling, then 'the same approach' vertically)."""
    I = -1.0
    D = np.array([[3, I, 3], [0, I, 20], [3, 3, 3]], np.float32)
    P = np.where(D >= 0, 1.0, -1.0).astype(np.float32)
    Df, _ = oracle.fill_gaps(D, P, 1.0)
    assert Df[0, 1] == 3 and Df[1, 1] == 3


def test_edge_reject_hand_cases():
    """Sec. 2.2: predicted pixels next to a disparity discontinuity are rejected (reading: any
    valid 8-neighbour differing by >= edge_thr), both sides of the edge, nothing else."""
    I = -1.0
    # a vertical step between columns 2 and 3: those two columns go, the rest stays
    D = np.array([[10, 10, 10, 20, 20, 20]] * 4, np.float32)
    P = np.full_like(D, 2.0)
    De, Pe = oracle.edge_reject(D, P, 1.0)
    keep = np.ones_like(D, bool)
    keep[:, 2:4] = False
    assert np.array_equal(De[keep], D[keep]) and np.array_equal(Pe[keep], P[keep])
    assert np.all(De[~keep] == -1) and np.all(Pe[~keep] == -1)
    # a ramp whose steps (0.4 px across, 0.8 px diagonally) stay below the threshold: untouched
    y, x = np.mgrid[0:5, 0:7].astype(np.float32)
    R = (np.float32(10) + np.float32(0.4) * x + np.float32(0.4) * y).astype(np.float32)
    Re, _ = oracle.edge_reject(R, np.ones_like(R), 1.0)
    assert np.array_equal(Re, R)
    # a difference equal to the threshold is a discontinuity (the similarity of Eq. 8 is strict)
    E = np.array([[5, 6]], np.float32)
    Ee, _ = oracle.edge_reject(E, np.ones_like(E), 1.0)
    assert np.all(Ee == -1)
    Ee2, _ = oracle.edge_reject(E, np.ones_like(E), 1.5)
    assert np.array_equal(Ee2, E)
    # holes are not edges: a valid pixel among invalid ones (or ones with an invalid variance)
    # stays; a diagonal neighbour counts
    H = np.array([[I, I, I], [I, 7, 30], [I, 40, I]], np.float32)
    HP = np.where(H >= 0, 1.0, -1.0).astype(np.float32)
    HP[1, 2] = -1.0                                  # (1, 2) has an invalid variance: a hole
    He, _ = oracle.edge_reject(H, HP, 1.0)
    assert He[1, 1] == -1 and He[2, 1] == -1         # 7 vs 40 (below): both rejected
    assert He[1, 2] == 30                            # invalid pixels are left as they are
    # a valid pixel whose neighbours are all holes stays, and so does one whose only valid-looking
    # neighbour, far away in disparity, has an invalid variance
    O = np.array([[I, I, I], [I, 7, I], [I, I, I]], np.float32)
    assert oracle.edge_reject(O, np.where(O >= 0, 1.0, -1.0).astype(np.float32), 1.0)[0][1, 1] == 7
    V = np.array([[I, I, I], [I, 7, 30], [I, I, I]], np.float32)
    VP = np.array([[I, I, I], [I, 1, I], [I, I, I]], np.float32)
    assert oracle.edge_reject(V, VP, 1.0)[0][1, 1] == 7
    G = np.array([[I, I, I], [I, 7, I], [I, I, 90]], np.float32)
    Ge, _ = oracle.edge_reject(G, np.where(G >= 0, 1.0, -1.0).astype(np.float32), 1.0)
    assert Ge[1, 1] == -1 and Ge[2, 2] == -1         # diagonal neighbours: an edge
    # one pixel, one row, one column: no neighbours beyond the image
    assert oracle.edge_reject(np.array([[3.0]], np.float32), np.array([[1.0]], np.float32), 1.0)[0][0, 0] == 3.0


def test_edge_reject_runs_before_gap_filling_in_the_tracker():
    """The tracker refines the prediction in the paper's order: edge rejection, then gap filling
    (Sec. 2.2); a one-pixel hole between two rejected edge pixels stays a hole."""
    from paper_1708_06301_gb300 import synth
    seq = synth.small_pair(1)
    W, H = seq.cam.W, seq.cam.H
    base = dict(d_max=63, census_w=5, census_h=5, n_paths=4)
    outs = {}
    for er in (False, True):
        prm = oracle.Params(W, H, fill_gaps=True, edge_reject=er, **base)
        tr = oracle.Tracker(prm)
        tr.frame(seq.left[0], seq.right[0], None, None, seq.K, seq.cam.b)
        outs[er] = tr.frame(seq.left[1], seq.right[1], seq.R[1], seq.t[1], seq.K, seq.cam.b, keep=True)
    pd0, pd1 = outs[False]["Dpred"], outs[True]["Dpred"]
    assert (pd1 < 0).sum() > (pd0 < 0).sum()        # the scene's object edges lose predictions
    raw = (outs[True]["Dpred_raw"], outs[True]["Ppred_raw"])
    ref = oracle.fill_gaps(*oracle.edge_reject(*raw, 1.0), 1.0)
    swapped = oracle.edge_reject(*oracle.fill_gaps(*raw, 1.0), 1.0)
    assert np.array_equal(ref[0], pd1) and np.array_equal(ref[1], outs[True]["Ppred"])
    assert not np.array_equal(swapped[0], pd1)       # the order matters on this scene


def test_pred_lr_check_hand_cases():
    """Sec. 2.2 / Fig. 3(d): the prediction's left-right check against the right view formed from
    it (each predicted pixel lands on x - round(d); the right view keeps the nearest surface)."""
    I = -1.0
    # one row worked by hand: landing columns 1, 1, 0, 2, 2, 6, 0 for x = 1..7
    d = np.array([[I, 0.4, 1.0, 3.0, 2.0, 2.6, 0.0, 7.2]], np.float32)
    p = np.where(d >= 0, 1.0, -1.0).astype(np.float32)
    De, Pe = oracle.pred_lr_check(d, p, 0.5)
    # right view: col 0 <- max(3.0, 7.2) = 7.2, col 1 <- max(0.4, 1.0) = 1.0, col 2 <- 2.6, col 6 <- 0
    expect = np.array([[I, I, 1.0, I, I, 2.6, 0.0, 7.2]], np.float32)
    assert np.array_equal(De, expect)
    assert np.array_equal(Pe, np.where(expect >= 0, 1.0, -1.0).astype(np.float32))
    # the same row with a looser threshold: 0.6 apart is now consistent, 4.2 apart still not
    De2, _ = oracle.pred_lr_check(d, p, 0.6)
    assert np.array_equal(De2, np.array([[I, 0.4, 1.0, I, 2.0, 2.6, 0.0, 7.2]], np.float32))
    # a difference equal to the threshold is consistent: x=2 (2.0) and x=3 (2.5, rounds to 3)
    # land on column 0 with x=0 (0.0), which the nearer 2.5 hides; x=1 (0.0) keeps column 1
    e = np.array([[0, 0, 2.0, 2.5]], np.float32)
    Ee, _ = oracle.pred_lr_check(e, np.ones_like(e), 0.5)
    assert np.array_equal(Ee, np.array([[I, 0, 2.0, 2.5]], np.float32))
    Ee2, _ = oracle.pred_lr_check(e, np.ones_like(e), 0.49)
    assert np.array_equal(Ee2, np.array([[I, 0, I, 2.5]], np.float32))


def test_pred_lr_check_geometry():
    """Closed forms: a fronto-parallel plane at disparity d is seen by both cameras exactly where
    x >= round(d) (the left-border band of Fig. 3(d)); a nearer block hides from the right camera
    the band of background of width (d_F - d_B) just left of it, and nothing else."""
    W, H = 40, 3
    for dv in (0.0, 3.0, 7.49, 7.5, 12.2):
        D = np.full((H, W), dv, np.float32)
        De, _ = oracle.pred_lr_check(D, np.ones_like(D), 0.25)
        k = int(math.floor(dv + 0.5))
        assert np.all(De[:, :k] == -1) and np.array_equal(De[:, k:], D[:, k:])
    dB, dF, a, b = 4.0, 10.0, 20, 30
    D = np.full((1, W), dB, np.float32)
    D[0, a:b] = dF
    De, _ = oracle.pred_lr_check(D, np.ones_like(D), 0.5)
    hidden = np.zeros(W, bool)
    hidden[:4] = True                                   # background not seen by the right camera
    hidden[a - int(dF - dB):a] = True                   # background behind the block
    assert np.all(De[0, hidden] == -1)
    assert np.array_equal(De[0, ~hidden], D[0, ~hidden])


def test_sad_check_hand_cases():
    """Sec. 2.4: a pixel of the updated map is rejected when its left/right patch SAD exceeds the
    threshold times the patch area; coordinates clamp at the image border."""
    I = -1.0
    L = np.array([[10, 20, 30, 40, 50]], np.uint8)
    R = np.array([[20, 30, 40, 50, 99]], np.uint8)  # the left row moved one pixel left
    D = np.array([[1.0, 1.0, 1.0, 0.0, I]], np.float32)
    P = np.where(D >= 0, 1.0, -1.0).astype(np.float32)
    # 3 x 1 patches. x=0, d=1: left (10,10,20) vs right cols clamp(-2..0) = (20,20,20): SAD 30;
    # x=1, d=1: (10,20,30) vs (20,20,30): 10; x=2, d=1: (20,30,40) vs (20,30,40): 0;
    # x=3, d=0: (30,40,50) vs (40,50,99): 10 + 10 + 49 = 69
    De, Pe = oracle.sad_check(L, R, D, P, 3, 1, 10.0)   # limit 30: 30 stays (not above), 69 goes
    assert np.array_equal(De, np.array([[1.0, 1.0, 1.0, I, I]], np.float32))
    assert np.array_equal(Pe, np.array([[1.0, 1.0, 1.0, I, I]], np.float32))
    De2, _ = oracle.sad_check(L, R, D, P, 3, 1, 3.0)    # limit 9: only the exact match stays
    assert np.array_equal(De2, np.array([[I, I, 1.0, I, I]], np.float32))
    # rounding of the disparity: 1.49 uses 1, 1.5 uses 2 (x=2: right cols 0..2 = (20,30,40) vs
    # cols -1..1 clamped = (20,20,30))
    D3 = np.array([[I, I, 1.49, I, I]], np.float32)
    assert oracle.sad_check(L, R, D3, np.abs(D3), 3, 1, 0.0)[0][0, 2] == 1.49
    D4 = np.array([[I, I, 1.5, I, I]], np.float32)
    assert oracle.sad_check(L, R, D4, np.abs(D4), 3, 1, 6.6)[0][0, 2] == -1   # SAD 20 > 19.8
    assert oracle.sad_check(L, R, D4, np.abs(D4), 3, 1, 6.7)[0][0, 2] == 1.5  # 20 <= 20.1
    # the limit scales with the patch area sw * sh: 3 x 5 patches of two constant images 2 apart
    # have SAD 30, which a threshold of 2 (limit 30) keeps and one of 1.99 (limit 29.85) rejects
    L5 = np.full((5, 5), 10, np.uint8)
    R5 = np.full((5, 5), 12, np.uint8)
    D5 = np.full((5, 5), I, np.float32)
    D5[2, 2] = 0.0
    P5 = np.abs(D5)
    assert oracle.sad_check(L5, R5, D5, P5, 3, 5, 2.0)[0][2, 2] == 0.0
    assert oracle.sad_check(L5, R5, D5, P5, 3, 5, 1.99)[0][2, 2] == -1


def test_sad_check_shifted_texture():
    """A right image that is the left one shifted by s: every pixel far enough from the borders
    passes at d = s with SAD 0 and fails at a wrong disparity."""
    rng = np.random.default_rng(3)
    W, H, s = 48, 9, 5
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = np.zeros_like(L)
    R[:, :W - s] = L[:, s:]
    D = np.full((H, W), float(s), np.float32)
    De, _ = oracle.sad_check(L, R, D, np.ones_like(D), 5, 5, 0.0)
    inner = (slice(2, H - 2), slice(s + 2, W - s - 2))
    assert np.all(De[inner] == s)
    Dw = np.full((H, W), float(s + 3), np.float32)
    Dwe, _ = oracle.sad_check(L, R, Dw, np.ones_like(Dw), 5, 5, 20.0)
    assert np.all(Dwe[inner] == -1)


def test_pred_lr_and_sad_checks_in_the_tracker():
    """The tracker checks the prediction after gap filling (Fig. 3(c) then (d)) and the updated
    map with the SAD check after the Kalman update; both only ever invalidate pixels."""
    seq = synth.small_pair(1)
    W, H = seq.cam.W, seq.cam.H
    base = dict(d_max=63, census_w=5, census_h=5, n_paths=4, fill_gaps=True)
    prm = oracle.Params(W, H, pred_lr_check=True, sad_check=True, **base)
    tr = oracle.Tracker(prm)
    tr.frame(seq.left[0], seq.right[0], None, None, seq.K, seq.cam.b)
    out = tr.frame(seq.left[1], seq.right[1], seq.R[1], seq.t[1], seq.K, seq.cam.b, keep=True)
    raw = (out["Dpred_raw"], out["Ppred_raw"])
    ref = oracle.pred_lr_check(*oracle.fill_gaps(*raw, prm.gamma_f), prm.pred_lr_tol)
    assert np.array_equal(ref[0], out["Dpred"]) and np.array_equal(ref[1], out["Ppred"])
    filled = oracle.fill_gaps(*raw, prm.gamma_f)[0]
    assert (out["Dpred"] < 0).sum() > (filled < 0).sum()     # the left border band goes
    chk = oracle.sad_check(seq.left[1], seq.right[1], out["D_unchecked"], out["P_unchecked"],
                           prm.sad_w, prm.sad_h, prm.sad_thr)
    assert np.array_equal(chk[0], out["D"]) and np.array_equal(chk[1], out["P"])
    changed = out["D"] != out["D_unchecked"]
    assert np.all(out["D"][changed] == -1)
