"""Pins of the oracle's binary64 adjoint references (no GPU needed)."""
import numpy as np

import oracle
from paper_1708_06301_gb300 import synth

B = np.float32(0.54)


def _setup(seed, W=180, H=60):
    D, P = synth.random_maps(seed, W, H, invalid_frac=0.1)
    Dz, rz = synth.random_maps(seed + 1, W, H, p_range=(0.5, 4), invalid_frac=0.1)
    R, t = synth.random_pose(seed + 2)
    w = np.array([0.03, -0.02, 0.04])
    pose6 = np.concatenate([w, t.astype(np.float64)])
    K = synth.Camera(W, H, 721.0, 0.54).K
    _, H32 = oracle.build_H(oracle.rodrigues(w).astype(np.float32), t, 721.0, float(B))
    _, _, win = oracle.warp_predict(D, P, H32, K[0, 2], K[1, 2], 0.25)
    rs = np.random.default_rng(seed)
    gD = rs.normal(size=(H, W)).astype(np.float32)
    gP = rs.normal(size=(H, W)).astype(np.float32)
    return D, P, Dz, rz, win, pose6, K, gD, gP


def test_rodrigues_is_a_rotation_about_its_axis():
    w = np.array([0.3, -0.2, 0.5])
    R = oracle.rodrigues(w)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
    np.testing.assert_allclose(R @ w, w, atol=1e-14)          # the axis is fixed
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-14)
    # quarter turn about z maps x to y
    np.testing.assert_allclose(oracle.rodrigues([0, 0, np.pi / 2]) @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def test_fixed_winner_forward_matches_the_binary32_pipeline():
    D, P, Dz, rz, win, pose6, K, _, _ = _setup(1)
    D64, P64 = oracle.warp_kalman_f64(D, P, win, pose6, K, B, 0.25, 1.0, Dz, rz)
    _, H32 = oracle.build_H(oracle.rodrigues(pose6[:3]).astype(np.float32), pose6[3:].astype(np.float32),
                            721.0, float(B))
    Dp, Pp, _ = oracle.warp_predict(D, P, H32, K[0, 2], K[1, 2], 0.25)
    D32, P32 = oracle.kalman(Dp, Pp, Dz, rz)
    assert np.array_equal(D64 < 0, D32 < 0)
    v = D32 >= 0
    np.testing.assert_allclose(D64[v], D32[v], rtol=2e-5, atol=1e-4)
    np.testing.assert_allclose(P64[v], P32[v], rtol=2e-5)


def test_analytic_gradient_matches_finite_differences():
    for seed in (1, 7):
        args = _setup(seed)
        D, P, Dz, rz, win, pose6, K, gD, gP = args
        g_fd = oracle.adjoint_fd(D, P, win, pose6, K, B, 0.25, 1.3, Dz, rz, gD, gP)
        g_an = oracle.adjoint_grad_f64(D, P, win, pose6, K, B, 0.25, 1.3, Dz, rz, gD, gP)
        scale = np.abs(g_fd).max()
        np.testing.assert_allclose(g_an, g_fd, rtol=1e-6, atol=1e-9 * scale)
        assert g_fd[3] == 0 and g_fd[4] == 0  # lateral translation: no depth change


def test_gradient_closed_forms_for_one_sided_pixels():
    """Prediction only: P = p' = (d'/d)^2 p + q, so dL/dq = sum of gP over predicted pixels.
    Measurement only: P = s_r r_z, so dL/ds_r = sum of gP r_z."""
    D, P, Dz, rz, win, pose6, K, gD, gP = _setup(3)
    none = np.full_like(Dz, -1.0)
    g = oracle.adjoint_grad_f64(D, P, win, pose6, K, B, 0.25, 1.0, none, none, gD, gP)
    assert np.isclose(g[6], gP.reshape(-1)[win.reshape(-1) >= 0].astype(np.float64).sum())
    nowin = np.full_like(win, -1)
    g = oracle.adjoint_grad_f64(D, P, nowin, pose6, K, B, 0.25, 2.0, Dz, rz, gD, gP)
    mv = (Dz >= 0) & (rz >= 0)
    assert np.isclose(g[7], (gP[mv].astype(np.float64) * rz[mv]).sum())
    assert np.all(g[:6] == 0)
