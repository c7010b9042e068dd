"""Accuracy of the reduced search against full-range SGM on a longer driving sequence.

Sec. 3 (Table 1) reports the reduced search at least as accurate as plain SGM on every scene.
Here the kitti-shaped sequence is run for 30 frames twice through tsgm_frame: with the +-3 sigma
windows around the gap-filled prediction, and with every window the full range (prediction and
update as usual). The bad-3px rate of the updated map against the rendered ground truth
(|d - gt| > 3, invalid pixels counted bad) must be no worse with the reduced windows on every
frame, while the windows cover well under half of the range. Both runs equal the oracle
bit for bit (tests/test_gpu_sequence.py checks the first ten frames element by element), so this
is a property of the method with the readings taken here, checked on the GPU path.
"""
import numpy as np
import pytest

from paper_1708_06301_gb300 import synth

from gpu_util import dev, empty, f32, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_FRAMES = 30


@pytest.fixture(scope="module")
def tsgm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_06301_gb300 import tsgm as t
    t.load()
    return t


def _run(tsgm, seq, flags):
    W, H = seq.cam.W, seq.cam.H
    bad, frac = [], []
    with tsgm.Context(tsgm.default_params(W, H, flags=flags)) as ctx:
        D, P = empty((H, W), np.float32), empty((H, W), np.float32)
        for k in range(len(seq.left)):
            ctx.frame(dev(seq.left[k]), dev(seq.right[k]), seq.R[k], seq.t[k], seq.K,
                      f32(seq.cam.b), D, P)
            frac.append(ctx.cells() / (W * H * 128))
            d = host(D, np.float32)
            bad.append(float(np.mean((d < 0) | (np.abs(d - seq.gt_disp[k]) > 3))))
    return np.array(bad), np.array(frac)


@pytest.mark.slow
def test_reduced_no_worse_than_full_range_for_30_frames(tsgm):
    seq = synth.kitti_like(2, n_frames=N_FRAMES)
    bad_red, frac_red = _run(tsgm, seq, tsgm.FLAG_FILL_GAPS)
    bad_full, frac_full = _run(tsgm, seq, tsgm.FLAG_FULL_RANGE)
    assert np.all(frac_full == 1.0)
    assert frac_red[0] == 1.0 and np.all(frac_red[1:] < 0.5)
    # the per-frame table (shown with pytest -s)
    print("\nframe  searched  bad3px_reduced  bad3px_full")
    for k in range(N_FRAMES):
        print(f"{k + 1:5d}  {frac_red[k]:8.4f}  {100 * bad_red[k]:14.3f}  {100 * bad_full[k]:11.3f}")
    worse = [(k + 1, bad_red[k], bad_full[k]) for k in range(N_FRAMES) if bad_red[k] > bad_full[k]]
    assert not worse, f"frames where the reduced search is less accurate: {worse}"
