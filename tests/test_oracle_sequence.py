"""Whole-pipeline properties of the oracle on the driving-shaped synthetic sequence."""
import json
import os

import numpy as np

import oracle
from paper_1708_06301_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_search_space.json")


def test_search_space_fraction_matches_paper_claim():
    """Sec. 3: the first frame searches the whole range (100%), later frames consider less than
    half of the search space (the paper reports 49.05 / 47.24 / 46.05 % on one KITTI scene)."""
    gold = json.load(open(GOLD))
    seq = synth.kitti_like(2, n_frames=3)
    prm = oracle.Params(1242, 375, d_max=127, census_w=9, census_h=7, n_paths=8)
    tr = oracle.Tracker(prm)
    full = 1242 * 375 * 128
    fr = []
    for k in range(3):
        o = tr.frame(seq.left[k], seq.right[k], seq.R[k], seq.t[k], seq.K, 0.54, keep=True)
        fr.append(100.0 * o["n_cells"] / full)
    assert fr[0] == gold["considered_percent_frames_0_to_3"][0]
    assert all(f < gold["claim_most_scenes_below_percent"] for f in fr[1:])
    # the paper's accuracy trend (Table 1): on the last frame the updated map has no more bad
    # pixels (error > 3 px, invalid counted as bad) than full-range SGM on the same images
    lo = np.zeros((375, 1242), np.int16)
    hi = np.full((375, 1242), 127, np.int16)
    Dz_full, _ = oracle.match(seq.left[2], seq.right[2], lo, hi, prm)
    gt = seq.gt_disp[2]

    def bad(d):
        return float(np.mean((d < 0) | (np.abs(d - gt) > 3)))

    assert bad(o["D"]) <= bad(Dz_full)
