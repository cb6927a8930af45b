"""The test helper that finds Gaussians composited differently by two
projections of one scene (CPU)."""
import numpy as np

import gs_inputs as gi
import oracle as O
from flips import decision_flips


def test_decision_flips_finds_a_planted_threshold_crossing():
    sc = gi.make_scene(200, 0, 9)
    sc[1, :, :3] += 1.0
    cams = gi.ring_cameras(1, 48, 48)
    f = O.forward(sc, 0, cams)
    flags, npix = decision_flips(cams, f["proj"], f["vals"], f["ranges"], f["proj"], f["vals"], f["ranges"])
    assert npix == 0 and not flags.any()
    # move one visible Gaussian's opacity so that one fragment crosses 1/255
    p2 = f["proj"].copy()
    g = int(np.nonzero(p2[0, :, 14] > p2[0, :, 12])[0][0])
    p2[0, g, 3] *= 0.5
    flags, npix = decision_flips(cams, f["proj"], f["vals"], f["ranges"], p2, f["vals"], f["ranges"])
    assert npix > 0 and flags[0, g]
