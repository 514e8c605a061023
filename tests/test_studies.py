"""The image-quality scores of the paper's studies (CR and CNR, its evaluation paragraph) on
hand-made images (CPU), and one small synthetic study through the GPU path."""
import numpy as np
import pytest

from conftest import gpu_available


def studies():
    import importlib
    import sys
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    return importlib.import_module("paper_2405_11105_b300.studies")


def test_cr_cnr_closed_form():
    """Blood 4 and 6 (mean 5), background 1 and 3 (mean 2, SD 1): CR = 10 log10(5/2),
    CNR = 10 log10((5 - 2) / 1)."""
    pytest.importorskip("torch")
    try:
        S = studies()
    except ImportError:
        pytest.skip("library not built")
    pd = np.array([[4.0, 6.0, 1.0, 3.0]])
    blood = np.array([[True, True, False, False]])
    bg = ~blood
    cr, cnr = S.cr_cnr(pd, blood, bg)
    assert cr == pytest.approx(10 * np.log10(2.5), rel=1e-14)
    assert cnr == pytest.approx(10 * np.log10(3.0), rel=1e-14)
    cr, cnr = S.cr_cnr(np.array([[1.0, 1.0, 2.0, 4.0]]), blood, bg)   # background brighter: no CNR
    assert cr < 0 and np.isnan(cnr)


def test_rois_geometry():
    try:
        S = studies()
    except ImportError:
        pytest.skip("library not built")
    m = np.zeros((20, 20), bool)
    m[8:12, 5:15] = True                    # a 4-row vessel
    blood, bg = S.rois(m, margin=3)
    assert blood.sum() == 2 * 8             # shrunk by one pixel on every side
    assert not (bg & m).any()
    rows = np.nonzero(bg.any(axis=1))[0]
    assert rows.min() == 9 and rows.max() == 10     # background at the blood region's depths
    cols = set(np.nonzero(bg[9])[0].tolist())
    assert cols == {0, 1, 18, 19}           # three pixels of margin around the vessel


@pytest.mark.gpu
@pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")
def test_small_study_on_the_gpu():
    """A 96 x 96 sequence with laterally varying motion: every rule's best CR beats the
    unfiltered image by 3 dB, and method 6's CR has its maximum inside its factor sweep."""
    import paper_2405_11105_b300 as L
    S = studies()
    from synth import Recipe, generate_frames
    rec = Recipe(96, 96, 40, n_vessels=4, width_px=(3.0, 6.0), phi_rad=(0.1, 0.8), tbr_db=40.0, noise_db=-60.0,
                 motion_amp_px=1.0, motion_period=30.0, motion_lateral_gain=(0.2, 2.0))
    frames, truth = generate_frames(rec, 40 + 4 * 5, seed=3, return_truth=True)
    mask = truth["blood_mask"]
    base = S.score_sequence(frames, mask, 40, 5, (1, 1), L.LCF_T_NONE, 1.0)
    table = S.subset_study(frames, mask, 40, 5, grids=((1, 1), (2, 2)),
                           rules=(L.LCF_T_CURVATURE, L.LCF_T_MEDIAN, L.LCF_T_NCC, L.LCF_T_ADAPTIVE_SOFT))
    for key, row in table.items():
        print(key, {k: round(v, 3) for k, v in row.items()})
        assert np.isfinite(row["cr"]) and row["cr"] >= base["cr"] + 3.0, (key, row, base)
    sweep = S.beta_sweep(frames, mask, 40, 5, (1, 1), L.LCF_T_ADAPTIVE_SOFT)
    crs = [r["cr"] for r in sweep]
    print("unfiltered CR", base["cr"], "method 6 sweep", crs)
    assert 0 < int(np.argmax(crs)) < len(crs) - 1
