"""Synthetic re-runs of the paper's image-quality studies, on the GPU path.

The paper scores each thresholding rule, each subset grid and each packet
length by the contrast ratio and the contrast-to-noise ratio of the power-Doppler
image inside a blood region and a background region at similar depths
(CR = 10 log10(mean PD_blood / mean PD_background),
CNR = 10 log10((mean PD_blood - mean PD_background) / SD_background)), over packets
taken from a frame sequence with a sliding window, mean and SD over the packets
(the evaluation paragraph of its methods section, Figs. 4-10).  Here the frames
come from the seeded synthetic generator, whose vessel masks are known, so the
regions need no drawing: the blood region is the vessels shrunk by one pixel, the
background every pixel at least ``margin`` pixels from any vessel within the rows
the blood region spans.

Every filter runs in the CUDA library (lcf_filter_stream: all packets of a
sequence as one graph launch); this module only chooses configurations, scores
the images and tabulates.
"""
from __future__ import annotations

import numpy as np

from . import (LCF_T_ADAPTIVE_SOFT, LCF_T_CURVATURE, LCF_T_MEDIAN, LCF_T_NCC, LCF_T_NONE, LCF_T_SIGMOID, LCF_T_SLOPE,
               Plan)

# scaling-factor ranges swept per rule (the paper sweeps each rule's factor and keeps the best)
BETAS = {
    LCF_T_CURVATURE: (0.05, 0.1, 0.15, 0.25, 0.5, 1.0, 2.0),
    LCF_T_SLOPE: (0.5, 1.0, 1.5, 2.0, 3.0, 4.0),
    LCF_T_MEDIAN: (1.43, 3.0, 10.0, 30.0, 100.0, 300.0, 1000.0),
    LCF_T_SIGMOID: (0.5, 1.0, 2.0, 4.0),          # sigmoid sharpness at method 4's cutoff
    LCF_T_ADAPTIVE_SOFT: (0.1, 0.25, 0.5, 0.75, 1.0),
    LCF_T_NCC: (1.0,),                            # method 4 has no factor
}
RULE_NAMES = {LCF_T_NONE: "no filtering", LCF_T_CURVATURE: "method 1 (curvature)", LCF_T_SLOPE: "method 2 (slope)",
              LCF_T_MEDIAN: "method 3 (median)", LCF_T_NCC: "method 4 (NCC)",
              LCF_T_SIGMOID: "method 5 (sigmoid at method 4's k)", LCF_T_ADAPTIVE_SOFT: "method 6 (adaptive soft)"}


def _erode(m):
    out = m.copy()
    out[1:, :] &= m[:-1, :]
    out[:-1, :] &= m[1:, :]
    out[:, 1:] &= m[:, :-1]
    out[:, :-1] &= m[:, 1:]
    return out


def _dilate(m, r):
    out = m.copy()
    for _ in range(r):
        d = out.copy()
        d[1:, :] |= out[:-1, :]
        d[:-1, :] |= out[1:, :]
        d[:, 1:] |= out[:, :-1]
        d[:, :-1] |= out[:, 1:]
        out = d
    return out


def rois(blood_mask, margin: int = 3):
    """(blood ROI, background ROI) boolean images from the true vessel mask."""
    blood = _erode(np.asarray(blood_mask, bool))
    if not blood.any():
        blood = np.asarray(blood_mask, bool)
    rows = np.nonzero(blood.any(axis=1))[0]
    band = np.zeros_like(blood)
    if rows.size:
        band[rows.min():rows.max() + 1, :] = True
    bg = band & ~_dilate(np.asarray(blood_mask, bool), margin)
    return blood, bg


def cr_cnr(pd, blood, bg):
    """The paper's contrast ratio and contrast-to-noise ratio (dB) of one PD image;
    CNR is NaN when the blood mean does not exceed the background mean."""
    pd = np.asarray(pd, np.float64)
    mb, mg = float(pd[blood].mean()), float(pd[bg].mean())
    sg = float(pd[bg].std())
    cr = 10.0 * np.log10(mb / mg) if mb > 0 and mg > 0 else float("nan")
    cnr = 10.0 * np.log10((mb - mg) / sg) if mb > mg and sg > 0 else float("nan")
    return cr, cnr


def score_sequence(frames, blood_mask, nt, stride, grid, rule, beta, device=0, margin=3, **cfg):
    """Filter every packet of ``frames`` (nt frames every ``stride``) with one configuration:
    CR and CNR mean and SD over the packets and the GPU time per packet (ms).  grid (1, 1)
    is the paper's global processing (one window covering the image, g = 1)."""
    import torch
    nf, nz, nx = frames.shape
    kw = dict(thresh_mode=rule, beta=float(beta), device=device)
    if rule == LCF_T_SIGMOID:
        kw.update(k_src=LCF_T_NCC)
    if tuple(grid) == (1, 1):
        kw.update(all_ones_window=1)
    kw.update(cfg)
    plan = Plan.make(nz, nx, nt, grid[0], grid[1], **kw)
    d = frames if torch.is_tensor(frames) else torch.from_numpy(np.ascontiguousarray(frames)).to(f"cuda:{device}")
    out = plan.filter_stream(d, stride)          # capture
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = plan.filter_stream(d, stride, out)
    e1.record()
    torch.cuda.synchronize()
    npk = out.shape[0]
    blood, bg = rois(blood_mask, margin)
    pds = out.cpu().numpy()
    sc = np.array([cr_cnr(p, blood, bg) for p in pds])
    plan.close()
    return {"cr": float(np.nanmean(sc[:, 0])), "cr_sd": float(np.nanstd(sc[:, 0])),
            "cnr": float(np.nanmean(sc[:, 1])), "cnr_sd": float(np.nanstd(sc[:, 1])),
            "ms_per_packet": e0.elapsed_time(e1) / npk, "packets": int(npk)}


def beta_sweep(frames, blood_mask, nt, stride, grid, rule, betas=None, **kw):
    """CR / CNR against the rule's scaling factor (the paper's Figs. 4d, 6d, 8d)."""
    rows = []
    for b in (betas if betas is not None else BETAS[rule]):
        r = score_sequence(frames, blood_mask, nt, stride, grid, rule, b, **kw)
        r["beta"] = float(b)
        rows.append(r)
    return rows


def best_of(rows):
    """The maximum achievable CR and CNR over a sweep (each at its own factor)."""
    cr = max(rows, key=lambda r: -np.inf if np.isnan(r["cr"]) else r["cr"])
    cnr = max(rows, key=lambda r: -np.inf if np.isnan(r["cnr"]) else r["cnr"])
    return {"cr": cr["cr"], "cr_beta": cr["beta"], "cnr": cnr["cnr"], "cnr_beta": cnr["beta"],
            "ms_per_packet": float(np.mean([r["ms_per_packet"] for r in rows]))}


def subset_study(frames, blood_mask, nt, stride, grids=((1, 1), (2, 2), (3, 3), (8, 8)), rules=None, **kw):
    """Maximum achievable CR / CNR per rule and subset grid, with the GPU time per packet
    (the paper's Figs. 5, 7, 9 d-f)."""
    table = {}
    for rule in (rules if rules is not None else BETAS):
        for g in grids:
            table[(RULE_NAMES[rule], f"{g[0]}x{g[1]}")] = best_of(
                beta_sweep(frames, blood_mask, nt, stride, g, rule, **kw))
    return table


def packet_size_study(make_frames, nts=(50, 70, 90), stride=5, grids=((1, 1), (3, 3)), rule=LCF_T_CURVATURE, **kw):
    """Maximum achievable CR / CNR and time per packet against the packet length (Fig. 10);
    make_frames(nt) -> (frames, blood_mask) gives a sequence long enough for the packets."""
    table = {}
    for nt in nts:
        frames, mask = make_frames(nt)
        for g in grids:
            table[(nt, f"{g[0]}x{g[1]}")] = best_of(beta_sweep(frames, mask, nt, stride, g, rule, **kw))
    return table
