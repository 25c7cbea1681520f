"""GPU-vs-oracle comparison at the tolerances of the renderer's contract.

  coverage / segmentation: bit-exact, except pixels whose two nearest oracle
      fragments are within 1e-6 relative in depth (ties); those are counted
      and must stay under 0.01% of the pixels
  depth: 1e-6 relative (the kernels compute it bit-identically in practice)
  rgb_linear: 1e-4 absolute;  rgb8: 1 LSB;  normal: 1 binary16 ulp per component
"""

import numpy as np

TIE_REL = 1e-6
MAX_TIE_FRACTION = 1e-4


def f16_ordered(bits):
    b = bits.astype(np.int32)
    mag = b & 0x7FFF
    return np.where(b & 0x8000, -mag, mag)


def compare(gpu, orc, label=""):
    """Assert the contract; returns a dict of statistics."""
    N = len(orc["seg"])
    d1 = orc["depth"].astype(np.float64)
    d2 = orc["depth2"].astype(np.float64)
    tie = np.isfinite(d2) & (d1 > 0) & (np.abs(d2 - d1) <= TIE_REL * d1)
    seg_bad = gpu["seg"] != orc["seg"]
    depth_bad = np.abs(gpu["depth"].astype(np.float64) - d1) > TIE_REL * np.abs(d1)
    flip = seg_bad | depth_bad
    untied = flip & ~tie
    stats = dict(pixels=N, ties=int(tie.sum()), flips=int(flip.sum()), depth_exact=float((gpu["depth"] == orc["depth"]).mean()))
    assert untied.sum() == 0, f"{label}: {int(untied.sum())} coverage/depth mismatches outside ties " \
                              f"(first at {np.nonzero(untied)[0][:5]})"
    assert flip.sum() <= MAX_TIE_FRACTION * N + 0.5, f"{label}: {int(flip.sum())} tie flips of {N}"
    ok = ~flip
    if "rgb_linear" in gpu and "rgb_linear" in orc:
        e = np.abs(gpu["rgb_linear"][ok].astype(np.float64) - orc["rgb_linear"][ok])
        stats["rgb_linear_max_err"] = float(e.max()) if e.size else 0.0
        assert stats["rgb_linear_max_err"] <= 1e-4, f"{label}: rgb_linear error {stats['rgb_linear_max_err']}"
    e8 = np.abs(gpu["rgb"][ok].astype(np.int32) - orc["rgb"][ok].astype(np.int32))
    stats["rgb8_max_err"] = int(e8.max()) if e8.size else 0
    assert stats["rgb8_max_err"] <= 1, f"{label}: rgb8 error {stats['rgb8_max_err']}"
    en = np.abs(f16_ordered(gpu["normal"][ok]) - f16_ordered(orc["normal"][ok]))
    stats["normal_max_ulp"] = int(en.max()) if en.size else 0
    assert stats["normal_max_ulp"] <= 1, f"{label}: normal error {stats['normal_max_ulp']} ulp"
    return stats
