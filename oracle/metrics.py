"""Accuracy measures for central eigenvalues (oracle side, test infrastructure).

* relative error eta = |E - E_exact| / |E_exact| (Sec. III, Fig. 2);
* error in units of the local mean level spacing: the mean of the exact
  spacings over the +-10 levels around the matched exact level;
* matching: each computed value is paired with the nearest exact level; a
  level used twice or a value with no level within half a local spacing is
  reported as unmatched.
"""

from __future__ import annotations

import numpy as np


def central_exact(spectrum, n: int) -> np.ndarray:
    """The n exact levels of smallest |E|, ascending."""
    spectrum = np.sort(np.asarray(spectrum))
    order = np.argsort(np.abs(spectrum), kind="stable")[:n]
    return np.sort(spectrum[order])


def local_spacing(spectrum, idx: int, half: int = 10) -> float:
    sp = np.asarray(spectrum)
    lo = max(0, idx - half)
    hi = min(len(sp) - 1, idx + half)
    return float((sp[hi] - sp[lo]) / max(1, hi - lo))


def match(computed, spectrum):
    """Pair computed values with exact levels.

    Returns dict with abs_err, spacing_err (error / local mean spacing), idx
    (exact index per computed value) and n_unmatched.
    """
    sp = np.sort(np.asarray(spectrum))
    comp = np.sort(np.asarray(computed))
    pos = np.clip(np.searchsorted(sp, comp), 1, len(sp) - 1)
    left = sp[pos - 1]
    right = sp[pos]
    idx = np.where(np.abs(comp - left) <= np.abs(comp - right), pos - 1, pos)
    abs_err = np.abs(comp - sp[idx])
    spc = np.array([local_spacing(sp, i) for i in idx])
    used, counts = np.unique(idx, return_counts=True)
    dup = int((counts > 1).sum())
    far = int((abs_err > 0.5 * spc).sum())
    return {"abs_err": abs_err, "spacing_err": abs_err / spc, "idx": idx,
            "n_unmatched": dup + far}
