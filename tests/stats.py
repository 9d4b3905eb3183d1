"""Goodness-of-fit helpers shared by the statistical tests."""
from __future__ import annotations

import numpy as np
from scipy import stats as _st


def tv(counts, probs) -> float:
    """Total-variation distance between empirical counts and a probability vector."""
    counts = np.asarray(counts, dtype=np.float64)
    probs = np.asarray(probs, dtype=np.float64)
    return 0.5 * float(np.abs(counts / counts.sum() - probs / probs.sum()).sum())


def chisq_p(counts, probs, min_expected: float = 5.0) -> float:
    """Chi-square goodness-of-fit p-value; categories with small expectation are pooled."""
    counts = np.asarray(counts, dtype=np.float64)
    probs = np.asarray(probs, dtype=np.float64)
    probs = probs / probs.sum()
    exp = probs * counts.sum()
    order = np.argsort(exp)
    oc, oe = [], []
    acc_c = acc_e = 0.0
    for i in order:
        acc_c += counts[i]
        acc_e += exp[i]
        if acc_e >= min_expected:
            oc.append(acc_c)
            oe.append(acc_e)
            acc_c = acc_e = 0.0
    if acc_e > 0 or acc_c > 0:
        if oe:
            oc[-1] += acc_c
            oe[-1] += acc_e
        else:
            oc.append(acc_c)
            oe.append(acc_e)
    oc, oe = np.array(oc), np.array(oe)
    if len(oc) < 2:
        return 1.0
    stat = float(((oc - oe) ** 2 / oe).sum())
    return float(_st.chi2.sf(stat, len(oc) - 1))


def binned(counts, probs, max_bins: int = 1000):
    """Merge consecutive categories into at most max_bins bins with their exact masses."""
    counts = np.asarray(counts, dtype=np.float64)
    probs = np.asarray(probs, dtype=np.float64)
    k = len(counts)
    if k <= max_bins:
        return counts, probs
    edges = np.linspace(0, k, max_bins + 1).astype(np.int64)
    return np.add.reduceat(counts, edges[:-1]), np.add.reduceat(probs, edges[:-1])
