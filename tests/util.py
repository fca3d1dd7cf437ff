"""Comparison helpers shared by the tests (no solver arithmetic here)."""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def orth(X: np.ndarray) -> np.ndarray:
    q, _ = np.linalg.qr(X)
    return q


def max_subspace_angle(X: np.ndarray, Y: np.ndarray) -> float:
    """Largest principal angle (radians) between span(X) and span(Y)."""
    return float(np.max(sla.subspace_angles(X, Y))) if X.shape[1] else 0.0


def clusters(lam: np.ndarray, rel: float = 1e-8):
    """Group sorted eigenvalues whose gap is below rel*max(1,|lambda|)."""
    groups, cur = [], [0]
    for j in range(1, len(lam)):
        if abs(lam[j] - lam[j - 1]) < rel * max(1.0, abs(lam[j])):
            cur.append(j)
        else:
            groups.append(cur)
            cur = [j]
    groups.append(cur)
    return groups


def cluster_angles(lam_ref: np.ndarray, V_ref: np.ndarray, V: np.ndarray, rel: float = 1e-8):
    """Per-cluster largest principal angle between matching columns of V and V_ref.

    A cluster that is cut by the end of the block is compared as a whole anyway; callers
    should include a guard column if that matters.
    """
    out = []
    for g in clusters(lam_ref, rel):
        out.append(max_subspace_angle(V_ref[:, g], V[:, g]))
    return np.array(out)


def rel_eig_err(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


def golden(name: str = "paper_printed_values.json") -> dict:
    """A fixture of values printed in the paper (tests/golden/, each entry with its citation)."""
    import json
    import pathlib
    return json.loads((pathlib.Path(__file__).resolve().parent / "golden" / name).read_text())
