"""Error norms used to report accuracy."""
import numpy as np


def gre(phi, ref) -> float:
    """Global relative error, sum|phi - phi*| / sum|phi*| (Eq. 63)."""
    phi = np.asarray(phi, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.abs(phi - ref).sum() / np.abs(ref).sum())


def rel_l2(phi, ref) -> float:
    """||phi - ref||_2 / ||ref||_2."""
    phi = np.asarray(phi, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((phi - ref).ravel()) / np.linalg.norm(ref.ravel()))
