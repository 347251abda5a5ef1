"""Shared test helpers (no method arithmetic): error metric and fixtures."""

import numpy as np


def floored_rel_err(a, ref, n_qubits, floor=0.1):
    """Per-amplitude error |a - ref| / max(|ref|, floor * rms), maximised.

    rms is taken over the amplitudes of the call; for a single amplitude it is
    2^(-n/2), the Porter-Thomas mean magnitude of an n-qubit amplitude. With
    the default floor 0.1, amplitudes at or above a tenth of the rms are held
    to a relative bound and smaller ones to the same bound relative to 0.1 rms
    (their relative error is ill-conditioned: near-zero amplitudes are common
    under Porter-Thomas statistics)."""
    a = np.asarray(a).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    if ref.size == 1:
        rms = 2.0 ** (-n_qubits / 2)
    else:
        rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
    den = np.maximum(np.abs(ref), floor * rms)
    return float(np.max(np.abs(a - ref) / den))
