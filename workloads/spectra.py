"""Seeded band tables ``(C, v, tau)`` standing in for first-principles spectra.

Units: C in J/(m^3 K), v in m/s, tau in s.
"""
from __future__ import annotations

import numpy as np

C_SILICON = 1.66e6  # J/(m^3 K), total heat capacity used for the synthetic spectra


def gray(C: float = C_SILICON, v: float = 6000.0, tau: float = 16.7e-12):
    return (np.array([C], dtype=np.float64), np.array([v], dtype=np.float64),
            np.array([tau], dtype=np.float64))


def _weights(rng, B, total):
    cw = rng.uniform(0.5, 1.5, size=B)
    return cw / cw.sum() * total


def silicon_like(B: int, seed: int, C_total: float = C_SILICON,
                 v_range=(1e3, 8e3), tau_range=(1e-12, 1e-8)):
    """Group velocity uniform in ``v_range``, relaxation time log-uniform in
    ``tau_range``, heat-capacity weights uniform in [0.5, 1.5] normalised to
    ``C_total``."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(*v_range, size=B)
    tau = np.exp(rng.uniform(np.log(tau_range[0]), np.log(tau_range[1]), size=B))
    C = _weights(rng, B, C_total)
    return C, v, tau


def knudsen_spread(B: int, seed: int, mfp_range=(5e-9, 500e-9), C_total: float = C_SILICON,
                   v_range=(1e3, 8e3)):
    """Velocity uniform in ``v_range``; mean free path log-uniform in
    ``mfp_range`` (so Kn spans a chosen window for a given length);
    ``tau = mfp / v``."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(*v_range, size=B)
    mfp = np.exp(rng.uniform(np.log(mfp_range[0]), np.log(mfp_range[1]), size=B))
    C = _weights(rng, B, C_total)
    return C, v, mfp / v
