"""Discrete-ordinates direction sets (inputs: unit vectors ``s`` and weights ``w``).

* ``inplane(n)``: in-plane transport in a 2D material, ``n`` azimuths
  ``phi_k = (k + 1/2) 2 pi / n`` with equal weights ``2 pi / n`` (total 2 pi).
* ``gl_azimuth(n_pol, n_az)``: 3D product set, Gauss-Legendre nodes in
  ``mu = cos(theta)`` times uniform half-offset azimuths; total weight 4 pi.
* ``projected_3d_on_plane(n_pol_half, n_az)``: a 3D material on a 2D domain;
  half-range Gauss-Legendre nodes in ``mu`` in (0, 1), each standing for +mu
  and -mu (weights doubled), times uniform azimuths; total weight 4 pi.  Only
  the in-plane components of ``s`` enter a 2D domain's transport.

The half offset of the azimuths keeps every direction off axis-aligned walls,
and the sets map onto themselves under reflection in x-, y- and z-planes when
``n_az`` is a multiple of 4.
"""
from __future__ import annotations

import numpy as np


def inplane(n: int):
    phi = (np.arange(n) + 0.5) * 2.0 * np.pi / n
    s = np.stack([np.cos(phi), np.sin(phi), np.zeros(n)], axis=1)
    w = np.full(n, 2.0 * np.pi / n)
    return s, w


def gl_azimuth(n_pol: int, n_az: int):
    mu, wmu = np.polynomial.legendre.leggauss(n_pol)
    phi = (np.arange(n_az) + 0.5) * 2.0 * np.pi / n_az
    M, P = np.meshgrid(mu, phi, indexing="ij")
    WM = np.repeat(wmu[:, None], n_az, axis=1)
    st = np.sqrt(1.0 - M ** 2)
    s = np.stack([st * np.cos(P), st * np.sin(P), M], axis=-1).reshape(-1, 3)
    w = (WM * 2.0 * np.pi / n_az).reshape(-1)
    return s, w


def projected_3d_on_plane(n_pol_half: int, n_az: int):
    x, wx = np.polynomial.legendre.leggauss(n_pol_half)
    mu = 0.5 * (x + 1.0)          # nodes on (0, 1)
    wmu = 0.5 * wx * 2.0          # half-range weights, doubled for -mu
    phi = (np.arange(n_az) + 0.5) * 2.0 * np.pi / n_az
    M, P = np.meshgrid(mu, phi, indexing="ij")
    WM = np.repeat(wmu[:, None], n_az, axis=1)
    st = np.sqrt(1.0 - M ** 2)
    s = np.stack([st * np.cos(P), st * np.sin(P), M], axis=-1).reshape(-1, 3)
    w = (WM * 2.0 * np.pi / n_az).reshape(-1)
    return s, w
