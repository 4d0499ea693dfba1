"""Pins that tie the FP64 oracle to something other than itself.

Each test names what the paper or mathematics fixes and which plausible
mistake in the oracle it would expose.  Nothing here touches a GPU.
"""
import numpy as np
import pytest

import workloads as W
from workloads.problems import Boundary, Problem, THERMALIZING, DIFFUSE, SPECULAR, PARTIAL
from oracle import OracleSolver, quadrature_moments

from bruteforce import solve_fixed_point
from cases import CASES


# ----------------------------------------------------------------------------- I1
@pytest.mark.parametrize("kind,args,W_expect,second", [
    ("inplane", (16,), 2 * np.pi, np.diag([np.pi, np.pi, 0.0])),
    ("gl_azimuth", (8, 16), 4 * np.pi, np.eye(3) * 4 * np.pi / 3),
    ("gl_azimuth", (10, 20), 4 * np.pi, np.eye(3) * 4 * np.pi / 3),
    ("projected_3d_on_plane", (4, 16), 4 * np.pi, np.eye(3) * 4 * np.pi / 3),
])
def test_quadrature_moments(kind, args, W_expect, second):
    """Eq. (11): W_Omega = sum_i w_i is the full solid angle (2 pi in-plane,
    4 pi for 3D sets); the first moment vanishes and the second is isotropic.
    A wrong weight or a dropped half of the polar range fails here."""
    s, w = getattr(W.quadrature, kind)(*args)
    W0, W1, W2 = quadrature_moments(s, w)
    assert W0 == pytest.approx(W_expect, rel=1e-13)
    # the projected set stores +mu only (each node stands for +-mu), so only its
    # in-plane first moment is meaningful
    k = 2 if kind == "projected_3d_on_plane" else 3
    assert np.abs(W1[:k]).max() < 1e-12
    assert np.abs(W2 - second).max() < 1e-12
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)


@pytest.mark.parametrize("kind,args", [("inplane", (16,)), ("gl_azimuth", (8, 16)),
                                       ("projected_3d_on_plane", (4, 16))])
def test_quadrature_reflection_closure(kind, args):
    """Specular walls need the mirror image of every direction in the set for
    axis-aligned walls; the half-offset azimuths give that exactly."""
    s, w = getattr(W.quadrature, kind)(*args)
    for n in np.eye(3):
        if kind != "gl_azimuth" and n[2] == 1.0:
            continue
        mirror = s - 2.0 * (s @ n)[:, None] * n[None, :]
        d = np.min(np.sum((mirror[:, None] - s[None]) ** 2, axis=2), axis=1)
        assert d.max() < 1e-24


# ----------------------------------------------------------------------------- I4
def _ballistic_square(n_dirs=16, nx=20):
    return W.problems.square_inplane(n=nx, n_dirs=n_dirs, tau=1e-3)


@pytest.mark.parametrize("n_dirs", [8, 16, 32])
def test_ballistic_gray_slab_closed_form(n_dirs):
    """Ballistic limit (Kn ~ 6e7) of the in-plane square with thermalizing
    left/right walls and specular top/bottom (Sec. III A): every interior cell
    sits at the mean wall temperature (a jump of dT/2 at each wall) and the flux
    is q_x = C v dT sum_{s_x>0} w s_x / W = C v dT / (n sin(pi/n)) for the
    n-direction in-plane set.  A swapped upwind side, a wrong specular map or a
    wrong weight changes one of them."""
    p = _ballistic_square(n_dirs)
    r = OracleSolver(p).solve(tol=1e-13, max_iter=50)
    dT = p.meta["T_left"] - p.meta["T_right"]
    assert np.abs(r["T"] - 0.5 * (p.meta["T_left"] + p.meta["T_right"])).max() < 1e-6 * dT
    q_exact = p.C[0] * p.v[0] * dT / (n_dirs * np.sin(np.pi / n_dirs))
    assert np.abs(r["q"][:, 0] / q_exact - 1.0).max() < 1e-6
    assert np.abs(r["q"][:, 1]).max() < 1e-9 * q_exact


# ----------------------------------------------------------------------------- I6
def test_square_symmetries():
    """Specular top/bottom make the square a 1D problem (rows identical) and
    301/299 K walls around 300 K make T' antisymmetric in x; the wall heat
    flows balance.  An index or transposition slip breaks one of these."""
    p = W.problems.square_inplane()
    r = OracleSolver(p).solve()
    T = r["T"].reshape(40, 40) - 300.0
    assert np.abs(T - T[:1]).max() < 1e-10
    assert np.abs(T + T[:, ::-1]).max() < 1e-10
    f = r["wall_flux"]
    assert abs(f[1] + f[2]) < 1e-10 * abs(f[1])
    assert abs(f[3]) < 1e-10 * abs(f[1]) and abs(f[4]) < 1e-10 * abs(f[1])
    # L = MFP sits between the ballistic profile (T' = 0 in the first cell) and
    # the diffusive one (T' = 1 - 1/40 at the first cell centre)
    assert 0.1 < T[0, 0] < 1.0 - 1.0 / 40


# ----------------------------------------------------------------------------- I2
def _uniform_variants():
    out = []
    p = W.problems.square_inplane(n=4, n_dirs=8)
    p.boundaries = [Boundary(1, THERMALIZING, 303.0), Boundary(2, DIFFUSE),
                    Boundary(3, SPECULAR, 0.0, 1.0), Boundary(4, PARTIAL, 0.0, 0.4)]
    out.append(p)
    p = W.problems.finfet2d(h=25e-9, B=3, n_pol_half=2, n_az=8, q_peak=0.0)
    p.boundaries = [Boundary(1, THERMALIZING, 303.0), Boundary(2, DIFFUSE), Boundary(3, SPECULAR, 0, 1),
                    Boundary(4, PARTIAL, 0.0, 0.5), Boundary(5, DIFFUSE)]
    p.Q = None
    out.append(p)
    p = W.problems.finfet3d(h=40e-9, B=2, n_pol=2, n_az=8, q_fin=0.0)
    for b in p.boundaries:
        if b.type == THERMALIZING:
            b.T_wall = 303.0
    p.Q = None
    out.append(p)
    p = W.problems.cube3d(n=3, B=2, n_pol=2, n_az=8, T_hot=303.0, T_cold=303.0)
    out.append(p)
    return out


@pytest.mark.parametrize("k", range(4))
def test_uniform_wall_temperature_is_exact_fixed_point(k):
    """All thermalizing walls at T_w and no heat source: the exact solution is
    T = T_w everywhere with zero flux, on every mesh type and wall mix.  From
    T_init = T_w one sweep reproduces it; from T_ref the iteration reaches it.
    A wrong C/W normalisation, source split or wall formula breaks it."""
    p = _uniform_variants()[k]
    o = OracleSolver(p)
    r1 = o.solve(n_iter=1, T_init=np.full(p.n_cells, 303.0))
    assert np.abs(r1["T"] - 303.0).max() < 1e-11
    qs = p.C.sum() * p.v.max() * 3.0
    assert np.abs(r1["q"]).max() < 1e-11 * qs
    r = o.solve(scheme="synthetic", tol=1e-12, max_iter=3000)
    assert r["converged"]
    assert np.abs(r["T"] - 303.0).max() < 1e-9


# ----------------------------------------------------------------------------- I3
@pytest.mark.parametrize("which", ["tri", "tet"])
def test_energy_conservation(which):
    """At convergence the net heat leaving through the thermalizing walls
    equals the integrated volumetric source (Sec. III B: the source enters as
    equilibrium phonons, uniform over directions, split by heat capacity), and
    diffuse/specular walls carry no net heat.  A dropped 1/W or C_l/C_tot in the
    source, or a sign slip in the wall flux, fails it."""
    if which == "tri":
        p = W.problems.finfet2d(h=10e-9, B=3, n_pol_half=2, n_az=8, sigma=15e-9)
    else:
        p = W.problems.finfet3d(h=25e-9, B=2, n_pol=2, n_az=8)
    o = OracleSolver(p)
    r = o.solve(scheme="synthetic", tol=1e-12, max_iter=3000)
    assert r["converged"]
    assert r["Q_total"] > 0
    assert r["energy_imbalance"] < 1e-9
    for t, f in r["wall_flux"].items():
        kinds = {b.tag: b.type for b in p.boundaries}
        if kinds[t] != THERMALIZING:
            assert abs(f) < 1e-9 * r["Q_total"]


# ----------------------------------------------------------------------------- I7
def _tiny_cases():
    cases = []
    p = W.problems.square_inplane(n=3, ny=2, n_dirs=8, tau=5e-12)
    p.boundaries = [Boundary(1, THERMALIZING, 302.0), Boundary(2, THERMALIZING, 299.0),
                    Boundary(3, DIFFUSE), Boundary(4, SPECULAR, 0, 1)]
    p.Q = np.linspace(0, 3e17, p.n_cells)
    cases.append(p)
    p = W.problems.square_inplane(n=3, n_dirs=8)
    p.C, p.v, p.tau = np.array([1e6, 6e5]), np.array([6e3, 2e3]), np.array([10e-12, 40e-12])
    p.boundaries = [Boundary(1, THERMALIZING, 302.0), Boundary(2, PARTIAL, 0, 0.3),
                    Boundary(3, DIFFUSE), Boundary(4, SPECULAR, 0, 1)]
    p.Q = np.full(p.n_cells, 1e17)
    cases.append(p)
    p = W.problems.finfet2d(h=50e-9, B=2, n_pol_half=2, n_az=8, sigma=20e-9)
    p.boundaries = [Boundary(1, THERMALIZING, 300.5), Boundary(2, DIFFUSE), Boundary(3, SPECULAR, 0, 1),
                    Boundary(4, PARTIAL, 0, 0.5), Boundary(5, DIFFUSE)]
    cases.append(p)
    p = W.problems.finfet3d(h=60e-9, B=1, n_pol=2, n_az=8)
    cases.append(p)
    p = W.problems.cube3d(n=2, B=2, n_pol=2, n_az=4)
    cases.append(p)
    return cases


@pytest.mark.parametrize("k", range(5))
def test_fixed_point_equals_dense_direct_solve(k):
    """The iteration's limit is the solution of one linear system (every
    (cell, band, direction) balance with T' eliminated and every wall written
    in terms of the current distribution).  A plain-loop dense assembly with
    its own geometry, solved by LAPACK, must agree with the oracle's converged
    field: this catches any dropped term, sign, index or transposed operand in
    the transport, source, moment or wall arithmetic."""
    p = _tiny_cases()[k]
    r = OracleSolver(p).solve(scheme="synthetic", tol=1e-14, max_iter=5000)
    assert r["converged"]
    TL, q = solve_fixed_point(p)
    dev = np.abs(TL - p.T_ref).max()
    assert np.abs(r["T"] - TL).max() < 1e-10 * dev
    assert np.abs(r["q"] - q).max() < 1e-9 * np.abs(q).max()


# ----------------------------------------------------------------------------- I8
def test_sequential_and_synthetic_reach_same_field():
    """Both schemes share one fixed point; the DSA form of the synthetic update
    (the default) on a ballistic-dominated 2D fin."""
    p = W.problems.finfet2d(h=12e-9, B=4, n_pol_half=2, n_az=8, sigma=10e-9)
    o = OracleSolver(p)
    a = o.solve(scheme="sequential", tol=1e-13, max_iter=20000)
    b = o.solve(scheme="synthetic", tol=1e-13, max_iter=20000)
    dev = np.abs(a["T"] - 300).max()
    assert a["converged"] and b["converged"]
    assert np.abs(a["T"] - b["T"]).max() < 1e-10 * dev


def test_literal_synthetic_same_fixed_point():
    """The literal form of Eq. (9) (gradient at T^n) converges where the
    correction dominates (Kn 0.01-1 cube) and to the same field; it stalls in
    the ballistic regime, which is why the DSA form is the default."""
    p = W.problems.cube3d(n=6, B=3, n_pol=2, n_az=8)
    o = OracleSolver(p)
    a = o.solve(scheme="sequential", tol=1e-13, max_iter=20000)
    c = o.solve(scheme="synthetic_literal", tol=1e-13, max_iter=20000)
    b = o.solve(scheme="synthetic", tol=1e-13, max_iter=20000)
    dev = np.abs(a["T"] - 300).max()
    assert a["converged"] and b["converged"] and c["converged"]
    assert b["iterations"] < a["iterations"] / 4
    assert np.abs(a["T"] - c["T"]).max() < 1e-10 * dev
    assert np.abs(a["T"] - b["T"]).max() < 1e-10 * dev


# ----------------------------------------------------------------------------- I9
def test_face_divergence_identity():
    """Summing the discrete balance of Eq. (4) over bands and directions:
    Qdot V - div_h q = V beta (T'_L - T'^n) per cell, every iteration, when
    div_h q uses the sweep's own upwind face values (the identity that lets the
    synthetic right-hand side of Eq. (10) be formed from T_L)."""
    p = W.problems.finfet2d(h=20e-9, B=2, n_pol_half=2, n_az=8, sigma=15e-9)
    o = OracleSolver(p)
    T = np.zeros(p.n_cells) + 0.3
    eb = o.equilibrium_walls(T)
    for _ in range(3):
        out = o.sweep(T, eb, store_e=True)
        div = o.face_divergence(out["e"], out["e_in"])
        TL = out["NL"] / o.beta
        lhs = o.Qdot * o.g.V - div
        rhs = o.g.V * o.beta * (TL - T)
        assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(rhs).max()
        T, eb = TL, out["eb"]


# ----------------------------------------------------------------------------- scaling
def test_knudsen_scaling_invariance():
    """Scaling every length and every tau by a (fixed Knudsen numbers) and the
    heat source by 1/a leaves the steady temperature unchanged exactly; a length
    or volume entering a coefficient with the wrong power breaks it."""
    base = W.problems.finfet2d(h=20e-9, B=2, n_pol_half=2, n_az=8, sigma=15e-9)
    a = 7.0
    big = W.problems.finfet2d(h=20e-9, B=2, n_pol_half=2, n_az=8, sigma=15e-9)
    big.mesh.nodes = big.mesh.nodes * a
    big.tau = big.tau * a
    big.Q = base.Q / a
    r0 = OracleSolver(base).solve(scheme="synthetic", tol=1e-13, max_iter=3000)
    r1 = OracleSolver(big).solve(scheme="synthetic", tol=1e-13, max_iter=3000)
    dev = np.abs(r0["T"] - 300).max()
    assert np.abs(r0["T"] - r1["T"]).max() < 1e-9 * dev


def test_fourier_limit_scaling_eq15():
    """Eq. (15): in the diffusive limit the rise is dT ~ Q L^2 / kappa, so
    doubling every length and cutting Q by 4 keeps the rise (the paper's
    scaling of its device sizes).  Square with thermalizing walls, resolved
    cells (h = mfp/2): the scaled rise dT kappa / (Q L^2) settles as Kn drops."""
    from workloads.problems import THERMALIZING
    v, tau = 6000.0, 1e-12
    mfp = v * tau
    ratios = []
    for l_over_mfp in (10, 20, 40):
        L = l_over_mfp * mfp
        p = W.problems.square_inplane(n=2 * l_over_mfp, n_dirs=8, tau=tau, v=v,
                                      T_left=300.0, T_right=300.0)
        p.mesh.nodes = p.mesh.nodes * (L / 100e-9)
        p.boundaries = [Boundary(t, THERMALIZING, 300.0) for t in (1, 2, 3, 4)]
        Q = 1e18 * (20 * mfp / L) ** 2
        p.Q = np.full(p.n_cells, Q)
        r = OracleSolver(p).solve(scheme="synthetic", tol=1e-10, max_iter=300)
        assert r["converged"]
        kappa = p.C[0] * v * mfp / 2.0
        ratios.append((r["T"].max() - 300.0) * kappa / (Q * L ** 2))
    d1 = abs(ratios[1] / ratios[0] - 1.0)
    d2 = abs(ratios[2] / ratios[1] - 1.0)
    assert d2 < d1 and d2 < 0.12
    # same order as the continuum Dirichlet-square value 0.0737
    assert 0.04 < ratios[2] < 0.09


# ----------------------------------------------------------------------------- I5
def test_diffusive_limit_linear_profile():
    """Near the diffusive limit (Kn = 0.025) the profile between the
    thermalizing walls is linear away from the walls (Sec. III A, the 100 um
    case), with a small jump at each wall, and the flux is within a few per
    cent of C v dT / (pi + 2 L / mfp) for the in-plane gray medium (the
    interpolation that is exact in both the ballistic and diffusive limits)."""
    v, tau = 6000.0, 1e-12
    mfp = v * tau
    L = 40 * mfp
    n = 80
    p = W.problems.square_inplane(n=n, n_dirs=16, tau=tau, v=v)
    p.mesh.nodes = p.mesh.nodes * (L / 100e-9)
    r = OracleSolver(p).solve(scheme="synthetic", tol=1e-11, max_iter=300)
    assert r["converged"]
    T = r["T"].reshape(n, n)[0]
    xs = np.arange(n)
    core = slice(n // 4, n - n // 4)
    fit = np.polyfit(xs[core], T[core], 1)
    assert np.abs(np.polyval(fit, xs[core]) - T[core]).max() < 1e-5
    jump = 301.0 - T[0]
    assert 0.0 < jump < 0.1
    q_ref = p.C[0] * v * 2.0 / (np.pi + 2 * L / mfp)
    assert abs(r["q"][:, 0].mean() / q_ref - 1.0) < 0.03


def test_fourier_guess_linear_between_thermalizing_walls():
    """Diffusion-limit initial guess on the in-plane square (walls 301 / 299 K
    left / right, specular top / bottom, no source): the TPFA solution with
    uniform conductivity is exactly linear in x, T = 301 - 2 x / L, at every
    cell centre (the two-point flux of a linear field is exact, also at the
    half-cell wall distance)."""
    p = W.problems.square_inplane(n=20)
    o = OracleSolver(p)
    T = o.fourier_guess() + p.T_ref
    L = 100e-9
    x = o.g.xc[:, 0]
    assert np.abs(T - (301.0 - 2.0 * x / L)).max() < 1e-10


def test_fourier_guess_same_fixed_point():
    """Starting from the Fourier guess changes the iterates, not the limit."""
    p = CASES["square_mixed"]()
    o = OracleSolver(p)
    a = o.solve(scheme="synthetic", tol=1e-13, max_iter=20000)
    b = o.solve(scheme="synthetic", tol=1e-13, max_iter=20000, init="fourier")
    dev = np.abs(a["T"] - p.T_ref).max()
    assert np.abs(a["T"] - b["T"]).max() < 1e-10 * dev
