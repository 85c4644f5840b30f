"""Pins of the oracle's bonded terms (Sec. II.B, Eqs. 9-10; Sec. III names
the harmonic angle term), against what the mathematics and mechanics fix:

* Morse: zero at b_e, D_e at dissociation, curvature 2 D_e beta^2 at b_e,
  dV/dr by finite differences;
* the angle of known geometries (tetrahedral, right angle);
* F = -grad U by finite differences on every coordinate of ionised water and
  methane molecules (a wrong sign or index of any atom's share fails);
* zero net force and torque per molecule (translation and rotation
  invariance);
* the charge scaling of Eq. 9: 1 for neutral atoms, 0 from a mean charge of 1;
* the minimum image across a periodic boundary;
* a diatomic's small-amplitude period 2 pi / omega, omega = beta sqrt(2 D_e / mu),
  integrated with the oracle's velocity Verlet.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_03180_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def _deriv(f, x, h):
    return (f(x - 2 * h) - 8 * f(x - h) + 8 * f(x + h) - f(x + 2 * h)) / (12 * h)


def test_morse_zero_dissociation_and_curvature():
    De, be, beta = 420.0, 0.109, 18.0
    assert O.morse(be, De, be, beta)[0] == 0.0
    assert O.morse(be, De, be, beta)[1] == 0.0
    assert O.morse(be + 60.0 / beta, De, be, beta)[0] == pytest.approx(De, rel=1e-12)
    h = 1e-5
    v = [O.morse(be + k * h, De, be, beta)[0] for k in (-1, 0, 1)]
    assert (v[0] - 2 * v[1] + v[2]) / h ** 2 == pytest.approx(2 * De * beta ** 2, rel=1e-5)
    for r in (0.07, 0.1, 0.13, 0.25):
        assert O.morse(r, De, be, beta)[1] == pytest.approx(
            _deriv(lambda t: O.morse(t, De, be, beta)[0], r, 1e-6), rel=1e-8)


def test_bond_scale_limits():
    assert O.bond_scale(0, 2) == 1.0
    assert O.bond_scale(1, 2) == 0.5
    assert O.bond_scale(2, 2) == 0.0
    assert O.bond_scale(7, 2) == 0.0            # clamped
    assert O.bond_scale(1, 3) == pytest.approx(2.0 / 3.0, rel=1e-15)
    assert O.bond_scale(3, 3) == 0.0


def _topo(bonds, angles):
    return W.Topology(np.asarray(bonds, np.int32).reshape(-1, 3), W.BOND_PARAMS.copy(),
                      np.asarray(angles, np.int32).reshape(-1, 4), W.ANGLE_PARAMS.copy())


def _energy(x, q, box, topo):
    return O.bonded_forces(x, q, box, topo)[1].sum()


def test_angle_of_known_geometries():
    kt, th0 = W.ANGLE_PARAMS[1]
    d = 0.109 / math.sqrt(3.0)
    x = np.array([[0, 0, 0], [d, d, d], [d, -d, -d]], np.float64)   # tetrahedral H-C-H
    topo = _topo([], [[1, 0, 2, 1]])
    box = np.zeros((3, 3))
    F, U = O.bonded_forces(x, np.zeros(3), box, topo)
    assert abs(U.sum()) < 1e-20 and np.abs(F).max() < 1e-9
    x = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.12, 0]], np.float64)  # right angle
    F, U = O.bonded_forces(x, np.zeros(3), box, topo)
    assert U.sum() == pytest.approx(0.5 * kt * (math.pi / 2 - th0) ** 2, rel=1e-13)
    assert np.allclose(U, U.sum() / 3, rtol=1e-15)


@pytest.mark.parametrize("kind", ["water", "methane"])
def test_forces_are_minus_gradient_and_conserve_momentum(kind):
    rng = np.random.default_rng(7)
    s = W.with_topology(W.water_box(8, 1.2, 3) if kind == "water" else W.methane_cluster(4, 5))
    x = s.x + rng.normal(scale=0.01, size=s.x.shape)        # off equilibrium
    q = rng.integers(0, 3, s.n_atoms).astype(np.uint8)     # charges 0-2: c from 1 down to 0
    box = np.repeat(s.box, s.n_atoms, 0)
    F, U = O.bonded_forces(x, q, box, s.topology)
    h = 1e-6
    for a in range(s.n_atoms):
        for d in range(3):
            def e(t):
                y = x.copy(); y[a, d] = t
                return _energy(y, q, box, s.topology)
            assert F[a, d] == pytest.approx(-_deriv(e, x[a, d], h), rel=1e-6, abs=1e-6)
    for f in np.unique(s.fragment):
        m = s.fragment == f
        assert np.abs(F[m].sum(0)).max() < 1e-10
        c = x[m].mean(0)
        assert np.abs(np.cross(x[m] - c, F[m]).sum(0)).max() < 1e-10
    # the scaling actually varies here and a term of mean charge >= 1 drops out
    cb = O.bond_scale(q[s.topology.bonds[:, 0]].astype(float) + q[s.topology.bonds[:, 1]], 2)
    assert cb.min() == 0.0 and cb.max() == 1.0 and ((cb > 0) & (cb < 1)).any()


def test_ionised_term_scales_linearly():
    s = W.with_topology(W.water_box(1, 1.0, 2))
    x = s.x.copy()
    x[1] += 0.01
    box = np.zeros((3, 3))
    F0, U0 = O.bonded_forces(x, np.zeros(3), box, s.topology)
    F1, U1 = O.bonded_forces(x, np.array([0, 1, 0]), box, s.topology)
    # O-H1 bond: c = 1/2; O-H2 bond: 1; angle: 2/3
    one = W.Topology(s.topology.bonds[:1], s.topology.bond_params, np.zeros((0, 4), np.int32), s.topology.angle_params)
    Fb0, Ub0 = O.bonded_forces(x, np.zeros(3), box, one)
    Fb1, Ub1 = O.bonded_forces(x, np.array([0, 1, 0]), box, one)
    assert np.allclose(Fb1, 0.5 * Fb0, rtol=1e-15, atol=0) and Ub1.sum() == pytest.approx(0.5 * Ub0.sum(), rel=1e-15)
    ang = W.Topology(np.zeros((0, 3), np.int32), s.topology.bond_params, s.topology.angles, s.topology.angle_params)
    Fa0, Ua0 = O.bonded_forces(x, np.zeros(3), box, ang)
    Fa1, Ua1 = O.bonded_forces(x, np.array([0, 1, 0]), box, ang)
    Fa2, Ua2 = O.bonded_forces(x, np.array([1, 1, 1]), box, ang)
    assert np.allclose(Fa1, Fa0 * (2.0 / 3.0), rtol=1e-14, atol=0) and Ua1.sum() == pytest.approx(Ua0.sum() * 2 / 3, rel=1e-14)
    assert np.abs(Fa0).max() > 0 and not Fa2.any() and not Ua2.any()
    assert U1.sum() < U0.sum()


def test_minimum_image_across_the_box():
    L = 1.5
    s = W.with_topology(W.methane_cluster(1, 9))
    x = s.x - s.x[0] + np.array([0.02, 0.75, 0.75])             # C near the x = 0 face
    x += np.random.default_rng(1).normal(scale=0.005, size=x.shape)
    box = np.full((5, 3), L)
    F0, U0 = O.bonded_forces(x, np.zeros(5), box, s.topology)
    xw = np.mod(x, L)                                           # Hs wrapped to the far face
    assert (np.abs(xw - x) > 1.0).any()
    F1, U1 = O.bonded_forces(xw, np.zeros(5), box, s.topology)
    assert np.allclose(F1, F0, rtol=1e-9, atol=1e-9) and np.allclose(U1, U0, rtol=1e-9, atol=1e-15)


def test_diatomic_vibration_period():
    De, be, beta = W.BOND_PARAMS[0]
    m1, m2 = W.MASS[W.O], W.MASS[W.H]
    mu = m1 * m2 / (m1 + m2)
    omega = beta * math.sqrt(2 * De / mu)                      # 1/ps
    a0 = 0.002
    s = W.Sample(x=np.array([[0.0, 0.0, 0.0], [be + a0, 0.0, 0.0]]), v=np.zeros((2, 3)),
                 species=np.array([W.O, W.H], np.uint8), fragment=np.zeros(2, np.int32),
                 q0=np.zeros(2, np.uint8), replica_offset=np.array([0, 2], np.int32),
                 seed=np.array([1], np.uint64), box=np.zeros((1, 3)), volume=np.array([1.0]),
                 topology=_topo([[0, 1, 0]], []))
    md = O.OracleMD(s, W.atomic_data(8.0), cr_enabled=False, kappa_fixed=0.0)
    r = []
    for _ in range(700):
        md.step()
        r.append(np.linalg.norm(md.x[1] - md.x[0]) - be)
    r = np.array(r)
    t = (np.arange(len(r)) + 1) * md.dt
    up = np.flatnonzero((r[:-1] < 0) & (r[1:] >= 0))          # upward zero crossings
    tc = t[up] + md.dt * (-r[up]) / (r[up + 1] - r[up])
    period = np.diff(tc).mean()
    # Morse anharmonicity at this amplitude shifts omega by ~E/(2 D_e) ~ 1e-3
    assert period == pytest.approx(2 * math.pi / omega, rel=3e-3)
    assert len(up) >= 3
