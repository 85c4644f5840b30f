"""Pins of the oracle's hybrid ion-sphere / Debye electrostatics (Sec. II.A,
Eqs. 4-7), against what the paper and the mathematics fix:

* Eq. 7 as printed: (r' + lambda)^3 = R^3 + lambda^3;
* the continuity of phi, phi' and phi'' at r' (the matching the paper names);
* inside r' the curvature term is the uniform electron background's,
  c2 = -Q/(2R^3) = -2 pi n_e / 3 (Poisson), as in the ion-sphere form Eq. 5;
* limits: the uniform-electron-gas ion sphere of Eq. 5 as lambda -> 0,
  Coulomb as kappa -> 0, Debye (Eq. 2) as R -> 0;
* pair level: F = -dU/dr, symmetry in (i, j), Newton III in all-pairs sums.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

CASES = [(1.0, 50.0, 5.0), (2.0, 100.0, 10.0), (6.0, 300.0, 20.0), (3.0, 10.0, 3.0), (8.0, 600.0, 60.0)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def _R(Q, ne):
    return (3.0 * Q / (4.0 * math.pi * ne)) ** (1.0 / 3.0)


@pytest.mark.parametrize("Q,ne,kap", CASES)
def test_transition_radius_is_eq7(Q, ne, kap):
    rp, _, _, _ = O.hybrid_coeffs(Q, ne, kap)
    lam = 1.0 / kap
    R = _R(Q, ne)
    assert 0.0 < rp < R
    assert (rp + lam) ** 3 == pytest.approx(R ** 3 + lam ** 3, rel=1e-13)


@pytest.mark.parametrize("Q,ne,kap", CASES)
def test_inner_curvature_is_uniform_background(Q, ne, kap):
    _, _, c2, _ = O.hybrid_coeffs(Q, ne, kap)
    assert c2 == pytest.approx(-2.0 * math.pi * ne / 3.0, rel=1e-12)
    assert c2 == pytest.approx(-Q / (2.0 * _R(Q, ne) ** 3), rel=1e-12)


@pytest.mark.parametrize("Q,ne,kap", CASES)
def test_phi_and_two_derivatives_continuous_at_r_prime(Q, ne, kap):
    rp, _, _, _ = O.hybrid_coeffs(Q, ne, kap)
    eps = 1e-7 * rp
    lo = O.hybrid_phi(Q, ne, kap, rp * (1 - 1e-12))
    hi = O.hybrid_phi(Q, ne, kap, rp * (1 + 1e-12))
    assert lo[0] == pytest.approx(hi[0], rel=1e-9)        # phi
    assert lo[1] == pytest.approx(hi[1], rel=1e-9)        # -phi'
    # phi'': one-sided differences of -phi' on each side of r'
    h = 1e-4 * rp
    in1, in2 = O.hybrid_phi(Q, ne, kap, rp - h - eps)[1], O.hybrid_phi(Q, ne, kap, rp - eps)[1]
    out1, out2 = O.hybrid_phi(Q, ne, kap, rp + eps)[1], O.hybrid_phi(Q, ne, kap, rp + h + eps)[1]
    d_in = (in2 - in1) / h
    d_out = (out2 - out1) / h
    assert d_in == pytest.approx(d_out, rel=2e-3)


def test_ion_sphere_limit_is_eq5():
    # lambda -> 0 at fixed R: r' -> R and phi -> Q/r - (Q/2R)(3 - r^2/R^2) inside, 0 outside
    Q, ne = 4.0, 200.0
    R = _R(Q, ne)
    kap = 1e6 / R
    rp, _, _, _ = O.hybrid_coeffs(Q, ne, kap)
    assert rp == pytest.approx(R, rel=1e-5)
    for r in (0.1 * R, 0.5 * R, 0.9 * R):
        phi, mphi = O.hybrid_phi(Q, ne, kap, r)
        ref = Q / r - Q / (2 * R) * (3 - r * r / (R * R))
        mref = Q / r ** 2 - Q * r / R ** 3
        assert phi == pytest.approx(ref, rel=1e-5, abs=1e-9 * Q / R)
        assert mphi == pytest.approx(mref, rel=1e-5)
    assert abs(O.hybrid_phi(Q, ne, kap, 1.01 * R)[0]) < 1e-12


def test_coulomb_limit():
    Q, ne = 3.0, 100.0
    for r in (0.05, 0.3, 1.0):
        phi, mphi = O.hybrid_phi(Q, ne, 1e-9, r)
        assert phi == pytest.approx(Q / r, rel=1e-8)
        assert mphi == pytest.approx(Q / r ** 2, rel=1e-8)


def test_debye_limit():
    # R -> 0 at fixed kappa (dense electrons): r' -> 0, phi -> Q e^{-kappa r}/r
    Q, kap = 2.0, 8.0
    rp, _, _, a = O.hybrid_coeffs(Q, 1e12, kap)
    assert rp < 1e-10 and a == pytest.approx(Q, rel=1e-9)
    for r in (0.05, 0.4, 1.1):
        phi, mphi = O.hybrid_phi(Q, 1e12, kap, r)
        assert phi == pytest.approx(Q * math.exp(-kap * r) / r, rel=1e-9)
        assert mphi == pytest.approx(Q * math.exp(-kap * r) * (1 + kap * r) / r ** 2, rel=1e-9)


def test_no_ion_sphere_without_electrons_or_charge():
    assert O.hybrid_coeffs(2.0, 0.0, 5.0) == (0.0, 0.0, 0.0, 2.0)
    assert O.hybrid_coeffs(0.0, 100.0, 5.0) == (0.0, 0.0, 0.0, 0.0)
    r, q = 0.3, 2.0
    fr, u = O.pair_hybrid(r, q, 1.0, 0.0, 0.0, 5.0, 0.0, 1.2, lj_on=False)
    fr0, u0 = O.pair(r, q, 1.0, 0.0, 0.0, 5.0, 1.2, lj_on=False)
    assert fr == pytest.approx(fr0, rel=1e-13) and u == pytest.approx(u0, rel=1e-13)


@pytest.mark.parametrize("qi,qj", [(1.0, 1.0), (3.0, 1.0), (6.0, 2.0), (0.0, 4.0)])
def test_pair_force_is_minus_dU_dr(qi, qj):
    ne, kap, rc = 300.0, 25.0, 1.2
    c6, c12 = 2e-3, 3e-6
    rps = [O.hybrid_coeffs(q, ne, kap)[0] for q in (qi, qj) if q > 0]
    # radii inside both ion spheres, between the two transition radii, and outside
    rs = [0.3 * min(rps), 0.5 * (rps[0] + rps[-1]) if rps else 0.1, 0.35, 0.9] if rps else [0.2, 0.9]
    for r in rs:
        h = 1e-5 * r
        u = [O.pair_hybrid(r + k * h, qi, qj, c6, c12, kap, ne, rc)[1] for k in (-2, -1, 1, 2)]
        dudr = (u[0] - 8 * u[1] + 8 * u[2] - u[3]) / (12 * h)
        fr, _ = O.pair_hybrid(r, qi, qj, c6, c12, kap, ne, rc)
        assert fr * r == pytest.approx(-dudr, rel=1e-7, abs=1e-9)
        assert O.pair_hybrid(r, qj, qi, c6, c12, kap, ne, rc) == pytest.approx((fr, O.pair_hybrid(r, qi, qj, c6, c12, kap, ne, rc)[1]), rel=1e-14)
    assert O.pair_hybrid(rc, qi, qj, c6, c12, kap, ne, rc)[1] == pytest.approx(0.0, abs=1e-12)


def test_all_pairs_newton_iii_and_debye_when_no_electrons():
    from paper_2401_03180_gb300 import workloads as W
    wl = W.workload("c1_methane_1500", scale=0.2)
    s = wl.sample
    rng = np.random.default_rng(3)
    s.q0[:] = rng.integers(0, 3, s.n_atoms)
    atom = W.atomic_data(8.0)
    md = O.OracleMD(s, atom, r_cut=1.2, kappa_fixed=6.0, screening="hybrid")
    F, _, _ = md.forces(ne=np.array([150.0]))
    assert np.abs(F.sum(0)).max() < 1e-9 * np.abs(F).sum()
    Fd, _, _ = md.forces(ne=np.array([0.0]))
    md2 = O.OracleMD(s, atom, r_cut=1.2, kappa_fixed=6.0)
    assert np.allclose(Fd, md2.F, rtol=1e-12, atol=1e-9)
    assert not np.allclose(F, md2.F, rtol=1e-3)
