"""Pins of the oracle's pair potential and all-pairs forces (no GPU).

Sec. II.A Eq. 2 (Debye-screened Coulomb), Sec. II.B Eq. 8 (screened LJ) and
Eq. 11 (charge scaling of the LJ size), checked against facts that do not
come from the oracle's own formulas: a CODATA-derived Coulomb energy,
textbook LJ landmarks, finite-difference derivatives, Newton's third law,
translation/periodic-image invariance and a KD-tree pair count.
"""
import math
import os

import numpy as np
import pytest

from paper_2401_03180_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].split()
        if len(line) == 2:
            out[line[0]] = float(line[1])
    return out


def test_coulomb_prefactor_codata(oracle_mod):
    g = _golden("coulomb_two_charges_1nm.txt")
    fr, u = oracle_mod.pair(g["r_nm"], 1.0, 1.0, 0.0, 0.0, 0.0, rc=1e16)
    assert abs(u - g["u_kj_mol"]) / g["u_kj_mol"] < g["rel_tol"]
    # F = U/r for bare Coulomb: fr = F/r = U/r^2
    assert abs(fr - g["u_kj_mol"]) / g["u_kj_mol"] < g["rel_tol"]


@pytest.mark.parametrize("kappa,r", [(1.0, 1.0), (5.0, 1.0), (2.0, 0.5), (0.3, 2.0)])
def test_yukawa_ratio_and_coulomb_limit(oracle_mod, kappa, r):
    _, u0 = oracle_mod.pair(r, 2.0, 3.0, 0.0, 0.0, 0.0, rc=1e16)
    _, uk = oracle_mod.pair(r, 2.0, 3.0, 0.0, 0.0, kappa, rc=1e16)
    assert math.isclose(uk / u0, math.exp(-kappa * r), rel_tol=1e-13)
    _, ut = oracle_mod.pair(r, 2.0, 3.0, 0.0, 0.0, 1e-8, rc=1e16)
    assert math.isclose(ut, u0, rel_tol=2e-8 * r + 1e-14)


def test_lj_landmarks_and_charge_scaling(oracle_mod):
    z = W.Z
    c6, c12 = oracle_mod.lj_table(z, W.LJ_SIGMA0, W.LJ_EPS0)
    off = W.ts_offsets(z)
    for si in range(5):
        for sj in range(5):
            a, b = off[si], off[sj]
            sig = 0.5 * (W.LJ_SIGMA0[si] + W.LJ_SIGMA0[sj])
            eps = math.sqrt(W.LJ_EPS0[si] * W.LJ_EPS0[sj])
            rmin = 2 ** (1 / 6) * sig
            # zero crossing at sigma, minimum -eps at 2^(1/6) sigma (kappa = 0, no shift)
            _, u_sig = oracle_mod.pair(sig, 0, 0, c6[a, b], c12[a, b], 0.0, rc=1e9)
            _, u_min = oracle_mod.pair(rmin, 0, 0, c6[a, b], c12[a, b], 0.0, rc=1e9)
            fr_min, _ = oracle_mod.pair(rmin, 0, 0, c6[a, b], c12[a, b], 0.0, rc=1e9)
            assert abs(u_sig) < 1e-12 * eps
            assert math.isclose(u_min, -eps, rel_tol=1e-12)
            assert abs(fr_min) < 1e-9 * eps / sig ** 2
    # Eq. 11: a fully stripped atom has zero size -> c6 = c12 = 0 for (s, q=Z) with itself
    for s in range(5):
        full = off[s] + z[s]
        assert c6[full, full] == 0.0 and c12[full, full] == 0.0
    # half-stripped carbon (q = 3 of 6): sigma halves; C-C minimum moves to half
    cq3 = off[W.C] + 3
    rmin_half = 2 ** (1 / 6) * W.LJ_SIGMA0[W.C] * 0.5
    fr, u = oracle_mod.pair(rmin_half, 0, 0, c6[cq3, cq3], c12[cq3, cq3], 0.0, rc=1e9)
    assert abs(fr) < 1e-8 and math.isclose(u, -W.LJ_EPS0[W.C], rel_tol=1e-12)


def test_force_is_minus_energy_derivative(oracle_mod):
    c6, c12 = oracle_mod.lj_table(W.Z, W.LJ_SIGMA0, W.LJ_EPS0)
    off = W.ts_offsets(W.Z)
    rc = 1.2
    cases = [(off[W.O], off[W.O], 0, 0), (off[W.O] + 2, off[W.H] + 1, 2, 1),
             (off[W.C] + 1, off[W.S] + 5, 1, 5), (off[W.H], off[W.N] + 7, 0, 7)]
    for kappa in (0.0, 1.7, 6.0):
        for a, b, qa, qb in cases:
            for lj_on in (True, False):
                for r in np.linspace(0.12, rc - 0.01, 23):
                    h = 1e-5 * r
                    us = [oracle_mod.pair(r + k * h, qa, qb, c6[a, b], c12[a, b], kappa, rc, lj_on)[1]
                          for k in (-2, -1, 1, 2)]
                    dudr = (us[0] - 8 * us[1] + 8 * us[2] - us[3]) / (12 * h)
                    fr, _ = oracle_mod.pair(r, qa, qb, c6[a, b], c12[a, b], kappa, rc, lj_on)
                    F = fr * r
                    scale = max(abs(F), 1e-3)
                    assert abs(F + dudr) / scale < 1e-7, (kappa, a, b, r, F, -dudr)
    # energy shifted to zero at the cutoff
    _, u_rc = oracle_mod.pair(rc, 2, 3, c6[1, 1], c12[1, 1], 2.0, rc)
    assert abs(u_rc) < 1e-14


def _small_system(oracle_mod, name="c2", scale=0.02, q_every=2, kappa=3.0):
    wl = W.workload("c2_water_30k" if name == "c2" else "c1_methane_1500", scale=scale)
    s = wl.sample
    s.q0[::q_every] = 1
    atom = W.atomic_data(wl.photon_kev)
    rc = 0.9 if name == "c2" else 1.2
    md = oracle_mod.OracleMD(s, atom, r_cut=rc, cr_enabled=False, kappa_fixed=kappa)
    return md


@pytest.mark.parametrize("name", ["c2", "c1"])
def test_newton_third_law(oracle_mod, name):
    md = _small_system(oracle_mod, name)
    F = md.F
    net = F.sum(0)
    assert np.abs(net).max() < 1e-11 * np.abs(F).sum(0).max()


def test_translation_and_periodic_images(oracle_mod):
    md = _small_system(oracle_mod, "c2")
    F0 = md.F.copy()
    L = md.box[0]
    shifted = md.x + np.array([0.37, -1.91, 2.5])
    wrapped = shifted - L * np.floor(shifted / L)
    F1, U1, n1 = md.forces(x=wrapped)
    assert np.abs(F1 - F0).max() < 1e-9 * np.abs(F0).max()
    assert n1 == md.n_pairs
    # any atom moved by a whole box vector: nothing changes
    x2 = md.x.copy()
    x2[::7] += L * np.array([1, -2, 3])
    F2, _, n2 = md.forces(x=x2)
    assert np.abs(F2 - F0).max() < 1e-9 * np.abs(F0).max() and n2 == md.n_pairs


@pytest.mark.parametrize("name", ["c2", "c1"])
def test_pair_count_matches_kdtree(oracle_mod, name):
    from scipy.spatial import cKDTree
    md = _small_system(oracle_mod, name)
    L = md.box[0]
    periodic = L[0] > 0
    tree = cKDTree(np.mod(md.x, L) if periodic else md.x, boxsize=L if periodic else None)
    n_ref = len(tree.query_pairs(md.rc))
    assert md.n_pairs == n_ref


def test_excluded_pairs_keep_coulomb(oracle_mod):
    # two atoms of one fragment: LJ off, screened Coulomb on (Sec. II.B)
    s = W.Sample(x=np.array([[0.0, 0, 0], [0.25, 0, 0]]), v=np.zeros((2, 3)),
                 species=np.array([W.O, W.O], np.uint8), fragment=np.array([0, 0], np.int32),
                 q0=np.array([1, 2], np.uint8), replica_offset=np.array([0, 2], np.int32),
                 seed=np.array([1], np.uint64), box=np.zeros((1, 3)), volume=np.array([1.0]))
    md = oracle_mod.OracleMD(s, W.atomic_data(8.0), cr_enabled=False, kappa_fixed=2.0)
    fr, _ = oracle_mod.pair(0.25, 1, 2, 0.0, 0.0, 2.0, 1.2, lj_on=False)
    assert math.isclose(md.F[0, 0], fr * -0.25, rel_tol=1e-14)
    s.fragment[1] = 1
    md2 = oracle_mod.OracleMD(s, W.atomic_data(8.0), cr_enabled=False, kappa_fixed=2.0)
    assert abs(md2.F[0, 0] - md.F[0, 0]) > 1.0
