"""Pins of the oracle's fragment analysis (ion yields, Sec. III; reading:
fragments are connected components of atoms closer than r_frag):

* intact water and methane molecules are one fragment each, of mass number
  18 and 16 and charge the sum of their atoms' charges;
* an H pulled beyond r_frag splits a methane into CH3 (15) and H (1);
* a molecule split across a periodic face stays one fragment;
* the labels equal a brute-force all-pairs union-find on small random gases
  (a different algorithm: O(N^2) distances, union by relabelling);
* mass and charge summed over the fragments equal the atoms' totals.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_03180_gb300 import workloads as W

A = np.rint(W.MASS).astype(np.int64)     # mass numbers H 1, C 12, N 14, O 16, S 32


def _brute(x, box, rep_off, r_frag):
    lab = np.arange(len(x))
    for r in range(len(rep_off) - 1):
        a0, a1 = rep_off[r], rep_off[r + 1]
        L = box[r]
        for i in range(a0, a1):
            for j in range(i + 1, a1):
                d = x[i] - x[j]
                if (L > 0).all():
                    d -= L * np.round(d / L)
                if d @ d < r_frag * r_frag:
                    a, b = lab[i], lab[j]
                    if a != b:
                        lab[lab == max(a, b)] = min(a, b)
    return lab


def test_intact_molecules_are_one_fragment_each():
    for s, m in ((W.methane_cluster(20, 3), 16), (W.water_droplet(25, 4), 18)):
        rng = np.random.default_rng(1)
        q = rng.integers(0, 3, s.n_atoms)
        lab = O.fragments(s.x, s.box, s.replica_offset, 0.16)
        assert np.array_equal(lab, np.repeat(np.flatnonzero(np.r_[True, s.fragment[1:] != s.fragment[:-1]]),
                                             np.bincount(s.fragment)))
        h = O.ion_yield_counts(lab, q, A[s.species], s.replica_offset, 40, 20)
        zmol = np.bincount(s.fragment, weights=q).astype(int)
        assert h[0, m].sum() == len(zmol) and np.array_equal(h[0, m, :15], np.bincount(zmol, minlength=15)[:15])


def test_pulled_hydrogen_splits_off_and_periodic_face():
    s = W.methane_cluster(1, 2)
    x = s.x.copy()
    x[3] = x[0] + 3.0 * (x[3] - x[0])                       # C-H 0.109 -> 0.327 nm
    lab = O.fragments(x, s.box, s.replica_offset, 0.2)
    assert np.array_equal(lab, [0, 0, 0, 3, 0])
    q = np.array([2, 0, 1, 1, 0])
    h = O.ion_yield_counts(lab, q, A[s.species], s.replica_offset, 20, 5)
    assert h[0, 15, 3] == 1 and h[0, 1, 1] == 1 and h.sum() == 2
    L = 2.0
    xw = np.mod(s.x - s.x[0] + np.array([0.01, 1.0, 1.0]), L)   # C at the x = 0 face, Hs wrap
    assert (xw[:, 0] > 1.5).any()
    lab = O.fragments(xw, np.array([[L, L, L]]), s.replica_offset, 0.2)
    assert (lab == 0).all()


@pytest.mark.parametrize("periodic", [False, True])
def test_labels_equal_brute_force_union(periodic):
    rng = np.random.default_rng(5 + periodic)
    n = [60, 45, 80]
    off = np.r_[0, np.cumsum(n)]
    L = 1.6
    x = rng.uniform(0, L, (off[-1], 3))
    box = np.full((3, 3), L if periodic else 0.0)
    for rf in (0.15, 0.25):
        lab = O.fragments(x, box, off, rf)
        assert np.array_equal(lab, _brute(x, box, off, rf))
    sp = rng.integers(0, 5, off[-1])
    q = rng.integers(0, 4, off[-1])
    h = O.ion_yield_counts(lab, q, A[sp], off, 2_000, 300)
    r_, m_, z_ = np.nonzero(h)
    c_ = h[r_, m_, z_]
    assert (h.sum(2).sum(1) > 0).all() and (m_ < 2_000).all() and (z_ < 300).all()
    assert int((m_ * c_).sum()) == int(A[sp].sum()) and int((z_ * c_).sum()) == int(q.sum())
