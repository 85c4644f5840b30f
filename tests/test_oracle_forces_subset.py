"""Pin of the oracle's sampled forces (no GPU).

`oracle.forces_of_atoms` (the C routine `orc_forces_subset`) computes the
all-pairs forces of selected atoms only; it checks and times samples of the
200,000- to 2,000,000-atom systems, where all pairs would take hours.  It is
a second copy of the all-pairs loop, with its own replica lookup, minimum
image and hybrid electron density.  Here it must equal, atom by atom, the
full all-pairs forces of `OracleMD.forces()`, which are pinned themselves
(Newton's third law, translation and periodic-image invariance, F = -dU/dr,
the CODATA Coulomb energy, a KD-tree pair count; `test_oracle_forces.py`,
`test_oracle_hybrid.py`, `test_oracle_bonded.py`).

The systems mix what a wrong offset, image or density would break: charged
and neutral atoms, a periodic box and vacuum clusters in one batch, replicas
with different screening lengths and electron densities, bonded topology.
Forces of Sec. II.A Eq. 2 (Debye), Eqs. 4-7 (hybrid), Sec. II.B Eq. 8 (LJ)
and Eqs. 9-10 (bonded terms).
"""
import numpy as np
import pytest

from paper_2401_03180_gb300 import workloads as W

R_CUT = 1.2


def _charged(s, seed):
    """Charges 0..3 at random (capped at Z) on about half the atoms."""
    rng = np.random.default_rng(seed)
    q = rng.integers(0, 4, s.n_atoms).astype(np.uint8)
    q[rng.random(s.n_atoms) < 0.5] = 0
    s.q0 = np.minimum(q, W.Z[s.species]).astype(np.uint8)
    return s


def _water_box():
    return _charged(W.workload("c2_water_30k", scale=0.03).sample, 1)      # 300 H2O, periodic 2.08 nm


def _methane_cluster():
    return _charged(W.workload("c1_methane_1500", scale=0.4).sample, 2)    # 120 CH4, vacuum


def _batch():
    # three replicas: a vacuum methane cluster, a periodic water box, another cluster
    reps = [W.methane_cluster(60, seed=11), W.water_box(200, 1.82, seed=12), W.methane_cluster(90, seed=13)]
    return _charged(W.concat(reps, "mixed_batch"), 3)


SYSTEMS = {"water_box": _water_box, "methane_cluster": _methane_cluster, "batch3": _batch}


def _full_forces(oracle_mod, s, atom, kappa, ne):
    md = oracle_mod.OracleMD(s, atom, r_cut=R_CUT, cr_enabled=False,
                             screening="hybrid" if ne is not None else "debye")
    F, _, _ = md.forces(kappa=kappa, ne=ne)
    return F


def _selection(n, seed):
    rng = np.random.default_rng(seed)
    # first and last atoms of the system, the replica boundaries, and a random draw
    return np.unique(np.concatenate([[0, n - 1], rng.choice(n, min(n, 97), replace=False)]))


@pytest.mark.parametrize("mode", ["debye", "hybrid"])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_forces_of_atoms_equal_all_pairs(oracle_mod, name, mode):
    s = SYSTEMS[name]()
    atom = W.atomic_data(8.0)
    R = s.n_replicas
    kappa = np.linspace(0.7, 4.1, R)                       # a different screening per replica
    ne = np.linspace(2.0, 9.0, R) if mode == "hybrid" else None   # nm^-3
    F = _full_forces(oracle_mod, s, atom, kappa, ne)
    idx = np.unique(np.concatenate([_selection(s.n_atoms, 5), s.replica_offset[1:-1], s.replica_offset[1:-1] - 1]))
    Fs = oracle_mod.forces_of_atoms(s, atom, idx, r_cut=R_CUT, kappa=kappa, ne=ne)
    scale = np.abs(F).max()
    assert scale > 1.0
    err = np.abs(Fs - F[idx]).max() / scale
    assert err < 1e-12, (name, mode, err)


def test_forces_of_atoms_bonded(oracle_mod):
    """With the molecules' Morse bonds and angles (Eqs. 9-10) the sampled forces
    include the bonded terms as the full forces do."""
    s = W.with_topology(_water_box())
    atom = W.atomic_data(8.0)
    F = _full_forces(oracle_mod, s, atom, np.array([2.5]), None)
    idx = _selection(s.n_atoms, 6)
    Fs = oracle_mod.forces_of_atoms(s, atom, idx, r_cut=R_CUT, kappa=2.5)
    assert np.abs(Fs - F[idx]).max() < 1e-12 * np.abs(F).max()


def test_forces_of_atoms_catches_a_wrong_replica(oracle_mod):
    """The comparison is sharp enough to see a replica mix-up: the same atoms
    summed against the next replica's screening differ far beyond 1e-12."""
    s = _batch()
    atom = W.atomic_data(8.0)
    kappa = np.array([0.7, 2.4, 4.1])
    F = _full_forces(oracle_mod, s, atom, kappa, None)
    idx = np.arange(s.replica_offset[0], s.replica_offset[1])
    Fs = oracle_mod.forces_of_atoms(s, atom, idx, r_cut=R_CUT, kappa=kappa[[1, 2, 0]])
    assert np.abs(Fs - F[idx]).max() > 1e-6 * np.abs(F).max()
