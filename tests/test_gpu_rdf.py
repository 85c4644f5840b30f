"""Pair-distance histograms for the radial distribution functions and the
partial structure factors of Sec. II.C (Eq. 18), through the C ABI (-m gpu):
the GPU counts equal the all-pairs FP64 oracle's, up to pairs within 1e-5 nm
of a bin edge (where FP32 and FP64 distances may disagree), after some steps
(list built earlier, with and without the Verlet buffer); md_structure_factor
equals the oracle's quadrature on the same counts."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import methane, water

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"


def _edge_slack(x, sp, box, r_max, n_bins, ns, tol=1e-5):
    periodic = box is not None and box[0] > 0
    xx = np.mod(x, box) if periodic else x
    t = cKDTree(xx, boxsize=box if periodic else None)
    pr = np.array(sorted(t.query_pairs(r_max + tol)), dtype=np.int64).reshape(-1, 2)
    d = x[pr[:, 0]] - x[pr[:, 1]]
    if periodic:
        d -= box * np.round(d / box)
    r = np.sqrt((d * d).sum(1))
    dr = r_max / n_bins
    k = np.rint(r / dr)
    near = np.abs(r - k * dr) < tol                  # within tol of edge k*dr
    slack = np.zeros((ns, ns, n_bins + 1), dtype=np.int64)
    a, b = sp[pr[near, 0]], sp[pr[near, 1]]
    kk = k[near].astype(np.int64)
    for lo, hi, e in zip(np.minimum(a, b), np.maximum(a, b), kk):
        for kb in (e - 1, e):                        # the bins on both sides of the edge
            if 0 <= kb < n_bins:
                slack[lo, hi, kb] += 1
                if lo != hi:
                    slack[hi, lo, kb] += 1
    return slack[:, :, :n_bins]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("case", ["water", "water_skin", "methane"])
def test_rdf_counts_match_oracle(oracle_mod, prec, case):
    if case.startswith("water"):
        s, rc = water(1000, charge_frac=0.0)
    else:
        s, rc = methane(300, charge_frac=0.0), 1.2
    skin = 0.03 if case == "water_skin" else 0.0
    if skin:
        rc = 0.9                                     # 3 (r_cut + skin) within the 3.11 nm box
    atom = W.atomic_data(8.0)
    g = M.IonisingMD(s, atom, precision=prec, r_cut=rc, cr_enabled=False, max_steps=30, list_skin_nm=skin)
    g.step(25)
    x = g.get_state(M.MD_FIELD_X)["x"]
    r_max, n_bins, ns = min(1.0, rc), 50, len(atom.z)
    got = g.rdf(r_max, n_bins)
    g.close()
    ref = oracle_mod.rdf_counts(x, s.species, ns, s.box, s.replica_offset, r_max, n_bins)
    box = s.box[0] if s.box[0, 0] > 0 else None
    slack = _edge_slack(x, s.species.astype(np.int64), box, r_max, n_bins, ns)
    assert np.all(np.abs(got - ref) <= slack), np.argwhere(np.abs(got - ref) > slack)[:5]
    assert np.array_equal(got, got.transpose(1, 0, 2))
    heavy = 3 if case.startswith("water") else 1     # O-H pairs of the water box, C-H of methane
    assert got[heavy, 0].sum() > 1000
    # Eq. 18 on these counts: the library's quadrature equals the oracle's
    if box is not None:
        V = float(np.prod(box))
        n_a = int((s.species == 3).sum()); n_b = int((s.species == 0).sum())
        q = np.array([5.0, 10.0, 20.0, 30.0])
        S = M.md_structure_factor(got[3, 0], r_max, n_a, n_b, False, V, s.n_atoms / V, q)
        r, gr = oracle_mod.rdf(got[3, 0], n_a, n_b, False, V, r_max)
        ref_S = oracle_mod.structure_factor(r, gr, s.n_atoms / V, q, r_max / n_bins)
        assert np.allclose(S, ref_S, rtol=1e-10, atol=1e-12)
