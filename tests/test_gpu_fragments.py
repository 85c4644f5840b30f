"""Fragments and ion-yield counts (Sec. III) on the GPU, through the C ABI
(-m gpu), against the FP64 oracle on the same positions and charges:
labels (the smallest atom index of each fragment) and the counts by mass
number and charge equal, bit for bit, once no pair lies within 1e-5 nm of
r_frag (where FP32 and FP64 distances may decide differently)."""
import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import methane, water

pytestmark = pytest.mark.gpu

A = np.rint(W.MASS).astype(np.int64)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"


def _clear_r_frag(x, box, rep_off, r_frag, tol=1e-5):
    """r_frag moved, if needed, so that no pair lies within tol of it."""
    from scipy.spatial import cKDTree
    for _ in range(50):
        near = 0
        for r in range(len(rep_off) - 1):
            L = box[r]
            per = (L > 0).all()
            xr = np.mod(x[rep_off[r]:rep_off[r + 1]], L) if per else x[rep_off[r]:rep_off[r + 1]]
            t = cKDTree(xr, boxsize=L if per else None)
            near += t.count_neighbors(t, r_frag + tol) - t.count_neighbors(t, r_frag - tol)
        if near == 0:
            return r_frag
        r_frag += 3 * tol
    raise AssertionError("no clear r_frag")


def _check(oracle_mod, g, s, r_frag, mass_max=40, charge_max=20):
    st = g.get_state(M.MD_FIELD_X | M.MD_FIELD_Q)
    rf = _clear_r_frag(st["x"], s.box, s.replica_offset, r_frag)
    lab, cnt = g.fragments(rf, mass_max, charge_max)
    lab_o = oracle_mod.fragments(st["x"], s.box, s.replica_offset, rf)
    assert np.array_equal(lab, lab_o)
    cnt_o = oracle_mod.ion_yield_counts(lab_o, st["q"], A[s.species], s.replica_offset, mass_max, charge_max)
    assert np.array_equal(cnt, cnt_o)
    return lab, cnt


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_intact_molecules_match_oracle(oracle_mod, prec):
    for s, rc, m in ((methane(200), 1.2, 16), water(800) + (18,)):
        g = M.IonisingMD(s, W.atomic_data(8.0), precision=prec, r_cut=rc, cr_enabled=False, max_steps=5)
        lab, cnt = _check(oracle_mod, g, s, 0.16)
        g.close()
        n_mol = len(np.unique(s.fragment))
        assert cnt[0, m].sum() == n_mol and cnt.sum() == n_mol


@pytest.mark.parametrize("skin", [0.0, 0.05])
def test_exploding_clusters_match_oracle(oracle_mod, skin):
    """Batched methane clusters after a strong pulse: Coulomb explosion
    splits molecules into CH_n and H fragments of several charges."""
    reps = [methane(n, seed=k + 41, charge_frac=0.0) for k, n in enumerate((40, 90, 25))]
    for k, r in enumerate(reps):
        r.seed[:] = 900 + k
    s = W.concat(reps)
    atom = W.atomic_data(8.0, pi_scale=20000.0, ci_scale=40.0)
    g = M.IonisingMD(s, atom, max_steps=700, t_start_fs=-5.0, list_skin_nm=skin)
    g.set_pulse([W.Pulse(8.0, 5.0, 5e12, 0.0)])
    g.step(600)
    lab, cnt = _check(oracle_mod, g, s, 0.2)
    g.close()
    n_frag = (lab == np.arange(len(lab))).sum()
    assert n_frag > len(np.unique(s.fragment))               # molecules have broken up
    assert (cnt[:, 1, 1].sum() > 0)                          # protons
    assert cnt.sum() == n_frag


def test_fragments_argument_checks():
    s = methane(10)
    g = M.IonisingMD(s, W.atomic_data(8.0), max_steps=5)
    for bad in (0.0, 1.3):
        with pytest.raises(M.MDError) as e:
            g.fragments(bad)
        assert e.value.status == M.MD_ERR_INVALID_ARG
    g.close()
