"""Shared helpers of the -m gpu tests (not a test module)."""
import numpy as np

from paper_2401_03180_gb300 import workloads as W


def water(n_mol, r_cut=None, charge_frac=0.3, seed=7):
    """Periodic water box at 1 g/cm^3 with random ion charges 1..2."""
    wl = W.workload("c2_water_30k", scale=n_mol / 10_000)
    s = wl.sample
    rng = np.random.default_rng(seed)
    sel = rng.random(s.n_atoms) < charge_frac
    s.q0[sel] = np.minimum(rng.integers(1, 3, sel.sum()), W.Z[s.species[sel]]).astype(np.uint8)
    if r_cut is None:
        r_cut = min(1.2, s.box[0, 0] / 3.0 * 0.999)
    return s, r_cut


def methane(n_mol, charge_frac=0.3, seed=8):
    wl = W.workload("c1_methane_1500", scale=n_mol / 300)
    s = wl.sample
    rng = np.random.default_rng(seed)
    sel = rng.random(s.n_atoms) < charge_frac
    s.q0[sel] = np.minimum(rng.integers(1, 4, sel.sum()), W.Z[s.species[sel]]).astype(np.uint8)
    return s


def force_errors(F, Fref):
    """RMS relative error ||F - Fref|| / ||Fref||, and max |dF| / RMS|Fref|."""
    d = F - Fref
    rms_rel = float(np.linalg.norm(d) / np.linalg.norm(Fref))
    rms_f = float(np.sqrt((Fref ** 2).sum(1).mean()))
    max_rel = float(np.abs(d).max() / rms_f)
    return rms_rel, max_rel


def near_cutoff_pairs(x, box, rc, tol):
    """Pairs whose distance lies within tol of the cutoff (either count is valid)."""
    from scipy.spatial import cKDTree
    periodic = box is not None and box[0] > 0
    xx = np.mod(x, box) if periodic else x
    t = cKDTree(xx, boxsize=box if periodic else None)
    return len(t.query_pairs(rc + tol)) - len(t.query_pairs(rc - tol))
