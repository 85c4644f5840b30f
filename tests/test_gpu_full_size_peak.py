"""The five workloads at full size, in the middle of their runs, in the
benchmark's configuration, -m gpu.

The bench times each workload around the middle of its configured run (the
pulse peak; for the protein crystal the middle between pump and probe) with
the Verlet buffer (0.12 nm skin), autotuned launch shapes and eight steps per
graph launch; there the samples are ionised and the lists are rebuilt every
few steps.  After the first half of the run, with the charge dynamics on, the
state must hold:

* every pair within r_cut: the force kernel's in-cutoff pair count equals an
  exact KD-tree count of the pairs closer than r_cut in each replica
  (periodic replicas with the minimum image), up to the pairs within 1e-6 nm
  of r_cut (FP32 cell-relative distances are good to ~1e-7 nm there);
* the forces of 300 sampled atoms equal the FP64 oracle's all-pair forces at
  the GPU's positions, charges and kappa (Sec. II.A Eq. 2, Sec. II.B Eq. 8)
  within the mixed path's 1e-5 RMS relative error, and the FP64 path's 1e-12
  (the FP64 path on the four smaller workloads; on the droplet, 400 FP64 steps
  would take over a minute, and the bench checks its FP64 forces there);
* the screened Coulomb term is live (some replica has kappa > 0 and free
  electrons) and the buffer was used (fewer builds than steps).
"""
import dataclasses

import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import force_errors

pytestmark = pytest.mark.gpu
RC = 1.2
SKIN = 0.12          # the bench's skin
WORKLOADS = ["c1_methane_1500", "c2_water_30k", "c3_protein_200k", "c4_methane_batch", "c5_droplet_2m"]


def _pairs_within(x, box, r):
    """Unordered pairs closer than each radius in r (exact, KD-tree)."""
    from scipy.spatial import cKDTree
    periodic = box is not None and box[0] > 0
    xx = np.mod(x, box) if periodic else x
    tree = cKDTree(xx, boxsize=box if periodic else None)
    return (tree.count_neighbors(tree, np.asarray(r)) - len(x)) // 2


CASES = [(w, "mixed") for w in WORKLOADS] + [(w, "fp64") for w in WORKLOADS[:4]]
TOL = {"mixed": 1e-5, "fp64": 1e-12}


@pytest.mark.parametrize("name,prec", CASES)
def test_full_size_mid_run_in_the_bench_configuration(oracle_mod, name, prec):
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    wl = W.workload(name)
    s = wl.sample
    atom = W.atomic_data(wl.photon_kev)
    steps = wl.n_steps // 2
    g = M.IonisingMD(s, atom, precision=prec, r_cut=RC, max_steps=wl.n_steps, t_start_fs=wl.t_start_fs,
                     autotune=prec == "mixed", list_skin_nm=SKIN)
    for r in range(s.n_replicas):
        g.set_pulse(wl.pulses[r], replica=r)
    g.step(steps)
    st = g.get_state(M.MD_FIELD_X | M.MD_FIELD_Q | M.MD_FIELD_F | M.MD_FIELD_PLASMA | M.MD_FIELD_STEP)
    _, _, n_gpu = g.energies()
    t = g.timing()
    g.close()
    assert st["step"] == steps
    assert np.max(st["kappa"]) > 1.0 and np.max(st["n_e"]) > 0
    assert t.list_builds < steps, t.list_builds

    # every pair within r_cut, replica by replica
    tol = 1e-6
    lo = hi = 0
    off = s.replica_offset
    for r in range(s.n_replicas):
        a, b = _pairs_within(st["x"][off[r]:off[r + 1]], s.box[r], [RC - tol, RC + tol])
        lo += int(a)
        hi += int(b)
    assert lo <= n_gpu <= hi, (lo, n_gpu, hi)

    # sampled forces against the oracle's all pairs at the GPU's state
    idx = np.sort(np.random.default_rng(41).choice(s.n_atoms, min(300, s.n_atoms), replace=False))
    ss = dataclasses.replace(s, x=st["x"], q0=st["q"].astype(np.uint8))
    ref = oracle_mod.forces_of_atoms(ss, atom, idx, r_cut=RC, kappa=st["kappa"])
    rms, mx = force_errors(st["f"][idx], ref)
    assert rms <= TOL[prec], (rms, mx)
