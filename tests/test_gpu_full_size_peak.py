"""The 2 M-atom droplet at its pulse peak in the benchmark's configuration, -m gpu.

The bench times the droplet (the largest workload) around the peak of its
pulse with the Verlet buffer (0.12 nm skin), autotuned launch shapes and
eight steps per graph launch; there the ionised droplet Coulomb-explodes and
the list is rebuilt every few steps.  After 400 steps from the start of the
run (t = 0 fs, the peak, with the charge dynamics on), the state must hold:

* every pair within r_cut: the force kernel's in-cutoff pair count equals an
  exact KD-tree count of the pairs closer than r_cut, up to the pairs within
  1e-6 nm of it (FP32 cell-relative distances are good to ~1e-7 nm there);
* the forces of 300 sampled atoms equal the FP64 oracle's all-pair forces at
  the GPU's positions, charges and kappa (Sec. II.A Eq. 2, Sec. II.B Eq. 8)
  within the mixed path's 1e-5 RMS relative error;
* the screened Coulomb term is live (kappa > 0, free electrons present) and
  the buffer was used (fewer builds than steps, more than one).
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
STEPS = 400          # t_start = -20 fs, 50 as per step: the pulse peak


def test_droplet_at_the_pulse_peak_in_the_bench_configuration(oracle_mod):
    import torch
    from scipy.spatial import cKDTree
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    wl = W.workload("c5_droplet_2m")
    s = wl.sample
    atom = W.atomic_data(wl.photon_kev)
    g = M.IonisingMD(s, atom, r_cut=RC, max_steps=wl.n_steps, t_start_fs=wl.t_start_fs, autotune=True,
                     list_skin_nm=SKIN)
    g.set_pulse(wl.pulses[0])
    g.step(STEPS)
    st = g.get_state(M.MD_FIELD_X | M.MD_FIELD_Q | M.MD_FIELD_F | M.MD_FIELD_PLASMA | M.MD_FIELD_STEP)
    _, _, n_gpu = g.energies()
    t = g.timing()
    g.close()
    assert st["step"] == STEPS
    assert st["kappa"][0] > 1.0 and st["n_e"][0] > 0
    assert 1 < t.list_builds < STEPS, t.list_builds

    # every pair within r_cut
    tree = cKDTree(st["x"])
    tol = 1e-6
    lo, hi = (tree.count_neighbors(tree, np.array([RC - tol, RC + tol])) - s.n_atoms) // 2
    assert lo <= n_gpu <= hi, (lo, n_gpu, hi)

    # sampled forces against the oracle's all pairs at the GPU's state
    idx = np.sort(np.random.default_rng(41).choice(s.n_atoms, 300, replace=False))
    ss = dataclasses.replace(s, x=st["x"], q0=st["q"].astype(np.uint8))
    ref = oracle_mod.forces_of_atoms(ss, atom, idx, r_cut=RC, kappa=st["kappa"])
    rms, mx = force_errors(st["f"][idx], ref)
    assert rms <= 1e-5, (rms, mx)
