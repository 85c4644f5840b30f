"""Charge-state parity at the full sizes of the large workloads (-m gpu).

The stochastic integer charges (Sec. II.A; the reading "RCM-1": photo-
ionisation, Auger decay, collisional ionisation and recombination drawn from
Philox4x32-10 keyed by (seed, atom, step)) must be bit-exact against the FP64
oracle.  The small parity tests run the step kernel's variant for small
grids; these run, in the bench's launch configuration (Verlet-buffered list,
autotuned force kernel):

  * the 2,000,000-atom water droplet, whose grid of 62,500 blocks takes the
    step kernel's variant for grids of at least 16 blocks per SM, with the
    charge update on;
  * the 256-replica methane batch (500-20,000 atoms each, log-uniform, with
    its own fluence and seed per replica), whose per-replica plasma
    reduction runs in its own kernel (more than four replicas).

Charges never read positions (the electron gas is homogeneous and of fixed
volume), so the oracle advances the charge dynamics alone
(`OracleMD(with_forces=False)`, pinned to the full step in
`test_oracle_cr.py`) and no all-pairs forces are needed.  Every step the
charges, K holes, electron counts, gas energies, event counts, T_e and the
screening kappa of Eq. 3 must be equal, bit for bit.
"""
import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

pytestmark = pytest.mark.gpu
STEPS = 24
T_START_FS = -3.0    # near the pulse peak, where the rates are largest


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("name", ["c5_droplet_2m", "c4_methane_batch"])
def test_full_size_charge_sequences_bit_exact(oracle_mod, name):
    import torch
    wl = W.workload(name)
    s = wl.sample
    # 5 % of the atoms start singly ionised, so that collisional ionisation and
    # recombination act from the first step; photo-absorption scaled up 30x, so
    # that a 24-step window holds every channel
    rng = np.random.default_rng(5)
    s.q0[rng.random(s.n_atoms) < 0.05] = 1
    atom = W.atomic_data(wl.photon_kev, pi_scale=30.0)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    if name.startswith("c5"):
        assert (s.n_atoms + 31) // 32 >= 16 * n_sm      # the many-blocks variant of the step kernel
    else:
        assert s.n_replicas > 4                         # the separate per-replica reduction
    gpu = M.IonisingMD(s, atom, r_cut=1.2, max_steps=STEPS + 8, t_start_fs=T_START_FS, list_skin_nm=0.08,
                       autotune=True)
    for r in range(s.n_replicas):
        gpu.set_pulse(wl.pulses[r], replica=r)
    ora = oracle_mod.OracleMD(s, atom, r_cut=1.2, t_start_fs=T_START_FS, pulses=wl.pulses, n_steps_max=STEPS + 8,
                              with_forces=False)
    fields = M.MD_FIELD_Q | M.MD_FIELD_H | M.MD_FIELD_PLASMA | M.MD_FIELD_COUNTS
    for n in range(STEPS):
        gpu.step(1)
        ora.step()
        st = gpu.get_state(fields)
        assert np.array_equal(st["q"], ora.q), n
        assert np.array_equal(st["h"], ora.h), n
        assert np.array_equal(st["n_e"], ora.n_e), n
        assert np.array_equal(st["e_gas_mev"], ora.e_gas), n
        assert np.array_equal(st["event_counts"], ora.counts), n
        assert np.array_equal(st["kappa"], np.array([sc["kappa"] for sc in ora.scal])), n
        assert np.array_equal(st["te_ev"], np.array([sc["te_ev"] for sc in ora.scal])), n
    tot = ora.counts.sum(0)
    assert np.all(tot > 0), tot                     # every channel fired
    assert (ora.n_e > 0).all()
    gpu.close()
