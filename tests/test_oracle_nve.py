"""Pin of the oracle's integrator (Sec. II.B, Eq. 12; velocity Verlet).

With ionisation off, fixed charges and a fixed screening length, the total
energy (kinetic + cutoff-shifted potential) of a periodic water box is
conserved: its deviation stays bounded and shrinks 4x when dt halves
(second order).  A dropped half-kick or a kick with stale forces turns the
ratio into ~2 (first order) and fails this test.
"""
import numpy as np

from paper_2401_03180_gb300 import workloads as W


def _energies(oracle_mod, dt, steps, kappa=10.0, rc=0.95, nmol=300):
    wl = W.workload("c2_water_30k", scale=nmol / 10000)
    s = wl.sample
    s.q0[::2] = 1
    md = oracle_mod.OracleMD(s, W.atomic_data(6.0), dt_ps=dt, r_cut=rc, cr_enabled=False,
                             kappa_fixed=kappa)
    e = []
    for _ in range(steps):
        md.step()
        e.append(md.kinetic()[0] + md.potential()[0])
    return md.n, np.array(e)


def test_nve_second_order(oracle_mod):
    n, e1 = _energies(oracle_mod, 5e-5, 400)
    _, e2 = _energies(oracle_mod, 2.5e-5, 800)
    dev1 = np.abs(e1 - e1[0]).max() / n
    dev2 = np.abs(e2[1::2] - e2[1]).max() / n
    assert dev1 < 1e-2, dev1          # kJ/mol per atom over 20 fs
    assert 3.0 < dev1 / dev2 < 5.0, (dev1, dev2)
