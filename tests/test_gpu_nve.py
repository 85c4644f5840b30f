"""NVE energy behaviour of the GPU paths (-m gpu; Sec. II.B, Eq. 12, velocity
Verlet), with ionisation off, fixed charges and a fixed screening length, on
the periodic water box of the oracle's own NVE pin:

* FP64 path: the total energy's deviation stays below 1e-2 kJ/mol per atom
  over 20 fs and shrinks 3-5x when dt halves (second order), and it matches
  the oracle's deviation on the same run within 5 %;
* mixed path: the FP32 pair forces add noise but no drift beyond the FP64
  path's deviation plus 1e-4 kJ/mol per atom.
"""
import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RC, KAPPA, NMOL = 0.85, 10.0, 600


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"


def _sample():
    s = W.workload("c2_water_30k", scale=NMOL / 10000).sample
    s.q0[::2] = 1
    return s


def _gpu_dev(prec, dt, steps, every):
    s = _sample()
    g = M.IonisingMD(s, W.atomic_data(6.0), precision=prec, dt_ps=dt, r_cut=RC, cr_enabled=False,
                     kappa_fixed=KAPPA, max_steps=steps + 1)
    e = []
    for _ in range(steps // every):
        g.step(every)
        ek, ep, _ = g.energies()
        e.append(ek[0] + ep[0])
    g.close()
    e = np.array(e)
    return float(np.abs(e - e[0]).max() / s.n_atoms)


def test_nve_second_order_and_oracle(oracle_mod):
    dev1 = _gpu_dev("fp64", 5e-5, 400, 10)
    dev2 = _gpu_dev("fp64", 2.5e-5, 800, 20)
    assert dev1 < 1e-2, dev1
    assert 3.0 < dev1 / dev2 < 5.0, (dev1, dev2)
    s = _sample()
    md = oracle_mod.OracleMD(s, W.atomic_data(6.0), dt_ps=5e-5, r_cut=RC, cr_enabled=False, kappa_fixed=KAPPA)
    e = []
    for k in range(400):
        md.step()
        if (k + 1) % 10 == 0:
            e.append(md.kinetic()[0] + md.potential()[0])
    e = np.array(e)
    dev_o = float(np.abs(e - e[0]).max() / s.n_atoms)
    assert dev1 == pytest.approx(dev_o, rel=0.05), (dev1, dev_o)
    mixed = _gpu_dev("mixed", 5e-5, 400, 10)
    assert mixed <= dev1 + 1e-4, (mixed, dev1)
