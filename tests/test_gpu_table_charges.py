"""Table-driven charges (Sec. II.A: integer charges assigned so that, averaged,
they match the CR charge-state fractions) on the GPU, through the C ABI
(-m gpu): charge sequences bit-exact against the oracle at every step, and
the argument checks of md_set_charge_table."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("case", ["methane", "water"])
def test_table_charges_bit_exact(oracle_mod, prec, case):
    if case == "methane":
        s, rc = methane(200, charge_frac=0.0), 1.2
    else:
        s, rc = water(300, charge_frac=0.0)
    atom = W.atomic_data(8.0)
    steps = 40
    pulses = [W.Pulse(8.0, 1.0, 1e12, 0.5)]
    table = W.charge_fraction_table(pulses, 0.0, 0.05, steps + 1, mean_final=3.0)
    gpu = M.IonisingMD(s, atom, precision=prec, r_cut=rc, max_steps=steps, charge_mode="table")
    gpu.set_charge_table(table)
    ora = oracle_mod.OracleMD(s, atom, r_cut=rc, n_steps_max=steps, charge_table=table[None])
    for n in range(steps):
        gpu.step(1)
        ora.step()
        st = gpu.get_state(M.MD_FIELD_Q | M.MD_FIELD_H | M.MD_FIELD_PLASMA | M.MD_FIELD_COUNTS)
        assert np.array_equal(st["q"], ora.q), n
        assert not st["h"].any()
        assert st["n_e"][0] == ora.n_e[0] == int(ora.q.astype(np.int64).sum()), n
        assert np.array_equal(st["event_counts"][0], ora.counts[0]), n
    assert ora.q.mean() > 0.5          # the table ionised the sample
    gpu.close()


def test_set_charge_table_checks_its_arguments():
    s = methane(20, charge_frac=0.0)
    atom = W.atomic_data(8.0)
    n_ts = int(W.ts_offsets().max())
    good = W.charge_fraction_table([W.Pulse(8.0, 1.0, 1e12, 0.5)], 0.0, 0.05, 5)
    g = M.IonisingMD(s, atom, max_steps=4)                     # rates mode
    with pytest.raises(M.MDError):
        g.set_charge_table(good)
    g.close()
    g = M.IonisingMD(s, atom, max_steps=4, charge_mode="table")
    bad = good.copy()
    bad[2, 1] += 0.1                                           # hydrogen row sums to 1.1
    with pytest.raises(M.MDError):
        g.set_charge_table(bad)
    with pytest.raises(M.MDError):
        g.set_charge_table(np.zeros((6, n_ts)) + good[0])       # more rows than max_steps + 1
    g.set_charge_table(good)
    g.step(4)
    g.close()
