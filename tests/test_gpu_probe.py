"""Probe records and the probe-weighted displacement (Sec. II.C, Eq. 17) on
the GPU, through the C ABI (-m gpu), against the FP64 oracle:

* summed charges per species: bit-exact at every step;
* summed squared displacements: within the trajectory tolerance (positions
  RMS <= 1e-6 nm mixed, 1e-9 nm FP64) -- relative 2e-3 (mixed) and 1e-6 (FP64)
  over 30 steps, where |x - x0| grows to ~1e-3 nm -- plus the fixed point's
  rounding, half of 2^-40 nm^2 per atom;
* the library's Eq. 17 evaluation equals the oracle's on the same series;
* batched replicas record what their solo runs record, bit for bit, and a
  restored checkpoint rewrites its record bit for bit.
"""
import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import methane, water

pytestmark = pytest.mark.gpu

TOL_D2 = {"mixed": 2e-3, "fp64": 1e-6}
PROBE = [W.Pulse(6.0, 0.6, 1e12, -1.0)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_probe_series_and_displacement_match_oracle(oracle_mod, prec):
    s, rc = water(400)
    atom = W.atomic_data(6.0, pi_scale=3000.0)
    pulses = [W.Pulse(6.0, 5.0, 1e12, 0.0)]
    steps = 30
    gpu = M.IonisingMD(s, atom, precision=prec, r_cut=rc, max_steps=40, t_start_fs=-2.0, probe_record=True)
    gpu.set_pulse(pulses)
    ora = oracle_mod.OracleMD(s, atom, r_cut=rc, t_start_fs=-2.0, pulses=[pulses], n_steps_max=40)
    for _ in range(steps):
        gpu.step(1)
        ora.step()
    qg, dg = gpu.probe_series()
    qo, do = ora.probe_series(0)
    assert qg.shape == (steps + 1, len(atom.z))
    assert np.array_equal(qg, qo)
    assert qo[-1].sum() > qo[0].sum()                       # the pulse ionises
    assert not dg[0].any()
    present = do[-1] > 0
    n_of = np.bincount(s.species, minlength=len(atom.z))
    # the trajectory tolerance, plus half a 2^-40 nm^2 unit of rounding per atom
    assert (np.abs(dg - do) <= TOL_D2[prec] * do + n_of * 2.0 ** -41).all()
    Dg = gpu.probe_displacement(PROBE, first=0, n=steps + 1)
    Dq = oracle_mod.probe_weighted_displacement(PROBE, -2.0, 0.05, qg, dg, n_of, atom.z)
    assert np.allclose(Dg, Dq, rtol=1e-12, atol=0)
    Do = oracle_mod.probe_weighted_displacement(PROBE, -2.0, 0.05, qo, do, n_of, atom.z)
    assert np.allclose(Dg, Do, rtol=TOL_D2[prec], atol=0) and (Dg[present] > 0).all()
    # a window of the records
    Dw = gpu.probe_displacement(PROBE, first=10, n=15)
    assert np.allclose(Dw, oracle_mod.probe_weighted_displacement(PROBE, -2.0 + 10 * 0.05, 0.05, qg[10:25], dg[10:25],
                                                                  n_of, atom.z), rtol=1e-12, atol=0)
    with pytest.raises(M.MDError):
        gpu.probe_series(first=0, n=steps + 2)               # beyond the current step
    gpu.close()


def test_probe_records_batched_equal_solo_and_resume():
    reps = [methane(n, seed=k + 31) for k, n in enumerate((25, 60, 14))]
    for k, r in enumerate(reps):
        r.seed[:] = 800 + k
    atom = W.atomic_data(8.0, pi_scale=1500.0, ci_scale=10.0)
    pulses = [[W.Pulse(8.0, 10.0, f, 0.0)] for f in (1e12, 3e11, 2e12)]
    kw = dict(max_steps=50, t_start_fs=-5.0, probe_record=True)
    batch = W.concat(reps)
    g = M.IonisingMD(batch, atom, **kw)
    for k, p in enumerate(pulses):
        g.set_pulse(p, replica=k)
    g.step(20)
    ck = g.get_state(M.MD_FIELD_ALL)
    g.step(20)
    sb = [g.probe_series(replica=k) for k in range(3)]
    # restore the checkpoint of step 20: record 20 is rewritten identically,
    # and the next 20 steps record the same values again
    g.set_state(M.MD_FIELD_ALL, **{k: ck[k] for k in ("x", "v", "q", "h", "n_e", "e_gas_mev", "event_counts",
                                                      "x_list")}, step=ck["step"])
    g.step(20)
    for k in range(3):
        q2, d2 = g.probe_series(replica=k)
        assert np.array_equal(q2, sb[k][0]) and np.array_equal(d2, sb[k][1])
    g.close()
    for k, r in enumerate(reps):
        h = M.IonisingMD(r, atom, **kw)
        h.set_pulse(pulses[k])
        h.step(40)
        qs, ds = h.probe_series()
        h.close()
        assert np.array_equal(qs, sb[k][0]) and np.array_equal(ds, sb[k][1]), k


def test_probe_records_off_is_an_error():
    s = methane(10)
    g = M.IonisingMD(s, W.atomic_data(8.0), max_steps=5)
    with pytest.raises(M.MDError) as e:
        g.probe_series(n=1)
    assert e.value.status == M.MD_ERR_BAD_STATE
    g.close()
