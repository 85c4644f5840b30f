"""The widened rows together on the GPU (-m gpu): hybrid electrostatics,
Langevin coupling, bonded terms, probe records and table-driven charges in
one run, against the FP64 oracle running the same options; and a checkpoint
of such a run, resumed in a new handle through the Verlet-buffered list,
equal to the straight run bit for bit.

Tolerances are those of each row alone: charges bit-exact; positions RMS
<= 1e-6 nm (mixed) / 1e-9 nm (FP64); forces RMS relative <= 1e-5 / 1e-12;
velocities as in the Langevin test (the coupling heats the ions to T_e)."""
import dataclasses

import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import force_errors, water

pytestmark = pytest.mark.gpu

TOL_X = {"mixed": 1e-6, "fp64": 1e-9}
TOL_F = {"mixed": 1e-5, "fp64": 1e-12}
TOL_V = {"mixed": 1e-4, "fp64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"


def _sample(n_mol=400, shake=0.004, seed=5):
    s, rc = water(n_mol)
    s = W.with_topology(s)
    x = s.x + np.random.default_rng(seed).normal(scale=shake, size=s.x.shape)
    return dataclasses.replace(s, x=np.mod(x, s.box[0])), rc


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("charges", ["rates", "table"])
def test_all_rows_together_match_oracle(oracle_mod, prec, charges):
    s, rc = _sample()
    atom = W.atomic_data(6.0, pi_scale=3000.0)
    pulses = [W.Pulse(6.0, 5.0, 1e12, 0.0)]
    g_e = np.full(len(atom.z), 0.5)
    steps = 25
    kw = dict(r_cut=rc, max_steps=40, t_start_fs=-2.0, screening="hybrid", langevin_g=g_e, probe_record=True)
    okw = dict(r_cut=rc, t_start_fs=-2.0, pulses=[pulses], n_steps_max=40, screening="hybrid", langevin_g=g_e)
    if charges == "table":
        tab = W.charge_fraction_table(pulses, -2.0, 0.05, 41, mean_final=1.5)
        kw.update(charge_mode="table")
        okw.update(charge_table=tab[None])
    gpu = M.IonisingMD(s, atom, precision=prec, **kw)
    gpu.set_pulse(pulses)
    if charges == "table":
        gpu.set_charge_table(tab)
    ora = oracle_mod.OracleMD(s, atom, **okw)
    for _ in range(steps):
        gpu.step(1)
        ora.step()
    st = gpu.get_state(M.MD_FIELD_X | M.MD_FIELD_V | M.MD_FIELD_Q | M.MD_FIELD_F | M.MD_FIELD_PLASMA)
    qg, dg = gpu.probe_series()
    gpu.close()
    assert np.array_equal(st["q"], ora.q) and st["n_e"][0] == ora.n_e[0]
    assert (ora.q != s.q0).sum() > 50               # the charges moved (the table resets the start's)
    L = s.box[0]
    d = st["x"] - ora.x
    d -= L * np.round(d / L)
    assert float(np.sqrt((d ** 2).sum(1).mean())) <= TOL_X[prec]
    rms, mx = force_errors(st["f"], ora.F)
    assert rms <= TOL_F[prec], (rms, mx)
    scale = np.linalg.norm(ora.v, axis=1) + 1.0
    assert np.percentile(np.abs(st["v"] - ora.v).max(1) / scale, 98) <= TOL_V[prec]
    qo, do = ora.probe_series(0)
    assert np.array_equal(qg, qo)
    n_of = np.bincount(s.species, minlength=len(atom.z))
    assert (np.abs(dg - do) <= 2e-3 * do + n_of * 2.0 ** -41).all()


def test_checkpoint_of_all_rows_resumes_bit_exact():
    s, rc = _sample(300)
    rc -= 0.06                                      # room for the skin: box >= 3 (r_cut + skin)
    atom = W.atomic_data(6.0, pi_scale=1500.0, ci_scale=20.0)
    p = [W.Pulse(6.0, 4.0, 3e12, 0.0)]
    kw = dict(r_cut=rc, max_steps=60, t_start_fs=-1.5, screening="hybrid", langevin_g=np.full(5, 0.3),
              probe_record=True, list_skin_nm=0.05)
    ALL = M.MD_FIELD_ALL
    g = M.IonisingMD(s, atom, **kw)
    g.set_pulse(p)
    g.step(40)
    straight = g.get_state(ALL)
    series = g.probe_series()
    g.close()
    g = M.IonisingMD(s, atom, **kw)
    g.set_pulse(p)
    g.step(20)
    ck = g.get_state(ALL)
    g.close()
    h = M.IonisingMD(s, atom, **kw)
    h.set_pulse(p)
    h.set_state(ALL, **{k: ck[k] for k in ("x", "v", "q", "h", "n_e", "e_gas_mev", "event_counts", "x_list")},
                step=ck["step"])
    h.step(20)
    resumed = h.get_state(ALL)
    q2, d2 = h.probe_series(first=20, n=21)
    h.close()
    for k in ("x", "v", "f", "q", "h", "n_e", "e_gas_mev", "event_counts", "x_list"):
        assert np.array_equal(straight[k], resumed[k]), k
    assert np.array_equal(q2, series[0][20:]) and np.array_equal(d2, series[1][20:])
