"""Bonded terms (Sec. II.B, Eqs. 9-10) on the GPU against the FP64 CPU oracle,
through the C ABI (-m gpu).

The tolerances are those of the non-bonded path:
  * forces: RMS relative error <= 1e-5 (mixed) and 1e-12 (FP64);
  * energy: within 1e-5 (mixed) and 1e-10 (FP64) of sum |U_i|;
  * charges: bit-exact;
  * positions over the first steps: RMS <= 1e-6 nm (mixed) and 1e-9 nm (FP64).

The states are displaced from the molecules' equilibrium geometry and carry
charges 0-3, so the Morse and angle forces are large and the charge scaling
of Eq. 9 takes every value from 1 down to 0.
"""
import dataclasses

import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import force_errors, methane, water

pytestmark = pytest.mark.gpu

TOL_F = {"mixed": 1e-5, "fp64": 1e-12}
TOL_U = {"mixed": 1e-5, "fp64": 1e-10}
TOL_X = {"mixed": 1e-6, "fp64": 1e-9}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"


def _bonded(s, seed=3, shake=0.008):
    """The sample with its molecules' bonded terms, atoms shaken off equilibrium
    (kept inside a periodic box)."""
    s = W.with_topology(s)
    rng = np.random.default_rng(seed)
    x = s.x + rng.normal(scale=shake, size=s.x.shape)
    if s.box[0, 0] > 0:
        x = np.mod(x, s.box[0])
    return dataclasses.replace(s, x=x)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("case", ["water", "methane"])
def test_bonded_forces_and_energy_match_oracle(oracle_mod, prec, case):
    if case == "water":
        s, rc = water(1000)
    else:
        s, rc = methane(300), 1.2
    s = _bonded(s)
    t = s.topology
    cb = oracle_mod.bond_scale(s.q0[t.bonds[:, 0]].astype(float) + s.q0[t.bonds[:, 1]], 2)
    assert (cb == 0).any() and (cb == 1).any() and ((cb > 0) & (cb < 1)).any()
    atom = W.atomic_data(8.0)
    gpu = M.IonisingMD(s, atom, precision=prec, r_cut=rc, cr_enabled=False, max_steps=10)
    ora = oracle_mod.OracleMD(s, atom, r_cut=rc, cr_enabled=False)
    st = gpu.get_state(M.MD_FIELD_F | M.MD_FIELD_PLASMA)
    assert st["kappa"][0] == ora.scal[0]["kappa"]
    rms, mx = force_errors(st["f"], ora.F)
    assert rms <= TOL_F[prec], (rms, mx)
    # the bonded terms change the forces: not the non-bonded result
    plain = oracle_mod.OracleMD(dataclasses.replace(s, topology=None), atom, r_cut=rc, cr_enabled=False)
    assert force_errors(plain.F, ora.F)[0] > 1e-2
    assert np.abs(st["f"].sum(0)).max() <= (1e-6 if prec == "mixed" else 1e-12) * np.abs(st["f"]).sum(0).max()
    ek, ep, _ = gpu.energies()
    assert abs(ep[0] - ora.potential()[0]) <= TOL_U[prec] * np.abs(ora.U).sum()
    gpu.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_bonded_trajectory_matches_oracle(oracle_mod, prec):
    s, rc = water(400)
    s = _bonded(s, shake=0.004)
    atom = W.atomic_data(6.0, pi_scale=3000.0)
    pulses = [W.Pulse(6.0, 5.0, 1e12, 0.0)]
    gpu = M.IonisingMD(s, atom, precision=prec, r_cut=rc, max_steps=40, t_start_fs=-2.0)
    gpu.set_pulse(pulses)
    ora = oracle_mod.OracleMD(s, atom, r_cut=rc, t_start_fs=-2.0, pulses=[pulses], n_steps_max=40)
    for _ in range(30):
        gpu.step(1)
        ora.step()
    st = gpu.get_state(M.MD_FIELD_X | M.MD_FIELD_Q | M.MD_FIELD_F)
    gpu.close()
    assert np.array_equal(st["q"], ora.q)
    assert ora.n_e[0] > 0
    L = s.box[0]
    d = st["x"] - ora.x
    d -= L * np.round(d / L)
    assert float(np.sqrt((d ** 2).sum(1).mean())) <= TOL_X[prec]
    rms, mx = force_errors(st["f"], ora.F)
    assert rms <= TOL_F[prec], (rms, mx)


def test_bonded_with_verlet_buffer_and_replicas():
    """Bonded terms through the buffered list and in a batch of replicas:
    each replica equals its solo run bit for bit, and the buffered run
    equals the unbuffered one to FP32 rounding."""
    reps = [_bonded(methane(n, seed=k + 21), seed=k) for k, n in enumerate((30, 55, 17))]
    for k, r in enumerate(reps):
        r.seed[:] = 700 + k
    atom = W.atomic_data(8.0, pi_scale=1500.0, ci_scale=10.0)
    pulses = [[W.Pulse(8.0, 10.0, f, 0.0)] for f in (1e12, 4e11, 2e12)]
    kw = dict(max_steps=60, t_start_fs=-5.0)
    batch = W.concat(reps)
    assert len(batch.topology.bonds) == sum(len(r.topology.bonds) for r in reps)
    g = M.IonisingMD(batch, atom, **kw)
    for k, p in enumerate(pulses):
        g.set_pulse(p, replica=k)
    g.step(40)
    sb = g.get_state(M.MD_FIELD_ALL)
    g.close()
    off = batch.replica_offset
    for k, r in enumerate(reps):
        h = M.IonisingMD(r, atom, **kw)
        h.set_pulse(pulses[k])
        h.step(40)
        so = h.get_state(M.MD_FIELD_ALL)
        h.close()
        sl = slice(off[k], off[k + 1])
        for key in ("x", "v", "f", "q", "h"):
            assert np.array_equal(sb[key][sl], so[key]), (k, key)
    out = []
    for skin in (0.0, 0.02):
        g = M.IonisingMD(reps[1], atom, list_skin_nm=skin, **kw)
        g.set_pulse(pulses[1])
        g.step(40)
        out.append(g.get_state(M.MD_FIELD_F | M.MD_FIELD_Q))
        g.close()
    assert np.array_equal(out[0]["q"], out[1]["q"])
    assert force_errors(out[1]["f"], out[0]["f"])[0] <= 1e-5


def test_bonded_energy_is_conserved_without_ionisation():
    """NVE with Morse bonds and angles (no pulse, no charges): the total
    energy stays within a small fraction of the vibrational energy."""
    s, rc = water(300, charge_frac=0.0)
    s = _bonded(s, shake=0.003)
    atom = W.atomic_data(6.0)
    g = M.IonisingMD(s, atom, precision="fp64", r_cut=rc, cr_enabled=False, max_steps=2000, kappa_fixed=0.0)
    e = []
    for _ in range(10):
        ek, ep, _ = g.energies()
        e.append(ek[0] + ep[0])
        g.step(100)
    g.close()
    e = np.array(e)
    # ~9 vibrational periods of the O-H bonds; Verlet at 50 as keeps the
    # fluctuation of the total well below 1e-3 of the kinetic energy
    assert np.abs(e - e[0]).max() <= 1e-3 * abs(ek[0])
