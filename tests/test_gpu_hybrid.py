"""Hybrid ion-sphere / Debye electrostatics (Sec. II.A, Eqs. 4-7) on the GPU
against the FP64 CPU oracle, through the C ABI (-m gpu).

The tolerances are those of the Debye path:
  * forces: RMS relative error <= 1e-5 (mixed) and 1e-12 (FP64);
  * energy: within 1e-5 (mixed) and 1e-10 (FP64) of sum |U_i|;
  * charges: bit-exact;
  * positions over the first steps: RMS <= 1e-6 nm (mixed) and 1e-9 nm (FP64).

The states are chosen so that bonded and close pairs lie inside the ion
spheres (r' of 0.1-0.3 nm): both branches of the potential are exercised.
"""
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


def _pairs_inside(x, box, rp):
    from scipy.spatial import cKDTree
    periodic = box is not None and box[0] > 0
    t = cKDTree(np.mod(x, box) if periodic else x, boxsize=box if periodic else None)
    return len(t.query_pairs(rp))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("case", ["water", "methane"])
def test_hybrid_forces_and_energy_match_oracle(oracle_mod, prec, case):
    if case == "water":
        s, rc = water(1000)
    else:
        s, rc = methane(300), 1.2
    atom = W.atomic_data(8.0)
    gpu = M.IonisingMD(s, atom, precision=prec, r_cut=rc, cr_enabled=False, max_steps=10, screening="hybrid")
    ora = oracle_mod.OracleMD(s, atom, r_cut=rc, cr_enabled=False, screening="hybrid")
    ne, kap = ora.scal[0]["n_e"], ora.scal[0]["kappa"]
    rp = max(oracle_mod.hybrid_coeffs(q, ne, kap)[0] for q in np.unique(s.q0) if q > 0)
    box = s.box[0] if s.box[0, 0] > 0 else None
    assert ne > 0 and kap > 0 and _pairs_inside(s.x, box, rp) > 100, (ne, kap, rp)

    st = gpu.get_state(M.MD_FIELD_F | M.MD_FIELD_PLASMA)
    assert st["kappa"][0] == kap
    rms, mx = force_errors(st["f"], ora.F)
    assert rms <= TOL_F[prec], (rms, mx)
    # the ion spheres change the forces: not the Debye result
    deb = oracle_mod.OracleMD(s, atom, r_cut=rc, cr_enabled=False)
    assert force_errors(deb.F, ora.F)[0] > 1e-3
    # Newton's third law to float rounding of the block sums
    assert np.abs(st["f"].sum(0)).max() <= (1e-6 if prec == "mixed" else 1e-12) * np.abs(st["f"]).sum(0).max()
    ek, ep, _ = gpu.energies()
    assert abs(ep[0] - ora.potential()[0]) <= TOL_U[prec] * np.abs(ora.U).sum()
    gpu.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_hybrid_trajectory_matches_oracle(oracle_mod, prec):
    s, rc = water(400)
    atom = W.atomic_data(6.0, pi_scale=3000.0)
    pulses = [W.Pulse(6.0, 5.0, 1e12, 0.0)]
    gpu = M.IonisingMD(s, atom, precision=prec, r_cut=rc, max_steps=40, t_start_fs=-2.0, screening="hybrid")
    gpu.set_pulse(pulses)
    ora = oracle_mod.OracleMD(s, atom, r_cut=rc, t_start_fs=-2.0, pulses=[pulses], n_steps_max=40,
                              screening="hybrid")
    for _ in range(30):
        gpu.step(1)
        ora.step()
    st = gpu.get_state(M.MD_FIELD_X | M.MD_FIELD_Q | M.MD_FIELD_F | M.MD_FIELD_PLASMA)
    assert np.array_equal(st["q"], ora.q)
    assert st["n_e"][0] == ora.n_e[0] and st["kappa"][0] == ora.scal[0]["kappa"]
    L = s.box[0]
    d = st["x"] - ora.x
    d -= L * np.round(d / L)
    assert float(np.sqrt((d ** 2).sum(1).mean())) <= TOL_X[prec]
    rms, mx = force_errors(st["f"], ora.F)
    assert rms <= TOL_F[prec], (rms, mx)
    gpu.close()


def test_hybrid_with_verlet_buffer_matches_unbuffered():
    """The hybrid term through the buffered list (trimmed masks, fragment
    flags): same forces as a list rebuilt every step, to FP32 rounding."""
    s, rc = water(1000)
    rc = 0.9
    atom = W.atomic_data(6.0, pi_scale=800.0)
    p = [W.Pulse(6.0, 4.0, 3e12, 0.0)]
    out = []
    for skin in (0.0, 0.01):
        g = M.IonisingMD(s, atom, r_cut=rc, max_steps=40, t_start_fs=-1.5, list_skin_nm=skin, screening="hybrid")
        g.set_pulse(p)
        g.step(25)
        out.append(g.get_state(M.MD_FIELD_F | M.MD_FIELD_Q))
        g.close()
    assert np.array_equal(out[0]["q"], out[1]["q"])
    rms, _ = force_errors(out[1]["f"], out[0]["f"])
    assert rms <= 1e-5, rms
