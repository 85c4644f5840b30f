"""GPU path vs the FP64 CPU oracle, through the C ABI (-m gpu).

Tolerances (the method's stated targets; the FP64 ones from the fixed-point
rounding of 2^-32 per contribution against forces of ~1e2-1e4 kJ/mol/nm):
  * charges, K-holes, electron counts, gas energy, event counts: bit-exact;
  * kappa (double, Eq. 3): bit-exact;
  * forces, mixed path: RMS relative error <= 1e-5; FP64 path: <= 1e-12;
  * in-cutoff pair count: equal up to pairs within 1e-5 nm of r_cut;
  * positions over the first 50 steps: RMS <= 1e-6 nm (mixed), 1e-9 nm (FP64).
"""
import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import force_errors, methane, near_cutoff_pairs, water

pytestmark = pytest.mark.gpu

TOL_F = {"mixed": 1e-5, "fp64": 1e-12}
TOL_X = {"mixed": 1e-6, "fp64": 1e-9}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a GPU"


def _pair(sample, atomic, prec, oracle_mod, **kw):
    gpu = M.IonisingMD(sample, atomic, precision=prec, **kw)
    ora = oracle_mod.OracleMD(sample, atomic, dt_ps=kw.get("dt_ps", 5e-5), r_cut=kw.get("r_cut", 1.2),
                              cr_enabled=kw.get("cr_enabled", True), kappa_fixed=kw.get("kappa_fixed", -1.0),
                              t_start_fs=kw.get("t_start_fs", 0.0), n_steps_max=kw.get("max_steps", 1000))
    return gpu, ora


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("case", ["water", "methane", "protein"])
def test_forces_match_oracle(oracle_mod, prec, case):
    if case == "water":
        s, rc = water(1000)
    elif case == "methane":
        s, rc = methane(300), 1.2
    else:
        s, rc = W.workload("c3_protein_200k", scale=0.03).sample, 1.2
        s.q0[::3] = 1
    atom = W.atomic_data(8.0)
    gpu, ora = _pair(s, atom, prec, oracle_mod, r_cut=rc, cr_enabled=False, kappa_fixed=2.5, max_steps=10)
    st = gpu.get_state(M.MD_FIELD_F)
    rms, mx = force_errors(st["f"], ora.F)
    assert rms <= TOL_F[prec], (rms, mx)
    # Newton's third law holds to float rounding of the block sums
    net = st["f"].sum(0)
    assert np.abs(net).max() <= (1e-6 if prec == "mixed" else 1e-12) * np.abs(st["f"]).sum(0).max()
    ek, ep, npairs = gpu.energies()
    box = s.box[0] if s.box[0, 0] > 0 else None
    slack = near_cutoff_pairs(s.x, box, rc, 1e-5)
    assert abs(npairs - ora.n_pairs) <= slack, (npairs, ora.n_pairs, slack)
    # forces unchanged by the energy pass (same decomposition -> same bits)
    st2 = gpu.get_state(M.MD_FIELD_F)
    assert np.array_equal(st["f"], st2["f"])
    assert abs(ep[0] - ora.potential()[0]) <= (1e-5 if prec == "mixed" else 1e-10) * np.abs(ora.U).sum()
    assert abs(ek[0] - ora.kinetic()[0]) <= 1e-12 * ek[0]
    gpu.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_charge_sequences_bit_exact(oracle_mod, prec):
    s = methane(60, charge_frac=0.0)
    atom = W.atomic_data(8.0, pi_scale=2000.0, ci_scale=20.0, rec_scale=500.0)
    pulses = [W.Pulse(8.0, 10.0, 1e12, 0.0)]
    kw = dict(r_cut=1.2, cr_enabled=True, max_steps=300, t_start_fs=-7.0)
    gpu = M.IonisingMD(s, atom, precision=prec, **kw)
    gpu.set_pulse(pulses)
    ora = oracle_mod.OracleMD(s, atom, r_cut=1.2, cr_enabled=True, t_start_fs=-7.0, pulses=[pulses],
                              n_steps_max=300)
    seen = np.zeros(4, np.int64)
    for n in range(300):
        gpu.step(1)
        ora.step()
        st = gpu.get_state(M.MD_FIELD_Q | M.MD_FIELD_H | M.MD_FIELD_PLASMA | M.MD_FIELD_COUNTS)
        assert np.array_equal(st["q"], ora.q), n
        assert np.array_equal(st["h"], ora.h), n
        assert st["n_e"][0] == ora.n_e[0] and st["e_gas_mev"][0] == ora.e_gas[0], n
        assert np.array_equal(st["event_counts"][0], ora.counts[0]), n
        assert st["kappa"][0] == ora.scal[0]["kappa"], n
        assert st["te_ev"][0] == ora.scal[0]["te_ev"], n
        seen = st["event_counts"][0]
    assert np.all(seen > 0), seen          # every channel exercised
    gpu.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_trajectory_50_steps(oracle_mod, prec):
    s, rc = water(400)
    atom = W.atomic_data(6.0, pi_scale=3000.0)
    pulses = [W.Pulse(6.0, 5.0, 1e12, 0.0)]
    gpu = M.IonisingMD(s, atom, precision=prec, r_cut=rc, max_steps=60, t_start_fs=-2.0)
    gpu.set_pulse(pulses)
    ora = oracle_mod.OracleMD(s, atom, r_cut=rc, t_start_fs=-2.0, pulses=[pulses], n_steps_max=60)
    L = s.box[0]
    for n in range(50):
        gpu.step(1)
        ora.step()
    st = gpu.get_state(M.MD_FIELD_X | M.MD_FIELD_V | M.MD_FIELD_Q)
    assert np.array_equal(st["q"], ora.q)
    d = st["x"] - ora.x
    d -= L * np.round(d / L)
    rms = float(np.sqrt((d ** 2).sum(1).mean()))
    assert rms <= TOL_X[prec], rms
    # a pair within an FP32 ulp of r_cut may be inside on one side and outside on
    # the other; the truncated force then kicks its two atoms differently, so
    # velocities are compared on the 98th percentile, positions on the RMS
    # velocities drift as (force error / m) * t: with |F| ~ 1e4 kJ/mol/nm, m = 1 amu
    # and t = 50 dt = 2.5e-3 ps, a 1e-5 relative force error gives ~2.5e-4 nm/ps
    dv = np.abs(st["v"] - ora.v).max(1)
    bound = {"mixed": 2.5e-4, "fp64": 2.5e-11}[prec]
    assert np.percentile(dv, 98) <= bound, np.percentile(dv, 98)
    gpu.close()


def test_philox_device_matches_oracle(oracle_mod):
    import torch
    n = 1 << 20
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:1000] = 0
    ctr[:1000, 0] = np.arange(1000)
    for seed in (0, 1001, 0xDEADBEEF12345678):
        d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
        d_out = torch.empty_like(d_ctr)
        M.md_philox(seed, d_ctr.data_ptr(), n, d_out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint32)
        ref = oracle_mod.philox_blocks(seed, ctr)
        assert np.array_equal(got, ref)


def test_full_size_water_sampled(oracle_mod):
    """The bench workload (30,000-atom water box) in its bench configuration,
    checked on sampled atoms against the oracle."""
    wl = W.workload("c2_water_30k")
    s = wl.sample
    rng = np.random.default_rng(3)
    sel = rng.random(s.n_atoms) < 0.3
    s.q0[sel] = 1
    atom = W.atomic_data(wl.photon_kev)
    gpu = M.IonisingMD(s, atom, r_cut=1.2, cr_enabled=False, kappa_fixed=1.5, max_steps=10, autotune=True)
    st = gpu.get_state(M.MD_FIELD_F)
    idx = rng.choice(s.n_atoms, 400, replace=False)
    ref = _subset_forces(oracle_mod, s, atom, 1.2, 1.5, idx)
    rms, mx = force_errors(st["f"][idx], ref)
    assert rms <= 1e-5, (rms, mx)
    gpu.close()


def test_full_size_droplet_sampled(oracle_mod):
    """2,000,000-atom droplet (the largest workload): sampled force parity."""
    wl = W.workload("c5_droplet_2m")
    s = wl.sample
    rng = np.random.default_rng(4)
    s.q0[rng.random(s.n_atoms) < 0.2] = 1
    atom = W.atomic_data(wl.photon_kev)
    gpu = M.IonisingMD(s, atom, r_cut=1.2, cr_enabled=False, kappa_fixed=2.0, max_steps=4)
    gpu.step(2)
    st = gpu.get_state(M.MD_FIELD_F | M.MD_FIELD_X | M.MD_FIELD_Q)
    idx = rng.choice(s.n_atoms, 300, replace=False)
    s2 = W.Sample(x=st["x"], v=s.v, species=s.species, fragment=s.fragment, q0=st["q"],
                  replica_offset=s.replica_offset, seed=s.seed, box=s.box, volume=s.volume)
    ref = _subset_forces(oracle_mod, s2, atom, 1.2, 2.0, idx)
    rms, mx = force_errors(st["f"][idx], ref)
    assert rms <= 1e-5, (rms, mx)
    gpu.close()


def _subset_forces(oracle_mod, s, atom, rc, kappa, idx):
    return oracle_mod.forces_of_atoms(s, atom, idx, r_cut=rc, kappa=kappa)
