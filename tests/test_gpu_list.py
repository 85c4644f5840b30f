"""Cluster-pair list and asynchronous stepping (-m gpu): enqueued steps equal
synchronous ones, profile timing keeps every step, and a list that has to
grow while the atoms crowd together gives the same trajectory, bit for bit,
as a list that had room from the start."""
import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import water

pytestmark = pytest.mark.gpu
ALL = M.MD_FIELD_ALL
DT = 5e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _same(a, b):
    for k in ("x", "v", "f", "q", "h", "n_e", "e_gas_mev", "event_counts"):
        assert np.array_equal(a[k], b[k]), k
    assert a["step"] == b["step"]


def test_async_steps_equal_sync_steps():
    s, rc = water(500)
    atom = W.atomic_data(6.0, pi_scale=800.0, ci_scale=20.0)
    p = [W.Pulse(6.0, 4.0, 3e12, 0.0)]
    kw = dict(r_cut=rc, max_steps=60, t_start_fs=-1.5)
    states = []
    for mode in ("sync", "async", "async_then_get"):
        g = M.IonisingMD(s, atom, **kw)
        g.set_pulse(p)
        if mode == "sync":
            for _ in range(30):
                g.step(1)
        elif mode == "async":
            for _ in range(3):
                g.step(10, wait=False)
            g.sync()
        else:
            g.step(30, wait=False)   # get_state reads the status of pending steps itself
        states.append(g.get_state(ALL))
        g.close()
    _same(states[0], states[1])
    _same(states[0], states[2])
    assert states[0]["step"] == 30
    # fields read without host-side reordering: the copies and the status of
    # the pending steps come back in one round trip
    fused = M.MD_FIELD_V | M.MD_FIELD_F | M.MD_FIELD_Q | M.MD_FIELD_H | M.MD_FIELD_PLASMA | M.MD_FIELD_COUNTS | M.MD_FIELD_STEP
    g = M.IonisingMD(s, atom, **kw)
    g.set_pulse(p)
    got = []
    for _ in range(3):
        g.step(10, wait=False)
        got.append(g.get_state(fused))
    g.close()
    for k in ("v", "f", "q", "h", "n_e", "e_gas_mev", "te_ev", "kappa", "event_counts"):
        assert np.array_equal(got[-1][k], states[0][k]), k
    assert [st["step"] for st in got] == [10, 20, 30]


def test_profile_timing_counts_every_step():
    s, rc = water(300)
    atom = W.atomic_data(6.0)
    g = M.IonisingMD(s, atom, r_cut=rc, max_steps=700, profile=True)
    g.step(300, wait=False)          # more steps than event pairs kept in flight
    t = g.timing()
    assert t.pair_launches == 300 and t.steps == 300
    assert 0.0 < t.pair_ms / 300 < 10.0
    g.reset_timing()
    g.step(5)
    t = g.timing()
    assert t.pair_launches == 5 and t.steps == 5
    g.close()


def _compressing_box(n_mol, steps, f=0.5):
    """A periodic water box whose atoms move straight towards the box centre,
    ending at f times their distance from it in `steps` steps (density up by
    1/f^3 in the centre).  Cells then hold several super-clusters and the
    cluster pairs per cell grow with the square of the occupancy.  LJ is made
    negligible (and charges are zero), so the motion stays ballistic."""
    s, _ = water(n_mol, r_cut=1.0, charge_frac=0.0)
    c = 0.5 * s.box[0]
    target = c + f * (s.x - c)
    s.v = (target - s.x) / (steps * DT)
    return s, target


def _weak_lj():
    return dict(eps0=np.asarray(W.LJ_EPS0, dtype=np.float64) * 1e-6)


def _roomy_run(s, atom, kw, steps):
    """Step one at a time with a list that never fills; entries per build."""
    g = M.IonisingMD(s, atom, list_reserve=4096, **kw)
    t = g.timing()
    cluster_cap = t.list_capacity // 4096
    need = [t.list_entries]
    for _ in range(steps):
        g.step(1)
        need.append(g.timing().list_entries)
    st = g.get_state(ALL)
    assert g.timing().list_grows == 0
    g.close()
    return st, need, cluster_cap


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_list_growth_keeps_the_trajectory(prec):
    steps = 60
    s, _ = _compressing_box(3000, steps)
    atom = W.atomic_data(8.0)
    kw = dict(r_cut=1.0, max_steps=steps + 5, precision=prec, **_weak_lj())
    ref, need, cluster_cap = _roomy_run(s, atom, kw, steps)
    reserve = -(-need[0] // cluster_cap)            # room for the first build only
    assert reserve * cluster_cap < max(need), f"compression too weak: {need[0]} -> {max(need)}"
    g = M.IonisingMD(s, atom, list_reserve=reserve, **kw)
    t0 = g.timing()
    g.step(steps)                                   # one call: the list grows inside md_step
    t1 = g.timing()
    got = g.get_state(ALL)
    g.close()
    assert t1.list_grows > t0.list_grows
    assert t1.list_capacity >= max(need)
    _same(ref, got)
    # the same with the steps in flight when the state is read: the one-round-trip
    # read sees the overflow flag, lets md_sync grow the list, and copies again
    g = M.IonisingMD(s, atom, list_reserve=reserve, **kw)
    g.step(steps, wait=False)
    got2 = g.get_state(M.MD_FIELD_V | M.MD_FIELD_F | M.MD_FIELD_Q | M.MD_FIELD_PLASMA | M.MD_FIELD_STEP)
    assert g.timing().list_grows > 0
    g.close()
    for k in ("v", "f", "q", "n_e", "e_gas_mev"):
        assert np.array_equal(got2[k], ref[k]), k
    assert got2["step"] == steps


def test_list_growth_on_set_state():
    steps = 60
    s, target = _compressing_box(3000, steps)
    atom = W.atomic_data(8.0)
    kw = dict(r_cut=1.0, max_steps=20, **_weak_lj())
    out = {}
    for reserve in (None, 4096):
        if reserve is None:
            g = M.IonisingMD(s, atom, list_reserve=4096, **kw)
            reserve = -(-g.timing().list_entries // (g.timing().list_capacity // 4096))
            g.close()
            key = "tight"
        else:
            key = "roomy"
        g = M.IonisingMD(s, atom, list_reserve=reserve, **kw)
        grows0 = g.timing().list_grows
        g.set_state(M.MD_FIELD_X, x=target)          # about twice the list entries
        g.step(3)
        out[key] = (g.get_state(ALL), g.timing().list_grows - grows0)
        g.close()
    assert out["tight"][1] >= 1 and out["roomy"][1] == 0
    _same(out["tight"][0], out["roomy"][0])


# ---- Verlet-buffered list (list_skin_nm > 0) ----
SKIN = 0.01   # thermal atoms close half of it in ~15 steps: several builds in 50


def _buffered_water():
    s, _ = water(1000)               # 3.11 nm box: r_cut + skin <= box / 3
    return s, 0.9


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_buffered_trajectory_matches_oracle(oracle_mod, prec):
    s, rc = _buffered_water()
    atom = W.atomic_data(6.0, pi_scale=3000.0)
    pulses = [W.Pulse(6.0, 5.0, 1e12, 0.0)]
    gpu = M.IonisingMD(s, atom, precision=prec, r_cut=rc, max_steps=60, t_start_fs=-2.0, list_skin_nm=SKIN)
    gpu.set_pulse(pulses)
    ora = oracle_mod.OracleMD(s, atom, r_cut=rc, t_start_fs=-2.0, pulses=[pulses], n_steps_max=60)
    L = s.box[0]
    for _ in range(50):
        gpu.step(1)
        ora.step()
    st = gpu.get_state(M.MD_FIELD_X | M.MD_FIELD_V | M.MD_FIELD_Q | M.MD_FIELD_F)
    t = gpu.timing()
    gpu.close()
    assert 1 <= t.list_builds < 50, t.list_builds          # the buffer skipped builds
    assert np.array_equal(st["q"], ora.q)
    d = st["x"] - ora.x
    d -= L * np.round(d / L)
    rms = float(np.sqrt((d ** 2).sum(1).mean()))
    assert rms <= {"mixed": 1e-6, "fp64": 1e-9}[prec], rms
    dv = np.abs(st["v"] - ora.v).max(1)
    assert np.percentile(dv, 98) <= {"mixed": 2.5e-4, "fp64": 2.5e-11}[prec]
    # forces at the final state, from the list built some steps earlier
    F = ora.F
    rel = np.linalg.norm(st["f"] - F) / np.linalg.norm(F)
    assert rel <= {"mixed": 1e-5, "fp64": 1e-12}[prec], rel


def test_buffered_checkpoint_resume_bit_exact():
    s, rc = _buffered_water()
    atom = W.atomic_data(6.0, pi_scale=800.0, ci_scale=20.0)
    p = [W.Pulse(6.0, 4.0, 3e12, 0.0)]
    kw = dict(r_cut=rc, max_steps=80, t_start_fs=-1.5, list_skin_nm=SKIN)
    g = M.IonisingMD(s, atom, **kw)
    g.set_pulse(p)
    g.step(60)
    straight = g.get_state(ALL)
    g.close()
    g = M.IonisingMD(s, atom, **kw)
    g.set_pulse(p)
    g.step(23)                       # mid-way between two list builds
    ck = g.get_state(ALL)
    g.close()
    assert not np.array_equal(ck["x_list"], ck["x"])
    h = M.IonisingMD(s, atom, **kw)
    h.set_pulse(p)
    h.set_state(ALL, **{k: ck[k] for k in ("x", "v", "q", "h", "n_e", "e_gas_mev", "event_counts", "x_list")},
                step=ck["step"])
    h.step(37)
    resumed = h.get_state(ALL)
    h.close()
    _same(straight, resumed)
    assert np.array_equal(straight["x_list"], resumed["x_list"])


def test_buffered_energy_pass_changes_nothing():
    s, rc = _buffered_water()
    atom = W.atomic_data(6.0, pi_scale=800.0)
    p = [W.Pulse(6.0, 4.0, 3e12, 0.0)]
    kw = dict(r_cut=rc, max_steps=50, t_start_fs=-1.5, list_skin_nm=SKIN)
    out = []
    for with_energy in (False, True):
        g = M.IonisingMD(s, atom, **kw)
        g.set_pulse(p)
        g.step(17)
        if with_energy:
            f0 = g.get_state(M.MD_FIELD_F)["f"]
            _, _, n = g.energies()
            assert n > 0
            assert np.array_equal(f0, g.get_state(M.MD_FIELD_F)["f"])
        g.step(13)
        out.append(g.get_state(ALL))
        g.close()
    _same(out[0], out[1])


def test_unbuffered_list_builds_every_step():
    s, rc = water(300)
    g = M.IonisingMD(s, W.atomic_data(6.0), r_cut=rc, max_steps=20)
    g.step(7)
    assert g.timing().list_builds == 7
    g.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_list_blocks_loop_over_super_clusters(oracle_mod, prec):
    """More super-clusters than list blocks (each block loops over several) and
    cells of more than 32 clusters (the write pass re-tests the boxes of its
    later batches): a 60,000-atom protein-crystal box with r_cut + skin = 1.24 nm
    (1,042 super-clusters, 162 cells above 256 atoms), sampled forces."""
    from gpu_common import force_errors
    wl = W.workload("c3_protein_200k", scale=0.3)
    s = wl.sample
    rng = np.random.default_rng(21)
    s.q0[rng.random(s.n_atoms) < 0.2] = 1
    atom = W.atomic_data(wl.photon_kev)
    g = M.IonisingMD(s, atom, precision=prec, r_cut=1.2, cr_enabled=False, kappa_fixed=1.5, max_steps=4,
                     list_skin_nm=0.04)
    f = g.get_state(M.MD_FIELD_F)["f"]
    g.close()
    idx = rng.choice(s.n_atoms, 500, replace=False)
    ref = oracle_mod.forces_of_atoms(s, atom, idx, r_cut=1.2, kappa=1.5)
    rms, mx = force_errors(f[idx], ref)
    assert rms <= {"mixed": 1e-5, "fp64": 1e-12}[prec], (rms, mx)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_cells_beyond_the_sort_shared_memory(oracle_mod, prec):
    """Cells of more atoms than the cell sort keeps in shared memory (2,048):
    a 12,000-atom water droplet (6 nm across) with r_cut = 3.1 nm is one cell of
    12,000 atoms, which the sort ranks from global memory and whose cluster
    boxes it builds without the shared-memory path.  Forces
    against the oracle's all pairs, and a short ionising run with rebuilds."""
    from gpu_common import force_errors
    s = W.water_droplet(4000, seed=31)
    rng = np.random.default_rng(22)
    s.q0[rng.random(s.n_atoms) < 0.2] = 1
    atom = W.atomic_data(8.0)
    rc = 3.1
    assert s.n_atoms > 2 * 2048 and (s.x.max(0) - s.x.min(0)).max() < 2 * (rc + 0.04)
    g = M.IonisingMD(s, atom, precision=prec, r_cut=rc, cr_enabled=False, kappa_fixed=1.0, max_steps=8,
                     list_skin_nm=0.04)
    f = g.get_state(M.MD_FIELD_F)["f"]
    ref = oracle_mod.OracleMD(s, atom, r_cut=rc, cr_enabled=False, kappa_fixed=1.0).F
    rms, mx = force_errors(f, ref)
    assert rms <= {"mixed": 1e-5, "fp64": 1e-12}[prec], (rms, mx)
    g.step(5)
    st = g.get_state(M.MD_FIELD_X | M.MD_FIELD_Q | M.MD_FIELD_F)
    g.close()
    s2 = W.Sample(x=st["x"], v=s.v, species=s.species, fragment=s.fragment, q0=st["q"],
                  replica_offset=s.replica_offset, seed=s.seed, box=s.box, volume=s.volume)
    ref2 = oracle_mod.OracleMD(s2, atom, r_cut=rc, cr_enabled=False, kappa_fixed=1.0).F
    rms2, mx2 = force_errors(st["f"], ref2)
    assert rms2 <= {"mixed": 1e-5, "fp64": 1e-12}[prec], (rms2, mx2)
