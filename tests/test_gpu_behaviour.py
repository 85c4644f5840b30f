"""GPU path properties that need no oracle value (-m gpu): determinism
across runs and launch shapes, replica independence in a batch,
checkpoint/resume, edge cases, and error reporting."""
import numpy as np
import pytest

from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

from gpu_common import methane, water

pytestmark = pytest.mark.gpu
ALL = M.MD_FIELD_ALL


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    from paper_2401_03180_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _run(sample, atom, steps, pulses=None, **kw):
    g = M.IonisingMD(sample, atom, **kw)
    if pulses is not None:
        g.set_pulse(pulses)
    g.step(steps)
    st = g.get_state(ALL)
    g.close()
    return st


def _same(a, b):
    for k in ("x", "v", "f", "q", "h", "n_e", "e_gas_mev", "event_counts"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_runs_are_bit_identical_and_tile_invariant(prec):
    s, rc = water(800)
    atom = W.atomic_data(6.0, pi_scale=500.0)
    p = [W.Pulse(6.0, 5.0, 2e12, 0.0)]
    kw = dict(precision=prec, r_cut=rc, max_steps=40, t_start_fs=-1.0)
    a = _run(s, atom, 30, p, **kw)
    b = _run(s, atom, 30, p, **kw)
    c = _run(s, atom, 30, p, autotune=True, **kw)
    _same(a, b)
    _same(a, c)


SHAPES = [dict(pair_warps=4, pair_blocks_per_sm=2, sort_threads=1024, list_blocks_per_sm=1),
          dict(pair_warps=12, pair_blocks_per_sm=1, sort_threads=256, list_blocks_per_sm=16),
          dict(pair_warps=8, pair_blocks_per_sm=3, sort_threads=256, list_blocks_per_sm=2)]


@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_launch_shapes_give_identical_runs(shape):
    """Every launch shape the autotuner may pick (force-kernel warps and blocks
    per SM, cell-sort block size, list-build blocks per SM, which also sets how
    many warps share a super-cluster's cells) gives the same trajectory, bit
    for bit, with the Verlet-buffered list rebuilt during the run: on a
    periodic water box and on a vacuum batch of methane clusters."""
    s, rc = water(800)
    atom = W.atomic_data(6.0, pi_scale=500.0)
    p = [W.Pulse(6.0, 5.0, 2e12, 0.0)]
    kw = dict(r_cut=rc - 0.04, max_steps=40, t_start_fs=-1.0, list_skin_nm=0.03)   # box >= 3 (r_cut + skin)
    _same(_run(s, atom, 30, p, **kw), _run(s, atom, 30, p, launch_shape=SHAPES[shape], **kw))
    reps = [methane(n, seed=k + 31) for k, n in enumerate((40, 75, 23, 31, 52, 18))]
    b = W.concat(reps)
    atom8 = W.atomic_data(8.0, pi_scale=1500.0, ci_scale=10.0)
    kw8 = dict(max_steps=40, t_start_fs=-5.0, list_skin_nm=0.03)
    p8 = [W.Pulse(8.0, 10.0, 1e12, 0.0)]
    _same(_run(b, atom8, 30, p8, **kw8), _run(b, atom8, 30, p8, launch_shape=SHAPES[shape], **kw8))


def test_launch_shape_outside_occupancy_is_rejected():
    s, rc = water(200)
    with pytest.raises(M.MDError) as e:
        M.IonisingMD(s, W.atomic_data(6.0), r_cut=rc, max_steps=4,
                     launch_shape=dict(pair_warps=12, pair_blocks_per_sm=40))
    assert e.value.status == M.MD_ERR_INVALID_ARG


def test_batched_replicas_equal_solo_runs():
    # six replicas: more than the step kernel reduces itself, so the batch takes
    # the warp-per-replica reduction and each solo run the in-kernel one
    reps = [methane(n, seed=k + 1) for k, n in enumerate((40, 75, 23, 31, 52, 18))]
    for k, r in enumerate(reps):
        r.seed[:] = 500 + k
    atom = W.atomic_data(8.0, pi_scale=1500.0, ci_scale=10.0)
    pulses = [[W.Pulse(8.0, 10.0, f, 0.0)] for f in (1e12, 3e11, 2e12, 5e11, 1.5e12, 8e11)]
    batch = W.concat(reps)
    g = M.IonisingMD(batch, atom, max_steps=80, t_start_fs=-5.0)
    for k, p in enumerate(pulses):
        g.set_pulse(p, replica=k)
    g.step(60)
    sb = g.get_state(ALL)
    g.close()
    off = batch.replica_offset
    for k, r in enumerate(reps):
        so = _run(r, atom, 60, pulses[k], max_steps=80, t_start_fs=-5.0)
        sl = slice(off[k], off[k + 1])
        for key in ("x", "v", "f", "q", "h"):
            assert np.array_equal(sb[key][sl], so[key]), (k, key)
        assert sb["n_e"][k] == so["n_e"][0] and sb["e_gas_mev"][k] == so["e_gas_mev"][0]


@pytest.mark.parametrize("mode", ["hybrid_langevin", "table"])
def test_batched_replicas_equal_solo_runs_in_the_widened_modes(mode):
    """The per-replica tables of the hybrid electrostatics, the Langevin
    coupling and the charge-state fractions: each replica of a batch of six
    equals its solo run, bit for bit."""
    reps = [methane(n, seed=k + 11) for k, n in enumerate((40, 75, 23, 31, 52, 18))]
    for k, r in enumerate(reps):
        r.seed[:] = 900 + k
    atom = W.atomic_data(8.0, pi_scale=1500.0, ci_scale=10.0)
    pulses = [[W.Pulse(8.0, 10.0, f, 0.0)] for f in (1e12, 3e11, 2e12, 5e11, 1.5e12, 8e11)]
    if mode == "table":
        kw = dict(max_steps=80, t_start_fs=-5.0, charge_mode="table")
        tabs = [W.charge_fraction_table(p, -5.0, 0.05, 81, mean_final=1.0 + 0.3 * k) for k, p in enumerate(pulses)]
    else:
        kw = dict(max_steps=80, t_start_fs=-5.0, screening="hybrid", langevin_g=np.full(len(atom.z), 0.5))
    batch = W.concat(reps)
    g = M.IonisingMD(batch, atom, **kw)
    for k, p in enumerate(pulses):
        g.set_pulse(p, replica=k)
        if mode == "table":
            g.set_charge_table(tabs[k], replica=k)
    g.step(60)
    sb = g.get_state(ALL)
    g.close()
    off = batch.replica_offset
    for k, r in enumerate(reps):
        h = M.IonisingMD(r, atom, **kw)
        h.set_pulse(pulses[k])
        if mode == "table":
            h.set_charge_table(tabs[k])
        h.step(60)
        so = h.get_state(ALL)
        h.close()
        sl = slice(off[k], off[k + 1])
        for key in ("x", "v", "f", "q", "h"):
            assert np.array_equal(sb[key][sl], so[key]), (k, key)
        assert sb["n_e"][k] == so["n_e"][0] and sb["kappa"][k] == so["kappa"][0]
    assert sb["q"].any()


def test_checkpoint_resume_bit_exact():
    s, rc = water(500)
    atom = W.atomic_data(6.0, pi_scale=800.0, ci_scale=20.0)
    p = [W.Pulse(6.0, 4.0, 3e12, 0.0)]
    kw = dict(r_cut=rc, max_steps=60, t_start_fs=-1.5)
    straight = _run(s, atom, 40, p, **kw)
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
    h.close()
    _same(straight, resumed)


def test_edge_cases_single_atom_and_tiny_cluster():
    one = W.Sample(x=np.array([[0.1, 0.2, 0.3]]), v=np.array([[1.0, 0.0, 0.0]]),
                   species=np.array([W.C], np.uint8), fragment=np.array([0], np.int32),
                   q0=np.array([2], np.uint8), replica_offset=np.array([0, 1], np.int32),
                   seed=np.array([1], np.uint64), box=np.zeros((1, 3)), volume=np.array([1.0]))
    st = _run(one, W.atomic_data(8.0), 10, cr_enabled=False, max_steps=10)
    assert np.all(st["f"] == 0)
    np.testing.assert_allclose(st["x"][0], [0.1 + 10 * 5e-5, 0.2, 0.3], rtol=0, atol=1e-15)
    # a cluster smaller than one cell; fully stripped atoms have no LJ
    s = methane(3, charge_frac=0.0)
    s.q0[:] = W.Z[s.species]
    st = _run(s, W.atomic_data(8.0), 5, cr_enabled=False, max_steps=5, kappa_fixed=0.0)
    assert np.isfinite(st["f"]).all() and np.abs(st["f"]).max() > 0


def test_periodic_wrap_keeps_atoms_in_box():
    s, rc = water(300)
    s.v[:] = 0.0
    s.v[:, 0] = 200.0          # 0.01 nm per step along x
    st = _run(s, W.atomic_data(6.0), 60, cr_enabled=False, r_cut=rc, max_steps=60, kappa_fixed=3.0)
    L = s.box[0]
    assert np.all(st["x"] >= 0) and np.all(st["x"] < L)


def test_expanding_cluster_regrids():
    s = methane(50, charge_frac=0.0)
    s.q0[:] = np.minimum(3, W.Z[s.species])          # strongly charged -> explodes
    st = _run(s, W.atomic_data(8.0), 200, cr_enabled=False, max_steps=200, kappa_fixed=0.0)
    r0 = np.linalg.norm(s.x - s.x.mean(0), axis=1).max()
    r1 = np.linalg.norm(st["x"] - st["x"].mean(0), axis=1).max()
    assert r1 > r0 and np.isfinite(st["x"]).all()


def test_errors_are_reported_not_faulted():
    s = methane(20)
    atom = W.atomic_data(8.0)
    with pytest.raises(M.MDError) as e:
        M.IonisingMD(s, atom, r_cut=-1.0)
    assert e.value.status == M.MD_ERR_INVALID_ARG
    w, rc = water(100)
    with pytest.raises(M.MDError) as e:
        M.IonisingMD(w, atom, r_cut=1.2)               # box < 3 r_cut
    assert e.value.status == M.MD_ERR_INVALID_ARG
    g = M.IonisingMD(s, atom, max_steps=5)
    with pytest.raises(M.MDError) as e:
        g.step(6)
    assert e.value.status == M.MD_ERR_TABLE_END
    g.step(5)
    with pytest.raises(M.MDError) as e:
        g.set_pulse([W.Pulse(9.0, 10.0, 1e12, 0.0)])   # photon energy of another table
    assert e.value.status == M.MD_ERR_INVALID_ARG
    g.close()
    # two highly charged ions almost on top of each other: the fixed-point
    # range is exceeded and reported; the handle then refuses to step
    two = W.Sample(x=np.array([[0.0, 0.0, 0.0], [1e-4, 0.0, 0.0]]), v=np.zeros((2, 3)),
                   species=np.array([W.S, W.S], np.uint8), fragment=np.array([0, 1], np.int32),
                   q0=np.array([16, 16], np.uint8), replica_offset=np.array([0, 2], np.int32),
                   seed=np.array([1], np.uint64), box=np.zeros((1, 3)), volume=np.array([1.0]))
    with pytest.raises(M.MDError) as e:
        M.IonisingMD(two, atom, cr_enabled=False, kappa_fixed=0.0, max_steps=3)
    assert e.value.status == M.MD_ERR_FIXED_OVERFLOW


def test_fluence_per_step_equals_pulse_tables():
    """md_set_fluence_at (one step, every replica) reproduces per-replica pulse
    tables set up front, bit for bit."""
    wl = W.workload("c4_methane_batch", scale=0.05)
    s = wl.sample
    atom = W.atomic_data(wl.photon_kev, pi_scale=3000.0)
    steps = 30
    kw = dict(r_cut=1.2, max_steps=steps + 1, t_start_fs=wl.t_start_fs)
    a = M.IonisingMD(s, atom, **kw)
    for r in range(s.n_replicas):
        a.set_pulse(wl.pulses[r], replica=r)
    a.step(steps)
    ref = a.get_state(ALL)
    a.close()
    tab = np.stack([M.md_pulse_table(wl.pulses[r], wl.t_start_fs, 5e-5 * 1000.0, steps + 1)
                    for r in range(s.n_replicas)])
    b = M.IonisingMD(s, atom, **kw)
    for k in range(steps):
        M.md_set_fluence_at(b.h, k, np.ascontiguousarray(tab[:, k]))
        b.step(1)
    got = b.get_state(ALL)
    b.close()
    assert s.n_replicas > 1 and ref["event_counts"].sum() > 0
    _same(ref, got)
    with pytest.raises(M.MDError):
        c = M.IonisingMD(s, atom, **kw)
        try:
            M.md_set_fluence_at(c.h, steps + 1, np.ascontiguousarray(tab[:, 0]))
        finally:
            c.close()
