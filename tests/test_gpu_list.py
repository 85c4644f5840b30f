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
