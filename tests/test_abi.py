"""The C-ABI library without a GPU: it builds, loads, exports every function
include/md.h declares, and its ctypes mirror has the C struct layout.  The
one host-only entry point (md_pulse_table) is compared with the oracle."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2401_03180_gb300 import build as B
from paper_2401_03180_gb300 import md as M
from paper_2401_03180_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "md.h")


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:md_status|void|const char\*)\s+(md_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(libpath):
    names = _declared()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (md_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in names:
        assert hasattr(lib, n)
    assert M.md_version().startswith("gb300")
    hdr = open(HEADER).read()
    assert int(re.search(r"#define MD_NOALLOC_MAX_ATOMS (\d+)", hdr).group(1)) == M.MD_NOALLOC_MAX_ATOMS
    assert int(re.search(r"#define MD_NOALLOC_MAX_CELLS (\d+)", hdr).group(1)) == M.MD_NOALLOC_MAX_CELLS


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    fields = {
        "md_config": [f[0] for f in M.MDConfig._fields_],
        "md_system": [f[0] for f in M.MDSystem._fields_],
        "md_pulse": [f[0] for f in M.MDPulse._fields_],
        "md_state": [f[0] for f in M.MDState._fields_],
        "md_timing": [f[0] for f in M.MDTiming._fields_],
        "md_forces_input": [f[0] for f in M.MDForcesInput._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-o", str(exe), str(src)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    pys = {"md_config": M.MDConfig, "md_system": M.MDSystem, "md_pulse": M.MDPulse,
           "md_state": M.MDState, "md_timing": M.MDTiming, "md_forces_input": M.MDForcesInput}
    for st, cls in pys.items():
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f in fields[st]:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def test_host_pulse_table_bit_exact_vs_oracle(libpath, oracle_mod):
    cases = [
        ([W.Pulse(8.0, 10.0, 1e12, 0.0)], -10.0, 400),
        ([W.Pulse(6.0, 25.0, 5e12, 0.0)], -25.0, 1000),
        ([W.Pulse(9.0, 10.0, 1e13, 0.0), W.Pulse(9.0, 10.0, 1e13, 50.0)], -10.0, 1400),
        ([W.Pulse(8.0, 15.0, 1e13, 3.0, W.FLAT_TOP)], -20.0, 900),
        ([W.Pulse(8.0, 0.3, 2e12, 0.01)], -1.0, 60),
    ]
    for pulses, t0, n in cases:
        a = M.md_pulse_table(pulses, t0, 0.05, n)
        b = oracle_mod.pulse_table(pulses, t0, 0.05, n)
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_host_pulse_table_rejects_bad_input(libpath):
    with pytest.raises(M.MDError) as e:
        M.md_pulse_table([W.Pulse(8.0, -1.0, 1e12, 0.0)], 0.0, 0.05, 10)
    assert e.value.status == M.MD_ERR_INVALID_ARG
    with pytest.raises(M.MDError):
        M.md_pulse_table([W.Pulse(8.0, 10.0, 1e12, 0.0)], 0.0, 0.0, 10)


def test_binding_fails_loudly_without_gpu(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    wl = W.workload("c1_methane_1500", scale=0.02)
    with pytest.raises(RuntimeError):
        M.IonisingMD(wl.sample, W.atomic_data(8.0))


def _init_status(sample):
    """md_init's status and message for a system whose bonded terms are
    invalid: the host-side checks run before any CUDA call."""
    cfg, keep_c = M.make_config(W.atomic_data(8.0))
    sysd, keep_s = M.make_system(sample)
    h = ctypes.c_void_p()
    st = M.lib().md_init(ctypes.byref(cfg), ctypes.byref(sysd), ctypes.byref(h))
    return st, M.lib().md_last_error(None).decode()


def test_bonded_topology_is_validated_on_the_host(libpath):
    import dataclasses
    base = W.with_topology(W.concat([W.methane_cluster(3, 1), W.methane_cluster(2, 2)]))
    t = base.topology
    cases = []
    b = t.bonds.copy(); b[0, 1] = b[0, 0]
    cases.append((dataclasses.replace(t, bonds=b), "atoms out of range or equal"))
    b = t.bonds.copy(); b[1, 1] = base.n_atoms
    cases.append((dataclasses.replace(t, bonds=b), "atoms out of range or equal"))
    b = t.bonds.copy(); b[2, 2] = 2
    cases.append((dataclasses.replace(t, bonds=b), "type out of range"))
    b = t.bonds.copy(); b[3, 1] = 7                     # another methane: another fragment
    cases.append((dataclasses.replace(t, bonds=b), "different replicas or fragments"))
    a = t.angles.copy(); a[0, 2] = base.replica_offset[1] + 1   # an atom of the second replica
    cases.append((dataclasses.replace(t, angles=a), "different replicas or fragments"))
    a = t.angles.copy(); a[1, 2] = a[1, 0]
    cases.append((dataclasses.replace(t, angles=a), "atoms must be distinct"))
    bp = t.bond_params.copy(); bp[0, 2] = 0.0
    cases.append((dataclasses.replace(t, bond_params=bp), "beta > 0"))
    ap = t.angle_params.copy(); ap[1, 1] = 4.0
    cases.append((dataclasses.replace(t, angle_params=ap), "theta_0 in [0, pi]"))
    for topo, msg in cases:
        st, err = _init_status(dataclasses.replace(base, topology=topo))
        assert st == M.MD_ERR_INVALID_ARG and msg in err, (st, err)


def test_system_is_validated_on_the_host(libpath):
    """Degenerate and malformed samples are refused with MD_ERR_INVALID_ARG
    before any device work: no atoms, a replica without atoms, offsets that do
    not span the atoms, a species or charge outside the tables, non-finite
    coordinates and a periodic box shorter than three interaction ranges."""
    import dataclasses
    base = W.concat([W.methane_cluster(3, 1), W.methane_cluster(2, 2)])
    n = base.n_atoms
    cases = []
    cases.append((dataclasses.replace(base, x=base.x[:0], v=base.v[:0], species=base.species[:0],
                                      fragment=base.fragment[:0], q0=base.q0[:0],
                                      replica_offset=np.array([0, 0], np.int32), seed=base.seed[:1],
                                      box=base.box[:1], volume=base.volume[:1]), "n_atoms must be >= 1"))
    off = base.replica_offset.copy(); off[1] = 0
    cases.append((dataclasses.replace(base, replica_offset=off), "at least one atom"))
    off = base.replica_offset.copy(); off[-1] = n - 1
    cases.append((dataclasses.replace(base, replica_offset=off), "from 0 to n_atoms"))
    sp = base.species.copy(); sp[4] = 200
    cases.append((dataclasses.replace(base, species=sp), "species index out of range"))
    q = base.q0.copy(); q[1] = W.Z[base.species[1]] + 1
    cases.append((dataclasses.replace(base, q0=q), "q0 above Z"))
    x = base.x.copy(); x[2, 1] = np.nan
    cases.append((dataclasses.replace(base, x=x), "non-finite"))
    v = base.v.copy(); v[3, 0] = np.inf
    cases.append((dataclasses.replace(base, v=v), "non-finite"))
    vol = base.volume.copy(); vol[1] = 0.0
    cases.append((dataclasses.replace(base, volume=vol), "volume must be > 0"))
    box = base.box.copy(); box[0] = [3.0, 3.0, 3.0]           # r_cut 1.2 + skin: 3.6 nm needed
    cases.append((dataclasses.replace(base, box=box), "periodic box edges"))
    for s, msg in cases:
        st, err = _init_status(s)
        assert st == M.MD_ERR_INVALID_ARG and msg in err, (msg, st, err)
