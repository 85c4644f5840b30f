"""Thin Python binding of the C ABI in include/md.h (ctypes).

Argument marshalling only: every step of the method runs in libmdgb.so's
CUDA kernels.  The module-level functions carry the C names (md_init,
md_set_pulse, md_step, md_get_state, ...); ``IonisingMD`` wraps them for
convenience.  PyTorch provides device memory (through the library's
allocation hooks) and the current CUDA stream.  There is no CPU fallback:
if libmdgb.so is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

MD_OK, MD_ERR_INVALID_ARG, MD_ERR_BAD_STATE, MD_ERR_OOM, MD_ERR_CUDA = 0, 1, 2, 3, 4
MD_ERR_FIXED_OVERFLOW, MD_ERR_TIMEOUT, MD_ERR_NONFINITE, MD_ERR_CELL_OVERFLOW, MD_ERR_TABLE_END = 5, 6, 7, 8, 9
MD_PREC_MIXED, MD_PREC_FP64 = 0, 1
MD_PLASMA_BOOKKEEPING, MD_PLASMA_PRESCRIBED = 0, 1
MD_SCREEN_DEBYE, MD_SCREEN_HYBRID = 0, 1
MD_CHARGE_RATES, MD_CHARGE_TABLE = 0, 1
MD_FIELD_X, MD_FIELD_V, MD_FIELD_F, MD_FIELD_Q, MD_FIELD_H = 1, 2, 4, 8, 16
MD_FIELD_PLASMA, MD_FIELD_COUNTS, MD_FIELD_STEP, MD_FIELD_XLIST, MD_FIELD_ALL = 32, 64, 128, 256, 511
MD_MAX_SPECIES = 8
MD_NOALLOC_MAX_ATOMS = 16384
MD_NOALLOC_MAX_CELLS = 4096
COULOMB_F = 138.935458

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_S = MD_MAX_SPECIES


class MDConfig(C.Structure):
    _fields_ = [("dt_ps", C.c_double), ("r_cut", C.c_double), ("precision", C.c_int),
                ("cr_enabled", C.c_int), ("plasma_mode", C.c_int), ("max_steps", C.c_int),
                ("kappa_fixed", C.c_double), ("t_start_fs", C.c_double), ("te_floor_ev", C.c_double),
                ("coulomb_f", C.c_double), ("photon_kev", C.c_double), ("n_species", C.c_int),
                ("z", C.c_int * _S), ("mass", C.c_double * _S), ("lj_sigma0", C.c_double * _S),
                ("lj_eps0", C.c_double * _S), ("tau_auger_ps", C.c_double * _S),
                ("sigma_pi", C.c_void_p), ("k_ci", C.c_void_p), ("k_rec", C.c_void_p),
                ("ip_mev", C.c_void_p), ("e_pi_mev", C.c_void_p), ("e_auger_mev", C.c_void_p),
                ("n_te", C.c_int), ("dte_ev", C.c_double), ("dev_alloc", ALLOC_FN),
                ("dev_free", FREE_FN), ("alloc_ctx", C.c_void_p), ("autotune", C.c_int),
                ("profile", C.c_int), ("list_reserve", C.c_int), ("list_skin_nm", C.c_double),
                ("screening", C.c_int), ("langevin_g", C.c_double * MD_MAX_SPECIES),
                ("charge_mode", C.c_int), ("probe_record", C.c_int), ("pair_warps", C.c_int),
                ("pair_blocks_per_sm", C.c_int), ("sort_threads", C.c_int), ("list_blocks_per_sm", C.c_int),
                ("list_skin_adaptive", C.c_int)]


class MDSystem(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("x", C.c_void_p), ("v", C.c_void_p), ("species", C.c_void_p),
                ("fragment", C.c_void_p), ("q0", C.c_void_p), ("n_replicas", C.c_int),
                ("replica_offset", C.c_void_p), ("seed", C.c_void_p), ("box", C.c_void_p),
                ("volume", C.c_void_p), ("n_bonds", C.c_int), ("bonds", C.c_void_p), ("n_bond_types", C.c_int),
                ("bond_params", C.c_void_p), ("n_angles", C.c_int), ("angles", C.c_void_p),
                ("n_angle_types", C.c_int), ("angle_params", C.c_void_p)]


class MDPulse(C.Structure):
    _fields_ = [("photon_kev", C.c_double), ("fwhm_fs", C.c_double), ("fluence_ph_um2", C.c_double),
                ("t_center_fs", C.c_double), ("shape", C.c_int)]


class MDState(C.Structure):
    _fields_ = [("x", C.c_void_p), ("v", C.c_void_p), ("f", C.c_void_p), ("q", C.c_void_p),
                ("h", C.c_void_p), ("n_e", C.c_void_p), ("e_gas_mev", C.c_void_p), ("te_ev", C.c_void_p),
                ("kappa", C.c_void_p), ("event_counts", C.c_void_p), ("step", C.c_int64),
                ("x_list", C.c_void_p)]


class MDTiming(C.Structure):
    _fields_ = [("pair_ms", C.c_double), ("pair_launches", C.c_int64), ("steps", C.c_int64),
                ("pair_count_last", C.c_int64), ("tile_warps", C.c_int), ("tile_blocks_per_sm", C.c_int),
                ("list_capacity", C.c_int64), ("list_entries", C.c_int64), ("list_grows", C.c_int64),
                ("list_builds", C.c_int64), ("sort_threads", C.c_int), ("list_blocks_per_sm", C.c_int),
                ("build_kernels", C.c_int), ("list_unbuffered_builds", C.c_int64)]


class MDForcesInput(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("d_x", C.c_void_p), ("d_species", C.c_void_p), ("d_q", C.c_void_p),
                ("d_fragment", C.c_void_p), ("box", C.c_double * 3), ("kappa", C.c_double),
                ("r_cut", C.c_double), ("coulomb_f", C.c_double), ("precision", C.c_int),
                ("n_species", C.c_int), ("z", C.c_int * _S), ("lj_sigma0", C.c_double * _S),
                ("lj_eps0", C.c_double * _S)]


class MDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"md status {status}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libmdgb.so (built in-tree); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                                   "(no CPU fallback exists)")
            L = C.CDLL(path)
            P = C.c_void_p
            L.md_init.argtypes = [C.POINTER(MDConfig), C.POINTER(MDSystem), C.POINTER(C.c_void_p)]
            L.md_set_stream.argtypes = [P, P]
            L.md_set_pulse.argtypes = [P, C.c_int, C.POINTER(MDPulse), C.c_int]
            L.md_set_pulse_table.argtypes = [P, C.c_int, P, C.c_int]
            L.md_set_pulse_table_at.argtypes = [P, C.c_int, C.c_int, P, C.c_int]
            L.md_set_plasma_table.argtypes = [P, C.c_int, P, P, C.c_int]
            L.md_set_charge_table.argtypes = [P, C.c_int, P, C.c_int]
            L.md_rdf.argtypes = [P, C.c_double, C.c_int, P]
            L.md_get_probe_series.argtypes = [P, C.c_int, C.c_int, C.c_int, P, P]
            L.md_fragments.argtypes = [P, C.c_double, C.c_int, C.c_int, P, P]
            L.md_probe_displacement.argtypes = [P, C.c_int, C.c_int, C.c_int, C.POINTER(MDPulse), C.c_int, P]
            L.md_structure_factor.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double,
                                              C.c_double, P, C.c_int, P]
            L.md_set_fluence_at.argtypes = [P, C.c_int, P]
            L.md_step.argtypes = [P, C.c_int]
            L.md_step_async.argtypes = [P, C.c_int]
            L.md_sync.argtypes = [P]
            L.md_get_state.argtypes = [P, C.POINTER(MDState), C.c_uint]
            L.md_set_state.argtypes = [P, C.POINTER(MDState), C.c_uint]
            L.md_get_energies.argtypes = [P, P, P, P]
            L.md_get_timing.argtypes = [P, C.POINTER(MDTiming)]
            L.md_reset_timing.argtypes = [P]
            L.md_last_error.argtypes = [P]
            L.md_last_error.restype = C.c_char_p
            L.md_finalize.argtypes = [P]
            L.md_finalize.restype = None
            L.md_pulse_table.argtypes = [C.POINTER(MDPulse), C.c_int, C.c_double, C.c_double, C.c_int, P]
            L.md_philox.argtypes = [C.c_uint64, P, C.c_int64, P, P]
            L.md_fma_peak.argtypes = [C.c_int, C.c_int64, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), P]
            L.md_forces_noalloc.argtypes = [C.POINTER(MDForcesInput), P, P]
            L.md_version.restype = C.c_char_p
            _lib = L
    return _lib


def _check(status, handle=None):
    if status != MD_OK:
        msg = lib().md_last_error(handle).decode(errors="replace")
        raise MDError(status, msg)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _pulses(pulses):
    arr = (MDPulse * max(len(pulses), 1))()
    for k, p in enumerate(pulses):
        arr[k] = MDPulse(p.photon_kev, p.fwhm_fs, p.fluence_ph_um2, p.t_center_fs, int(p.shape))
    return arr


# ---------------------------------------------------------------------------
# C-named functions (marshalling only)
# ---------------------------------------------------------------------------
def md_init(config: MDConfig, system: MDSystem) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().md_init(C.byref(config), C.byref(system), C.byref(h)))
    return h


def md_set_stream(h, stream_ptr: int):
    _check(lib().md_set_stream(h, C.c_void_p(stream_ptr)), h)


def md_set_pulse(h, replica: int, pulses):
    arr = _pulses(pulses)
    _check(lib().md_set_pulse(h, int(replica), arr, len(pulses)), h)


def md_set_pulse_table(h, replica: int, dF):
    dF = _c(dF, np.float64)
    _check(lib().md_set_pulse_table(h, int(replica), _p(dF), len(dF)), h)


def md_set_pulse_table_at(h, replica: int, first_step: int, dF):
    dF = _c(dF, np.float64)
    _check(lib().md_set_pulse_table_at(h, int(replica), int(first_step), _p(dF), len(dF)), h)


def md_set_fluence_at(h, step: int, dF):
    """dF[r]: fluence of `step` for each replica r (float64 array, pinned for overlap)."""
    _check(lib().md_set_fluence_at(h, int(step), _p(dF)), h)


def md_rdf(h, n_species: int, r_max: float, n_bins: int):
    out = np.zeros((n_species, n_species, n_bins), dtype=np.int64)
    _check(lib().md_rdf(h, float(r_max), int(n_bins), _p(out)), h)
    return out


def md_fragments(h, n_atoms: int, n_replicas: int, r_frag: float, mass_max: int, charge_max: int):
    label = np.zeros(n_atoms, dtype=np.int32)
    counts = np.zeros((n_replicas, mass_max + 1, charge_max + 1), dtype=np.int64)
    _check(lib().md_fragments(h, float(r_frag), int(mass_max), int(charge_max), _p(label), _p(counts)), h)
    return label, counts


def md_get_probe_series(h, n_species: int, replica: int, first: int, n: int):
    q = np.zeros((n, n_species), dtype=np.int64)
    d2 = np.zeros((n, n_species), dtype=np.float64)
    _check(lib().md_get_probe_series(h, int(replica), int(first), int(n), _p(q), _p(d2)), h)
    return q, d2


def md_probe_displacement(h, n_species: int, replica: int, first: int, n: int, probe):
    out = np.zeros(n_species)
    arr = _pulses(probe)
    _check(lib().md_probe_displacement(h, int(replica), int(first), int(n), arr, len(probe), _p(out)), h)
    return out


def md_structure_factor(counts_ab, r_max, n_a, n_b, same, volume, rho0, q):
    c = np.ascontiguousarray(counts_ab, dtype=np.int64)
    qq = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(len(qq))
    _check(lib().md_structure_factor(_p(c), len(c), float(r_max), float(n_a), float(n_b), int(bool(same)),
                                     float(volume), float(rho0), _p(qq), len(qq), _p(out)), None)
    return out


def md_set_charge_table(h, replica: int, frac):
    f = np.ascontiguousarray(frac, dtype=np.float64)
    _check(lib().md_set_charge_table(h, int(replica), _p(f), int(f.shape[0])), h)


def md_set_plasma_table(h, replica: int, ne, te_ev):
    ne = _c(ne, np.float64); te = _c(te_ev, np.float64)
    _check(lib().md_set_plasma_table(h, int(replica), _p(ne), _p(te), len(ne)), h)


def md_step(h, n_steps: int):
    _check(lib().md_step(h, int(n_steps)), h)


def md_step_async(h, n_steps: int):
    _check(lib().md_step_async(h, int(n_steps)), h)


def md_sync(h):
    _check(lib().md_sync(h), h)


def md_get_state(h, state: MDState, fields: int):
    _check(lib().md_get_state(h, C.byref(state), int(fields)), h)


def md_set_state(h, state: MDState, fields: int):
    _check(lib().md_set_state(h, C.byref(state), int(fields)), h)


def md_get_energies(h, e_kin, e_pot):
    n = C.c_int64()
    _check(lib().md_get_energies(h, _p(e_kin), _p(e_pot), C.byref(n)), h)
    return int(n.value)


def md_get_timing(h) -> MDTiming:
    t = MDTiming()
    _check(lib().md_get_timing(h, C.byref(t)), h)
    return t


def md_reset_timing(h):
    _check(lib().md_reset_timing(h), h)


def md_last_error(h=None) -> str:
    return lib().md_last_error(h).decode(errors="replace")


def md_finalize(h):
    lib().md_finalize(h)


def md_pulse_table(pulses, t_start_fs: float, dt_fs: float, n_steps: int) -> np.ndarray:
    out = np.empty(n_steps)
    arr = _pulses(pulses)
    _check(lib().md_pulse_table(arr, len(pulses), float(t_start_fs), float(dt_fs), int(n_steps), _p(out)))
    return out


def md_fma_peak(precision: int, iters: int, blocks_per_sm: int = 4, stream_ptr: int = 0):
    """Measured FMA-pipe throughput of the current device: (flop/s, kernel seconds)."""
    f, s = C.c_double(0.0), C.c_double(0.0)
    _check(lib().md_fma_peak(int(precision), C.c_int64(iters), int(blocks_per_sm), C.byref(f), C.byref(s),
                             C.c_void_p(stream_ptr)))
    return f.value, s.value


def md_philox(seed: int, d_ctr4_ptr: int, n: int, d_out_ptr: int, stream_ptr: int = 0):
    _check(lib().md_philox(C.c_uint64(seed), C.c_void_p(d_ctr4_ptr), C.c_int64(n), C.c_void_p(d_out_ptr),
                           C.c_void_p(stream_ptr)))


def md_forces_noalloc(inp: MDForcesInput, d_f_ptr: int, stream_ptr: int = 0):
    """Forces of one configuration from device buffers, with no device
    allocation inside the library (fixed scratch compiled into it)."""
    _check(lib().md_forces_noalloc(C.byref(inp), C.c_void_p(d_f_ptr), C.c_void_p(stream_ptr)))


def md_version() -> str:
    return lib().md_version().decode()


# ---------------------------------------------------------------------------
# Torch-backed device allocator for the library's hooks
# ---------------------------------------------------------------------------
class TorchAllocator:
    def __init__(self):
        import torch
        self._torch = torch
        self._live = {}
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.free_fn = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device="cuda")
        ptr = t.data_ptr()
        self._live[ptr] = t
        return ptr

    def _free(self, ptr, ctx):
        self._live.pop(ptr, None)


def make_config(atomic, *, dt_ps=5e-5, r_cut=1.2, precision="mixed", cr_enabled=True,
                plasma_mode=MD_PLASMA_BOOKKEEPING, max_steps=1000, kappa_fixed=-1.0, t_start_fs=0.0,
                te_floor_ev=1.0, coulomb_f=COULOMB_F, autotune=False, profile=False, list_reserve=0,
                list_skin_nm=0.0, screening="debye", langevin_g=None, charge_mode="rates",
                sigma0=None, eps0=None, mass=None, list_skin_adaptive=False):
    """An md_config for the atomic data and options (argument marshalling);
    returns it with the arrays it points into, which must outlive md_init."""
    from . import workloads as W
    ns = len(atomic.z)
    cfg = MDConfig()
    cfg.dt_ps, cfg.r_cut = float(dt_ps), float(r_cut)
    cfg.precision = MD_PREC_FP64 if precision == "fp64" else MD_PREC_MIXED
    cfg.cr_enabled, cfg.plasma_mode, cfg.max_steps = int(bool(cr_enabled)), int(plasma_mode), int(max_steps)
    cfg.kappa_fixed, cfg.t_start_fs, cfg.te_floor_ev = float(kappa_fixed), float(t_start_fs), float(te_floor_ev)
    cfg.coulomb_f, cfg.photon_kev, cfg.n_species = float(coulomb_f), float(atomic.photon_kev), ns
    mass = W.MASS if mass is None else mass
    sigma0 = W.LJ_SIGMA0 if sigma0 is None else sigma0
    eps0 = W.LJ_EPS0 if eps0 is None else eps0
    for k in range(ns):
        cfg.z[k] = int(atomic.z[k]); cfg.mass[k] = float(mass[k])
        cfg.lj_sigma0[k] = float(sigma0[k]); cfg.lj_eps0[k] = float(eps0[k])
        cfg.tau_auger_ps[k] = float(atomic.tau_auger_ps[k])
    keep = [_c(atomic.sigma_pi, np.float64), _c(atomic.k_ci, np.float64), _c(atomic.k_rec, np.float64),
            _c(atomic.ip_mev, np.int64), _c(atomic.e_pi_mev, np.int64), _c(atomic.e_auger_mev, np.int64)]
    (cfg.sigma_pi, cfg.k_ci, cfg.k_rec, cfg.ip_mev, cfg.e_pi_mev,
     cfg.e_auger_mev) = [a.ctypes.data for a in keep]
    cfg.n_te, cfg.dte_ev = int(atomic.n_te), float(atomic.dte_ev)
    cfg.autotune, cfg.profile = int(bool(autotune)), int(bool(profile))
    cfg.list_reserve = int(list_reserve)
    cfg.list_skin_nm = float(list_skin_nm)
    cfg.list_skin_adaptive = int(list_skin_adaptive)
    if screening not in ("debye", "hybrid"):
        raise ValueError("screening must be 'debye' or 'hybrid'")
    cfg.screening = MD_SCREEN_HYBRID if screening == "hybrid" else MD_SCREEN_DEBYE
    if charge_mode not in ("rates", "table"):
        raise ValueError("charge_mode must be 'rates' or 'table'")
    cfg.charge_mode = MD_CHARGE_TABLE if charge_mode == "table" else MD_CHARGE_RATES
    if langevin_g is not None:
        g = np.broadcast_to(np.asarray(langevin_g, np.float64), (ns,))
        for k in range(len(g)):
            cfg.langevin_g[k] = float(g[k])
    return cfg, keep


def make_system(sample):
    """An md_system for a Sample, with its bonded terms when it has a
    topology; returns it with the arrays it points into."""
    s = sample
    arrs = [_c(s.x, np.float64), _c(s.v, np.float64), _c(s.species, np.uint8), _c(s.fragment, np.int32),
            _c(s.q0, np.uint8), _c(s.replica_offset, np.int32), _c(s.seed, np.uint64),
            _c(s.box, np.float64), _c(s.volume, np.float64)]
    sysd = MDSystem(s.n_atoms, *[a.ctypes.data for a in arrs[:5]], s.n_replicas, *[a.ctypes.data for a in arrs[5:]])
    topo = getattr(s, "topology", None)
    if topo is not None:
        t = [_c(topo.bonds, np.int32), _c(topo.bond_params, np.float64), _c(topo.angles, np.int32),
             _c(topo.angle_params, np.float64)]
        arrs += t
        sysd.n_bonds, sysd.bonds = len(t[0]), t[0].ctypes.data
        sysd.n_bond_types, sysd.bond_params = len(t[1]), t[1].ctypes.data
        sysd.n_angles, sysd.angles = len(t[2]), t[2].ctypes.data
        sysd.n_angle_types, sysd.angle_params = len(t[3]), t[3].ctypes.data
    return sysd, arrs


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------
class IonisingMD:
    """One handle of the GB300 hot path for a Sample and its atomic data."""

    def __init__(self, sample, atomic, *, dt_ps=5e-5, r_cut=1.2, precision="mixed", cr_enabled=True,
                 plasma_mode=MD_PLASMA_BOOKKEEPING, max_steps=1000, kappa_fixed=-1.0, t_start_fs=0.0,
                 te_floor_ev=1.0, coulomb_f=COULOMB_F, autotune=False, profile=False, list_reserve=0,
                 list_skin_nm=0.0, screening="debye", langevin_g=None, charge_mode="rates",
                 probe_record=False, torch_allocator=True, sigma0=None, eps0=None, mass=None,
                 launch_shape=None, list_skin_adaptive=False):
        """launch_shape: optional dict pinning md_config's launch-shape fields
        (pair_warps, pair_blocks_per_sm, sort_threads, list_blocks_per_sm)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("IonisingMD needs a CUDA GPU (no CPU fallback)")
        self.n = sample.n_atoms
        self.R = sample.n_replicas
        self.ns = len(atomic.z)
        cfg, keep_c = make_config(atomic, dt_ps=dt_ps, r_cut=r_cut, precision=precision, cr_enabled=cr_enabled,
                                  plasma_mode=plasma_mode, max_steps=max_steps, kappa_fixed=kappa_fixed,
                                  t_start_fs=t_start_fs, te_floor_ev=te_floor_ev, coulomb_f=coulomb_f,
                                  autotune=autotune, profile=profile, list_reserve=list_reserve,
                                  list_skin_nm=list_skin_nm, screening=screening, langevin_g=langevin_g,
                                  charge_mode=charge_mode, sigma0=sigma0, eps0=eps0, mass=mass,
                                  list_skin_adaptive=list_skin_adaptive)
        cfg.probe_record = int(bool(probe_record))
        for k, v in (launch_shape or {}).items():
            if k not in ("pair_warps", "pair_blocks_per_sm", "sort_threads", "list_blocks_per_sm"):
                raise ValueError(f"unknown launch-shape field {k}")
            setattr(cfg, k, int(v))
        self._keep = keep_c
        self._alloc = TorchAllocator() if torch_allocator else None
        if self._alloc is not None:
            cfg.dev_alloc, cfg.dev_free = self._alloc.alloc_fn, self._alloc.free_fn
        sysd, arrs = make_system(sample)
        self.config = cfg
        self.stream = torch.cuda.current_stream().cuda_stream
        self.h = md_init(cfg, sysd)
        md_set_stream(self.h, self.stream)

    # pass-throughs ---------------------------------------------------------
    def set_pulse(self, pulses, replica=-1):
        md_set_pulse(self.h, replica, pulses)

    def set_pulse_table(self, dF, replica=-1):
        md_set_pulse_table(self.h, replica, dF)

    def rdf(self, r_max, n_bins):
        """Pair counts [n_species][n_species][n_bins] by distance bin (md_rdf)."""
        return md_rdf(self.h, self.ns, r_max, n_bins)

    def fragments(self, r_frag, mass_max=64, charge_max=32):
        """Fragment label of every atom and fragment counts [R][mass][charge] (md_fragments)."""
        return md_fragments(self.h, self.n, self.R, r_frag, mass_max, charge_max)

    def probe_series(self, replica=0, first=0, n=None):
        """Probe records (q_sum, d2_sum), [n][n_species], of the states after
        steps first .. first + n - 1 (md_get_probe_series)."""
        if n is None:
            n = self.get_state(MD_FIELD_STEP)["step"] + 1 - first
        return md_get_probe_series(self.h, self.ns, replica, first, n)

    def probe_displacement(self, probe, replica=0, first=0, n=1):
        """Probe-weighted RMS displacement per species (Eq. 17, md_probe_displacement)."""
        return md_probe_displacement(self.h, self.ns, replica, first, n, probe)

    def set_charge_table(self, frac, replica=-1):
        """Charge-state fractions [rows][n_ts] for charge_mode="table"."""
        md_set_charge_table(self.h, replica, frac)

    def set_plasma_table(self, ne, te_ev, replica=-1):
        md_set_plasma_table(self.h, replica, ne, te_ev)

    def step(self, n=1, wait=True):
        """Advance n steps; wait=False only enqueues them (status read by sync())."""
        if wait:
            md_step(self.h, n)
        else:
            md_step_async(self.h, n)

    def sync(self):
        md_sync(self.h)

    def get_state(self, fields=MD_FIELD_ALL, out=None):
        o = out or {}
        n, R = self.n, self.R
        spec = [("x", MD_FIELD_X, (n, 3), np.float64), ("v", MD_FIELD_V, (n, 3), np.float64),
                ("f", MD_FIELD_F, (n, 3), np.float64), ("q", MD_FIELD_Q, (n,), np.uint8),
                ("h", MD_FIELD_H, (n,), np.uint8), ("n_e", MD_FIELD_PLASMA, (R,), np.int64),
                ("e_gas_mev", MD_FIELD_PLASMA, (R,), np.int64), ("te_ev", MD_FIELD_PLASMA, (R,), np.float64),
                ("kappa", MD_FIELD_PLASMA, (R,), np.float64),
                ("event_counts", MD_FIELD_COUNTS, (R, 4), np.int64),
                ("x_list", MD_FIELD_XLIST, (n, 3), np.float64)]
        st = MDState()
        for name, bit, shape, dt in spec:
            if fields & bit:
                if name not in o:
                    o[name] = np.empty(shape, dtype=dt)
                setattr(st, name, o[name].ctypes.data)
        md_get_state(self.h, st, fields)
        if fields & MD_FIELD_STEP:
            o["step"] = int(st.step)
        return o

    def set_state(self, fields, **arrays):
        st = MDState()
        keep = []
        for name, dt in [("x", np.float64), ("v", np.float64), ("q", np.uint8), ("h", np.uint8),
                         ("n_e", np.int64), ("e_gas_mev", np.int64), ("event_counts", np.int64),
                         ("x_list", np.float64)]:
            if name in arrays and arrays[name] is not None:
                a = _c(arrays[name], dt)
                keep.append(a)
                setattr(st, name, a.ctypes.data)
        st.step = int(arrays.get("step", 0))
        md_set_state(self.h, st, fields)

    def energies(self):
        ek = np.zeros(self.R); ep = np.zeros(self.R)
        n = md_get_energies(self.h, ek, ep)
        return ek, ep, n

    def timing(self):
        return md_get_timing(self.h)

    def reset_timing(self):
        md_reset_timing(self.h)

    def close(self):
        if getattr(self, "h", None):
            md_finalize(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
