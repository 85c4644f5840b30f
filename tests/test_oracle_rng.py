"""Pins of the oracle's random-number pieces (no GPU).

Philox4x32-10 is checked block by block against the cuRAND host generator
(CURAND_RNG_PSEUDO_PHILOX4_32_10), run as a library on the CPU: its k-th
output block is Philox(counter = (0, 0, k, 0), key = (seed_lo, seed_hi)).
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest


def _curand():
    for cand in ("libcurand.so", "libcurand.so.10",
                 os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so")):
        try:
            return ctypes.CDLL(cand)
        except OSError:
            continue
    return None


def _curand_host_philox(lib, seed, n_words, offset=0):
    g = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(g), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
        buf = (ctypes.c_uint32 * n_words)()
        assert lib.curandGenerate(g, buf, ctypes.c_size_t(n_words)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return np.frombuffer(buf, dtype=np.uint32).copy()


@pytest.mark.parametrize("seed", [0, 1, 12345, 0xDEADBEEF12345678, 2**64 - 1])
def test_philox_matches_curand_host(oracle_mod, seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not present")
    n_blocks = 4096
    ref = _curand_host_philox(lib, seed, 4 * n_blocks).reshape(-1, 4)
    ctr = np.zeros((n_blocks, 4), dtype=np.uint32)
    ctr[:, 2] = np.arange(n_blocks)
    got = oracle_mod.philox_blocks(seed, ctr)
    np.testing.assert_array_equal(got, ref)


def test_philox_counter_words_all_matter(oracle_mod):
    base = oracle_mod.philox_blocks(7, [[1, 2, 3, 4]])[0]
    for w in range(4):
        c = [1, 2, 3, 4]
        c[w] ^= 1
        assert not np.array_equal(oracle_mod.philox_blocks(7, [c])[0], base)
    # distinct counters -> distinct blocks (bijection for a fixed key)
    ids = np.arange(200_000, dtype=np.uint32)
    out = oracle_mod.philox(99, ids, ids * 3 + 1)
    assert len(np.unique(out.view(np.dtype((np.void, 16))))) == len(ids)


def test_u53_extremes_and_uniformity(oracle_mod):
    assert oracle_mod.u53(0, 0) == 0.0
    assert oracle_mod.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle_mod.u53(0x80000000, 0) == 0.5
    assert oracle_mod.u53(0, 64) == 2.0 ** -53
    ids = np.arange(100_000, dtype=np.uint32)
    w = oracle_mod.philox(2024, ids, np.zeros_like(ids))
    u = np.array([oracle_mod.u53(int(a), int(b)) for a, b in w[:20000, :2]])
    from scipy import stats
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_one_minus_exp_neg_vs_expm1(oracle_mod):
    rng = np.random.default_rng(3)
    x = np.concatenate([np.logspace(-300, 0, 4000), rng.uniform(0, 40, 20000),
                        np.arange(0, 640) / 16.0, np.arange(1, 640) / 16.0 - 1e-15,
                        [1e-320, 5e-324, 0.0625, 0.5, 1.0, 39.99]])
    p = oracle_mod.one_minus_exp_neg(x)
    ref = -np.expm1(-x)
    rel = np.abs(p - ref) / np.maximum(np.abs(ref), np.finfo(float).tiny)
    assert rel.max() < 8 * np.finfo(float).eps, rel.max()
    # p <= x holds exactly (used as an exact shortcut by the GPU path)
    assert np.all(p <= x)
    assert np.all(np.diff(p[np.argsort(x)]) >= -4e-16)
    assert oracle_mod.one_minus_exp_neg(np.array([0.0, -1.0, 40.0, 1e9])).tolist() == [0.0, 0.0, 1.0, 1.0]
