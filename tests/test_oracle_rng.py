"""Pins of the oracle's random streams and logarithm.

Philox4x32-10 is pinned against cuRAND's host-side generator (a library
routine running on the CPU): with the default ordering, block j of its output
is Philox(counter = (j // 65536, 0, j % 65536, 0), key = seed).
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and (os.path.exists(cand) or not cand.startswith("/")):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    pytest.skip("libcurand not found")


def _curand_host_words(seed, n):
    lib = _curand()
    g = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        buf = np.empty(n, np.uint32)
        assert lib.curandGenerate(g, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return buf


@pytest.mark.parametrize("seed", [0, 1, 0xFEDCBA9876543210, 0x00000001FFFFFFFF])
def test_philox_matches_curand_host(seed):
    n_blocks = 65536 + 300
    ref = _curand_host_words(seed, 4 * n_blocks).reshape(-1, 4)
    j = np.arange(n_blocks, dtype=np.uint64)
    sel = np.concatenate([np.arange(0, 2000), np.arange(65000, n_blocks)])
    ctr = np.zeros((sel.size, 4), np.uint32)
    ctr[:, 0] = (j[sel] // 65536).astype(np.uint32)
    ctr[:, 2] = (j[sel] % 65536).astype(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    got = oracle.philox(ctr, key)
    np.testing.assert_array_equal(got, ref[sel])


def test_stream_layout():
    # Stream of history hid at angle a: counters (k, a, hid lo, hid hi), k = 0, 1, ...
    seed, a, hid = 0x1234_5678_9ABC_DEF0, 7, (3 << 32) | 11
    words = oracle.stream_words(seed, a, hid, 3).reshape(3, 4)
    ctr = np.array([[k, a, 11, 3] for k in range(3)], np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    np.testing.assert_array_equal(words, oracle.philox(ctr, key))


def test_stream_words_are_uniform():
    # Top-24-bit uniforms of one long stream: Kolmogorov-Smirnov against U(0,1].
    from scipy import stats
    w = oracle.stream_words(99, 0, 5, 50000)
    u = ((w >> 8).astype(np.float64) + 1.0) * 2.0**-24
    assert u.min() > 0.0 and u.max() <= 1.0
    assert stats.kstest(u, "uniform").pvalue > 0.01


def test_logf_accuracy():
    # Every uniform the transport can draw is k * 2^-24, k = 1..2^24; check a
    # dense sample of them plus all powers of two, against the FP64 log.
    rng = np.random.default_rng(0)
    k = np.unique(np.concatenate([rng.integers(1, 2**24 + 1, 400000), 2 ** np.arange(25),
                                  np.arange(1, 5000), 2**24 - np.arange(5000)]))
    x = (k.astype(np.float64) * 2.0**-24).astype(np.float32)
    got = oracle.logf(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    ulp[ref == 0] = np.spacing(np.float32(0))
    err = np.abs(got - ref)
    assert np.all(err <= 2.0 * ulp), (err / ulp).max()
    assert got[x == 1.0].item() == 0.0


def test_logf_general_range():
    x = np.geomspace(1e-30, 1e30, 20001).astype(np.float32)
    got = oracle.logf(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3)
    assert rel.max() < 4e-7
