"""Pins for the oracle's random test-vector init (Alg. 1, "x_i <- rand(-0.5, 0.5)").

The init is Philox4x32-10 (Salmon et al., SC'11).  The oracle's generator is
checked against cuRAND's host-side Philox4x32-10 generator, a separate
implementation of the same published function: block b of cuRAND's host
stream is Philox(counter = (lo32(b >> 16), hi32(b >> 16), b & 0xffff, 0),
key = (seed_lo, seed_hi)).  The grid/range of the derived uniforms and their
statistics are checked from first principles.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so",
                 "/usr/local/cuda/lib64/libcurand.so.10"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def _curand_host_blocks(seed, first_block, n_blocks):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        lib.curandSetPseudoRandomGeneratorSeed.argtypes = [ctypes.c_void_p, ctypes.c_ulonglong]
        lib.curandSetGeneratorOffset.argtypes = [ctypes.c_void_p, ctypes.c_ulonglong]
        lib.curandGenerate.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, seed) == 0
        assert lib.curandSetGeneratorOffset(gen, 4 * first_block) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data, out.size) == 0
        return out.reshape(n_blocks, 4)
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0x1601055270000000, 2**64 - 1])
@pytest.mark.parametrize("first_block", [0, 65530, ((1 << 32) + 7) << 16, (123456789 << 16) | 4321])
def test_philox_matches_curand_host_generator(seed, first_block):
    blocks = _curand_host_blocks(seed, first_block, 8)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    for t in range(8):
        b = first_block + t
        c = b >> 16
        ctr = np.array([c & 0xFFFFFFFF, c >> 32, b & 0xFFFF, 0], dtype=np.uint32)
        np.testing.assert_array_equal(oracle.philox4x32_10(ctr, key), blocks[t])


def test_stream_word_changes_output():
    key = np.array([1, 2], dtype=np.uint32)
    a = oracle.philox4x32_10(np.array([3, 4, 5, 0], dtype=np.uint32), key)
    b = oracle.philox4x32_10(np.array([3, 4, 5, 1], dtype=np.uint32), key)
    # one flipped input bit changes about half of the 128 output bits
    flipped = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b))
    assert 40 < flipped < 88


def test_init_values_lie_on_the_2p24_grid_in_half_open_interval():
    x = oracle.init_vectors(4096, 16, seed=11)
    assert x.min() >= -0.5 and x.max() <= 0.5 - 2.0 ** -24
    q = (x + 0.5) * 2.0 ** 24
    np.testing.assert_array_equal(q, np.round(q))
    # exactly representable in binary32
    np.testing.assert_array_equal(x.astype(np.float32).astype(np.float64), x)


def test_init_value_is_the_top_24_bits_of_the_philox_word():
    seed, stream = 0xDEADBEEF12345678, 3
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    for i, r in [(0, 0), (5, 3), (2**33 + 9, 7), (1000, 30)]:
        ctr = np.array([i & 0xFFFFFFFF, i >> 32, r // 4, stream], dtype=np.uint32)
        u = int(oracle.philox4x32_10(ctr, key)[r % 4])
        assert oracle.test_value(seed, stream, i, r) == (u >> 8) / 2.0 ** 24 - 0.5


def test_init_statistics_uniform():
    x = oracle.init_vectors(1 << 15, 8, seed=5).ravel()
    N = x.size
    # mean 0, variance 1/12 of U(-1/2, 1/2)
    assert abs(x.mean()) < 5 * np.sqrt(1 / 12 / N)
    assert abs(x.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / N)
    # chi-square over 64 equal bins (dof 63): reject only far tails
    h, _ = np.histogram(x, bins=64, range=(-0.5, 0.5))
    chi2 = ((h - N / 64) ** 2 / (N / 64)).sum()
    assert 25 < chi2 < 115
    # serial correlation between consecutive draws
    c = np.corrcoef(x[:-1], x[1:])[0, 1]
    assert abs(c) < 5 / np.sqrt(N)


def test_init_depends_only_on_seed_vertex_and_vector():
    a = oracle.init_vectors(100, 12, seed=9)
    b = oracle.init_vectors(300, 20, seed=9)
    np.testing.assert_array_equal(a, b[:100, :12])
    c = oracle.init_vectors(100, 12, seed=10)
    assert not np.any(a == c).all()
    d = oracle.init_vectors(100, 12, seed=9, stream=1)
    assert np.mean(a == d) < 0.01
