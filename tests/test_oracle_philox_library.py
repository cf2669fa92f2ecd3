"""Bit-level pin of the oracle's Philox4x32-10 block (Salmon, Moraes, Dror &
Shaw, SC'11: ten rounds, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key
increments 0x9E3779B9 / 0xBB67AE85) against an independent implementation:
the host-side Philox4_32_10 generator of the cuRAND library, which needs no
GPU.

cuRAND keys the generator with the 64-bit seed (low word first) and emits
whole blocks; the block at output offset 4b has the counter
(c0, c1, c2, c3) = (q mod 2^32, q div 2^32, b mod 2^16, 0) with q = b div 2^16.
Random seeds and offsets therefore pin both key words, all 32 bits of
counter word 0, the low 14 bits of word 1 and the low 16 bits of word 2
through the library.  Counter word 3 stays 0 there; the avalanche test of the
oracle covers it."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle as O

_PHILOX4_32_10 = 161  # curandRngType_t value of the Philox generator


def _curand():
    names = [ctypes.util.find_library("curand")]
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    names += [os.path.join(cuda, "lib64", "libcurand.so"), os.path.join(cuda, "lib64", "libcurand.so.10")]
    for nm in names:
        if not nm:
            continue
        try:
            return ctypes.CDLL(nm)
        except OSError:
            continue
    pytest.skip("cuRAND library not found")


def _library_words(L, seed, n_words, offset=0):
    g = ctypes.c_void_p()
    assert L.curandCreateGeneratorHost(ctypes.byref(g), _PHILOX4_32_10) == 0
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert L.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert L.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n_words)) == 0
    finally:
        L.curandDestroyGenerator(g)
    return out


def _counter(b):
    q, r = divmod(b, 1 << 16)
    return [q & 0xFFFFFFFF, q >> 32, r, 0]


def _key(seed):
    return [seed & 0xFFFFFFFF, seed >> 32]


@pytest.mark.parametrize("seed", [0, 1, 0xFEDCBA9876543210, 0xFFFFFFFFFFFFFFFF])
def test_oracle_blocks_equal_library_stream(seed):
    """A stream of 65,600 blocks from offset 0 (past the first wrap of counter
    word 2 into word 0): sampled blocks, the wrap and the first ones equal the
    oracle's block for the same key and counter, word for word."""
    L = _curand()
    n_blocks = (1 << 16) + 64
    blocks = _library_words(L, seed, 4 * n_blocks).reshape(-1, 4)
    rng = np.random.default_rng(seed & 0xFFFF)
    picks = set(range(40)) | set(range((1 << 16) - 8, n_blocks)) | set(int(v) for v in rng.integers(0, n_blocks, 400))
    for b in sorted(picks):
        assert np.array_equal(O.philox4x32_10(_counter(b), _key(seed)), blocks[b]), f"seed {seed:#x}, block {b}"


def test_oracle_blocks_equal_library_at_random_offsets():
    """Random keys and counters (word 0 over its full 32 bits, word 1 up to
    2^14, word 2 up to 2^16): the library's block at that offset equals the
    oracle's block."""
    L = _curand()
    rng = np.random.default_rng(2312)
    for _ in range(200):
        seed = int(rng.integers(0, 1 << 63, dtype=np.uint64)) * 2 + int(rng.integers(0, 2))
        c0 = int(rng.integers(0, 1 << 32, dtype=np.uint64))
        c1 = int(rng.integers(0, 1 << 14))
        c2 = int(rng.integers(0, 1 << 16))
        b = ((c1 << 32) + c0) * (1 << 16) + c2
        got = _library_words(L, seed, 4, offset=4 * b)
        assert _counter(b) == [c0, c1, c2, 0]
        assert np.array_equal(O.philox4x32_10([c0, c1, c2, 0], _key(seed)), got), (seed, c0, c1, c2)


def test_zero_key_zero_counter_block():
    """The all-zero key and counter: the library's first block equals the
    oracle's block and is not the identity or zero."""
    L = _curand()
    lib = _library_words(L, 0, 4)
    assert np.array_equal(O.philox4x32_10([0, 0, 0, 0], [0, 0]), lib)
    assert lib.any() and len(set(int(v) for v in lib)) == 4


def test_counter_word_roles_are_distinguished():
    """The library's third block has counter word 2 = 2: the oracle's block
    with that value in word 0 or word 3 instead differs, so a transposed
    counter word in the oracle would fail the pins above."""
    L = _curand()
    lib = _library_words(L, 0x0123456789ABCDEF, 4 * 3).reshape(-1, 4)
    key = _key(0x0123456789ABCDEF)
    assert np.array_equal(O.philox4x32_10([0, 0, 2, 0], key), lib[2])
    assert not np.array_equal(O.philox4x32_10([0, 0, 0, 2], key), lib[2])
    assert not np.array_equal(O.philox4x32_10([2, 0, 0, 0], key), lib[2])
    assert not np.array_equal(O.philox4x32_10([0, 0, 2, 0], key[::-1]), lib[2])
