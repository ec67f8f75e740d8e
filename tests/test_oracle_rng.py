"""Pin of the oracle's Philox4x32-10 against an independent implementation.

cuRAND's host-side generator (CURAND_RNG_PSEUDO_PHILOX4_32_10, run on the CPU,
no GPU involved) emits, for seed s and stream offset 4*(65536*(c0 + 2^32*c1) + c2),
the block Philox4x32-10(counter = (c0, c1, c2, 0), key = (s mod 2^32, s >> 32))
as its first four words.  The method's draws use counters of exactly this form
(the last counter word is always 0), so this pins every draw the oracle makes.
"""
import ctypes
import ctypes.util
import glob
import os

import numpy as np
import pytest


def _find_curand():
    cands = []
    lib = ctypes.util.find_library("curand")
    if lib:
        cands.append(lib)
    for base in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/*/lib"):
        cands += sorted(glob.glob(os.path.join(base, "libcurand.so*")))
    try:
        import nvidia  # noqa: F401  (pip-packaged CUDA libraries, if any)
        for p in nvidia.__path__:
            cands += sorted(glob.glob(os.path.join(p, "*", "lib", "libcurand.so*")))
    except Exception:
        pass
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


CURAND = _find_curand()


def curand_block(seed: int, c0: int, c1: int, c2: int) -> np.ndarray:
    lib = CURAND
    gen = ctypes.c_void_p()
    PHILOX = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        off = 4 * (65536 * (c0 + (c1 << 32)) + c2)
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(off)) == 0
        out = np.zeros(4, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), 4) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.skipif(CURAND is None, reason="libcurand not found")
@pytest.mark.parametrize("seed", [1, 0x123456789ABCDEF, 2**64 - 1, 0xDEADBEEF00000000])
def test_philox_matches_curand_host_generator(oracle_mod, seed):
    rng = np.random.default_rng(seed % 1000)
    cases = [(0, 0, 0), (1, 0, 0), (0, 0, 1), (5, 1, 7), (65535, 3, 65535), (2**32 - 1, 2**14 - 1, 65535)]
    cases += [(int(rng.integers(0, 2**32)), int(rng.integers(0, 2**14)), int(rng.integers(0, 65536)))
              for _ in range(6)]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for c0, c1, c2 in cases:
        ours = oracle_mod.philox4x32_10([c0, c1, c2, 0], key)
        assert np.array_equal(ours, curand_block(seed, c0, c1, c2)), (seed, c0, c1, c2)


def test_bounded_draws_are_uniform(oracle_mod):
    # init draws: S(v) uniform over D(v) \ {0}; chi-square on an empty 6x6 grid
    I = oracle_mod.Instance(np.zeros((6, 6), dtype=np.int8))
    P = I.init_population(3000, 7)
    counts = np.bincount(P.ravel(), minlength=7)[1:]
    expected = P.size / 6
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert counts.sum() == P.size and chi2 < 30.0      # 5 dof; p ~ 1e-5 threshold
