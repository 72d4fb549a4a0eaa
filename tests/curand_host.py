"""Philox4x32-10 blocks from cuRAND's host generator, an implementation independent of this
project, used to pin the oracle's generator (and the GPU's) to the published algorithm.

cuRAND's host generator of type CURAND_RNG_PSEUDO_PHILOX4_32_10 (curandCreateGeneratorHost, no
GPU needed) keys Philox4x32-10 by its 64-bit seed, key = (seed low word, seed high word), and
emits 4-word blocks; with the generator offset set to 4 j0, the i-th block it emits is the block
of counter (q, 0, s, 0) with j = j0 + i, q = j div 65536 and s = j mod 65536 (its 65,536
subsequences interleaved).  So the counters it reaches are (q low, q high, s, 0) for any q < 2^46
and s < 65,536: every word but the last, and any key.
"""
import ctypes
import os

import numpy as np

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
_SUBSEQ = 65536


def library():
    """The cuRAND shared library, or None when it is not installed."""
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        for name in ("libcurand.so", "libcurand.so.10"):
            p = os.path.join(d, "lib64", name)
            if d and os.path.exists(p):
                return ctypes.CDLL(p)
    try:
        return ctypes.CDLL("libcurand.so.10")
    except OSError:
        return None


def blocks(lib, seed: int, first_block: int, n: int) -> np.ndarray:
    """Blocks first_block .. first_block + n - 1 of the host generator: [n, 4] uint32."""
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * first_block)) == 0
        out = np.zeros(4 * n, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(4 * n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(n, 4)


def counter_of(j: int):
    """Philox counter (4 words) of the generator's block j."""
    q, s = divmod(j, _SUBSEQ)
    return [q & 0xFFFFFFFF, (q >> 32) & 0xFFFFFFFF, s, 0]


def key_of(seed: int):
    return [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]


# seeds and first blocks spanning every key bit pattern and counter words 0, 1 and 2
CASES = [(0, 0), (1, 0), (0xFFFFFFFFFFFFFFFF, 0), (0x243F6A8885A308D3, 12345),
         (0x13198A2E03707344, (1 << 16) * 0xA4093822 + 777), ((1 << 63) + 5, (1 << 16) * ((1 << 45) + 3) + 65530)]
