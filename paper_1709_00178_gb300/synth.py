"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle runs.

This module holds no coding arithmetic: it only produces uniform random bytes. The generator is
SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
used in counter mode: 64-bit word i of a stream with seed s is mix(s + (i + 1) * gamma), so any
word range can be produced independently, here with numpy and on the device by the library's
``pyrit_synth_fill`` (which implements the same published definition).

Bytes are the little-endian bytes of consecutive words; byte offset o of a stream is byte o % 8
of word o // 8.
"""
import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

#: Base seed of the workloads; workload c uses BASE_SEED + c.
BASE_SEED = 0x5059524954


def splitmix64_words(seed: int, start: int, count: int) -> np.ndarray:
    """Words [start, start + count) of the counter-mode SplitMix64 stream ``seed``."""
    i = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.uint64(GAMMA) * i
        z ^= z >> np.uint64(30)
        z *= np.uint64(MIX1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(MIX2)
        z ^= z >> np.uint64(31)
    return z


def synth_bytes(seed: int, offset: int, nbytes: int) -> np.ndarray:
    """Bytes [offset, offset + nbytes) of stream ``seed`` as a uint8 array."""
    if nbytes <= 0:
        return np.zeros(0, np.uint8)
    w0 = offset // 8
    w1 = (offset + nbytes + 7) // 8
    words = splitmix64_words(seed, w0, w1 - w0)
    b = words.astype("<u8").view(np.uint8)
    s = offset - w0 * 8
    return b[s:s + nbytes].copy()


def stripe_layout(k: int, m: int, w: int, P: int):
    """Byte sizes of the contiguous stripe layout used by the benchmark and tests:
    a stripe is k+m blocks, a block is w packets of P bytes (packet q at q*P)."""
    block = w * P
    return block, (k + m) * block


def mixed_batch_specs(seed: int, count: int = 4096):
    """The mixed-batch workload: ``count`` stripes (w, k, m, P, op, erasures) drawn with numpy's
    PCG64 generator from ``seed``. Per stripe: the ring n uniform in {5, 11, 13} (w = n - 1); k in
    4..32 and m in 2..8, both drawn again until k + m <= 2^w (the Cauchy code needs distinct
    points); P log-uniform over [512 B, 256 KiB], rounded down to a multiple of 16; encode or decode
    with equal odds, a decode losing e blocks, e uniform in 1..m, chosen uniformly among the k + m.
    Random draws only: no coding arithmetic."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        n = int(rng.choice([5, 11, 13]))
        w = n - 1
        while True:
            k, m = int(rng.integers(4, 33)), int(rng.integers(2, 9))
            if k + m <= (1 << w):
                break
        P = max(16, int(2 ** rng.uniform(9, 18)) // 16 * 16)
        op = int(rng.integers(0, 2))
        er = 0
        if op:
            e = int(rng.integers(1, m + 1))
            er = sum(1 << int(x) for x in rng.choice(k + m, e, replace=False))
        specs.append((w, k, m, P, op, er))
    return specs


def stripe_offsets(specs, align: int = 256):
    """Byte offsets of stripes (w, k, m, P, ...) laid out one after another in one buffer, each
    starting on an ``align``-byte boundary; returns (offsets, total bytes)."""
    offs, total = [], 0
    for s in specs:
        w, k, m, P = s[:4]
        offs.append(total)
        total += ((k + m) * w * P + align - 1) // align * align
    return offs, total
