"""Seeded random bitstrings inside the (n_up, n_dn) particle-number sector."""
import numpy as np

from .rng import SplitMix64


def random_sector_bits(n_orb: int, n_up: int, n_dn: int, count: int, seed: int) -> np.ndarray:
    """count uint64 bitstrings, each with a uniformly random n_up-subset of spin-up orbitals
    (even bits) and n_dn-subset of spin-down orbitals (odd bits)."""
    rng = SplitMix64(seed)
    out = np.zeros(count, dtype=np.uint64)
    for spin, k in ((0, n_up), (1, n_dn)):
        if k == 0:
            continue
        keys = rng.uniform(count * n_orb).reshape(count, n_orb)
        chosen = np.argsort(keys, axis=1, kind="stable")[:, :k]
        bits = (np.uint64(1) << (2 * chosen + spin).astype(np.uint64))
        out |= np.bitwise_or.reduce(bits, axis=1)
    return out
