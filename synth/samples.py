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


def random_sector_bits_words(n_orb: int, n_up: int, n_dn: int, count: int, seed: int,
                             words: int) -> np.ndarray:
    """random_sector_bits for registers of W words: uint64 [count, W] (qubit j in bit j % 64 of
    word j // 64); the same draws as random_sector_bits."""
    rng = SplitMix64(seed)
    out = np.zeros((count, words), dtype=np.uint64)
    for spin, k in ((0, n_up), (1, n_dn)):
        if k == 0:
            continue
        keys = rng.uniform(count * n_orb).reshape(count, n_orb)
        chosen = np.argsort(keys, axis=1, kind="stable")[:, :k]
        q = 2 * chosen + spin
        for w in range(words):
            sel = (q // 64) == w
            bits = np.where(sel, np.uint64(1) << (q % 64).astype(np.uint64), np.uint64(0))
            out[:, w] |= np.bitwise_or.reduce(bits, axis=1)
    return out
