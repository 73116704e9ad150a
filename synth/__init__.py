"""Seeded synthetic inputs shared by the tests, the bench and the oracle's tests.

This package generates inputs only: molecule-shaped Jordan-Wigner Hamiltonians from seeded
one- and two-electron integrals, model parameters, random in-sector bitstrings and the named
workload configurations.  It holds none of the method's arithmetic (grouping, term sweep,
network, sampling, energy statistics, gradient); both the CUDA library and the oracle consume
what it produces.
"""
from .rng import SplitMix64
from .configs import CONFIGS, WorkloadConfig, get_config
from .hamiltonian import integrals, jordan_wigner, hamiltonian_for, jordan_wigner_words, hamiltonian_words_for
from .params import init_params, param_shapes, default_order, hf_occupied
from .samples import random_sector_bits, random_sector_bits_words

__all__ = [
    "SplitMix64", "CONFIGS", "WorkloadConfig", "get_config", "integrals", "jordan_wigner",
    "hamiltonian_for", "init_params", "param_shapes", "default_order", "hf_occupied",
    "random_sector_bits", "jordan_wigner_words", "hamiltonian_words_for", "random_sector_bits_words",
]
