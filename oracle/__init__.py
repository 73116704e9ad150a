"""FP64 CPU oracle for the NQS local-energy hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct restatement of what the paper's method computes, used to check
the CUDA library.  Only the test suite, the package's smoke check and the bench's CPU-baseline
leg may import it; the library itself never does, and this package imports nothing from the
library.  It shares no code with the CUDA path: the only common inputs come from the separate
`synth` package (seeded integrals, parameters, bitstrings), which holds none of the method's
arithmetic.

Modules (each function cites the part of the paper it restates):
  pauli      matrix elements from the 2x2 sigma matrices, dense H, Pauli decomposition
  fermion    dense H from second-quantised operators acting on occupation bitstrings
  grouping   merge / group Pauli strings by X flip mask with the (-i)^r phase folded in
  models     MADE, decoder-only transformer and product models in FP64 (torch CPU), with the
             Hamming-weight constraint and optional bf16 quantisation emulation
  sampler    Philox4x32-10 and unique-sample autoregressive sampling with counts
  eloc       local energy by the per-term definition
  vmc        energy statistics, VMC gradient (autograd in FP64), Adam
  lanczos    sector-restricted Hamiltonian and a textbook Lanczos eigensolver

Parity status: every function here is pinned by a CPU test against a closed form, an invariant,
a library routine or brute force (tests/test_oracle_*.py); none is "parity unpinned".
"""
