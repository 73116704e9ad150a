"""The named synthetic workloads (molecule-shaped stand-ins for the paper's Table 1 systems).

Each workload fixes the spatial-orbital count, the electron split, the integral generator's
symmetry and decay options, the model and the nominal sample count.  Seeds: integrals 1000+id,
parameters 2000+id, sampler 3000+id.
"""
from dataclasses import dataclass, field


@dataclass(frozen=True)
class WorkloadConfig:
    cid: int
    name: str
    n_orb: int            # spatial orbitals; qubits n = 2 * n_orb
    n_up: int
    n_dn: int
    irreps: int           # 0 (no symmetry labels), 2 (Z2) or 4 (Z2 x Z2)
    decay: bool           # multiply h_pq and L_pq by exp(-|p-q|/3)
    arch: str             # "made" | "transformer" | "product"
    hidden: int           # MADE hidden width or transformer d_model
    layers: int           # MADE hidden layers or transformer blocks
    heads: int            # transformer heads (0 for MADE)
    n_samples: int        # nominal sample count N_s
    mini_batches: int
    precisions: tuple = field(default=("fp32",))

    @property
    def n_qubits(self) -> int:
        return 2 * self.n_orb

    @property
    def seed_integrals(self) -> int:
        return 1000 + self.cid

    @property
    def seed_params(self) -> int:
        return 2000 + self.cid

    @property
    def seed_sampler(self) -> int:
        return 3000 + self.cid


CONFIGS = {
    1: WorkloadConfig(1, "h2_like_4q_made16", 2, 1, 1, 2, False, "made", 16, 1, 0, 1024, 1, ("fp32",)),
    2: WorkloadConfig(2, "lih_like_12q_made2x64", 6, 2, 2, 4, True, "made", 64, 2, 0, 10_000, 1, ("fp32",)),
    3: WorkloadConfig(3, "n2_like_20q_tf64x2", 10, 7, 7, 4, True, "transformer", 64, 2, 4, 100_000, 1,
                      ("fp32", "bf16")),
    4: WorkloadConfig(4, "li2o_like_30q_tf128x4", 15, 5, 5, 4, True, "transformer", 128, 4, 8, 1 << 17, 8,
                      ("fp32", "bf16")),
    5: WorkloadConfig(5, "large_52q_tf128x4", 26, 8, 8, 0, True, "transformer", 128, 4, 8, 1 << 18, 16,
                      ("fp32", "bf16")),
    # two-word registers (64 < n <= 128): the paper's largest system has 76 qubits (Table 1);
    # the term sweep and the MADE local energy run on seeded in-sector configurations
    6: WorkloadConfig(6, "wide_76q_made2x64", 38, 8, 8, 2, True, "made", 64, 2, 0, 1 << 14, 1, ("fp32",)),
}


def get_config(cid: int) -> WorkloadConfig:
    return CONFIGS[int(cid)]
