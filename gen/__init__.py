"""Seeded synthetic input generators (input recipe only, no method arithmetic)."""
from .synth import (SystemSpec, SMALL_2x2x2, DIAMOND_3x3x3, DIAMOND_4x4x4, BATCHED_UNEVEN, kpoints,
                    chol_block, cholesky, one_body, trial, walkers, fields, perturbation,
                    upstream)

__all__ = ["SystemSpec", "SMALL_2x2x2", "DIAMOND_3x3x3", "DIAMOND_4x4x4", "BATCHED_UNEVEN", "kpoints",
           "chol_block", "cholesky", "one_body", "trial", "walkers", "fields", "perturbation",
           "upstream"]
