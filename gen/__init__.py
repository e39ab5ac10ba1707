"""Seeded synthetic input generators (input recipe only, no method arithmetic)."""
from .synth import (SystemSpec, SMALL_2x2x2, DIAMOND_3x3x3, DIAMOND_4x4x4, BATCHED_UNEVEN, kpoints,
                    chol_block, cholesky, one_body, trial, trial_dense, walkers, near_trial_walkers, fields, perturbation,
                    upstream, DenseSpec, DENSE_1x1x2, KPOINT_1x1x2, dense_cholesky, dense_one_body,
                    dense_trial, dense_walkers, dense_near_trial_walkers, dense_fields)

__all__ = ["SystemSpec", "SMALL_2x2x2", "DIAMOND_3x3x3", "DIAMOND_4x4x4", "BATCHED_UNEVEN", "kpoints",
           "chol_block", "cholesky", "one_body", "trial", "trial_dense", "walkers", "near_trial_walkers", "fields", "perturbation",
           "upstream", "DenseSpec", "DENSE_1x1x2", "KPOINT_1x1x2", "dense_cholesky", "dense_one_body",
           "dense_trial", "dense_walkers", "dense_near_trial_walkers", "dense_fields"]
