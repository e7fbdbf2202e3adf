"""Seeded synthetic pooling instances shared by the oracle tests, the GPU tests and the bench.

This package draws pooling designs, true positives and noisy pool outcomes.  It holds none of the
decoding method's arithmetic (no likelihoods, no weights, no tables, no estimator): both the CPU
oracle and the CUDA library receive its arrays as plain inputs.
"""
from .designs import (Instance, SplitMix64, kset_design, tapestry_like_design, mixed_degree_design,
                      draw_outcomes, make_instance, make_mixed_instance, make_tapestry_like_instance, tiny_config, paper_shaped_config, high_noise_config,
                      batched_configs, budget_horizon)

__all__ = ["Instance", "SplitMix64", "kset_design", "tapestry_like_design", "mixed_degree_design",
           "draw_outcomes", "make_instance", "make_mixed_instance", "make_tapestry_like_instance", "tiny_config", "paper_shaped_config", "high_noise_config",
           "batched_configs", "budget_horizon"]
