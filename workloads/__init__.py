"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library."""
from .circuits import (Circuit, Op, repetition_code, surface_code, random_layered,
                       batch_suite, perturbed_probabilities, channel_probabilities,
                       random_small_circuit, random_clifford_circuit, mirror_circuit,
                       random_feedforward_circuit, with_channel_probabilities,
                       surface_code_all_channels)

__all__ = ["Circuit", "Op", "repetition_code", "surface_code", "random_layered",
           "batch_suite", "perturbed_probabilities", "channel_probabilities",
           "random_small_circuit", "random_clifford_circuit", "mirror_circuit",
           "random_feedforward_circuit", "with_channel_probabilities",
           "surface_code_all_channels"]
