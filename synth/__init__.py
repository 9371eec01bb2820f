"""Seeded synthetic inputs for the symmetry-reduced BSE block builder.

A fixture shared by the CPU oracle, the tests and the benchmark; it contains
no Bethe-Salpeter arithmetic of its own.
"""
from .generate import CONFIGS, HA_EV, Config, generate, subset_pairs  # noqa: F401
