"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This package only draws numbers (network topology, ReacLib-form fit
coefficients, per-zone temperature / density / abundances).  It holds none
of the burn's arithmetic: no rates, no right-hand side, no integrator.
"""
from .workloads import (CONFIGS, network, zones, problem, largest_species,
                        NetworkSpec)

__all__ = ["CONFIGS", "network", "zones", "problem", "largest_species",
           "NetworkSpec"]
