"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the simulation method: it only draws
Hamiltonians (Pauli strings with real coefficients), initial states and
observables, with the shapes and value distributions of the workloads the
simulator is measured on.  Both the CUDA path and the CPU oracle read the
same arrays from here.
"""
from .generators import *  # noqa: F401,F403
