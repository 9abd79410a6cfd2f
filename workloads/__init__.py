"""Seeded synthetic inputs: Hamiltonians and collapse operators.

This package builds the operators H and C_k (sparse, d x d, complex128) of the
quantum-optics systems the solver is exercised on. It holds none of the
steady-state method's arithmetic (no Liouvillian, no ordering, no
factorisation, no Krylov step): both the CUDA path's tests and the CPU oracle
take their inputs from here.
"""
from .quantum_optics import (  # noqa: F401
    System,
    destroy,
    sigma_minus,
    sigma_x,
    sigma_y,
    sigma_z,
    identity,
    tensor,
    driven_cavity,
    thermal_cavity,
    jaynes_cummings_rwa,
    optomechanics,
    kerr_oscillator,
    kerr_sweep,
    kerr_chain,
    two_level_atom,
    random_system,
    paper_jc_nonrwa,
    paper_spin_chain,
    paper_optomechanics,
    config_systems,
)
