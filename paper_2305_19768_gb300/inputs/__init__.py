"""Seeded input generators shared by the CUDA path and the CPU oracle.

Nothing here evaluates the lattice rule: these modules build sector
descriptions (Feynman polynomials, sector decomposition, prefactor series),
kinematic points and rank-1 lattice generating vectors, which are inputs to
both sides.
"""
