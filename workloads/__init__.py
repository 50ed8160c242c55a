"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This package holds only input generation: random matrices from the
ensembles the paper samples, unitary-group geodesic points, and uniformly
random residues.  It contains none of the permanent method's arithmetic
(no row sums, products, modular reduction, primes or Chinese remaindering),
so both the CUDA path and the oracle can take inputs from it without sharing
any of the computation being checked.
"""
from .ensembles import (  # noqa: F401
    ENSEMBLES,
    dft_matrix,
    ensemble,
    geodesic_cycle,
    geodesic_dft,
    ginibre_c,
    ginibre_r,
    goe,
    gue,
    haar_orthogonal,
    haar_unitary,
    random_residues,
    rng,
)
