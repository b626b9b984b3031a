"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the benchmark.

This package holds none of the inversion method's arithmetic: it builds tau
grids, frequency grids, peak spectra, their exact Laplace transforms, noise
and the two sum constants A and B of Sec. 2.2, and nothing else.
"""
from .spectra import Peak, laplace, mass, first_moment, bin_masses  # noqa: F401
from .problems import (  # noqa: F401
    Problem,
    make_problem,
    tiny_double_lorentz,
    paper_scale_double_lorentz,
    precision_random_peaks,
    random_batch_problem,
    random_peaks,
    lorentzian_band,
    lorentzian_band_peaks,
    skew,
)
