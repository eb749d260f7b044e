"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds none of the matched filter's arithmetic: no noise-weighted
inner products, no correlation, no SNR normalisation, threshold, clustering,
coincidence or neighbourhood union.  It only builds the things both
implementations start from: the analytic detector PSD, coloured Gaussian
noise, TaylorF2 templates and injections, sine-Gaussian glitches, template
banks and their neighbourhood maps.  Everything is drawn from
``numpy.random.default_rng(seed)`` so the same seed gives the same inputs on
any machine.
"""

from .generators import (  # noqa: F401
    MTSUN_S,
    psd_analytic,
    psd_bins,
    chirp_times,
    masses_from_chirp_times,
    chirp_mass,
    duration_2pn,
    f_isco,
    taylorf2_phase,
    taylorf2,
    taylorf2_torch,
    taylorf2_chunks_torch,
    coloured_noise_fd,
    sine_gaussian,
    sine_gaussian_amplitude,
    taylorf2_norm_continuum,
    strain_from_fd,
    sample_bank_uniform_masses,
    sample_bank_chirp_times,
    nbhd_map,
    metric_match,
)
from .configs import (  # noqa: F401
    Config1,
    make_config1,
    Config2,
    make_config2,
    make_banks,
    Config3,
    make_config3,
    Config4,
    make_config4,
)
