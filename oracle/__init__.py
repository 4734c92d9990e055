"""CPU FP64 oracle for the RSFT hot path (test infrastructure only).

This package is a plain, slow, deliberately literal restatement of the RSFT of
Wang, Patel and Petropulu ("An Efficient High-Dimensional Sparse Fourier
Transform"): Algorithm 1 step by step (§III-C, Algorithm 1), the estimation rule
of §III (last paragraphs before Algorithm 1), and the threshold design of §IV
(eq. (bpd), eq. (opt)).  It exists to check the CUDA path and is never part of
it: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code, table or constant generator with
the CUDA library; both sides only read the same seeded cubes from
``rsft_inputs``.

``refine.py`` is the bucket-domain refinement loss of off-grid tones and its gradient
(beyond the paper), pinned by central finite differences.

The first stage has two modes: known noise (the paper's model, sigma_n^2 given) and an
estimate mode in which each loop's noise floor is the lower median of its bucket powers
divided by ln 2 (eq. (exp): the median of an exponential is its mean times ln 2).  The
second-stage design has the paper's Normal vote approximation (Claims 2-3) and an exact
binomial vote law (``design.optimal_thresholds_binomial``).

``bartlett.py`` is the dense comparison system of Appendix A (Algorithm 2, one
segment): window, full N-D DFT, exact NP threshold on the bin power.

Parity pins (tests marked ``not gpu``) tie every function here to something
other than itself: published constants, closed forms, library routines,
exhaustive brute force and the identities the paper states.  The one function
without such a pin is the off-grid, noisy amplitude estimate
(``estimate_amplitudes`` on off-grid input): parity unpinned beyond its exact
on-grid case.
"""
from .perm import splitmix64, splitmix64_at, draw_sigmas, inverse_mod
from .windows import (chebyshev_window, flat_window, flat_gain, window_6db_bins,
                      chebyshev_poly)
from .pipeline import (OraclePlan, make_plan, rsft, fold_loop, bucket_spectrum,
                       fold_bucket_direct, reverse_map, mapping, estimate_amplitudes,
                       permute, alias, noise_floor_gamma, spectrum_at)
from .refine import tone_field, refine_loss, refine_grad
from .bartlett import bartlett, bartlett_window, bartlett_gamma, bartlett_pd_swerling1
from .design import (beta_sigma, alpha_sigma, mean_alpha, mean_beta, q_func,
                     solve_pd_bar, solve_pfa1, optimal_thresholds, optimal_thresholds_binomial,
                     binomial_vote_tail, solve_pd_bar_binomial, solve_pfa1_binomial,
                     complexity_rsft, complexity_bartlett, first_stage_gamma)

__all__ = [
    "splitmix64", "splitmix64_at", "draw_sigmas", "inverse_mod",
    "chebyshev_window", "flat_window", "flat_gain", "window_6db_bins", "chebyshev_poly",
    "OraclePlan", "make_plan", "rsft", "fold_loop", "bucket_spectrum",
    "fold_bucket_direct", "reverse_map", "mapping", "estimate_amplitudes",
    "permute", "alias", "noise_floor_gamma", "spectrum_at",
    "beta_sigma", "alpha_sigma", "mean_alpha", "mean_beta", "q_func",
    "solve_pd_bar", "solve_pfa1", "optimal_thresholds", "optimal_thresholds_binomial",
    "binomial_vote_tail", "solve_pd_bar_binomial", "solve_pfa1_binomial", "complexity_rsft",
    "complexity_bartlett", "first_stage_gamma",
    "bartlett", "bartlett_window", "bartlett_gamma", "bartlett_pd_swerling1",
    "tone_field", "refine_loss", "refine_grad",
]
