"""psum: periodic Coulomb sums on one GB300 by the periodisation method of
Gumerov & Duraiswami (arXiv 1310.4374).

The computation lives in ``libpsum.so`` (C-ABI, ``include/psum.h``); this
package holds its build script, a thin ctypes binding with the same function
names, and the seeded input generators used by the tests and the benchmark.
"""
from .binding import (PSUM_ERR_ARG, PSUM_ERR_CUDA, PSUM_ERR_NOMEM, PSUM_ERR_NONFINITE, PSUM_ERR_NONNEUTRAL,
                      PSUM_ERR_OUT_OF_BOX, PSUM_ERR_RANK, PSUM_ERR_TIMEOUT, PSUM_FP32C, PSUM_FP64,
                      PSUM_MEAN_NONE, PSUM_MEAN_ZERO, PSUM_OK, PeriodicCoulomb, PsumError, load, psum_destroy,
                      psum_eval, psum_eval_host, psum_get_coeffs, psum_last_timings, psum_opts_default,
                      psum_plan_create, psum_plan_create_ex, psum_plan_info, psum_profile, psum_strerror,
                      psum_sync, psum_energy, psum_energy_backward)

__all__ = [n for n in dir() if n.startswith(("psum_", "PSUM_"))] + ["PeriodicCoulomb", "PsumError", "load"]
