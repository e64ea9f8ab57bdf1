"""GB300-native multi-product imaginary-time propagation (Chin, Janecek,
Krotscheck): a CUDA library with a C ABI (include/itp.h, libitp.so) and its
ctypes binding."""
from .itp import (ITP_EVAL_FP64, ITP_FP64, ITP_MIXED, ITP_RITZ, ITP_RITZ_VALUES,  # noqa: F401
                  ITP_STEP_FP64,
                  itp_autotune, itp_get_tuning, itp_set_tuning,
                  ItpBatch, ItpError, ItpGrid, itp_batch_destroy, itp_batch_problem,
                  itp_batch_step, itp_create_batch, itp_create_grid, itp_destroy,
                  itp_energies, itp_get_phi, itp_get_states, itp_kernel_launches,
                  itp_last_error, itp_orthonormalize, itp_orthonormalize_noalloc, itp_polish,
                  itp_profile, itp_profile_read, itp_propagate, itp_propagate_romberg6,
                  itp_set_potential,
                  itp_set_states, itp_set_states_device, itp_solve_adaptive, itp_step, itp_step_host,
                  itp_synchronize, itp_test_expire_waits, itp_peak_probe, load)
