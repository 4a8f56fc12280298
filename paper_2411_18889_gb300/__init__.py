"""GB300 (sm_103a) all-pairs Plummer-softened gravity: Python binding of libnbody.

The computation is the N-body demonstration of Miki & Hanawa, Sec. III.A
(Eq. 1 and Listing 4), written as hand-written CUDA behind a C ABI
(include/nbody.h); this package only marshals arguments to it.
"""
from ._lib import (NBODY_ACC_COMPENSATED, NBODY_ACC_FP32, NBODY_ACC_KAHAN_PAIR, NBODY_EINVAL, NBODY_ENOMEM, NBODY_ENOTSUP, NBODY_ECUDA, NBODY_EBOUNDS,
                   NBODY_ETIMEOUT, NBODY_OK, NBODY_PREC_MIXED, NBODY_PREC_MIXED_UNSORTED, NBODY_PREC_PLAIN, NbodyError,
                   load)
from .api import (accel, nbody_accel, nbody_accel_batched, nbody_accel_f32, nbody_accel_ij, nbody_accel_ij_f32, nbody_accel_vjp,
                  nbody_leapfrog_batched,
                  nbody_leapfrog_record, nbody_leapfrog_vjp, nbody_leapfrog_vjp_tape, nbody_tape_bytes, nbody_config_block, nbody_energy, nbody_energy_f32,
                  nbody_finalize, nbody_last_device_error, nbody_leapfrog, nbody_leapfrog_f32, nbody_num_configs,
                  nbody_num_batched_configs, nbody_profile_enable, nbody_profile_read, nbody_profile_read_kind, nbody_selftest_wait, nbody_version)

from .autograd import Trajectory  # noqa: E402

__all__ = [
    "NBODY_ACC_COMPENSATED", "NBODY_ACC_FP32", "NBODY_ACC_KAHAN_PAIR", "NBODY_EINVAL", "NBODY_ENOMEM", "NBODY_ENOTSUP", "NBODY_ECUDA", "NBODY_EBOUNDS",
    "NBODY_ETIMEOUT", "NBODY_OK", "NBODY_PREC_MIXED", "NBODY_PREC_MIXED_UNSORTED", "NBODY_PREC_PLAIN", "NbodyError", "load", "accel",
    "nbody_accel", "nbody_accel_ij", "nbody_accel_ij_f32", "nbody_accel_vjp", "nbody_leapfrog_record", "nbody_leapfrog_vjp", "nbody_leapfrog_vjp_tape", "nbody_tape_bytes",
    "Trajectory", "nbody_accel_batched", "nbody_leapfrog_batched", "nbody_accel_f32", "nbody_config_block", "nbody_energy", "nbody_energy_f32", "nbody_finalize",
    "nbody_last_device_error", "nbody_leapfrog", "nbody_leapfrog_f32", "nbody_num_configs", "nbody_num_batched_configs", "nbody_selftest_wait", "nbody_version",
    "nbody_profile_enable", "nbody_profile_read", "nbody_profile_read_kind",
]
