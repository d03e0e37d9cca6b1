"""GB300-native PMWA (parallelized multiple-worm algorithm) sweep.

The compute path is libpmwa.so (hand-written sm_103a CUDA behind the C ABI in
include/pmwa.h); this package only marshals arguments to it.  PyTorch
provides the device arena and the CUDA stream.
"""
from ._lib import (PMWA_OK, PMWA_EINVAL, PMWA_ECAPACITY, PMWA_ETIMEOUT, PMWA_ECUDA,
                   PMWA_EINVARIANT, PMWA_EROWS, CHECK_NAMES, Batch, PmwaError, Sim, load, make_params,
                   observables, pmwa_boundary, pmwa_check, pmwa_create, pmwa_destroy, pmwa_export,
                   pmwa_export_bytes, pmwa_footprint, pmwa_get_sweep, pmwa_green, pmwa_green_tau, pmwa_import,
                   pmwa_measure, pmwa_npoint, pmwa_profile, pmwa_profile_phases, pmwa_profile_read, pmwa_rho_alpha, pmwa_rho_slices, pmwa_rho_slices_static, pmwa_set_n_cycle, pmwa_set_sweep, pmwa_slot_capacity, pmwa_tile_smem, pmwa_tile_plan, pmwa_strerror, pmwa_sweep,
                   pmwa_tables, pmwa_tile, ROW_DTYPE, KERNELS, SERIES, summary, n_cycle, pmwa_set_loop_caps,
                   pmwa_philox_blocks, pmwa_temporal, pmwa_npoint_alpha)

__all__ = [n for n in dir() if not n.startswith("_")]
