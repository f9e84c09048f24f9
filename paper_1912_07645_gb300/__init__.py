"""GB300 (sm_103a) finite-volume Monte Carlo solver for hyperbolic conservation laws.

Implements the data-parallel core of Alsvinn (arXiv:1912.07645): the semi-discrete finite-volume
update of eq. (2.1) with HLLC / Rusanov / HLL fluxes, PC / MC / WENO3 reconstruction and SSP-RK
time stepping (Sec. 2.1), run over many Monte Carlo samples with per-cell mean and variance kept
on the device (Sec. 2.2). All arithmetic runs in libalsv.so (hand-written CUDA); this package only
marshals arguments (``_abi``, same names as include/alsv.h) and allocates caller-owned buffers
with torch (``Solver``).
"""
from __future__ import annotations

from ._abi import (BC, EQ, FLUX, INIT, PRECISION, RECON, RK, RVARS, AlsvError, alsv_adjoint_evolve, alsv_adjoint_get_plan,  # noqa: F401
                   alsv_adjoint_workspace_bytes, alsv_autotune, alsv_bind_adjoint_workspace,
                   alsv_bind_workspace, alsv_conservation_totals, alsv_conservation_totals_noalloc, alsv_destroy, alsv_evolve_to_T,
                   alsv_get_launch_count, alsv_get_parameters, alsv_get_profile, alsv_get_tile, alsv_get_time, alsv_grid_desc,
                   alsv_init_grid, alsv_kinetic_energy, alsv_last_error, alsv_mlmc_accumulate, alsv_mlmc_bytes,
                   alsv_correlator_accumulate, alsv_joint_pdf_accumulate, alsv_mlmc_read, alsv_mlmc_reset,
                   alsv_point_pdf_accumulate,
                   alsv_structure_function_accumulate, alsv_structure_function_bytes,
                   alsv_structure_function_read, alsv_num_samples,
                   alsv_num_tile_variants, alsv_num_vars, alsv_set_graphs, alsv_set_initial_data,
                   alsv_set_profiling, alsv_set_tile_variant, alsv_set_time, alsv_state_bytes, alsv_stats_accumulate,
                   alsv_stats_bytes, alsv_stats_merge, alsv_stats_read, alsv_stats_reset, alsv_step, alsv_sync,
                   alsv_version, load, alsv_halo_info, alsv_bind_halo, alsv_halo_pack, alsv_stage,
                   alsv_speed_max, alsv_speed_max_combine, alsv_stage_part, alsv_evolve_resident, alsv_finish_step, alsv_set_end_time, alsv_mixing_width,
                   OBSERVABLE)
from .provenance import provenance, save_result  # noqa: F401
from .solver import Solver, make_desc  # noqa: F401
