"""GB300 shifted-COCG / Dyson transport library: Python binding of the C ABI in ``include/rsfd.h``.

Every function here only marshals arguments (numpy host arrays, torch device
tensors, the current CUDA stream) into the C entry points of ``librsfd.so``;
all arithmetic of the method runs in the library's CUDA kernels (or, for the
lead self-energy helper, in its host C++).  There is no Python or CPU
fallback: importing the binding fails if the library has not been built.

Paper: S. Iwase, T. Hoshi, T. Ono, "Efficient numerical solver for
first-principles transport calculation based on real-space finite-difference
method" -- shifted COCG for the unperturbed Green's functions (Sec. III B,
Appendix) and the OBM/Dyson relation to the perturbed ones (Eq. sec3-01a).
"""

from .binding import (  # noqa: F401
    RSFD_OK, RSFD_ERR_ARG, RSFD_ERR_ALLOC, RSFD_ERR_CUDA, RSFD_ERR_NOT_CONVERGED, RSFD_ERR_BREAKDOWN,
    RSFD_ERR_TIMEOUT, RSFD_ERR_UNSUPPORTED, RSFD_FP64, RSFD_MIXED, RSFD_DF64, RSFD_SEED_MID, RSFD_SEED_FIRST, RSFD_SEED_INDEX, RSFD_SEED_AUX,
    RSFD_PASS_AUTO, RSFD_PASS_RECOMPUTE, RSFD_PASS_STORED, RSFD_PASS_SPLIT, RSFD_PASS_SPLIT_BFP, RSFD_DYSON_AUTO, RSFD_DYSON_FP64, RSFD_DYSON_TC,
    RsfdError, lib_path, load_library,
    rsfd_create, rsfd_boundary_rows, rsfd_set_tracked_planes, rsfd_tracked_rows, rsfd_dyson_tracked,
    rsfd_set_solve_options, rsfd_shifted_cocg, rsfd_get_stats, rsfd_autotune, rsfd_shifted_cocg_regions, rsfd_shifted_cocg_sweep, rsfd_sweep_load_energies,
    rsfd_dyson_boundary, rsfd_dyson_boundary_noalloc, rsfd_cgemm_tf32x3, rsfd_transmission, rsfd_lead_sigma_uniform, rsfd_lead_sigma_decimation, rsfd_last_error, rsfd_destroy,
    Handle,
)
