"""GB300 (sm_103a) implementation of ADOP's differentiable one-pixel point
rasterizer (Rueckert et al., arXiv 2110.06635, Sec. 3.1).

The compute path is the CUDA library ``libadop.so`` behind the C ABI of
``include/adop.h``; this package is its build step and a thin ctypes binding
(``_abi``) with the same entry-point names.  There is no CPU fallback.
"""
from ._build import build  # noqa: F401
from ._abi import (  # noqa: F401
    ADOP_BF16, ADOP_F16, ADOP_F32, ADOP_FLAG_DISCARD, ADOP_FLAG_EPILOGUE, ADOP_FLAG_GRAD_ALL_PROJECTED, ADOP_FLAG_GRAD_ASSIGN, ADOP_FLAG_LEAKY_CRF, ADOP_FLAG_LOG_DESCRIPTORS,
    ADOP_FLAG_NORMAL_CULL, ADOP_MAX_CAMERAS, ADOP_MAX_LEVELS, SIGNATURES, AdopError, Frame, Params, Points,
    adop_abi_version, adop_atomic_probe, adop_env_backward, adop_last_error, adop_photometric_backward, adop_point_radius, adop_profile_collect, adop_profile_enable, adop_render_backward, adop_render_backward_noalloc, adop_render_forward, adop_workspace_bytes,
    Server, alloc_workspace, camera_struct, lib_path, load, output_numel, pyramid_offsets, split_output)
