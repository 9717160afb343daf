"""GB300-native ramp-preconditioned primal-dual TV reconstruction for CT
(Kudo, Yamazaki, Nemoto, Takaki, arXiv 1609.06041).

The compute path is libctpd.so (hand-written CUDA for sm_103a) behind the
C ABI of include/ctpd.h; ``ctpd`` is its thin Python binding.
"""
from .ctpd import (  # noqa: F401
    CT_BATCH_AUTO,
    CT_BATCH_POOL,
    CT_FEWVIEW,
    CT_LOWDOSE,
    CT_TAPS_HIGH_BAND,
    CT_TAPS_LOW_BAND,
    BatchedSolve,
    CTError,
    Geometry,
    PDTVParams,
    ct_backproject,
    ct_batched_options,
    ct_geometry_autotune,
    ct_geometry_create,
    ct_geometry_destroy,
    ct_geometry_get_tuning,
    ct_geometry_set_tuning,
    ct_kernel_launches,
    ct_last_error,
    ct_pdtv_solve,
    ct_pdtv_status,
    ct_pdtv_solve_batched,
    ct_pdtv_workspace_bytes,
    ct_probe_fp32_fma,
    ct_project,
    ct_project_bands,
    ct_project_bands_count,
    ct_ramp_filter,
    ct_ramp_filter_noalloc,
    ct_sym_toeplitz_eig,
    ct_ramp_filter_split,
    ct_ramp_taps,
    ct_version,
    workspace_for,
    ct_unrolled_workspace_bytes,
    ct_unrolled_forward,
    ct_unrolled_backward,
)
from .autograd import (  # noqa: F401
    Backproject,
    Project,
    UnrolledPDTV,
    UnrolledReconstructor,
    backproject,
    project,
)
