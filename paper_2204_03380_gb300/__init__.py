"""GB300-native (sm_103a) seismic modeling and reverse time migration with
random boundary conditions (Barbosa & Coutinho, arXiv:2204.03380).

The compute path is the C-ABI library ``librbc`` (include/rbc.h), hand-written
CUDA kernels for sm_103a; this package only binds it.  PyTorch provides device
memory and streams.
"""
from ._native import (  # noqa: F401
    RBC_REINJECT_SOURCE, RBC_ZERO_FIRST, RBCError, make_grid, rbc_build_velocity, rbc_create, rbc_destroy,
    rbc_fwi_backward, rbc_fwi_forward, rbc_batch_create, rbc_batch_destroy, rbc_batch_rtm, rbc_batch_info,
    rbc_batch_timing, rbc_cnn_param_count, rbc_cnn_workspace_bytes, rbc_cnn_forward, rbc_cnn_infer, rbc_cnn_backward,
    rbc_cnn_mse, rbc_cnn_adam, rbc_inject_fault,
    rbc_get_panels, rbc_grid, rbc_image_stack, rbc_last_error, rbc_launch_count, rbc_model, rbc_model_static,
    rbc_phase_timing, rbc_rtm_shot, rbc_set_coef, rbc_set_snapshots, rbc_nyquist_stride, rbc_storage_bytes, rbc_rtm_storage,
    LIB_PATH, EXPORTED,
)
