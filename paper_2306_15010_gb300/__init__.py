"""GB300-native VQ-NNF template matching (Gupta & Sintorn, arXiv 2306.15010).

The hot path -- k-means codebook, nearest-neighbour field, integral-image filter
responses and the Eq. 2 similarity heatmap -- runs in the hand-written CUDA kernels of
``libvqnnf.so``; this package only marshals torch tensors (device memory and the current
stream) into the C ABI of ``include/vqnnf.h``.
"""
from .api import (  # noqa: F401
    vqnnf_assign,
    vqnnf_assign_noalloc,
    vqnnf_fit_codebook,
    vqnnf_filter_responses,
    vqnnf_last_device_error,
    vqnnf_match_host,
    vqnnf_match_host_workspace_bytes,
    vqnnf_score,
    vqnnf_selftest_bounded_wait,
    vqnnf_set_kernel_events,
    vqnnf_version,
    vqnnf_workspace_bytes,
    Bank,
    Workspace,
)
from ._lib import VqnnfError  # noqa: F401
from .soft import SoftHeatmap, soft_heatmap, soft_workspace_bytes  # noqa: F401
from .batch import BatchPlan, vqnnf_batch_tune, vqnnf_batch_workspace_bytes, vqnnf_match_batch  # noqa: F401
