"""GB300-native (sm_103a) hot path of DIGS dynamic cone-beam CT reconstruction (arXiv 2506.22280).

The compute path is the CUDA library ``libdigs.so`` behind the C-ABI in ``include/digs.h``;
``paper_2506_22280_gb300.digs`` is its thin ctypes binding (tensor marshalling only, no CPU fallback).
"""
from .digs import (  # noqa: F401
    DigsError,
    DigsRender,
    Projector,
    Reconstruction,
    WeightPredictor,
    Workspace,
    adam_config,
    exported_symbols,
    ffd_eval,
    lib,
    sync_status,
    workspace_size,
)
