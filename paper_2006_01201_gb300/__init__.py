"""GB300-native asymmetric bidirectional optical-flow blend of overlap strips.

Python face of ``libpanoflow.so`` (C ABI: ``include/pano_flow.h``); the
method is Section III-C of Meng & Liu, "High-quality Panorama Stitching based
on Asymmetric Bidirectional Optical Flow". Importing this package does not
load the library; the first call that needs it does, and fails loudly if it
has not been built.
"""
from .binding import (  # noqa: F401
    FlowContext,
    PanoError,
    Params,
    load_library,
    stage_lk,
    stage_luma,
    stage_pyr_down,
    stage_warp,
)

__all__ = ["FlowContext", "PanoError", "Params", "load_library", "stage_lk", "stage_luma",
           "stage_pyr_down", "stage_warp"]
