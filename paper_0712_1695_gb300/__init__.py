"""GB300-native Biot-Savart velocity on tetrahedral meshes (ray-traced near field, Gauss far field).

The compute path is libbs.so (hand-written sm_103a CUDA behind the C ABI of
include/bs.h); ``binding`` is the Python view of that ABI.
"""
from .binding import (  # noqa: F401
    BS_FP32,
    BS_FP64,
    BS_NEAR_EXACT,
    BS_NEAR_RAY,
    INF,
    Batch,
    BSError,
    Mesh,
    bs_create,
    bs_direction_table,
    bs_num_variants,
    bs_variant_shape,
    bs_tet_rule,
    load,
)
from .build import build  # noqa: F401
