"""GB300-native HENN: Hierarchical epsilon-Net Navigation graph (arXiv 2505.17368).

The index build (eps-net layers, navigable graphs) and the batched query
run in CUDA kernels for sm_103a behind the C ABI of include/henn.h; this
package is the Python binding.  `build()` compiles the library in tree.
"""
from .binding import (  # noqa: F401
    ANGULAR, BF16, F32, FP8E4M3, GRAPH_KNN, GRAPH_NSW, L2, SAMPLER_HALVING, SAMPLER_SAMPLING, TILES_AUTO, TILES_SIMT,
    TILES_TCGEN05, EXACT_SORT, EXACT_TILES, EXACT_SCAN,
    HennError, Index, Server, exact_knn, load, quantize_rows,
)


def build(force: bool = False) -> str:
    from .build import build as _build

    return _build(force=force)
