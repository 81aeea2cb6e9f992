"""GB300-native (sm_103a) splatting renderer and point-to-ellipsoid
estimator of "Low Latency Point Cloud Rendering with Learned Splatting"
(arXiv 2409.16504).

The compute path lives in ``libp2e.so`` (``csrc/``, C ABI in
``include/p2e.h``); this package only marshals arguments and owns buffers.
"""
from ._lib import P2EError, load  # noqa: F401
from .render import (DEFAULT_CONFIG, Bins, GaussianSet, Images, Projected, Renderer,  # noqa: F401
                     p2e_bins_check, p2e_project, p2e_render, p2e_render_backward, p2e_sort_bin, point_raster, relight,
                     render_differentiable, total_tiles)
