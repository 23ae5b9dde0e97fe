"""GB300-native differentiable 2D Gaussian surfel rasterizer (2DGS-SLAM hot path).

Importing the package loads nothing native; ``paper_2506_00970_gb300.gs2d``
binds the CUDA library and raises if it has not been built.
"""
