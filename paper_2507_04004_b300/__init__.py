"""B300-native differentiable tile-based 3D Gaussian splatting rasterizer
(the mapping/tracking hot path of Gaussian-LIC2, arxiv 2507.04004).

``synth`` draws seeded synthetic inputs; ``raster`` (imported lazily) holds
the PyTorch face of the CUDA library ``libgsb300.so``.
"""

__all__ = ["raster", "synth", "build"]


def __getattr__(name):
    if name == "raster":
        from . import raster
        return raster
    raise AttributeError(name)
