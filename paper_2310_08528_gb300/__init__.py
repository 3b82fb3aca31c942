"""GB300-native per-frame render path of 4D Gaussian Splatting (arXiv 2310.08528).

The CUDA library (``libfs4d.so``) is loaded lazily by :mod:`.fs4d`, so that the
input generator (:mod:`.scenegen`) can be imported on machines without a GPU.
"""
__all__ = ["scenegen", "fs4d"]
