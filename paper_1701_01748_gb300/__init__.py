"""GB300-native preconditioned primal-dual (PPD) radio-interferometric imaging.

The compute path is the CUDA library ``libppd.so`` (C ABI in
``include/ppd.h``); ``ppd`` is its Python binding, ``torch_ops`` wraps the
measurement operator for autograd and ``synth`` makes seeded test problems.
"""
__all__ = ["ppd", "torch_ops", "synth", "build"]
