"""GB300-native TensorNet energy and forces (arXiv 2402.17660, TorchMD-Net 2.0).

The computation lives in the C-ABI CUDA library libtnet (include/tnet.h,
csrc/); `tnet` holds the PyTorch-facing wrapper and `synth` the seeded
synthetic workloads.
"""
__all__ = ["synth", "build", "tnet"]
