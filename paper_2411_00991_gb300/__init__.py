"""GB300-native posterior-sampling sweep of Bayesian deconvolution
(arXiv 2411.00991).  ``bdecon`` is the ctypes binding of the C-ABI CUDA
library (libbdecon.so, built in-tree by ``build``); ``synth`` draws seeded
synthetic inputs."""
__all__ = ["bdecon", "build", "synth"]
