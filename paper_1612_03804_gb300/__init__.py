"""GB300-native self-learning determinantal QMC (arXiv:1612.03804).

The compute path is the CUDA library under csrc/ behind the C ABI of
include/sldqmc.h; `sldqmc` is its ctypes binding and `inputs` draws seeded
synthetic field configurations.  Importing the package loads nothing.
"""
