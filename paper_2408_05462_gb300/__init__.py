"""GB300-native topology-preserving compression and marching cubes
(arXiv 2408.05462).  The compute path is the CUDA library ``libchr.so``
behind the C-ABI declared in ``include/chr.h``; ``chr`` is its ctypes binding.
"""
