"""GB300-native Difference Potentials Method hot path (arXiv:1811.03557).

The compute path is the CUDA library ``libdpm.so`` (C ABI, ``include/dpm.h``);
``paper_1811_03557_gb300.abi`` is its thin ctypes binding.
"""
