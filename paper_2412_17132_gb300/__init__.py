"""GB300-native GW+C core-level satellite engine (arXiv 2412.17132 hot path).

The compute path is the C-ABI library ``libgwc.so`` (hand-written CUDA for sm_103a);
``paper_2412_17132_gb300.gwc`` is its thin ctypes binding and ``synth`` the seeded
synthetic input generator.
"""
