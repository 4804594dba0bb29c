"""GB300-native implicit APIC-MPM surface-energy path (arXiv 2101.12408).

``scenes`` generates seeded synthetic inputs; ``mpm`` is the ctypes binding of
the CUDA library (``libmpm_gb300.so``), built by ``build.py``.
"""
