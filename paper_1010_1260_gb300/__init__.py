"""GB300-native inverse spherical harmonic transform (alm2map) and its adjoint.

Nothing heavy happens at import time: the CUDA library is loaded by
``paper_1010_1260_gb300.sht`` on first use.
"""
