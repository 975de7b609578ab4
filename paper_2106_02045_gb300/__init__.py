"""GB300-native batched least-squares fitting of 2-D Gaussian spots with implicit
amplitudes (Leutenegger & Weber, arXiv 2106.02045).

``fitspots`` binds the CUDA library (``include/fitspots.h``); ``synth`` draws seeded
synthetic workloads; ``build`` compiles the library for sm_103a.
"""
