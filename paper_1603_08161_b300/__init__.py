"""B300-native VolumeDeform lattice solve (arXiv 1603.08161).

``paper_1603_08161_b300.vd`` is the thin ctypes binding of ``libvd.so`` (the CUDA
library in ``csrc/``); ``paper_1603_08161_b300.synth`` builds seeded synthetic inputs.
Importing the package loads neither; ``vd`` loads the library on first import and
raises if it is missing.
"""
__all__ = ["vd", "synth"]
