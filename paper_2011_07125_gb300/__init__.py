"""GB300-native FermiNet VMC hot path (arXiv:2011.07125).

``synth`` holds the seeded input generators; ``binding`` wraps the C-ABI library
``libferminet.so`` built from ``csrc/`` (imported lazily so that input generation
works on machines without the CUDA build).
"""
__all__ = ["synth"]
