"""GB300-native convergent cross mapping (CCM).

The package holds the CUDA hot path behind a C ABI (``csrc/``, built into
``libccm_gb300.so``), a thin ctypes binding (:mod:`.ccm`) and the seeded
synthetic input generators (:mod:`.inputs`).  Nothing is imported eagerly:
``import paper_1905_00565_gb300.ccm`` loads the shared library and fails
loudly if it has not been built.
"""

__all__ = ["ccm", "inputs"]
