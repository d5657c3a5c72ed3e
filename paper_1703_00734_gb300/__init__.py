"""GB300-native BPMF Gibbs sweep with posterior propagation (Qin et al., arXiv 1703.00734).

The compute path lives in ``csrc/`` (CUDA for sm_103a behind the C ABI of ``include/bmf.h``);
``bmf`` is the thin ctypes binding.  ``synth`` produces seeded synthetic inputs.  Importing
this package does not load the CUDA library; ``bmf.load()`` does, and fails loudly when the
library has not been built.
"""
__all__ = ["bmf", "synth"]
