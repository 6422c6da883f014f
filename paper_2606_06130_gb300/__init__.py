"""GB300-native per-ping coherent echo formation for volumetric 3D sonar.

The compute path is the C-ABI library ``libsonar.so`` (hand-written sm_103a CUDA);
``paper_2606_06130_gb300.sonar`` is its thin ctypes binding. Importing this package
loads nothing; the library is loaded on first use and fails loudly when missing.
"""
__all__ = ["sonar", "inputs"]
