"""GB300-native (sm_103a) ILE extrinsic-marginalisation hot path (arXiv:2210.07912).

The compute path is the C-ABI library ``libile.so`` (hand-written CUDA kernels, declared in
``include/ile.h``).  ``paper_2210_07912_gb300.ile`` is its thin ctypes binding; importing the
package itself loads nothing, and every call into the binding fails loudly if the library is
missing.  ``synthetic`` draws seeded inputs and holds none of the likelihood's arithmetic.
"""
__all__ = ["ile", "synthetic"]
