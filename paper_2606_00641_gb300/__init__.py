"""GB300-native vectorial lattice Boltzmann method for MHD.

The compute path is the C-ABI library ``libvlbm.so`` (hand-written sm_103a
CUDA kernels); ``vlbm`` is its thin ctypes binding and ``fields`` the seeded
input generators.  Import ``paper_2606_00641_gb300.vlbm`` explicitly: this
package ``__init__`` loads nothing.
"""
__all__ = ["vlbm", "fields"]
