"""GB300-native recursive Green's function (RGF) transport for armchair graphene nanoribbons.

The compute path is the CUDA library ``librgf.so`` (C ABI in ``include/rgf.h``),
built in-tree for sm_103a by ``paper_1107_5300_gb300.build``.  ``rgf`` is its
thin Python binding (argument marshalling only); importing it fails loudly if
the library has not been built.
"""

__all__ = ["rgf"]
