"""GB300-native composite-polynomial projection onto the PSD cone.

The compute path is the CUDA library ``libpsdproj.so`` (built from
``csrc/`` for sm_103a) behind the C ABI declared in ``include/psdproj.h``;
``binding`` is a thin ctypes layer with the same names.  Importing this
package loads nothing: the library is opened on the first call, and a
missing or unbuilt library raises instead of falling back to anything else.
"""
__all__ = ["binding", "synth"]
