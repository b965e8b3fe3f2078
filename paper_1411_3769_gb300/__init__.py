"""GB300 (sm_103a) Polya/SDP robust-stability library.

The compute path lives in the C-ABI shared library ``lib/libpolya_sdp.so``
(sources in ``csrc/``, declarations in ``include/polya_sdp.h``); ``binding``
is its thin ctypes binding and ``build`` compiles it.  ``synth`` draws the
seeded synthetic systems.  Importing the package loads nothing: the library is
opened on first use and its absence is an error, never a fallback.
"""

__all__ = ["binding", "build", "synth"]
