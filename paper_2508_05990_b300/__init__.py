"""B300-native Bayer-domain block motion estimation and MV feature propagation.

The compute path is the CUDA library ``libbayer_me.so`` (sources in ``csrc/``)
behind the C ABI declared in ``include/bayer_me.h``; ``bayer_me`` is its thin
ctypes binding and ``synth`` draws the seeded synthetic inputs.  Importing the
package loads nothing; ``bayer_me`` loads the library on first use and raises
if it is missing.
"""
__all__ = ["bayer_me", "synth"]
