"""GB300-native compression-enabled column operators (MorphStore's processing model).

The compute path is libms.so (CUDA, sm_103a) behind the C ABI in
include/morphstore.h; ``morphstore`` is its thin ctypes binding.  Importing this
package loads nothing: ``paper_2004_09350_gb300.morphstore`` loads the library on
first use and raises if it has not been built.
"""
__all__ = ["morphstore", "synth"]
