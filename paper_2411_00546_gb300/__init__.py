"""GB300-native (sm_103a) solver for the RAS / RASPEN hot path of arXiv 2411.00546.

The CUDA library `libras.so` (built from `csrc/`) holds every step of the path;
`ras.py` is the thin ctypes binding with the C-ABI's names. Importing this
package loads nothing: the library is loaded on first use of `ras`, and that
fails loudly when it has not been built.
"""
