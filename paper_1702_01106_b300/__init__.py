"""B300-native implicit EMHD zone step (grim, Chandra, Foucart & Gammie 2017).

The compute path is the C-ABI library libgrim.so (hand-written sm_103a CUDA
kernels); `grim` below is its thin ctypes binding.  Importing this package
does not load the library; the first call into `grim` does, and fails loudly
if the library is missing.
"""
