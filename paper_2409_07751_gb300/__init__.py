"""GB300-native RNS-CKKS and encrypted KAN inference (arXiv 2409.07751).

The compute path is the CUDA library `libckks_kan.so` behind the C ABI in
`include/ckks_kan.h`; `paper_2409_07751_gb300.ckks` is its ctypes binding.
Importing this package does not load the library; the binding does, and it
raises if the library is missing.
"""
