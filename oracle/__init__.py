"""Oracle — test infrastructure only.

Plain, slow CPU implementations of what the GPU library computes: RNS-CKKS
arithmetic (C, `ckks_oracle.c`), the FP64 plaintext KAN (Eqs. 1-5), the
SiLU range and weighted least-squares fit (Eqs. 11-12), the comparison
composite, and the encrypted KAN layer schedule (Algorithms 1-3, BSGS).

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package. Nothing here is shared with the GPU
library, and nothing here imports it.
"""
