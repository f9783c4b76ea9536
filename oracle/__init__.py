"""CPU FP64 oracle for the directional fast multipole matvec.

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library and its Python
binding) never imports, calls or links anything here; only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline / reference leg do.  The
oracle shares no code with the CUDA path: it is written independently from the
paper (arXiv:1311.4257) in plain numpy, FP64 throughout.
"""
