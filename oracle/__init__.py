"""CPU oracle for black-and-white connected component analysis.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it; the product path never imports it. It shares no code
with the CUDA library.

Modules:
  oracle.reference   plain C flood fill (ccl_oracle.c) behind ctypes; the
                     definition the GPU path is held to, bit for bit.
  oracle.twin        the same definition written again in pure Python with a
                     different traversal (pixel union-find), for tiny images.
  oracle.paper_lsl   Algorithms 1-3 of the paper restated step by step
                     (segments, B&W unification, B&W transitive closure),
                     used to pin the definition to the paper's own method.
  oracle.checks      independent properties: Euler number by bit-quads,
                     surround test by barrier search, brute-force hole fill.
"""
