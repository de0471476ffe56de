"""CPU oracle for the batched-einsum engine -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything from this package.  The product path (the
``paper_2601_12220_b300`` package and its CUDA library) never calls into it,
and this package imports nothing from the product path.

Contents
  spec.py      independent reader of the textual batched-einsum spec
  canon.py     brute-force canonical form C_lex and isomorphism judge
               (Sec. "Isomorphic Batched Einstein Summations", Defs. of
               einsum / batched-einsum isomorphism; Sec. "A Canonical form
               for Batched Einsums", Def. of a canonicalization function)
  einsum_ref.c plain FP64 nested-loop evaluation of Eq. (1) and of the
               functional form (Def. "Functional Batched Einstein
               Summation"), plus the absolute contraction used for
               tolerances; host libm for sin / cos / exp
  evaluate.py  Python driver for einsum_ref.c (materialises each lambda
               operand over its domain, then contracts)

Parity status per function is listed in each module's header.
"""
