"""Plain, slow, CPU-only FP64 oracle for the preconditioned shifted block FOM.

THIS PACKAGE IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of
``bench.py`` may import or execute anything under ``oracle/``.  The CUDA library never
calls into it, and it never calls into the CUDA library: the two share no code, tables
or constant generators.  Inputs come from seeded generators that hold none of the
method's arithmetic.

Modules
-------
cf         Caratheodory-Fejer poles/residues of e^x on (-inf, 0]  (paper Section 2)
operators  the test operators as scipy sparse matrices plus their closed-form
           eigen-decompositions (diagonal similarity + discrete sine transform)
psbfom     Algorithm 1 (SBFOM) and Algorithm 2 (PSBFOM), written step by step
           in the paper's order and notation (Sections 3 and 4)

Every function cites the passage of the paper it follows.
"""
