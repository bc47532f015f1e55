"""CPU FP64 oracle for the non-extensive sparsification of H^2 matrices.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import anything from
this package.  The product path (the CUDA library and its Python binding)
never imports, links or executes it, and shares no code with it: the only
module both sides use is the seeded input generator
``paper_1705_04601_gb300.synth``, which holds no step of the method.

Contents, in the order of the method:

* ``h2``          -- the H^2 matrix as defined in Definition 4.9 (§4.1):
                     expanded cluster bases, dense form, matrix-vector product.
* ``householder`` -- Householder QR with square completion Q = [Q^b | Q^perp]
                     (§4.2: orthogonal completion of the cluster bases).
* ``sparsify``    -- the level-by-level construction A = U S V^T of §2.1-2.3
                     built from H^2 parameters as in §4.2-4.3, the sparse S in
                     a variable-block (VBR) layout, and the applies of U, V.
* ``factor``      -- nested-dissection ordering of S by cluster closure, the
                     symbolic elimination, a right-looking block LU with
                     partial pivoting inside each pivot block, the solve
                     S y = U^T b, x = V y of §1 (Eq. sp0), log|det A|
                     from the pivots (§5.3), and the block Cholesky of an
                     SPD S on the same supernodes.
* ``ilu``         -- the threshold incomplete LU (ILUt) of S that §5.5 uses
                     as the preconditioner, on dense arrays for small cases.
* ``iterate``     -- iterative refinement and restarted GMRES driven by the
                     H^2 matvec and preconditioned by the factored S (§5.5).

Every function states which passage of the paper it follows.  Where the paper
is silent or garbled the reading taken is written in the docstring.
"""
