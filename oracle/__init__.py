"""FP64 CPU oracle for the first-order bilevel topology optimiser (TEST INFRASTRUCTURE).

This package is the slow, plain statement of what the GPU path computes.  It
exists only to check that path: ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it; the
library itself never imports, links or runs anything from here.  It shares no
code with the CUDA sources (no kernels, headers, tables or constant
generators); the only common module is ``workloads`` (seeded inputs, no
arithmetic of the method).

Everything is numpy / scipy in float64.  Each function names the passage of the
paper it restates (section, equation or algorithm of arXiv 2204.06204):

* ``fem``      -- Sec. III: potential energy, element stiffness K_e, assembled
                  K(v), fixtures and loads; the power-law (SIMP) parameterisation.
* ``filt``     -- Remark 3.1 (material filtering): a linear cone density filter
                  and its transpose (chain rule).
* ``sens``     -- Sec. III, exact gradient -1/2 u^T dK/dv u (here for
                  J = f^T u = 2 l, so twice the paper's value).
* ``project``  -- Sec. IV-B, Eq. (piecewiseLinearEQ) and Algorithm 4 (sorted
                  breakpoints, running SLOPE / RHS).
* ``solve``    -- Algorithm 1 / 3 lower-level steps, exact solves for the nested
                  method (PGD, Sec. V), and the multigrid V-cycle used as M.
* ``outer``    -- Algorithms 1 and 3 (FBTO / CPFBTO outer loop) and PGD.
* ``adjoint``  -- reverse mode of a truncated lower-level solve.

Pins (``tests/test_oracle_*.py``, run with ``-m "not gpu"``) tie each part to
something other than itself: the closed-form element matrix, rigid-body null
space, the patch test, beam theory, finite differences, KKT conditions and
brute force for the projection, the Galerkin identity for the multigrid
transfer, and the nested-exact limit of the bilevel loop.

Parity unpinned: the paper prints no 3-D trajectory, so the outer loop's
iterates on the measured workloads are pinned only through their parts and
the nested-exact limit, not to printed values.
"""
