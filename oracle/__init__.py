"""FP64 CPU oracle for the matrix-free finite-element Kohn-Sham operator Y = H X.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle is written directly from the paper's definitions (Panigrahi &
Motamarri, "Matrix-free algorithms for fast ab initio calculations on
distributed CPU architectures using finite-element discretization"):

* ``basis``     -- 1D Gauss-Legendre / Gauss-Lobatto-Legendre rules and Lagrange
                   bases (Sec. 2.2, eq. FEdiscr; Sec. 3.1, eq. cellIntegrals).
* ``operator``  -- cell matrices T, L, G, K assembled by quadrature with
                   physical gradients (Sec. 2.2, eq. Hloc / eq. HlocIntegral),
                   the nonlocal projector matrices F (eq. Vnonloc) and the
                   assembled action Y = H X (eq. HX), i.e. the paper's
                   cell-matrix (CM) baseline method.
* ``chfsi``     -- the residual-based Chebyshev filter (Algorithm 4), the
                   Rayleigh-Ritz outer step (Algorithm 3) and a Lanczos
                   spectral upper bound, all in the standard form
                   D^{-1/2} H D^{-1/2} with D the GLL-lumped mass.
* ``flops``     -- the paper's operation-count model (eq. flopRealMF,
                   eq. flopComplexMF, eq. flopRealCM, eq. flopComplexCM).

It shares no code with the CUDA path.  Inputs come from ``synth`` (seeded
generators that hold none of the method's arithmetic).
"""
