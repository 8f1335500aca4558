"""Plain, slow CPU oracle for the fast Fourier spectral linearized Boltzmann
collision operator (Yin, Cai, Wang, arXiv 2503.09580).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The product path (the CUDA library and its Python binding) never calls it and
shares no code, header, table or helper with it.

Everything here is FP64 (numpy) unless a function says otherwise, follows the
paper's steps in the paper's order, and cites the passage it implements:

* ``quadrature``  -- radial rule of Eq. (2.13) and the hemisphere rule.
* ``grid``        -- the collocation grid and cyclic multi-indices (Sec. 2.3).
* ``linearized``  -- Algorithm 1 (the M-free linearized operator L[g]).
* ``quadratic``   -- the M-point quadratic operator Q(f,f), Eq. (2.14), and its
                     bilinear form Q(f,g)+Q(g,f).
* ``moments``     -- density, velocity, temperature, stress, heat flux
                     (Sec. 2.1) and the FP64 conservation projection.
* ``direct``      -- O(J n^6) direct real-/Fourier-space sums of the same
                     discrete operators (no FFT), in plain C, for tiny grids.

Pins (tests marked ``not gpu``) tie every function to something other than
itself: closed forms, collision invariants, the Maxwell-molecule eigenvalue,
the BKW solution, quadrature exactness and brute-force sums.
"""
