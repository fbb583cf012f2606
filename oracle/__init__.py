"""Exact CPU oracle for the resultant / gcd path (TEST INFRASTRUCTURE ONLY).

This package is the slow, plainly written reference that the CUDA path is checked
against.  It uses Python's arbitrary-precision integers and ``fractions.Fraction`` and
follows the definitions of the paper directly:

* ``sylvester``  -- the Sylvester matrix of Sec. 2 ("Resultants") and three determinant
  routines (Leibniz expansion, fraction-free Bareiss elimination, Gaussian elimination
  over Z_p);
* ``resultant``  -- res(f, g; y) and res(f, g; x) in Z[x] as that determinant, the
  per-(prime, point) values of step (c) of the modular algorithm (Sec. 5.1), the
  Hadamard-type coefficient bound and the plan (degree bound, prime count);
* ``gcd``        -- gcd in Z_p[x] (Euclid, and the Sylvester-echelon route of the
  theorem in Sec. 5.1), gcd in Z[x], Yun's square-free factorisation (Sec. 2.1) and the
  square-free part;
* ``numtheory``  -- Miller-Rabin, the table of transform-friendly 31-bit primes,
  primitive roots;
* ``subresultant`` -- principal subresultant coefficients (Sec. 3.3), exact and modulo
  a prime, the fiber counts N, N^- and N^+, the bivariate gcd and Teissier's Q, and the
  split of R* by the multiplicity of Q at its roots; ``gcd`` also holds the content of
  a bivariate polynomial with respect to one variable (Sec. 4).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import anything from here.  The product path (``paper_1201_1548_gb300``) never
does, and this package never imports the product path: the two share no code.

Parity status: every public function is pinned by ``tests/test_oracle_*.py`` against
brute force, closed forms or algebraic identities; none is marked "parity unpinned".
"""
