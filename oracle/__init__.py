"""FP64 CPU oracle for Positively Split Ewald (PSE) Brownian sampling.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
anything from this package.  The product (``paper_1611_09322_gb300``) never
imports it and shares no code with it; the only thing the two sides have in
common is the seeded workload generator (``paper_1611_09322_gb300.workloads``),
which holds none of the method's arithmetic.

Everything here is plain numpy/scipy in float64, written from the paper
(Fiore, Balboa Usabiaga, Donev & Swan, "Rapid sampling of stochastic
displacements in Brownian dynamics simulations", J. Chem. Phys. 146, 124116,
arXiv:1611.09322).  Each function cites the section / equation it restates.

Modules
-------
rpy      real-space scalar functions F, G (Appendix A), self term (eq. self),
         free-space RPY (eq. RPY_free_space), integral forms (eqs. int1/int2)
ewald    splitting function H, truncation / quadrature parameters (Sec. II C),
         dense real- and wave-space mobilities (eqs. Mreal, Mwave)
philox   Philox4x32-10 counter-based generator and Box-Muller normals
pse      real-space Lanczos sample and wave-space NUFFT sample (Sec. II B);
         Lanczos on the whole mobility (Sec. IV's comparison method)
poly     polydisperse spheres: the size-dependent shape factor of Sec. V
precond  block-diagonal preconditioner network (forward/backward in FP64)

Parity status of every function is pinned by ``tests/test_oracle_*.py``
against facts the paper and mathematics fix; functions without such a pin
say "parity unpinned" in their docstring.
"""
