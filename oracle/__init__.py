"""Plain FP64 CPU oracle for the energy-based DG / Galerkin-difference method.

TEST INFRASTRUCTURE ONLY.  Nothing in the library path may import, call or
link this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA path (its own basis, quadrature, assembly,
eigen-solves, fluxes and time stepping, written from the paper's
definitions in numpy FP64).

Modules
-------
gd_basis   1-D GD basis with the extrapolation boundary basis (Section 2.1,
           Eq. GD_basis_lagrange, Section 2.1.1), 1-D mass/stiffness by
           Gauss quadrature (Section 3.1), simultaneous diagonalisation
           (Section 3.2).
dg_const   Energy-DG semi-discretisation on Cartesian constant-coefficient
           meshes in nodal form (Eqs. DG1, DG2, DG1_extra and the fluxes of
           Section 2.2.1), with dense element solves.
dg_var     Variable c^2 and mapped elements (Section 7.1): quadrature
           assembly, face fluxes by quadrature, dense solves and PCG with
           IC(0) (the paper's preconditioner) or a frozen-coefficient
           diagonalisation preconditioner.
timeint    Classic RK4 (Sections 3.3, 6), discrete energy, L2 / energy-norm
           errors (Section 6).

Parity status: every function is pinned by the not-gpu tests in
``tests/test_oracle_*.py`` (worked example of Section 2.1.1, polynomial
reproduction, matrix structure, energy identities, brute-force dense
operators, convergence on exact solutions).  Nothing here is "parity
unpinned".
"""
