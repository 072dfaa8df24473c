"""Plain, slow CPU FP64 oracle for the butterfly-accelerated VIE method.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this package.  The CUDA library
never calls it and shares no code, tables or helpers with it; both sides
read only the seeded inputs of the ``workloads`` module.

Contents (each function cites the passage of the paper it follows):
  mesh        voxel -> Kuhn tetrahedra, faces, SWG support data (Sec. II, Eq. 3)
  quadrature  Gauss rules on tetrahedra and triangles (reading of the silent
              quadrature choice, see ``entries``)
  entries     Galerkin SWG entries Z(m, n) and V(m) (Eqs. 1-5), dense blocks
  dense       dense solve, far field and RCS
  mie         Mie series for a homogeneous sphere (exact reference RCS)
  hodbf       cluster tree, interpolative decomposition, butterfly (Eqs. 7-10),
              HOD-BF apply and a dense-defined HOD-BF inverse (Algorithm 1)
  gmres       restarted right-preconditioned GMRES

Parity pins (what fixes each part independently of itself) live in
``tests/test_oracle_*.py``.  Parts without such a pin say "parity unpinned".
"""
