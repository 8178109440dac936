"""Plain, slow FP64 CPU oracle for the directional equispaced-interpolation FMM.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call or execute it.  It
shares no code, header, table or constant generator with the CUDA library;
the two meet only through the seeded inputs of
``paper_2202_04894_gb300.workloads``.

Every function follows a passage of the paper (arXiv 2202.04894, "A
Directional Equispaced interpolation-based Fast Multipole Method for
oscillatory kernels"), cited in its docstring by section / equation /
algorithm.  Arithmetic is float64 / complex128 throughout.

Modules
  direct      O(N^2) direct sum of Eq. (1.1) (``fmmsum``), numpy + plain C.
  tree        bounding cube, Morton order, Ncrit 2^d-tree (Sec. 4.2.1).
  directions  cube-face direction sets and the direction tree (Sec. 2.1, 4.1.2).
  dtt         MACs (Sec. 3, Eq. macdirref), dual tree traversal (Alg. 1),
              blank DTT (Alg. 2) and blank downward pass (Alg. 3).
  interp      equispaced Lagrange interpolation and the P2M / M2M / L2L / L2P
              operators (Sec. 2.2-2.3), dense and tensorised (Sec. 5.2).
  m2l         kernel samples on the difference grid, circulant embedding, DFT
              diagonalisation and Fourier-domain symmetries (Sec. 2.3, 4.3).
  fmm         the plan and the application phase, step by step.

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except where its docstring says "parity unpinned".
"""
