"""CPU FP64 oracle for adaptive-multilevel BDDC (Sousedik & Mandel).

TEST INFRASTRUCTURE ONLY.  Plain NumPy/SciPy, dense per-substructure
matrices, loops over substructures and edges, written from the paper's
definitions so that a reader can check it against the text by eye:

* ``fem``       - Q1 model problem of Sec. 2, eq. (1), and plane linear
                  elasticity with bilinear elements (the problem of the
                  experiments of Sec. 5).
* ``levels``    - substructures, interface, corners / edges, stiffness
                  weights (Sec. 2, 2.1).
* ``bddc``      - coarse degrees of freedom, coarse basis, the multilevel
                  hierarchy (Sec. 2.1) and Algorithm 1 (eqs. 4-11).
* ``adaptive``  - the local generalized eigenproblems of Theorem 1, the
                  optimal augmentation of Theorem 2 and Algorithm 2 (eq. 14).
* ``pcg``       - preconditioned conjugate gradients with the Lanczos
                  condition-number estimate reported in Tables 1-7.
* ``reduced``   - level 1 reduced to the interface (the closing remark of
                  Sec. 4): PCG on the Schur complement with eqs. (6)-(9).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library; the two meet only through the seeded inputs of
``paper_0911_5730_gb300.inputs``.

Pins: every function is checked in ``tests/test_oracle_*.py`` against closed
forms, a sparse direct solve, exactness invariants and brute-force
eigenvalues; see the docstring of each test module.
"""
