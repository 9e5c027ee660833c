"""FP64 CPU oracle for the LDG diffusion operator of FESTUNG Part I (arXiv:1408.3877).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) may import, call or link anything in this package.  Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.

The oracle is a plain, slow, obviously-correct restatement of the paper:

* ``basis``       orthonormal modal basis on the reference triangle (Sec. 2.4.1)
* ``quadrature``  triangle and Gauss rules (Sec. 3.3, routines quadRule1D/2D)
* ``grid``        grid lists of Tab. 1 (routine generateGridData, Sec. 3.1)
* ``reference``   reference-element integrals M^, H^, G^, S^, R^ (Sec. 3.6)
* ``assemble``    global block matrices and right-hand sides (Sec. 2.4.3-2.4.4, 3.6)
* ``solve``       the implicit-Euler system (Sec. 2.5), its elimination of z,
                  the stationary problem (Sec. 3.9) and the sparse direct solve
* ``project``     L2 projection (Sec. 3.4) and the discretisation error (Sec. 3.5)

Every floating-point computation is FP64.  Parity status of each function is
stated in its docstring; all functions are pinned by ``tests/test_oracle_*.py``.
"""
