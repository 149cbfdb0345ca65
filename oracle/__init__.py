"""Oracle for the arc x constant-latitude intersection: TEST INFRASTRUCTURE ONLY.

This package is the slow, obviously correct CPU reference that the CUDA path is
checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or execute anything in it. The product library never routes through it,
and it shares no code with the CUDA path (no kernels, headers, helpers, tables
or pre/post-processing); neither side imports the other.

Contents
--------
``exact``      The plain definition: Eq. 2.2 evaluated in exact rational
               arithmetic (Python integers) on the FP64 inputs taken as exact
               reals, the test that a point lies between the endpoints
               decided exactly, and each coordinate correctly rounded to
               nearest-even FP64 (Sec. 1.2, Sec. 2, Sec. 3).
``steps``      The paper's algorithms executed step by step in FP64 with
               correctly rounded operations (Algorithms 1, 2, 4, 5, 6, 7 and
               8, plus the AccSqrt reading), and the direct FP64 evaluation of
               Eq. 2.2 (Sec. 4). Written in plain C (``accux_ref.c``) with libm
               ``fma``/``sqrt``, built with ``-ffp-contract=off``.
``ragged``     Brute force over every (edge, latitude) pair of a mesh batch,
               using ``exact``.
``exact_arcs`` Intersection of two great circle arcs (three cross products
               followed by a normalisation, Sec. 1): v = n_a x n_b exactly, the
               on-arc signs exactly, v / |v| correctly rounded.

Pinning
-------
``exact`` is pinned by closed forms (equator, meridian and mirror-symmetric
arcs), exact invariants, and brute-force bisection in high precision
(``tests/test_oracle_exact.py``). ``steps`` is pinned by the per-algorithm
error bounds the paper states, checked against exact rational values, and by
the final AccuX bound against ``exact`` (``tests/test_oracle_steps.py``).
"""
