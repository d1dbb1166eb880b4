"""Plain, slow CPU reference ("oracle") for multi-baryon two-point correlators.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library may import, call or link
anything in this package; it exists so that tests, the smoke check and the benchmark's
CPU-baseline leg can check the CUDA path against an independent statement of the
method.  It shares no code with the CUDA path; only the seeded input generator in
``mbc_inputs`` is common to both sides.

What it computes (arXiv 2201.04269, Eq. 1 and Sec. 1, with the determinant
formulation of the Wick contractions cited there):

    C(t) = sum_x sum_{(a, a') in I} W_{a, a'} <q(a_1)...q(a_n) qbar(a'_1)...qbar(a'_n)>

with the quark-level contraction equal to a signed product of an up and a down
determinant.  Modules:

* ``dirac``      gamma matrices, C, P_+- (Sec. 1, baryon operators)
* ``operators``  Grassmann expansion of p, n, p_+-, n_+-, D_I, D_II, 3He_I, 3He_II (Eq. 2)
* ``wick``       brute-force Wick pairings, Leibniz and pivoted-LU determinants (Sec. 1)
* ``canonical``  per-flavour canonical ordering and multiplicity merging (Sec. 3)
* ``correlator`` the correlator by definition, by the canonical form, per site
* ``factor_tree`` abstract and linearised factor trees (Sec. 4, Figs. 4-5)
* ``egraph``     tensor e-graph with union-find, class map and hash-cons (Sec. 5)
* ``blocks``     hadron blocks, their momentum projection and the expanded block form of
                 the correlator (Secs. 2-3)
* ``native``     the same per-site sums written in plain C for speed (``csrc/oracle.c``)

Pins: every function is checked by ``tests/test_oracle_*.py`` against closed forms,
brute force on tiny inputs, invariants and the paper's worked examples.
"""
