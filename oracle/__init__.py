"""Plain, slow, FP64 CPU oracle for the RAS / RASPEN method of
Ciaramella, Kartmann & Mueller, "Solving semi-linear elliptic optimal control
problems with L1-cost via regularization and RAS-preconditioned Newton methods"
(arXiv 2411.00546).

THIS PACKAGE IS TEST INFRASTRUCTURE. It exists only to check the CUDA library
(`paper_2411_00546_gb300`) against the paper. Only `tests/`,
`__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference` legs of
`bench.py` may import it. The product path never calls it and has no CPU
fallback. It shares no code with the CUDA path: the two meet only in the seeded
input generator (`paper_2411_00546_gb300.inputs`), which holds none of the
method's arithmetic.

Every routine follows the paper's definitions in its own order and notation:

* pointwise.py      smoothed projection P_eps, P_eps' (Sec. 3.1, Lemma 5), phi
* discretization.py 5-point finite-difference A_h, residual F_eps and its
                    Jacobian (Sec. 3.3 and the model problem of Sec. 4)
* decomposition.py  non-overlapping blocks, overlapping subdomains, R_i, P_i,
                    restricted prolongation (Sec. 4.2)
* newton.py         damped Newton with eps-continuation and relaxed backtracking
                    (Alg. 1)
* gmres.py          restarted GMRES with classical Gram-Schmidt applied twice
* ras.py            local corrections C_i (Sec. 4.2), the RASPEN function
                    (Alg. 3), its Jacobian action (Alg. 4), linear RAS
* solvers.py        RASPEN (Alg. 2), Newton_RAS (Alg. 1 + linear RAS GMRES),
                    dense brute-force Newton and sparse monolithic Newton

Pins (what ties each routine to something other than itself) are in
`tests/test_oracle_*.py`. Functions without such a pin say "parity unpinned".
"""
