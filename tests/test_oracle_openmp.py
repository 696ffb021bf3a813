"""The OpenMP build of the oracle (used only to time the CPU baseline on all
host cores) gives bitwise the results of the single-thread parity oracle: each
point is computed by the same expression, only the loop over points is split."""
import os

import numpy as np

from paper_1307_7867_gb300 import inputs


def test_openmp_build_is_bitwise_the_serial_oracle(oracle):
    os.environ.setdefault("OMP_NUM_THREADS", "4")
    fine, coarse = (15, 4, 5), (7, 2, 3)
    u0 = inputs.smooth_random_field(15, seed=3, kmax=4)
    runs = []
    for omp in (False, True):
        prob = oracle.Prob(nu=0.1, forcing=1, kappa=1.0, mg_tol=1e-11, mg_max=100, interp=8)
        if omp:
            with oracle.openmp():
                a = oracle.mlsdc_run(fine, coarse, prob, 1 / 16, 2, u0, max_iters=3, tol=-1.0)
                b = oracle.pfasst_run(fine, coarse, prob, 1 / 16, 4, 4, u0, max_iters=2)
                c = oracle.laplacian(u0, oracle.COMPACT)
        else:
            a = oracle.mlsdc_run(fine, coarse, prob, 1 / 16, 2, u0, max_iters=3, tol=-1.0)
            b = oracle.pfasst_run(fine, coarse, prob, 1 / 16, 4, 4, u0, max_iters=2)
            c = oracle.laplacian(u0, oracle.COMPACT)
        runs.append((a, b, c))
    (a0, b0, c0), (a1, b1, c1) = runs
    assert np.array_equal(a0[0], a1[0]) and a0[2]["vcycles"] == a1[2]["vcycles"]
    assert np.array_equal(b0[2]["slice_nodes"], b1[2]["slice_nodes"])
    assert np.array_equal(c0, c1)
