"""CPU checks of the closed forms bench.py uses to report accuracy: the
amplitude of the PDE solution (Eqs. 3-4) and the semi-discrete decay rates of
the wide and compact stencils on the (1,1,1) sine mode."""
import math

import numpy as np

import bench
from paper_1307_7867_gb300 import inputs
from tests import independent as ind


def test_analytic_amplitude_matches_independent_form():
    for t in (0.0, 0.1, 1.0, 6.0):
        for lam in (None, -2.9, -0.5):
            lam_ind = -3 * 0.1 * math.pi**2 if lam is None else lam
            a = bench.analytic_amplitude(t, lam=lam)
            b = ind.semidiscrete_amplitude(lam_ind, t, 0.1, 1.0)
            assert abs(a - b) <= 1e-14 * max(1.0, abs(b))


def test_semidiscrete_rates_are_the_stencil_symbols(oracle):
    """nu times the symbol on the (1,1,1) mode, checked by applying the oracle's
    operators to the mode (compact: L Phi = lam_L Phi, W Phi = lam_W Phi)."""
    N = 15
    phi = inputs.sine_mode(N)
    lap_w = oracle.laplacian(phi, 4)
    lam_w = float(np.sum(lap_w * phi) / np.sum(phi * phi))
    assert abs(bench.wide_lambda(N) - 0.1 * lam_w) <= 1e-12 * abs(lam_w)
    lam_l = float(np.sum(oracle.laplacian(phi, oracle.COMPACT) * phi) / np.sum(phi * phi))
    lam_m = float(np.sum(oracle.weight(phi, oracle.COMPACT) * phi) / np.sum(phi * phi))
    assert abs(bench.compact_lambda(N) - 0.1 * lam_l / lam_m) <= 1e-12 * abs(lam_l / lam_m)


def test_workload_config_keys():
    cfg = bench.workload_config(bench.WORKLOADS["c2"], 1)
    assert cfg["N_fine"] == 255 and cfg["interp"] == 2 and cfg["mg_rel"] == 0.0
    assert cfg["parallelism"] == "single GPU"
    assert bench.workload_config(bench.WORKLOADS["c2"], 4)["parallelism"] == "replicas x4"


def test_workload_config_names_the_solve_path_and_l2_regime():
    """The persistent solve kernel's setting and whether the working set fits
    in L2 are stated in the JSON line's config."""
    c1 = bench.workload_config(bench.WORKLOADS["c1"], 1)
    c2 = bench.workload_config(bench.WORKLOADS["c2"], 1)
    assert c1["persistent_solves"] == "N <= 31" and c2["persistent_solves"] == "N <= 31"
    assert "fits in L2" in c1["l2"] and "no flush needed" in c2["l2"]
    off = bench.workload_config(dict(bench.WORKLOADS["c1"], persistent=0), 1)
    assert off["persistent_solves"] == "off"
