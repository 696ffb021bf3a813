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


def test_stored_step_counts_come_from_the_oracle_script():
    """The reference timing's per-step counts exist for the default workload
    and are those of the oracle's own run (oracle/step_counts.py): the V-cycle
    work over N_fine^3 lies between the fine V-cycles alone and all V-cycles."""
    c2 = bench.stored_step_counts("c2")
    assert c2 is not None and c2["status"] == 0 and c2["steps"] >= 1
    fine_equiv = c2["vcycle_points_per_step"] / 255.0**3
    assert 0 < fine_equiv < c2["vcycles_per_step"]
    assert c2["iters_per_step"] >= 1
    assert bench.stored_step_counts("no-such-workload") is None


def test_reference_arm_without_counts_reports_unavailable():
    import argparse
    a = argparse.Namespace(steps=1, warmup=0)
    out = bench.run_reference(a, bench.WORKLOADS["c3"], "c3")
    assert out["impl"] == "reference" and "unavailable" in out


def test_host_info_names_threads_and_cpu():
    cores, model = bench.host_info()
    assert cores >= 1 and isinstance(model, str) and model


def test_mixed_inner_follows_the_tolerance_rule(monkeypatch):
    monkeypatch.delenv("HEAT3D_INNER", raising=False)
    assert bench.mixed_inner() == 0 and bench.mixed_inner(0.02) == 2
    monkeypatch.setenv("HEAT3D_INNER", "5")
    assert bench.mixed_inner() == 5
