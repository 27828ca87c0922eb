"""The autotuner's cost model (Section 4, eq. (cost)): t(n) = N^2 s + 4 tau / n
per sub-step, fitted to two probes. CPU only: the fit recovers s and tau from
exact model data, its ranking follows the model, and the per-node optimum of
eq. (cost), n* = (2 tau / s)^(1/3), is where the model's derivative vanishes."""
import pytest

from paper_1602_07558_gb300.autotune import fit_cost_model, predict


@pytest.mark.parametrize("s,tau", [(2e-12, 3e-6), (8e-12, 1e-7), (1e-11, 0.0)])
def test_fit_recovers_s_and_tau(s, tau):
    N2 = 4096.0 * 4096.0
    probes = [(n, predict(N2, s, tau, n)) for n in (16, 64)]
    s_fit, tau_fit = fit_cost_model(N2, probes)
    assert s_fit == pytest.approx(s, rel=1e-9)
    assert tau_fit == pytest.approx(tau, rel=1e-9, abs=1e-18)
    assert predict(N2, s_fit, tau_fit, 32) == pytest.approx(predict(N2, s, tau, 32), rel=1e-9)


def test_larger_tiles_rank_first_when_tau_is_positive():
    N2 = 1024.0 * 1024.0
    pred = {n: predict(N2, 5e-12, 2e-6, n) for n in (16, 32, 64)}
    assert sorted(pred, key=pred.get) == [64, 32, 16]


def test_per_node_optimum_of_eq_cost():
    """On one node of n x n points eq. (cost) is n^2 s + 4 tau / n; its minimum
    is at n* = (2 tau / s)^(1/3)."""
    s, tau = 0.6e-9, 150e-6            # Table 1 / Table 2 orders of magnitude
    f = lambda n: n * n * s + 4 * tau / n
    n_star = (2 * tau / s) ** (1.0 / 3.0)
    h = 1e-3 * n_star
    assert f(n_star) < f(n_star - h) and f(n_star) < f(n_star + h)
    assert (f(n_star + h) - f(n_star - h)) / (2 * h) == pytest.approx(0.0, abs=1e-9)


def test_fit_falls_back_when_the_probes_fall_faster_than_one_over_n():
    """Probes t(16) = 10, t(64) = 1 (per sub-step) fall faster than 1/n: the
    exact fit would give s < 0; the fit keeps s = 0 and takes tau from the
    larger tile, so the model goes through that probe and ranks by 1/n."""
    N2 = 1.0e6
    s_fit, tau_fit = fit_cost_model(N2, [(16, 10.0), (64, 1.0)])
    assert s_fit == 0.0
    assert predict(N2, s_fit, tau_fit, 64) == pytest.approx(1.0)
    assert predict(N2, s_fit, tau_fit, 16) > predict(N2, s_fit, tau_fit, 32) > 1.0
