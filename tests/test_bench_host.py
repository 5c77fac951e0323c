"""Host logic of bench.py that needs no GPU: the equal-error comparison of the
work-against-accuracy study (log eta linear in log error between bracketing runs)."""

import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _first_order_runs(c_err=0.16, c_eta=640.0, n=6):
    # error = c_err dt and eta = c_eta dt: a first-order method whose cost grows like 1/dt
    runs = []
    for r in range(n):
        dt = 2.0 ** -r
        runs.append({"dt": dt, "rel_err": c_err * dt, "eta": c_eta * dt})
    return runs


def test_interpolation_is_exact_for_a_power_law():
    runs = _first_order_runs()
    # eta = (c_eta / c_err) err on every run, so also between them
    for err in (0.15, 0.05, 0.0123, 0.006):
        got = bench._eta_at_error(runs, err)
        assert got["eta"] == pytest.approx(640.0 / 0.16 * err, rel=1e-12)
        assert not got["extrapolated"]
        lo, hi = got["between_dt"]
        assert 0.16 * hi <= err <= 0.16 * lo


def test_error_on_a_run_gives_that_run():
    runs = _first_order_runs()
    got = bench._eta_at_error(runs, runs[3]["rel_err"])
    assert got["eta"] == pytest.approx(runs[3]["eta"], rel=1e-12)


def test_below_every_run_is_extrapolated_from_the_last_two():
    runs = _first_order_runs()
    runs[-1]["eta"] *= 0.9  # the last pair sets the slope
    err = runs[-1]["rel_err"] / 8.0
    got = bench._eta_at_error(runs, err)
    assert got["extrapolated"]
    assert got["between_dt"] == [runs[-2]["dt"], runs[-1]["dt"]]
    e = np.log([runs[-2]["rel_err"], runs[-1]["rel_err"]])
    eta = np.log([runs[-2]["eta"], runs[-1]["eta"]])
    slope = (eta[1] - eta[0]) / (e[1] - e[0])
    assert got["eta"] == pytest.approx(np.exp(eta[1] + slope * (np.log(err) - e[1])), rel=1e-12)
