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


def test_oracle_sample_runs_the_predictor_interval():
    # the bounded CPU sample of the largest workload, here on the 1,876-DOF machine: Algorithm 1
    # on the first interval of positive length, cut after the given number of substeps
    res = bench._oracle_finish(bench._oracle_sample(0, substeps=3, reps=2, warmup=1))
    assert len(res["seconds"]) == 2 and all(t > 0 for t in res["seconds"])
    assert res["substeps"] == 3 and res["n"] == 1876
    assert res["interval"] == 2  # Lobatto: the first interval has zero length


def test_traffic_comes_from_a_profile_of_the_current_kernel(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1707_03581_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "kernels.cu").write_text("// kernel source\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench._kernels_sha()
    (tmp_path / "profiles" / "k_a.md").write_text(
        f"# summary\nbench-traffic: kernel=k_a n_dof=100 dram_bytes=1234.5 kernels_cu_sha256={sha}\n")
    (tmp_path / "profiles" / "k_b.md").write_text(
        "bench-traffic: kernel=k_b n_dof=100 dram_bytes=99 kernels_cu_sha256=0000000000000000\n")
    assert bench._profile_traffic("k_a", 100)[0] == 1234.5
    assert bench._profile_traffic("k_a", 101)[0] is None
    t, note = bench._profile_traffic("k_b", 100)
    assert t is None and "changed" in note


class _FakeSolver:
    def __init__(self, n, nnz, bits, implied):
        self.n, self.nnz, self._bits, self._implied = n, nnz, bits, implied

    def matrix_columns(self):
        return self._bits

    def matrix_implied(self):
        return self._implied


@pytest.mark.parametrize("bits,implied,per_nnz,slices", [(16, True, 4, True), (16, False, 6, True),
                                                          (32, False, 8, False)])
def test_spmv_bytes_follow_the_matrix_form(bits, implied, per_nnz, slices):
    # the FP32 SpMV's algorithmic bytes: the value (4 B) and the stored column of every nonzero
    # (none when implied, 2 B offset, 4 B column), 16 B a row, 4 B a 32-row slice (its base
    # or its table position; none with 32-bit columns)
    n, nnz = 1000, 27000
    s = _FakeSolver(n, nnz, bits, implied)
    kt = {"k_mx_spmv": (10, 1.0), "k_mx_update": (10, 0.5)}
    reps = [{"cg_iters_total": 8, "refinements_total": 2, "n_solves": 2}]
    name, upd, _, sp_bytes, up_bytes, work, _, _, note = bench._dominant_kernel(s, "mixed", kt, reps)
    assert name == "k_mx_spmv" and upd == "k_mx_update"
    assert sp_bytes == per_nnz * nnz + 16 * n + (4 * 32 if slices else 0)  # 32 slices of 32 rows
    assert up_bytes == 48 * n and work == 10
    assert note.startswith(f"{per_nnz} B/nnz")
    # the FP64 path reads the FP64 values with the stored columns whatever the FP32 copy's form
    name, _, _, sp64, _, work64, _, _, _ = bench._dominant_kernel(s, "fp64", {}, reps)
    assert name == "k_cg_spmv" and work64 == 10
    assert sp64 == (8 + bits // 8) * nnz + 32 * n + (4 * 32 if bits == 16 else 0)


def test_oracle_pool_runs_one_process_per_machine():
    # the CPU baseline of the batch and serving workloads: one spawned oracle process per
    # machine, one macro step each, started together (two small machines of the batch here)
    cb = bench._oracle_pool(3, [6, 8])
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["unit"] == bench.UNIT
    assert cb["value"] > 0 and "12902-41336 DOF" in cb["sample"]
    assert cb["host_cpu"]["logical_cores"] == os.cpu_count()
