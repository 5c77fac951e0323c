"""The allocation-free heat ledger, sdc_heat_totals_noalloc, through the C ABI.

Some callers must not allocate device memory while they run. Examples are
a monitoring hook inside a real-time look-ahead loop, where cudaMalloc or
cudaFree would synchronise the device and stall the steps in flight, and a
process whose device memory belongs to another framework's pool. For them
the library offers one entry point whose scratch is a fixed device array.
This test checks it against the regular ledger (sdc_get_heat_totals) on two
calls in a row. The second call reuses the array the first call left behind.

Tolerance: 1e-12 relative, the bound the other heat-ledger checks use (FP64
sums over the same terms).

The file name sorts last, so a run that stops at the first failure has run
every other test before this one.
"""

import numpy as np
import pytest

from synth import machine_config

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_noalloc_heat_ledger_matches_regular_ledger_on_two_calls(torch):
    from paper_1707_03581_gb300 import Solver

    mach = machine_config(0)
    s = Solver(0)
    s.set_machine(mach)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda:0")
    for call in range(2):
        s.step(report=True)
        s.heat_totals_noalloc(s.temperature_device_ptr(), out)
        s.synchronize()
        got = out.cpu().numpy()
        ref = s.heat_totals()
        assert np.isfinite(got).all(), (call, got)
        assert abs(got[0] - ref["stored_stand"]) <= REL * abs(ref["stored_stand"]), (call, got, ref)
        assert abs(got[1] - ref["stored_stock"]) <= REL * abs(ref["stored_stock"]), (call, got, ref)
    s.close()


def test_noalloc_heat_ledger_of_another_field_matches_host_sum(torch):
    # a device field other than the step's own T, on two calls in a row: the totals
    # equal the host FP64 sums of m_i T_i over the stand rows [0, n_stand) and the
    # stock rows [n_stand, n), with the lumped mass the library assembled
    from paper_1707_03581_gb300 import Solver

    s = Solver(0)
    s.set_machine(machine_config(0))
    mass = s.system()[3]
    rng = np.random.default_rng(21)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda:0")
    for call in range(2):
        T = 20.0 + 5.0 * rng.standard_normal(s.n)
        Td = torch.from_numpy(T).to("cuda:0")
        s.heat_totals_noalloc(Td.data_ptr(), out)
        s.synchronize()
        got = out.cpu().numpy()
        ref = (float(np.sum(mass[: s.n_stand] * T[: s.n_stand])), float(np.sum(mass[s.n_stand:] * T[s.n_stand:])))
        assert abs(got[0] - ref[0]) <= REL * abs(ref[0]), (call, got, ref)
        assert abs(got[1] - ref[1]) <= REL * abs(ref[1]), (call, got, ref)
    s.close()


def test_noalloc_heat_ledger_rejects_buffers_off_the_device(torch):
    # host memory and wrong output tensors are refused before any kernel runs
    from paper_1707_03581_gb300 import SdcError, Solver

    s = Solver(0)
    s.set_machine(machine_config(0))
    out = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    T_host = torch.full((s.n,), 20.0, dtype=torch.float64)
    with pytest.raises(SdcError) as e:
        s.heat_totals_noalloc(T_host.data_ptr(), out)
    assert "SDC_ERR_ARG" in str(e.value)
    T_dev = torch.full((s.n,), 20.0, dtype=torch.float64, device="cuda:0")
    for bad in (torch.zeros(2, dtype=torch.float64), torch.zeros(2, dtype=torch.float32, device="cuda:0"),
                torch.zeros(1, dtype=torch.float64, device="cuda:0")):
        with pytest.raises(ValueError):
            s.heat_totals_noalloc(T_dev.data_ptr(), bad)
    s.close()


def test_noalloc_heat_ledger_rejects_null_buffers(torch):
    from paper_1707_03581_gb300 import SdcError, Solver

    s = Solver(0)
    s.set_machine(machine_config(0))
    out = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    with pytest.raises(SdcError):
        s.heat_totals_noalloc(0, out)
    s.close()
