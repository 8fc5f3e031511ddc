"""Measurement probes: the Newton reciprocal of the outer residual kernels
against the device's own double division, and the FMA-rate probe that gives
the double kernels' roofline."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")


def test_newton_reciprocal_is_within_two_ulp_of_division():
    """Two Newton steps from the float reciprocal: the relative error after
    the steps is below 2^-52 plus the roundings of the last two FMAs, so the
    result lies within 2 units in the last place of the correctly rounded 1/d
    over the whole valid range [2^-126, 2^127] (log-uniform samples, the
    range ends, powers of two and the s^2 + s_sat^2 values of the workloads)."""
    rng = np.random.default_rng(0)
    d = np.concatenate([
        np.exp2(rng.uniform(-126, 127, 2_000_000)),
        np.exp2(np.arange(-126, 128, dtype=np.float64)),
        np.array([2.0 ** -126, 2.0 ** 127, 1.0, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52]),
        rng.uniform(0, 50, 100_000) ** 2 + rng.uniform(0.5, 2.0, 100_000) ** 2,
    ])
    dt = torch.tensor(d, device="cuda")
    out = torch.empty_like(dt)
    ptp.probe_recip_dev(dt, out)
    ref = 1.0 / dt                      # the device's correctly rounded division
    ulp = torch.abs(torch.nextafter(ref, torch.full_like(ref, float("inf"))) - ref)
    err_ulp = (torch.abs(out - ref) / ulp).max().item()
    assert err_ulp <= 2.0, err_ulp


def test_fma_probe_rates_are_plausible():
    """FP64 and FP32 FMA rates: positive, FP32 well above FP64, and neither
    above the unit-count bound at the maximum clock (152 SMs at 2.07 GHz:
    128 FP32 lanes per SM; 2 FP64 FMAs per clock and SM on this part)."""
    f64 = ptp.probe_fma(0, fp64=True)
    f32 = ptp.probe_fma(0, fp64=False)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 0 < f64 < f32
    assert f32 <= sms * 128 * 2 * 2.07e9 / 1e12 * 1.05
