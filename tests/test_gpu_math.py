"""The device exponential, logarithm and reciprocal used by the generated code
(table-driven Tang-style reductions; a series-refined reciprocal) against the
CUDA library functions and exact values."""
from decimal import Decimal, getcontext

import numpy as np
import pytest
import torch

from paper_2405_05974_b300 import binding

pytestmark = pytest.mark.gpu


def ulp_err(y, ref):
    y = np.asarray(y, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(y - ref) / np.spacing(np.abs(ref))


def _inputs():
    rng = np.random.default_rng(3)
    parts = [rng.uniform(-700.0, 700.0, 400000), rng.uniform(-1.0, 1.0, 200000),
             rng.uniform(-1e-3, 1e-3, 50000), np.arange(-90000, 90000) * (np.log(2.0) / 128.0),
             (np.arange(-2000, 2000) + 0.5) * (np.log(2.0) / 128.0),
             np.array([0.0, -0.0, 1e-300, -1e-300, 707.9, -707.9, 1.0, -1.0])]
    return np.concatenate(parts)


def test_table_exp_vs_library():
    x = _inputs()
    xd = torch.from_numpy(x).cuda()
    y = binding.selftest_math(0, xd).cpu().numpy()
    ref = binding.selftest_math(1, xd).cpu().numpy()
    e = ulp_err(y, ref)
    assert np.all(np.isfinite(y))
    assert e.max() <= 2.0, (e.max(), x[np.argmax(e)])


def test_table_exp_vs_exact():
    getcontext().prec = 50
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(-700.0, 700.0, 300), rng.uniform(-2.0, 2.0, 300)])
    y = binding.selftest_math(0, torch.from_numpy(x).cuda()).cpu().numpy()
    exact = np.array([float(Decimal(float(v)).exp()) for v in x])
    assert ulp_err(y, exact).max() <= 1.5


def test_table_exp_out_of_fast_range():
    x = np.array([708.0, 709.7, 710.0, -708.0, -745.0, -746.0, -1000.0, 1000.0, np.inf, -np.inf, np.nan])
    xd = torch.from_numpy(x).cuda()
    y = binding.selftest_math(0, xd).cpu().numpy()
    ref = binding.selftest_math(1, xd).cpu().numpy()
    assert np.array_equal(np.isnan(y), np.isnan(ref))
    m = ~np.isnan(ref)
    assert np.array_equal(y[m], ref[m])


# ---------------------------------------------------------------------------
# table-driven log
# ---------------------------------------------------------------------------

def _log_inputs():
    rng = np.random.default_rng(5)
    parts = [np.exp(rng.uniform(-700.0, 700.0, 300000)), rng.uniform(200.0, 5000.0, 200000),
             1.0 + rng.uniform(-1e-2, 1e-2, 100000), 1.0 + rng.uniform(-1e-9, 1e-9, 20000),
             rng.uniform(1e-3, 1.0, 100000),
             np.ldexp(1.0, np.arange(-1020, 1020)).astype(np.float64),
             np.array([1.0, 2.0, 0.5, np.sqrt(0.5), np.nextafter(1.0, 0.0), np.nextafter(1.0, 2.0),
                       2.2250738585072014e-308, 1.7976931348623157e308])]
    return np.concatenate(parts)


def test_table_log_vs_library():
    x = _log_inputs()
    xd = torch.from_numpy(x).cuda()
    y = binding.selftest_math(2, xd).cpu().numpy()
    ref = binding.selftest_math(4, xd).cpu().numpy()
    nz = ref != 0
    assert np.all(y[~nz] == 0)
    e = ulp_err(y[nz], ref[nz])
    assert e.max() <= 2.0, (e.max(), x[nz][np.argmax(e)])


def test_table_log_vs_exact():
    getcontext().prec = 50
    rng = np.random.default_rng(6)
    x = np.concatenate([np.exp(rng.uniform(-700.0, 700.0, 300)), rng.uniform(250.0, 4000.0, 300),
                        1.0 + rng.uniform(-1e-3, 1e-3, 300)])
    y = binding.selftest_math(2, torch.from_numpy(x).cuda()).cpu().numpy()
    exact = np.array([float(Decimal(float(v)).ln()) for v in x])
    assert ulp_err(y, exact).max() <= 1.5


def test_table_log_special_arguments():
    x = np.array([0.0, -0.0, -1.0, 5e-324, 1e-310, np.inf, -np.inf, np.nan])
    xd = torch.from_numpy(x).cuda()
    y = binding.selftest_math(2, xd).cpu().numpy()
    ref = binding.selftest_math(4, xd).cpu().numpy()
    assert np.array_equal(np.isnan(y), np.isnan(ref))
    m = ~np.isnan(ref)
    assert np.array_equal(y[m], ref[m])


# ---------------------------------------------------------------------------
# series-refined reciprocal
# ---------------------------------------------------------------------------

def test_rcp_vs_exact():
    # numpy's 1/x is the correctly rounded reciprocal: the exact value to 1/2 ulp
    rng = np.random.default_rng(7)
    x = np.concatenate([np.ldexp(rng.uniform(1.0, 2.0, 400000), rng.integers(-1020, 1020, 400000)),
                        -np.ldexp(rng.uniform(1.0, 2.0, 100000), rng.integers(-1020, 1020, 100000)),
                        rng.uniform(200.0, 5000.0, 100000), 1.0 + rng.uniform(-1e-9, 1e-9, 20000),
                        np.ldexp(1.0, np.arange(-1022, 1021)).astype(np.float64),
                        np.array([1.0, 3.0, 7.0, np.nextafter(1.0, 2.0), np.nextafter(2.0, 0.0)])])
    y = binding.selftest_math(3, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = 1.0 / x
    e = ulp_err(y, ref)
    assert e.max() <= 1.0, (e.max(), x[np.argmax(e)])
    assert np.mean(y == ref) > 0.99        # nearly always the correctly rounded value
    lib = binding.selftest_math(5, torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(lib, ref)


def test_rcp_special_arguments():
    x = np.array([0.0, -0.0, 5e-324, -1e-310, 2.2250738585072014e-308, 2.0 ** 1021, -(2.0 ** 1022),
                  1.7976931348623157e308, np.inf, -np.inf, np.nan])
    xd = torch.from_numpy(x).cuda()
    y = binding.selftest_math(3, xd).cpu().numpy()
    ref = binding.selftest_math(5, xd).cpu().numpy()
    assert np.array_equal(np.isnan(y), np.isnan(ref))
    m = ~np.isnan(ref)
    assert np.array_equal(y[m], ref[m])
    assert np.array_equal(np.signbit(y[m]), np.signbit(ref[m]))
