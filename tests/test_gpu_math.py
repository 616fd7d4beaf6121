"""The device exponential used by the generated code (table-driven, Tang's
method) against the CUDA library exp and against exact values."""
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
