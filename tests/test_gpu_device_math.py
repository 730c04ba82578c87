"""The fit's scalar device routines against their error bounds (ksdf_device_math):

  * the kernel-entry exponential 2^(-e/2^16) (Sec. IV-B kernel matrix; a two-level table method) within
    3 units of 2^-53 relative, from a binary64 argument and from the 40-bit fixed-point one;
  * the pivot reciprocal square root of the Cholesky factorisation within 0.51 ulp (FP32 seed plus an exact
    integer second-order correction: half an ulp from the final rounding, the rest below 2^-60).

References are computed with 50-digit decimal arithmetic.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2603_29227_gb300 import ksdf  # noqa: E402

getcontext().prec = 50


@pytest.fixture(scope="module")
def h():
    import __graft_entry__

    __graft_entry__.build()
    m = ksdf.KernelSDF(dict(dim=3, origin=(0.0, 0.0, 0.0), cell=0.5, margin=0.1, n_max=64, k_cand=4,
                            **{"lambda": 300.0}))
    yield m.h  # the context lives as long as m


def _ulps(got, exact):
    ulp = Decimal(2) ** (math.frexp(got)[1] - 53)
    return float(abs((Decimal(got) - exact) / ulp))


def _exp_args(rng):
    e = np.concatenate([rng.uniform(0, 2.0 ** 22, 6000), rng.uniform(0, 64, 2000), rng.uniform(0, 0.5, 500),
                        np.arange(0, 2 ** 22, 65536, dtype=np.float64), np.arange(0, 65536, 256, dtype=np.float64),
                        [0.0, 2.0 ** -60, 0.5, 0.5 - 2 ** -54, 1.0, 2.0 ** 22 - 2 ** -30]])
    return e


def test_exp_binary64_argument(h):
    e = _exp_args(np.random.default_rng(11))
    y = ksdf.ksdf_device_math(h, 0, e)
    worst = max(_ulps(float(v), Decimal(2) ** (-Decimal(float(a)) / 65536)) for a, v in zip(e, y))
    assert worst <= 3.0, worst


def test_exp_fixed_point_argument(h):
    e = _exp_args(np.random.default_rng(12))
    y = ksdf.ksdf_device_math(h, 1, e)
    worst = 0.0
    for a, v in zip(e, y):
        F = int(math.floor(float(a) * 2.0 ** 40))  # the routine's argument, exactly
        worst = max(worst, _ulps(float(v), Decimal(2) ** (-Decimal(F) / (Decimal(2) ** 56))))
    assert worst <= 3.0, worst


def test_exp_domain(h):
    y = ksdf.ksdf_device_math(h, 0, np.array([-1.0, 2.0 ** 22, np.inf, np.nan]))
    assert np.all(np.isnan(y))
    y = ksdf.ksdf_device_math(h, 1, np.array([-1.0, 2.0 ** 22, np.nan]))
    assert np.all(np.isnan(y))


def test_pivot_rsqrt(h):
    rng = np.random.default_rng(13)
    d = np.concatenate([np.ldexp(rng.uniform(1, 2, 8000), rng.integers(-1020, 1020, 8000)),
                        rng.uniform(1e-4, 300.0, 4000), rng.uniform(1.0, 4.0, 4000),
                        np.ldexp(1.0, np.arange(-1022, 1023, 7)),
                        [1.0, 2.0, 4.0, np.nextafter(4.0, 0), np.nextafter(1.0, 2), np.nextafter(2.0, 0),
                         np.finfo(np.float64).tiny, np.finfo(np.float64).max]])
    y = ksdf.ksdf_device_math(h, 2, d)
    worst = max(_ulps(float(v), Decimal(1) / Decimal(float(a)).sqrt()) for a, v in zip(d, y))
    assert worst <= 0.51, worst


def test_pivot_rsqrt_domain(h):
    y = ksdf.ksdf_device_math(h, 2, np.array([0.0, -1.0, 5e-324, np.inf, np.nan]))
    assert np.all(np.isnan(y))


def test_arguments(h):
    with pytest.raises(ksdf.KsdfError):
        ksdf.ksdf_device_math(h, 3, np.ones(4))
    assert ksdf.ksdf_device_math(h, 0, np.zeros(0)).size == 0
