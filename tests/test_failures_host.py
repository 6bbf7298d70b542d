"""Invalid input is rejected on the host with BIOT_EINVAL and a message, before any CUDA call
(so these run without a GPU): non-finite or non-positive permeabilities, coefficients out of
their ranges (paper §Poroelasticity: 0 < b < 1, 1/M >= 0, K_dr, mu, eta > 0, lambda >= 0) or
non-finite, bad mesh sizes, time orders and boundary codes."""
import numpy as np
import pytest

from paper_1801_04984_gb300 import binding as B

GOOD = dict(lam=1.0, mu=1.0, b=0.8, invM=0.05, eta=1.0, K_dr=5.0 / 3.0)
UBC, FBC = [2, 2, 2, 2, 2, 0], [1, 1, 1, 1, 1, 0]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1801_04984_gb300 import build
    build.build()


def _setup(n=(3, 2, 2), r=1, K=None, ubc=UBC, fbc=FBC, **co):
    K = np.full(int(np.prod(n)), 1e-2) if K is None else K
    return B.Context(len(n), n, dict(GOOD, K=K, **co), r, ubc, fbc)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -1e-2, 0.0])
def test_bad_permeability_is_rejected(bad):
    K = np.full(12, 1e-2)
    K[7] = bad
    with pytest.raises(B.BiotError) as e:
        _setup(K=K)
    assert e.value.code == B.EINVAL and "K_cell[7]" in str(e.value)


@pytest.mark.parametrize("name,value", [("b", 1.0), ("b", 0.0), ("b", np.nan), ("invM", -0.1), ("invM", np.inf),
                                        ("mu", 0.0), ("lam", -1.0), ("eta", 0.0), ("K_dr", 0.0), ("K_dr", np.nan)])
def test_bad_coefficient_is_rejected(name, value):
    with pytest.raises(B.BiotError) as e:
        _setup(**{name: value})
    assert e.value.code == B.EINVAL


def test_bad_mesh_order_and_boundary_codes_are_rejected():
    for kw in (dict(r=3), dict(r=-1), dict(ubc=[5, 2, 2, 2, 2, 0]), dict(fbc=[1, 1, 1, 1, 1, 7])):
        with pytest.raises(B.BiotError) as e:
            _setup(**kw)
        assert e.value.code == B.EINVAL
    with pytest.raises(B.BiotError):
        B.Context(3, (0, 2, 2), dict(GOOD, K=np.zeros(0)), 1, UBC, FBC)


def test_host_only_entry_points_reject_bad_arguments():
    lib = B.load()
    assert lib.biot_time_tables(3, None, None, None, None, None, None, None, None, None) == B.EINVAL
    assert lib.biot_fma_peak(7, None, None, None) == B.EINVAL
