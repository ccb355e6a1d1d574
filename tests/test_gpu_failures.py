"""Failure handling through the C ABI: every error comes back as an nc_status (NatConvError in
Python) and leaves the problem usable; nothing traps or faults on the device. The failures are made
on the host side (bad inputs, call order, a tiny time limit, an iteration limit)."""

import numpy as np
import pytest

from synthetic import filtered_random

pytestmark = pytest.mark.gpu

N = 8


@pytest.fixture(scope="module")
def nc():
    from paper_1904_00182_gb300 import build
    build.build()
    import paper_1904_00182_gb300
    return paper_1904_00182_gb300


def _status(exc):
    return exc.value.status_name


def test_bad_designs_are_rejected_and_the_problem_stays_usable(nc):
    pb = nc.Problem(N, N, N, alpha=1e4)
    rho = filtered_random(N, N, N, seed=1, volfrac=0.2)
    for bad in (np.where(np.arange(rho.size) == 5, np.nan, rho), np.where(np.arange(rho.size) == 7, 1.5, rho),
                np.where(np.arange(rho.size) == 9, -0.1, rho)):
        with pytest.raises(nc.NatConvError) as e:
            pb.set_design(bad)
        assert _status(e) == "NC_ERR_ARG"
    with pytest.raises(ValueError):
        pb.set_design(rho[:-1])
    pb.set_design(rho)
    st = pb.solve_state()
    assert st["rel_residual"] <= 1e-8
    pb.close()


def test_call_order_is_enforced(nc):
    pb = nc.Problem(N, N, N, alpha=1e4)
    with pytest.raises(nc.NatConvError) as e:
        pb.solve_state()
    assert _status(e) == "NC_ERR_STATE"
    pb.set_design(filtered_random(N, N, N, seed=2, volfrac=0.2))
    with pytest.raises(nc.NatConvError) as e:
        pb.solve_adjoint()
    assert _status(e) == "NC_ERR_STATE"
    pb.solve_state()
    with pytest.raises(nc.NatConvError) as e:
        pb.sensitivities()
    assert _status(e) == "NC_ERR_STATE"
    pb.solve_adjoint()
    assert np.all(np.isfinite(pb.sensitivities().cpu().numpy()))
    pb.close()


def test_time_and_iteration_limits(nc):
    rho = filtered_random(N, N, N, seed=3, volfrac=0.2)
    pb = nc.Problem(N, N, N, alpha=1e4, timeout_s=1e-9)
    pb.set_design(rho)
    with pytest.raises(nc.NatConvError) as e:
        pb.solve_state()
    assert _status(e) == "NC_ERR_TIMEOUT"
    pb.set_params(timeout_s=600.0, newton_maxit=1, newton_rtol=1e-12)
    pb.set_design(rho)
    with pytest.raises(nc.NatConvError) as e:
        pb.solve_state()
    assert _status(e) == "NC_ERR_MAXIT"
    pb.set_params(newton_maxit=50, newton_rtol=1e-8)
    pb.set_design(rho)
    assert pb.solve_state()["rel_residual"] <= 1e-8
    pb.close()


def test_fixed_parameters_cannot_change(nc):
    pb = nc.Problem(N, N, N, alpha=1e4)
    with pytest.raises(nc.NatConvError) as e:
        pb.set_params(precision=nc.NC_PREC_FP64)
    assert _status(e) == "NC_ERR_ARG"
    with pytest.raises(nc.NatConvError) as e:
        pb.set_params(outer_arith=7)
    assert _status(e) == "NC_ERR_ARG"
    pb.close()
