"""Host set-up of libhz (hz_plan, no GPU) against the oracle's set-up on the same inputs:
spectrum rectangle (Lemma 3.1), contour nodes (eq:quad-points) and the polynomial-scheme
parameters (eq:fix-pt-conv)."""
import numpy as np
import pytest

import paper_1811_12378_gb300 as hzpkg
import workloads as W
from oracle import hz_oracle as O


def cases():
    return [W.small_case(3, 13, 9, 7, layer=2, J=4),
            W.small_case(4, 16, 16, 16, layer=4, J=6, medium="layered"),
            W.small_case(5, 5, 1, 3, layer=1, J=3, medium="const"),
            W.point_source_32(),
            W.gaussian_bumps_64()]


@pytest.mark.parametrize("wl", cases(), ids=lambda w: w.name)
def test_plan_matches_oracle(wl):
    info, tb = hzpkg.plan(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps)
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    (b1, b2, rho2), nodes = O.setup_nodes(op, wl.J, wl.t, wl.eps)
    assert info["s"] == pytest.approx(op.s, rel=1e-15)
    assert info["b1"] == pytest.approx(b1, rel=1e-13, abs=1e-13)
    assert info["b2"] == pytest.approx(b2, rel=1e-13)
    assert info["rho2"] == pytest.approx(rho2, rel=1e-14)
    assert info["n"] == op.n and info["J"] == wl.J
    assert info["stages"] == max(nd.q * nd.sweeps for nd in nodes)
    for j, nd in enumerate(nodes):
        assert abs(tb["z"][j] - nd.z) <= 1e-13 * abs(nd.z)
        assert abs(tb["sigma"][j] - nd.sigma) <= 1e-13 * abs(nd.sigma)
        assert abs(tb["z0"][j] - nd.z0) <= 1e-13 * abs(nd.z0)
        assert tb["q"][j] == nd.q
        assert tb["sweeps"][j] == nd.sweeps
        assert tb["delta"][j] == pytest.approx(nd.delta, rel=1e-7)
        assert tb["nu"][j] == pytest.approx(nd.nu, rel=1e-9)


def spectral_cases():
    return [W.small_case(3, 12, 10, 9, layer=2, J=4, ppw=2.5),
            W.small_case(6, 7, 16, 5, layer=1, J=6, ppw=3.0),
            W.spectral_bumps(24, 3),
            W.spectral_bumps(64, 1)]


@pytest.mark.parametrize("t", [1.0, 0.6])
@pytest.mark.parametrize("wl", spectral_cases(), ids=lambda w: w.name)
def test_spectral_plan_matches_oracle(wl, t):
    """The same for the Fourier spectral Laplacian (its rectangle from the closed-form
    wavenumbers, eq:eig-Laplacian-spectral), on circles and ellipses of ratio t = 0.6."""
    info, tb = hzpkg.plan(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, t, wl.eps,
                          discretization=hzpkg.HZ_DISC_SPECTRAL)
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, kind="spectral")
    (b1, b2, rho2), nodes = O.setup_nodes(op, wl.J, t, wl.eps)
    assert info["b1"] == pytest.approx(b1, rel=1e-13, abs=1e-13)
    assert info["b2"] == pytest.approx(b2, rel=1e-13)
    assert info["rho2"] == pytest.approx(rho2, rel=1e-14)
    for j, nd in enumerate(nodes):
        assert abs(tb["z"][j] - nd.z) <= 1e-13 * abs(nd.z)
        assert abs(tb["sigma"][j] - nd.sigma) <= 1e-13 * abs(nd.sigma)
        assert tb["q"][j] == nd.q and tb["sweeps"][j] == nd.sweeps
        assert tb["delta"][j] == pytest.approx(nd.delta, rel=1e-7)


def test_plan_rejects_bad_input():
    c = np.ones((4, 4, 4))
    with pytest.raises(hzpkg.HzError):
        hzpkg.plan(c, 0.2, 1.0, 1, 1.0, 0, 1.0, 1.0)      # J = 0
    with pytest.raises(hzpkg.HzError):
        hzpkg.plan(-c, 0.2, 1.0, 1, 1.0, 4, 1.0, 1.0)     # negative speed
    with pytest.raises(hzpkg.HzError):
        hzpkg.plan(c, 0.2, 1.0, 1, 1.0, 17, 1.0, 1.0)     # J > 16
