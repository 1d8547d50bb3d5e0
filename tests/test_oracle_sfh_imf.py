"""Parametric SFH models (Section 2.2 S1-S4) and the Kroupa IMF: the oracle against quadrature
and closed forms, and the library's host helper against the oracle (CPU)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_1904_00011_gb300 import workloads as W

EDGES = np.linspace(6.0, 10.15, 22)       # 21 bins in log age, 1 Myr .. 14 Gyr (Section 2.2)


def _bin_masses(rate):
    ages = 10.0 ** EDGES
    t0 = ages[-1]
    return np.array([integrate.quad(rate, t0 - ages[j + 1], t0 - ages[j], limit=200)[0]
                     for j in range(len(EDGES) - 1)])


@pytest.mark.parametrize("model,tau", [(O.SFH_TAU, 1.5), (O.SFH_TAU, 8.0),
                                       (O.SFH_DELAYED_TAU, 2.0), (O.SFH_DELAYED_TAU, 0.7)])
def test_tau_models_match_quadrature(model, tau):
    t = tau * 1e9
    rate = (lambda x: math.exp(-x / t)) if model == O.SFH_TAU else (lambda x: x * math.exp(-x / t))
    m = _bin_masses(rate)
    ref = 1e4 * m / m.sum()
    got = 10.0 ** O.sfh_bins(model, [4.0, tau], EDGES)
    ok = ref > 1e-25
    assert np.allclose(got[ok], ref[ok], rtol=1e-6)
    assert abs(got.sum() - 1e4) < 1e-6


def test_constant_and_ssp():
    got = 10.0 ** O.sfh_bins(O.SFH_CONSTANT, [2.0], EDGES)
    widths = 10.0 ** EDGES[1:] - 10.0 ** EDGES[:-1]
    assert np.allclose(got / got.sum(), widths / widths.sum(), rtol=1e-12)
    assert abs(got.sum() - 100.0) < 1e-9
    s = O.sfh_bins(O.SFH_SSP, [3.0, 9.03], EDGES)
    j = np.nonzero(s > -30)[0]
    assert len(j) == 1 and EDGES[j[0]] <= 9.03 < EDGES[j[0] + 1]
    assert abs(10.0 ** s[j[0]] - 1000.0) < 1e-9


@pytest.mark.parametrize("model,theta", [(1, [3.0, 9.03]), (2, [2.0]), (3, [4.0, 1.5]), (4, [5.0, 2.0]),
                                         (3, [1.0, 30.0])])
def test_library_helper_matches_oracle(model, theta):
    import paper_1904_00011_gb300 as P
    got = P.sfh_bins(model, theta, EDGES)
    ref = O.sfh_bins(model, theta, EDGES)
    assert np.allclose(got, ref, rtol=0, atol=1e-10)


def test_library_helper_rejects_bad_input():
    import paper_1904_00011_gb300 as P
    with pytest.raises(P.PcmdError):
        P.sfh_bins(9, [2.0], EDGES)
    with pytest.raises(P.PcmdError):
        P.sfh_bins(O.SFH_TAU, [2.0, -1.0], EDGES)
    with pytest.raises(P.PcmdError):
        P.sfh_bins(O.SFH_SSP, [2.0, 12.0], EDGES)
    with pytest.raises(P.PcmdError):
        P.sfh_bins(O.SFH_CONSTANT, [2.0], EDGES[::-1])


def _kroupa_density(m):
    if m < 0.08:
        return m ** -0.3
    if m < 0.5:
        return 0.08 * m ** -1.3
    return 0.04 * m ** -2.3


def test_kroupa_imf_cells_match_quadrature_and_are_continuous():
    w = W.tiny()
    wk = W.Workload(**{**w.__dict__, "imf": 1})
    lam = O.weights(wk, wk.params[0]).reshape(-1)
    m = wk.iso.mass.reshape(-1)
    e = np.empty(m.size + 1)
    e[1:-1] = np.sqrt(m[:-1] * m[1:])
    e[0] = m[0] ** 2 / e[1]
    e[-1] = m[-1] ** 2 / e[-2]
    cells = np.array([integrate.quad(_kroupa_density, e[i], e[i + 1], points=[0.08, 0.5])[0]
                      for i in range(m.size)])
    ref = cells / cells.sum() * lam.sum()
    assert np.allclose(lam, ref, rtol=1e-9)
    # continuity of the density at the breaks
    for b in (0.08, 0.5):
        assert math.isclose(_kroupa_density(b * (1 - 1e-12)), _kroupa_density(b), rel_tol=1e-9)
    # Kroupa differs from Salpeter on the same grid (more weight below 0.5 Msun relative to above)
    lam_s = O.weights(w, w.params[0]).reshape(-1)
    low = m < 0.5
    assert lam[low].sum() / lam.sum() != pytest.approx(lam_s[low].sum() / lam_s.sum(), rel=1e-3)
