"""M1, one [Fe/H] (Section 2.2: isochrones interpolated between the grid metallicities), in the
oracle.  Pins: on a grid point M1 equals the Gaussian MDF in its zero-width limit; isochrones
whose magnitudes and masses are linear in [Fe/H] are reproduced at any [Fe/H] (fluxes against
the zero-point closed form, IMF weights against quadrature over the interpolated mass cells);
approaching the next grid point converges to it; outside the grid the end isochrone is used."""
import dataclasses
import math

import numpy as np
from scipy import integrate

import oracle as O
from paper_1904_00011_gb300 import workloads as W

FEH = (-1.0, -0.75, -0.5, -0.25)


def _linear_workload(n_mass=40):
    """Two ages; magnitudes a + s [Fe/H] and masses c + d [Fe/H] per point (closed forms)."""
    rng = np.random.default_rng(3)
    na, nf = 2, len(FEH)
    feh = np.asarray(FEH)
    base_m = np.geomspace(0.2, 3.0, n_mass)
    dm = 0.05 * base_m                                    # masses grow with [Fe/H]
    mass = np.empty((na, nf, n_mass))
    mags = np.empty((na, nf, n_mass, 2))
    a = rng.uniform(2.0, 9.0, (na, n_mass, 2))
    sl = rng.uniform(0.1, 0.6, (na, n_mass, 2))
    for j in range(na):
        for k in range(nf):
            mass[j, k] = base_m + dm * feh[k]
            mags[j, k] = a[j] + sl[j] * feh[k]
    iso = W.Isochrones(np.array([9.0, 10.0]), feh, mass, mags)
    p = W.Params(log_sfh=np.array([1.0, 1.5]), feh_mean=-0.6, feh_sigma=0.0, log_ebv=-1.0,
                 dust_sigma=0.0, dmod=24.0)
    w = W.Workload("m1", iso, 2, 16, [p], [16], psf=None, hess_c_lo=-1.0, hess_m_lo=21.0, seed=1)
    return w, base_m, dm, a, sl


def _imf_quadrature(m, slope=2.35):
    e = np.empty(m.size + 1)
    e[1:-1] = np.sqrt(m[:-1] * m[1:])
    e[0] = m[0] ** 2 / e[1]
    e[-1] = m[-1] ** 2 / e[-2]
    cells = np.array([integrate.quad(lambda x: x ** -slope, e[i], e[i + 1], epsabs=0, epsrel=1e-13)[0]
                      for i in range(m.size)])
    return cells / cells.sum()


def test_m1_on_a_grid_point_equals_the_narrow_gaussian_mdf():
    w = W.full()
    for k in (0, 3, 6):
        mu = W.FULL_FEH[k]
        p1 = dataclasses.replace(w.params[0], feh_mean=mu, feh_sigma=0.0)
        p2 = dataclasses.replace(w.params[0], feh_mean=mu, feh_sigma=1e-3)   # neighbours vanish
        assert np.array_equal(O.weights(w, p1), O.weights(w, p2))
        assert np.array_equal(O.fluxes(w, p1), O.fluxes(w, p2))


def test_m1_reproduces_isochrones_linear_in_feh():
    w, base_m, dm, a, sl = _linear_workload()
    for mu in (-0.9, -0.6, -0.3):
        p = dataclasses.replace(w.params[0], feh_mean=mu)
        k, t = O.m1_bracket(np.asarray(FEH), mu)
        assert 0.0 < t < 1.0
        f = O.fluxes(w, p).reshape(2, len(FEH), -1, 2)
        zp, et = np.asarray(w.zeropoint[:2]), np.asarray(w.exptime[:2])
        want = et * 10.0 ** (-0.4 * (a + sl * mu + p.dmod - zp))
        assert np.allclose(f[:, k], want, rtol=1e-12, atol=0)
        lam = O.weights(w, p)
        assert np.count_nonzero(lam.sum(axis=(0, 2))) == 1
        imf = _imf_quadrature(base_m + dm * mu)
        for j in range(2):
            assert np.allclose(lam[j, k] / lam[j, k].sum(), imf, rtol=1e-9, atol=0)
            assert math.isclose(lam[j, k].sum(), 10.0 ** p.log_sfh[j], rel_tol=1e-13)


def test_m1_converges_to_the_next_grid_isochrone():
    w, *_ = _linear_workload()
    p_near = dataclasses.replace(w.params[0], feh_mean=-0.5 - 1e-10)   # just below the grid -0.5
    p_grid = dataclasses.replace(w.params[0], feh_mean=-0.5)
    k, t = O.m1_bracket(np.asarray(FEH), p_near.feh_mean)
    assert k == 1 and t > 0.999999
    ln, lg = O.weights(w, p_near), O.weights(w, p_grid)
    fn, fg = O.fluxes(w, p_near).reshape(2, 4, -1, 2), O.fluxes(w, p_grid).reshape(2, 4, -1, 2)
    assert np.allclose(ln[:, 1], lg[:, 2], rtol=1e-8)
    assert np.allclose(fn[:, 1], fg[:, 2], rtol=1e-8)


def test_m1_outside_the_grid_takes_the_end_isochrone():
    feh = np.asarray(FEH)
    assert O.m1_bracket(feh, -3.0) == (0, 0.0)
    assert O.m1_bracket(feh, 0.5) == (3, 0.0)
    assert O.m1_bracket(feh, -0.25) == (3, 0.0)
    assert O.m1_bracket(np.array([-0.5]), -0.1) == (0, 0.0)
    w, *_ = _linear_workload()
    hi = O.weights(w, dataclasses.replace(w.params[0], feh_mean=0.7))
    assert np.count_nonzero(hi.sum(axis=(0, 2))) == 1 and hi[:, 3].sum() > 0
