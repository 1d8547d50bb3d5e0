"""The binding's two ways of passing parameter sets to the C ABI give the same pcmd_params
records: a list of workloads.Params, and a float64 matrix in the struct's layout (the
surrogate's fast path).  CPU only: no library call."""
import numpy as np
import pytest

import paper_1904_00011_gb300 as P
from paper_1904_00011_gb300 import workloads as W
from paper_1904_00011_gb300 import surrogate as S


def _fields(rec):
    return list(rec.log_sfh) + [rec.feh_mean, rec.feh_sigma, rec.log_ebv, rec.dust_sigma, rec.dmod]


def test_matrix_and_list_marshalling_agree():
    th = np.random.default_rng(0).uniform(-0.5, 0.5, size=(7, 12))
    sur = S.Surrogate.__new__(S.Surrogate)       # only the parameter mapping, no device state
    sur.base = W.surrogate(n_sets=1, n_im=64)
    w = W.surrogate_from_theta(th, n_im=64, base=sur.base)
    a = P.params_array(w.params)
    b = P.params_array(sur.param_matrix(th))
    assert len(a) == len(b) == 7
    for k in range(7):
        assert _fields(a[k]) == _fields(b[k])


def test_matrix_of_wrong_width_is_rejected():
    with pytest.raises(ValueError):
        P.params_array(np.zeros((3, 12)))
