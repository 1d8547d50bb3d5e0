"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no compute calls: no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(pcmd_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libpcmd():
    from paper_1904_00011_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["pcmd_create", "pcmd_simulate", "pcmd_hess", "pcmd_loglike", "pcmd_destroy",
              "pcmd_evaluate", "pcmd_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpcmd):
    missing = [n for n in _declared() if not hasattr(libpcmd, n)]
    assert not missing, missing


def test_package_fails_loudly_without_gpu(libpcmd):
    import torch
    import paper_1904_00011_gb300 as P
    from paper_1904_00011_gb300 import workloads as W
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        P.Simulator(W.tiny())
