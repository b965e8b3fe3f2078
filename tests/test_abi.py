"""The C-ABI library builds, loads and exports every symbol its header declares;
host-side argument checks (no GPU needed)."""

import os
import re

import numpy as np
import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_1411_3769_gb300 import build
    build.build()
    from paper_1411_3769_gb300 import binding
    return binding._lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "polya_sdp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psdp_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    from paper_1411_3769_gb300 import binding
    names = _declared()
    assert len(names) >= 20
    for nm in names:
        assert hasattr(lib, nm), nm
    assert sorted(binding.EXPORTS) == names


def test_default_opts_and_strerror(lib):
    from paper_1411_3769_gb300 import binding as b
    o = b.psdp_default_opts()
    assert o.delta == 1.0 and o.eps == 1e-7 and abs(o.sigma - 1 / 3) < 1e-15 and o.tau == 0.95
    assert o.d2 == -1 and o.d_a == 1 and o.max_iter == 100 and o.crit_sms == 0
    assert b.psdp_strerror(0) == "ok"
    assert "positive definite" in b.psdp_strerror(5)


@pytest.mark.parametrize("args", [
    dict(n=0, l=2, d_p=1, d1=1), dict(n=113, l=2, d_p=1, d1=1), dict(n=4, l=0, d_p=1, d1=1),
    dict(n=4, l=2, d_p=-1, d1=1), dict(n=4, l=2, d_p=1, d1=-2), dict(n=4, l=17, d_p=1, d1=1),
])
def test_setup_rejects_bad_sizes(lib, args):
    from paper_1411_3769_gb300 import binding as b
    A = np.zeros((max(args["l"], 1), max(args["n"], 1), max(args["n"], 1)))
    with pytest.raises(b.PsdpError) as e:
        b.psdp_setup(args["n"], args["l"], args["d_p"], args["d1"], A)
    assert e.value.name == "EINVAL"


def test_setup_rejects_nonfinite_and_bad_options(lib):
    from paper_1411_3769_gb300 import binding as b
    A = np.zeros((2, 3, 3))
    A[1, 2, 2] = np.nan
    with pytest.raises(b.PsdpError) as e:
        b.psdp_setup(3, 2, 1, 1, A)
    assert e.value.name == "EINVAL"
    with pytest.raises(b.PsdpError) as e:
        b.psdp_setup(3, 2, 1, 1, np.zeros((2, 3, 3)), b.psdp_default_opts(tau=1.5))
    assert e.value.name == "EINVAL"
    with pytest.raises(b.PsdpError) as e:
        b.psdp_setup(3, 2, 1, 1, np.zeros((2, 3, 3)), b.psdp_default_opts(precision=1, crit_sms=-1))
    assert e.value.name == "EINVAL"


def test_null_context_is_einval(lib):
    assert lib.psdp_step(None, None) == 1
    assert lib.psdp_certify(None, None, None, None) == 1
    lib.psdp_destroy(None)
