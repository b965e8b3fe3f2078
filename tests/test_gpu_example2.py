"""Example 2 of Sec. V on the GPU: the bisection search over the library
against the oracle's bisection, and the batched multisection against the
bisection.

Bands.  Near the certifiability threshold the certificate margin of the final
iterate is of the order of the stopping tolerance (the optimal dual has a
singular Lyapunov coefficient, reading R-A5), so there the verdict depends on
where a correct solver stops.  `verdict_is_determined` (oracle) marks the
scales where it does not: the margin at eps is within a stated factor of its
change when the tolerance moves by a decade.  At every other visited scale the
library's verdict must equal the oracle's.  Two bisections from the same
interval visit the same scales until their verdicts first differ, which can
only happen at an undetermined scale; from there both stay inside the interval
of that step, so their bounds differ by at most its width.  Two searches over
the library's own verdicts (bisection, multisection) end within their
resolutions of each other plus the extent of the undetermined scales they
visited."""

import numpy as np
import pytest

from tests.test_oracle_example2 import L_OPT, determined_many, load_example2, oracle_bisect

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_3769_gb300 import build
    build.build()
    from paper_1411_3769_gb300 import binding
    binding._lib()
    return binding


def test_substitution_matches_oracle(bd):
    from oracle import polya
    from paper_1411_3769_gb300 import robust
    from tests.test_oracle_example2 import coeffs_on_simplex, g_matrix
    for L in (-0.1, 0.0, 0.3):
        ours = robust.substitute(load_example2(), robust.simplex_scale_map(L, 3))
        assert np.allclose(ours, coeffs_on_simplex(L), rtol=1e-13, atol=1e-14)
    assert np.array_equal(robust.simplex_scale_map(0.25, 3), g_matrix(0.25))
    assert robust.monomials(3, 3) == polya.monomials(3, 3)


@pytest.mark.parametrize("d_p,d1", [(1, 1), (2, 2)])
def test_bisection_matches_oracle(bd, d_p, d1):
    from paper_1411_3769_gb300 import robust
    lo, hi, iters = -0.2, 1.0, 10
    ours, trace = robust.bisect(load_example2(), lo, hi, d_p, d1, iters=iters)
    ref_trace = []
    ref = oracle_bisect(d_p, d1, lo, hi, iters=iters, trace=ref_trace)
    assert ours > L_OPT
    det = dict(zip([s for s, _ in trace], determined_many([(s, d_p, d1) for s, _ in trace])))
    for s, v in trace:
        if det[s][0]:
            assert v == det[s][1], (s, v, det[s])
    band = 0.0
    for (s, v), (s_ref, v_ref) in zip(trace, ref_trace):
        assert s == s_ref                  # same interval so far
        if v != v_ref:
            assert not det[s][0], (s, v, v_ref)
            band = hi - lo
            break
        if v:
            hi = s
        else:
            lo = s
    assert abs(ours - ref) <= band


def test_batched_multisection_brackets_the_bisection_bound(bd):
    from paper_1411_3769_gb300 import robust
    lo, hi = -0.2, 1.0
    b_bis, t_bis = robust.bisect(load_example2(), lo, hi, 2, 3, iters=12)
    b_mul, t_mul = robust.multisection(load_example2(), lo, hi, 2, 3, points=7, rounds=4)
    assert len(t_mul) == 28
    res_bis, res_mul = (hi - lo) / 2 ** 12, (hi - lo) / 8 ** 4
    visited = sorted(set(s for s, _ in t_bis + t_mul))
    det = dict(zip(visited, determined_many([(s, 2, 3) for s in visited])))
    for s, v in t_bis + t_mul:
        if det[s][0]:
            assert v == det[s][1], (s, v, det[s])
    und = [s for s in visited if not det[s][0]]
    band = res_bis + res_mul + ((max(und) - min(und)) if und else 0.0)
    assert abs(b_mul - b_bis) <= band
    assert b_mul > L_OPT and b_bis > L_OPT
    assert dict(t_mul)[b_mul] == 1
