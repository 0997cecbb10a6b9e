"""dq_theory (the library's theory-mode counts, host arithmetic) against the oracle's
eq. choose_ein / Sec. 5 helpers; runs without a GPU."""
import math

import numpy as np
import pytest

import oracle as O

ALGS = {"DGM": O.DGM, "DFGM": O.DFGM, "ADGM": O.ADGM, "ADFGM": O.ADFGM}


@pytest.mark.parametrize("alg", list(ALGS))
@pytest.mark.parametrize("eps,Rd,D_U,lmax,lmin,normG2", [
    (1e-3, 1.0, 2.0, 100.0, 1.0, 3.0),
    (1e-2, 0.3, 44.7, 4.01, 0.01, 2.9),
    (1e-4, 5.0, 10.0, 1e4, 1.0, 0.5),
    (1e-3, 2.0, 2.0, 10.0, 0.0, 1.0),      # singular Q: only the augmented algorithms
])
def test_library_counts_match_oracle(alg, eps, Rd, D_U, lmax, lmin, normG2):
    from paper_1504_05708_gb300 import duquad as D
    a = ALGS[alg]
    if lmin == 0.0 and a in (O.DGM, O.DFGM):
        with pytest.raises(D.DuquadError) as e:
            D.theory(alg, eps, Rd, D_U, lmax, lmin, normG2)
        assert e.value.status == D.ERR_INVALID
        return
    t = D.theory(alg, eps, Rd, D_U, lmax, lmin, normG2)
    rho = O.rho_star(eps, Rd) if a in (O.ADGM, O.ADFGM) else 0.0
    LL, Ld = lmax + rho * normG2, normG2 / (lmin + rho * normG2)
    ein = O.default_eps_in(a, eps, Ld, Rd)
    assert t["rho"] == pytest.approx(rho, rel=1e-15)
    assert t["LL"] == pytest.approx(LL, rel=1e-15) and t["sigma"] == lmin
    assert t["Ld"] == pytest.approx(Ld, rel=1e-14)
    assert t["eps_in"] == pytest.approx(ein, rel=1e-14)
    assert t["k_out"] == max(1, math.ceil(O.k_out(a, eps, Ld, Rd) * (1 - 1e-14)))
    assert t["k_in"] == max(1, math.ceil(O.k_in(LL, lmin, D_U, ein) * (1 - 1e-14)))
    assert t["k_total"] == t["k_out"] * t["k_in"]


def test_library_counts_with_given_rho_and_invalid_inputs():
    from paper_1504_05708_gb300 import duquad as D
    t = D.theory("ADFGM", 1e-3, 1.0, 2.0, 100.0, 1.0, 3.0, rho=0.5)
    assert t["rho"] == 0.5 and t["LL"] == pytest.approx(101.5)
    for bad in (dict(eps=0.0), dict(Rd=-1.0), dict(D_U=float("nan")), dict(lmin_Q=-1.0)):
        kw = dict(alg="DGM", eps=1e-3, Rd=1.0, D_U=2.0, lmax_Q=10.0, lmin_Q=1.0, normG2=1.0)
        kw.update(bad)
        with pytest.raises(D.DuquadError):
            D.theory(**kw)
    with pytest.raises(D.DuquadError):
        D.theory("DFGM", 1e-3, 1.0, 2.0, 10.0, 1.0, 1.0, rho=0.5)     # rho > 0 is ADGM/ADFGM only
