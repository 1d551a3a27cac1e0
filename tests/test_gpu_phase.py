"""Phase-boundary scans on the GPU (hotrg_phase_scan).

The scan's chi and C_V tables are the runs and arithmetic of
hotrg_observables_batch, so they must equal its chi / chi1 / cv bit for bit;
its peaks and fit are the host routines on those tables; and the whole scan
is compared with the oracle's (same model, FP64 form) on a case whose chi
maxima lead their neighbours by more than 1 % (peak decisions well
conditioned)."""
import math

import numpy as np
import pytest

from oracle import phase as OP

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2609_20536_b300 import build
    build.build()
    from paper_2609_20536_b300 import hotrg
    return hotrg


@pytest.fixture(scope="module")
def C(H):
    c = H.Context()
    yield c
    c.close()


@pytest.mark.parametrize("delta,prec,bs", [(0.8, 0, 0), (0.3, 0, 0), (0.8, 1, 1)])
def test_scan_equals_observables_batch(H, C, delta, prec, bs):
    temps = [0.8, 0.95, 1.1, 1.25]
    hbars = [0.01, 0.03]
    base = H.params(1.0, delta, 2, 8, 8, prec=prec, block_sparse=bs)
    res = C.phase_scan(base, temps, hbars, nstreams=2)
    assert res["field"] == (H.T_IMP_M if delta > 0.36 else H.T_IMP_M1)
    pts = [H.params(1.0 / T, delta, 2, 8, 8, prec=prec, block_sparse=bs) for T in temps]
    for k, hb in enumerate(hbars):
        obs = C.observables_batch(pts, hbar=hb, dh=1e-3, nstreams=2)
        ref = [o.chi if delta > 0.36 else o.chi1 for o in obs]
        assert list(res["chi"][k]) == ref
        assert list(res["cv"]) == [o.cv for o in obs]
    # without C_V: no pure runs, the same chi
    res2 = C.phase_scan(base, temps, hbars, nstreams=1, with_cv=False)
    assert np.array_equal(res2["chi"], res["chi"]) and res2["cv"] is None


def test_peaks_and_fit_are_the_host_routines(H, C):
    temps = np.linspace(0.8, 1.4, 13)
    hbars = [0.01, 0.02, 0.04]
    res = C.phase_scan(H.params(1.0, 0.8, 2, 8, 10), temps, hbars, nstreams=2)
    for k in range(len(hbars)):
        (pk,), _ = H.hotrg_find_peaks(temps, res["chi"][k], 0.0, 1)
        assert res["t_peak"][k] == pk[0]
    f = H.hotrg_fit_tc(hbars, res["t_peak"])
    assert (res["fit"].a, res["fit"].b, res["fit"].c, res["fit"].n) == (f.a, f.b, f.c, f.n)


@pytest.fixture(scope="module")
def oracle_scan():
    temps = np.linspace(0.8, 1.4, 13)
    hbars = [0.01, 0.02, 0.04]
    chi = OP.chi_scan(0.8, 2, 8, 10, temps, hbars)
    cv = OP.cv_scan(0.8, 2, 8, 10, temps)
    tp = [OP.chi_peak(temps, row) for row in chi]
    return temps, hbars, chi, cv, tp, OP.fit_tc(hbars, tp)


def test_scan_against_oracle(H, C, oracle_scan):
    temps, hbars, chi, cv, tp, fit = oracle_scan
    res = C.phase_scan(H.params(1.0, 0.8, 2, 8, 10), temps, hbars, nstreams=2)
    # chi: a difference quotient of impurity ratios over 2 dh = 2e-3
    assert np.abs(res["chi"] - chi).max() <= 1e-7 * max(1.0, np.abs(chi).max())
    # C_V multiplies the ln Z error by beta^2 / hb^2 = 1e6
    assert np.abs(res["cv"] - cv).max() <= 1e-4
    assert np.abs(res["t_peak"] - np.array(tp)).max() <= 1e-6
    assert abs(res["fit"].a - fit["a"]) <= 1e-5 and res["fit"].n == 3
    # the chi peak moves up in T with the field; the zero-field limit lies below
    assert res["t_peak"][0] < res["t_peak"][1] < res["t_peak"][2] and res["fit"].a < res["t_peak"][0]


def test_scan_without_peaks_has_no_fit(H, C):
    # a window well inside the low-temperature side: chi rises monotonically, no interior peak
    res = C.phase_scan(H.params(1.0, 0.8, 2, 8, 8), [0.5, 0.55, 0.6], [0.01, 0.02, 0.03], nstreams=1,
                       with_cv=False)
    assert all(math.isnan(v) for v in res["t_peak"])
    assert res["fit"].n == 0 and math.isnan(res["fit"].a)


def test_scan_rejects_bad_arguments(H, C):
    base = H.params(1.0, 0.8, 2, 8, 4)
    bad = [dict(temps=[0.8, 0.9], hbars=[0.01]),                 # n_t < 3
           dict(temps=[0.9, 0.8, 1.0], hbars=[0.01]),            # not ascending
           dict(temps=[0.8, 0.9, 1.0], hbars=[0.0005]),          # hbar < dh
           dict(temps=[0.8, 0.9, 1.0], hbars=[0.01], field=5),
           dict(temps=[0.8, 0.9, 1.0], hbars=[0.01], nstreams=17),
           dict(temps=[0.8, 0.9, 1.0], hbars=[0.01], c_lo=1.0, c_hi=0.5)]
    for kw in bad:
        temps, hbars = kw.pop("temps"), kw.pop("hbars")
        with pytest.raises(H.HotrgError) as e:
            C.phase_scan(base, temps, hbars, **kw)
        assert e.value.status == H.EINVAL
    with pytest.raises(H.HotrgError):
        C.phase_scan(H.params(0.6, 0.0, 0, 8, 4, tkind=H.T_ISING), [0.8, 0.9, 1.0], [0.01])
