"""What the trained surrogate gains, on the GPU: the project's network and HOTRG.

The same experiment as test_oracle_surrogate_gain.py, with every step on the
library: the observables of an 11 x 4 (beta, Delta) training grid come from
hotrg_observables_batch, the 4-member MLP ensemble is trained by the library's
own forward / backward / Adam kernels (hotrg_surrogate_fit), and
hotrg_surrogate_peaks places the refinement window at the ensemble's chi
maximum for a Delta between the training rows.  Five HOTRG solves in that
window, and five spread uniformly over the beta range, each locate the chi
peak (hotrg_find_peaks); a dense HOTRG scan (a coarse pass, then a fine one
around its peak) is the judge.  n_max = 2, D_cut = 8, 10 steps, chi at
hbar = 0.01, dh = 1e-3: the peak is an interior maximum at this size.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NM, DC, ST = 2, 8, 10
DELTA = 0.75  # between the training grid's Delta rows
B_LO, B_HI = 0.6, 1.6
HB, HBAR, DH = 1e-3, 0.01, 1e-3


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


def observables(H, C, X):
    pts = [H.params(b, d, NM, DC, ST) for b, d in X]
    out = C.observables_batch(pts, hb=HB, hbar=HBAR, dh=DH, nstreams=3)
    assert all(o.status == 0 for o in out)
    return np.array([[o.f, o.cv, o.chi, o.chi1] for o in out])


def chi_peak(H, C, betas):
    chi = observables(H, C, [(b, DELTA) for b in betas])[:, 2]
    peaks, _ = H.hotrg_find_peaks(np.asarray(betas, dtype=np.float64), chi, 0.0, 4)
    assert peaks, "no interior chi maximum"
    return max(peaks, key=lambda p: p[2])[0]  # the most prominent one


def test_gpu_surrogate_steering_beats_uniform_refinement(H, C):
    betas = np.linspace(B_LO, B_HI, 11)
    X = np.array([[b, d] for d in (0.6, 0.7, 0.8, 0.9) for b in betas])
    Y = observables(H, C, X)
    sur = H.Surrogate(ensemble=4, seed=20536)
    try:
        sur.fit(X, Y, epochs=2000, batch=len(X), lr=2e-3)
        _, pk = sur.peaks([DELTA], B_LO, B_HI, 401, 2, 0.05)
    finally:
        sur.close()
    b_sur = pk[0, 1]  # the ensemble mean's chi maximum at DELTA
    # the judge: a dense HOTRG scan, coarse then fine around its peak
    b0 = chi_peak(H, C, np.linspace(B_LO, B_HI, 21))
    b_ref = chi_peak(H, C, np.linspace(b0 - 0.05, b0 + 0.05, 21))
    # five HOTRG solves either way
    err_steered = abs(chi_peak(H, C, np.linspace(b_sur - 0.05, b_sur + 0.05, 5)) - b_ref)
    err_uniform = abs(chi_peak(H, C, np.linspace(B_LO, B_HI, 5)) - b_ref)
    assert abs(b_sur - b_ref) < 0.03, (b_sur, b_ref)
    assert err_steered < 1e-3, err_steered
    assert err_steered < 0.1 * err_uniform, (err_steered, err_uniform)
