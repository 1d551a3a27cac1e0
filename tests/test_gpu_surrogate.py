"""Batched observables and the surrogate driver.

hotrg_observables_batch must equal hotrg_observables bit for bit (the same
runs through the batch runner).  The surrogate's prediction is checked
against the FP64 oracle network on the members' BF16-rounded weights, its
refinement points against a brute-force argmax of the oracle network, and
its re-solve step against hotrg_observables_batch on the flagged points."""
import numpy as np
import pytest

from oracle import mlp as OM
from oracle import observables as OO

pytestmark = pytest.mark.gpu

FIELDS = ("lnz", "f", "cv", "m", "m1", "chi", "chi1")


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


def grid_params(H, betas, deltas, nm=2, dcut=8, steps=10, prec=0):
    return [H.params(b, d, nm, dcut, steps, prec=prec) for d in deltas for b in betas]


@pytest.mark.parametrize("nstreams", [1, 3])
def test_observables_batch_equals_sequential(H, C, nstreams):
    pts = grid_params(H, [0.7, 1.1, 1.5], [0.3, 0.9])
    a = C.observables(pts)
    b = C.observables_batch(pts, nstreams=nstreams)
    for x, y in zip(a, b):
        assert y.status == 0
        assert [getattr(x, f) for f in FIELDS] == [getattr(y, f) for f in FIELDS]


def test_observables_batch_against_oracle(H, C):
    args = (1.0, 0.5, 2, 8, 10)
    o = C.observables_batch([H.params(*args)], hb=1e-3, hbar=0.01, dh=1e-3)[0]
    ref = OO.observables(*args, hb=1e-3, hbar=0.01, dh=1e-3)
    assert abs(o.lnz - ref.lnz) < 1e-10
    assert abs(o.cv - ref.cv) < 1e-3  # central difference amplifies rounding by beta^2 / hb^2
    assert abs(o.m - ref.m) < 1e-10 and abs(o.chi - ref.chi) < 1e-6 and abs(o.chi1 - ref.chi1) < 1e-6


def test_observables_batch_rejects_bad_arguments(H, C):
    with pytest.raises(H.HotrgError):
        C.observables_batch([H.params(1.0, 0.5, 2, 8, 4)], hbar=0.0, dh=1e-3)
    with pytest.raises(H.HotrgError):
        C.observables_batch([H.params(1.0, 0.5, 2, 8, 4)], nstreams=17)  # 0 means the autotuned count


def oracle_members(sur):
    """The members' networks as the GPU holds them: BF16 weights, FP32 biases."""
    nets = []
    for e in range(sur.mlp.ensemble):
        flat = sur.mlp.get_params(e).astype(np.float64)
        net, o = [], 0
        for a, b in zip(OM.SIZES[:-1], OM.SIZES[1:]):
            W = flat[o:o + a * b].reshape(a, b)
            o += a * b
            net.append((OM.weights_bf16(W), flat[o:o + b].copy()))
            o += b
        nets.append(net)
    return nets


def oracle_predict(sur, X):
    s = sur.scaling
    Xs = ((X - np.array(s.x_mean[:])) / np.array(s.x_std[:])).astype(np.float32).astype(np.float64)
    outs = np.stack([OM.forward(net, Xs)[0] for net in oracle_members(sur)])
    return outs.mean(0) * np.array(s.y_std[:]) + np.array(s.y_mean[:]), outs.std(0)


@pytest.fixture(scope="module")
def trained(H, C):
    betas = np.linspace(0.6, 1.6, 11)
    deltas = np.linspace(0.2, 0.8, 5)
    pts = grid_params(H, betas, deltas)
    obs = C.observables_batch(pts, nstreams=3)
    X = np.array([[p.beta, p.delta] for p in pts])
    Y = np.array([[o.f, o.cv, o.chi, o.chi1] for o in obs])
    sur = H.Surrogate(ensemble=4, seed=9)
    loss = sur.fit(X, Y, epochs=1500, batch=64, lr=2e-3)
    yield sur, X, Y, loss
    sur.close()


def test_surrogate_fits_and_matches_oracle_network(H, trained):
    sur, X, Y, loss = trained
    assert loss < 0.05
    y, sd = sur.predict(X)
    ref, ref_sd = oracle_predict(sur, X)
    scale = np.array(sur.scaling.y_std[:])
    assert np.abs((y - ref) / scale).max() < 1e-4
    assert np.abs(sd - ref_sd).max() < 1e-4
    # the fit itself: standardised residual on the training grid
    assert np.sqrt(np.mean(((y - Y) / scale) ** 2)) < 0.25


def test_refinement_points_sit_at_the_oracle_maxima(H, trained):
    sur, _, _, _ = trained
    deltas = np.array([0.25, 0.5, 0.75])
    Xr, pk = sur.peaks(deltas, 0.6, 1.6, 201, 5, 0.05)
    assert Xr.shape == (len(deltas) * 2 * 5, 2)
    betas = np.linspace(0.6, 1.6, 201)
    for a, d in enumerate(deltas):
        ref, _ = oracle_predict(sur, np.column_stack([betas, np.full_like(betas, d)]))
        for o in (1, 2):
            got = ref[np.argmin(np.abs(betas - pk[a, o - 1])), o]
            # the GPU's argmax is the oracle's up to FP32 rounding of near-equal values
            assert got >= ref[:, o].max() - 3e-4 * sur.scaling.y_std[o]
            win = Xr[(a * 2 + o - 1) * 5:(a * 2 + o) * 5]
            assert np.all(win[:, 1] == d)
            assert np.all(np.abs(win[:, 0] - pk[a, o - 1]) <= 0.05 + 1e-12)


def test_refine_resolves_exactly_the_uncertain_points(H, C, trained):
    sur, _, _, _ = trained
    Xr, _ = sur.peaks(np.array([0.3, 0.7]), 0.6, 1.6, 101, 4, 0.1)
    _, sd = sur.predict(Xr)
    thr = float(np.median(sd.max(1)))
    base = H.params(1.0, 0.5, 2, 8, 10)
    y, sd2, solved = sur.refine(C, base, Xr, threshold=thr, nstreams=2)
    assert np.array_equal(solved, sd.max(1) > thr)
    assert 0 < solved.sum() < len(Xr)
    pred, _ = sur.predict(Xr)
    assert np.array_equal(y[~solved], pred[~solved])
    obs = C.observables_batch([H.params(b, d, 2, 8, 10) for b, d in Xr[solved]], nstreams=2)
    assert np.array_equal(y[solved], np.array([[o.f, o.cv, o.chi, o.chi1] for o in obs]))
