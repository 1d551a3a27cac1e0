"""hotrg_run_batch: points of several classes on several worker streams, the
first point of each class run directly and the rest replayed from a captured
CUDA graph.  The kernels and their inputs are the same as hotrg_run's, so the
results must be bitwise identical; a few are also checked against the oracle."""
import pytest

from oracle import hotrg as OH

from parity_points import BATCH, BATCH_ORACLE

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


def points(H, prec):
    return [H.params(*pt, prec=prec) for pt in BATCH]


@pytest.mark.parametrize("prec_name", ["FP64", "SPLIT_BF16"])
@pytest.mark.parametrize("nstreams", [1, 3])
def test_batch_equals_single_runs(H, C, prec_name, nstreams):
    prec = getattr(H, prec_name)
    pts = points(H, prec)
    single = [C.run([p])[0].lnz_per_site for p in pts]
    for repeat in range(2):  # the second call replays graphs only
        got = C.run_batch(pts, nstreams=nstreams)
        assert [r.status for r in got] == [0] * len(pts)
        assert [r.lnz_per_site for r in got] == single
        for r, p in zip(got, pts):
            assert r.n_steps == p.n_steps and r.step[p.n_steps - 1].dprime > 0


def test_batch_against_oracle(H, C):
    pts = [H.params(*pt, prec=H.SPLIT_BF16) for pt in BATCH_ORACLE]
    got = C.run_batch(pts, nstreams=2)
    for r, p in zip(got, pts):
        ref = OH.run_gxy(p.beta, p.delta, p.n_max, p.d_cut, p.n_steps).lnz_per_site
        assert abs(r.lnz_per_site - ref) < 1e-9


def test_batch_with_invalid_entries(H, C):
    pts = points(H, H.SPLIT_BF16)[:3]
    pts.insert(1, H.params(-1.0, 0.5, 2, 12, 14))
    got = H.hotrg_run_batch(C.handle, pts, nstreams=2, check=False)
    assert got[1].status == H.EINVAL
    assert all(got[i].status == 0 for i in (0, 2, 3))


def test_batch_with_profiling_equals_graph_replay(H, C):
    pts = points(H, H.SPLIT_BF16)[:4]
    replay = [r.lnz_per_site for r in C.run_batch(pts, nstreams=2)]
    H.hotrg_profile_enable(C.handle, True)
    got = [r.lnz_per_site for r in C.run_batch(pts, nstreams=2)]
    prof = H.hotrg_profile_read(C.handle)
    H.hotrg_profile_enable(C.handle, False)
    assert got == replay
    assert prof.steps == sum(p.n_steps for p in pts)
    assert prof.gemm_calls[1] > 0 and prof.gemm_ms[1] > 0 and prof.eig_ms > 0


def test_autotune_batch_and_tuned_stream_count(H, C):
    pts = points(H, H.SPLIT_BF16)[:4]
    best, secs = C.autotune_batch(pts, max_streams=3)
    assert 1 <= best <= 3 and len(secs) == 3 and all(t > 0 for t in secs)
    single = [C.run([p])[0].lnz_per_site for p in pts]
    got = [r.lnz_per_site for r in C.run_batch(pts, nstreams=0)]  # 0: the tuned count
    assert got == single


# A point whose block-sparse products cannot be planned: with n_max = 34 the labels
# run over [-34, 34] and the first environment's signed label sums span 137 values,
# more than the planner's 128-slot table, so the device planner records HOTRG_ENOTSUP
# in that point's status slot (the out-of-table elements are left out of every pass).
def enotsup_point(H, prec):
    return H.params(1.0, 0.5, 34, 4, 1, prec=prec, block_sparse=1)


@pytest.mark.parametrize("prec_name", ["FP64", "SPLIT_BF16"])
def test_batch_device_failure_fails_that_point_alone(H, C, prec_name):
    prec = getattr(H, prec_name)
    good = [H.params(*pt, prec=prec, block_sparse=1) for pt in BATCH[:3]]
    single = [C.run([p])[0].lnz_per_site for p in good]
    pts = [good[0], enotsup_point(H, prec), good[1], good[2]]
    for _ in range(2):  # the second call replays every class from its graph, the failing one too
        got = H.hotrg_run_batch(C.handle, pts, nstreams=2, check=False)
        assert got[1].status == H.ENOTSUP
        assert [got[i].status for i in (0, 2, 3)] == [0, 0, 0]
        assert [got[i].lnz_per_site for i in (0, 2, 3)] == single
    # with invalid parameters on the host as well: each failing entry fails alone
    pts.insert(2, H.params(1.0, 1.5, 2, 12, 4, prec=prec))
    got = H.hotrg_run_batch(C.handle, pts, nstreams=3, check=False)
    assert got[1].status == H.ENOTSUP and got[2].status == H.EINVAL
    assert [got[i].lnz_per_site for i in (0, 3, 4)] == single


def test_run_device_failure_does_not_leak_into_the_next_point(H, C):
    got = H.hotrg_run(C.handle, [enotsup_point(H, H.SPLIT_BF16), H.params(*BATCH[0], prec=H.SPLIT_BF16)],
                      check=False)
    assert got[0].status == H.ENOTSUP and got[1].status == 0
    ref = OH.run_gxy(*BATCH[0]).lnz_per_site
    assert abs(got[1].lnz_per_site - ref) < 1e-9
