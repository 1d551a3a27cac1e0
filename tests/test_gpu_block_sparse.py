"""Block-sparse coarse contraction (block_sparse = 1) against the oracle and
against the dense split form.

The charge blocks hold every nonzero product of the dense contraction, so the
result equals the dense form's up to the split form's own error (the slices
accumulate over different exact chunks once the zeros are dropped), and the
oracle's within the split form's tolerance.
"""
import numpy as np
import pytest

from oracle import gxy
from oracle import hotrg as OH

from parity_points import BATCH, DRIFT_SHAPES, FP64_SHAPES, SPLIT_SHAPES

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


@pytest.mark.parametrize("beta,delta,nm,dcut,steps", SPLIT_SHAPES)
def test_block_sparse_lnz_against_oracle(H, C, beta, delta, nm, dcut, steps):
    ref = OH.run_gxy(beta, delta, nm, dcut, steps)
    bs = C.run([H.params(beta, delta, nm, dcut, steps, prec=H.SPLIT_BF16, block_sparse=1)])[0]
    dense = C.run([H.params(beta, delta, nm, dcut, steps, prec=H.SPLIT_BF16)])[0]
    assert bs.status == 0
    assert abs(bs.lnz_per_site - ref.lnz_per_site) <= 1e-9, bs.lnz_per_site - ref.lnz_per_site
    # both carry the split form's ~1e-11..1e-10 error, from different exact chunks (the blocks drop zeros)
    assert abs(bs.lnz_per_site - dense.lnz_per_site) <= 2e-10
    for k, rs in enumerate(ref.steps):
        assert bs.step[k].dprime == rs.Dp
        # the side is compared where the eps_1 / eps_2 decision is well conditioned (as in the
        # FP64 parity tests): away from the 1e-6 margin and above rounding-level discarded weight
        margin = abs(rs.eps_right - rs.eps_left * (1 - 1e-6)) / max(abs(rs.eps_left), 1e-300)
        if margin > 1e-9 and rs.eps_left > 1e-13:
            assert bs.step[k].side == rs.side
        assert abs(bs.step[k].ln_c - rs.ln_c) <= 1e-7 * max(1.0, abs(rs.ln_c))


@pytest.mark.parametrize("beta,delta,nm,dcut,steps", DRIFT_SHAPES)
def test_block_sparse_drifted_charge_window(H, C, beta, delta, nm, dcut, steps):
    # the kept U(1) window has drifted far from charge 0: the planner's value table
    # follows the products' label range instead of failing with HOTRG_ENOTSUP
    ref = OH.run_gxy(beta, delta, nm, dcut, steps)
    bs = C.run([H.params(beta, delta, nm, dcut, steps, prec=H.SPLIT_BF16, block_sparse=1)])[0]
    dense = C.run([H.params(beta, delta, nm, dcut, steps, prec=H.SPLIT_BF16)])[0]
    assert bs.status == 0
    assert abs(bs.lnz_per_site - ref.lnz_per_site) <= 1e-9, bs.lnz_per_site - ref.lnz_per_site
    assert abs(bs.lnz_per_site - dense.lnz_per_site) <= 2e-10


def test_block_sparse_z2_field(H, C):
    # h1 != 0 keeps only the parity of the charge: two blocks
    ref = OH.run_gxy(1.1, 0.4, 3, 16, 14, h1=0.03)
    bs = C.run([H.params(1.1, 0.4, 3, 16, 14, h1=0.03, prec=H.SPLIT_BF16, block_sparse=1)])[0]
    assert abs(bs.lnz_per_site - ref.lnz_per_site) <= 1e-9


def test_block_sparse_ising(H, C):
    ref = OH.hotrg_run(gxy.ising_tensor(0.6), gxy.ising_charges(), 30, 16, "z2")
    bs = C.run([H.params(0.6, 0.0, 0, 16, 30, tkind=H.T_ISING, prec=H.SPLIT_BF16, block_sparse=1)])[0]
    assert abs(bs.lnz_per_site - ref.lnz_per_site) <= 1e-9


def test_block_sparse_without_structure_is_the_dense_form(H, C):
    # h != 0 leaves no conserved label, and the cos(theta) impurity (parity odd) breaks the
    # Z2 rule of h1 != 0: both keep the dense path, bitwise equal
    a = C.run([H.params(1.1, 0.4, 2, 12, 10, h=0.02, prec=H.SPLIT_BF16, block_sparse=1)])[0]
    b = C.run([H.params(1.1, 0.4, 2, 12, 10, h=0.02, prec=H.SPLIT_BF16)])[0]
    assert a.lnz_per_site == b.lnz_per_site
    a = C.run([H.params(1.1, 0.4, 2, 12, 10, h1=0.02, prec=H.SPLIT_BF16, block_sparse=1)], imp_kind=H.T_IMP_M)[0]
    b = C.run([H.params(1.1, 0.4, 2, 12, 10, h1=0.02, prec=H.SPLIT_BF16)], imp_kind=H.T_IMP_M)[0]
    assert a.lnz_per_site == b.lnz_per_site and a.imp_ratio == b.imp_ratio


# The cos(2 theta) impurity (Eq. 3.21) at h = 0, h1 != 0 keeps the charge parity of the pure
# tensor, so its co-update (the impurity rule above T and below T) runs in the Z2 block form.
M1_POINTS = [(1.1, 0.4, 2, 10, 10, 0.03), (1.3, 0.2, 3, 16, 14, 0.02), (0.9, 0.3, 3, 13, 12, 0.01)]


@pytest.mark.parametrize("beta,delta,nm,dcut,steps,h1", M1_POINTS)
@pytest.mark.parametrize("prec_name,tol_lnz,tol_imp", [("SPLIT_BF16", 1e-9, 1e-8), ("FP64", 1e-10, 1e-10)])
def test_block_sparse_m1_impurity_against_oracle(H, C, beta, delta, nm, dcut, steps, h1, prec_name, tol_lnz,
                                                 tol_imp):
    prec = getattr(H, prec_name)
    ref = OH.run_gxy(beta, delta, nm, dcut, steps, h1=h1, impurity=gxy.IMP_M1)
    bs = C.run([H.params(beta, delta, nm, dcut, steps, h1=h1, prec=prec, block_sparse=1)], imp_kind=H.T_IMP_M1)[0]
    dense = C.run([H.params(beta, delta, nm, dcut, steps, h1=h1, prec=prec)], imp_kind=H.T_IMP_M1)[0]
    assert bs.status == 0
    assert abs(bs.lnz_per_site - ref.lnz_per_site) <= tol_lnz
    assert abs(bs.imp_ratio - ref.imp_ratio) <= tol_imp, (bs.imp_ratio, ref.imp_ratio)
    assert abs(bs.imp_ratio - dense.imp_ratio) <= tol_imp
    assert bs.imp_ratio != 0.0


def test_block_sparse_m1_impurity_is_cheaper(H, C):
    # the co-update runs per block: fewer algorithmic flops than the dense co-update
    p = H.params(1.1, 0.4, 3, 16, 12, h1=0.02, prec=H.SPLIT_BF16, block_sparse=1)
    H.hotrg_profile_enable(C.handle, True)
    C.run([p], imp_kind=H.T_IMP_M1)
    bs = H.hotrg_profile_read(C.handle)
    H.hotrg_profile_enable(C.handle, False)
    # three coarse contractions per step (pure, impurity above, impurity below), all per block
    assert bs.gemm_calls[1] == 3 * 3 * 12 and bs.operand_elems[1] > 0


def test_block_sparse_batch_replay_equals_single_runs(H, C):
    pts = [H.params(*pt, prec=H.SPLIT_BF16, block_sparse=1) for pt in BATCH]
    single = [C.run([p])[0].lnz_per_site for p in pts]
    for _ in range(2):  # the second call replays the captured graphs
        got = C.run_batch(pts, nstreams=3)
        assert [r.lnz_per_site for r in got] == single


@pytest.mark.parametrize("beta,delta,nm,dcut,steps", FP64_SHAPES)
def test_block_sparse_fp64_form_against_oracle(H, C, beta, delta, nm, dcut, steps):
    # the FP64 form per charge block (the block-sparse remark of §2.3.1 with FP64 FMA):
    # the FP64 parity bar of the dense FP64 form, per step and for ln Z / N
    ref = OH.run_gxy(beta, delta, nm, dcut, steps)
    bs = C.run([H.params(beta, delta, nm, dcut, steps, prec=H.FP64, block_sparse=1)])[0]
    dense = C.run([H.params(beta, delta, nm, dcut, steps, prec=H.FP64)])[0]
    assert bs.status == 0
    assert abs(bs.lnz_per_site - ref.lnz_per_site) <= 1e-10, bs.lnz_per_site - ref.lnz_per_site
    assert abs(bs.lnz_per_site - dense.lnz_per_site) <= 1e-12
    for k, rs in enumerate(ref.steps):
        g = bs.step[k]
        assert g.dprime == rs.Dp
        assert abs(g.ln_c - rs.ln_c) <= 1e-11 * max(1.0, abs(rs.ln_c)), (k, g.ln_c, rs.ln_c)
        assert abs(g.eps_left - rs.eps_left) <= 1e-13 + 1e-8 * abs(rs.eps_left)


def test_block_sparse_fp64_form_z2_and_ising(H, C):
    ref = OH.run_gxy(1.1, 0.4, 3, 16, 14, h1=0.03)
    bs = C.run([H.params(1.1, 0.4, 3, 16, 14, h1=0.03, prec=H.FP64, block_sparse=1)])[0]
    assert abs(bs.lnz_per_site - ref.lnz_per_site) <= 1e-10
    ref = OH.hotrg_run(gxy.ising_tensor(0.6), gxy.ising_charges(), 30, 16, "z2")
    bs = C.run([H.params(0.6, 0.0, 0, 16, 30, tkind=H.T_ISING, prec=H.FP64, block_sparse=1)])[0]
    assert abs(bs.lnz_per_site - ref.lnz_per_site) <= 1e-10


def test_block_sparse_fp64_form_counts_block_flops(H, C):
    p = H.params(1.0, 0.5, 2, 16, 12, prec=H.FP64, block_sparse=1)
    H.hotrg_profile_enable(C.handle, True)
    C.run([p])
    bs = H.hotrg_profile_read(C.handle)
    H.hotrg_profile_enable(C.handle, True)
    C.run([H.params(1.0, 0.5, 2, 16, 12, prec=H.SPLIT_BF16, block_sparse=1)])
    split = H.hotrg_profile_read(C.handle)
    H.hotrg_profile_enable(C.handle, False)
    # the same planner: the same algorithmic block flops in both forms
    assert bs.gemm_flops[1] == split.gemm_flops[1] and bs.gemm_flops[0] == split.gemm_flops[0]


def test_block_sparse_profile_counts_block_flops(H, C):
    p = H.params(1.0, 0.5, 2, 16, 12, prec=H.SPLIT_BF16, block_sparse=1)
    H.hotrg_profile_enable(C.handle, True)
    C.run([p])
    bs = H.hotrg_profile_read(C.handle)
    H.hotrg_profile_enable(C.handle, True)
    C.run([H.params(1.0, 0.5, 2, 16, 12, prec=H.SPLIT_BF16)])
    dense = H.hotrg_profile_read(C.handle)
    H.hotrg_profile_enable(C.handle, False)
    # the blocks hold a small fraction of the dense products
    assert 0 < bs.gemm_flops[1] < 0.5 * dense.gemm_flops[1]
    assert bs.gemm_calls[1] == dense.gemm_calls[1]


def random_charged_tensor(rng, qh, qv):
    """T[l,r,u,d] random where q_l + q_u = q_r + q_d, zero elsewhere (no mirror symmetry)."""
    Dh, Dv = len(qh), len(qv)
    T = rng.standard_normal((Dh, Dh, Dv, Dv))
    mask = (qh[:, None, None, None] + qv[None, None, :, None]) == (qh[None, :, None, None] + qv[None, None, None, :])
    T = T * mask
    return T / np.linalg.norm(T)


@pytest.mark.parametrize("seed", [0, 1])
def test_block_sparse_step_matches_dense_step(H, C, seed):
    # one hotrg_step on a tensor without left-right or up-down symmetry: the
    # block-sparse step must give the dense step's environments (eps_1, eps_2 in
    # their places) and the same output tensor in the same frame
    from gpu_util import dev_f64, dev_i32, to_dev, torch
    rng = np.random.default_rng(seed)
    qh = rng.integers(-2, 3, size=7).astype(np.int32)
    qv = rng.integers(-2, 3, size=6).astype(np.int32)
    T = random_charged_tensor(rng, qh, qv)
    Dh, Dv, dcut = len(qh), len(qv), 12
    outs = []
    for bs in (0, 1):
        p = H.params(1.0, 0.5, 2, dcut, 1, prec=H.SPLIT_BF16, block_sparse=bs)
        Tin, qhd, qvd = to_dev(T), to_dev(qh, torch.int32), to_dev(qv, torch.int32)
        Tout = dev_f64(Dh * Dh * 64 * 64)
        qout = dev_i32(64)
        info = torch.zeros(5, dtype=torch.float64, device="cuda")
        dp = H.hotrg_step(C.handle, p, Tin.data_ptr(), qhd.data_ptr(), qvd.data_ptr(), Dh, Dv, Tout.data_ptr(),
                          qout.data_ptr(), info.data_ptr())
        torch.cuda.synchronize()
        outs.append((dp, info.cpu().numpy().copy(), Tout[: Dv * Dv * dp * dp].cpu().numpy().copy(),
                     qout[:dp].cpu().numpy().copy()))
    (d0, i0, t0, q0), (d1, i1, t1, q1) = outs
    assert d0 == d1 == dcut
    assert abs(i0[1] - i1[1]) <= 1e-9 * i0[1] and abs(i0[2] - i1[2]) <= 1e-9 * i0[2], (i0[1:3], i1[1:3])
    assert abs(i0[1] - i0[2]) > 1e-6 * i0[1]  # the two sides differ on this tensor
    assert np.array_equal(q0, q1)
    assert np.abs(t0 - t1).max() <= 1e-9 * np.abs(t0).max()


# Tile shapes of the tensor-core products (hotrg_set_tiles): 128 or 64 output columns per
# tile, for the environments and the coarse contraction separately.  The products of every
# output element are the same; only the tiling and the TMEM double buffering differ.
@pytest.mark.parametrize("tiles", [(64, 64), (128, 64), (64, 128)])
@pytest.mark.parametrize("beta,delta,nm,dcut,steps", SPLIT_SHAPES[:4] + DRIFT_SHAPES[:1])
def test_tile_shapes_match_oracle(H, C, tiles, beta, delta, nm, dcut, steps):
    ref = OH.run_gxy(beta, delta, nm, dcut, steps)
    try:
        C.set_tiles(128, 128)
        base = C.run([H.params(beta, delta, nm, dcut, steps, prec=H.SPLIT_BF16, block_sparse=1)])[0]
        C.set_tiles(*tiles)
        got = C.run([H.params(beta, delta, nm, dcut, steps, prec=H.SPLIT_BF16, block_sparse=1)])[0]
    finally:
        C.set_tiles(128, 128)
    assert got.status == 0
    assert abs(got.lnz_per_site - ref.lnz_per_site) <= 1e-9
    assert abs(got.lnz_per_site - base.lnz_per_site) <= 1e-12, got.lnz_per_site - base.lnz_per_site


def test_tile_autotuner_and_graph_rebuild(H, C):
    pts = [H.params(*pt, prec=H.SPLIT_BF16, block_sparse=1) for pt in BATCH[:4]]
    single = [C.run([p])[0].lnz_per_site for p in pts]
    try:
        (e, c), secs = C.autotune_tiles(pts, nstreams=2)
        assert e in (64, 128) and c in (64, 128) and len(secs) == 4 and all(t > 0 for t in secs)
        # the worker graphs were rebuilt for the chosen shapes: the batch still equals the single runs
        got = C.run_batch(pts, nstreams=2)
        assert max(abs(r.lnz_per_site - x) for r, x in zip(got, single)) <= 1e-12
        with pytest.raises(H.HotrgError):
            C.set_tiles(96, 128)
    finally:
        C.set_tiles(128, 128)
