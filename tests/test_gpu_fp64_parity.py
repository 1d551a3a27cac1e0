"""Parity of the CUDA FP64 form against the oracle (element by element where
the quantity is gauge invariant: ln c_k, eps_1, eps_2, side, D', ln Z/N,
impurity ratios; element by element for the initial tensors)."""
import math

import numpy as np
import pytest

from oracle import exact, gxy
from oracle import hotrg as OH
from oracle import observables as OO

pytestmark = pytest.mark.gpu

from gpu_util import ctx as make_ctx, dev_f64, dev_i32, to_dev, torch  # noqa: E402
from parity_points import FP64_SHAPES  # noqa: E402


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


KINDS = {"pure": 0, "imp_m": 1, "imp_m1": 2}


@pytest.mark.parametrize("beta,delta,nm,h,h1,kind", [
    (1.0, 0.5, 2, 0.0, 0.0, "pure"), (1.6, 0.3, 4, 0.0, 0.0, "pure"), (0.7, 0.0, 3, 0.0, 0.0, "pure"),
    (1.1, 0.4, 3, 0.05, 0.0, "pure"), (1.1, 0.4, 3, 0.0, 0.04, "pure"), (1.1, 0.4, 3, 0.03, 0.02, "imp_m"),
    (1.3, 0.2, 2, 0.0, 0.05, "imp_m1"), (0.9, 1.0, 5, 0.0, 0.0, "pure"), (1.2, 0.6, 0, 0.0, 0.0, "pure"),
])
def test_init_tensor_elementwise(H, C, beta, delta, nm, h, h1, kind):
    p = H.params(beta, delta, nm, 8, 1, h=h, h1=h1)
    D0 = 2 * nm + 1
    T = dev_f64(D0 ** 4)
    q = dev_i32(D0)
    H.hotrg_init_tensor(C.handle, p, KINDS[kind], T.data_ptr(), q.data_ptr())
    torch.cuda.synchronize()
    ref = gxy.site_tensor(beta, delta, nm, h, h1, {"pure": gxy.PURE, "imp_m": gxy.IMP_M, "imp_m1": gxy.IMP_M1}[kind])
    got = T.cpu().numpy().reshape(D0, D0, D0, D0)
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) <= 1e-14 * scale
    qref = gxy.leg_charges(nm, gxy.symmetry_of(h, h1))
    assert np.array_equal(q.cpu().numpy(), qref)


def test_init_ising(H, C):
    p = H.params(0.4, 0.0, 0, 4, 1, tkind=H.T_ISING)
    T = dev_f64(16)
    q = dev_i32(2)
    H.hotrg_init_tensor(C.handle, p, H.T_ISING, T.data_ptr(), q.data_ptr())
    torch.cuda.synchronize()
    assert np.allclose(T.cpu().numpy().reshape(2, 2, 2, 2), gxy.ising_tensor(0.4), rtol=1e-15, atol=1e-15)


def compare_run(res, ref, lnz_tol, step_rtol=1e-11, eps_atol=1e-13):
    assert res.status == 0
    assert abs(res.lnz_per_site - ref.lnz_per_site) <= lnz_tol, (res.lnz_per_site, ref.lnz_per_site)
    assert abs(res.ln_c0 - ref.ln_c0) <= 1e-14 * max(1.0, abs(ref.ln_c0))
    for k, rs in enumerate(ref.steps):
        g = res.step[k]
        assert g.dprime == rs.Dp
        assert abs(g.ln_c - rs.ln_c) <= step_rtol * max(1.0, abs(rs.ln_c)), (k, g.ln_c, rs.ln_c)
        assert abs(g.eps_left - rs.eps_left) <= eps_atol + 1e-8 * abs(rs.eps_left), (k, g.eps_left, rs.eps_left)
        if not math.isnan(rs.eps_right):
            assert abs(g.eps_right - rs.eps_right) <= eps_atol + 1e-8 * abs(rs.eps_right)
            # same side unless the oracle's own decision sits within rounding of the 1e-6 margin
            margin = abs(rs.eps_right - rs.eps_left * (1 - 1e-6)) / max(abs(rs.eps_left), 1e-300)
            if margin > 1e-9 and rs.eps_left > 1e-13:
                assert g.side == rs.side, (k, g.side, rs.side, rs.eps_left, rs.eps_right)


def test_small_config_lnz(H, C):
    """beta = 1.0, Delta = 0.5, n_max = 2 (D0 = 5), D_cut = 16, 20 steps (2^20 sites)."""
    ref = OH.run_gxy(1.0, 0.5, 2, 16, 20)
    res = C.run([H.params(1.0, 0.5, 2, 16, 20)])[0]
    compare_run(res, ref, 1e-10)


@pytest.mark.parametrize("beta,delta,nm,dcut,steps", FP64_SHAPES)
def test_varied_shapes(H, C, beta, delta, nm, dcut, steps):
    ref = OH.run_gxy(beta, delta, nm, dcut, steps)
    res = C.run([H.params(beta, delta, nm, dcut, steps)])[0]
    compare_run(res, ref, 1e-10)


def test_env_policy_left_only(H, C):
    ref = OH.run_gxy(1.0, 0.5, 2, 16, 12, env_policy=1)
    res = C.run([H.params(1.0, 0.5, 2, 16, 12, env_policy=1)])[0]
    compare_run(res, ref, 1e-10)
    assert all(res.step[k].side == 0 for k in range(12))


@pytest.mark.parametrize("nm,steps", [(1, 2), (2, 2), (1, 4)])
def test_exact_small_lattices(H, C, nm, steps):
    L = 2 if steps == 2 else 4
    T0 = gxy.site_tensor(1.0, 0.5, nm)
    ref = exact.tensor_network_lnz(T0, L, L) / (L * L)
    res = C.run([H.params(1.0, 0.5, nm, 10 ** 2 if steps == 4 else 128, steps)])[0]
    assert abs(res.lnz_per_site - ref) < 1e-13


@pytest.mark.parametrize("beta,tol", [(0.3, 1e-9), (0.6, 1e-9), (0.4406868, 1e-6)])
def test_ising_vs_onsager(H, C, beta, tol):
    res = C.run([H.params(beta, 0.0, 0, 16, 30, tkind=H.T_ISING)])[0]
    assert abs(res.lnz_per_site - exact.onsager_lnz(beta)) < tol
    ref = OH.hotrg_run(gxy.ising_tensor(beta), gxy.ising_charges(), 30, 16, "z2")
    assert abs(res.lnz_per_site - ref.lnz_per_site) < 1e-12


def test_delta0_equals_xy(H, C):
    g, x = C.run([H.params(1.3, 0.0, 4, 12, 16), H.params(1.3, 1.0, 2, 12, 16)])
    assert abs(g.lnz_per_site - x.lnz_per_site) < 1e-13


@pytest.mark.parametrize("h,h1,kind", [(0.0, 0.03, "imp_m1"), (0.04, 0.0, "imp_m"), (0.02, 0.01, "imp_m")])
def test_impurity_ratio(H, C, h, h1, kind):
    ref = OH.run_gxy(1.1, 0.4, 2, 10, 10, h=h, h1=h1, impurity={"imp_m": gxy.IMP_M, "imp_m1": gxy.IMP_M1}[kind])
    res = C.run([H.params(1.1, 0.4, 2, 10, 10, h=h, h1=h1)], imp_kind=KINDS[kind])[0]
    compare_run(res, ref, 1e-10)
    assert abs(res.imp_ratio - ref.imp_ratio) < 1e-10


def test_observables_api(H, C):
    args = (1.0, 0.5, 2, 8, 10)
    o = C.observables([H.params(*args)], hb=1e-3, hbar=0.01, dh=1e-3)[0]
    ref = OO.observables(*args, hb=1e-3, hbar=0.01, dh=1e-3)
    assert o.status == 0
    assert abs(o.lnz - ref.lnz) < 1e-10
    assert abs(o.cv - ref.cv) < 1e-3  # FD amplifies rounding by beta^2 / hb^2 = 1e6
    assert abs(o.m - ref.m) < 1e-10 and abs(o.m1 - ref.m1) < 1e-10
    assert abs(o.chi - ref.chi) < 1e-6 and abs(o.chi1 - ref.chi1) < 1e-6


def test_step_entry_point_matches_run(H, C):
    # two explicit steps through hotrg_step == the first two steps of hotrg_run
    beta, delta, nm, dcut = 1.2, 0.5, 2, 12
    p = H.params(beta, delta, nm, dcut, 2)
    D0 = 2 * nm + 1
    T0 = gxy.site_tensor(beta, delta, nm)
    c0 = np.linalg.norm(T0)
    T = to_dev(T0 / c0)
    q = to_dev(gxy.leg_charges(nm, "u1"), torch.int32)
    info = torch.zeros(10 * 5, dtype=torch.float64, device="cuda")
    T1 = dev_f64(D0 * D0 * 25 * 25)
    q1 = dev_i32(64)
    dp = H.hotrg_step(C.handle, p, T.data_ptr(), q.data_ptr(), q.data_ptr(), D0, D0, T1.data_ptr(),
                      q1.data_ptr(), info.data_ptr())
    torch.cuda.synchronize()
    ref = OH.run_gxy(beta, delta, nm, dcut, 2)
    assert dp == ref.steps[0].Dp
    assert abs(info[0].item() - ref.steps[0].ln_c) < 1e-13
    # gauge-invariant check of the output tensor: its closing trace and norm
    Tn = T1[: D0 * D0 * dp * dp].cpu().numpy().reshape(D0, D0, dp, dp)
    assert abs(np.linalg.norm(Tn) - 1.0) < 1e-14
    Tref, _, _, _, _ = OH.hotrg_step(T0 / c0, gxy.leg_charges(nm, "u1"), gxy.leg_charges(nm, "u1"), dcut)
    assert abs(np.einsum("xxyy->", Tn) - np.einsum("xxyy->", Tref)) < 1e-13


def test_invalid_parameters_are_rejected(H, C):
    bad = [H.params(-1.0, 0.5, 2, 8, 4), H.params(1.0, 1.5, 2, 8, 4), H.params(1.0, 0.5, -1, 8, 4),
           H.params(1.0, 0.5, 2, 0, 4), H.params(1.0, 0.5, 2, 8, 65), H.params(1.0, 0.5, 2, 8, 4, h=-0.1)]
    for p in bad:
        with pytest.raises(H.HotrgError) as e:
            C.run([p])
        assert e.value.status == H.EINVAL
    # the context stays usable
    assert C.run([H.params(1.0, 0.5, 1, 4, 3)])[0].status == 0
