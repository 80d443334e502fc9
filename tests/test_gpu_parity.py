"""GPU parity: every step of the solve path, called through the C ABI, against
the FP64 oracle on the same seeded inputs.

FP64 path: element-wise agreement to 1e-11 relative (the two sides differ
only in rounding order); full solve to 1e-10 relative at the oracle's
iteration count and iteration counts within +-1.  FP32 V-cycle: level
operators within FP32 rounding (1e-5 relative), and the outer FP64 CG still
reaches the 1e-8 relative residual.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import gmg as ogmg
from paper_1904_03317_gb300 import gmg as G
from tests.helpers import workload_rhs, from_slots, level_maps, oracle_hierarchy, small_workloads, to_slots

pytestmark = pytest.mark.gpu

NAMES = list(small_workloads())


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03317_gb300 import build
    build.build()
    return T


_cache = {}


def gpu_hier(torch, name, prec=G.PREC_FP64, fixed=True, solve_graph=True):
    key = (name, prec, fixed, solve_graph)
    if key not in _cache:
        O = oracle_hierarchy(name)
        w = small_workloads()[name]
        lam = [lev.lam for lev in O.levels] if fixed else None
        ctx = G.Context(0)
        m = G.build_mesh(w)
        H = G.Hierarchy(ctx, m, w.degree, w.coeff, cheb_degree=O.cheb_degree, vcycle_prec=prec,
                        fixed_lambda=lam, solve_graph=solve_graph)
        _cache[key] = (O, H, ctx, m)
    return _cache[key][:2]


def dev(torch, a, prec=G.PREC_FP64):
    dt = torch.float64 if prec == G.PREC_FP64 else torch.float32
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def host(t):
    return t.double().cpu().numpy()


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_level_apply(torch, name, prec):
    O, H = gpu_hier(torch, name, prec)
    rng = np.random.default_rng(11)
    for l in range(1, len(O.levels)):
        lev = O.levels[l]
        idx, cls = level_maps(H, O, l)
        x = rng.uniform(-1, 1, len(lev.keys))
        want = np.zeros(len(lev.keys))
        want[lev.S] = lev.A_S @ x[lev.S] + lev.A_SI @ x[lev.I]
        xs = dev(torch, to_slots(x, idx, len(idx)), prec)
        ys = torch.zeros_like(xs)
        H.level_apply(l, xs, ys)
        torch.cuda.synchronize()
        got = host(ys)
        assert np.all(got[cls != 1] == 0.0)  # only S slots written
        tol = 1e-11 if prec == G.PREC_FP64 else 2e-5
        assert rel_err(from_slots(got, idx, len(lev.keys))[lev.S], want[lev.S]) < tol


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_residual_restrict(torch, name, prec):
    O, H = gpu_hier(torch, name, prec)
    rng = np.random.default_rng(12)
    for l in range(1, len(O.levels)):
        lev, levc = O.levels[l], O.levels[l - 1]
        idx, cls = level_maps(H, O, l)
        u = np.zeros(len(lev.keys)); u[lev.S] = rng.uniform(-1, 1, len(lev.S))
        g = np.zeros(len(lev.keys)); g[lev.S] = rng.uniform(-1, 1, len(lev.S))
        t = np.zeros(len(lev.keys))
        t[lev.S] = g[lev.S] - lev.A_S @ u[lev.S]
        t[lev.I] = -lev.A_IS @ u[lev.S]
        want = lev.P.T @ t
        idc, clsc = level_maps(H, O, l - 1)
        gc = torch.zeros(len(idc), dtype=torch.float64 if prec == G.PREC_FP64 else torch.float32, device="cuda")
        H.level_residual_restrict(l, dev(torch, to_slots(u, idx, len(idx)), prec),
                                  dev(torch, to_slots(g, idx, len(idx)), prec), gc)
        torch.cuda.synchronize()
        got = from_slots(host(gc), idc, len(levc.keys))
        tol = 1e-11 if prec == G.PREC_FP64 else 2e-5
        assert rel_err(got, want) < tol
        assert not np.any(want[levc.I])  # complete layer: R lands on S nodes only


@pytest.mark.parametrize("name", NAMES)
def test_prolongate(torch, name):
    O, H = gpu_hier(torch, name)
    rng = np.random.default_rng(13)
    for l in range(1, len(O.levels)):
        lev, levc = O.levels[l], O.levels[l - 1]
        idx, cls = level_maps(H, O, l)
        idc, clsc = level_maps(H, O, l - 1)
        uc = rng.uniform(-1, 1, len(levc.keys))
        u = np.zeros(len(lev.keys)); u[lev.S] = rng.uniform(-1, 1, len(lev.S))
        pu = lev.P @ uc
        ud = dev(torch, to_slots(u, idx, len(idx)))
        u2 = torch.zeros_like(ud)
        H.level_prolongate(l, dev(torch, to_slots(uc, idc, len(idc))), ud, u2)
        torch.cuda.synchronize()
        got = from_slots(host(ud), idx, len(lev.keys))
        got2 = from_slots(host(u2), idx, len(lev.keys))
        want = u.copy(); want[lev.S] += pu[lev.S]; want[lev.I] = pu[lev.I]
        assert rel_err(got, want) < 1e-13
        assert rel_err(got2[lev.I], pu[lev.I]) < 1e-13 if len(lev.I) else True
        assert np.all(got2[lev.S] == 0.0)


@pytest.mark.parametrize("name", NAMES)
def test_inverse_diagonal(torch, name):
    O, H = gpu_hier(torch, name)
    for l in range(1, len(O.levels)):
        lev = O.levels[l]
        idx, cls = level_maps(H, O, l)
        out = torch.zeros(len(idx), dtype=torch.float64, device="cuda")
        H.level_inv_diag(l, out)
        torch.cuda.synchronize()
        got = host(out)
        assert np.all(got[cls != 1] == 0.0)
        assert rel_err(from_slots(got, idx, len(lev.keys))[lev.S], lev.dinv) < 1e-13


@pytest.mark.parametrize("name", NAMES)
def test_fp32_inverse_diagonal_is_the_rounded_fp64_one(torch, name):
    """An FP32 hierarchy's inverse diagonal is its FP64 one rounded to
    nearest (numpy's float32 cast), bit for bit: the two precisions share
    the diagonal's FP64 evaluation."""
    O, H64 = gpu_hier(torch, name)
    _, H32 = gpu_hier(torch, name, G.PREC_FP32)
    for l in range(1, len(O.levels)):
        n = int(H64.info.slots[l])
        d64 = torch.zeros(n, dtype=torch.float64, device="cuda")
        d32 = torch.zeros(n, dtype=torch.float32, device="cuda")
        H64.level_inv_diag(l, d64)
        H32.level_inv_diag(l, d32)
        torch.cuda.synchronize()
        want = d64.cpu().numpy().astype(np.float32)
        assert np.array_equal(d32.cpu().numpy().view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("name", NAMES)
def test_coarse_solve(torch, name):
    O, H = gpu_hier(torch, name)
    lev = O.levels[0]
    idx, cls = level_maps(H, O, 0)
    rng = np.random.default_rng(14)
    g = rng.uniform(-1, 1, len(lev.keys))
    want = sla.cho_solve(O.coarse_chol, g)
    u0 = torch.zeros(len(idx), dtype=torch.float64, device="cuda")
    H.coarse_solve(dev(torch, to_slots(g, idx, len(idx))), u0)
    torch.cuda.synchronize()
    got = host(u0)
    assert np.all(got[cls == 3] == 0.0)
    assert rel_err(from_slots(got, idx, len(lev.keys)), want) < 1e-12


@pytest.mark.parametrize("name", NAMES)
def test_chebyshev_smoother(torch, name):
    O, H = gpu_hier(torch, name)
    rng = np.random.default_rng(15)
    m = O.cheb_degree
    for l in range(1, len(O.levels)):
        lev = O.levels[l]
        idx, cls = level_maps(H, O, l)
        g = np.zeros(len(lev.keys)); g[lev.S] = rng.uniform(-1, 1, len(lev.S))
        # from zero
        want = np.zeros(len(lev.keys))
        want[lev.S] = ogmg.chebyshev(lev.A_S, lev.dinv, np.zeros(len(lev.S)), g[lev.S], lev.lam, m, x0_is_zero=True)
        ud = torch.zeros(len(idx), dtype=torch.float64, device="cuda")
        tmp = torch.zeros_like(ud)
        gd = dev(torch, to_slots(g, idx, len(idx)))
        H.level_smooth(l, gd, ud, tmp, True)
        torch.cuda.synchronize()
        assert rel_err(from_slots(host(ud), idx, len(lev.keys)), want) < 1e-11
        # from a nonzero start with fixed interface values
        u0 = rng.uniform(-1, 1, len(lev.keys))
        want = u0.copy()
        want[lev.S] = ogmg.chebyshev(lev.A_S, lev.dinv, u0[lev.S], g[lev.S] - lev.A_SI @ u0[lev.I], lev.lam, m)
        ud = dev(torch, to_slots(u0, idx, len(idx)))
        H.level_smooth(l, gd, ud, tmp, False)
        torch.cuda.synchronize()
        assert rel_err(from_slots(host(ud), idx, len(lev.keys)), want) < 1e-11


@pytest.mark.parametrize("name", NAMES)
def test_chebyshev_smoother_fp32(torch, name):
    """The FP32 smoothers (full and partial bricks, single groups, groups at
    coefficient jumps) against the FP64 oracle: m Chebyshev steps in FP32
    from zero and from a nonzero start, to single-precision rounding."""
    O, H = gpu_hier(torch, name, G.PREC_FP32)
    rng = np.random.default_rng(18)
    m = O.cheb_degree
    for l in range(1, len(O.levels)):
        lev = O.levels[l]
        idx, cls = level_maps(H, O, l)
        g = np.zeros(len(lev.keys)); g[lev.S] = rng.uniform(-1, 1, len(lev.S))
        want = np.zeros(len(lev.keys))
        want[lev.S] = ogmg.chebyshev(lev.A_S, lev.dinv, np.zeros(len(lev.S)), g[lev.S], lev.lam, m, x0_is_zero=True)
        ud = torch.zeros(len(idx), dtype=torch.float32, device="cuda")
        tmp = torch.zeros_like(ud)
        gd = dev(torch, to_slots(g, idx, len(idx)), G.PREC_FP32)
        H.level_smooth(l, gd, ud, tmp, True)
        torch.cuda.synchronize()
        assert rel_err(from_slots(host(ud), idx, len(lev.keys)), want) < 5e-5
        u0 = rng.uniform(-1, 1, len(lev.keys))
        want = u0.copy()
        want[lev.S] = ogmg.chebyshev(lev.A_S, lev.dinv, u0[lev.S], g[lev.S] - lev.A_SI @ u0[lev.I], lev.lam, m)
        ud = dev(torch, to_slots(u0, idx, len(idx)), G.PREC_FP32)
        H.level_smooth(l, gd, ud, tmp, False)
        torch.cuda.synchronize()
        got = from_slots(host(ud), idx, len(lev.keys))
        assert rel_err(got[lev.S], want[lev.S]) < 5e-5
        assert np.array_equal(got[lev.I], u0[lev.I].astype(np.float32).astype(np.float64))  # I values kept


@pytest.mark.parametrize("name", NAMES)
def test_eigenvalue_estimates(torch, name):
    O, H = gpu_hier(torch, name, fixed=False)
    for l in range(1, len(O.levels)):
        assert H.info.lambda_max[l] == pytest.approx(O.levels[l].lam, rel=1e-10)


@pytest.mark.parametrize("name", NAMES)
def test_vcycle(torch, name):
    O, H = gpu_hier(torch, name)
    rng = np.random.default_rng(16)
    r = rng.uniform(-1, 1, O.disc.n)
    want = ogmg.vcycle(O, r)
    z = torch.zeros(O.disc.n, dtype=torch.float64, device="cuda")
    H.vcycle(dev(torch, r), z)
    torch.cuda.synchronize()
    assert rel_err(host(z), want) < 1e-11


@pytest.mark.parametrize("name", NAMES)
def test_vcycle_fp32(torch, name):
    O, H = gpu_hier(torch, name, G.PREC_FP32)
    rng = np.random.default_rng(17)
    r = rng.uniform(-1, 1, O.disc.n)
    want = ogmg.vcycle(O, r)
    z = torch.zeros(O.disc.n, dtype=torch.float64, device="cuda")
    H.vcycle(dev(torch, r), z)
    torch.cuda.synchronize()
    assert rel_err(host(z), want) < 1e-4
    # z is the FP32 level solution widened to FP64: every value is a float
    zh = host(z)
    assert np.array_equal(zh.astype(np.float32).astype(np.float64), zh)


@pytest.mark.parametrize("name", NAMES)
def test_active_apply(torch, name):
    O, H = gpu_hier(torch, name)
    rng = np.random.default_rng(18)
    x = rng.uniform(-1, 1, O.disc.n)
    y = torch.zeros(O.disc.n, dtype=torch.float64, device="cuda")
    H.apply(dev(torch, x), y)
    torch.cuda.synchronize()
    assert rel_err(host(y), O.disc.A @ x) < 1e-12


@pytest.mark.parametrize("name", NAMES)
def test_active_apply_wide_range(torch, name):
    """Inputs spanning sixteen decades, with exact zeros and subnormals: the
    leaf operator stays within FP64 rounding of |A| |x| in the max norm (the
    cubic-cell kernels split each group's values against its largest one)."""
    O, H = gpu_hier(torch, name)
    rng = np.random.default_rng(19)
    n = O.disc.n
    x = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-8, 8, n)
    x[rng.random(n) < 0.1] = 0.0
    x[rng.random(n) < 0.02] = 5e-324
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    H.apply(dev(torch, x), y)
    torch.cuda.synchronize()
    A = O.disc.A
    bound = (abs(A) @ np.abs(x)).max()
    assert np.all(np.isfinite(host(y)))
    assert np.abs(host(y) - A @ x).max() <= 1e-13 * bound


def test_active_apply_propagates_nan(torch):
    O, H = gpu_hier(torch, "3d_q2_patches")
    x = np.ones(O.disc.n)
    x[O.disc.n // 2] = np.nan
    y = torch.zeros(O.disc.n, dtype=torch.float64, device="cuda")
    H.apply(dev(torch, x), y)
    torch.cuda.synchronize()
    yh = host(y)
    assert np.isnan(yh).any()
    # the NaN reaches every row that couples to it
    rows = O.disc.A[:, O.disc.n // 2].nonzero()[0]
    assert np.all(np.isnan(yh[rows]))


@pytest.mark.parametrize("name", NAMES)
def test_level_apply_wide_range(torch, name):
    """FP64 level operators on inputs spanning sixteen decades, with exact
    zeros and subnormals: within FP64 rounding of |A| |x| in the max norm.
    On cubic cells the brick and single-group kernels split each brick's or
    group's values against its largest one (the leaf operator's scheme)."""
    O, H = gpu_hier(torch, name)
    rng = np.random.default_rng(23)
    for l in range(1, len(O.levels)):
        lev = O.levels[l]
        idx, cls = level_maps(H, O, l)
        n = len(lev.keys)
        x = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-8, 8, n)
        x[rng.random(n) < 0.1] = 0.0
        x[rng.random(n) < 0.02] = 5e-324
        want = lev.A_S @ x[lev.S] + lev.A_SI @ x[lev.I]
        bound = (abs(lev.A_S) @ np.abs(x[lev.S]) + abs(lev.A_SI) @ np.abs(x[lev.I])).max()
        xs = dev(torch, to_slots(x, idx, len(idx)))
        ys = torch.zeros_like(xs)
        H.level_apply(l, xs, ys)
        torch.cuda.synchronize()
        got = from_slots(host(ys), idx, n)[lev.S]
        assert np.all(np.isfinite(got))
        assert np.abs(got - want).max() <= 1e-13 * bound


def test_level_apply_propagates_nan(torch):
    """A NaN in the input reaches every S row of the level operator that
    couples to it (the split-integer kernels turn the outputs of the brick
    or group whose halo holds it into NaN)."""
    O, H = gpu_hier(torch, "3d_q2_patches")
    for l in range(1, len(O.levels)):
        lev = O.levels[l]
        idx, cls = level_maps(H, O, l)
        x = np.ones(len(lev.keys))
        k = len(lev.S) // 2
        x[lev.S[k]] = np.nan
        xs = dev(torch, to_slots(x, idx, len(idx)))
        ys = torch.zeros_like(xs)
        H.level_apply(l, xs, ys)
        torch.cuda.synchronize()
        got = from_slots(host(ys), idx, len(lev.keys))[lev.S]
        rows = lev.A_S[:, k].nonzero()[0]
        assert len(rows) > 0 and np.all(np.isnan(got[rows]))


@pytest.mark.parametrize("name", [n for n in NAMES if small_workloads()[n].coeff is None])
def test_rhs_sine(torch, name):
    O, H = gpu_hier(torch, name)
    b = torch.zeros(O.disc.n, dtype=torch.float64, device="cuda")
    H.assemble_rhs(b)
    torch.cuda.synchronize()
    assert rel_err(host(b), O.disc.rhs_sine()) < 1e-12


@pytest.mark.parametrize("seed", [0, 20190403, 2**64 - 1])
def test_rhs_random_equals_seeded_generator(torch, seed):
    """gmg_assemble_rhs(GMG_RHS_RANDOM, seed) is the seeded U[-1, 1) input of
    the variable-coefficient, batched and served workloads: the same counter
    generator as inputs.random_rhs, so the two agree bit for bit, in the
    canonical order, for every unknown (a ragged last block included)."""
    from paper_1904_03317_gb300 import inputs
    O, H = gpu_hier(torch, "3d_q2_checker")
    n = O.disc.n
    b = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    H.assemble_rhs(b, "random", seed)
    torch.cuda.synchronize()
    want = inputs.random_rhs(seed, n)
    assert np.array_equal(host(b), want)
    assert want.min() >= -1.0 and want.max() < 1.0 and n % 256 != 0


def test_rhs_rejects_unknown_kind(torch):
    O, H = gpu_hier(torch, "2d_q1_circle")
    b = torch.zeros(O.disc.n, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GmgError) as e:
        G._check(G.load_library().gmg_assemble_rhs(H.handle, 7, 0, G._ptr(b)), "gmg_assemble_rhs")
    assert e.value.status == G.EINVAL


def _rhs(O, w):
    from paper_1904_03317_gb300 import inputs
    return workload_rhs(O, w)


@pytest.mark.parametrize("name", NAMES)
def test_solve_fp64_matches_oracle(torch, name):
    O, H = gpu_hier(torch, name)
    w = small_workloads()[name]
    b = _rhs(O, w)
    ref = ogmg.solve(O, b, 1e-10)
    x = torch.zeros(O.disc.n, dtype=torch.float64, device="cuda")
    st = H.solve(dev(torch, b), x, tol=1e-10)
    assert abs(st.iterations - ref.iterations) <= 1
    # same iteration count: the iterates agree to rounding
    st = H.solve(dev(torch, b), x, fixed_iterations=ref.iterations)
    assert st.iterations == ref.iterations
    assert rel_err(host(x), ref.x) < 1e-10


@pytest.mark.parametrize("name", NAMES)
def test_solve_fp32_vcycle_reaches_tolerance(torch, name):
    O, H = gpu_hier(torch, name, G.PREC_FP32)
    w = small_workloads()[name]
    b = _rhs(O, w)
    x = torch.zeros(O.disc.n, dtype=torch.float64, device="cuda")
    st = H.solve(dev(torch, b), x, tol=1e-8)
    assert st.converged and st.rel_residual <= 1e-8
    xs = host(x)
    true_res = np.linalg.norm(b - O.disc.A @ xs) / np.linalg.norm(b)
    assert true_res < 2e-8
    ref = ogmg.solve(O, b, 1e-12)
    assert rel_err(xs, ref.x) < 1e-6


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_solve_graph_equals_stream(torch, name, prec):
    """The graph-mode loop performs the stream-mode operations in the same
    order, so iterates and statistics agree to rounding (the leaf operator
    and the restriction scatter with atomics, whose order varies from run to
    run: FP64 rounding for an FP64 V-cycle, FP32 rounding of the
    preconditioner for an FP32 one); the launch accounting agrees too."""
    O, Hg = gpu_hier(torch, name, prec)
    _, Hs = gpu_hier(torch, name, prec, solve_graph=False)
    w = small_workloads()[name]
    b = dev(torch, _rhs(O, w))
    xtol = 1e-10 if prec == G.PREC_FP64 else 1e-4
    for kw in (dict(tol=1e-9), dict(fixed_iterations=3)):
        xg = torch.full_like(b, 7.0)
        xs = torch.full_like(b, -7.0)
        Hg.profile_reset()
        sg = Hg.solve(b, xg, **kw)
        pg = Hg.profile_read()
        Hs.profile_reset()
        ss = Hs.solve(b, xs, **kw)
        ps = Hs.profile_read()
        assert sg.norm_b == ss.norm_b
        if prec == G.PREC_FP32 and "tol" in kw and sg.iterations != ss.iterations:
            # a residual within rounding of the tolerance may stop one pass apart
            assert abs(sg.iterations - ss.iterations) == 1 and sg.converged and ss.converged
            continue
        assert (sg.iterations, sg.converged) == (ss.iterations, ss.converged)
        assert abs(sg.rel_residual - ss.rel_residual) <= xtol * ss.rel_residual
        assert rel_err(host(xg), host(xs)) < xtol
        lg = {k: v["launches"] for k, v in pg.items()}
        ls = {k: v["launches"] for k, v in ps.items()}
        it = sg.iterations
        # graph mode adds one loop-control kernel before the loop and one per
        # pass
        assert lg.pop("other") == ls.pop("other") + 1 + it
        assert lg == ls
    # a second graph solve reuses the graph and starts from scratch again
    xg2 = torch.zeros_like(b)
    sg2 = Hg.solve(b, xg2, fixed_iterations=3)
    assert sg2.iterations == 3 and rel_err(host(xg2), host(xs)) < xtol


@pytest.mark.parametrize("solve_graph", [True, False])
def test_solve_error_paths(torch, solve_graph):
    O, H = gpu_hier(torch, "3d_q2_sphere", solve_graph=solve_graph)
    b = dev(torch, O.disc.rhs_sine())
    x = torch.zeros_like(b)
    st = H.solve(b, x, tol=1e-12, max_iter=2, raise_on_error=False)
    assert H.last_status == G.ENOTCONV and st.iterations == 2 and not st.converged
    bn = b.clone()
    bn[3] = float("nan")
    H.solve(bn, x, tol=1e-8, raise_on_error=False)
    assert H.last_status == G.ENAN
    z = torch.zeros_like(b)
    st = H.solve(z, x, tol=1e-8)
    assert st.iterations == 0 and torch.count_nonzero(x).item() == 0


VARIANTS = {
    "cheb_coarse": dict(smoother="chebyshev", coarse="chebyshev", degree=None),
    "cg_coarse": dict(smoother="chebyshev", coarse="cg", degree=None),
    "jacobi1_cg": dict(smoother="jacobi", coarse="cg", degree=1),
    "jacobi2_cheb": dict(smoother="jacobi", coarse="chebyshev", degree=2),
}


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("name", ["2d_q1_circle", "3d_q2_sphere", "3d_q2_checker"])
def test_solver_variants_match_oracle(torch, name, variant):
    """Chebyshev coarse solver (Sec. 4.1), unpreconditioned CG coarse solver and
    undamped Jacobi smoothing (Sec. 4.3) against the oracle's same variant,
    FP64 V-cycle: iteration counts within one; with the linear coarse solvers
    the iterates agree to 1e-10 at the oracle's count."""
    v = VARIANTS[variant]
    O = oracle_hierarchy(name)
    w = small_workloads()[name]
    deg = v["degree"] or O.cheb_degree
    lam = [lev.lam for lev in O.levels]
    ctx = G.Context(0)
    H = G.Hierarchy(ctx, G.build_mesh(w), w.degree, w.coeff, cheb_degree=deg, vcycle_prec=G.PREC_FP64,
                    fixed_lambda=lam,
                    smoother=G.SMOOTHER_JACOBI if v["smoother"] == "jacobi" else G.SMOOTHER_CHEBYSHEV,
                    coarse_solver={"cholesky": G.COARSE_CHOLESKY, "chebyshev": G.COARSE_CHEBYSHEV,
                                   "cg": G.COARSE_CG}[v["coarse"]])
    saved = (O.smoother, O.coarse, O.cheb_degree)
    try:
        O.smoother, O.cheb_degree = v["smoother"], deg
        ogmg.setup_coarse(O, v["coarse"])
        b = _rhs(O, w)
        ref = ogmg.solve(O, b, 1e-8)
        x = torch.zeros(O.disc.n, dtype=torch.float64, device="cuda")
        st = H.solve(dev(torch, b), x, tol=1e-8, max_iter=200)
        assert st.converged and abs(st.iterations - ref.iterations) <= 1
        true_res = np.linalg.norm(b - O.disc.A @ host(x)) / np.linalg.norm(b)
        assert true_res <= 2e-8
        if v["coarse"] != "cg":  # a linear preconditioner: same iterates to rounding
            st = H.solve(dev(torch, b), x, fixed_iterations=ref.iterations)
            assert rel_err(host(x), ref.x) < 1e-10
    finally:
        O.smoother, O.cheb_degree = saved[0], saved[2]
        ogmg.setup_coarse(O, saved[1])
        H.close()


@pytest.mark.parametrize("prec,tol", [(G.PREC_FP64, 1e-8), (G.PREC_FP32, 1e-3)])
def test_cg_coarse_solver_meets_its_tolerance(torch, prec, tol):
    """The unpreconditioned CG coarse solver (Sec. 4.3) iterates in the
    V-cycle's precision until ||g - A_0 u|| <= tol ||g||: on the Fichera
    coarse problem (279 unknowns) the true residual of its result, taken
    with the oracle's A_0 in FP64, meets the tolerance (1e-8 in FP64; the
    default 1e-3 in FP32, whose rounding stays far below it)."""
    name = "3d_q2_fichera"
    O = oracle_hierarchy(name)
    w = small_workloads()[name]
    H = G.Hierarchy(G.Context(0), G.build_mesh(w), w.degree, w.coeff, cheb_degree=w.cheb_degree,
                    vcycle_prec=prec, coarse_solver=G.COARSE_CG, coarse_tol=tol)
    lev = O.levels[0]
    idx, cls = level_maps(H, O, 0)
    rng = np.random.default_rng(23)
    for _ in range(2):
        g = rng.uniform(-1, 1, len(lev.keys))
        u0 = torch.zeros(len(idx), dtype=torch.float64 if prec == G.PREC_FP64 else torch.float32, device="cuda")
        H.coarse_solve(dev(torch, to_slots(g, idx, len(idx)), prec), u0)
        torch.cuda.synchronize()
        u = from_slots(host(u0), idx, len(lev.keys))
        res = np.linalg.norm(g - lev.A @ u) / np.linalg.norm(g)
        assert res <= 1.05 * tol, res
    H.close()


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_fichera_mf_setting_matches_oracle(torch, prec):
    """The Laplace example of Sec. 4.3 on the Fichera corner with the paper's
    "MF" solver: one undamped Jacobi step per smoothing, unpreconditioned CG
    on the coarse level, CG to 1e-10 with f = 1 (assembled on the device).
    The right-hand side equals the oracle's to 1e-12; FP64 V-cycles take the
    oracle's iteration count within one, FP32 V-cycles (the paper's single
    precision) reach the tolerance too; both solutions agree with the
    oracle's to the tolerance, and the true residual meets it."""
    from paper_1904_03317_gb300 import inputs
    w = inputs.fichera(3, 1)
    O = ogmg.setup(w)
    b_ref = O.disc.rhs_one()
    ref = ogmg.solve(O, b_ref, w.tol)
    assert ref.converged
    ctx = G.Context(0)
    H = G.Hierarchy(ctx, G.build_mesh(w), w.degree, w.coeff, cheb_degree=w.cheb_degree, vcycle_prec=prec,
                    smoother=G.SMOOTHER_JACOBI, coarse_solver=G.COARSE_CG)
    try:
        b = torch.zeros(O.disc.n, dtype=torch.float64, device="cuda")
        H.assemble_rhs(b, "one")
        torch.cuda.synchronize()
        assert rel_err(host(b), b_ref) < 1e-12
        x = torch.zeros_like(b)
        st = H.solve(b, x, tol=w.tol, max_iter=500)
        assert st.converged
        if prec == G.PREC_FP64:
            assert abs(st.iterations - ref.iterations) <= 1
        true_res = np.linalg.norm(b_ref - O.disc.A @ host(x)) / np.linalg.norm(b_ref)
        assert true_res <= 2 * w.tol
        assert rel_err(host(x), ref.x) < 1e-8
    finally:
        H.close()


@pytest.mark.parametrize("name", ["3d_q2_sphere", "3d_q2_checker", "3d_q2_fichera", "2d_q1_circle"])
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_deterministic_mode_is_bitwise_repeatable(torch, name, prec):
    """gmg_params.deterministic: the leaf operator and the restriction add to
    shared nodes one colour of elements at a time, without atomics, so
    repeated solves give the same bits, in graph and stream mode alike (the
    same operations in the same order); the FP64 result still agrees with
    the oracle to 1e-10 at the oracle's iteration count, and with the
    default (atomic) mode to rounding."""
    O = oracle_hierarchy(name)
    w = small_workloads()[name]
    lam = [lev.lam for lev in O.levels]
    ctx = G.Context(0)
    m = G.build_mesh(w)
    kw = dict(cheb_degree=O.cheb_degree, vcycle_prec=prec, fixed_lambda=lam)
    Hd = G.Hierarchy(ctx, m, w.degree, w.coeff, deterministic=True, **kw)
    Hs = G.Hierarchy(ctx, m, w.degree, w.coeff, deterministic=True, solve_graph=False, **kw)
    Ha = G.Hierarchy(ctx, m, w.degree, w.coeff, **kw)
    try:
        b = dev(torch, _rhs(O, w))
        ref = ogmg.solve(O, _rhs(O, w), 1e-8)
        xs = []
        for H in (Hd, Hd, Hs):
            x = torch.zeros_like(b)
            H.solve(b, x, fixed_iterations=ref.iterations)
            xs.append(x)
        torch.cuda.synchronize()
        assert torch.equal(xs[0], xs[1]) and torch.equal(xs[0], xs[2])
        xa = torch.zeros_like(b)
        Ha.solve(b, xa, fixed_iterations=ref.iterations)
        tol = 1e-10 if prec == G.PREC_FP64 else 1e-4
        assert rel_err(host(xs[0]), host(xa)) < tol
        if prec == G.PREC_FP64:
            assert rel_err(host(xs[0]), ref.x) < 1e-10
        y1, y2 = torch.zeros_like(b), torch.zeros_like(b)
        Hd.apply(b, y1)
        Hd.apply(b, y2)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
    finally:
        for H in (Hd, Hs, Ha):
            H.close()
