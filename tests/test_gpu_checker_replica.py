"""The checkerboard-coefficient workload (a in {1, 100} on the 4^3 subcubes,
random refinement at the subcube planes) on a replica of its generator that
the FP64 oracle can solve: 2 global rounds and random rounds to level 4
(212k unknowns; the full configuration has 5 and 9 and 100.7M unknowns).
Iteration counts and the error of the GPU solutions against the oracle's."""
import numpy as np
import pytest

from oracle import gmg as ogmg
from paper_1904_03317_gb300 import gmg as G
from paper_1904_03317_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def case():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03317_gb300 import build
    build.build()
    w = inputs.checkerboard3d(2, 4)
    O = ogmg.setup(w)
    b = inputs.random_rhs(w.seed, O.disc.n)
    return torch, w, O, b


def test_checker_replica_against_oracle(case):
    torch, w, O, b = case
    ref = ogmg.solve(O, b, 1e-8)
    tight = ogmg.solve(O, b, 1e-13).x
    lam = [lev.lam for lev in O.levels]
    ctx = G.Context(0)
    m = G.build_mesh(w)
    H64 = G.Hierarchy(ctx, m, w.degree, w.coeff, cheb_degree=w.cheb_degree, vcycle_prec=G.PREC_FP64,
                      fixed_lambda=lam)
    H32 = G.Hierarchy(ctx, m, w.degree, w.coeff, cheb_degree=w.cheb_degree, vcycle_prec=G.PREC_FP32)
    db = torch.tensor(b, dtype=torch.float64, device="cuda")
    x64, x32 = torch.zeros_like(db), torch.zeros_like(db)
    s64 = H64.solve(db, x64, tol=1e-8)
    s32 = H32.solve(db, x32, tol=1e-8)
    assert s64.converged and abs(s64.iterations - ref.iterations) <= 1
    assert s32.converged and abs(s32.iterations - ref.iterations) <= 1
    err32 = float(np.linalg.norm(x32.cpu().numpy() - tight) / np.linalg.norm(tight))
    err_ref = float(np.linalg.norm(ref.x - tight) / np.linalg.norm(tight))
    # the FP32-V-cycle solution is as close to the converged answer as the
    # oracle's own 1e-8 solution, up to a small factor
    assert err32 <= 10 * err_ref + 1e-12
    H64.solve(db, x64, fixed_iterations=ref.iterations)
    err64 = float(np.linalg.norm(x64.cpu().numpy() - ref.x) / np.linalg.norm(ref.x))
    assert err64 < 1e-10
    print(f"checker replica: n={O.disc.n} its oracle={ref.iterations} gpu64={s64.iterations} gpu32={s32.iterations} "
          f"err32_vs_converged={err32:.2e} oracle_err={err_ref:.2e} gpu64_vs_oracle_same_its={err64:.2e}")
