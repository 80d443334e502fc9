"""gmg_level_smooth_noalloc: the level smoother for callers that cannot call
cudaMalloc while they run (their device memory belongs to another allocator,
or they cannot pay the synchronisation of cudaMalloc/cudaFree).  It keeps the
recurrence's second vector in the library's static scratch array; its result
must equal gmg_level_smooth's with a caller buffer, call after call."""
import numpy as np
import pytest

from paper_1904_03317_gb300 import gmg as G
from paper_1904_03317_gb300 import inputs

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 8 << 20


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03317_gb300 import build
    build.build()
    return T


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_noalloc_smoother_matches_caller_buffer_version(torch, prec):
    w = inputs.poisson3d_sphere(2, 2)
    ctx = G.Context(0)
    mesh = G.build_mesh(w)
    H = G.Hierarchy(ctx, mesh, w.degree, cheb_degree=w.cheb_degree, vcycle_prec=prec)
    dt = torch.float64 if prec == G.PREC_FP64 else torch.float32
    esz = 8 if prec == G.PREC_FP64 else 4
    rng = np.random.default_rng(5)
    checked = 0
    for level in range(1, H.info.n_levels):
        n = len(H.export(G.EXPORT_LEVEL_KEYS, level))
        cls = H.export(G.EXPORT_LEVEL_CLASS, level)
        if n * esz > SCRATCH_BYTES:
            continue
        s_mask = torch.tensor(cls == 1, device="cuda")
        g = torch.tensor(rng.uniform(-1, 1, n), dtype=dt, device="cuda") * s_mask
        u_ref = torch.zeros(n, dtype=dt, device="cuda")
        u_new = torch.zeros(n, dtype=dt, device="cuda")
        tmp = torch.zeros(n, dtype=dt, device="cuda")
        kept_ref = [torch.empty_like(u_ref) for _ in range(2)]
        kept_new = [torch.empty_like(u_ref) for _ in range(2)]
        torch.cuda.synchronize()
        # every tensor of this level exists now, and nothing below allocates
        # until the window closes: the no-allocation calls, the first one
        # included, must leave the device's free memory unchanged (the
        # library looked the array up when H was built)
        free_before = torch.cuda.mem_get_info()[0]
        # two calls in a row: from zero, then from the first result
        for i, from_zero in enumerate((True, False)):
            H.level_smooth(level, g, u_ref, tmp, from_zero)
            H.level_smooth_noalloc(level, g, u_new, from_zero)
            kept_ref[i].copy_(u_ref)
            kept_new[i].copy_(u_new)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        # both paths launch the same kernels on the same values, so they
        # agree bit for bit
        for i in range(2):
            assert torch.equal(kept_new[i], kept_ref[i])
            assert float(kept_ref[i].abs().max()) > 0.0
        checked += 1
    assert checked >= 2


def test_noalloc_smoother_rejects_aliased_vectors(torch):
    w = inputs.poisson3d_sphere(2, 0)
    ctx = G.Context(0)
    H = G.Hierarchy(ctx, G.build_mesh(w), w.degree, cheb_degree=w.cheb_degree, vcycle_prec=G.PREC_FP32)
    n = len(H.export(G.EXPORT_LEVEL_KEYS, 1))
    u = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(G.GmgError) as e:
        H.level_smooth_noalloc(1, u, u, True)
    assert e.value.status == G.EINVAL


def test_noalloc_smoother_rejects_levels_beyond_the_scratch(torch):
    w = inputs.poisson3d_sphere(4, 0)  # level 4: 64^3 cells, 2^21 slots of 8 bytes > 8 MiB
    ctx = G.Context(0)
    H = G.Hierarchy(ctx, G.build_mesh(w), w.degree, cheb_degree=w.cheb_degree, vcycle_prec=G.PREC_FP64)
    n = len(H.export(G.EXPORT_LEVEL_KEYS, 4))
    assert n * 8 > SCRATCH_BYTES
    g = torch.zeros(n, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(g)
    with pytest.raises(G.GmgError) as e:
        H.level_smooth_noalloc(4, g, u, True)
    assert e.value.status == G.EINVAL and "static scratch" in str(e.value)
