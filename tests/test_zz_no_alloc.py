"""cs_recover_gomp_noalloc, the entry point for callers that cannot allocate device
memory while they recover a cube, against the context-based cs_recover_gomp.

Two calls in a row, on two different dictionaries and cubes, must each reproduce the
context-based result: the second call re-derives the shared static scratch the first
call left behind.  Collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

from gpu_common import REL_L2_FP32, Problem, gpu_run, library, rel_l2, support

pytestmark = pytest.mark.gpu


def _noalloc_run(cs, torch, A, pr, kappa, G):
    P = pr.P
    Ad = torch.from_numpy(A).cuda()
    Yd = torch.from_numpy(pr.Y).cuda()
    Xd = torch.full((P, pr.N), float("nan"), device="cuda")
    it = torch.full((P,), -1, device="cuda", dtype=torch.int32)
    opts = cs.make_opts(iters_out=it)
    cs.cs_recover_gomp_noalloc(Ad, pr.M, pr.N, Yd, Xd, kappa, G, opts=opts)
    torch.cuda.synchronize()
    return Xd.cpu().numpy(), it.cpu().numpy()


def test_noalloc_matches_context_call_on_two_calls_in_a_row():
    cs = library()
    import torch
    cases = [(Problem(80, 200, 32 * 9 + 5, "powerlaw", seed=2, noise_var=1e-3), 20, 4),
             (Problem(48, 120, 32 * 8 + 3, "sparse", seed=1, S=8), 8, 2)]
    for pr, kappa, G in cases:
        ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
        A = cs.cs_get_dictionary(ctx)
        Xref, itref, _ = gpu_run(cs.cs_recover_gomp, ctx, pr.Y, pr.N, kappa, G)
        cs.cs_destroy(ctx)
        Xn, itn = _noalloc_run(cs, torch, A, pr, kappa, G)
        assert np.all(support(Xn) == support(Xref))
        assert rel_l2(Xn, Xref) <= REL_L2_FP32
        assert np.array_equal(itn, itref)


def test_noalloc_rejects_oversize_shapes_and_host_memory():
    cs = library()
    import torch
    A = torch.zeros((128, 256), dtype=torch.float64, device="cuda")
    Y = torch.zeros((4, 128), device="cuda")
    X = torch.zeros((4, 256), device="cuda")
    with pytest.raises(cs.CsError) as e:
        cs.cs_recover_gomp_noalloc(A, 128, 256, Y, X, 8, 2)
    assert e.value.status == cs.CS_ERR_SHAPE and "static scratch" in str(e.value)
    A = torch.zeros((48, 120), dtype=torch.float64, device="cuda")
    Yh = np.zeros((4, 48), dtype=np.float32)
    Xh = np.zeros((4, 120), dtype=np.float32)
    with pytest.raises(cs.CsError) as e:
        cs.cs_recover_gomp_noalloc(A, 48, 120, Yh, Xh, 8, 2)
    assert e.value.status == cs.CS_ERR_ARG
