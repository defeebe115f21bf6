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


def _noalloc_run(cs, torch, A, pr, kappa, G, Y=None):
    P = pr.P
    Ad = torch.from_numpy(A).cuda()
    Yd = torch.from_numpy(pr.Y if Y is None else Y).cuda()
    Xd = torch.full((P, pr.N), float("nan"), device="cuda")
    it = torch.full((P,), -1, device="cuda", dtype=torch.int32)
    cv = torch.full((P,), 255, device="cuda", dtype=torch.uint8)
    opts = cs.make_opts(iters_out=it, converged_out=cv)
    cs.cs_recover_gomp_noalloc(Ad, pr.M, pr.N, Yd, Xd, kappa, G, opts=opts)
    torch.cuda.synchronize()
    return Xd.cpu().numpy(), it.cpu().numpy(), cv.cpu().numpy()


def test_noalloc_matches_context_call_on_two_calls_in_a_row():
    cs = library()
    import torch
    cases = [(Problem(80, 200, 32 * 9 + 5, "powerlaw", seed=2, noise_var=1e-3), 20, 4),
             (Problem(48, 120, 32 * 8 + 3, "sparse", seed=1, S=8), 8, 2)]
    for pr, kappa, G in cases:
        ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
        A = cs.cs_get_dictionary(ctx)
        Xref, itref, cvref = gpu_run(cs.cs_recover_gomp, ctx, pr.Y, pr.N, kappa, G)
        cs.cs_destroy(ctx)
        Xn, itn, cvn = _noalloc_run(cs, torch, A, pr, kappa, G)
        assert np.all(support(Xn) == support(Xref))
        assert rel_l2(Xn, Xref) <= REL_L2_FP32
        assert np.array_equal(itn, itref) and np.array_equal(cvn, cvref)


@pytest.mark.parametrize("M,N,kappa,G", [(102, 256, 24, 4), (128, 256, 32, 2)])
def test_noalloc_largest_shapes(M, N, kappa, G):
    """The 2048x2048-cube shape (M = 102, N = 256, support up to 96 atoms) and the largest
    shape the library accepts: every shape fits the static scratch.  The allocation-free
    call keeps its FP64 fallback factors in shared memory (the context call uses global
    slots), so wide supports take its own register and shared-memory plan."""
    cs = library()
    import torch
    pr = Problem(M, N, 128 + 37, "powerlaw", seed=5, noise_var=1e-3)
    ctx = cs.cs_create(M, N, Phi=pr.Phi)
    A = cs.cs_get_dictionary(ctx)
    Xref, itref, cvref = gpu_run(cs.cs_recover_gomp, ctx, pr.Y, N, kappa, G)
    cs.cs_destroy(ctx)
    Xn, itn, cvn = _noalloc_run(cs, torch, A, pr, kappa, G)
    assert np.all(support(Xn) == support(Xref))
    assert rel_l2(Xn, Xref) <= REL_L2_FP32
    assert np.array_equal(itn, itref) and np.array_equal(cvn, cvref)


def test_noalloc_reports_nonfinite_pixels():
    """No status word reaches the caller of the allocation-free call: a pixel whose
    measurements are not finite is marked 3 in converged_out, as in the context call."""
    cs = library()
    import torch
    pr = Problem(80, 200, 70, "powerlaw", seed=6, noise_var=1e-3)
    Y = pr.Y.copy()
    Y[3, 7] = np.nan
    Y[40, 0] = np.inf
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    A = cs.cs_get_dictionary(ctx)
    cs.cs_destroy(ctx)
    Xn, itn, cvn = _noalloc_run(cs, torch, A, pr, 20, 4, Y=Y)
    assert cvn[3] == 3 and cvn[40] == 3
    good = np.ones(pr.P, bool)
    good[[3, 40]] = False
    assert np.all(cvn[good] != 3)
    # the next call starts clean: the shared scratch's status word is cleared
    Xn2, itn2, cvn2 = _noalloc_run(cs, torch, A, pr, 20, 4)
    assert np.all(cvn2 != 3)


def test_noalloc_rejects_bad_shapes_options_and_host_memory():
    cs = library()
    import torch
    A = torch.zeros((128, 300), dtype=torch.float64, device="cuda")
    Y = torch.zeros((4, 128), device="cuda")
    X = torch.zeros((4, 300), device="cuda")
    with pytest.raises(cs.CsError) as e:
        cs.cs_recover_gomp_noalloc(A, 128, 300, Y, X, 8, 2)
    assert e.value.status == cs.CS_ERR_SHAPE
    A = torch.zeros((48, 120), dtype=torch.float64, device="cuda")
    Y = torch.zeros((4, 48), device="cuda")
    X = torch.zeros((4, 120), device="cuda")
    # the same option checks as the context call: an unknown precision is an error
    with pytest.raises(cs.CsError) as e:
        cs.cs_recover_gomp_noalloc(A, 48, 120, Y, X, 8, 2, opts=cs.make_opts(prec=7))
    assert e.value.status == cs.CS_ERR_ARG
    Yh = np.zeros((4, 48), dtype=np.float32)
    Xh = np.zeros((4, 120), dtype=np.float32)
    with pytest.raises(cs.CsError) as e:
        cs.cs_recover_gomp_noalloc(A, 48, 120, Yh, Xh, 8, 2)
    assert e.value.status == cs.CS_ERR_ARG
