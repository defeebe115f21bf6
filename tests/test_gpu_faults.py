"""Failure detection without a GPU fault: every wait of the tensor-core kernels is
bounded (100 ms on the global timer).  A test hook (CS_HSI_INJECT_MMA_TIMEOUT=1 in the
environment) makes FISTA's and ADMM's first product go unissued, so its wait runs out:
the call must report CS_ERR_TIMEOUT through the status word, release its tensor memory
and leave the context usable for the next call."""
import pytest

from gpu_common import Problem, library, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    return library()


@pytest.mark.parametrize("algo", ["fista", "admm"])
def test_unfinished_product_times_out_and_context_survives(cs, algo, monkeypatch):
    torch = torch_cuda()
    M, N, P = 80, 200, 300
    pr = Problem(M, N, P, "powerlaw", seed=31, noise_var=1e-3)
    ctx = cs.cs_create(M, N, Phi=pr.Phi, admm_rho=1.0)
    Y = torch.from_numpy(pr.Y).cuda()
    opts = cs.make_opts(eps=0.0, prec=cs.CS_BF16)

    def call(X):
        if algo == "fista":
            cs.cs_recover_fista(ctx, Y, X, 1e-3, 50, opts)
        else:
            cs.cs_recover_admm(ctx, Y, X, 1.0, 1e-3, 50, opts)

    ref = torch.empty((P, N), device="cuda")
    call(ref)
    cs.cs_sync(ctx)
    monkeypatch.setenv("CS_HSI_INJECT_MMA_TIMEOUT", "1")
    X = torch.zeros((P, N), device="cuda")
    call(X)
    with pytest.raises(cs.CsError) as e:
        cs.cs_sync(ctx)
    assert e.value.status == cs.CS_ERR_TIMEOUT
    monkeypatch.delenv("CS_HSI_INJECT_MMA_TIMEOUT")
    # the status word was cleared by cs_sync; the same context recovers normally again
    call(X)
    cs.cs_sync(ctx)
    assert torch.equal(X, ref)
