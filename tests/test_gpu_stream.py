"""cs_recover_stream (pushbroom recovery of a host-memory cube, chunk by chunk, through
double device buffers): every chunking gives, bit for bit, the single-cube call's X and
iteration counts, since each pixel's recovery depends on that pixel alone (Section II)."""
import numpy as np
import pytest

from gpu_common import Problem, library, torch_cuda
from paper_2401_14762_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    return library()


ALGOS = ["fista", "admm", "gomp", "biht", "cosamp"]


def _device_call(cs, ctx, algo, Y, N, opts):
    torch = torch_cuda()
    Yd = torch.from_numpy(Y).cuda()
    Xd = torch.full((Y.shape[0], N), float("nan"), device="cuda")
    if algo == "fista":
        cs.cs_recover_fista(ctx, Yd, Xd, 1e-3, 120, opts)
    elif algo == "admm":
        cs.cs_recover_admm(ctx, Yd, Xd, 1.0, 1e-3, 120, opts)
    elif algo == "gomp":
        cs.cs_recover_gomp(ctx, Yd, Xd, 20, 4, opts)
    elif algo == "biht":
        cs.cs_recover_biht(ctx, Yd, Xd, 20, opts)
    else:
        cs.cs_recover_cosamp(ctx, Yd, Xd, 20, opts)
    cs.cs_sync(ctx)
    return Xd.cpu().numpy()


def _stream_call(cs, ctx, algo, Y, X, chunk, opts):
    code = {"fista": cs.CS_ALGO_FISTA, "admm": cs.CS_ALGO_ADMM, "gomp": cs.CS_ALGO_GOMP,
            "biht": cs.CS_ALGO_BIHT, "cosamp": cs.CS_ALGO_COSAMP}[algo]
    cs.cs_recover_stream(ctx, code, Y, X, chunk, lam=1e-3, rho=1.0, iters=120, kappa=20, G=4,
                         opts=opts)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("chunk,pinned", [(64, True), (37, False), (1000, True)])
def test_stream_equals_single_call(cs, algo, chunk, pinned):
    torch = torch_cuda()
    M, N, P = 80, 200, 301
    pr = Problem(M, N, P, "powerlaw", seed=17, noise_var=1e-3)
    ctx = cs.cs_create(M, N, Phi=pr.Phi, admm_rho=1.0)
    prec = cs.CS_BF16 if algo in ("fista", "admm") else cs.CS_FP32
    it_d = torch.full((P,), -1, dtype=torch.int32, device="cuda")
    it_s = torch.full((P,), -1, dtype=torch.int32, device="cuda")
    cv_s = torch.full((P,), 255, dtype=torch.uint8, device="cuda")
    Xd = _device_call(cs, ctx, algo, pr.Y, N,
                      cs.make_opts(eps=1e-8, prec=prec, iters_out=it_d))
    if pinned:
        Yh = torch.from_numpy(pr.Y).pin_memory()
        Xh = torch.full((P, N), float("nan")).pin_memory()
    else:
        Yh = pr.Y.copy()
        Xh = np.full((P, N), np.nan, dtype=np.float32)
    _stream_call(cs, ctx, algo, Yh, Xh, chunk,
                 cs.make_opts(eps=1e-8, prec=prec, iters_out=it_s, converged_out=cv_s))
    Xs = Xh.numpy() if pinned else Xh
    assert np.array_equal(Xs.view(np.uint32), Xd.view(np.uint32))
    assert torch.equal(it_s, it_d)
    assert (cv_s.cpu().numpy() <= 1).all()


def test_stream_per_pixel_kappa(cs):
    """gOMP with per-pixel sparsity (G = 0: G = max(1, kappa_p / 5)): the chunks read their
    own slice of kappa_per_pixel."""
    torch = torch_cuda()
    M, N, P = 48, 120, 257
    pr = Problem(M, N, P, "sparse", seed=23, S=6, amplitude="separated")
    kp = torch.from_numpy(sy.kappa_per_pixel(P, 2, 12, 23).astype(np.int16)).cuda()
    ctx = cs.cs_create(M, N, Phi=pr.Phi)
    Yd = torch.from_numpy(pr.Y).cuda()
    Xd = torch.zeros((P, N), device="cuda")
    cs.cs_recover_gomp(ctx, Yd, Xd, 12, 0, cs.make_opts(kappa_per_pixel=kp))
    cs.cs_sync(ctx)
    Xh = np.zeros((P, N), dtype=np.float32)
    cs.cs_recover_stream(ctx, cs.CS_ALGO_GOMP, pr.Y, Xh, 50, kappa=12, G=0,
                         opts=cs.make_opts(kappa_per_pixel=kp))
    assert np.array_equal(Xh.view(np.uint32), Xd.cpu().numpy().view(np.uint32))


def test_stream_argument_errors(cs):
    torch = torch_cuda()
    ctx = cs.cs_create(20, 50, Phi=sy.gaussian_phi(20, 50, 2))
    Y = np.zeros((10, 20), dtype=np.float32)
    X = np.zeros((10, 50), dtype=np.float32)
    for args, kw in (((Y, X, 0), {}),                                   # chunk < 1
                     ((torch.zeros((10, 20), device="cuda"), X, 4), {}),  # device Y
                     ((Y, X, 4), {"kappa": 26})):                      # 2 kappa > N
        with pytest.raises(cs.CsError) as e:
            cs.cs_recover_stream(ctx, cs.CS_ALGO_COSAMP, *args, **kw)
        assert e.value.status == cs.CS_ERR_ARG
    cs.cs_recover_stream(ctx, cs.CS_ALGO_COSAMP, Y[:0], X[:0], 4, kappa=5)  # P = 0


@pytest.mark.parametrize("pinned", [True, False])
def test_measure_host_cube_is_chunked_bit_for_bit(cs, pinned):
    """cs_measure on a host-memory cube runs in chunks of 262,144 pixels with the copies
    overlapped: Y equals the device-memory call's bit for bit, over two whole chunks and a
    ragged third, with and without E."""
    torch = torch_cuda()
    M, N, P = 48, 120, 2 * 262144 + 777
    Phi = sy.gaussian_phi(M, N, 5)
    ctx = cs.cs_create(M, N, Phi=Phi)
    X = torch.from_numpy(sy.sparse_coeffs(P, N, 6, 5)).float()
    E = torch.from_numpy(sy.noise(P, M, 1e-3, 5)).float()
    if pinned:
        X, E = X.pin_memory(), E.pin_memory()
    for noise in (E, None):
        Yd = torch.empty((P, M), device="cuda")
        cs.cs_measure(ctx, X.cuda(), Yd, None if noise is None else noise.cuda())
        cs.cs_sync(ctx)
        Yh = torch.full((P, M), float("nan"))
        if pinned:
            Yh = Yh.pin_memory()
        cs.cs_measure(ctx, X, Yh, noise)
        assert torch.equal(Yh, Yd.cpu())
