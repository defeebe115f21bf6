"""cs_recover_batch: several cubes of different shapes, sizes and per-pixel sparsity in one
call.  Each cube's result must equal the single-cube call bit for bit (the batch runs the
same per-pixel arithmetic), and the greedy results must match the FP64 oracle exactly."""
import numpy as np
import pytest

import oracle as orc
from gpu_common import Problem, exact_check, gpu_run, library, rel_l2, torch_cuda
from paper_2401_14762_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    return library()


def _cubes(kind="sparse"):
    # (M, N, P): the three band counts of the batching workload, M = 0.4 N, uneven sizes,
    # one empty cube in the middle
    shapes = [(48, 120, 37), (80, 200, 150), (80, 200, 0), (90, 224, 70)]
    out = []
    for i, (M, N, P) in enumerate(shapes):
        if P == 0:
            out.append(None)
            continue
        pr = Problem(M, N, P, kind, seed=40 + i, S=6, amplitude="separated")
        pr.kp = sy.kappa_per_pixel(P, 4, 12, 40 + i)
        out.append(pr)
    return shapes, out


def _batch(cs, algo, probs, shapes, ctxs, kappa=12, G=0, per_pixel=True, **kw):
    torch = torch_cuda()
    items, outs = [], []
    for (M, N, P), pr, ctx in zip(shapes, probs, ctxs):
        Y = torch.from_numpy(pr.Y).cuda() if pr else torch.zeros((0, M), device="cuda")
        X = torch.full((P, N), float("nan"), device="cuda")
        it = torch.full((P,), -1, device="cuda", dtype=torch.int32)
        cv = torch.full((P,), 255, device="cuda", dtype=torch.uint8)
        item = {"ctx": ctx, "Y": Y, "X": X}
        if P > 0:  # an empty cube passes no per-pixel arrays
            item.update(iters_out=it, converged_out=cv)
        if per_pixel and pr is not None:
            item["kappa_per_pixel"] = torch.from_numpy(pr.kp.astype(np.int16)).cuda()
        items.append(item)
        outs.append((X, it, cv))
    cs.cs_recover_batch(items, algo, kappa=kappa, G=G, opts=cs.make_opts(**kw))
    cs.cs_sync(ctxs[0])
    return [(X.cpu().numpy(), it.cpu().numpy(), cv.cpu().numpy()) for X, it, cv in outs]


@pytest.mark.parametrize("algo", ["gomp", "biht", "cosamp"])
def test_batch_greedy_equals_single_calls_and_oracle(cs, algo):
    shapes, probs = _cubes()
    ctxs = [cs.cs_create(M, N, Phi=pr.Phi if pr else sy.gaussian_phi(M, N, 1))
            for (M, N, _), pr in zip(shapes, probs)]
    code = {"gomp": cs.CS_ALGO_GOMP, "biht": cs.CS_ALGO_BIHT, "cosamp": cs.CS_ALGO_COSAMP}[algo]
    res = _batch(cs, code, probs, shapes, ctxs, mu=1.0)
    call = {"gomp": cs.cs_recover_gomp, "biht": cs.cs_recover_biht,
            "cosamp": cs.cs_recover_cosamp}[algo]
    for (M, N, P), pr, ctx, (Xb, itb, cvb) in zip(shapes, probs, ctxs, res):
        if pr is None:
            assert Xb.shape == (0, N)
            continue
        args = (12, 0) if algo == "gomp" else (12,)
        Xs, its, cvs = gpu_run(call, ctx, pr.Y, N, *args, mu=1.0, kappa_pp=pr.kp)
        assert np.array_equal(Xb.view(np.uint32), Xs.view(np.uint32))
        assert np.array_equal(itb, its) and np.array_equal(cvb, cvs)
        # oracle, per sparsity level
        Xo = np.zeros((P, N))
        ito = np.zeros(P, dtype=np.int32)
        for k in np.unique(pr.kp):
            sel = pr.kp == k
            k = int(k)
            if algo == "gomp":
                Xo[sel], ito[sel], _ = orc.gomp(pr.A, pr.Y[sel], k, max(1, k // 5))
            elif algo == "biht":
                Xo[sel], ito[sel], _ = orc.biht(pr.A, pr.Y[sel], k, 1.0)
            else:
                Xo[sel], ito[sel], _ = orc.cosamp(pr.A, pr.Y[sel], k)
        exact_check(Xb, itb, Xo, ito, 12)


@pytest.mark.parametrize("algo,prec", [("fista", 1), ("admm", 1), ("fista", 0), ("admm", 0)])
def test_batch_convex_equals_single_calls(cs, algo, prec):
    shapes, probs = _cubes("powerlaw")
    ctxs = [cs.cs_create(M, N, Phi=pr.Phi if pr else sy.gaussian_phi(M, N, 1), admm_rho=1.0)
            for (M, N, _), pr in zip(shapes, probs)]
    code = cs.CS_ALGO_FISTA if algo == "fista" else cs.CS_ALGO_ADMM
    torch = torch_cuda()
    items, outs = [], []
    for (M, N, P), pr, ctx in zip(shapes, probs, ctxs):
        Y = torch.from_numpy(pr.Y).cuda() if pr else torch.zeros((0, M), device="cuda")
        X = torch.full((P, N), float("nan"), device="cuda")
        it = torch.full((P,), -1, device="cuda", dtype=torch.int32)
        items.append({"ctx": ctx, "Y": Y, "X": X, "iters_out": it if P > 0 else None})
        outs.append((X, it))
    cs.cs_recover_batch(items, code, lam=1e-3, rho=1.0, iters=120,
                        opts=cs.make_opts(eps=0.0, prec=prec))
    cs.cs_sync(ctxs[0])
    for (M, N, P), pr, ctx, (X, it) in zip(shapes, probs, ctxs, outs):
        if pr is None:
            continue
        if algo == "fista":
            Xs, its, _ = gpu_run(cs.cs_recover_fista, ctx, pr.Y, N, 1e-3, 120, eps=0.0, prec=prec)
        else:
            Xs, its, _ = gpu_run(cs.cs_recover_admm, ctx, pr.Y, N, 1.0, 1e-3, 120, eps=0.0,
                                 prec=prec)
        assert np.array_equal(X.cpu().numpy().view(np.uint32), Xs.view(np.uint32))
        assert np.array_equal(it.cpu().numpy(), its)


def test_batch_argument_errors(cs):
    torch = torch_cuda()
    ctx_a = cs.cs_create(48, 120, Phi=sy.gaussian_phi(48, 120, 1))
    ctx_b = cs.cs_create(24, 60, Phi=sy.gaussian_phi(24, 60, 2))
    Y = torch.zeros((4, 48), device="cuda")
    X = torch.zeros((4, 120), device="cuda")
    Yb = torch.zeros((4, 24), device="cuda")
    Xb = torch.zeros((4, 60), device="cuda")
    ok = {"ctx": ctx_a, "Y": Y, "X": X}
    with pytest.raises(cs.CsError) as e:   # 2 kappa > N for the second cube
        cs.cs_recover_batch([ok, {"ctx": ctx_b, "Y": Yb, "X": Xb}], cs.CS_ALGO_COSAMP, kappa=31)
    assert e.value.status == cs.CS_ERR_ARG
    with pytest.raises(cs.CsError) as e:   # host memory
        cs.cs_recover_batch([{"ctx": ctx_a, "Y": Y.cpu().numpy(), "X": X.cpu().numpy()}],
                            cs.CS_ALGO_GOMP, kappa=8, G=2)
    assert e.value.status == cs.CS_ERR_ARG
    with pytest.raises(cs.CsError) as e:   # G = 0 without per-pixel kappa
        cs.cs_recover_batch([ok], cs.CS_ALGO_GOMP, kappa=8, G=0)
    assert e.value.status == cs.CS_ERR_ARG
    with pytest.raises(cs.CsError) as e:   # ADMM needs rho > 0
        cs.cs_recover_batch([ok], cs.CS_ALGO_ADMM, lam=1e-3, rho=0.0, iters=5)
    assert e.value.status == cs.CS_ERR_ARG
    with pytest.raises(cs.CsError):
        cs.cs_recover_batch([], cs.CS_ALGO_GOMP, kappa=8, G=2)


def test_batch_many_small_cubes(cs):
    """More cubes than one descriptor upload carries (32), several of one dictionary:
    every cube equals its single-cube call bit for bit."""
    torch = torch_cuda()
    ctxs = [cs.cs_create(48, 120, Phi=sy.gaussian_phi(48, 120, 70 + i % 5)) for i in range(5)]
    probs, items = [], []
    for i in range(41):
        pr = Problem(48, 120, 3 + (7 * i) % 19, "sparse", seed=70 + i % 5, S=5,
                     amplitude="separated")
        ctx = ctxs[i % 5]
        X = torch.full((pr.P, 120), float("nan"), device="cuda")
        it = torch.full((pr.P,), -1, device="cuda", dtype=torch.int32)
        items.append({"ctx": ctx, "Y": torch.from_numpy(pr.Y).cuda(), "X": X, "iters_out": it})
        probs.append((pr, ctx, X, it))
    cs.cs_recover_batch(items, cs.CS_ALGO_COSAMP, kappa=6, opts=cs.make_opts())
    cs.cs_sync(ctxs[0])
    for pr, ctx, X, it in probs:
        Xs, its, _ = gpu_run(cs.cs_recover_cosamp, ctx, pr.Y, 120, 6)
        assert np.array_equal(X.cpu().numpy().view(np.uint32), Xs.view(np.uint32))
        assert np.array_equal(it.cpu().numpy(), its)


@pytest.mark.parametrize("algo", ["cosamp", "fista"])
def test_batch_replays_in_cuda_graph(cs, algo):
    """cs_recover_batch queues only stream-ordered work (kernels, memsets, and event waits
    that fork its per-cube FISTA/ADMM launches over several streams and join them back),
    so it can be captured in a CUDA graph: replaying the graph on new measurements in the
    same buffers gives, bit for bit, what a direct call gives on them."""
    torch = torch_cuda()
    s = torch.cuda.Stream()
    kind = "sparse" if algo == "cosamp" else "powerlaw"
    shapes, first = _cubes(kind)
    second = [Problem(M, N, P, kind, seed=80 + i, S=6, amplitude="separated") if P else None
              for i, (M, N, P) in enumerate(shapes)]
    ctxs = [cs.cs_create(M, N, Phi=pr.Phi if pr else sy.gaussian_phi(M, N, 1),
                         stream=s.cuda_stream) for (M, N, _), pr in zip(shapes, first)]
    # the second set reuses each cube's dictionary: measure it with the first set's A
    Ys, Xs, its = [], [], []
    for (M, N, P), pr in zip(shapes, first):
        Ys.append(torch.zeros((P, M), device="cuda"))
        Xs.append(torch.zeros((P, N), device="cuda"))
        its.append(torch.zeros((P,), device="cuda", dtype=torch.int32))
    items = [{"ctx": c, "Y": Y, "X": X, "iters_out": it if Y.shape[0] else None}
             for c, Y, X, it in zip(ctxs, Ys, Xs, its)]

    def call():
        if algo == "cosamp":
            cs.cs_recover_batch(items, cs.CS_ALGO_COSAMP, kappa=12, opts=cs.make_opts())
        else:
            cs.cs_recover_batch(items, cs.CS_ALGO_FISTA, lam=1e-3, iters=80,
                                opts=cs.make_opts(eps=0.0, prec=1))

    def load(probs):
        torch.cuda.synchronize()
        for Y, pr, p1 in zip(Ys, probs, first):
            if pr is not None:
                Y.copy_(torch.from_numpy(orc.measure(p1.A, pr.Xt).astype(np.float32)))
        torch.cuda.synchronize()

    def outputs():
        torch.cuda.synchronize()
        return [(X.cpu().numpy().copy(), it.cpu().numpy().copy()) for X, it in zip(Xs, its)]

    load(first)
    with torch.cuda.stream(s):
        call()  # warm-up: creates the fork-join streams, sizes the greedy scratch
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        call()
    cs.cs_sync(ctxs[0])
    for probs in (second, first):
        load(probs)
        g.replay()
        replayed = outputs()
        with torch.cuda.stream(s):
            call()
        cs.cs_sync(ctxs[0])
        direct = outputs()
        for (Xg, ig), (Xd, idd), (M, N, P) in zip(replayed, direct, shapes):
            assert np.array_equal(Xg.view(np.uint32), Xd.view(np.uint32))
            assert np.array_equal(ig, idd)
            if P:
                assert np.isfinite(Xd).all() and (idd > 0).all()


@pytest.mark.parametrize("prec", [1, 0])
def test_batch_fista_meets_the_oracle(cs, prec):
    """The batching workload's FISTA (lambda = 0.1, Delta < 1e-6 or 3,000 iterations) on
    exactly sparse, noiseless cubes of the three band counts, all in one
    cs_recover_batch call: every cube within rel-L2 1e-3 of the FP64 oracle run with the
    same stop rule, on the split-BF16 tensor path and on the FP32 path."""
    torch = torch_cuda()
    shapes = [(48, 120, 37), (80, 200, 150), (90, 224, 70)]
    probs, ctxs, items, outs = [], [], [], []
    for i, (M, N, P) in enumerate(shapes):
        S = sy.kappa_per_pixel(P, 4, 32, 60 + i)
        Phi = sy.gaussian_phi(M, N, 60 + i)
        A = orc.dictionary(Phi)
        Y = orc.measure(A, sy.sparse_coeffs(P, N, S, 60 + i), np.zeros((P, M))).astype(np.float32)
        ctx = cs.cs_create(M, N, Phi=Phi)
        X = torch.full((P, N), float("nan"), device="cuda")
        items.append({"ctx": ctx, "Y": torch.from_numpy(Y).cuda(), "X": X})
        probs.append((A, Y))
        ctxs.append(ctx)
        outs.append(X)
    cs.cs_recover_batch(items, cs.CS_ALGO_FISTA, lam=0.1, iters=3000,
                        opts=cs.make_opts(eps=1e-6, prec=prec))
    cs.cs_sync(ctxs[0])
    for (A, Y), X in zip(probs, outs):
        Xo, _ = orc.fista(A, Y.astype(np.float64), orc.lipschitz(A), 0.1, 1e-6, 3000)
        err = rel_l2(X.cpu().numpy(), Xo)
        print(f"batch FISTA prec {prec}, N = {A.shape[1]}: rel-L2 {err:.2e}")
        assert err <= 1e-3
