"""The autotuner of the greedy kernels' launch configuration (cs_autotune): it times the
candidate configurations on a sample and installs the fastest; results do not depend on
the configuration, so the tuned calls must reproduce the built-in ones bit for bit, and a
choice cached to JSON must be installed again without measuring."""
import json

import numpy as np
import pytest

from gpu_common import Problem, gpu_run, library, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    return library()


@pytest.mark.parametrize("algo,kappa,G", [("gomp", 20, 4), ("cosamp", 20, 0), ("biht", 20, 0)])
def test_tuned_calls_equal_builtin_ones(cs, algo, kappa, G, tmp_path):
    torch = torch_cuda()
    pr = Problem(80, 200, 32 * 40 + 9, "powerlaw", seed=12, noise_var=1e-3)
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    code = {"gomp": cs.CS_ALGO_GOMP, "cosamp": cs.CS_ALGO_COSAMP, "biht": cs.CS_ALGO_BIHT}[algo]
    call = {"gomp": lambda c, Y, X, opts: cs.cs_recover_gomp(c, Y, X, kappa, G, opts=opts),
            "cosamp": lambda c, Y, X, opts: cs.cs_recover_cosamp(c, Y, X, kappa, opts=opts),
            "biht": lambda c, Y, X, opts: cs.cs_recover_biht(c, Y, X, kappa, opts=opts)}[algo]
    X0, it0, cv0 = gpu_run(call, ctx, pr.Y, pr.N)
    Yd = torch.from_numpy(pr.Y).cuda()
    cache = str(tmp_path / "tune.json")
    rec = cs.cs_autotune(ctx, code, Yd, kappa, G, cache=cache)
    print(algo, rec)
    assert rec["cached"] is False and rec["ms"] > 0 and rec["ms_default"] > 0
    assert rec["ms"] <= rec["ms_default"]
    assert 2 <= rec["warps_per_cta"] <= 8 or rec["tuned"] == 0
    X1, it1, cv1 = gpu_run(call, ctx, pr.Y, pr.N)
    assert np.array_equal(X0, X1) and np.array_equal(it0, it1) and np.array_equal(cv0, cv1)
    # a second context takes the cached choice without measuring
    ctx2 = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    rec2 = cs.cs_autotune(ctx2, code, Yd, kappa, G, cache=cache)
    assert rec2["cached"] is True and rec2["warps_per_cta"] == rec["warps_per_cta"]
    assert json.load(open(cache))
    X2, it2, _ = gpu_run(call, ctx2, pr.Y, pr.N)
    assert np.array_equal(X0, X2) and np.array_equal(it0, it2)


def test_autotune_rejects_convex_and_host_samples(cs):
    torch = torch_cuda()
    pr = Problem(48, 120, 64, "sparse", seed=1, S=6)
    ctx = cs.cs_create(pr.M, pr.N, Phi=pr.Phi)
    with pytest.raises(cs.CsError) as e:
        cs.cs_autotune(ctx, cs.CS_ALGO_FISTA, torch.from_numpy(pr.Y).cuda(), 6, 2)
    assert e.value.status == cs.CS_ERR_ARG
    with pytest.raises(cs.CsError) as e:
        cs.cs_autotune(ctx, cs.CS_ALGO_GOMP, pr.Y, 6, 2)
    assert e.value.status == cs.CS_ERR_ARG
