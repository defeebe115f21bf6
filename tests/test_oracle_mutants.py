"""Plants plausible mistakes in copies of the oracle and checks that the pins catch each.

Every mutant is a one-line textual change of ``oracle/cs_oracle.c`` (a dropped term,
a wrong sign, index or operand, a misread step), compiled to a temporary library and
run through all pins of ``oracle_pins`` in a child process.  A mutant that no pin
rejects means the oracle's arithmetic at that spot is not pinned.  CPU only.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cs_oracle.c")

MUTANTS = {
    "fista_momentum": ("((t - 1.0) / t_new)", "((t_new - 1.0) / t_new)"),
    "fista_grad_sign": ("aux[n] = z[n] - g[n] / L", "aux[n] = z[n] + g[n] / L"),
    "fista_threshold": ("soft(aux[n], lambda / L)", "soft(aux[n], lambda)"),
    "fista_t_update": ("sqrt(1.0 + 4.0 * t * t)", "sqrt(1.0 + 2.0 * t * t)"),
    "soft_drops_sign": ("return a > 0.0 ? mag : (a < 0.0 ? -mag : 0.0);", "return mag;"),
    "admm_threshold_lambda_alpha": ("soft(x[n] + w[n], lambda / alpha)",
                                    "soft(x[n] + w[n], lambda * alpha)"),
    "admm_dual_sign": ("w[n] = w[n] + x[n] - z[n]", "w[n] = w[n] - x[n] + z[n]"),
    "admm_rhs_sign": ("aty[n] + alpha * (z[n] - w[n])", "aty[n] + alpha * (z[n] + w[n])"),
    "admm_drops_alpha_I": ("K[i * N + j] = s + (i == j ? alpha : 0.0);", "K[i * N + j] = s;"),
    "gomp_no_union": ("nc = support_union(N, w.c, nc, w.theta, G, w.in_c);",
                      "nc = support_union(N, w.c, 0, w.theta, G, w.in_c);"),
    "gomp_no_cap": ("if (M / G < cap) cap = M / G;", ""),
    "cosamp_selects_kappa": ("argmax_k(w.p, w.cand, N, 2 * kappa, w.theta, w.taken)",
                             "argmax_k(w.p, w.cand, N, kappa, w.theta, w.taken)"),
    "cosamp_no_union": ("nc = support_union(N, w.c, nc, w.theta, 2 * kappa, w.in_c);",
                        "nc = support_union(N, w.c, 0, w.theta, 2 * kappa, w.in_c);"),
    "biht_drops_support": ("if (xa[n] != 0.0) w.c[nc++] = n;", "if (0) w.c[nc++] = n;"),
    "biht_step_sign": ("w.p[n] = xa[n] + mu * w.p[n];", "w.p[n] = xa[n] - mu * w.p[n];"),
    "argmax_tie_break": ("(a == b && cand[i] < cand[best])", "(a == b && cand[i] > cand[best])"),
    "delta_not_difference": ("d += (r[m] - r_prev[m]) * (r[m] - r_prev[m]);", "d += r[m] * r[m];"),
    "lipschitz_min_eig": ("if (S[i * M + i] > lmax)", "if (S[i * M + i] < lmax)"),
    "dct_a0": ("sqrt(1.0 / N) : sqrt(2.0 / N)", "sqrt(2.0 / N) : sqrt(2.0 / N)"),
    "dct_phase": ("(2.0 * n + 1.0) * k", "(2.0 * n) * k"),
    "qr_transposed_R": ("acc -= R[j * nc + k] * s[k];", "acc -= R[k * nc + j] * s[k];"),
    "measure_noise_sign": ("Y[p * M + m] += E[p * M + m];", "Y[p * M + m] -= E[p * M + m];"),
    "svd_cutoff_inverted": ("if (sig[j] <= tol) continue;\n      double uty",
                            "if (sig[j] > tol) continue;\n      double uty"),
    "sparsify_population_std": ("sqrt(ss / (N - ddof))", "sqrt(ss / N)"),
    "sparsify_no_abs": ("      a[i] = fabs(s);", "      a[i] = s;"),
    "sparsify_strict_keep": ("if (a[i] - mu < T * sigma) x[i] = 0.0;",
                             "if (a[i] - mu <= T * sigma) x[i] = 0.0;"),
    "sparsify_transposed_psi": ("s += Psi[(size_t)n * N + i] * f[n];",
                                "s += Psi[(size_t)i * N + n] * f[n];"),
    "sparsify_std_uncentred": ("ss += (a[i] - mu) * (a[i] - mu);", "ss += a[i] * a[i];"),
    "dft_inverse_sign": ("const double ang = -2.0 * pi", "const double ang = 2.0 * pi"),
    "complex_no_conjugate": ("s += conj(A[(size_t)m * N + n]) * v[m];",
                             "s += A[(size_t)m * N + n] * v[m];"),
    "csoft_real_sign": ("return a * ((mag - t) / mag);",
                        "return (creal(a) >= 0.0 ? 1.0 : -1.0) * (mag - t);"),
    "cqr_drops_phase": ("const cplx alpha = -phase * nrm;", "const cplx alpha = -nrm;"),
    "cgomp_no_refit": ("        fail |= cqr_lstsq(M, N, A, cw.q, nq, y, cw.s, cw.lsw);\n", ""),
    "ccosamp_selects_kappa": ("argmax_k(cw.mag, cw.cand, N, 2 * kappa, cw.theta, cw.taken);",
                              "argmax_k(cw.mag, cw.cand, N, kappa, cw.theta, cw.taken);"),
    "cfista_grad_sign": ("aux[n] = z[n] - (g[n] / L);", "aux[n] = z[n] + (g[n] / L);"),
    "ccholesky_no_conjugate": ("acc -= K[(size_t)i * n + k] * conj(K[(size_t)j * n + k]);",
                               "acc -= K[(size_t)i * n + k] * K[(size_t)j * n + k];"),
    "cadmm_threshold_times_alpha": ("const double zthr = lambda / alpha;",
                                    "const double zthr = lambda * alpha;"),
    "cbiht_step_sign": ("cabs(xa[n] + mu * cw.p[n])", "cabs(xa[n] - mu * cw.p[n])"),
}

_RUNNER = r"""
import json, sys
sys.path[:0] = [sys.argv[2], sys.argv[3]]
import oracle, oracle_pins
oracle.use_library(sys.argv[1])
failed = []
for pin in oracle_pins.ALL_PINS:
    try:
        pin()
    except Exception:
        failed.append(pin.__name__)
        break  # one failing pin is enough to reject the mutant
print(json.dumps(failed))
"""


def _run_pins(lib):
    return subprocess.run([sys.executable, "-c", _RUNNER, str(lib), ROOT,
                           os.path.join(ROOT, "tests")],
                          capture_output=True, text=True, timeout=600)


def test_control_unmutated(tmp_path):
    """The unmutated source, built the same way, passes every pin through the runner."""
    lib = tmp_path / "libcontrol.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(lib), SRC,
                           "-lm"])
    out = _run_pins(lib)
    assert out.returncode == 0, out.stderr
    assert json.loads(out.stdout.strip().splitlines()[-1]) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(lib),
                           str(mutated), "-lm"])
    out = _run_pins(lib)
    if out.returncode != 0:
        return  # the mutant crashed or hung the pins: caught
    failed = json.loads(out.stdout.strip().splitlines()[-1])
    assert failed, f"no pin catches mutant {name}"
