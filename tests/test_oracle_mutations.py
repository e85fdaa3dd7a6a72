"""Mutation check of the oracle's pins.

Each entry below plants one plausible mistake in one oracle module (a
dropped term, a flipped sign, a wrong index or normalisation, a transposed
operand, a skipped step) and runs that module's pin file against the mutant
in a child process (tests/_oracle_mutant_plugin.py swaps the module in before
the pins import it).  The pins must fail on every mutant, and must pass on
the unmodified source re-executed the same way (the control runs).

The mutants run in parallel child processes, on the CPU only.
"""

import concurrent.futures as cf
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")

PINS = {m: ["tests/test_oracle_%s.py" % m]
        for m in ("philox", "transform", "prox", "svt", "admm", "learned", "tucker", "ctv",
                  "onebit")}

# (id, module, text in the module's source, its replacement)
MUTANTS = [
    # Philox4x32-10 and Box-Muller
    ("philox-swapped-key-words", "philox",
     "(hi_b ^ c1 ^ k0), lo_b, (hi_a ^ c3 ^ k1), lo_a",
     "(hi_b ^ c1 ^ k1), lo_b, (hi_a ^ c3 ^ k0), lo_a"),
    ("philox-half-angle", "philox", "theta = 2.0 * np.pi * u2", "theta = np.pi * u2"),
    ("philox-row-major-block", "philox", "return vals.reshape(cols, rows).T.copy()",
     "return vals.reshape(rows, cols).copy()"),
    # the transform (Eq. trans, Eq. orth)
    ("transform-dc-scale", "transform", "s[0, 0] = np.sqrt(1.0 / n)", "s[0, 0] = np.sqrt(2.0 / n)"),
    ("transform-untransposed-inverse", "transform", "return dct_matrix(n).T",
     "return dct_matrix(n)"),
    ("transform-mode-axis", "transform", "return d - mode   #", "return mode - 3   #"),
    ("transform-dft-inverse-scale", "transform", "return dft_matrix(n).conj().T / n",
     "return dft_matrix(n).conj().T"),
    # scalar proximal maps (Eq. equ_gst1)
    ("prox-l1-threshold", "prox", "return sgn * np.maximum(a - mu * theta, 0.0)",
     "return sgn * np.maximum(a - 0.5 * mu * theta, 0.0)"),
    ("prox-mcp-dropped-denominator", "prox",
     "mid = sgn * (a - mu * theta) / (1.0 - mu / gamma)", "mid = sgn * (a - mu * theta)"),
    ("prox-mcp-hard-threshold", "prox", "thr = theta * np.sqrt(gamma * mu)", "thr = theta * mu"),
    ("prox-mcp-penalty-plateau", "prox", "gamma * theta * theta / 2.0", "gamma * theta / 2.0"),
    # GNHTSVT engines (Alg. 1-4, Def. gNtsvt)
    ("svt-full-no-shrink", "svt", "return (U * s2) @ Vt, s, s2", "return (U * s) @ Vt, s, s2"),
    ("svt-power-step-discarded", "svt", "        Y = Ab @ W\n", "        Y = Ab @ Omega\n"),
    ("svt-defl-qr-unpermuted", "svt", "R[:, piv] = Rt[:s, :]", "R[:, :] = Rt[:s, :]"),
    ("svt-blbp-dropped-L-term", "svt", "E -= float(np.sum(Lt * Lt))",
     "E -= 0.0 * float(np.sum(Lt * Lt))"),
    ("svt-blbp-sign-of-U-L", "svt", "defl_qr(A @ V - U_prev @ L, delta)",
     "defl_qr(A @ V + U_prev @ L, delta)"),
    ("svt-learned-no-fallback", "svt", "            if j in set(fb.tolist()):",
     "            if j in set():"),
    ("svt-forward-for-inverse", "svt", "out = transform.inverse(Gbar, tdims, transform_kind)",
     "out = transform.forward(Gbar, tdims, transform_kind)"),
    # the pure-L ADMM step (Alg. 5)
    ("admm-L-multiplier-sign", "admm", "(st.G - st.Lam / mu))", "(st.G + st.Lam / mu))"),
    ("admm-Y-update-sign", "admm", "Y = st.Y + mu * (M - L - E)", "Y = st.Y - mu * (M - L - E)"),
    ("admm-tau-times-mu", "admm", "tau = 1.0 / mu", "tau = 1.0 * mu"),
    ("admm-E-zero-off-omega", "admm", "E = np.where(omega, E_on, H)",
     "E = np.where(omega, E_on, 0.0)"),
    # the learned engine (rank predictor and width plan)
    ("learned-dropped-bias", "learned", "h = np.maximum(h @ W.T + b, 0.0)",
     "h = np.maximum(h @ W.T, 0.0)"),
    ("learned-backprop-no-relu-mask", "learned", "dz = (dz @ W) * (inp > 0)", "dz = dz @ W"),
    ("learned-adam-no-v-bias-correction", "learned", "vhat = v / (1.0 - beta2 ** step)",
     "vhat = v"),
    ("learned-width-rounded-down", "learned", "l = (r + p + 7) // 8 * 8", "l = (r + p) // 8 * 8"),
    ("learned-judge-eps-not-squared", "learned", "a2 - cap < eps * eps * a2",
     "a2 - cap < eps * a2"),
    ("learned-judge-missed-energy-sign", "learned", "a2 - cap < eps * eps * a2",
     "a2 + cap < eps * eps * a2"),
    ("learned-judge-margin-ignores-oversampling", "learned", "margin = rank[j] <= width[j] - p",
     "margin = rank[j] <= width[j]"),
    # shared and fixed-accuracy Tucker forms (Alg. 1, Alg. AD-RSTHOSVD-BLBP)
    ("tucker-transposed-mode-product", "tucker", '"jia,ba->jib", C, F', '"jia,ab->jib", C, F'),
    ("tucker-trailing-singular-vectors", "tucker", "return canonical_signs(Z @ U[:, :r]), Z",
     "return canonical_signs(Z @ U[:, -r:]), Z"),
    ("tucker-krylov-block", "tucker", "blocks.append(A @ (A.T @ blocks[-1]))",
     "blocks.append(A @ (A.T @ blocks[0]))"),
    ("svt-eps-not-squared", "svt", "if E < eps * eps * normA2", "if E < eps * normA2"),
    ("tucker-ad-factor-signs-free", "tucker", "        Fm = canonical_signs(Fm)\n", "\n"),
    # the gradient-domain step (Eq. coef-tensor, Eq. gnrhtc-L, Alg. 5)
    ("ctv-missing-conjugate", "ctv", "num = num + np.conj(FD) * np.fft.fftn",
     "num = num + FD * np.fft.fftn"),
    ("ctv-tau-without-gamma", "ctv", "tau = 1.0 / (gam * mu)", "tau = 1.0 / mu"),
    ("ctv-kernel-offset", "ctv", "idx[ax] = Dk.shape[ax] - 1", "idx[ax] = 1"),
    ("ctv-adjoint-untransposed", "ctv", "difference_matrix(X.shape[ax]).T, ax)",
     "difference_matrix(X.shape[ax]), ax)"),
    ("ctv-Lambda-sign", "ctv", "st.Lam[k] + mu * (gradL[k] - G[k])",
     "st.Lam[k] - mu * (gradL[k] - G[k])"),
    # the one-bit step (Alg. 6)
    ("onebit-L-sign-of-Y", "onebit", "(m * mu * Z + J1 - m * Y)", "(m * mu * Z + J1 + m * Y)"),
    ("onebit-Y-update-sign", "onebit", "Y = st.Y + mu * (L - Z)", "Y = st.Y + mu * (Z - L)"),
    ("onebit-tau-without-gamma", "onebit", "tau = p.lam / (gam * mu)", "tau = p.lam / mu"),
    ("onebit-Z-step-old-L", "onebit", "Z = ctv.l_update(L + st.Y / mu",
     "Z = ctv.l_update(st.L + st.Y / mu"),
    ("onebit-no-clip", "onebit", "/ (m * mu + J2), -alpha, alpha)",
     "/ (m * mu + J2), -1e300, 1e300)"),
]


def _run(module, old, new):
    env = dict(os.environ)
    env["PYTHONPATH"] = os.pathsep.join([ROOT, TESTS, env.get("PYTHONPATH", "")])
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[var] = "1"   # the children run side by side
    env["TR_ORACLE_MUTANT"] = json.dumps({"module": module, "old": old, "new": new})
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           "-p", "_oracle_mutant_plugin", "-m", "not gpu"] + PINS[module]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-1500:]


@pytest.fixture(scope="module")
def outcomes():
    jobs = {("mutant", mid): (mod, old, new) for mid, mod, old, new in MUTANTS}
    jobs.update({("control", mod): (mod, "", "") for mod in PINS})
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {key: ex.submit(_run, *args) for key, args in jobs.items()}
        return {key: f.result() for key, f in futs.items()}


def test_mutation_texts_occur_once():
    for mid, mod, old, new in MUTANTS:
        with open(os.path.join(ROOT, "oracle", mod + ".py")) as f:
            assert f.read().count(old) == 1, mid


@pytest.mark.parametrize("module", sorted(PINS))
def test_control_run_passes(outcomes, module):
    code, tail = outcomes[("control", module)]
    assert code == 0, tail


@pytest.mark.parametrize("mid", [m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(outcomes, mid):
    code, tail = outcomes[("mutant", mid)]
    # exit code 1: the pin tests ran and at least one failed
    assert code == 1, "mutant %s survived or broke collection (exit %d)\n%s" % (mid, code, tail)
