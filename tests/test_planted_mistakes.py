"""The oracle's pins against planted mistakes: each case below copies the oracle's C source with one
plausible error in it (a dropped term, a flipped sign, a transposed index, a wrong constant), builds that
copy, and runs the oracle's pin tests (tests/test_oracle_*.py) on it in a child process.  Every copy must
fail at least one pin, and the unchanged source, built the same way, must pass them all.  The mistakes
are planted in the oracle only, on the CPU."""
import concurrent.futures as cf
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rmge_oracle.c")

# (name, text in the oracle's source, replacement): each text occurs exactly once
MISTAKES = [
    # Philox4x32-10 and the draws (Def. 4.1, Ex. 5.1, Ex. 5.2)
    ("philox nine rounds", "for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {"),
    ("philox wrong key bump", "k[1] += 0xBB67AE85u;", "k[1] += 0x9E3779B9u;"),
    ("box-muller radius without the factor 2", "const double r = sqrt(-2.0 * log(u1));",
     "const double r = sqrt(-log(u1));"),
    ("uniform draw not centred", "out[e] = 2.0 * ((double)bits53(x[0], x[1]) * two_m53) - 1.0;",
     "out[e] = 2.0 * ((double)bits53(x[0], x[1]) * two_m53);"),
    ("unitary spectrum not Hermitian", "ui[n - j] = -ui[j];", "ui[n - j] = ui[j];"),
    # products and structured multipliers (Fact 4.1, Sec. 5)
    ("matmul drops the last term", "        for (int64_t t = 0; t < k; ++t) {\n            const double a = A[i * k + t];",
     "        for (int64_t t = 0; t + 1 < k; ++t) {\n            const double a = A[i * k + t];"),
    ("matmul subtracts", "for (int64_t j = 0; j < n; ++j) c[j] += a * b[j];",
     "for (int64_t j = 0; j < n; ++j) c[j] -= a * b[j];"),
    ("circulant transposed", "C[i * n + j] = c[((i - j) % n + n) % n];", "C[i * n + j] = c[((j - i) % n + n) % n];"),
    ("toeplitz transposed", "T[i * n + j] = c2[((i - j) % N + N) % N];", "T[i * n + j] = c2[((j - i) % N + N) % N];"),
    ("dft sign", "const double ang = (double)sign * 2.0", "const double ang = -(double)sign * 2.0"),
    # GENP (Sec. 3, eq. (3.1)) and GEPP
    ("genp schur update adds", "/ piv;\n            M[i * n + s] = l;\n"
     "            for (int64_t j = s + 1; j < n; ++j) M[i * n + j] -= l * M[s * n + j];",
     "/ piv;\n            M[i * n + s] = l;\n"
     "            for (int64_t j = s + 1; j < n; ++j) M[i * n + j] += l * M[s * n + j];"),
    ("gepp without the row swap", "        if (p != s)\n            for (int64_t j = 0; j < n; ++j) {",
     "        if (0)\n            for (int64_t j = 0; j < n; ++j) {"),
    ("genp multiplier transposed", "            const double l = M[i * n + s] / piv;\n            M[i * n + s] = l;\n"
     "            for (int64_t j = s + 1; j < n; ++j)",
     "            const double l = M[s * n + i] / piv;\n            M[i * n + s] = l;\n"
     "            for (int64_t j = s + 1; j < n; ++j)"),
    ("genp misses a zero pivot", "        const double piv = M[s * n + s];\n        if (piv == 0.0 || !isfinite(piv)) return (int)(s + 1);\n#pragma",
     "        const double piv = M[s * n + s];\n        if (!isfinite(piv)) return (int)(s + 1);\n#pragma"),
    ("blocked genp schur update skips a column", "                for (int64_t j = k + b; j < n; ++j) M[i * n + j] -= l * M[t * n + j];",
     "                for (int64_t j = k + b + 1; j < n; ++j) M[i * n + j] -= l * M[t * n + j];"),
    # solves, residual, norms, growth (Sec. 1.2, Sec. 7.1, Thm 3.2)
    ("lu solve skips the diagonal of U", "        for (int64_t c = 0; c < k; ++c) B[i * k + c] /= LU[i * n + i];\n    }\n}\n\n/* B <- U^{-T}",
     "    }\n}\n\n/* B <- U^{-T}"),
    ("residual sign", "const double p = -A[i * n + t] * X[t * k + c];", "const double p = A[i * n + t] * X[t * k + c];"),
    ("backward error without the norm of b", "const double den = an * xn + bn;", "const double den = an * xn;"),
    ("infinity norm of the first row only", "if (s > best || isnan(s)) best = s;", "if (i == 0) best = s;"),
    ("growth from the lower factor", "if (j >= i) um = fmax(um, fabs(LU[i * n + j]));",
     "if (j <= i) um = fmax(um, fabs(LU[i * n + j]));"),
    # the randomized solve (Fact 4.1) and refinement
    ("solution not recovered by H", "    orc_lu_solve(n, k, LU, Y);\n    apply_H(kind, n, k, H, Y, X);",
     "    orc_lu_solve(n, k, LU, Y);\n    memcpy(X, Y, sizeof(double) * (size_t)(n * k));"),
    ("refinement correction without H", "    orc_lu_solve(n, k, LU, R);\n    apply_H(kind, n, k, H, R, D);",
     "    orc_lu_solve(n, k, LU, R);\n    memcpy(D, R, sizeof(double) * (size_t)(n * k));"),
    ("two-sided solve drops F on the right-hand side", "        orc_matmul(n, n, k, DF, B, Y);",
     "        memcpy(Y, B, sizeof(double) * (size_t)(n * k));"),
    # Algorithm 6.1 and the adjoint
    ("qr without the sign fix", "        if (R[j * l + j] < 0.0) {", "        if (0) {"),
    ("low-rank Z from the wrong side", "for (int64_t t = 0; t < m; ++t) z += Q[t * l + i] * A[t * n + j];",
     "for (int64_t t = 0; t < m; ++t) z += Q[t * l + i] * A[j * n + t];"),
    ("adjoint dA sign", "                dA[i * n + j] = -s;", "                dA[i * n + j] = s;"),
    ("adjoint solves with A, not its transpose", "AT[j * n + i] = A[i * n + j];", "AT[i * n + j] = A[i * n + j];"),
    # more of the draws, the structured products and the checks
    ("phases scaled by a half", "out[e] = (double)bits53(x[0], x[1]) * two_m53;",
     "out[e] = 0.5 * (double)bits53(x[0], x[1]) * two_m53;"),
    ("fp32 box-muller radius without the factor 2", "const float r = sqrtf(-2.0f * logf(u1));",
     "const float r = sqrtf(-logf(u1));"),
    ("unitary circulant column not divided by n", "        c[t] /= (double)n;\n", ""),
    ("toeplitz kinds taken as circulants", "else if (kind <= 3)", "else if (kind <= 5)"),
    ("circulant rows transposed", "s += A[i * n + k] * c[((k - j) % N + N) % N];",
     "s += A[i * n + k] * c[((j - k) % N + N) % N];"),
    ("low-rank multiplier block transposed", ": H[((i - j) % n + n) % n];", ": H[((j - i) % n + n) % n];"),
    ("complex genp imaginary update adds", "im[i * n + j] -= lr * ui + li * ur;", "im[i * n + j] += lr * ui + li * ur;"),
    ("transposed solve reads L for U", "            const double u = LU[t * n + i];\n"
     "            for (int64_t c = 0; c < k; ++c) B[i * k + c] -= u * B[t * k + c];",
     "            const double u = LU[i * n + t];\n"
     "            for (int64_t c = 0; c < k; ++c) B[i * k + c] -= u * B[t * k + c];"),
    ("blocked genp U12 substitution drops a term",
     "for (int64_t t = k; t < i; ++t) M[i * n + j] -= M[i * n + t] * M[t * n + j];",
     "for (int64_t t = k; t + 1 < i; ++t) M[i * n + j] -= M[i * n + t] * M[t * n + j];"),
    ("residual without its compensation", "R[i * k + c] = s + err;", "R[i * k + c] = s;"),
    ("backward error blind to non-finite entries",
     "if (!isfinite(R[i * k + c]) || !isfinite(X[i * k + c])) { free(R); return INFINITY; }", ""),
    ("relative residual without the square root of b", "const double v = sqrt(rn) / sqrt(bn);",
     "const double v = sqrt(rn) / bn;"),
    ("growth denominator from the factors", "mm = fmax(mm, fabs(M[i * n + j]));", "mm = fmax(mm, fabs(LU[i * n + j]));"),
    ("two-sided solve drops H from X", "        orc_matmul(n, n, k, DH, Y, X);",
     "        memcpy(X, Y, sizeof(double) * (size_t)(n * k));"),
    ("qr reflection by half", "const double f = 2.0 * d / vv;\n                for (int64_t i = j; i < m; ++i) W[i * l + c]",
     "const double f = 1.0 * d / vv;\n                for (int64_t i = j; i < m; ++i) W[i * l + c]"),
]


def _run_pins(lib_path):
    # one thread per child, for the oracle's OpenMP and for numpy's BLAS (the pins may ask for more): the
    # children run side by side
    env = dict(os.environ, RMGE_ORACLE_LIB=lib_path, RMGE_ORACLE_THREADS="1", OMP_THREAD_LIMIT="1",
               OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    tests = sorted(os.path.join("tests", f) for f in os.listdir(os.path.join(ROOT, "tests"))
                   if f.startswith("test_oracle_") and f.endswith(".py"))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *tests],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-400:]


def _build(text, path):
    from oracle import build as B
    src = path + ".c"
    with open(src, "w") as f:
        f.write(text)
    return B.compile_source(src, path + ".so")


def test_every_planted_mistake_fails_a_pin(tmp_path):
    source = open(SRC).read()
    for name, old, _ in MISTAKES:
        assert source.count(old) == 1, f"{name}: the text to replace occurs {source.count(old)} times"
    jobs = [("unchanged", source)] + [(name, source.replace(old, new)) for name, old, new in MISTAKES]

    def build_and_run(i):
        return _run_pins(_build(jobs[i][1], str(tmp_path / f"m{i}")))

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = dict(zip((name for name, _ in jobs), ex.map(build_and_run, range(len(jobs)))))
    code, tail = results.pop("unchanged")
    assert code == 0, f"the unchanged oracle fails its pins when built this way:\n{tail}"
    # 1: some pin failed; a negative code: the copy crashed (a signal), which a pin run also reports
    survivors = {name: (c, t) for name, (c, t) in results.items() if not (c == 1 or c < 0)}
    assert not survivors, "mistakes no pin catches: " + "; ".join(f"{n} (exit {c})" for n, (c, _) in survivors.items())
