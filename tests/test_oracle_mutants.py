"""The pins catch planted mistakes.

Each mutant is oracle.c with one plausible slip (a dropped term, a wrong
sign, a wrong index, a transposed operand, a broken heap or sort) compiled
to a temporary library; at least one quick pin must fail against it.  This
keeps the oracle's pins honest: a pin set that passes a broken oracle pins
nothing.
"""
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1306_4743_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")

MUTANTS = [
    ("3D branch dropped",
     "  if (u <= a3) return u;\n  double b2", "  return u;\n  double b2"),
    ("wrong root sign, 2 terms",
     "u = a1 + 0.5 * (b + sqrt(disc2));", "u = a1 + 0.5 * (b - sqrt(disc2));"),
    ("dropped term in 3-term discriminant",
     "3.0 * (b2 * b2 + b3 * b3 - s * s)", "3.0 * (b2 * b2 - s * s)"),
    ("wrong divisor, 3 terms",
     "return a1 + (p + sqrt(disc3)) / 3.0;", "return a1 + (p + sqrt(disc3)) / 2.0;"),
    ("third compare-swap of the sort dropped",
     "  if (a1 > a2) { t = a1; a1 = a2; a2 = t; }\n  if (isinf(a1)) return INFINITY; /* no finite",
     "  if (isinf(a1)) return INFINITY; /* no finite"),
    ("y stride uses ny",
     "if (j > 0 && V[c - nx] < m) m = V[c - nx];",
     "if (j > 0 && V[c - ny] < m) m = V[c - ny];"),
    ("transposed operands of s = h / F in FMM",
     "double v = orc_local_solve(ax, ay, az, h / (double)F[y]);",
     "double v = orc_local_solve(ax, ay, az, (double)F[y] / h);"),
    ("heap compares the wrong way",
     "if (H->key[H->heap[parent]] <= H->key[H->heap[p]]) break;",
     "if (H->key[H->heap[parent]] >= H->key[H->heap[p]]) break;"),
    ("z neighbour skipped",
     "if (k + 1 < nz && V[c + nx * ny] < m) m = V[c + nx * ny];", ""),
    ("exit nodes recomputed in FMM",
     "      if (accepted[y] || mask[y]) continue;", "      if (accepted[y]) continue;"),
    ("residual takes a signed difference",
     "double e = fabs(U[x] - v);", "double e = U[x] - v;"),
    ("residual keeps the smallest difference",
     "if (e > r) r = e;", "if (e < r) r = e;"),
    ("residual includes exit nodes",
     "        if (mask[x]) continue;\n        double ax, ay, az;\n        axis_minima(U, i, j, k,",
     "        double ax, ay, az;\n        axis_minima(U, i, j, k,"),
    ("residual does not count non-finite values",
     "if (!isfinite(U[x])) { ++bad; continue; }", "if (!isfinite(U[x])) continue;"),
    ("residual uses s = F / h",
     "double v = orc_local_solve(ax, ay, az, h / (double)F[x]);\n        double e",
     "double v = orc_local_solve(ax, ay, az, (double)F[x] / h);\n        double e"),
]


def _pin_closed_forms():
    s = 1.0 / 64
    assert oracle.local_solve(0.0, 0.0, 0.0, s) == pytest.approx(s / math.sqrt(3), rel=1e-14)
    assert oracle.local_solve(0.0, 0.0, math.inf, s) == pytest.approx(s / math.sqrt(2), rel=1e-14)
    assert oracle.local_solve(0.0, math.inf, math.inf, s) == s


def _pin_equation():
    rng = np.random.default_rng(5)
    for _ in range(300):
        s = float(10 ** rng.uniform(-3, 0))
        a = [float(v) for v in rng.permutation(rng.uniform(0, 1.2, 3) * s + 0.5)]
        u = oracle.local_solve(*a, s)
        lhs = sum(max(u - ad, 0.0) ** 2 for ad in a) - s * s
        assert abs(lhs) <= 1e-12 * s * s


def _pin_tiny_brute_force():
    rng = np.random.default_rng(6)
    for _ in range(10):
        nx, ny, nz = (int(v) for v in rng.integers(3, 7, 3))
        F = rng.uniform(0.2, 2.0, (nz, ny, nx)).astype(np.float32)
        mask = np.zeros_like(F, dtype=np.uint8)
        q = np.zeros(F.shape)
        mask.reshape(-1)[rng.integers(0, F.size)] = 1
        U = oracle.fmm(F, mask, q, 0.1)
        V, _ = oracle.value_iteration(F, mask, q, 0.1)
        with np.errstate(invalid="ignore"):  # a mutant may leave inf - inf
            assert np.max(np.abs(U - V)) <= 1e-14 * U.max()


def _pin_exact_1d():
    f = np.linspace(0.5, 1.5, 20).astype(np.float32).reshape(1, 1, 20)
    mask = np.zeros(f.shape, np.uint8)
    mask[0, 0, 0] = 1
    U = oracle.fmm(f, mask, np.zeros(f.shape), 0.1).reshape(-1)
    expect = np.concatenate([[0.0], np.cumsum(0.1 / f.reshape(-1)[1:].astype(np.float64))])
    np.testing.assert_allclose(U, expect, rtol=1e-15)


def _pin_table5_head():
    p = W.paper_example(2, 24)
    U, sweeps, mc, nc = oracle.fsm(p.F, p.mask, p.q, p.h, dir_order=(0, 1, 3, 2, 4, 5, 7, 6))
    V = oracle.fmm(p.F, p.mask, p.q, p.h)
    with np.errstate(invalid="ignore"):  # a mutant may leave inf - inf
        assert np.max(np.abs(U - V)) <= 1e-13 * V.max()


def _pin_exit_dirichlet():
    F = np.ones((3, 4, 5), np.float32)
    mask = np.zeros(F.shape, np.uint8)
    q = np.zeros(F.shape)
    mask[0, 0, 0] = 1
    mask[0, 0, 1] = 1
    q[0, 0, 1] = 3.0
    U = oracle.fmm(F, mask, q, 0.2)
    assert U[0, 0, 1] == 3.0


def _pin_residual():
    # closed-form residuals of perturbed exact solutions (see
    # test_oracle_residual.py): a raised interior node and a lowered end
    # node of the exact 1D line give delta, an inconsistent exit gives 0,
    # non-finite values are counted
    N, h = 30, 1.0 / 29
    f = np.linspace(0.6, 1.4, N).astype(np.float32)
    F = f.reshape(1, 1, N)
    mask = np.zeros(F.shape, np.uint8)
    mask[0, 0, 3] = 1
    s = h / f.astype(np.float64)
    U = np.empty(N)
    U[3] = 0.0
    for i in range(4, N):
        U[i] = U[i - 1] + s[i]
    for i in range(2, -1, -1):
        U[i] = U[i + 1] + s[i]
    delta = 1e-3
    for node, sign in ((15, 1.0), (N - 1, -1.0)):
        V = U.copy()
        V[node] += sign * delta
        r, bad = oracle.residual(V.reshape(F.shape), F, mask, h)
        assert bad == 0 and abs(r - delta) <= 1e-14
    m2 = mask.copy()
    m2[0, 0, 20] = 1
    q2 = np.zeros(F.shape)
    q2[0, 0, 20] = 5.0
    W2 = U.copy()
    W2[20] = 5.0
    for i in range(21, N):
        W2[i] = W2[i - 1] + s[i]
    r, bad = oracle.residual(W2.reshape(F.shape), F, m2, h)
    assert bad == 0 and r == 0.0
    V = U.copy()
    V[0] = np.inf
    V[N - 1] = np.nan
    r, bad = oracle.residual(V.reshape(F.shape), F, mask, h)
    assert bad == 2


PINS = [_pin_closed_forms, _pin_equation, _pin_tiny_brute_force, _pin_exact_1d,
        _pin_table5_head, _pin_exit_dirichlet, _pin_residual]


def test_unmutated_oracle_passes_quick_pins():
    for pin in PINS:
        pin()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found: " + name
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    "-w", "-o", str(so), str(mut), "-lm"], check=True)
    lib = oracle.load_library(str(so))
    failures = 0
    with oracle.use_library(lib):
        for pin in PINS:
            try:
                pin()
            except (AssertionError, oracle.OracleError):
                failures += 1
    assert failures > 0, "no pin caught: " + name
