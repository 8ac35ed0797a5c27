"""The solver's host-side decisions (csrc/host_logic.h: the look-ahead to restart
criterion (iii), the restart kind, Algorithm 3's primal weight), compiled with g++ and
checked on the CPU against brute force, the restart rules of Sec. 3 and the oracle's
primal weight update."""
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import pdlp_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2501_07018_gb300", "csrc", "host_logic.h")
NEVER = (2**63 - 1) // 4

DRIVER = r"""
#include <cstdio>
#include "host_logic.h"
int main() {
  char op;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'S') {
      long long k, t; double b;
      std::scanf("%lld %lld %la", &k, &t, &b);
      std::printf("%lld\n", (long long)pdlp::steps_to_artificial(k, t, b));
    } else if (op == 'K') {
      int c, a, h; double mc, mr, mp, bs, bn;
      std::scanf("%d %d %d %la %la %la %la %la", &c, &a, &h, &mc, &mr, &mp, &bs, &bn);
      std::printf("%d\n", pdlp::restart_kind(c, a, h, mc, mr, mp, bs, bn));
    } else if (op == 'W') {
      double om, dx, dy, th, ez;
      std::scanf("%la %la %la %la %la", &om, &dx, &dy, &th, &ez);
      std::printf("%a\n", pdlp::primal_weight(om, dx, dy, th, ez));
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def run():
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "driver.cpp"), os.path.join(d, "driver")
    with open(src, "w") as f:
        f.write(DRIVER)
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", os.path.dirname(HEADER), "-o", exe, src],
                   check=True)

    def call(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout.split()
        assert len(out) == len(lines)
        return out

    yield call
    for p in (src, exe):
        os.remove(p)
    os.rmdir(d)


def _first_art(k, t, beta):
    """Smallest j >= 1 with t + j >= beta (k + j), the test of criterion (iii) in the same
    double arithmetic, by stepping j."""
    if not beta < 1.0:
        return NEVER
    j = 1
    while not (float(t + j) >= beta * float(k + j)):
        j += 1
    return j


def test_lookahead_to_criterion_iii_matches_brute_force(run):
    rng = np.random.default_rng(3)
    cases = []
    for beta in (0.5, 0.25, 0.1, 0.3, 0.7, 0.9, 0.99, 1.0, 1.5):
        big = [int(v) for v in rng.integers(70, 5000, 40)] if beta < 0.95 else []
        for k in list(range(0, 70)) + big:
            for t in sorted({0, 1, k // 3, k // 2, k} | {int(v) for v in rng.integers(0, k + 1, 4)}):
                if t <= k:
                    cases.append((k, t, beta))
    got = run([f"S {k} {t} {float(b).hex()}" for k, t, b in cases])
    for (k, t, b), g in zip(cases, got):
        assert int(g) == _first_art(k, t, b), (k, t, b)


def test_lookahead_at_large_counts(run):
    # the closed-form estimate path: j follows from one division, then settles exactly
    cases = [(10**12, 3, 0.5), (10**12 + 7, 10**11, 0.25), (2**40 + 1, 2**39, 0.5)]
    got = run([f"S {k} {t} {float(b).hex()}" for k, t, b in cases])
    for (k, t, b), g in zip(cases, got):
        j = int(g)
        assert float(t + j) >= b * float(k + j)
        assert j == 1 or not (float(t + j - 1) >= b * float(k + j - 1))


def test_lookahead_beyond_range_is_never(run):
    """beta_art just below 1 at large k: the next (iii) iteration lies beyond 2^52 steps
    (here ~1e19), where a double no longer resolves single iterations; the look-ahead
    answers "never" at once instead of converting that count to an integer or stepping
    towards it; NaN likewise."""
    b = 1.0 - 2.0**-53
    cases = [(1000, 0, b), (10**6, 3, b), (2**40, 1, 1.0 - 2.0**-40), (5, 1, math.nan)]
    got = run([f"S {k} {t} {float(bb).hex()}" for k, t, bb in cases])
    assert [int(g) for g in got] == [NEVER] * len(cases)
    # just inside the range the exact answer is still returned
    k, t, bb = 2**20, 0, 1.0 - 2.0**-30
    j = int(run([f"S {k} {t} {float(bb).hex()}"])[0])
    assert float(t + j) >= bb * float(k + j) and not (float(t + j - 1) >= bb * float(k + j - 1))


def _kind(is_check, is_art, have, mu_c, mu_ref, mu_prev, bs, bn):
    # Sec. 3: (i) sufficient decay, (ii) necessary decay without progress -- both at the
    # periodic evaluations once the reference gap exists -- else (iii) artificial
    if is_check and have and mu_c <= bs * mu_ref:
        return 1
    if is_check and have and mu_c <= bn * mu_ref and mu_c > mu_prev:
        return 2
    return 3 if is_art else 0


def test_restart_kind_follows_the_criteria(run):
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(3000):
        mu_ref = float(rng.choice([0.0, 1.0, rng.random() * 10]))
        mu_c = float(rng.choice([0.0, 0.1 * mu_ref, 0.5 * mu_ref, 0.9 * mu_ref, mu_ref,
                                 rng.random() * 10]))
        mu_prev = float(rng.choice([math.inf, mu_c, 0.5 * mu_c, 2 * mu_c, rng.random() * 10]))
        cases.append((int(rng.integers(2)), int(rng.integers(2)), int(rng.integers(2)),
                      mu_c, mu_ref, mu_prev, 0.1, 0.9))
    # the boundaries: equality in (i) and (ii), and no (ii) on the first check (+inf)
    cases += [(1, 0, 1, 0.1, 1.0, math.inf, 0.1, 0.9), (1, 1, 1, 0.9, 1.0, 0.5, 0.1, 0.9),
              (1, 1, 1, 0.9, 1.0, math.inf, 0.1, 0.9), (0, 1, 1, 0.0, 1.0, 1.0, 0.1, 0.9),
              (1, 1, 0, 0.0, 1.0, 1.0, 0.1, 0.9)]
    lines = [f"K {c} {a} {h} " + " ".join(float(v).hex() for v in (mc, mr, mp, bs, bn))
             for c, a, h, mc, mr, mp, bs, bn in cases]
    got = run(lines)
    for cs, g in zip(cases, got):
        assert int(g) == _kind(*cs), cs
    assert [int(g) for g in got[-5:]] == [1, 2, 3, 3, 3]


def test_primal_weight_matches_the_oracle(run):
    rng = np.random.default_rng(7)
    cases = []
    for _ in range(500):
        omega = float(np.exp(rng.uniform(-5, 5)))
        dx = float(rng.choice([0.0, 1e-11, 1e11, np.exp(rng.uniform(-8, 8))]))
        dy = float(rng.choice([0.0, 1e-11, 1e11, np.exp(rng.uniform(-8, 8))]))
        theta = float(rng.choice([0.5, 0.2, 1.0]))
        cases.append((omega, dx, dy, theta, 1e-10))
    got = run(["W " + " ".join(float(v).hex() for v in cs) for cs in cases])
    for (om, dx, dy, th, ez), g in zip(cases, got):
        want = O.primal_weight_update(np.array([dx]), np.array([dy]), np.zeros(1), np.zeros(1),
                                      om, th, ez)
        assert float.fromhex(g) == pytest.approx(want, rel=1e-14), (om, dx, dy, th)
        if not (ez < dx < 1 / ez and ez < dy < 1 / ez):
            assert float.fromhex(g) == om  # unchanged outside (eps_zero, 1/eps_zero)
