"""Pins of the FP64 oracle against facts the mathematics fixes.

The oracle (``oracle/``) restates the Bellman operator, value iteration and
exact policy iteration of a discounted cost-minimising MDP (madupite, "Problem
Setting and Solution Methods"; Bertsekas 2007).  None of these checks re-types
the oracle's formulas: each compares it with a closed form, a hand derivation,
brute force over every deterministic policy, an exact rational solve, or an
invariant of the Bellman operator.  ``test_pins_reject_planted_mistakes``
shows that every planted mistake in the oracle fails at least one pin.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from mdp_helpers import from_dense, random_dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Pins, written as functions of an oracle module so they can be replayed on a
# mutated oracle.
# ---------------------------------------------------------------------------

def pin_uniform_single_action(orc):
    """m = 1 and P(s'|s) = 1/n: V(s) = g(s) + gamma * mean(g) / (1 - gamma)."""
    rng = np.random.default_rng(11)
    n, gamma = 9, 0.8
    g = rng.random((n, 1))
    mdp = from_dense(np.full((n, 1, n), 1.0 / n), g, gamma)
    expect = g[:, 0] + gamma * g.mean() / (1 - gamma)
    V, pi, _, _ = orc.value_iteration(mdp, 1e-13)
    Vp, pip, _, _ = orc.policy_iteration(mdp)
    # constant cost: V = c / (1 - gamma) on every state
    mdpc = from_dense(np.full((n, 1, n), 1.0 / n), np.full((n, 1), 0.7), gamma)
    Vc = orc.policy_evaluate(mdpc, np.zeros(n, dtype=np.int32))
    return (np.allclose(V, expect, rtol=0, atol=1e-11) and np.allclose(Vp, expect, rtol=0, atol=1e-12)
            and np.allclose(Vc, 0.7 / (1 - gamma), rtol=0, atol=1e-12)
            and not pi.any() and not pip.any())


def pin_deterministic_cycle(orc):
    """m = 1, s -> s+1 mod n: V(s) = sum_{j<n} gamma^j g(s+j) / (1 - gamma^n)."""
    rng = np.random.default_rng(12)
    n, gamma = 7, 0.9
    g = rng.random(n)
    P = np.zeros((n, 1, n))
    for s in range(n):
        P[s, 0, (s + 1) % n] = 1.0
    mdp = from_dense(P, g[:, None], gamma)
    expect = np.array([sum(gamma**j * g[(s + j) % n] for j in range(n)) for s in range(n)])
    expect /= 1 - gamma**n
    V, _, _, _ = orc.value_iteration(mdp, 1e-13)
    Vp, _, _, _ = orc.policy_iteration(mdp)
    return np.allclose(V, expect, rtol=0, atol=1e-11) and np.allclose(Vp, expect, rtol=0, atol=1e-12)


def _golden_mdp():
    with open(os.path.join(GOLDEN, "two_state_two_action.json")) as f:
        d = json.load(f)
    frac = lambda x: Fraction(x[0], x[1])
    n, m = 2, 2
    P = np.zeros((n, m, n))
    g = np.zeros((n, m))
    for row in d["rows"]:
        g[row["s"], row["a"]] = float(frac(row["cost"]))
        for sp, p in row["succ"]:
            P[row["s"], row["a"], sp] = float(frac(p))
    return d, from_dense(P, g, float(frac(d["gamma"])))


def pin_golden_two_state(orc):
    """The hand-derived 2-state, 2-action example in tests/golden."""
    d, mdp = _golden_mdp()
    frac = lambda x: float(Fraction(x[0], x[1]))
    Vstar = np.array([frac(x) for x in d["V_star"]])
    Qstar = np.array([[frac(x) for x in row] for row in d["Q_star"]])
    gap = np.array([frac(x) for x in d["gap"]])
    V, pi, _, _ = orc.policy_iteration(mdp)
    Vv, piv, _, _ = orc.value_iteration(mdp, 1e-14)
    TV, tpi, Q, gp = orc.bellman(mdp, Vstar, want_q=True, want_gap=True)
    ok = np.allclose(V, Vstar, rtol=0, atol=1e-15) and np.allclose(Vv, Vstar, rtol=0, atol=1e-13)
    ok &= list(pi) == d["pi_star"] and list(piv) == d["pi_star"] and list(tpi) == d["pi_star"]
    ok &= np.allclose(Q, Qstar, rtol=0, atol=1e-15) and np.allclose(gp, gap, rtol=0, atol=1e-15)
    ok &= np.allclose(TV, Vstar, rtol=0, atol=1e-15)
    for key, vals in d["policy_values"].items():
        pol = np.array([int(x) for x in key.split(",")], dtype=np.int32)
        ok &= np.allclose(orc.policy_evaluate(mdp, pol), [frac(x) for x in vals], rtol=0, atol=1e-14)
    return bool(ok)


def _bruteforce(mdp):
    """Componentwise minimum over all m^n deterministic policies (numpy solves)."""
    n, m = mdp.n, mdp.m
    from mdp_helpers import to_dense
    P, g = to_dense(mdp)
    best = np.full(n, np.inf)
    for pol in itertools.product(range(m), repeat=n):
        Pp = P[np.arange(n), pol]
        gp = g[np.arange(n), pol]
        v = np.linalg.solve(np.eye(n) - mdp.gamma * Pp, gp)
        best = np.minimum(best, v)
    return best


def pin_bruteforce(orc):
    """V* from VI and exact PI equals the minimum over all m^n policies (n <= 6)."""
    rng = np.random.default_rng(13)
    ok = True
    for n, m in [(1, 3), (2, 2), (3, 3), (4, 2), (5, 3), (6, 4)]:
        gamma = float(rng.uniform(0.5, 0.95))
        mdp = from_dense(random_dense(n, m, rng), rng.random((n, m)), gamma)
        Vb = _bruteforce(mdp)
        V, pi, _, _ = orc.value_iteration(mdp, 1e-12)
        Vp, pip, _, _ = orc.policy_iteration(mdp)
        ok &= np.allclose(V, Vb, rtol=0, atol=1e-10) and np.allclose(Vp, Vb, rtol=0, atol=1e-10)
        # the returned policy attains V*
        ok &= np.allclose(orc.policy_evaluate(mdp, pip), Vb, rtol=0, atol=1e-10)
    return bool(ok)


def pin_exact_rational(orc):
    """Policy values against exact rational Gauss-Jordan elimination (Fraction)."""
    rng = np.random.default_rng(14)
    ok = True
    for n in (2, 3, 4):
        m = 2
        num = rng.integers(0, 5, size=(n, m, n))
        num[:, :, 0] += 1
        P = [[[Fraction(int(num[s, a, t]), int(num[s, a].sum())) for t in range(n)]
              for a in range(m)] for s in range(n)]
        g = [[Fraction(int(rng.integers(0, 9)), 4) for a in range(m)] for s in range(n)]
        gamma = Fraction(3, 4)
        pol = [int(x) for x in rng.integers(0, m, size=n)]
        # exact solve of (I - gamma P_pi) v = g_pi
        A = [[(1 if i == j else 0) - gamma * P[i][pol[i]][j] for j in range(n)] + [g[i][pol[i]]]
             for i in range(n)]
        for c in range(n):
            piv = next(r for r in range(c, n) if A[r][c] != 0)
            A[c], A[piv] = A[piv], A[c]
            A[c] = [x / A[c][c] for x in A[c]]
            for r in range(n):
                if r != c and A[r][c] != 0:
                    f = A[r][c]
                    A[r] = [x - f * y for x, y in zip(A[r], A[c])]
        exact = np.array([float(A[i][n]) for i in range(n)])
        Pd = np.array([[[float(x) for x in row] for row in st] for st in P])
        gd = np.array([[float(x) for x in row] for row in g])
        mdp = from_dense(Pd, gd, float(gamma))
        v = orc.policy_evaluate(mdp, np.array(pol, dtype=np.int32))
        ok &= np.allclose(v, exact, rtol=1e-14, atol=1e-14)
        # T_pi applied to the exact fixed point returns it
        ok &= np.allclose(orc.policy_apply(mdp, np.array(pol, dtype=np.int32), exact), exact,
                          rtol=0, atol=1e-14)
    return bool(ok)


def pin_operator_invariants(orc):
    """gamma-contraction and monotonicity of T; bounds on V*; V_pi >= V*."""
    rng = np.random.default_rng(15)
    mdp = synth.random_sparse(60, 3, 5, 1.0, 0.85, seed=7)
    ok = True
    for _ in range(20):
        V = rng.normal(size=mdp.n) * 3
        W = V + rng.normal(size=mdp.n)
        TV, _ = orc.bellman(mdp, V)
        TW, _ = orc.bellman(mdp, W)
        ok &= np.max(np.abs(TV - TW)) <= mdp.gamma * np.max(np.abs(V - W)) * (1 + 1e-12)
        Wup = V + np.abs(rng.normal(size=mdp.n))
        TWup, _ = orc.bellman(mdp, Wup)
        ok &= bool(np.all(TWup >= TV - 1e-12))
    Vs, _, _, _ = orc.policy_iteration(mdp)
    gmin, gmax = mdp.g.min(), mdp.g.max()
    ok &= bool(np.all(Vs >= gmin / (1 - mdp.gamma) - 1e-12) and np.all(Vs <= gmax / (1 - mdp.gamma) + 1e-12))
    for _ in range(5):
        pol = rng.integers(0, mdp.m, size=mdp.n).astype(np.int32)
        ok &= bool(np.all(orc.policy_evaluate(mdp, pol) >= Vs - 1e-11))
    return bool(ok)


def pin_greedy_tie_break(orc):
    """Identical actions tie exactly: the greedy policy takes the lowest index."""
    rng = np.random.default_rng(16)
    n, m = 5, 3
    P1 = random_dense(n, 1, rng)
    P = np.repeat(P1, m, axis=1)
    g = np.repeat(rng.random((n, 1)), m, axis=1)
    mdp = from_dense(P, g, 0.9)
    _, pi = orc.bellman(mdp, rng.random(n))
    # action 2 strictly better at state 0 only
    g2 = g.copy()
    g2[0, 2] -= 0.5
    _, pi2 = orc.bellman(from_dense(P, g2, 0.9), rng.random(n))
    return (not pi.any()) and pi2[0] == 2 and not pi2[1:].any()


PINS = [pin_uniform_single_action, pin_deterministic_cycle, pin_golden_two_state, pin_bruteforce,
        pin_exact_rational, pin_operator_invariants, pin_greedy_tie_break]


@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin):
    assert pin(oracle)


# ---------------------------------------------------------------------------
# Further properties of the oracle's iterations
# ---------------------------------------------------------------------------

def test_value_iteration_residual_contracts():
    mdp = synth.random_sparse(200, 4, 6, 1.0, 0.9, seed=21)
    _, _, _, hist = oracle.value_iteration(mdp, 1e-10)
    h = np.array(hist)
    assert np.all(h[1:] <= mdp.gamma * h[:-1] * (1 + 1e-12) + 1e-15)


def test_policy_iteration_monotone_and_matches_vi():
    mdp = synth.random_sparse_n1000()
    Vp, pip, it, hist = oracle.policy_iteration(mdp)
    for a, b in zip(hist[:-1], hist[1:]):
        assert np.all(b <= a + 1e-12)
    Vv, piv, _, _ = oracle.value_iteration(mdp, 1e-11)
    assert np.max(np.abs(Vp - Vv)) <= 1e-10
    # the greedy policies agree wherever the Q-gap is clearly positive
    cert = oracle.certificate(mdp, Vp)
    clear = cert["gap"] > 1e-8
    assert np.array_equal(pip[clear], piv[clear])
    assert cert["res_inf"] <= 1e-12


def test_certificate_bounds_error():
    mdp = synth.random_sparse(300, 3, 5, 1.0, 0.95, seed=22)
    Vs, _, _, _ = oracle.policy_iteration(mdp)
    rng = np.random.default_rng(23)
    for scale in (1e-1, 1e-4, 1e-8):
        V = Vs + scale * rng.normal(size=mdp.n)
        c = oracle.certificate(mdp, V)
        assert np.max(np.abs(V - Vs)) <= c["bound"] * (1 + 1e-9) + 1e-13


def test_bellman_on_subrange_matches_whole():
    full = synth.banded(3000, 4, 6, 200, 0.5, 0.95, seed=24)
    part = synth.banded(3000, 4, 6, 200, 0.5, 0.95, seed=24, s0=1000, s1=1700)
    V = np.random.default_rng(25).random(3000)
    TV, pi = oracle.bellman(full, V)
    TVp, pip = oracle.bellman(part, V)
    assert np.array_equal(TV[1000:1700], TVp) and np.array_equal(pi[1000:1700], pip)


def test_fp32_storage_is_read_exactly():
    m32 = synth.random_sparse(100, 3, 4, 1.0, 0.9, seed=26, dtype=np.float32)
    m64 = synth.CSRMDP(n=m32.n, m=m32.m, gamma=m32.gamma, row_ptr=m32.row_ptr, col=m32.col,
                       val=m32.val.astype(np.float64), g=m32.g.astype(np.float64))
    V = np.random.default_rng(27).random(100)
    a, b = oracle.bellman(m32, V), oracle.bellman(m64, V)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ---------------------------------------------------------------------------
# Planted mistakes: each mutation of the oracle must fail at least one pin.
# ---------------------------------------------------------------------------

class _Mutant:
    """A copy of the oracle's public API with ``bellman``/``policy_apply`` swapped."""

    def __init__(self, bellman=None, policy_apply=None, policy_matrix=None):
        import types
        import builtins
        self.mod = types.ModuleType("oracle_mutant")
        self.mod.__dict__["__builtins__"] = builtins
        for k in dir(oracle):
            if not k.startswith("__"):
                setattr(self.mod, k, getattr(oracle, k))
        # rebind the module-level functions so that internal calls use the mutants
        src_funcs = ["value_iteration", "policy_iteration", "policy_evaluate", "greedy",
                     "certificate"]
        import types as _t
        for name in src_funcs:
            f = getattr(oracle, name)
            setattr(self.mod, name, _t.FunctionType(f.__code__, self.mod.__dict__, name,
                                                    f.__defaults__, f.__closure__))
        if bellman:
            self.mod.bellman = bellman
        if policy_apply:
            self.mod.policy_apply = policy_apply
        if policy_matrix:
            self.mod.policy_matrix = policy_matrix


def _with_gamma(mdp, gamma):
    return synth.CSRMDP(n=mdp.n, m=mdp.m, gamma=gamma, row_ptr=mdp.row_ptr, col=mdp.col,
                        val=mdp.val, g=mdp.g, s0=mdp.s0)


def _mut_gamma_squared():
    def b(mdp, V, want_q=False, want_gap=False):
        return oracle.bellman(_with_gamma(mdp, mdp.gamma**2), V, want_q, want_gap)

    def pm(mdp, pi):
        P, gp = oracle.policy_matrix(mdp, pi)
        return P * mdp.gamma, gp
    return _Mutant(bellman=b, policy_matrix=pm)


def _mut_argmax():
    def b(mdp, V, want_q=False, want_gap=False):
        TV, pi, Q, gap = oracle.bellman(mdp, V, want_q=True, want_gap=True)
        pi = np.argmax(Q, axis=1).astype(np.int32)
        TV = Q.max(axis=1)
        return (TV, pi, Q if want_q else None, gap) if (want_q or want_gap) else (TV, pi)
    return _Mutant(bellman=b)


def _mut_tie_highest():
    def b(mdp, V, want_q=False, want_gap=False):
        TV, pi, Q, gap = oracle.bellman(mdp, V, want_q=True, want_gap=True)
        pi = (Q.shape[1] - 1 - np.argmin(Q[:, ::-1], axis=1)).astype(np.int32)
        return (TV, pi, Q if want_q else None, gap) if (want_q or want_gap) else (TV, pi)
    return _Mutant(bellman=b)


def _transpose(mdp):
    from mdp_helpers import to_dense
    P, g = to_dense(mdp)
    Pt = np.transpose(P, (2, 1, 0))  # P'(s'|s,a) = P(s|s',a): a transposed operand
    return from_dense(Pt, g, mdp.gamma)


def _mut_transposed():
    def b(mdp, V, want_q=False, want_gap=False):
        return oracle.bellman(_transpose(mdp), V, want_q, want_gap)

    def pm(mdp, pi):
        P, gp = oracle.policy_matrix(mdp, pi)
        return P.T.copy(), gp

    def pa(mdp, pi, V):
        return oracle.policy_apply(_transpose(mdp), pi, V)
    return _Mutant(bellman=b, policy_matrix=pm, policy_apply=pa)


def _mut_cost_row_shift():
    """Off-by-one row index for the cost: g(s, a+1) read as g(s, a)."""
    def shifted(mdp):
        g = np.roll(np.asarray(mdp.g), -1)
        return synth.CSRMDP(n=mdp.n, m=mdp.m, gamma=mdp.gamma, row_ptr=mdp.row_ptr,
                            col=mdp.col, val=mdp.val, g=g, s0=mdp.s0)

    def b(mdp, V, want_q=False, want_gap=False):
        return oracle.bellman(shifted(mdp), V, want_q, want_gap)

    def pm(mdp, pi):
        return oracle.policy_matrix(shifted(mdp), pi)
    return _Mutant(bellman=b, policy_matrix=pm)


def _mut_dropped_last_term():
    """Each row's last successor dropped from the expectation."""
    def dropped(mdp):
        keep = np.ones(mdp.nnz, dtype=bool)
        keep[mdp.row_ptr[1:] - 1] = False
        counts = np.diff(mdp.row_ptr) - 1
        rp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        return synth.CSRMDP(n=mdp.n, m=mdp.m, gamma=mdp.gamma, row_ptr=rp, col=mdp.col[keep],
                            val=mdp.val[keep], g=mdp.g, s0=mdp.s0)

    def b(mdp, V, want_q=False, want_gap=False):
        return oracle.bellman(dropped(mdp), V, want_q, want_gap)

    def pm(mdp, pi):
        return oracle.policy_matrix(dropped(mdp), pi)

    def pa(mdp, pi, V):
        return oracle.policy_apply(dropped(mdp), pi, V)
    return _Mutant(bellman=b, policy_matrix=pm, policy_apply=pa)


MUTANTS = {"gamma_squared": _mut_gamma_squared, "argmax": _mut_argmax,
           "tie_highest": _mut_tie_highest, "transposed_P": _mut_transposed,
           "cost_row_shift": _mut_cost_row_shift, "dropped_term": _mut_dropped_last_term}


def _fails(pin, mod):
    try:
        return not pin(mod)
    except (AssertionError, RuntimeError, ValueError, IndexError, np.linalg.LinAlgError):
        return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistakes(name):
    mod = MUTANTS[name]().mod
    failed = [p.__name__ for p in PINS if _fails(p, mod)]
    assert failed, f"mutant {name} passed every pin"
