"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each ``pin_*`` takes a loaded oracle library (the real one or a deliberately
broken copy) and returns a list of failure messages; an empty list means the
pin holds. ``tests/test_oracle.py`` requires every pin to hold on the real
oracle; ``tests/test_oracle_mutants.py`` requires every planted mistake to
break at least one pin.

Sources of truth:
* hand-computed rationals for Eq. 4, Eq. 1 and Eq. 3 (``golden/*.json``);
* the closed form sum_j u_ij^m d_ij^2 = (sum_k d_ik^(-2/(m-1)))^(1-m), which
  holds whenever U comes from Eq. 4 (algebra: u_j = w_j / W with
  w_j = d_j^(-2/(m-1)), and u_j^m d_j^2 = w_j / W^m);
* optimality (Bezdek): Eq. 3 minimises J over V for fixed U, and Eq. 4
  minimises J over each pixel's membership simplex for fixed V;
* special cases: C = 1 gives the mean; point masses are fixed points;
* metamorphic relations: translating, scaling or reflecting x moves V the
  same way and leaves U unchanged; permuting pixels permutes U;
* monotone descent of J along the iteration (alternating minimisation);
* a naive nested-loop Algorithm 1 on tiny inputs, with Eq. 4 in its
  ratio-of-distances form and real powers;
* the fixed-point property of a run stopped at a tight tolerance.
"""
from __future__ import annotations

import json
import os
from fractions import Fraction

import numpy as np

import oracle
import phantom

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _frac(a):
    return np.array([[float(Fraction(str(v))) for v in row] for row in a])


def _check(fails, cond, msg):
    if not cond:
        fails.append(msg)


def pin_toy_rationals(L):
    fails = []
    g = _golden("toy_two_cluster.json")
    x, V = g["x"], g["V"]
    for name, c in g["cases"].items():
        m = c["m"]
        U = oracle.memberships(x, V, m, L=L)
        _check(fails, np.allclose(U, _frac(c["U"]), rtol=0, atol=1e-15),
               f"toy {name}: U {U.tolist()}")
        if "J" in c:
            J = oracle.objective(x, U, V, m, L=L)
            ref = float(Fraction(c["J"]))
            _check(fails, abs(J - ref) <= 1e-13 * ref, f"toy {name}: J {J} vs {ref}")
        if "V_next" in c:
            Vn = oracle.centers(x, U, m, L=L)[0]
            ref = [float(Fraction(v)) for v in c["V_next"]]
            _check(fails, np.allclose(Vn, ref, rtol=1e-14, atol=0),
                   f"toy {name}: V_next {Vn}")
    return fails


def pin_singular_points(L):
    fails = []
    for c in _golden("singular_points.json")["cases"]:
        U = oracle.memberships(c["x"], c["V"], c["m"], L=L)
        _check(fails, np.allclose(U, _frac(c["U"]), rtol=0, atol=1e-15),
               f"singular {c['x']} {c['V']}: {U.tolist()}")
    # a fixed point of the loop: V0 on the two pixels gives U = I, delta = 0
    r = oracle.fcm([0.0, 10.0], 2, 2.0, 1e-5, 50, V0=[0.0, 10.0], L=L)
    _check(fails, r["iters"] == 1 and r["status"] == oracle.CONVERGED
           and r["delta"][0] == 0.0 and np.array_equal(r["V"], [0.0, 10.0])
           and np.array_equal(r["U"], np.eye(2)), f"fixed point run: {r['iters']} {r['V']}")
    return fails


def pin_closed_form_objective(L):
    fails = []
    g = np.random.default_rng(7)
    for m in (1.5, 2.0, 2.5, 3.0, 4.0):
        for C in (2, 3, 5, 8):
            x = g.uniform(0, 255, 200)
            V = g.uniform(0, 255, C)
            U = oracle.memberships(x, V, m, L=L)
            J = oracle.objective(x, U, V, m, L=L)
            d2 = (x[None, :] - V[:, None]) ** 2
            ref = np.sum(np.sum(d2 ** (-1.0 / (m - 1.0)), axis=0) ** (1.0 - m))
            _check(fails, abs(J - ref) <= 1e-11 * ref, f"closed form m={m} C={C}: {J} vs {ref}")
    return fails


def pin_optimality(L):
    """Eq. 3 minimises J(U, .) and Eq. 4 minimises J(., V) on the simplex."""
    fails = []
    g = np.random.default_rng(11)
    for m in (1.5, 2.0, 3.0):
        x = g.uniform(0, 255, 60)
        C = 4
        V = np.sort(g.uniform(0, 255, C))
        U = oracle.memberships(x, V, m, L=L)
        # perturb one pixel's membership along e_a - e_b; compare that
        # pixel's own term of J so the change is not lost in rounding
        for t in range(40):
            i = int(g.integers(0, x.size))
            a, b = g.choice(C, 2, replace=False)
            h = 1e-3 * min(U[b, i], 1 - U[a, i]) if g.random() < 0.5 else -1e-3 * min(U[a, i], 1 - U[b, i])
            if abs(h) < 1e-6:
                continue
            xi, Ui = x[i:i + 1], U[:, i:i + 1]
            U2 = Ui.copy()
            U2[a, 0] += h
            U2[b, 0] -= h
            _check(fails, oracle.objective(xi, U2, V, m, L=L) > oracle.objective(xi, Ui, V, m, L=L),
                   f"membership not a minimiser m={m} pixel {i}")
        # centers from a random membership minimise J(U, .)
        Ur = g.dirichlet(np.ones(C), x.size).T
        Vs = oracle.centers(x, Ur, m, L=L)[0]
        Js = oracle.objective(x, Ur, Vs, m, L=L)
        for j in range(C):
            for h in (1e-3, -1e-3):
                V2 = Vs.copy()
                V2[j] += h
                _check(fails, oracle.objective(x, Ur, V2, m, L=L) > Js,
                       f"center not a minimiser m={m} j={j}")
    return fails


def pin_special_cases(L):
    fails = []
    g = np.random.default_rng(3)
    x = g.uniform(0, 255, 101)
    # C = 1: u = 1, V = mean(x); delta_1 = 0 with U0 = 1
    r = oracle.fcm(x, 1, 2.0, 1e-5, 10, U0=np.ones((1, x.size)), L=L)
    _check(fails, np.allclose(r["U"], 1.0, rtol=0, atol=0), "C=1: U != 1")
    _check(fails, abs(r["V"][0] - np.mean(x)) <= 1e-12 * np.mean(x), f"C=1: V {r['V']} vs mean")
    _check(fails, r["iters"] == 1 and r["status"] == oracle.CONVERGED, "C=1: iters")
    # stopping rule is strict: delta = 0 is not < eps = 0
    r = oracle.fcm(x, 1, 2.0, 0.0, 4, U0=np.ones((1, x.size)), L=L)
    _check(fails, r["iters"] == 4 and r["status"] == oracle.NOT_CONVERGED,
           f"strict stop: iters {r['iters']} status {r['status']}")
    # point masses are the fixed point, for every m
    xp = np.array([20.0] * 30 + [100.0] * 50 + [180.0] * 20)
    u0 = phantom.dirichlet_u0((9, 1), 3, xp.size)
    for m in (1.5, 2.0, 3.0):
        r = oracle.fcm(xp, 3, m, 1e-12, 1000, U0=u0, L=L)
        _check(fails, np.allclose(np.sort(r["V"]), [20, 100, 180], rtol=0, atol=1e-9)
               and r["status"] == oracle.CONVERGED, f"point masses m={m}: {r['V']}")
    # defuzzification ties go to the lowest cluster index
    lab = oracle.labels(np.array([[0.5, 0.2, 0.4], [0.5, 0.4, 0.4], [0.0, 0.4, 0.2]]), L=L)
    _check(fails, lab.tolist() == [0, 1, 0], f"labels ties {lab.tolist()}")
    return fails


def _small_phantom():
    img, _ = phantom.phantom2d(21, 48, 40, 8.0)
    x = img.reshape(-1).astype(np.float64)
    return x, phantom.dirichlet_u0((21, 2), 4, x.size)


def pin_descent_and_invariants(L):
    fails = []
    x, u0 = _small_phantom()
    for m in (1.5, 2.0, 3.0):
        r = oracle.fcm(x, 4, m, 1e-7, 400, U0=u0, L=L)
        U = r["U"]
        _check(fails, np.max(np.abs(U.sum(0) - 1)) <= 1e-14, f"sum u != 1 (m={m})")
        _check(fails, U.min() >= 0 and U.max() <= 1, f"u outside [0, 1] (m={m})")
        J = r["J"]
        _check(fails, np.all(np.diff(J) <= 1e-12 * J[0]), f"J increases (m={m})")
        _check(fails, np.all(r["Vtrace"] >= x.min()) and np.all(r["Vtrace"] <= x.max()),
               f"V outside [min x, max x] (m={m})")
        # the reported delta is max |U^k - U^{k-1}|: recompute the last one
        if r["iters"] >= 2:
            Uk = oracle.memberships(x, r["Vtrace"][-1], m, L=L)
            Uk1 = oracle.memberships(x, r["Vtrace"][-2], m, L=L)
            _check(fails, abs(np.max(np.abs(Uk - Uk1)) - r["delta"][-1]) <= 1e-15,
                   f"delta is not max|dU| (m={m})")
        _check(fails, r["status"] == oracle.CONVERGED and r["delta"][-1] < 1e-7, f"no convergence m={m}")
    return fails


def pin_metamorphic(L):
    fails = []
    x, u0 = _small_phantom()
    m = 2.0
    base = oracle.fcm(x, 4, m, 1e-6, 300, U0=u0, L=L)
    for name, fx, fv in (("translate", lambda a: a + 37.0, lambda v: v + 37.0),
                         ("scale", lambda a: a * 0.75, lambda v: v * 0.75),
                         ("reflect", lambda a: 255.0 - a, lambda v: 255.0 - v)):
        r = oracle.fcm(fx(x), 4, m, 1e-6, 300, U0=u0, L=L)
        _check(fails, r["iters"] == base["iters"], f"{name}: iters {r['iters']} vs {base['iters']}")
        _check(fails, np.allclose(r["V"], fv(base["V"]), rtol=1e-9, atol=1e-9), f"{name}: V")
        _check(fails, np.allclose(r["U"], base["U"], rtol=0, atol=1e-9), f"{name}: U")
    perm = np.random.default_rng(5).permutation(x.size)
    r = oracle.fcm(x[perm], 4, m, 1e-6, 300, U0=u0[:, perm], L=L)
    _check(fails, r["iters"] == base["iters"] and np.allclose(r["V"], base["V"], rtol=1e-10)
           and np.allclose(r["U"], base["U"][:, perm], atol=1e-10), "permutation")
    return fails


def pin_quantized_matches_plain(L):
    """The 256-bin loop equals the per-pixel loop (brFCM identity)."""
    fails = []
    img, _ = phantom.phantom2d(31, 72, 64, 9.0)
    xq = img.reshape(-1)
    x = xq.astype(np.float64)
    u0 = phantom.dirichlet_u0((31, 2), 4, x.size)
    for m in (1.5, 2.0, 3.0):
        a = oracle.fcm(x, 4, m, 1e-5, 300, U0=u0, L=L)
        b = oracle.fcm_quantized(xq, 4, m, 1e-5, 300, U0=u0, want_U=True, L=L)
        _check(fails, a["iters"] == b["iters"], f"quantized iters m={m}: {a['iters']} {b['iters']}")
        k = min(a["iters"], b["iters"])
        _check(fails, np.allclose(a["Vtrace"][:k], b["Vtrace"][:k], rtol=1e-9, atol=1e-9),
               f"quantized V trace m={m}")
        _check(fails, np.allclose(a["J"][:k], b["J"][:k], rtol=1e-9), f"quantized J m={m}")
        _check(fails, np.allclose(a["delta"][:k], b["delta"][:k], rtol=1e-6, atol=1e-12),
               f"quantized delta m={m}")
        _check(fails, np.allclose(a["U"], b["U"], atol=1e-9), f"quantized U m={m}")
        # warm start from given centers
        V0 = np.array([10.0, 50.0, 120.0, 160.0])
        a = oracle.fcm(x, 4, m, 1e-5, 300, V0=V0, L=L)
        b = oracle.fcm_quantized(xq, 4, m, 1e-5, 300, V0=V0, L=L)
        _check(fails, a["iters"] == b["iters"] and np.allclose(a["V"], b["V"], rtol=1e-9),
               f"quantized init-V m={m}")
    return fails


def pin_dsc(L):
    """Dice similarity (Eq. 5) on a hand example with rational values, on
    identical and on disjoint segmentations, and through a label-to-class
    map: PR = [0, 0, 1, 1], GT = [0, 1, 1, 1] gives class 0: 2*1/(2+1) = 2/3,
    class 1: 2*2/(2+3) = 4/5; an absent class scores 1."""
    fails = []
    d, c = oracle.dsc([0, 0, 1, 1], [0, 1, 1, 1], [0, 1], 3, L=L)
    _check(fails, abs(d[0] - 2 / 3) < 1e-15 and abs(d[1] - 4 / 5) < 1e-15 and d[2] == 1.0,
           f"dsc hand example {d}")
    _check(fails, c.tolist() == [[2, 1, 1], [2, 3, 2], [0, 0, 0]], f"dsc counts {c.tolist()}")
    g = np.random.default_rng(3)
    t = g.integers(0, 4, 500)
    d, _ = oracle.dsc(t, t, [0, 1, 2, 3], 4, L=L)
    _check(fails, np.all(d == 1.0), f"dsc identical {d}")
    d, _ = oracle.dsc((t + 1) % 4, t, [0, 1, 2, 3], 4, L=L)
    _check(fails, np.all(d == 0.0), f"dsc disjoint {d}")
    # labels 0..3 named in reverse order: mapping them back restores DSC 1
    d, _ = oracle.dsc(3 - t, t, [3, 2, 1, 0], 4, L=L)
    _check(fails, np.all(d == 1.0), f"dsc through a map {d}")
    return fails


def pin_multi_feature(L):
    """Multi-feature FCM (Euclidean norm over D channels):
    * a 2-D hand example with rational memberships: V = [(0,0), (6,8)],
      pixels (3,4), (0,3), (6,0), m = 2 give u_1 = 1/2, 61/70, 16/25, and
      J = 25/2 + 549/70 + 2304/100 (closed form 1 / sum_k 1/d_k^2 per pixel);
    * one channel reproduces the scalar oracle; two identical channels give
      the scalar memberships and the scalar centers in both channels;
    * rotating the feature plane rotates V and leaves U unchanged;
      translating it translates V."""
    fails = []
    x = np.array([[3.0, 0.0, 6.0], [4.0, 3.0, 0.0]])
    V = np.array([[0.0, 0.0], [6.0, 8.0]])
    U = oracle.memberships_multi(x, V, 2.0, L=L)
    ref = np.array([[1 / 2, 61 / 70, 16 / 25], [1 / 2, 9 / 70, 9 / 25]])
    _check(fails, np.allclose(U, ref, rtol=0, atol=1e-15), f"multi toy U {U.tolist()}")
    J = oracle.objective_multi(x, U, V, 2.0, L=L)
    _check(fails, abs(J - (25 / 2 + 549 / 70 + 2304 / 100)) < 1e-12, f"multi toy J {J}")
    img, _ = phantom.phantom2d(11, 30, 30, 8.0)
    xs = img.reshape(-1).astype(np.float64)
    u0 = phantom.dirichlet_u0((11, 1), 3, xs.size).astype(np.float64)
    a = oracle.fcm(xs, 3, 2.0, 1e-9, 200, U0=u0, L=L)
    b = oracle.fcm_multi(xs[None, :], 3, 2.0, 1e-9, 200, U0=u0, L=L)
    _check(fails, a["iters"] == b["iters"] and np.max(np.abs(a["U"] - b["U"])) < 1e-12
           and np.max(np.abs(a["V"] - b["V"][:, 0])) < 1e-9, "multi D=1 vs scalar")
    c = oracle.fcm_multi(np.stack([xs, xs]), 3, 2.0, 1e-9, 200, U0=u0, L=L)
    _check(fails, c["iters"] == a["iters"] and np.max(np.abs(c["U"] - a["U"])) < 1e-12
           and np.max(np.abs(c["V"] - np.stack([a["V"], a["V"]], 1))) < 1e-9, "multi duplicated channel")
    g = np.random.default_rng(4)
    x2 = np.stack([xs, g.permutation(xs)])
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    d = oracle.fcm_multi(x2, 3, 2.0, 1e-9, 60, U0=u0, L=L)
    e = oracle.fcm_multi(R @ x2, 3, 2.0, 1e-9, 60, U0=u0, L=L)
    _check(fails, d["iters"] == e["iters"] and np.max(np.abs(d["U"] - e["U"])) < 1e-9
           and np.max(np.abs(d["V"] @ R.T - e["V"])) < 1e-7, "multi rotation")
    f = oracle.fcm_multi(x2 + np.array([[5.0], [-3.0]]), 3, 2.0, 1e-9, 60, U0=u0, L=L)
    _check(fails, np.max(np.abs(f["V"] - (d["V"] + np.array([5.0, -3.0])))) < 1e-7, "multi translation")
    return fails


def _naive_fcm(x, C, m, eps, max_iter, U0):
    """Algorithm 1 written as literal nested loops over tiny inputs, for
    pixels that sit on no center: Eq. 4 in the ratio-of-distances form with a
    real power (u_ij = 1 / sum_l (|x_i - v_j| / |x_i - v_l|)^(2/(m-1))), Eq. 3
    with u^m, Eq. 1 for J and the L-inf stopping test."""
    n = len(x)
    p = 2.0 / (m - 1.0)

    def centers(U):
        V = []
        for j in range(C):
            num = den = 0.0
            for i in range(n):
                w = U[j][i] ** m
                num += w * x[i]
                den += w
            V.append(num / den)
        return V

    Uprev = [[float(U0[j][i]) for i in range(n)] for j in range(C)]
    V = centers(Uprev)
    for k in range(1, max_iter + 1):
        U = [[0.0] * n for _ in range(C)]
        for i in range(n):
            for j in range(C):
                s = 0.0
                for l in range(C):
                    s += (abs(x[i] - V[j]) / abs(x[i] - V[l])) ** p
                U[j][i] = 1.0 / s
        delta = max(abs(U[j][i] - Uprev[j][i]) for j in range(C) for i in range(n))
        J = sum(U[j][i] ** m * (x[i] - V[j]) ** 2 for j in range(C) for i in range(n))
        if delta < eps or k == max_iter:  # V^k is the set that produced U^k
            return np.array(U), np.array(V), k, J
        V = centers(U)
        Uprev = U


def pin_brute_force(L):
    """The oracle agrees with the naive loop to 1e-12 on tiny random inputs
    (n <= 64, several C and m)."""
    fails = []
    g = np.random.default_rng(11)
    for n, C, m in [(7, 2, 2.0), (33, 3, 1.5), (64, 4, 2.7), (48, 3, 3.0), (64, 2, 2.0)]:
        x = g.uniform(0.0, 100.0, n)
        u0 = g.dirichlet(np.ones(C), n).T.copy()
        U, V, k, J = _naive_fcm(x, C, m, 1e-6, 40, u0)
        r = oracle.fcm(x, C, m, 1e-6, 40, U0=u0, L=L)
        _check(fails, r["iters"] == k, f"brute force n={n} C={C} m={m}: iters {r['iters']} vs {k}")
        if r["iters"] == k:
            _check(fails, np.max(np.abs(r["U"] - U)) < 1e-12, f"brute force n={n} C={C} m={m}: U")
            _check(fails, np.max(np.abs(r["V"] - V) / np.maximum(np.abs(V), 1.0)) < 1e-12,
                   f"brute force n={n} C={C} m={m}: V")
            _check(fails, abs(r["J"][-1] - J) <= 1e-12 * abs(J), f"brute force n={n} C={C} m={m}: J")
    return fails


def pin_converged_fixed_point(L):
    """A run stopped at a tight tolerance is a fixed point: one more center
    update (Eq. 3 from the returned U) moves no center by more than 1e-6."""
    fails = []
    img, _ = phantom.phantom2d(17, 40, 40, 8.0)
    x = img.reshape(-1).astype(np.float64)
    for C, m in [(4, 2.0), (3, 1.5)]:
        u0 = phantom.dirichlet_u0((17, C), C, x.size).astype(np.float64)
        r = oracle.fcm(x, C, m, 1e-10, 5000, U0=u0, L=L)
        _check(fails, r["status"] == 0, f"fixed point C={C} m={m}: not converged")
        W = r["U"] ** m
        Vn = (W @ x) / W.sum(1)
        _check(fails, np.max(np.abs(Vn - r["V"])) < 1e-6,
               f"fixed point C={C} m={m}: center moved {np.max(np.abs(Vn - r['V']))}")
    return fails


ALL_PINS = [pin_toy_rationals, pin_singular_points, pin_closed_form_objective,
            pin_optimality, pin_special_cases, pin_descent_and_invariants,
            pin_metamorphic, pin_quantized_matches_plain, pin_dsc, pin_multi_feature,
            pin_brute_force, pin_converged_fixed_point]
