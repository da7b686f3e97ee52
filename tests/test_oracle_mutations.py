"""The oracle's pins fail on plausible mistakes.

Each test plants one mistake in the FP64 oracle on the CPU (a monkeypatched solver function,
or a transformed projector matrix standing for a projector with that bug) and checks that the
pin written for that part rejects it: a dropped term, lambda in place of lambda^2, a wrong
trace, a reversed bisection, a mirrored detector, transposed image axes, a missing weight.
"""
import math

import numpy as np
import pytest

import synth
from oracle import proj as OP
from oracle import solver as S
from tests.test_oracle_explicit import GEOMS, explicit_A, explicit_B, oracle_matrix


def _hessenberg(k, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.triu(rng.standard_normal((k + 1, k)), -1) * np.logspace(0, -5, k)[None, :]


def _dense_pin(k=12, seed=7):
    """The Tikhonov / GCV / residual pin: the oracle against the stacked least-squares
    problem and the dense GCV definition."""
    H = _hessenberg(k, seed)
    beta = 2.5
    s, c, Vt = S.projected_svd(H, beta)
    e1 = np.zeros(k + 1)
    e1[0] = beta
    for lam in (1e-3, 0.05, 0.8):
        yd = np.linalg.lstsq(np.vstack([H, lam * np.eye(k)]), np.concatenate([e1, np.zeros(k)]),
                             rcond=None)[0]
        np.testing.assert_allclose(S.tikhonov_y(lam, s, c, Vt), yd, rtol=1e-8,
                                   atol=1e-10 * np.abs(yd).max())
        num = np.linalg.norm(H @ yd - e1) ** 2
        Hl = np.linalg.solve(H.T @ H + lam ** 2 * np.eye(k), H.T)
        tr = np.trace(np.eye(k + 1) - H @ Hl)
        np.testing.assert_allclose(S.residual_sq(lam, s, c), num, rtol=1e-8)
        np.testing.assert_allclose(S.gcv_value(lam, s, c), num / tr ** 2, rtol=1e-8)


def _dp_pin(k=12, seed=11):
    H = _hessenberg(k, seed)
    s, c, _ = S.projected_svd(H, 1.0)
    lo = math.sqrt(S.residual_sq(s[0] * 1e-8, s, c))
    hi = math.sqrt(S.residual_sq(s[0], s, c))
    target = 0.5 * (lo + hi)
    lam = S.dp_lambda(s, c, target)
    assert abs(math.sqrt(S.residual_sq(lam, s, c)) - target) <= 1e-10 * target


def test_pins_pass_on_the_oracle_as_it_is():
    _dense_pin()
    _dp_pin()


def test_dropped_residual_term_is_caught(monkeypatch):
    def residual_sq(lam, s, c):          # c_{k+1}^2 left out
        f = lam * lam / (s * s + lam * lam)
        return float(np.sum((f * c[:len(s)]) ** 2))
    monkeypatch.setattr(S, "residual_sq", residual_sq)
    with pytest.raises(AssertionError):
        _dense_pin()


def test_lambda_for_lambda_squared_is_caught(monkeypatch):
    def tikhonov_y(lam, s, c, Vt):       # s c / (s^2 + lambda)
        return Vt.T @ (s * c[:len(s)] / (s * s + lam))
    monkeypatch.setattr(S, "tikhonov_y", tikhonov_y)
    with pytest.raises(AssertionError):
        _dense_pin()


def test_wrong_gcv_trace_is_caught(monkeypatch):
    orig = S.residual_sq

    def gcv_value(lam, s, c):            # trace of I_k instead of I_{k+1}
        tr = len(s) - float(np.sum(s * s / (s * s + lam * lam)))
        return orig(lam, s, c) / (tr * tr)
    monkeypatch.setattr(S, "gcv_value", gcv_value)
    with pytest.raises(AssertionError):
        _dense_pin()


def test_reversed_dp_bisection_is_caught(monkeypatch):
    def dp_lambda(s, c, target):         # moves the wrong end of the bracket
        lo, hi = math.log(s[0] * 1e-8), math.log(s[0])
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if math.sqrt(S.residual_sq(math.exp(mid), s, c)) < target:
                hi = mid
            else:
                lo = mid
        return math.exp(0.5 * (lo + hi))
    monkeypatch.setattr(S, "dp_lambda", dp_lambda)
    with pytest.raises(AssertionError):
        _dp_pin()


# ----------------------------------------------------------------------------- projectors
def _mismatch(M, E):
    return np.max(np.abs(M - E)) > 1e-13 * np.max(np.abs(E))


SQUARE = {"fan_square_6": synth.fanflat2d(6, 5, 11, 20.0, 32.0,
                                         angles=np.array([0.2, 0.9, 1.7, 2.8, 4.0])),
          "parallel_square_7": synth.parallel2d(7, 4, 13, pitch=0.8,
                                                angles=np.array([0.1, 0.7, 1.3, 2.5]))}


@pytest.mark.parametrize("name", ["parallel_9x7", "fan_8x10", "fan_square_6", "parallel_square_7"])
def test_projector_pins_catch_planted_mistakes(name):
    """Matrices of A and B with a mirrored detector, transposed image axes or no ray weight
    are told apart from the explicit definitions (the oracle itself matches them)."""
    g = GEOMS.get(name) or SQUARE[name]
    nd, nv = g.n_det_u, g.n_views
    Ao = oracle_matrix(lambda e: OP.forward(g, e.reshape(g.image_shape)), g.n)
    Bo = oracle_matrix(lambda e: OP.back_pixel(g, e), g.m)
    A, B = explicit_A(g), explicit_B(g)
    assert not _mismatch(Ao, A) and not _mismatch(Bo, B)
    mirror = np.concatenate([np.arange(v * nd, (v + 1) * nd)[::-1] for v in range(nv)])
    assert _mismatch(Ao[mirror], A)                       # detector bins reversed
    assert _mismatch(Bo[:, mirror], B)
    perm = np.arange(g.n).reshape(g.ny, g.nx).T.reshape(-1) if g.nx == g.ny else None
    if perm is not None:
        assert _mismatch(Ao[:, perm], A)                  # x and y swapped
    assert _mismatch(Ao / _ray_weights(g)[:, None], A)   # the h / |d_drive| weight dropped
    assert _mismatch(Bo * (g.pitch_u / g.h ** 2), B)      # the backprojector's scale dropped


def _ray_weights(g):
    """h |D| / |D_drive| of every ray (its Joseph sample weight)."""
    w = []
    for th in g.angles:
        c, s = math.cos(th), math.sin(th)
        for j in range(g.n_det_u):
            u = (j - (g.n_det_u - 1) / 2.0) * g.pitch_u
            D = (np.array([-s, c]) if g.kind == synth.PARALLEL2D else
                 np.array([-g.sdd * c - u * s, -g.sdd * s + u * c]))
            w.append(g.h * np.linalg.norm(D) / np.max(np.abs(D)))
    return np.array(w)


# ----------------------------------------------------------------------------- initial guess,
# restarting and the NCP: the function's own source with one plausible mistake substituted
import inspect
import textwrap

from tests import test_oracle_ncp as NCP_PINS
from tests import test_oracle_solver as SOLVER_PINS


def _mutant(fn, old, new):
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, (fn.__name__, old)
    ns = {}
    exec(compile(src.replace(old, new), f"<mutant of {fn.__name__}>", "exec"), fn.__globals__, ns)
    return ns[fn.__name__]


X0_PINS = [lambda: SOLVER_PINS.test_initial_guess_iterate_matches_shifted_krylov_minimiser("ab"),
           lambda: SOLVER_PINS.test_initial_guess_iterate_matches_shifted_krylov_minimiser("ba"),
           SOLVER_PINS.test_matched_ab_from_initial_guess_is_lsqr_of_shifted_data,
           SOLVER_PINS.test_restart_at_full_dimension_follows_the_closed_form]


def _some_pin_fails(pins):
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    return failed


def test_x0_and_restart_pins_pass_on_the_oracle_as_it_is():
    assert _some_pin_fails(X0_PINS) == 0
    SOLVER_PINS.test_restarted_cycles_are_shifted_krylov_minimisers("ab")


@pytest.mark.parametrize("old,new", [
    ("return x0v + (B(z)", "return 0 * x0v + (B(z)"),     # x0 dropped from the iterate
])
def test_dropped_initial_guess_in_the_iterate_is_caught(monkeypatch, old, new):
    monkeypatch.setattr(S, "_form_x", _mutant(S._form_x, old, new))
    assert _some_pin_fails(X0_PINS) >= 3


@pytest.mark.parametrize("old,new", [
    ("r0 = b - A(x0v)\n", "r0 = b + A(x0v)\n"),            # sign of the AB shift
    ("r0 = b - A(x0v)\n", "r0 = b - 0 * A(x0v)\n"),        # AB residual ignores x0
    ("r0 = B(b - A(x0v))", "r0 = B(b)"),                   # BA residual ignores x0
])
def test_wrong_initial_residual_is_caught(monkeypatch, old, new):
    monkeypatch.setattr(S, "hybrid_gmres", _mutant(S.hybrid_gmres, old, new))
    assert _some_pin_fails(X0_PINS) >= 1


@pytest.mark.parametrize("old,new", [
    ("cycle, x0=x,", "cycle, x0=x0,"),                       # every cycle starts from x0
    ("x = res[\"x\"]", "x = res[\"x\"] - (x if x is not None else 0)"),  # keeps only the update
])
def test_wrong_restart_is_caught(monkeypatch, old, new):
    monkeypatch.setattr(S, "restarted_hybrid_gmres", _mutant(S.restarted_hybrid_gmres, old, new))
    with pytest.raises(AssertionError):
        SOLVER_PINS.test_restart_at_full_dimension_follows_the_closed_form()
    with pytest.raises(AssertionError):
        SOLVER_PINS.test_restarted_cycles_are_shifted_krylov_minimisers("ba")


NCP_CLOSED_FORMS = [lambda: NCP_PINS.test_ncp_of_a_sinusoid_is_a_step(17),
                    lambda: NCP_PINS.test_ncp_of_a_sinusoid_is_a_step(768),
                    NCP_PINS.test_ncp_ignores_mean_scale_and_circular_shift,
                    NCP_PINS.test_ncp_averages_rows_and_skips_rows_without_power]


def test_ncp_pins_pass_on_the_oracle_as_it_is():
    assert _some_pin_fails(NCP_CLOSED_FORMS) == 0


@pytest.mark.parametrize("fn,old,new", [
    ("periodogram", "[:, 1:q + 1]", "[:, 0:q]"),            # zero frequency kept
    ("periodogram", "[:, 1:q + 1]", "[:, 1:]"),             # mirrored half kept (q = n - 1)
    ("ncp", "c.mean(axis=0)", "c.sum(axis=0)"),             # rows summed, not averaged
    ("ncp", "/ tot[keep, None]", "/ tot.sum()"),            # one normalisation for all rows
])
def test_ncp_mistakes_are_caught(monkeypatch, fn, old, new):
    monkeypatch.setattr(S, fn, _mutant(getattr(S, fn), old, new))
    assert _some_pin_fails(NCP_CLOSED_FORMS) >= 1


@pytest.mark.parametrize("old,new", [
    ("dist > ncp_prev[1]", "dist < ncp_prev[1]"),           # stops while the distance falls
    ("k_done, y = ncp_prev[0], ncp_prev[2]", "pass"),       # returns the step that grew
])
def test_ncp_stop_mistakes_are_caught(monkeypatch, old, new):
    monkeypatch.setattr(S, "hybrid_gmres", _mutant(S.hybrid_gmres, old, new))
    with pytest.raises(AssertionError):
        NCP_PINS.test_ncp_stop_returns_the_last_checked_iterate_before_the_distance_grows("ab", 1)
