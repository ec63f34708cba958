"""Pins of the oracle's explicit scheme (the paper's own method, Sec. 2.1) against closed forms
and against the exact solution (no GPU).

* A -> B with constant k and Y_B >= Y_A: every substep is limited by A to h = frac / k, so after
  N full substeps Y_A = Y_A0 (1 - frac)^N and the last, partial substep of length r multiplies it
  by (1 - k r) -- a wrong sign, a max instead of a min over species or a missing end clamp fails;
* the floor: with Y_A below y_floor each substep removes exactly frac * y_floor of A;
* forward Euler keeps every linear invariant (sum Y, element masses) to round-off, so a dropped
  W_k or a wrong stoichiometric sign in the update fails;
* the error against the FP64 Radau reference falls as the change limit is tightened, at first
  order once the substeps are small.
"""
import numpy as np

import oracle
import synth
from synth import P_ATM


def _cell(mech, T, p, Y):
    T = np.atleast_1d(np.asarray(T, float))
    p = np.atleast_1d(np.asarray(p, float))
    Y = np.asarray(Y, float).reshape(mech["ns"], -1)
    rho, e = oracle.state_from_TpY(mech, T, p, Y)
    return T, Y, rho, e


def test_first_order_decay_closed_form():
    k = 2.0e6
    mech = synth.toy_mechanism("A->B", A=k)
    T, Y, rho, e = _cell(mech, 1000.0, P_ATM, [0.1, 0.9])
    for frac, nfull, part in ((0.05, 10, 0.5), (0.01, 37, 0.25), (0.03, 0, 0.7)):
        dt = (nfull + part) * frac / k
        T1, _, Y1, steps = oracle.explicit(mech, rho, e, T, Y, dt, frac=frac)
        exact = 0.1 * (1 - frac) ** nfull * (1 - part * frac)
        assert steps[0] == nfull + 1
        assert abs(Y1[0, 0] - exact) <= 1e-12 * exact
        assert abs(Y1[0, 0] + Y1[1, 0] - 1.0) <= 1e-15
        assert abs(T1[0] - 1000.0) <= 1e-9 * 1000.0     # identical thermo: T is constant


def test_floor_closed_form():
    """Y_A0 = 1e-12 < y_floor = 1e-11: h = frac y_floor / (k Y_A), so each substep removes
    frac y_floor = 5e-13; after two substeps (t = 0.5/k + 1/k) A is gone and the last substep
    runs to dt with zero rates."""
    k = 1.0e5
    mech = synth.toy_mechanism("A->B", A=k)
    T, Y, rho, e = _cell(mech, 1200.0, P_ATM, [1e-12, 1.0 - 1e-12])
    T1, _, Y1, steps = oracle.explicit(mech, rho, e, T, Y, 2.0 / k, frac=0.05, y_floor=1e-11)
    assert steps[0] == 3
    assert abs(Y1[0, 0]) <= 1e-24


def test_linear_invariants_and_cold_cells(h2mech):
    T, p, Y, hot = synth.sheet_field(h2mech, n=6, seed=3, frac=0.2)
    rho, e = oracle.state_from_TpY(h2mech, T, p, Y)
    T1, _, Y1, steps = oracle.explicit(h2mech, rho, e, T, Y, 1e-8, frac=0.05, T_min=1000.0)
    assert np.all(steps[T < 1000.0] == 0) and np.all(steps[hot] > 0)
    assert np.array_equal(Y1[:, T < 1000.0], Y[:, T < 1000.0])
    assert np.allclose(Y1.sum(0), Y.sum(0), atol=1e-13)
    elem = h2mech["elem"] / h2mech["W"][:, None]          # mol of element per kg of species
    assert np.allclose(Y1.T @ elem, Y.T @ elem, rtol=1e-12, atol=1e-12)
    # e is held: T(e, Y1) reproduces the returned T
    T_e = oracle.temperature_from_energy(h2mech, Y1, e, T1)
    assert np.allclose(T_e, T1, rtol=1e-12)


def test_error_falls_with_the_change_limit(h2mech):
    T, p, Y, hot = synth.sheet_field(h2mech, n=24, seed=1, frac=0.05)
    idx = np.nonzero(hot)[0][:24]
    T, p, Y = T[idx], p[idx], Y[:, idx]
    rho, e = oracle.state_from_TpY(h2mech, T, p, Y)
    T_ref, _, Y_ref, _ = oracle.advance(h2mech, rho, e, T, Y, 1e-8)
    big = Y_ref >= 1e-6
    med = []
    for frac in (0.05, 0.01, 0.002, 0.0004):
        T1, _, Y1, steps = oracle.explicit(h2mech, rho, e, T, Y, 1e-8, frac=frac)
        assert np.all(steps > 0)
        err = np.where(big, np.abs(Y1 - Y_ref) / np.maximum(Y_ref, 1e-300), 0.0).max(0)
        med.append(np.median(err))
    assert all(a > 1.5 * b for a, b in zip(med, med[1:]))
    # first order once the substeps are small: a 5x tighter limit gives about 5x less error
    assert 3.5 < med[2] / med[3] < 7.0
    assert med[3] < 1e-4
