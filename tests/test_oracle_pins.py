"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: closed-form solutions,
conservation laws, the order conditions of its Runge-Kutta tableau, an independent
equilibrium solver, thermodynamic identities, and brute-force step-halving extrapolation.
"""
import numpy as np
import pytest
from scipy.optimize import root

import oracle
import synth
from synth import P_ATM, R_GAS


def _one_cell(mech, T, p, Y):
    T = np.atleast_1d(np.asarray(T, float))
    p = np.atleast_1d(np.asarray(p, float))
    Y = np.asarray(Y, float).reshape(mech["ns"], -1)
    rho, e = oracle.state_from_TpY(mech, T, p, Y)
    return T, p, Y, rho, e


# ---------------------------------------------------------------- tableau and thermo

def test_radau_tableau_order_conditions():
    """3-stage Radau IIA: B(5) quadrature and C(3) stage-order conditions, c3 = 1, b = last row."""
    A, c = oracle.radau_tableau()
    b = A[2]
    for k in range(1, 6):
        assert abs(np.sum(b * c ** (k - 1)) - 1.0 / k) < 1e-14
    for k in range(1, 4):
        assert np.max(np.abs(A @ c ** (k - 1) - c ** k / k)) < 1e-14
    assert c[2] == 1.0
    assert np.allclose(c, [(4 - 6 ** 0.5) / 10, (4 + 6 ** 0.5) / 10, 1.0], atol=1e-15)


def test_thermo_identities(h2mech):
    """cp = dh/dT and cp/T = ds/dT (finite differences), continuity at T_lo / T_hi."""
    T = np.array([250.0, 299.0, 301.0, 800.0, 1500.0, 3400.0, 3600.0, 5000.0])
    d = 1e-3
    cp, hRT, sR = oracle.thermo(h2mech, T)
    _, hRTp, sRp = oracle.thermo(h2mech, T + d)
    _, hRTm, sRm = oracle.thermo(h2mech, T - d)
    dh = ((T + d) * hRTp - (T - d) * hRTm) / (2 * d)
    ds = (sRp - sRm) / (2 * d)
    assert np.max(np.abs(dh - cp) / cp) < 1e-7
    assert np.max(np.abs(ds * T - cp) / cp) < 1e-7
    for Tb in (300.0, 3500.0):
        lo, hi = oracle.thermo(h2mech, np.array([Tb - 1e-9])), oracle.thermo(h2mech, np.array([Tb + 1e-9]))
        for a, b in zip(lo, hi):
            assert np.max(np.abs(a - b)) < 1e-8


def test_thermo_reference_values(h2mech):
    """h(300 K) and s(300 K) reproduce the drawn formation enthalpy / entropy of the generator
    (the reference species have h = 0 at 300 K)."""
    cp, hRT, sR = oracle.thermo(h2mech, np.array([300.0]))
    for k, name in enumerate(h2mech["names"]):
        if name in ("H2", "O2", "N2"):
            assert abs(hRT[k, 0]) < 1e-10
    assert np.all(sR[:, 0] * R_GAS > 100.0) and np.all(sR[:, 0] * R_GAS < 290.0)


def test_temperature_roundtrip(h2mech):
    rng = np.random.default_rng(3)
    n = 400
    Y = rng.dirichlet(np.full(h2mech["ns"], 0.5), size=n).T
    T = rng.uniform(120.0, 9000.0, size=n)
    rho, e = oracle.state_from_TpY(h2mech, T, np.full(n, P_ATM), Y)
    Tb = oracle.temperature_from_energy(h2mech, Y, e, np.full(n, 1000.0))
    assert np.max(np.abs(Tb - T) / T) < 1e-11


def test_state_from_TpY_ideal_gas(h2mech):
    """rho from the ideal-gas law; e is linear in Y at fixed T (mixture rule)."""
    Y = synth.premix_mass_fractions(h2mech)[:, None]
    T, p, Y, rho, e = _one_cell(h2mech, 300.0, P_ATM, Y)
    Wbar = 1.0 / np.sum(Y[:, 0] / h2mech["W"])
    assert abs(rho[0] - P_ATM * Wbar / (R_GAS * 300.0)) / rho[0] < 1e-14
    e_k = []
    for k in range(h2mech["ns"]):
        yk = np.zeros((h2mech["ns"], 1))
        yk[k] = 1.0
        e_k.append(oracle.state_from_TpY(h2mech, T, p, yk)[1][0])
    assert abs(np.dot(e_k, Y[:, 0]) - e[0]) < 1e-9 * max(1.0, abs(e[0]))


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("T0,b,Ea", [(900.0, 0.7, 4.0e4), (1800.0, -1.2, 1.2e5)])
def test_closed_form_first_order_reversible(T0, b, Ea):
    """A <=> B with identical thermo: K_c = 1, T constant,
    Y_A(t) = Y_eq + (Y_A0 - Y_eq) exp(-(k_f + k_r) t), Y_eq = (Y_A0 + Y_B0) / 2."""
    mech = synth.toy_mechanism("AB", A=3.0e7, b=b, Ea=Ea)
    T, p, Y, rho, e = _one_cell(mech, T0, 2 * P_ATM, [0.85, 0.15])
    kf = 3.0e7 * T0 ** b * np.exp(-Ea / (R_GAS * T0))
    dt = 2.0 / (2 * kf)
    T1, _, Y1, steps = oracle.advance(mech, rho, e, T, Y, dt)
    exact = 0.5 + (0.85 - 0.5) * np.exp(-2 * kf * dt)
    assert steps[0] > 0
    assert abs(Y1[0, 0] - exact) / exact < 1e-8
    assert abs(T1[0] - T0) < 1e-8 * T0


def test_closed_form_irreversible_first_order():
    mech = synth.toy_mechanism("A->B", A=2.0e6)
    T, p, Y, rho, e = _one_cell(mech, 1000.0, P_ATM, [1.0, 0.0])
    dt = 3.0e-6
    _, _, Y1, _ = oracle.advance(mech, rho, e, T, Y, dt)
    assert abs(Y1[0, 0] - np.exp(-2.0e6 * dt)) / np.exp(-2.0e6 * dt) < 1e-8


def test_closed_form_second_order():
    """2A -> B: dC_A/dt = -2 k C_A^2, so 1/C_A = 1/C_A0 + 2 k t."""
    k = 5.0e3
    mech = synth.toy_mechanism("2A->B", A=k)
    T, p, Y, rho, e = _one_cell(mech, 1200.0, 10 * P_ATM, [0.95, 0.05])
    CA0 = rho[0] * 0.95 / 0.02
    dt = 4.0 / (2 * k * CA0)
    T1, _, Y1, _ = oracle.advance(mech, rho, e, T, Y, dt)
    CA = 1.0 / (1.0 / CA0 + 2 * k * dt)
    assert abs(rho[0] * Y1[0, 0] / 0.02 - CA) / CA < 1e-8
    assert abs(T1[0] - 1200.0) < 1e-8 * 1200.0


@pytest.mark.parametrize("eff_inert", [1.0, 3.5])
def test_closed_form_third_body(eff_inert):
    """A + M -> B + M with [M] = C_A + C_B + eff_I C_I constant: first order with k [M]."""
    k = 1.0e3
    mech = synth.toy_mechanism("A+M->B", A=k, eff_inert=eff_inert)
    Y0 = np.array([0.3, 0.1, 0.6])
    T, p, Y, rho, e = _one_cell(mech, 1500.0, 5 * P_ATM, Y0)
    M = rho[0] * (Y0[0] + Y0[1] + eff_inert * Y0[2]) / 0.02
    dt = 1.5 / (k * M)
    _, _, Y1, _ = oracle.advance(mech, rho, e, T, Y, dt)
    exact = 0.3 * np.exp(-k * M * dt)
    assert abs(Y1[0, 0] - exact) / exact < 1e-8


# ---------------------------------------------------------------- invariants

def test_invariants_on_reacting_cells(h2mech):
    """sum Y, element moles and e(T, Y) are conserved; Y stays non-negative."""
    T, p, Y, hot = synth.sheet_field(h2mech, n=12, seed=1)
    idx = np.nonzero(hot)[0][:24]
    T, p, Y = T[idx], p[idx], Y[:, idx]
    rho, e = oracle.state_from_TpY(h2mech, T, p, Y)
    T1, p1, Y1, steps = oracle.advance(h2mech, rho, e, T, Y, 1e-8)
    assert np.all(steps > 0)
    assert np.max(np.abs(Y1.sum(0) - Y.sum(0))) < 1e-12
    el0 = h2mech["elem"].T @ (Y / h2mech["W"][:, None])
    el1 = h2mech["elem"].T @ (Y1 / h2mech["W"][:, None])
    assert np.max(np.abs(el1 - el0) / (np.abs(el0) + 1e-300)) < 1e-11
    rho1, e1 = oracle.state_from_TpY(h2mech, T1, p1, Y1)
    assert np.max(np.abs(e1 - e) / np.abs(e)) < 1e-11
    assert np.max(np.abs(rho1 - rho) / rho) < 1e-11
    assert Y1.min() > -1e-14


def test_cold_cells_skipped_below_T_min(h2mech):
    T, p, Y, hot = synth.slab_field(h2mech, n=4)
    rho, e = oracle.state_from_TpY(h2mech, T, p, Y)
    T1, p1, Y1, steps = oracle.advance(h2mech, rho, e, T, Y, 1e-7, T_min=600.0)
    cold = T < 600.0
    assert np.all(steps[cold] == 0) and np.all(steps[~cold] > 0)
    assert np.array_equal(Y1[:, cold], Y[:, cold]) and np.array_equal(T1[cold], T[cold])


# ---------------------------------------------------------------- thermodynamic consistency

def test_affinity_relation(h2mech):
    """For every reversible reaction, q_f / q_r = exp(-sum_k dnu_k mu_k / RT) with the
    chemical potential mu_k / RT = g_k / RT + ln(C_k R T / p0) of an ideal gas."""
    rng = np.random.default_rng(11)
    n = 64
    Y = rng.dirichlet(np.full(h2mech["ns"], 1.0), size=n).T
    T = rng.uniform(700.0, 3000.0, size=n)
    rho = rng.uniform(0.2, 5.0, size=n)
    _, qf, qr = oracle.rates(h2mech, rho, T, Y, with_progress=True)
    _, hRT, sR = oracle.thermo(h2mech, T)
    C = rho[None, :] * Y / h2mech["W"][:, None]
    mu = hRT - sR + np.log(C * R_GAS * T[None, :] / P_ATM)
    dnu = (h2mech["nu_r"].astype(float) - h2mech["nu_f"])
    lhs = np.log(qf) - np.log(qr)
    rhs_ = -(dnu @ mu)
    assert np.max(np.abs(lhs - rhs_)) < 1e-9


def _equilibrium(mech, rho, e, T_guess, Y_guess):
    """Element-constrained equilibrium at fixed (rho, e): C_k = (p0/RT) exp(-g_k/RT + a_k . pi),
    solved for the element potentials pi and T from element and energy balances."""
    a = mech["elem"].astype(float)
    W = mech["W"]
    b = a.T @ (Y_guess / W)

    def comp(x):
        pi, T = x[:-1], x[-1]
        _, hRT, sR = oracle.thermo(mech, np.array([T]))
        C = P_ATM / (R_GAS * T) * np.exp(-(hRT[:, 0] - sR[:, 0]) + a @ pi)
        return C, T, hRT[:, 0]

    def F(x):
        C, T, hRT = comp(x)
        n = C / rho
        u = (hRT - 1.0) * R_GAS * T
        return np.concatenate([(a.T @ n - b) / b, [(n @ u - e) / abs(e)]])

    C0 = rho * Y_guess / W
    for Tg in (T_guess, 1.25 * T_guess, 0.8 * T_guess, 1.5 * T_guess):
        pi0 = np.linalg.lstsq(a, np.log(np.maximum(C0, 1e-300) * R_GAS * Tg / P_ATM), rcond=None)[0]
        with np.errstate(all="ignore"):
            sol = root(F, np.concatenate([pi0, [Tg]]), method="hybr", tol=1e-13)
            res = np.max(np.abs(F(sol.x)))
        if res < 1e-12:
            C, T, _ = comp(sol.x)
            return T, C * W / rho
    raise AssertionError("equilibrium solver did not converge")


def test_long_time_equilibrium_and_detailed_balance(h2mech):
    """Long integrations reach the state an independent entropy-maximising solver predicts,
    and every reaction is in detailed balance there (q_f = q_r)."""
    Tin = np.array([2400.0, 1700.0])
    pin = np.array([20.0, 3.0]) * P_ATM
    Y = np.stack([synth.premix_mass_fractions(h2mech),
                  np.random.default_rng(5).dirichlet(np.full(h2mech["ns"], 1.0))], axis=1)
    rho, e = oracle.state_from_TpY(h2mech, Tin, pin, Y)
    T1, _, Y1, steps = oracle.advance(h2mech, rho, e, Tin, Y, 1e6)
    assert np.all(steps > 0)
    for i in range(2):
        Teq, Yeq = _equilibrium(h2mech, rho[i], e[i], T1[i], Y1[:, i])
        assert abs(Teq - T1[i]) / Teq < 1e-7
        big = Yeq > 1e-10
        assert np.max(np.abs(Y1[big, i] - Yeq[big]) / Yeq[big]) < 1e-5
        _, qf, qr = oracle.rates(h2mech, rho[[i]], T1[[i]], Y1[:, [i]], with_progress=True)
        sig = qf[:, 0] > 1e-30 * np.max(qf)
        assert np.max(np.abs(qf[sig, 0] - qr[sig, 0]) / qf[sig, 0]) < 1e-4


def test_same_elements_same_energy_same_equilibrium(h2mech):
    """Two different hot initial states with equal element moles and equal (rho, e) reach the
    same final state (path independence of the equilibrium)."""
    from scipy.optimize import brentq
    W = h2mech["W"]
    Ya = np.random.default_rng(8).dirichlet(np.full(h2mech["ns"], 2.0))
    # move along three reaction directions: element moles are unchanged
    dnu = (h2mech["nu_r"].astype(float) - h2mech["nu_f"])
    Yb = Ya + 0.004 * (dnu[3] + dnu[7] - dnu[11]) * W
    assert Yb.min() > 0
    rho_a, e_a = oracle.state_from_TpY(h2mech, np.array([2600.0]), np.array([5 * P_ATM]), Ya[:, None])

    def de(T):
        return oracle.state_from_TpY(h2mech, np.array([T]), np.array([1.0]), Yb[:, None])[1][0] - e_a[0]

    Tb = brentq(de, 50.0, 19000.0, xtol=1e-12)
    assert 1500.0 < Tb < 4000.0
    rho = np.array([rho_a[0], rho_a[0]])
    e = np.array([e_a[0], e_a[0]])
    T1, _, Y1, steps = oracle.advance(h2mech, rho, e, np.array([2600.0, Tb]),
                                      np.stack([Ya, Yb], axis=1), 1e6)
    assert np.all(steps > 0)
    assert abs(T1[0] - T1[1]) / T1[0] < 1e-7
    big = Y1[:, 0] > 1e-10
    assert np.max(np.abs(Y1[big, 0] - Y1[big, 1]) / Y1[big, 0]) < 1e-5


# ---------------------------------------------------------------- brute force

def test_step_halving_extrapolation(h2mech):
    """Uniform backward Euler with N, 2N, ..., extrapolated (Richardson, error in powers of h)
    agrees with the adaptive Radau oracle."""
    Y0 = np.random.default_rng(2).dirichlet(np.full(h2mech["ns"], 2.0))
    T, p, Y, rho, e = _one_cell(h2mech, 1300.0, P_ATM, Y0)
    # let the fast modes relax first, so the backward-Euler error expansion holds
    T, _, Y, _ = oracle.advance(h2mech, rho, e, T, Y, 1e-6)
    dt = 2e-7
    Tref, _, Yref, _ = oracle.advance(h2mech, rho, e, T, Y, dt, rtol=1e-12, atol=1e-18)
    levels = [256, 512, 1024, 2048, 4096]
    sols = [oracle.backward_euler(h2mech, rho[0], e[0], T[0], Y[:, 0], dt, n)[1] for n in levels]
    # Neville/Richardson tableau for an error expansion in h, h^2, h^3, ...
    tab = [np.array(s) for s in sols]
    for j in range(1, len(levels)):
        tab = [tab[i + 1] + (tab[i + 1] - tab[i]) / (2 ** j - 1) for i in range(len(tab) - 1)]
    ext = tab[0]
    big = Yref[:, 0] > 1e-8
    err = np.abs(ext[big] - Yref[big, 0]) / Yref[big, 0]
    raw = np.abs(sols[-1][big] - Yref[big, 0]) / Yref[big, 0]
    assert np.max(err) < 1e-8
    assert np.max(raw) > 10 * np.max(err)   # the extrapolation did the work


def test_temperature_ode_cross_check(h2mech):
    """The corrected form of Eq. 6, dT/dt = -sum_k u_k W_k omega_k / (rho c_v), integrated
    with (Y, T) as state, gives the T that the T(e) closure of the oracle gives."""
    Y0 = np.random.default_rng(4).dirichlet(np.full(h2mech["ns"], 2.0))
    T, p, Y, rho, e = _one_cell(h2mech, 1300.0, P_ATM, Y0)
    T, _, Y, _ = oracle.advance(h2mech, rho, e, T, Y, 1e-6)
    dt = 2e-7
    T1, _, Y1, _ = oracle.advance(h2mech, rho, e, T, Y, dt, rtol=1e-12, atol=1e-18)
    T2, Y2 = oracle.temperature_ode(h2mech, rho[0], T[0], Y[:, 0], dt, 200000)
    assert abs(T2 - T1[0]) / T1[0] < 1e-8
    assert abs(T1[0] - T[0]) > 1e-3   # the temperature actually moved
