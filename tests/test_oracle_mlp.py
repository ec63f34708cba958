"""Pins of the FP64 surrogate oracle (oracle/mlp.py) against what the mathematics fixes (no GPU).

* the reverse-mode gradient against central finite differences of the loss (small and full-width
  networks), so that a dropped term, a transposed product or a wrong activation derivative fails;
* GELU against x Phi(x) with the normal CDF of scipy (a different routine from erf);
* bfloat16 rounding against exact ties and against torch's own conversion;
* encode/decode as inverse maps, with the documented linear and logarithmic regimes and the
  physical clamps;
* the conservative correction: feasible, a minimiser of the weighted norm, the identity on
  feasible changes, and element-conserving for the mechanism's element matrix;
* the state error vanishes for an exact prediction;
* the optimiser (AdamW with a cosine-annealed learning rate) against closed forms: a constant
  gradient gives steps of exactly lr sign(g) (the bias corrections cancel the moments' zero
  start), a zero gradient shrinks the weights by prod (1 - lr_s wd) (the decay is decoupled from
  the adaptive step), a rescaled gradient gives the same steps, and the schedule starts at lr,
  passes lr / 2 half-way, is antisymmetric about it and sums to lr (S + 1) / 2 over S steps;
* everything also at the 53-species shape (56 inputs, 55 outputs).
"""
import numpy as np
import pytest
from scipy.special import ndtr

from oracle import mlp
import synth


def _small_layers(rng, widths):
    return [(rng.normal(0, 1 / np.sqrt(widths[l]), (widths[l + 1], widths[l])), rng.normal(0, 0.1, widths[l + 1]))
            for l in range(len(widths) - 1)]


def _fd_check(layers, x, t, e_star, w, picks, h=1e-6):
    loss, grads = mlp.loss_and_grad(layers, x, t, e_star, w)
    flat = mlp.flatten(layers)
    g = mlp.flatten(grads)
    widths = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
    for i in picks:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = mlp.loss_and_grad(mlp.unflatten(fp, widths), x, t, e_star, w)
        lm, _ = mlp.loss_and_grad(mlp.unflatten(fm, widths), x, t, e_star, w)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    return loss


def test_gradient_matches_finite_differences_small_net():
    rng = np.random.default_rng(0)
    widths = (12, 8, 7, 11)
    layers = _small_layers(rng, widths)
    x = rng.normal(size=(16, 12))
    t = rng.normal(size=(16, 10))
    e_star = rng.normal(size=16)
    _fd_check(layers, x, t, e_star, 0.3, range(sum(widths[l + 1] * (widths[l] + 1) for l in range(3))))


@pytest.mark.parametrize("ns", [9, 53])
def test_gradient_matches_finite_differences_full_width(ns):
    rng = np.random.default_rng(1)
    w = mlp.widths(ns)
    layers = _small_layers(rng, w)
    x = rng.normal(size=(8, ns + 3))
    t = rng.normal(size=(8, ns + 1))
    e_star = rng.normal(size=8)
    n = mlp.n_params(ns)
    picks = list(rng.choice(n, 40, replace=False)) + [0, n - 1, n - ns - 3]   # first W1, last bias, error-head row
    _fd_check(layers, x, t, e_star, 0.5, picks)


def test_parameter_counts():
    assert mlp.n_params(9) == 52619 and mlp.n_params(53) == 63927
    assert mlp.ns_of_params(52619) == 9 and mlp.ns_of_params(63927) == 53


def test_gelu_is_x_times_normal_cdf():
    z = np.linspace(-8, 8, 1001)
    assert np.allclose(mlp.gelu(z), z * ndtr(z), rtol=1e-13, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_bf16_rounding_ties_and_torch():
    one = 1.0
    assert mlp.bf16(one + 2 ** -7) == one + 2 ** -7          # representable (7 stored mantissa bits)
    assert mlp.bf16(one + 2 ** -8) == one                    # tie -> even (mantissa 0)
    assert mlp.bf16(one + 3 * 2 ** -8) == one + 2 ** -6      # tie -> even (mantissa 2)
    assert mlp.bf16(-(one + 2 ** -8 + 2 ** -12)) == -(one + 2 ** -7)
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(2).normal(size=10000).astype(np.float32) * 10.0 ** np.random.default_rng(3).integers(-8, 8, 10000)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_encode_decode_inverse_and_regimes():
    rng = np.random.default_rng(4)
    Y0 = 10.0 ** rng.uniform(-9, 0, 5000)
    ratio = np.concatenate([1 + 10.0 ** rng.uniform(-14, 0, 2500), 1 - 10.0 ** rng.uniform(-14, -0.01, 2500)])
    Y1 = (Y0 + mlp.EPS_Y) * ratio - mlp.EPS_Y
    keep = (Y1 >= 0) & (Y1 <= 1)   # physical states only (decoding clamps to [0, 1])
    Y0, Y1, ratio = Y0[keep], Y1[keep], ratio[keep]
    T0 = rng.uniform(300, 3000, Y0.size)
    T1 = T0 * ratio
    A = mlp.targets(T0, Y0[:, None], Y1[:, None], T1)
    assert np.allclose(mlp.decode_species(A[:, 0:1], Y0[:, None])[:, 0], Y1, rtol=1e-9, atol=1e-20)
    inT = ratio >= 0.1   # T1 within [T0 / 10, 10 T0]
    assert np.allclose(mlp.decode_temperature(A[inT, 1], T0[inT]), T1[inT], rtol=1e-12)
    # linear for |u| << u0: a = u / u0; logarithmic for |u| >> u0: a = sign(u) ln(2 |u| / u0)
    u = np.log(ratio)
    small = np.abs(u) < 1e-12
    assert np.allclose(A[small, 1], u[small] / mlp.U0, rtol=1e-3, atol=1e-6)   # u rounded at 1e-16
    big = u > 1e-3
    assert np.allclose(A[big, 1], np.log(2 * u[big] / mlp.U0), rtol=1e-6)
    assert np.all(np.diff(mlp.encode(np.linspace(-0.5, 5, 1000))) > 0)
    # the physical clamps: any output decodes to 0 <= Y1 <= 1 and T0/10 <= T1 <= 10 T0
    Yr = rng.uniform(0, 1, 2000)
    aa = rng.uniform(-80, 80, 2000)
    Yd = mlp.decode_species(aa, Yr)
    assert np.all(Yd >= -1e-15) and np.all(Yd <= 1 + 1e-12)
    Td = mlp.decode_temperature(aa, np.full(2000, 1000.0))
    assert np.all(Td >= 100.0 - 1e-9) and np.all(Td <= 10000.0 + 1e-9)


def test_conservative_correction(h2mech):
    C = mlp.conserved_basis(h2mech["elem"], h2mech["W"])
    assert C.shape[0] == np.linalg.matrix_rank(h2mech["elem"].astype(float))
    assert np.allclose(C @ C.T, np.eye(C.shape[0]), atol=1e-12)
    # every reaction vector W .* dnu is orthogonal to the conserved directions
    dnu = (h2mech["nu_r"] - h2mech["nu_f"]).astype(float)
    assert np.allclose(C @ (h2mech["W"][:, None] * dnu.T), 0.0, atol=1e-12)
    rng = np.random.default_rng(5)
    Y0 = rng.dirichlet(np.full(9, 0.5), size=50)
    dY = rng.normal(scale=1e-3, size=(50, 9)) * (Y0 + 1e-6)
    out = mlp.conserve(C, Y0, dY)
    assert np.allclose(out @ C.T, 0.0, atol=1e-15)
    # element mass conserved: sum_k elem_kj dY_k / W_k = 0
    assert np.allclose(out @ (h2mech["elem"] / h2mech["W"][:, None]), 0.0, atol=1e-15)
    assert np.allclose(out.sum(1), 0.0, atol=1e-15)
    # optimality: any other feasible change is farther from dY in the weighted norm
    P = np.eye(9) - C.T @ C
    for i in range(50):
        w2 = np.maximum(np.abs(Y0[i] + out[i]), mlp.EPS_Y) ** 2
        best = np.sum((out[i] - dY[i]) ** 2 / w2)
        for _ in range(20):
            v = P @ rng.normal(scale=1e-4, size=9)
            alt = out[i] + v * (Y0[i] + 1e-6)
            alt = alt - C.T @ (C @ alt)
            assert np.sum((alt - dY[i]) ** 2 / w2) >= best * (1 - 1e-9)
    # identity on changes that are already feasible
    feas = out.copy()
    assert np.allclose(mlp.conserve(C, Y0, feas), feas, rtol=1e-12, atol=1e-20)


def test_conserved_directions_of_both_mechanisms(h2mech, hcmech):
    """The complement of the reaction span: orthonormal, orthogonal to every reaction vector, of
    dimension ns - rank, and containing the element-mass directions.  The 53-species mechanism has
    one direction more than it has elements: its N2 takes part in no reaction while other
    N-bearing species do."""
    for mech, n_extra in ((h2mech, 0), (hcmech, 1)):
        C = mlp.conserved_directions(mech["W"], mech["nu_f"], mech["nu_r"])
        R = mech["W"][:, None] * (mech["nu_r"] - mech["nu_f"]).astype(float).T
        assert np.allclose(C @ C.T, np.eye(C.shape[0]), atol=1e-12)
        assert np.allclose(C @ R, 0.0, atol=1e-12)
        assert C.shape[0] == mech["ns"] - np.linalg.matrix_rank(R)
        E = mlp.conserved_basis(mech["elem"], mech["W"])
        assert np.allclose(E @ C.T @ C, E, atol=1e-12)
        assert C.shape[0] == E.shape[0] + n_extra <= mlp.MAX_CONS


def test_state_error_vanishes_for_exact_prediction(h2mech):
    rng = np.random.default_rng(6)
    n = 200
    T0 = rng.uniform(300, 3000, n)
    Y0 = rng.dirichlet(np.full(9, 0.5), size=n)
    C = mlp.conserved_basis(h2mech["elem"], h2mech["W"])
    Y1 = Y0 + mlp.conserve(C, Y0, rng.normal(scale=1e-2, size=(n, 9)) * Y0)
    T1 = T0 + rng.normal(scale=10, size=n)
    A = mlp.targets(T0, Y0, Y1, T1)
    norm = mlp.norm_from_data(A, A)
    norm.update(C=np.vstack([C, np.zeros((mlp.MAX_CONS - C.shape[0], 9))]), ncons=C.shape[0])
    assert norm["sd_y"][8] == 1.0   # N2 is inert: its encoding never changes
    o = (A - norm["mu_y"]) / norm["sd_y"]
    E = mlp.state_error(norm, o, Y0, T0, Y1, T1)
    assert np.all(E < 1e-10)
    # a perturbed prediction has an error of the size of the perturbation
    o2 = o.copy()
    o2[:, 0] += 1e-3 / norm["sd_y"][0]
    assert np.all(mlp.state_error(norm, o2, Y0, T0, Y1, T1) > 1e-12)


@pytest.mark.parametrize("ns", [9, 53])
def test_checkpoint_round_trip(ns):
    rng = np.random.default_rng(7)
    ni, nt = ns + 3, ns + 1
    norm = dict(mu_x=rng.normal(size=ni), sd_x=rng.uniform(1, 2, ni), mu_y=rng.normal(size=nt),
                sd_y=rng.uniform(1, 2, nt), lo_x=rng.normal(size=ni), hi_x=rng.normal(size=ni),
                C=rng.normal(size=(mlp.MAX_CONS, ns)), ncons=3)
    params = rng.normal(size=mlp.n_params(ns)).astype(np.float32)
    blob = mlp.pack_checkpoint(norm, params)
    n2, p2 = mlp.unpack_checkpoint(blob)
    assert n2["ncons"] == 3 and np.array_equal(p2, params.astype(np.float64))
    for k in ("mu_x", "sd_y", "lo_x", "hi_x"):
        assert np.array_equal(n2[k], np.asarray(norm[k], np.float32).astype(np.float64))
    assert np.array_equal(n2["C"], np.asarray(norm["C"], np.float32).astype(np.float64))
    assert len(blob) == 16 + 4 * (ni * 4 + nt * 2 + mlp.MAX_CONS * ns + 4) + 4 * mlp.n_params(ns)


def test_adamw_constant_gradient_steps_are_lr_sign_g():
    """With the same gradient every step, the bias-corrected moments equal g and g^2 exactly, so
    (without decay) every step is lr g / (|g| + eps): the running averages' zero start is undone."""
    rng = np.random.default_rng(8)
    w0 = rng.normal(size=1000)
    g = rng.normal(size=1000) * 10.0 ** rng.uniform(-3, 3, 1000)
    w, m, v = w0.copy(), np.zeros(1000), np.zeros(1000)
    lr = 1e-3
    for t in range(1, 26):
        w, m, v = mlp.adamw_step(w, g, m, v, t, lr, 0.0)
    expect = w0 - 25 * lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(w, expect, rtol=0, atol=1e-12)


def test_adamw_zero_gradient_decays_independently_of_the_moments():
    """Decoupled weight decay: with g = 0 the adaptive term vanishes and the weights shrink by
    (1 - lr_s wd) per step, whatever the second-moment estimate (the coupled L2 form would divide
    the decay by sqrt(v))."""
    rng = np.random.default_rng(9)
    w0 = rng.normal(size=100)
    lr, wd, S = 2e-3, 0.1, 40
    w, m, v = w0.copy(), np.zeros(100), np.full(100, 1e-6)
    shrink = 1.0
    for s in range(S):
        lr_s = mlp.cosine_lr(lr, s, S)
        w, m, v = mlp.adamw_step(w, np.zeros(100), m, v, s + 1, lr_s, wd)
        shrink *= 1.0 - lr_s * wd
    assert np.allclose(w, w0 * shrink, rtol=1e-14, atol=0)


def test_adamw_is_invariant_to_gradient_scale():
    rng = np.random.default_rng(10)
    w0 = rng.normal(size=500)
    gs = [rng.normal(size=500) * 10.0 ** rng.uniform(-2, 2, 500) for _ in range(12)]
    out = []
    for c in (1.0, 1e3):
        w, m, v = w0.copy(), np.zeros(500), np.zeros(500)
        for t, g in enumerate(gs, start=1):
            w, m, v = mlp.adamw_step(w, c * g, m, v, t, 1e-3, 1e-4, eps=1e-30)
        out.append(w)
    assert np.allclose(out[0], out[1], rtol=0, atol=1e-12)


def test_cosine_schedule_closed_forms():
    lr, S = 1e-3, 1000
    lrs = np.array([mlp.cosine_lr(lr, s, S) for s in range(S)])
    assert lrs[0] == lr and abs(lrs[S // 2] - lr / 2) < 1e-18
    assert np.all(np.diff(lrs) < 0) and lrs[-1] > 0
    # antisymmetric about lr / 2: lr_s + lr_{S - s} = lr
    assert np.allclose(lrs[1:] + lrs[1:][::-1], lr, rtol=0, atol=1e-18)
    # sum_{s < S} cos(pi s / S) = 1, so the schedule sums to lr (S + 1) / 2
    assert abs(lrs.sum() - lr * (S + 1) / 2) < 1e-15


def test_adamw_minimises_a_quadratic():
    """AdamW with the cosine schedule drives a separable quadratic to its minimiser (w* = 0 with
    zero decay; with decay the minimiser of the decayed objective lies between)."""
    rng = np.random.default_rng(11)
    target = rng.normal(size=50)
    w, m, v = np.zeros(50), np.zeros(50), np.zeros(50)
    S = 4000
    for s in range(S):
        g = w - target
        w, m, v = mlp.adamw_step(w, g, m, v, s + 1, mlp.cosine_lr(0.05, s, S), 0.0)
    assert np.max(np.abs(w - target)) < 1e-3
