"""FP64 CPU oracle of the chemistry surrogate (test infrastructure).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import
this module.  It shares no code with the CUDA library.

The paper defines no learned surrogate (its outlook, Sec. 6, mentions machine learning only for
performance prediction); what is computed here is the surrogate as the library's C interface
documents it, written out plainly in numpy FP64:

* features x = (T, ln p, ln dt, ln(max(Y_k, 0) + 1e-6)), standardised with the stored mean and
  standard deviation;
* a multilayer perceptron: z_l = a_{l-1} W_l^T + b_l, a_l = gelu(z_l) = z_l Phi(z_l) (exact erf
  form) for the hidden layers, outputs o = z_L (no activation);
* target encodings of the state after dt: u_k = ln((Y1_k + 1e-6) / (max(Y0_k, 0) + 1e-6)),
  u_T = ln(T1 / T0), a = asinh(u / 1e-8), standardised;
* the decoded new state (u clamped so that 0 <= Y1 <= 1 and T0/10 <= T1 <= 10 T0), made
  conservative by the weighted least-squares correction of dY = Y1 - Y0:
  dY <- dY - D C^T (C D C^T)^{-1} C dY, D = diag(max(|Y1|, 1e-6)^2), where the rows of C span
  the directions no reaction moves Y in;
* the training loss mean_b [ sum_j (o_bj - t_bj)^2 + w (o_b,err - e*_b)^2 ] with
  e*_b = log10(E_b + 1e-12) held constant, E_b the relative error of the corrected state;
* its gradient by plain reverse-mode differentiation (chain rule, layer by layer);
* the optimiser: AdamW, i.e. Adam's bias-corrected first and second moment estimates (Kingma &
  Ba, "Adam: a method for stochastic optimization", 2015) with the weight decay decoupled from
  the adaptive step (Loshchilov & Hutter, "Decoupled weight decay regularization", 2019), scaled
  by a cosine-annealed learning rate lr_s = lr (1 + cos(pi s / S)) / 2 (their SGDR schedule,
  one cycle without restart).

Everything is written for any species count ns: the network maps ns + 3 features to ns + 2
outputs (ns + 1 targets and the error head).

`bf16_products=True` rounds both operands of every matrix product to bfloat16 (round to nearest even)
before multiplying, as the interface states the tensor-core path does; everything else stays
FP64.  Parity status: pinned by central finite differences of the loss (gradient), the
closed form of GELU through the normal CDF, encode/decode round trips, and the optimality and
feasibility of the conservative correction (tests/test_oracle_mlp.py).
"""
import math

from scipy.special import erf as _erf

import numpy as np

EPS_Y = 1e-6     # Y floor of the log features and of the relative error
U0 = 1e-8        # linear range of the asinh compression
HIDDEN = 128
MAX_CONS = 8


def widths(ns):
    """Layer widths of the network for ns species: ns + 3 inputs, four hidden layers, ns + 2 outputs."""
    return (ns + 3, HIDDEN, HIDDEN, HIDDEN, HIDDEN, ns + 2)


# ------------------------------------------------------------------ parameters

def n_params(ns):
    w = widths(ns)
    return sum(w[l + 1] * w[l] + w[l + 1] for l in range(len(w) - 1))


def ns_of_params(n):
    """Species count of a flat parameter vector of n entries."""
    for ns in range(1, 1024):
        if n_params(ns) == n:
            return ns
    raise ValueError(f"no network has {n} parameters")


def unflatten(flat, widths):
    """Flat parameter vector (W_1 row-major [out][in], b_1, W_2, b_2, ...) -> [(W, b), ...]."""
    flat = np.asarray(flat, dtype=np.float64)
    layers, off = [], 0
    for l in range(len(widths) - 1):
        nin, nout = widths[l], widths[l + 1]
        W = flat[off:off + nin * nout].reshape(nout, nin)
        off += nin * nout
        b = flat[off:off + nout]
        off += nout
        layers.append((W, b))
    assert off == flat.size
    return layers


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


# ------------------------------------------------------------------ normalisation block

def norm_fields(ns):
    return (("mu_x", ns + 3), ("sd_x", ns + 3), ("mu_y", ns + 1), ("sd_y", ns + 1), ("lo_x", ns + 3), ("hi_x", ns + 3),
            ("C", MAX_CONS * ns))


def pack_checkpoint(norm, params):
    """Bytes of a surrogate checkpoint: int32 header ("CHSG", version 1, ns, nparams), the
    normalisation block (float32 fields, then int32 ncons and 3 pad words) and float32 params."""
    ns = len(norm["mu_y"]) - 1
    hdr = np.array([0x47534843, 1, ns, n_params(ns)], dtype=np.int32).tobytes()
    body = b"".join(np.asarray(norm[k], dtype=np.float32).reshape(n).tobytes() for k, n in norm_fields(ns))
    tail = np.array([norm["ncons"], 0, 0, 0], dtype=np.int32).tobytes()
    return hdr + body + tail + np.asarray(params, dtype=np.float32).tobytes()


def unpack_checkpoint(blob):
    hdr = np.frombuffer(blob[:16], dtype=np.int32)
    assert hdr[0] == 0x47534843 and hdr[1] == 1
    ns = int(hdr[2])
    off, norm = 16, {}
    for k, n in norm_fields(ns):
        norm[k] = np.frombuffer(blob[off:off + 4 * n], dtype=np.float32).astype(np.float64)
        off += 4 * n
    norm["C"] = norm["C"].reshape(MAX_CONS, ns)
    norm["ncons"] = int(np.frombuffer(blob[off:off + 4], dtype=np.int32)[0])
    off += 16
    params = np.frombuffer(blob[off:], dtype=np.float32).astype(np.float64)
    assert params.size == hdr[3]
    return norm, params


def conserved_basis(elem, W):
    """Orthonormal rows spanning {c : c = sum_j lambda_j elem[:, j] / W}: the element-mass
    directions, which every element-balanced reaction leaves unchanged."""
    A = (np.asarray(elem, float) / np.asarray(W, float)[:, None]).T        # [ne][ns]
    q, r = np.linalg.qr(A.T)                                               # columns span A's rows
    keep = np.abs(np.diag(r)) > 1e-12 * np.abs(r).max()
    return q[:, keep].T


def conserved_directions(W, nu_f, nu_r):
    """Orthonormal rows spanning the complement of span{W .* (nu_r - nu_f)_r}: every direction of
    Y that no reaction moves (the element masses, and a species that no reaction touches).  The
    null space of the reaction matrix by singular value decomposition."""
    from scipy.linalg import null_space
    R = (np.asarray(W, float)[:, None] * (np.asarray(nu_r, float) - np.asarray(nu_f, float)).T)   # [ns][nr]
    return null_space(R.T).T


# ------------------------------------------------------------------ encodings

def features(T, p, dt, Y):
    """[n][ns + 3] raw features; Y is [n][ns]."""
    T, p, dt = (np.asarray(v, float).reshape(-1) for v in (T, p, dt))
    Y = np.asarray(Y, float)
    return np.column_stack([T, np.log(p), np.log(dt), np.log(np.maximum(Y, 0.0) + EPS_Y)])


def encode(u):
    return np.arcsinh(u / U0)


def decode(a, u_lo, u_hi):
    """u of an encoding a (inverse of encode), clamped to [u_lo, u_hi]."""
    return np.clip(U0 * np.sinh(np.clip(a, -60.0, 60.0)), u_lo, u_hi)


def decode_species(a, Y0):
    """New mass fractions Y1 = base e^u - eps, base = max(Y0, 0) + eps, with u clamped to
    [ln(eps / base), ln((1 + eps) / base)] so that 0 <= Y1 <= 1."""
    base = np.maximum(Y0, 0.0) + EPS_Y
    return base * np.exp(decode(a, np.log(EPS_Y / base), np.log((1.0 + EPS_Y) / base))) - EPS_Y


def decode_temperature(a, T0):
    """New temperature T1 = T0 e^u with T0 / 10 <= T1 <= 10 T0."""
    return T0 * np.exp(decode(a, -np.log(10.0), np.log(10.0)))


def targets(T0, Y0, Y1, T1):
    """[n][ns + 1] raw target encodings of the state (Y1, T1) after dt."""
    base = np.maximum(np.asarray(Y0, float), 0.0) + EPS_Y
    aY = encode(np.log((np.asarray(Y1, float) + EPS_Y) / base))
    aT = encode(np.log(np.asarray(T1, float).reshape(-1) / np.asarray(T0, float).reshape(-1)))
    return np.column_stack([aY, aT])


def conserve(C, Y0, dY):
    """Weighted least-squares correction of each row of dY onto {dY : C dY = 0}: minimise
    sum_k (delta_k / w_k)^2, w_k = max(|Y0_k + dY_k|, eps) (the new state's tolerance scale), by
    the normal equations of the Lagrange conditions."""
    C = np.asarray(C, float)
    out = np.array(dY, dtype=float, copy=True)
    if C.shape[0] == 0:
        return out
    for i in range(out.shape[0]):
        w2 = np.maximum(np.abs(Y0[i] + out[i]), EPS_Y) ** 2     # w_k^2
        lam = np.linalg.solve((C * w2) @ C.T, C @ out[i])
        out[i] = out[i] - w2 * (C.T @ lam)
    return out


def decode_state(norm, o, Y0, T0):
    """Standardised outputs o [n][>= ns + 1] -> conservative new state Y1 [n][ns] and T1 [n]."""
    ns = Y0.shape[1]
    a = o[:, :ns + 1] * norm["sd_y"] + norm["mu_y"]
    Y1 = decode_species(a[:, :ns], Y0)
    T1 = decode_temperature(a[:, ns], T0)
    C = norm["C"][:norm["ncons"]]
    return Y0 + conserve(C, Y0, Y1 - Y0), T1


def state_error(norm, o, Y0, T0, Y1, T1):
    """Relative error of the corrected state: max_k |Y1'_k - Y1_k| / max(|Y1_k|, 1e-6) and
    |T1' - T1| / T1."""
    Yp, Tp = decode_state(norm, o, Y0, T0)
    eY = np.max(np.abs(Yp - Y1) / np.maximum(np.abs(Y1), EPS_Y), axis=1)
    eT = np.abs(Tp - T1) / T1
    return np.maximum(eY, eT)


def standardise_inputs(norm, X):
    return (X - norm["mu_x"]) / norm["sd_x"]


def norm_from_data(X, A):
    """Mean / standard deviation (population) of features X and target encodings A, and the range
    of every feature.  A standard deviation below 1e-12 (a quantity that never changes, e.g. an
    inert species) is replaced by 1."""
    sd_x, sd_y = X.std(0), A.std(0)
    sd_x[sd_x < 1e-12] = 1.0
    sd_y[sd_y < 1e-12] = 1.0
    return dict(mu_x=X.mean(0), sd_x=sd_x, mu_y=A.mean(0), sd_y=sd_y, lo_x=X.min(0), hi_x=X.max(0))


# ------------------------------------------------------------------ network

def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _mm(a, W, rnd):
    return (bf16(a) @ bf16(W).T) if rnd else (a @ W.T)


def forward(layers, x, bf16_products=False):
    """Returns the outputs and the cache (pre-activations z_l, activations a_l)."""
    a, zs, acts = np.asarray(x, float), [], [np.asarray(x, float)]
    for l, (W, b) in enumerate(layers):
        z = _mm(a, W, bf16_products) + b
        zs.append(z)
        a = gelu(z) if l < len(layers) - 1 else z
        acts.append(a)
    return a, (zs, acts)


def loss_and_grad(layers, x, t, e_star, err_weight, bf16_products=False):
    """Loss of a batch and its gradient (list of (dW, db)) by reverse-mode differentiation.
    x [B][n_in] standardised inputs, t [B][ns + 1] standardised targets, e_star [B]."""
    B = x.shape[0]
    nt = t.shape[1]
    o, (zs, acts) = forward(layers, x, bf16_products)
    r = o[:, :nt] - t
    de = o[:, nt] - e_star
    loss = (np.sum(r * r) + err_weight * np.sum(de * de)) / B
    dz = np.zeros_like(o)
    dz[:, :nt] = 2.0 * r / B
    dz[:, nt] = 2.0 * err_weight * de / B
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a_prev = acts[l]
        if bf16_products:
            dW = bf16(dz).T @ bf16(a_prev)
        else:
            dW = dz.T @ a_prev
        grads[l] = (dW, dz.sum(0))
        if l > 0:
            da = _mm(dz, W.T, bf16_products)
            dz = da * gelu_grad(zs[l - 1])
    return loss, grads


def surrogate_loss_and_grad(norm, params, Xraw, Yraw, err_weight, bf16_products=False):
    """The documented training loss of one batch in the library's data layout: Xraw rows
    (T, p, dt, Y[ns]), Yraw rows (Y1[ns], T1), the state after dt.  Returns (loss, flat gradient)."""
    ns = Xraw.shape[1] - 3
    T0, p, dt, Y0 = Xraw[:, 0], Xraw[:, 1], Xraw[:, 2], Xraw[:, 3:]
    Y1, T1 = Yraw[:, :ns], Yraw[:, ns]
    x = standardise_inputs(norm, features(T0, p, dt, Y0))
    t = (targets(T0, Y0, Y1, T1) - norm["mu_y"]) / norm["sd_y"]
    layers = unflatten(params, widths(ns))
    o, _ = forward(layers, x, bf16_products)
    e_star = np.log10(state_error(norm, o, Y0, T0, Y1, T1) + 1e-12)
    loss, grads = loss_and_grad(layers, x, t, e_star, err_weight, bf16_products)
    return loss, flatten(grads)


def surrogate_outputs(norm, params, Xraw, bf16_products=False):
    """Standardised network outputs [n][ns + 2] for raw rows (T, p, dt, Y[ns])."""
    x = standardise_inputs(norm, features(Xraw[:, 0], Xraw[:, 1], Xraw[:, 2], Xraw[:, 3:]))
    o, _ = forward(unflatten(params, widths(Xraw.shape[1] - 3)), x, bf16_products)
    return o


# ------------------------------------------------------------------ optimiser

def cosine_lr(lr, step, total):
    """Learning rate of step s = 0 .. total - 1: lr (1 + cos(pi s / total)) / 2."""
    return 0.5 * lr * (1.0 + math.cos(math.pi * step / total))


def adamw_step(w, g, m, v, t, lr, weight_decay, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW update of parameters w with gradient g at optimiser step t (1-based) and learning
    rate lr; returns the new (w, m, v).  m and v are Adam's running first and second moment
    estimates, divided by 1 - beta^t for the bias of their zero start; the decay of the weights is
    decoupled from the adaptive step and scaled by the same learning rate."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    w = w - lr * (m_hat / (np.sqrt(v_hat) + eps) + weight_decay * w)
    return w, m, v
