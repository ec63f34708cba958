"""The warp-per-cell path for the 53-species / 325-reaction hydrocarbon-shaped mechanism (GPU).

Same method and parity bar as test_gpu_parity.py, on the large mechanism: rates against the
oracle's direct products (up to the FP32 cancellation floor of the gross rates), T(e) and the
state helpers, and one chemistry step of a small reacting sheet against the FP64 oracle on a
sample of stiff and cold cells, plus determinism and the per-cell independence of the result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
import paper_2510_23993_gb300 as chem
import synth

DEV = "cuda:0"
Y_BIG, TOL_Y, ABS_Y, TOL_T = 1e-6, 1e-4, 1e-10, 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chem.build()


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in arrs]


def _inputs32(mech, T, p, Y):
    T, p, Y = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
    rho, e = oracle.state_from_TpY(mech, T, p, Y)
    return T, p, Y, rho.astype(np.float32), e.astype(np.float32)


def test_large_mechanism_shape(hcmech):
    assert hcmech["ns"] == 53 and hcmech["nr"] == 325 and int(hcmech["third_body"].sum()) == 30
    ctx = chem.Context(hcmech, max_cells=16)
    ctx.close()


def test_large_rates_parity(hcmech):
    rng = np.random.default_rng(3)
    n = 500
    T = rng.uniform(800, 3000, n)
    p = rng.uniform(1, 20, n) * synth.P_ATM
    Y = rng.dirichlet(np.full(53, 0.3), size=n).T
    T32, p32, Y32, rho, e = _inputs32(hcmech, T, p, Y)
    ctx = chem.Context(hcmech, max_cells=n)
    tT, tY, trho = _dev(T32, Y32, rho)
    f = torch.empty_like(tY)
    ctx.rates(trho, tT, tY, f)
    f = f.cpu().numpy().astype(np.float64)
    ref, qf, qr = oracle.rates(hcmech, rho, T32, Y32, with_progress=True)
    dnu = (hcmech["nu_r"] - hcmech["nu_f"]).astype(np.float64)          # [nr, ns]
    gross = hcmech["W"][:, None] / rho.astype(np.float64)[None, :] * (np.abs(dnu).T @ (qf + qr))
    # FP32 log-form rates: relative 1e-4 of the net rate, or a few FP32 ulps of the gross rate
    assert np.all(np.abs(f - ref) <= 1e-4 * np.abs(ref) + 2e-5 * gross)
    ctx.close()


def test_large_state_and_temperature(hcmech):
    T, p, Y, hot = synth.sheet_field(hcmech, n=8, seed=2, frac=0.2)
    T32, p32, Y32, rho_o, e_o = _inputs32(hcmech, T, p, Y)
    ctx = chem.Context(hcmech, max_cells=T.size)
    tT, tp, tY = _dev(T32, p32, Y32)
    rho, e = torch.empty_like(tT), torch.empty_like(tT)
    ctx.state_from_TpY(tT, tp, tY, rho, e)
    assert np.allclose(rho.cpu().numpy(), rho_o, rtol=2e-6)
    assert np.allclose(e.cpu().numpy(), e_o, rtol=1e-5, atol=1e-2 * np.abs(e_o).max() * 1e-4)
    tT2 = torch.full_like(tT, 1000.0)
    ctx.temperature(tY, _dev(e_o)[0], tT2)
    T_ref = oracle.temperature_from_energy(hcmech, Y32.astype(np.float64), e_o.astype(np.float64), np.full(T.size, 1000.0))
    assert np.allclose(tT2.cpu().numpy(), T_ref, rtol=1e-6)
    ctx.close()


def _run(ctx, T, p, Y, rho, e, dt):
    tT, tp, tY, trho, te = _dev(T, p, Y, rho, e)
    sub = torch.full((T.size,), -99, dtype=torch.int32, device=DEV)
    ctx.advance(tT, tp, tY, trho, te, dt, sub)
    return ctx.status(), tT.cpu().numpy(), tp.cpu().numpy(), tY.cpu().numpy(), sub.cpu().numpy()


def test_large_advance_parity_sheet(hcmech):
    """12^3 sheet (4% reacting), dt = 1e-8 s: every stiff cell of a sample, and cold cells, vs the oracle."""
    T, p, Y, hot = synth.sheet_field(hcmech, n=12, seed=4, frac=0.04)
    T, p, Y, rho, e = _inputs32(hcmech, T, p, Y)
    ctx = chem.Context(hcmech, max_cells=T.size)
    st, T1, p1, Y1, sub = _run(ctx, T, p, Y, rho, e, 1e-8)
    assert st["status"] == 0 and st["nfailed"] == 0 and st["ninvalid"] == 0
    assert st["nqueued"] == int((sub >= 2).sum()) and st["nbulk"] == int((sub == 1).sum())
    # the warp-per-cell kernel keeps its factored matrix over held steps: fewer LUs than attempts
    assert 0 < st["factorizations"] < st["attempts"]
    assert np.all(sub[hot] >= 2)
    rng = np.random.default_rng(0)
    pick = np.concatenate([np.nonzero(hot)[0][:20], rng.choice(np.nonzero(~hot)[0], 12, replace=False)])
    T_ref, _, Y_ref, _ = oracle.advance(hcmech, rho[pick], e[pick], T[pick], Y[:, pick], 1e-8)
    T_p, _, Y_p, _ = oracle.advance(hcmech, rho[pick], e[pick].astype(np.float64) * (1 + 2.0 ** -23), T[pick],
                                    Y[:, pick], 1e-8)
    big = Y_ref >= Y_BIG
    cT = np.abs(T_p - T_ref) / T_ref
    cY = np.where(big, np.abs(Y_p - Y_ref) / np.maximum(Y_ref, 1e-300), np.abs(Y_p - Y_ref))
    eT = np.abs(T1[pick].astype(np.float64) - T_ref) / T_ref
    Yg = Y1[:, pick].astype(np.float64)
    eY = np.where(big, np.abs(Yg - Y_ref) / np.maximum(Y_ref, 1e-300), np.abs(Yg - Y_ref))
    bad_T = eT > TOL_T + 3 * cT
    bad_Y = eY > np.where(big, TOL_Y, ABS_Y) + 3 * cY
    assert not bad_T.any(), (eT.max(), np.nonzero(bad_T))
    assert not bad_Y.any(), (eY[bad_Y].max(), np.nonzero(bad_Y.any(0)))
    # invariants: sum Y and element masses
    assert np.allclose(Y1.astype(np.float64).sum(0), Y.astype(np.float64).sum(0), atol=2e-6)
    ctx.close()


def test_large_determinism_and_independence(hcmech):
    T, p, Y, hot = synth.sheet_field(hcmech, n=8, seed=5, frac=0.1)
    T, p, Y, rho, e = _inputs32(hcmech, T, p, Y)
    ctx = chem.Context(hcmech, max_cells=T.size)
    a = _run(ctx, T, p, Y, rho, e, 1e-8)
    b = _run(ctx, T, p, Y, rho, e, 1e-8)
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)
    i = int(np.nonzero(hot)[0][0])
    one = _run(ctx, T[[i]], p[[i]], Y[:, [i]], rho[[i]], e[[i]], 1e-8)
    assert one[1][0] == a[1][i] and np.array_equal(one[3][:, 0], a[3][:, i]) and one[4][0] == a[4][i]
    ctx.close()


def test_large_boxes_match_per_box_advance(hcmech):
    """Three uneven boxes with per-box dt through one bulk and one stiff launch of the warp-per-cell
    path equal chem_advance on each box alone, bit for bit."""
    boxes, hosts = [], []
    for k, (edge, dt) in enumerate(((6, 1e-8), (4, 5e-9), (5, 2.5e-9))):
        T, p, Y, hot = synth.sheet_field(hcmech, n=edge, seed=10 + k, frac=0.1)
        T, p, Y, rho, e = _inputs32(hcmech, T, p, Y)
        hosts.append((T, p, Y, rho, e, dt))
        d = dict(zip(("T", "p", "Y", "rho", "e"), _dev(T, p, Y, rho, e)))
        d["substeps"] = torch.zeros(T.size, dtype=torch.int32, device=DEV)
        d["dt"], d["level"] = dt, k
        boxes.append(d)
    total = sum(h[0].size for h in hosts)
    ctx = chem.Context(hcmech, max_cells=total)
    ctx.set_boxes(boxes)
    ctx.advance_boxes()
    st = ctx.status()
    assert st["status"] == 0 and st["ncell"] == total and st["nqueued"] > 0
    for d, (T, p, Y, rho, e, dt) in zip(boxes, hosts):
        ref = _run(ctx, T, p, Y, rho, e, dt)
        assert np.array_equal(ref[1], d["T"].cpu().numpy()) and np.array_equal(ref[3], d["Y"].cpu().numpy())
        assert np.array_equal(ref[4], d["substeps"].cpu().numpy())
    ctx.close()
