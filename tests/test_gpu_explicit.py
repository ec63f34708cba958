"""The paper's own integration loop on the GPU (chem_advance_explicit): the explicit first-order
scheme of Sec. 2.1 under the bulk / sparse control of Algorithm 3.

* Algorithm 3 only decides how a cell's substeps are split over launches, so every split (no
  bulk launch at all, i.e. Algorithm 2; bulk launches until every cell is done; mixtures) gives
  the same bits for every cell;
* the counters add up (skipped + finished in bulk + entering the sparse launch + invalid = n);
* against the oracle's FP64 restatement of the same scheme, with FP64 rates (CHEM_FLAG_FP64_RATES):
  the usual bar, 1e-4 relative (1e-10 absolute below Y = 1e-6), plus 3x the oracle's own largest
  response to rounding-size perturbations of the inputs; in cells where the scheme amplifies
  rounding, alternatively an error against the exact solution within that of the perturbed FP64
  runs; and the same median error against the exact solution;
* with FP32 rates (the default) the error against the exact solution has the oracle's distribution;
* failure reporting: a k_max too small for the stiff cells marks them -1 with CHEM_EMAXSTEPS,
  invalid input is reported, bad arguments are refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
import paper_2510_23993_gb300 as chem
import synth

DEV = "cuda:0"
TOL_T, TOL_Y, ABS_Y, Y_BIG = 1e-4, 1e-4, 1e-10, 1e-6
# a tenth of the benchmark step: the stiffest reacting cells of the synthetic fields need more
# than the paper's 1e5 explicit substeps at 1e-8 s, so the tests use a step that every cell finishes
DT = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chem.build()


@pytest.fixture(scope="module")
def sheet(h2mech):
    T, p, Y, hot = synth.sheet_field(h2mech, n=16, seed=7, frac=0.05)
    T, p, Y = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
    rho, e = oracle.state_from_TpY(h2mech, T, p, Y)
    return T, p, Y, rho.astype(np.float32), e.astype(np.float32), hot


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in arrs]


def _run(ctx, T, p, Y, rho, e, k_steps, n_star, dt=DT):
    tT, tp, tY, trho, te = _dev(T, p, Y, rho, e)
    sub = torch.full((T.size,), -99, dtype=torch.int32, device=DEV)
    nl = ctx.advance_explicit(tT, tp, tY, trho, te, dt, sub, k_steps=k_steps, n_star=n_star)
    return nl, ctx.status(), tT.cpu().numpy(), tp.cpu().numpy(), tY.cpu().numpy(), sub.cpu().numpy()


def test_split_over_launches_does_not_change_cells(h2mech, sheet):
    T, p, Y, rho, e, hot = sheet
    ctx = chem.Context(h2mech, max_cells=T.size)   # FP32 rates (FP64 where they overflow)
    runs = {(k, ns): _run(ctx, T, p, Y, rho, e, k, ns) for k, ns in ((5, 10 ** 9), (5, 0), (3, 20), (1, 100), (5, 10000))}
    ref = runs[(5, 10 ** 9)]
    assert ref[0] == 0                                   # Algorithm 2: the sparse launch alone
    assert runs[(5, 0)][0] >= ref[5].max() // 5          # bulk launches until every cell is done
    for key, r in runs.items():
        assert r[1]["status"] == 0 and r[1]["nfailed"] == 0, key
        for a, b in zip(r[2:], ref[2:]):
            assert np.array_equal(a, b), key
        st = r[1]
        assert st["nskipped"] + st["nbulk"] + st["nqueued"] + st["ninvalid"] == T.size, key
        assert st["substeps"] == int(r[5].sum()), key
    assert runs[(5, 0)][1]["nqueued"] == 0 and runs[(5, 10 ** 9)][1]["nbulk"] == 0
    assert np.all(ref[5][hot] > 1) and np.all(ref[5] >= 1)
    ctx.close()


def test_explicit_parity_vs_oracle(h2mech, sheet):
    """Cell by cell against the oracle's FP64 explicit scheme.  The scheme runs stiff modes at the
    edge of forward-Euler stability (the change rule does not bound h |lambda|), so many reacting
    cells amplify rounding: a one-ulp FP64 change of e moves their final state by up to ~1e-3.  An
    ensemble of eight rounding-size perturbations of the oracle's inputs (e by 1 and 2 FP64 ulps
    either way and by one FP32 ulp either way, rho by 1e-15 either way) measures that per cell:
      * cells that do not amplify (one-ulp response below 1e-10) hold the plain bar;
      * every cell holds the bar plus 3x the ensemble's largest deviation from the oracle, or, where
        the cell amplifies (a response above 1e-6), lies within the bar plus 3x the ensemble's
        largest error against the exact solution -- it is as accurate as an FP64 run of the scheme;
      * over the reacting cells, the median error against the exact solution matches the oracle's."""
    T, p, Y, rho, e, hot = sheet
    ctx = chem.Context(h2mech, max_cells=T.size, flags=chem.CHEM_FLAG_FP64_RATES)
    nl, st, T1, p1, Y1, sub = _run(ctx, T, p, Y, rho, e, 5, 10000)
    assert st["status"] == 0
    rng = np.random.default_rng(1)
    pick = np.concatenate([np.nonzero(hot)[0], rng.choice(np.nonzero(~hot)[0], 64, replace=False)])
    nh = int(hot.sum())
    # the kernel reads the change limit and the floor in FP32: the oracle takes the same values
    kw = dict(frac=float(np.float32(ctx.params.bulk_frac)), y_floor=float(np.float32(ctx.params.y_floor)))
    r, ee, Tp, Yp = rho[pick].astype(np.float64), e[pick].astype(np.float64), T[pick], Y[:, pick]
    T_ref, _, Y_ref, s_ref = oracle.explicit(h2mech, r, ee, Tp, Yp, DT, **kw)
    T_ex, _, Y_ex, _ = oracle.advance(h2mech, r, ee, Tp, Yp, DT)
    big = Y_ref >= Y_BIG
    bar_Y = np.where(big, TOL_Y, ABS_Y)

    def dev(Ta, Ya, Tb, Yb):
        dY = np.where(big, np.abs(Ya - Yb) / np.maximum(Yb, 1e-300), np.abs(Ya - Yb))
        return np.abs(Ta - Tb) / Tb, dY

    cT, cY, cS = np.zeros(pick.size), np.zeros_like(Y_ref), np.zeros(pick.size)
    xT, xY = dev(T_ref, Y_ref, T_ex, Y_ex)
    ens = [(r, ee * (1 + k * 2.0 ** -52)) for k in (1, 2, -1, -2)] + \
          [(r * (1 + 1e-15), ee), (r * (1 - 1e-15), ee), (r, ee * (1 + 2.0 ** -23)), (r, ee * (1 - 2.0 ** -23))]
    calm = None
    for rr, e2 in ens:
        Ta, _, Ya, sa = oracle.explicit(h2mech, rr, e2, Tp, Yp, DT, **kw)
        dT, dY = dev(Ta, Ya, T_ref, Y_ref)
        if calm is None:   # the response to one FP64 ulp of e
            calm = (dT < 1e-10) & (dY.max(0) < 1e-10)
        cT, cY, cS = np.maximum(cT, dT), np.maximum(cY, dY), np.maximum(cS, np.abs(sa - s_ref))
        aT, aY = dev(Ta, Ya, T_ex, Y_ex)
        xT, xY = np.maximum(xT, aT), np.maximum(xY, aY)
    amp = (cT > 1e-6) | (cY.max(0) > 1e-6)
    Tg, Yg = T1[pick].astype(np.float64), Y1[:, pick].astype(np.float64)
    eT, eY = dev(Tg, Yg, T_ref, Y_ref)
    gT, gY = dev(Tg, Yg, T_ex, Y_ex)
    assert calm[:nh].sum() > nh // 2
    assert np.all(eT[calm] <= TOL_T) and np.all(eY[:, calm] <= bar_Y[:, calm])
    parity = (eT <= TOL_T + 3 * cT) & np.all(eY <= bar_Y + 3 * cY, axis=0)
    envelope = (gT <= TOL_T + 3 * xT) & np.all(gY <= bar_Y + 3 * xY, axis=0)
    bad = ~(parity | (amp & envelope))
    assert not bad.any(), (np.nonzero(bad)[0], eT[bad], eY[:, bad].max(0))
    assert np.all((np.abs(sub[pick] - s_ref) <= 2 + 3 * cS) | amp)
    assert 0.67 < np.median(gT[:nh]) / np.median(np.abs(T_ref - T_ex)[:nh] / T_ex[:nh]) < 1.5
    ctx.close()


def test_fp32_rates_same_accuracy(h2mech, sheet):
    """Default mode (FP32 rates): the rates' 1e-7..1e-6 rounding acts on the scheme like a model
    perturbation, so cells are not compared one by one; the error against the exact solution over
    the reacting cells has the oracle's distribution (50th, 90th, 99th percentiles within 1.5x)."""
    T, p, Y, rho, e, hot = sheet
    ctx = chem.Context(h2mech, max_cells=T.size)
    nl, st, T1, p1, Y1, sub = _run(ctx, T, p, Y, rho, e, 5, 10000)
    assert st["status"] == 0
    idx = np.nonzero(hot)[0]
    kw = dict(frac=float(np.float32(ctx.params.bulk_frac)), y_floor=float(np.float32(ctx.params.y_floor)))
    r, ee, Tp, Yp = rho[idx].astype(np.float64), e[idx].astype(np.float64), T[idx], Y[:, idx]
    T_ref, _, Y_ref, _ = oracle.explicit(h2mech, r, ee, Tp, Yp, DT, **kw)
    T_ex, _, Y_ex, _ = oracle.advance(h2mech, r, ee, Tp, Yp, DT)
    big = Y_ex >= Y_BIG

    def err(Ta, Ya):
        return np.abs(Ta - T_ex) / T_ex, np.where(big, np.abs(Ya - Y_ex) / Y_ex, 0.0).max(0)

    gT, gY = err(T1[idx].astype(np.float64), Y1[:, idx].astype(np.float64))
    oT, oY = err(T_ref, Y_ref)
    for q in (50, 90, 99):
        assert 0.67 < np.percentile(gT, q) / np.percentile(oT, q) < 1.5, q
        assert 0.67 < np.percentile(gY, q) / np.percentile(oY, q) < 1.5, q
    ctx.close()


def test_failures_invalid_input_and_arguments(h2mech, sheet):
    T, p, Y, rho, e, hot = sheet
    ctx = chem.Context(h2mech, max_cells=T.size, flags=chem.CHEM_FLAG_FP64_RATES)
    ctx.set_params(k_max=20)
    nl, st, T1, p1, Y1, sub = _run(ctx, T, p, Y, rho, e, 5, 0)
    assert nl == 4                                       # ceil(k_max / k_steps) bulk launches
    assert st["status"] == chem.CHEM_EMAXSTEPS and st["nfailed"] == int((sub == -1).sum()) > 0
    assert np.all(sub[~hot] >= 1)
    ctx.set_params(k_max=100000)
    Tb = T.copy()
    Tb[3] = np.nan
    nl, st, T1, p1, Y1, sub = _run(ctx, Tb, p, Y, rho, e, 5, 10000)
    assert st["status"] == chem.CHEM_EINVAL and st["ninvalid"] == 1 and sub[3] == -1
    tT, tp, tY, trho, te = _dev(T, p, Y, rho, e)
    s = torch.zeros(T.size, dtype=torch.int32, device=DEV)
    with pytest.raises(chem.ChemError):
        ctx.advance_explicit(tT, tp, tY, trho, te, DT, s, k_steps=0)
    with pytest.raises(chem.ChemError):
        ctx.advance_explicit(tT, tp, tY, trho, te, DT, s, n_star=-1)
    ctx.close()
