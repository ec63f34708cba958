"""The paper's own integration loop on the GPU (chem_advance_explicit): the explicit first-order
scheme of Sec. 2.1 under the bulk / sparse control of Algorithm 3.

* Algorithm 3 only decides how a cell's substeps are split over launches, so every split (no
  bulk launch at all, i.e. Algorithm 2; bulk launches until every cell is done; mixtures) gives
  the same bits for every cell;
* the counters add up (skipped + finished in bulk + entering the sparse launch + invalid = n);
* against the oracle's FP64 restatement of the same scheme: the FP32 state and FP32 rates of the
  kernel perturb the model at the 1e-7 level, so the bar is the usual 1e-4 relative (1e-10
  absolute below Y = 1e-6) plus 3x the oracle's own response to a one-ulp (FP32) change of e;
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
DT = 1e-8


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
    ctx = chem.Context(h2mech, max_cells=T.size)
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
    T, p, Y, rho, e, hot = sheet
    ctx = chem.Context(h2mech, max_cells=T.size)
    nl, st, T1, p1, Y1, sub = _run(ctx, T, p, Y, rho, e, 5, 10000)
    assert st["status"] == 0
    rng = np.random.default_rng(1)
    pick = np.concatenate([np.nonzero(hot)[0], rng.choice(np.nonzero(~hot)[0], 64, replace=False)])
    frac = ctx.params.bulk_frac
    T_ref, p_ref, Y_ref, s_ref = oracle.explicit(h2mech, rho[pick], e[pick], T[pick], Y[:, pick], DT, frac=frac)
    T_p, _, Y_p, _ = oracle.explicit(h2mech, rho[pick], e[pick].astype(np.float64) * (1 + 2.0 ** -23), T[pick],
                                     Y[:, pick], DT, frac=frac)
    big = Y_ref >= Y_BIG
    cT = np.abs(T_p - T_ref) / T_ref
    cY = np.where(big, np.abs(Y_p - Y_ref) / np.maximum(Y_ref, 1e-300), np.abs(Y_p - Y_ref))
    eT = np.abs(T1[pick].astype(np.float64) - T_ref) / T_ref
    Yg = Y1[:, pick].astype(np.float64)
    eY = np.where(big, np.abs(Yg - Y_ref) / np.maximum(Y_ref, 1e-300), np.abs(Yg - Y_ref))
    assert not np.any(eT > TOL_T + 3 * cT), eT.max()
    bad = eY > np.where(big, TOL_Y, ABS_Y) + 3 * cY
    assert not bad.any(), (eY[bad].max(), np.nonzero(bad.any(0)))
    # the substep counts follow the same rule: equal up to a few where FP32 moves a boundary
    assert np.all(np.abs(sub[pick] - s_ref) <= np.maximum(2, 0.01 * s_ref))
    ctx.close()


def test_failures_invalid_input_and_arguments(h2mech, sheet):
    T, p, Y, rho, e, hot = sheet
    ctx = chem.Context(h2mech, max_cells=T.size)
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
