"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (the accuracy target: 1e-4 relative on T and on every non-negligible Y):
  * advanced state: |T - T_ref| / T_ref <= 1e-4; Y_ref >= 1e-6: |Y - Y_ref| / Y_ref <= 1e-4;
    Y_ref < 1e-6: |Y - Y_ref| <= 1e-10.  This bar is applied as is to the FP64-rate mode and to
    every well-conditioned cell.  The default mode evaluates rates from FP32-rounded tables,
    which perturbs the model at the 1e-7 level; cells whose exact solution itself moves by more
    than the bar under such a perturbation (runaway cells whose final radicals amplify input
    changes ~1000x) get the bar plus 3x the oracle's own response to a one-ulp (FP32) change of
    the internal energy, measured cell by cell;
  * FP32 rates: |f - f_ref| <= 3e-5 * s_k with s_k = W_k / rho * sum_r |dnu_kr| (q_f + q_r)
    (FP32 log-form kinetics: the error of ln q is ~|ln q| * 6e-8);
  * FP64 temperature inversion with FP32 output: 2 ulp of FP32 (relative 2.5e-7).
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chem.build()


def _inputs32(mech, T, p, Y):
    """FP32-rounded (T, p, Y) and the oracle's rho, e for them (rounded to FP32)."""
    T, p, Y = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
    rho, e = oracle.state_from_TpY(mech, T, p, Y)
    return T, p, Y, rho.astype(np.float32), e.astype(np.float32)


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in arrs]


def _run(ctx, T, p, Y, rho, e, dt, ld=None):
    n = T.shape[0]
    tT, tp, trho, te = _dev(T, p, rho, e)
    if ld is None:
        tY = _dev(Y)[0]
    else:   # padded leading dimension
        tY = torch.full((Y.shape[0], ld), -7.0, dtype=torch.from_numpy(Y).dtype, device=DEV)
        tY[:, :n] = torch.from_numpy(Y).to(DEV)
    sub = torch.full((n,), -99, dtype=torch.int32, device=DEV)
    rc = chem.chem_advance(ctx.handle, tT, tp, tY, tY.stride(0), trho, te, n, dt, sub)
    st = ctx.status()
    assert st["factorizations"] == st["attempts"]   # one thread per cell: one LU per attempted step
    Yo = tY.cpu().numpy()
    if ld is not None:
        assert np.all(Yo[:, n:] == -7.0)   # padding untouched
        Yo = Yo[:, :n]
    return rc, st, tT.cpu().numpy(), tp.cpu().numpy(), Yo, sub.cpu().numpy()


def _conditioning(mech, rho, e, T, Y, dt, T_ref, Y_ref):
    """The oracle's own response to a one-ulp (FP32) change of e, per cell and species."""
    e_p = np.asarray(e, np.float64) * (1.0 + 2.0 ** -23)
    T_p, _, Y_p, _ = oracle.advance(mech, rho, e_p, T, Y, dt)
    dT = np.abs(T_p - T_ref) / T_ref
    big = Y_ref >= Y_BIG
    dY = np.where(big, np.abs(Y_p - Y_ref) / np.maximum(Y_ref, 1e-300), np.abs(Y_p - Y_ref))
    return dT, dY


def _parity(T, Y, T_ref, Y_ref, mask=None, cond=None):
    """Check the bar; cond = (dT, dY) adds 3x the oracle's one-ulp response per cell."""
    if mask is not None:
        T, Y, T_ref, Y_ref = T[mask], Y[:, mask], T_ref[mask], Y_ref[:, mask]
        if cond is not None:
            cond = (cond[0][mask], cond[1][:, mask])
    T = T.astype(np.float64)
    Y = Y.astype(np.float64)
    big = Y_ref >= Y_BIG
    tolT = TOL_T + (3.0 * cond[0] if cond is not None else 0.0)
    tolY = np.where(big, TOL_Y, ABS_Y) + (3.0 * cond[1] if cond is not None else 0.0)
    eT = np.abs(T - T_ref) / T_ref
    eY = np.where(big, np.abs(Y - Y_ref) / np.maximum(Y_ref, 1e-300), np.abs(Y - Y_ref))
    bad_T = eT > tolT
    bad_Y = eY > tolY
    assert not bad_T.any(), f"T rel err {eT[bad_T].max():.3e} in {bad_T.sum()} cells"
    assert not bad_Y.any(), f"Y err {eY[bad_Y].max():.3e} in {bad_Y.any(0).sum()} cells"
    strict = (eT > TOL_T) | np.any(eY > np.where(big, TOL_Y, ABS_Y), axis=0)
    rel_big = np.where(big, eY, 0.0)
    return dict(maxT=eT.max(), maxY=rel_big.max(), maxabs=np.where(~big, eY, 0.0).max(),
                p999Y=float(np.percentile(rel_big.max(0), 99.9)), over_strict_bar=int(strict.sum()))


# ---------------------------------------------------------------- building blocks

def test_state_from_TpY_parity(h2mech):
    T, p, Y, hot = synth.sheet_field(h2mech, n=24, seed=3)
    T, p, Y, rho_ref, e_ref = _inputs32(h2mech, T, p, Y)
    ctx = chem.Context(h2mech, max_cells=T.size)
    tT, tp, tY = _dev(T, p, Y)
    rho = torch.empty_like(tT)
    e = torch.empty_like(tT)
    ctx.state_from_TpY(tT, tp, tY, rho, e)
    rho_ref64, e_ref64 = oracle.state_from_TpY(h2mech, T, p, Y)
    assert np.max(np.abs(rho.cpu().numpy() - rho_ref64) / rho_ref64) < 2.5e-7
    assert np.max(np.abs(e.cpu().numpy() - e_ref64) / np.abs(e_ref64)) < 2.5e-7
    ctx.close()


def test_temperature_parity(h2mech):
    rng = np.random.default_rng(5)
    n = 3000
    Y = rng.dirichlet(np.full(9, 0.5), size=n).T.astype(np.float32)
    T = rng.uniform(150.0, 9000.0, size=n)    # spans all three thermo regimes
    rho, e = oracle.state_from_TpY(h2mech, T, np.full(n, 1e5), Y)
    e32 = e.astype(np.float32)
    T_ref = oracle.temperature_from_energy(h2mech, Y, e32, T)
    ctx = chem.Context(h2mech, max_cells=n)
    tY, te = _dev(Y, e32)
    tT = torch.full((n,), 1500.0, dtype=torch.float32, device=DEV)
    ctx.temperature(tY, te, tT)
    assert np.max(np.abs(tT.cpu().numpy() - T_ref) / T_ref) < 2.5e-7
    ctx.close()


def test_rates_parity(h2mech):
    rng = np.random.default_rng(6)
    n = 4000
    Y = rng.dirichlet(np.full(9, 0.5), size=n).T.astype(np.float32)
    Y[:, :50] = synth.premix_mass_fractions(h2mech)[:, None]   # exact zeros (log floor path)
    T = rng.uniform(250.0, 5000.0, size=n).astype(np.float32)
    rho = rng.uniform(0.05, 10.0, size=n).astype(np.float32)
    f_ref, qf, qr = oracle.rates(h2mech, rho, T, Y, with_progress=True)
    dnu = np.abs(h2mech["nu_r"].astype(float) - h2mech["nu_f"]).T      # [ns, nr]
    scale = (h2mech["W"][:, None] / rho[None, :].astype(np.float64)) * (dnu @ (qf + qr))
    ctx = chem.Context(h2mech, max_cells=n)
    trho, tT, tY = _dev(rho, T, Y)
    f = torch.empty_like(tY)
    ctx.rates(trho, tT, tY, f)
    err = np.abs(f.cpu().numpy() - f_ref) / (scale + 1e-30)
    assert np.max(err) < 3e-5, np.max(err)
    # the statistic of the paper's App. A: the coefficient of determination of each species'
    # production rate over the random states (the inert species, identically zero, has none);
    # errors at the bar above would still give R^2 > 1 - 2e-9
    fo = f.cpu().numpy().astype(np.float64)
    for k in range(h2mech["ns"]):
        ss_tot = np.sum((f_ref[k] - f_ref[k].mean()) ** 2)
        if ss_tot > 0:
            assert 1.0 - np.sum((fo[k] - f_ref[k]) ** 2) / ss_tot > 0.999999, k
    ctx.close()


# ---------------------------------------------------------------- advance: small configurations

def test_advance_f64_slab_4096(h2mech):
    """16^3 premix with a hot slab, FP64 state, dt = 1e-7 s (the small FP64 workload)."""
    T, p, Y, hot = synth.slab_field(h2mech)
    rho, e = oracle.state_from_TpY(h2mech, T, p, Y)
    ctx = chem.Context(h2mech, max_cells=T.size)
    dt = 1e-7
    rc, st, To, po, Yo, sub = _run(ctx, T, p, Y, rho, e, dt)
    assert rc == 0 and st["status"] == 0, st
    T_ref, p_ref, Y_ref, steps = oracle.advance(h2mech, rho, e, T, Y, dt)
    assert np.all(steps > 0)
    errs = _parity(To, Yo, T_ref, Y_ref)
    assert np.all(sub[~hot] == 1) and np.all(sub[hot] >= 2)
    assert st["nqueued"] == hot.sum() and st["nbulk"] == (~hot).sum()
    assert np.max(np.abs(po - p_ref) / p_ref) < 1e-4
    print("slab parity", errs, "stiff substeps mean", sub[hot].mean())
    ctx.close()


@pytest.mark.parametrize("n_edge,seed", [(24, 0), (19, 1)])
def test_advance_f32_sheet(h2mech, n_edge, seed):
    """Reacting sheet (5%) in cold premix, FP32 state, dt = 1e-8 s; several tiles + ragged tail."""
    T, p, Y, hot = synth.sheet_field(h2mech, n=n_edge, seed=seed)
    T, p, Y, rho, e = _inputs32(h2mech, T, p, Y)
    n = T.size
    ctx = chem.Context(h2mech, max_cells=n)
    dt = 1e-8
    rc, st, To, po, Yo, sub = _run(ctx, T, p, Y, rho, e, dt)
    assert rc == 0 and st["status"] == 0, st
    T_ref, _, Y_ref, steps = oracle.advance(h2mech, rho, e, T, Y, dt)
    cond = _conditioning(h2mech, rho, e, T, Y, dt, T_ref, Y_ref)
    errs = _parity(To, Yo, T_ref, Y_ref, cond=cond)
    assert st["nqueued"] + st["nbulk"] + st["nskipped"] + st["ninvalid"] == n
    assert st["nqueued"] == np.sum(sub >= 2) and st["nbulk"] == np.sum(sub == 1)
    print("sheet parity", errs, st)
    ctx.close()


def test_fp64_rate_mode_meets_strict_bar(h2mech):
    """With FP64 rates (CHEM_FLAG_FP64_RATES) the integrator meets the bar on every cell,
    ill-conditioned ones included: the remaining difference of the default mode is the FP32
    rounding of the rate tables, not the integration."""
    T, p, Y, hot = synth.sheet_field(h2mech, n=24, seed=0)
    T, p, Y, rho, e = _inputs32(h2mech, T, p, Y)
    idx = np.nonzero(hot)[0]
    T, p, Y, rho, e = T[idx], p[idx], np.ascontiguousarray(Y[:, idx]), rho[idx], e[idx]
    ctx = chem.Context(h2mech, max_cells=T.size, flags=chem.CHEM_FLAG_FP64_RATES)
    rc, st, To, po, Yo, sub = _run(ctx, T, p, Y, rho, e, 1e-8)
    assert rc == 0 and st["status"] == 0, st
    T_ref, _, Y_ref, _ = oracle.advance(h2mech, rho, e, T, Y, 1e-8)
    errs = _parity(To, Yo, T_ref, Y_ref)
    print("fp64-rate mode parity", errs)
    ctx.close()


def test_padded_leading_dimension_and_k_bulk(h2mech):
    T, p, Y, hot = synth.sheet_field(h2mech, n=12, seed=4)
    T, p, Y, rho, e = _inputs32(h2mech, T, p, Y)
    ctx = chem.Context(h2mech, max_cells=T.size, k_bulk=2)
    rc, st, To, po, Yo, sub = _run(ctx, T, p, Y, rho, e, 1e-8, ld=T.size + 37)
    assert rc == 0 and st["status"] == 0
    T_ref, _, Y_ref, _ = oracle.advance(h2mech, rho, e, T, Y, 1e-8)
    _parity(To, Yo, T_ref, Y_ref, cond=_conditioning(h2mech, rho, e, T, Y, 1e-8, T_ref, Y_ref))
    assert np.all((sub == 2) | (sub >= 3))
    ctx.close()


# ---------------------------------------------------------------- edge cases

def test_edge_cases(h2mech):
    T, p, Y, hot = synth.sheet_field(h2mech, n=8, seed=2, frac=0.2)
    T, p, Y, rho, e = _inputs32(h2mech, T, p, Y)
    n = T.size
    ctx = chem.Context(h2mech, max_cells=n)
    # n = 0 is a no-op
    tT, tp, tY, trho, te = _dev(T, p, Y, rho, e)
    sub = torch.zeros(n, dtype=torch.int32, device=DEV)
    assert chem.chem_advance(ctx.handle, tT, tp, tY, n, trho, te, 0, 1e-8, sub) == 0
    # n > max_cells
    assert chem.chem_advance(ctx.handle, tT, tp, tY, n, trho, te, n + 1, 1e-8, sub) == chem.CHEM_ENOMEM
    # bad dt / ld
    assert chem.chem_advance(ctx.handle, tT, tp, tY, n, trho, te, n, -1.0, sub) == chem.CHEM_EINVAL
    assert chem.chem_advance(ctx.handle, tT, tp, tY, n - 1, trho, te, n, 1e-8, sub) == chem.CHEM_EINVAL
    # invalid cells are flagged, left untouched, and do not disturb the others
    Tb, rb = T.copy(), rho.copy()
    Tb[3] = np.nan
    rb[5] = -1.0
    rc, st, To, po, Yo, sub = _run(ctx, Tb, p, Y, rb, e, 1e-8)
    assert rc == 0 and st["ninvalid"] == 2 and st["status"] == chem.CHEM_EINVAL
    assert sub[3] == -1 and sub[5] == -1 and To[5] == T[5] and np.all(Yo[:, 5] == Y[:, 5])
    ok = np.ones(n, bool)
    ok[[3, 5]] = False
    T_ref, _, Y_ref, _ = oracle.advance(h2mech, rho, e, T, Y, 1e-8)
    _parity(To, Yo, T_ref, Y_ref, mask=ok, cond=_conditioning(h2mech, rho, e, T, Y, 1e-8, T_ref, Y_ref))
    # activity threshold: cold cells skipped and untouched
    ctx.set_params(T_min=600.0)
    rc, st, To, po, Yo, sub = _run(ctx, T, p, Y, rho, e, 1e-8)
    cold = T < 600
    assert np.all(sub[cold] == 0) and np.all(To[cold] == T[cold]) and np.array_equal(Yo[:, cold], Y[:, cold])
    assert st["nskipped"] == cold.sum()
    # k_max reached: stiff cells fail cleanly, bulk cells still fine
    ctx.set_params(T_min=0.0, k_max=2)
    rc, st, To, po, Yo, sub = _run(ctx, T, p, Y, rho, e, 1e-8)
    assert st["status"] == chem.CHEM_EMAXSTEPS and st["nfailed"] == hot.sum()
    assert np.all(sub[hot] == -1) and np.array_equal(Yo[:, hot], Y[:, hot])
    assert np.all(sub[~hot] == 1)
    ctx.close()


def test_single_cell_and_determinism(h2mech):
    T, p, Y, hot = synth.sheet_field(h2mech, n=10, seed=7, frac=0.1)
    T, p, Y, rho, e = _inputs32(h2mech, T, p, Y)
    i = int(np.nonzero(hot)[0][0])
    ctx = chem.Context(h2mech, max_cells=T.size)
    rc, st, T1, _, Y1, s1 = _run(ctx, T[[i]], p[[i]], Y[:, [i]], rho[[i]], e[[i]], 1e-8)
    assert rc == 0 and s1[0] >= 2
    rc, st, Ta, _, Ya, sa = _run(ctx, T, p, Y, rho, e, 1e-8)
    rc, st, Tb, _, Yb, sb = _run(ctx, T, p, Y, rho, e, 1e-8)
    assert np.array_equal(Ta, Tb) and np.array_equal(Ya, Yb) and np.array_equal(sa, sb)
    # a cell's result does not depend on its queue slot or neighbours
    assert T1[0] == Ta[i] and np.array_equal(Y1[:, 0], Ya[:, i])
    ctx.close()


def test_result_independent_of_queue_order_and_schedule(h2mech):
    """Each stiff cell is integrated from its own inputs alone (the cells of Algorithm 3's sparse
    phase are independent), so the order in which the stiff kernel takes them and the schedule of
    the stiff phase change nothing: compaction order (no key), the rate-keyed and the
    previous-count-keyed cost orders, and the two-pass schedule give the same T, p, Y bits, the
    same per-cell substep counts and the same counters."""
    T, p, Y, hot = synth.sheet_field(h2mech, n=24, seed=9, frac=0.08)
    T, p, Y, rho, e = _inputs32(h2mech, T, p, Y)
    runs = {}
    prev = None
    for name, flags in [("compaction", 0), ("order_rate", chem.CHEM_FLAG_ORDER_RATE),
                        ("order_prev", chem.CHEM_FLAG_ORDER_PREV), ("two_pass", chem.CHEM_FLAG_TWO_PASS),
                        ("order_rate_two_pass", chem.CHEM_FLAG_ORDER_RATE | chem.CHEM_FLAG_TWO_PASS)]:
        ctx = chem.Context(h2mech, max_cells=T.size, flags=flags)
        tT, tp, tY, trho, te = _dev(T, p, Y, rho, e)
        # ORDER_PREV keys on the counts already in substeps: hand it a previous call's counts
        sub = torch.from_numpy(prev.copy()).to(DEV) if flags == chem.CHEM_FLAG_ORDER_PREV else \
            torch.full((T.size,), -99, dtype=torch.int32, device=DEV)
        rc = chem.chem_advance(ctx.handle, tT, tp, tY, tY.stride(0), trho, te, T.size, 1e-8, sub)
        st = ctx.status()
        assert rc == 0 and st["status"] == 0 and st["nqueued"] == int(hot.sum())
        runs[name] = (tT.cpu().numpy(), tp.cpu().numpy(), tY.cpu().numpy(), sub.cpu().numpy(), st)
        if prev is None:
            prev = runs[name][3]
        ctx.close()
    ref = runs["compaction"]
    assert (ref[3] > 1 + 32).sum() > 10   # some cells outlive the two-pass probe
    for name, r in runs.items():
        assert np.array_equal(r[0], ref[0]) and np.array_equal(r[1], ref[1]), name
        assert np.array_equal(r[2], ref[2]), name
        assert np.array_equal(r[3], ref[3]), name
        for k in ("nqueued", "nbulk", "substeps", "attempts", "newton", "nfailed"):
            assert r[4][k] == ref[4][k], (name, k)


@pytest.mark.parametrize("order", [0, chem.CHEM_FLAG_ORDER_RATE])
def test_two_pass_equals_single_pass(h2mech, order):
    """The two-pass stiff phase parks unfinished cells with their full integration state and
    resumes them later: every cell's result and substep count are bit-identical, and so are the
    counters of attempts and Newton iterations."""
    T, p, Y, hot = synth.sheet_field(h2mech, n=24, seed=9, frac=0.08)
    T, p, Y, rho, e = _inputs32(h2mech, T, p, Y)
    ctx = chem.Context(h2mech, max_cells=T.size, flags=order)
    rc, st1, T1, p1, Y1, s1 = _run(ctx, T, p, Y, rho, e, 1e-8)
    ctx.set_params(flags=order | chem.CHEM_FLAG_TWO_PASS)
    rc2, st2, T2, p2, Y2, s2 = _run(ctx, T, p, Y, rho, e, 1e-8)
    assert rc == 0 and rc2 == 0
    assert (s1 > 1 + 32).sum() > 10   # some cells outlive the probe pass
    assert np.array_equal(T1, T2) and np.array_equal(Y1, Y2) and np.array_equal(p1, p2) and np.array_equal(s1, s2)
    for k in ("nqueued", "substeps", "attempts", "newton", "nfailed"):
        assert st1[k] == st2[k], k
    ctx.close()


def test_two_pass_equals_single_pass_f64_state(h2mech):
    """The same with FP64 state arrays (chem_advance_f64): the FP64 instantiation of the
    cooperative continuation launch sizes its grid for its own register use."""
    T, p, Y, hot = synth.sheet_field(h2mech, n=16, seed=11, frac=0.08)
    T, p, Y = T.astype(np.float64), p.astype(np.float64), np.ascontiguousarray(Y, dtype=np.float64)
    rho, e = oracle.state_from_TpY(h2mech, T, p, Y)
    ctx = chem.Context(h2mech, max_cells=T.size)
    outs = []
    for flags in (chem.CHEM_FLAG_ORDER_RATE, chem.CHEM_FLAG_ORDER_RATE | chem.CHEM_FLAG_TWO_PASS):
        ctx.set_params(flags=flags)
        outs.append(_run(ctx, T, p, Y, rho, e, 1e-8))
    (rc1, st1, T1, p1, Y1, s1), (rc2, st2, T2, p2, Y2, s2) = outs
    assert rc1 == 0 and rc2 == 0 and st2["status"] == 0 and (s1 > 1 + 32).sum() > 5
    assert np.array_equal(T1, T2) and np.array_equal(Y1, Y2) and np.array_equal(s1, s2)
    ctx.close()


def test_host_entry_point_matches_device(h2mech):
    T, p, Y, hot = synth.sheet_field(h2mech, n=10, seed=8)
    T, p, Y, rho, e = _inputs32(h2mech, T, p, Y)
    n = T.size
    ctx = chem.Context(h2mech, max_cells=n)
    rc, st, Td, pd, Yd, sd = _run(ctx, T, p, Y, rho, e, 1e-8)
    Th, ph, Yh = T.copy(), p.copy(), Y.copy()
    sh = np.zeros(n, np.int32)
    args = [torch.from_numpy(a) for a in (Th, ph, Yh, rho, e)] + [torch.from_numpy(sh)]
    ctx.advance_host(args[0], args[1], args[2], args[3], args[4], 1e-8, args[5])
    assert np.array_equal(Th, Td) and np.array_equal(Yh, Yd) and np.array_equal(sh, sd)
    ctx.close()


# ---------------------------------------------------------------- full size (bench launch config)

def test_full_size_sheet_sampled(h2mech):
    """128^3 cells (the benchmark workload) in one call: sampled cells against the oracle,
    conservation properties on every cell."""
    T, p, Y, hot = synth.sheet_field(h2mech, n=128, seed=0)
    T, p, Y = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
    n = T.size
    rho, e = oracle.state_from_TpY(h2mech, T, p, Y)
    rho, e = rho.astype(np.float32), e.astype(np.float32)
    ctx = chem.Context(h2mech, max_cells=n)
    tT, tp, tY, trho, te = _dev(T, p, Y, rho, e)
    sub = torch.zeros(n, dtype=torch.int32, device=DEV)
    ctx.advance(tT, tp, tY, trho, te, 1e-8, sub)
    st = ctx.status()
    assert st["status"] == 0 and st["nqueued"] == hot.sum()
    To, Yo, so = tT.cpu().numpy(), tY.cpu().numpy(), sub.cpu().numpy()
    # every cell: mass fractions still sum to their input sum, elements conserved
    assert np.max(np.abs(Yo.astype(np.float64).sum(0) - Y.astype(np.float64).sum(0))) < 2e-6
    el0 = h2mech["elem"].T @ (Y.astype(np.float64) / h2mech["W"][:, None])
    el1 = h2mech["elem"].T @ (Yo.astype(np.float64) / h2mech["W"][:, None])
    assert np.max(np.abs(el1 - el0) / (np.abs(el0).max(0) + 1e-30)) < 2e-6
    assert np.all(so[hot] >= 2) and np.all(so[~hot] == 1)
    # sampled cells against the oracle (the oracle is given the same FP32 inputs)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(np.nonzero(hot)[0], 160, replace=False),
                          rng.choice(np.nonzero(~hot)[0], 160, replace=False)])
    T_ref, _, Y_ref, _ = oracle.advance(h2mech, rho[idx], e[idx], T[idx], Y[:, idx], 1e-8)
    cond = _conditioning(h2mech, rho[idx], e[idx], T[idx], Y[:, idx], 1e-8, T_ref, Y_ref)
    print("full-size sampled parity", _parity(To[idx], Yo[:, idx], T_ref, Y_ref, cond=cond))
    ctx.close()


def test_fp64_peak_measurement_is_plausible():
    """The FMA-chain measurement that the stiff kernel's roofline is stated against: positive, and
    within a factor of two of the unit-count figure of this part (152 SMs x 2 FP64 FMA per clock at
    up to 2.07 GHz, 1.26 TFLOP/s); repeated measurements agree to 15%."""
    a = chem.chem_measure_fp64_peak(reps=3)
    b = chem.chem_measure_fp64_peak(reps=3)
    unit = 152 * 2 * 2 * 2.07e9 / 1e12
    assert 0.5 * unit < a < 2.0 * unit
    assert abs(a - b) <= 0.15 * max(a, b)
