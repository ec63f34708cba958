"""chem_advance_noalloc gives the results of chem_advance without allocating anything.

The entry point serves callers that cannot call cudaMalloc (real-time loops that may not block on
the allocator, plugins restricted to the buffers they are handed, capped allocators): its
mechanism tables and scratch live in fixed-size device arrays of the library.  Two calls in a row,
on two different fields, must give chem_advance's results bit for bit (same packed tables, same
kernels, and a cell's result does not depend on its queue slot), which also keeps them within the
parity tolerances of the other GPU tests; the counters of the second call must not carry anything
over from the first.  The file name makes pytest collect it last.
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


def _field(mech, seed):
    T, p, Y, hot = synth.sheet_field(mech, n=16, seed=seed)
    T, p, Y = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
    rho, e = oracle.state_from_TpY(mech, T, p, Y)
    return T, p, Y, rho.astype(np.float32), e.astype(np.float32), hot


def _tensors(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in arrs]


def test_noalloc_matches_chem_advance_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chem.build()
    mech = synth.h2_air_mechanism(0)
    cmech = chem.Mechanism(mech)
    params = chem.chem_default_params()
    dt = 1e-8
    for seed in (5, 6):
        T, p, Y, rho, e, hot = _field(mech, seed)
        n = T.size
        # the existing entry point
        ctx = chem.Context(mech, max_cells=n)
        rT, rp, rY, rrho, re = _tensors(T, p, Y, rho, e)
        rsub = torch.zeros(n, dtype=torch.int32, device=DEV)
        ctx.advance(rT, rp, rY, rrho, re, dt, rsub)
        ref_stats = ctx.status()
        ctx.close()
        # the entry point without allocation
        aT, ap, aY, arho, ae = _tensors(T, p, Y, rho, e)
        asub = torch.full((n,), -99, dtype=torch.int32, device=DEV)
        stats = chem.chem_stats()
        rc = chem.chem_advance_noalloc(cmech, params, aT, ap, aY, aY.stride(0), arho, ae, n, dt, asub, stats)
        assert rc == chem.CHEM_OK, chem.chem_strerror(rc)
        assert stats.status == chem.CHEM_OK
        assert stats.nqueued == int(hot.sum()) == ref_stats["nqueued"]
        assert stats.nbulk == ref_stats["nbulk"] and stats.ncell == n
        Tr, Yr = rT.cpu().numpy().astype(np.float64), rY.cpu().numpy().astype(np.float64)
        Ta, Ya = aT.cpu().numpy().astype(np.float64), aY.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(Ta - Tr) / Tr) <= TOL_T
        big = Yr >= Y_BIG
        assert np.max(np.abs(Ya[big] - Yr[big]) / Yr[big]) <= TOL_Y
        assert np.max(np.abs(Ya[~big] - Yr[~big]), initial=0.0) <= ABS_Y
        # both entry points pack the tables with the same host code and run the same kernels, and
        # a cell's integration does not depend on its queue slot: same bits, same substep counts
        assert np.array_equal(aT.cpu().numpy(), rT.cpu().numpy())
        assert np.array_equal(aY.cpu().numpy(), rY.cpu().numpy())
        assert np.array_equal(ap.cpu().numpy(), rp.cpu().numpy())
        assert np.array_equal(asub.cpu().numpy(), rsub.cpu().numpy())
        for k in ("substeps", "attempts", "newton", "nfailed"):
            assert getattr(stats, k) == ref_stats[k], k


def test_noalloc_rejects_more_cells_than_its_static_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chem.build()
    mech = chem.Mechanism(synth.h2_air_mechanism(0))
    t = torch.zeros(16, dtype=torch.float32, device=DEV)
    s = torch.zeros(16, dtype=torch.int32, device=DEV)
    n = (1 << 21) + 1   # rejected on the host before any device access
    rc = chem.chem_advance_noalloc(mech, None, t, t, t, n, t, t, n, 1e-8, s)
    assert rc == chem.CHEM_ENOMEM
