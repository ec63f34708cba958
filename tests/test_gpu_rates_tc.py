"""chem_rates_tc: the 53-species rates with the stoichiometric contractions on the tensor cores (GPU).

Same parity bar as the warp-per-cell rates of test_gpu_large.py (relative 1e-4 of the net rate,
or a few FP32 ulps of the gross rate): against the FP64 oracle at sizes that span several
128-cell tiles and a ragged tail, on a strided sample of a 1,048,576-cell batch (the size the rate
study times), below, above and across the thermo fit range (the per-regime reaction records), on
cells whose rates of progress leave the FP32 range (the FP64 fallback), with a leading
dimension larger than the cell count, and on degenerate inputs (no cells, one cell, species at
exactly zero).  Also: results are deterministic, and a 9-species context reports the call as
unsupported.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
import paper_2510_23993_gb300 as chem
import synth

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chem.build()


def _state(mech, n, seed, zero_frac=0.0):
    rng = np.random.default_rng(seed)
    T = rng.uniform(300, 3000, n)
    p = rng.uniform(0.1, 50, n) * synth.P_ATM
    Y = rng.dirichlet(np.full(mech["ns"], 0.3), size=n).T
    if zero_frac:
        Y[rng.random(Y.shape) < zero_frac] = 0.0
        Y /= Y.sum(0, keepdims=True)
    T32, Y32 = T.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
    rho, _ = oracle.state_from_TpY(mech, T32, p.astype(np.float32), Y32)
    return T32, Y32, rho.astype(np.float32)


def _bar(mech, rho, T, Y, f):
    """True where f meets the FP32 rate bar against the oracle."""
    ref, qf, qr = oracle.rates(mech, rho, T, Y, with_progress=True)
    dnu = (mech["nu_r"] - mech["nu_f"]).astype(np.float64)
    gross = mech["W"][:, None] / rho.astype(np.float64)[None, :] * (np.abs(dnu).T @ (qf + qr))
    return np.abs(f.astype(np.float64) - ref) <= 1e-4 * np.abs(ref) + 2e-5 * gross


def _run(ctx, rho, T, Y):
    tT, tY, trho = (torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (T, Y, rho))
    f = torch.full_like(tY, float("nan"))
    ctx.rates_tc(trho, tT, tY, f)
    torch.cuda.synchronize()
    assert ctx.status()["status"] == 0
    return f.cpu().numpy()


@pytest.mark.parametrize("n", [1, 127, 128, 129, 500, 1000])
def test_rates_tc_parity(hcmech, n):
    T, Y, rho = _state(hcmech, n, seed=n, zero_frac=0.1)
    ctx = chem.Context(hcmech, max_cells=n)
    f = _run(ctx, rho, T, Y)
    assert np.all(np.isfinite(f))
    assert np.all(_bar(hcmech, rho, T, Y, f))
    ctx.close()


@pytest.mark.parametrize("T_lo,T_hi", [(150.0, 299.0), (3600.0, 5500.0), (250.0, 4000.0)])
def test_rates_tc_thermo_regimes(hcmech, T_lo, T_hi):
    """Below, above and across the thermo fit range [300, 3500] K: the kernel takes the reaction
    records of each cell's regime (cp frozen outside the range, h and s continuous)."""
    n = 640
    rng = np.random.default_rng(int(T_lo))
    T = rng.uniform(T_lo, T_hi, n).astype(np.float32)
    p = (rng.uniform(0.5, 20, n) * synth.P_ATM).astype(np.float32)
    Y = np.ascontiguousarray(rng.dirichlet(np.full(hcmech["ns"], 0.3), size=n).T, dtype=np.float32)
    rho, _ = oracle.state_from_TpY(hcmech, T, p, Y)
    rho = rho.astype(np.float32)
    ctx = chem.Context(hcmech, max_cells=n)
    f = _run(ctx, rho, T, Y)
    assert np.all(np.isfinite(f))
    assert np.all(_bar(hcmech, rho, T, Y, f))
    ctx.close()


def test_rates_tc_matches_warp_kernel_bar(hcmech):
    """Both rate kernels meet the same bar on the same cells (and agree to it with each other)."""
    n = 2000
    T, Y, rho = _state(hcmech, n, seed=11)
    ctx = chem.Context(hcmech, max_cells=n)
    f_tc = _run(ctx, rho, T, Y)
    tT, tY, trho = (torch.from_numpy(a).to(DEV) for a in (T, Y, rho))
    f_w = torch.empty_like(tY)
    ctx.rates(trho, tT, tY, f_w)
    f_w = f_w.cpu().numpy()
    assert np.all(_bar(hcmech, rho, T, Y, f_tc)) and np.all(_bar(hcmech, rho, T, Y, f_w))
    ctx.close()


def test_rates_tc_fp64_fallback(hcmech):
    """Cells with a rate of progress beyond the FP32 range take the FP64 rates of progress."""
    n = 4096
    T, Y, rho = _state(hcmech, n, seed=5)
    rho = rho * np.float32(1e10)         # C = rho Y / W up 1e10: about half the cells pass e^87.5
    _, qf, qr = oracle.rates(hcmech, rho, T, Y, with_progress=True)
    lnq = np.log(np.maximum(np.maximum(qf, qr), 1e-300)).max(0)
    ref = oracle.rates(hcmech, rho, T, Y)
    keep = (lnq > 87.5) & (np.abs(ref).max(0) < 1e36)
    assert keep.sum() >= 16, "the recipe must produce cells beyond the FP32 exp range"
    T, Y, rho = T[keep], np.ascontiguousarray(Y[:, keep]), rho[keep]
    ctx = chem.Context(hcmech, max_cells=T.size)
    f = _run(ctx, rho, T, Y)
    assert np.all(np.isfinite(f))
    assert np.all(_bar(hcmech, rho, T, Y, f))
    ctx.close()


def test_rates_tc_leading_dimension(hcmech):
    n, ld = 300, 384
    T, Y, rho = _state(hcmech, n, seed=8)
    ctx = chem.Context(hcmech, max_cells=n)
    tT, trho = torch.from_numpy(T).to(DEV), torch.from_numpy(rho).to(DEV)
    tY = torch.zeros(hcmech["ns"], ld, device=DEV)
    tY[:, :n] = torch.from_numpy(Y).to(DEV)
    f = torch.full((hcmech["ns"], ld), 7.0, device=DEV)
    assert chem.chem_rates_tc(ctx.handle, trho, tT, tY, ld, n, f) == 0
    torch.cuda.synchronize()
    f = f.cpu().numpy()
    assert np.all(f[:, n:] == 7.0)                       # nothing written past n
    assert np.all(_bar(hcmech, rho, T, Y, f[:, :n]))
    ctx.close()


def test_rates_tc_full_size_sampled(hcmech):
    """1,048,576 cells in one call (the launch the rate study times); a strided sample of 4,096
    cells checked against the oracle, and a second call bit-identical to the first."""
    n = 1 << 20
    T, Y, rho = _state(hcmech, n, seed=21, zero_frac=0.05)
    ctx = chem.Context(hcmech, max_cells=n)
    tT, tY, trho = (torch.from_numpy(a).to(DEV) for a in (T, Y, rho))
    f1, f2 = torch.empty_like(tY), torch.empty_like(tY)
    ctx.rates_tc(trho, tT, tY, f1)
    ctx.rates_tc(trho, tT, tY, f2)
    torch.cuda.synchronize()
    assert ctx.status()["status"] == 0
    assert torch.equal(f1, f2)
    idx = np.arange(n)[::256]
    idx[-1] = n - 1                                      # the batch's last cell
    f = f1[:, torch.from_numpy(idx).to(DEV)].cpu().numpy()
    assert np.all(_bar(hcmech, rho[idx], T[idx], np.ascontiguousarray(Y[:, idx]), f))
    ctx.close()


def test_rates_tc_empty_and_unsupported(hcmech, h2mech):
    ctx = chem.Context(hcmech, max_cells=4)
    z = torch.empty(0, device=DEV)
    assert chem.chem_rates_tc(ctx.handle, z, z, torch.empty(hcmech["ns"], 0, device=DEV), 0, 0,
                              torch.empty(hcmech["ns"], 0, device=DEV)) == 0
    ctx.close()
    small = chem.Context(h2mech, max_cells=4)
    t = torch.ones(4, device=DEV)
    Y = torch.full((h2mech["ns"], 4), 1.0 / h2mech["ns"], device=DEV)
    with pytest.raises(chem.ChemError) as e:
        small.rates_tc(t, t * 1000.0, Y, torch.empty_like(Y))
    assert e.value.code == chem.CHEM_EUNSUPPORTED
    small.close()
