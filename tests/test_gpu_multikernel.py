"""The multi-kernel cuBLAS baseline of the rate evaluation (chem_mk_rates, Sec. 3.2.1 / App. C)
against the FP64 oracle and against the fused kernel (chem_rates), for the 9- and the 53-species
mechanisms.

Bar (FP32 log-form kinetics, as for chem_rates): |f - f_ref| <= 1e-4 |f_ref| + 2e-5 s_k with
s_k = W_k / rho sum_r |dnu_kr| (q_f + q_r), the FP32 cancellation floor of the gross rates.
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


def _states(mech, n, seed):
    rng = np.random.default_rng(seed)
    T = rng.uniform(800, 3000, n)
    p = rng.uniform(1, 20, n) * synth.P_ATM
    Y = rng.dirichlet(np.full(mech["ns"], 0.3), size=n).T
    Y[2:4, :5] = 0.0                     # absent species (ln C floor) in a few cells
    Y /= Y.sum(0)
    T32, p32, Y32 = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
    rho, _ = oracle.state_from_TpY(mech, T32, p32, Y32)
    return T32, Y32, rho.astype(np.float32)


def _bar(mech, rho, T, Y):
    ref, qf, qr = oracle.rates(mech, rho, T, Y, with_progress=True)
    dnu = (mech["nu_r"] - mech["nu_f"]).astype(np.float64)
    gross = mech["W"][:, None] / rho.astype(np.float64)[None, :] * (np.abs(dnu).T @ (qf + qr))
    return ref, 1e-4 * np.abs(ref) + 2e-5 * gross


@pytest.mark.parametrize("which", ["h2", "hc"])
def test_multikernel_rates_parity(which):
    mech = synth.h2_air_mechanism(0) if which == "h2" else synth.hydrocarbon_mechanism(0)
    ns = mech["ns"]
    n, ld = 1037, 1100                    # ragged against every block size; padded leading dimension
    T, Y, rho = _states(mech, n, 5)
    ref, bar = _bar(mech, rho, T, Y)
    mk = chem.MultiKernelRates(mech, max_cells=n)
    tT, trho = (torch.from_numpy(a).to(DEV) for a in (T, rho))
    tY = torch.zeros((ns, ld), dtype=torch.float32, device=DEV)
    tY[:, :n] = torch.from_numpy(Y).to(DEV)
    f = torch.full((ns, ld), -7.0, dtype=torch.float32, device=DEV)
    mk.rates(trho, tT, tY, f, n=n)
    torch.cuda.synchronize()
    fo = f.cpu().numpy()
    assert np.all(fo[:, n:] == -7.0)      # the padding is not written
    g = fo[:, :n].astype(np.float64)
    bad = np.abs(g - ref) > bar
    assert not bad.any(), (np.abs(g - ref)[bad].max(), np.nonzero(bad))
    # the fused kernel on the same inputs meets the same bar, so the two agree within twice it
    ctx = chem.Context(mech, max_cells=n)
    f2 = torch.empty((ns, n), dtype=torch.float32, device=DEV)
    ctx.rates(trho, tT, tY[:, :n].contiguous(), f2)
    assert np.all(np.abs(f2.cpu().numpy().astype(np.float64) - g) <= 2 * bar)
    ctx.close()
    # edge cases: nothing to do, and more cells than the scratch holds
    mk.rates(trho, tT, tY, f, n=0)
    with pytest.raises(chem.ChemError):
        mk.rates(trho, tT, tY, f, n=n + 1)
    mk.close()
