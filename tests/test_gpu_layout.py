"""The state load under the three storage layouts of chem_pressure_layout (Sec. 3.1 / Algorithm 1):
every layout gives the same bits (same arithmetic, same order) and matches the FP64 ideal-gas
pressure to FP32 rounding (ns + 3 roundings: relative 1e-5); ragged cell counts; bad arguments."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2510_23993_gb300 as chem
import synth

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chem.build()


@pytest.mark.parametrize("which", ["h2", "hc"])
def test_layouts_agree_and_match_ideal_gas(which):
    mech = synth.h2_air_mechanism(0) if which == "h2" else synth.hydrocarbon_mechanism(0)
    ns, W = mech["ns"], mech["W"]
    nv = ns + 2
    rng = np.random.default_rng(3)
    out = {}
    for n in (1, 37, 1000, 4133):
        rec = np.empty((nv, n), np.float32)                  # component-major record
        rec[0] = rng.uniform(0.05, 20.0, n)
        rec[1] = rng.uniform(300.0, 3000.0, n)
        rec[2:] = rng.dirichlet(np.full(ns, 0.5), size=n).T
        ref = rec[0].astype(np.float64) * 8.314462618 * rec[1] * (rec[2:].astype(np.float64).T @ (1.0 / W))
        ld = n + 5
        soa = np.zeros((nv, ld), np.float32)
        soa[:, :n] = rec
        aos = np.ascontiguousarray(rec.T)
        tiles = (n + 31) // 32
        aosoa = np.zeros((tiles, nv, 32), np.float32)
        pad = np.zeros((nv, tiles * 32), np.float32)
        pad[:, :n] = rec
        aosoa[:] = pad.reshape(nv, tiles, 32).transpose(1, 0, 2)
        res = {}
        for layout, arr, lda in ((chem.CHEM_LAYOUT_SOA, soa, ld), (chem.CHEM_LAYOUT_AOS, aos, 0),
                                 (chem.CHEM_LAYOUT_AOSOA, aosoa, 0), (chem.CHEM_LAYOUT_AOS_STAGED, aos, 0)):
            X = torch.from_numpy(np.ascontiguousarray(arr)).to(DEV)
            p = torch.full((n + 3,), -1.0, dtype=torch.float32, device=DEV)
            chem.pressure_layout(W, layout, X, n, p, ld=lda)
            torch.cuda.synchronize()
            po = p.cpu().numpy()
            assert np.all(po[n:] == -1.0)
            res[layout] = po[:n]
        for layout in res:
            assert np.array_equal(res[layout], res[chem.CHEM_LAYOUT_SOA]), (n, layout)
        assert np.allclose(res[chem.CHEM_LAYOUT_SOA], ref, rtol=1e-5, atol=0)
        out[n] = res
    # bad arguments
    X = torch.zeros(64 * nv + 1, dtype=torch.float32, device=DEV)
    p = torch.zeros(64, dtype=torch.float32, device=DEV)
    with pytest.raises(chem.ChemError):
        chem.pressure_layout(W, 7, X, 64, p)
    with pytest.raises(chem.ChemError):
        chem.pressure_layout(W, chem.CHEM_LAYOUT_AOS_STAGED, X[1:], 64, p)   # not 16-byte aligned
    with pytest.raises(chem.ChemError):
        chem.pressure_layout(W, chem.CHEM_LAYOUT_SOA, X, 64, p, ld=10)
