"""AMR box table: one persistent launch over uneven boxes, per-box dt, graph capture (GPU).

The multigrid kernel fusion of the paper (Sec. 3.2 / App. E) runs one kernel over the cells of all
grids, each cell finding its grid through an index map.  Here chem_advance_boxes advances every
registered box in one bulk launch and one persistent stiff launch; the result of each box must
equal chem_advance on that box alone (bit for bit: the per-cell arithmetic is the same), match
the oracle, and a captured CUDA graph must reproduce the direct call.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
import paper_2510_23993_gb300 as chem
import synth

DEV = "cuda:0"


def _make_boxes(mech, seed, n_boxes, edges, target):
    boxes = synth.amr_boxes(seed=seed, n_boxes=n_boxes, edges=edges, target_cells=target)
    fields = synth.helix_box_fields(mech, boxes, seed=seed, stiff_frac=0.05)
    out = []
    for bx, (T, p, Y, hot) in zip(boxes, fields):
        T, p, Y = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
        rho, e = oracle.state_from_TpY(mech, T, p, Y)
        out.append(dict(T=T, p=p, Y=Y, rho=rho.astype(np.float32), e=e.astype(np.float32), hot=hot,
                        dt=1e-8 / 2 ** bx["level"], level=bx["level"]))
    return out


def _to_dev(b):
    d = {k: torch.from_numpy(np.ascontiguousarray(b[k])).to(DEV) for k in ("T", "p", "Y", "rho", "e")}
    d["substeps"] = torch.full((b["T"].size,), -99, dtype=torch.int32, device=DEV)
    d["dt"], d["level"] = b["dt"], b["level"]
    return d


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chem.build()


def test_boxes_match_per_box_advance_oracle_and_graph(h2mech):
    boxes = _make_boxes(h2mech, seed=1, n_boxes=40, edges=(4, 8, 16), target=10 ** 9)
    total = sum(b["T"].size for b in boxes)
    ctx = chem.Context(h2mech, max_cells=total)
    dev = [_to_dev(b) for b in boxes]
    ctx.set_boxes(dev)
    ctx.advance_boxes()
    st = ctx.status()
    assert st["status"] == 0 and st["ncell"] == total
    assert st["nqueued"] == sum(int(b["hot"].sum()) for b in boxes)
    # each box alone through chem_advance gives the same bits
    for b, d in zip(boxes, dev):
        ref = _to_dev(b)
        ctx.advance(ref["T"], ref["p"], ref["Y"], ref["rho"], ref["e"], b["dt"], ref["substeps"])
        assert torch.equal(ref["T"], d["T"]) and torch.equal(ref["Y"], d["Y"])
        assert torch.equal(ref["substeps"], d["substeps"])
    # oracle on every hot cell of a few boxes of each level
    for lev in (0, 1, 2):
        pick = [k for k, b in enumerate(boxes) if b["level"] == lev and b["hot"].any()][:3]
        for k in pick:
            b, d = boxes[k], dev[k]
            idx = np.nonzero(b["hot"])[0][:40]
            T_ref, _, Y_ref, _ = oracle.advance(h2mech, b["rho"][idx], b["e"][idx], b["T"][idx], b["Y"][:, idx], b["dt"])
            To = d["T"].cpu().numpy()[idx].astype(np.float64)
            Yo = d["Y"].cpu().numpy()[:, idx].astype(np.float64)
            big = Y_ref >= 1e-6
            # conditioning allowance as in test_gpu_parity: 3x the oracle's one-ulp response of e
            e_p = b["e"][idx].astype(np.float64) * (1 + 2.0 ** -23)
            T_p, _, Y_p, _ = oracle.advance(h2mech, b["rho"][idx], e_p, b["T"][idx], b["Y"][:, idx], b["dt"])
            dY = np.where(big, np.abs(Y_p - Y_ref) / np.maximum(Y_ref, 1e-300), np.abs(Y_p - Y_ref))
            eY = np.where(big, np.abs(Yo - Y_ref) / np.maximum(Y_ref, 1e-300), np.abs(Yo - Y_ref))
            assert np.all(eY <= np.where(big, 1e-4, 1e-10) + 3 * dY)
            assert np.all(np.abs(To - T_ref) / T_ref <= 1e-4 + 3 * np.abs(T_p - T_ref) / T_ref)
    # the captured graph replays the same step
    direct = [(d["T"].clone(), d["Y"].clone()) for d in dev]
    stream = torch.cuda.Stream()
    for d, b in zip(dev, boxes):   # refill inputs in place (the graph refers to these arrays)
        d["T"].copy_(torch.from_numpy(b["T"]))
        d["Y"].copy_(torch.from_numpy(b["Y"]))
    torch.cuda.synchronize()
    ctx.capture_boxes(stream)
    for rep in range(2):
        with torch.cuda.stream(stream):
            for d, b in zip(dev, boxes):
                d["T"].copy_(torch.from_numpy(b["T"]))
                d["Y"].copy_(torch.from_numpy(b["Y"]))
        ctx.launch_boxes(stream)
        st2 = ctx.status(stream)
        assert st2["status"] == 0 and st2["nqueued"] == st["nqueued"]
        for (T1, Y1), d in zip(direct, dev):
            assert torch.equal(T1, d["T"]) and torch.equal(Y1, d["Y"])
    # the two-pass schedule (probe launch, then a cooperative launch of continuation rounds) in a
    # captured graph gives the same bits
    ctx.set_params(flags=ctx.params.flags | chem.CHEM_FLAG_TWO_PASS)
    with torch.cuda.stream(stream):
        for d, b in zip(dev, boxes):
            d["T"].copy_(torch.from_numpy(b["T"]))
            d["Y"].copy_(torch.from_numpy(b["Y"]))
    torch.cuda.synchronize()
    ctx.capture_boxes(stream)
    with torch.cuda.stream(stream):
        for d, b in zip(dev, boxes):
            d["T"].copy_(torch.from_numpy(b["T"]))
            d["Y"].copy_(torch.from_numpy(b["Y"]))
    ctx.launch_boxes(stream)
    st3 = ctx.status(stream)
    assert st3["status"] == 0 and st3["nqueued"] == st["nqueued"] and st3["attempts"] == st["attempts"]
    for (T1, Y1), d in zip(direct, dev):
        assert torch.equal(T1, d["T"]) and torch.equal(Y1, d["Y"])
    ctx.close()


def test_full_size_400_boxes_sampled(h2mech):
    """400 boxes over 3 levels (edges 8-64, ~8.1M cells, 3% stiff), one launch pair; sampled oracle."""
    boxes = synth.amr_boxes(seed=0)
    fields = synth.helix_box_fields(h2mech, boxes, seed=0, stiff_frac=0.03)
    dev, host = [], []
    for bx, (T, p, Y, hot) in zip(boxes, fields):
        d = {"T": torch.from_numpy(T.astype(np.float32)).to(DEV), "p": torch.from_numpy(p.astype(np.float32)).to(DEV),
             "Y": torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).to(DEV)}
        d["rho"], d["e"] = torch.empty_like(d["T"]), torch.empty_like(d["T"])
        d["substeps"] = torch.zeros(T.size, dtype=torch.int32, device=DEV)
        d["dt"], d["level"] = 1e-8 / 2 ** bx["level"], bx["level"]
        dev.append(d)
        host.append((T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32), hot))
    total = sum(h[0].size for h in host)
    ctx = chem.Context(h2mech, max_cells=total)
    rng = np.random.default_rng(0)
    samples = []
    for k, (d, (T, p, Y, hot)) in enumerate(zip(dev, host)):
        rho, e = oracle.state_from_TpY(h2mech, T, p, Y)
        d["rho"].copy_(torch.from_numpy(rho.astype(np.float32)))
        d["e"].copy_(torch.from_numpy(e.astype(np.float32)))
        if hot.any() and len(samples) < 60:
            samples.append((k, int(rng.choice(np.nonzero(hot)[0]))))
    ctx.set_boxes(dev)
    ctx.advance_boxes()
    st = ctx.status()
    assert st["status"] == 0 and st["ncell"] == total
    assert st["nqueued"] == sum(int(h[3].sum()) for h in host)
    for k, i in samples:
        T, p, Y, hot = host[k]
        rho, e = oracle.state_from_TpY(h2mech, T[[i]], p[[i]], Y[:, [i]])
        rho, e = rho.astype(np.float32), e.astype(np.float32)
        T_ref, _, Y_ref, _ = oracle.advance(h2mech, rho, e, T[[i]], Y[:, [i]], dev[k]["dt"])
        To = float(dev[k]["T"][i].item())
        Yo = dev[k]["Y"][:, i].cpu().numpy().astype(np.float64)
        big = Y_ref[:, 0] >= 1e-6
        e_p = e.astype(np.float64) * (1 + 2.0 ** -23)
        T_p, _, Y_p, _ = oracle.advance(h2mech, rho, e_p, T[[i]], Y[:, [i]], dev[k]["dt"])
        dY = np.where(big, np.abs(Y_p[:, 0] - Y_ref[:, 0]) / np.maximum(Y_ref[:, 0], 1e-300), np.abs(Y_p[:, 0] - Y_ref[:, 0]))
        eY = np.where(big, np.abs(Yo - Y_ref[:, 0]) / np.maximum(Y_ref[:, 0], 1e-300), np.abs(Yo - Y_ref[:, 0]))
        assert np.all(eY <= np.where(big, 1e-4, 1e-10) + 3 * dY)
        assert abs(To - T_ref[0]) / T_ref[0] <= 1e-4 + 3 * abs(T_p[0] - T_ref[0]) / T_ref[0]
    ctx.close()


def test_two_pass_with_4000_boxes(h2mech):
    """4000 small boxes: their offsets take 16 KB of shared memory per CTA, so fewer CTAs fit an
    SM; the cooperative continuation launch still runs (its grid is capped at what fits) and
    gives the bits of the single-pass schedule."""
    rng = np.random.default_rng(4)
    T, p, Y, hot = synth.sheet_field(h2mech, n=20, seed=12, frac=0.08)
    T, p, Y = T.astype(np.float32), p.astype(np.float32), np.ascontiguousarray(Y, dtype=np.float32)
    rho, e = oracle.state_from_TpY(h2mech, T, p, Y)
    n = T.size
    cuts = np.sort(rng.choice(np.arange(1, n), 3999, replace=False))
    off = np.concatenate([[0], cuts, [n]])
    res = []
    for flags in (chem.CHEM_FLAG_ORDER_RATE, chem.CHEM_FLAG_ORDER_RATE | chem.CHEM_FLAG_TWO_PASS):
        ctx = chem.Context(h2mech, max_cells=n, flags=flags)
        tT, tp, tY, trho, te = (torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
                                for a in (T, p, Y, rho.astype(np.float32), e.astype(np.float32)))
        sub = torch.zeros(n, dtype=torch.int32, device=DEV)
        boxes = [dict(T=tT[a:b], p=tp[a:b], Y=tY[:, a:b], rho=trho[a:b], e=te[a:b], substeps=sub[a:b], dt=1e-8,
                      level=0) for a, b in zip(off[:-1], off[1:])]
        ctx.set_boxes(boxes)
        ctx.advance_boxes()
        st = ctx.status()
        assert st["status"] == 0 and st["ncell"] == n
        res.append((tT.cpu().numpy(), tY.cpu().numpy(), sub.cpu().numpy()))
        ctx.close()
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)
