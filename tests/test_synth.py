"""The seeded input generators draw what their recipes state (no GPU)."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("make", [synth.h2_air_mechanism, synth.hydrocarbon_mechanism])
def test_mechanism_shape_and_balance(make):
    m = make(0)
    ns, nr = m["ns"], m["nr"]
    assert (ns, nr) == ((9, 21) if make is synth.h2_air_mechanism else (53, 325))
    dnu = m["nu_r"].astype(int) - m["nu_f"]
    assert np.all(dnu @ m["elem"] == 0)                      # element balance
    assert np.all((m["nu_f"] > 0) & (m["nu_r"] > 0) == False)  # no species on both sides
    assert m["nu_f"].max() <= 2 and m["nu_r"].max() <= 2
    assert np.all(m["nu_f"][:, m["inert"]] == 0) and np.all(m["nu_r"][:, m["inert"]] == 0)
    per_side = np.maximum(m["nu_f"].sum(1), m["nu_r"].sum(1))
    assert per_side.max() <= 3 and np.all(per_side[m["third_body"] == 1] <= 2)
    assert np.all((m["A_cgs"] >= 1e6) & (m["A_cgs"] <= 1e16))
    assert np.all((m["b"] >= -1.5) & (m["b"] <= 2.0)) and np.all((m["Ea"] >= 0) & (m["Ea"] <= 2e5))
    assert int(m["third_body"].sum()) == (4 if ns == 9 else 30)
    eff = m["eff"][m["third_body"] == 1]
    assert np.all((eff >= 0.5) & (eff <= 12.0))
    # cp/R within [1.5, 12] on [300, 3500] K
    T = np.linspace(300.0, 3500.0, 200)
    a = m["thermo"]
    cp = a[:, 0:1] + a[:, 1:2] * T + a[:, 2:3] * T**2 + a[:, 3:4] * T**3 + a[:, 4:5] * T**4
    assert cp.min() >= 1.5 and cp.max() <= 12.0


def test_reactions_written_exothermic(h2mech):
    """h(300 K) of products <= reactants for every reaction (the generator's orientation)."""
    a, T = h2mech["thermo"], 300.0
    h = a[:, 0] * T + a[:, 1] * T**2 / 2 + a[:, 2] * T**3 / 3 + a[:, 3] * T**4 / 4 + a[:, 4] * T**5 / 5 + a[:, 5]
    dnu = h2mech["nu_r"].astype(float) - h2mech["nu_f"]
    assert np.all(dnu @ h <= 1e-9)


def test_mechanism_is_seeded():
    a, b = synth.h2_air_mechanism(3), synth.h2_air_mechanism(3)
    c = synth.h2_air_mechanism(4)
    assert all(np.array_equal(a[k], b[k]) for k in ("nu_f", "A", "thermo"))
    assert not np.array_equal(a["A"], c["A"])


def test_slab_and_sheet_fields(h2mech):
    T, p, Y, hot = synth.slab_field(h2mech)
    assert T.shape == (4096,) and Y.shape == (9, 4096) and hot.sum() == 512
    assert np.all(T[hot] == 2500.0) and np.all(T[~hot] == 300.0)
    assert np.allclose(Y.sum(0), 1.0)
    T, p, Y, hot = synth.sheet_field(h2mech, n=32, seed=0)
    assert hot.sum() == round(0.05 * 32 ** 3)
    assert T[hot].min() >= 1500 and T[hot].max() <= 3000 and T[~hot].max() <= 400
    assert np.allclose(Y.sum(0), 1.0) and Y.min() >= 0


def test_amr_boxes():
    boxes = synth.amr_boxes(seed=0)
    assert len(boxes) == 400
    assert {b["level"] for b in boxes} == {0, 1, 2}
    total = sum(b["nx"] * b["ny"] * b["nz"] for b in boxes)
    assert 7_000_000 < total < 8_300_000
    assert all(b[k] in (4, 8, 16, 32, 64) for b in boxes for k in ("nx", "ny", "nz"))


def test_stratified_sample_keeps_fraction(h2mech):
    T, p, Y, hot = synth.sheet_field(h2mech, n=32, seed=0)
    idx = synth.stratified_sample(hot, 4096, seed=0)
    assert len(np.unique(idx)) == 4096
    assert abs(hot[idx].mean() - hot.mean()) < 2.0 / 4096
