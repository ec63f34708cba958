"""Seeded synthetic cell fields (T, p, Y) in structure-of-arrays layout.

Every function returns T [n], p [n] (Pa) and Y [ns, n] as float64 arrays; the caller casts
to the precision of the path under test.  Density and internal energy are NOT produced
here: they follow from (T, p, Y) through the thermochemistry, which both the oracle and
the library compute on their own.

Recipes (the paper's detonation and jet-in-crossflow states are not available; these
synthetic fields take the shapes the workloads describe):
  * premix: fuel : oxidizer : inert = 2 : 1 : 3.76 by moles (stoichiometric H2-air shape);
  * slab: a 16^3 grid of premix at 300 K / 1 atm, with the planes z = 7, 8 at 2500 K / 20 atm;
  * sheet: an n^3 grid; the `frac` of cells nearest to a seeded sinusoidally perturbed plane
    carry T ~ U[1500, 3000] K, Y ~ Dirichlet(0.5) over all species, p ~ U[1, 20] atm; the
    rest are premix with T ~ U[300, 400] K at 1 atm;
  * AMR boxes: seeded box sizes (edges from {8, 16, 32, 64}), 3 levels, reacting shear-layer
    states near a seeded helix.
"""
import numpy as np

from .mechanism import P_ATM


def premix_mass_fractions(mech):
    x = np.zeros(mech["ns"])
    x[mech["fuel"]] = 2.0
    x[mech["oxidizer"]] = 1.0
    x[mech["inert"]] = 3.76
    y = x * mech["W"]
    return y / y.sum()


def slab_field(mech, n=16, slab=(7, 8), T_cold=300.0, p_cold=P_ATM, T_hot=2500.0, p_hot=20 * P_ATM):
    """n^3 premix with a hot planar slab (cells with z in `slab`); cell index = x + n (y + n z)."""
    N = n ** 3
    z = np.arange(N) // (n * n)
    hot = np.isin(z, slab)
    T = np.where(hot, T_hot, T_cold).astype(np.float64)
    p = np.where(hot, p_hot, p_cold).astype(np.float64)
    Y = np.repeat(premix_mass_fractions(mech)[:, None], N, axis=1)
    return T, p, Y, hot


def sheet_field(mech, n=128, frac=0.05, seed=0, alpha=0.5, nx=None, ny=None, nz=None):
    """Curved reacting sheet in an nx*ny*nz grid (default n^3); returns T, p, Y, hot mask."""
    nx = nx or n
    ny = ny or n
    nz = nz or n
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    idx = np.arange(N)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    kx, ky = rng.integers(1, 4, size=2)
    ax, ay = rng.uniform(0.05, 0.15, size=2) * nz
    px, py = rng.uniform(0, 2 * np.pi, size=2)
    z0 = 0.5 * nz + ax * np.sin(2 * np.pi * kx * x / nx + px) + ay * np.sin(2 * np.pi * ky * y / ny + py)
    dist = np.abs(z + 0.5 - z0)
    n_hot = int(round(frac * N))
    hot = np.zeros(N, dtype=bool)
    if n_hot > 0:
        hot[np.argpartition(dist, n_hot - 1)[:n_hot]] = True
    ns = mech["ns"]
    T = rng.uniform(300.0, 400.0, size=N)
    p = np.full(N, P_ATM)
    Y = np.repeat(premix_mass_fractions(mech)[:, None], N, axis=1)
    nh = int(hot.sum())
    T[hot] = rng.uniform(1500.0, 3000.0, size=nh)
    p[hot] = rng.uniform(1.0, 20.0, size=nh) * P_ATM
    Y[:, hot] = rng.dirichlet(np.full(ns, alpha), size=nh).T
    return T, p, Y, hot


def stratified_sample(hot, n_sample, seed=0, hot_frac=None):
    """Seeded subsample of cell indices keeping the hot fraction of the full field (or hot_frac)."""
    rng = np.random.default_rng(seed + 7919)
    hot_idx = np.nonzero(hot)[0]
    cold_idx = np.nonzero(~hot)[0]
    frac = len(hot_idx) / max(1, len(hot)) if hot_frac is None else hot_frac
    n_hot = int(round(n_sample * frac))
    n_hot = min(n_hot, len(hot_idx))
    n_cold = min(n_sample - n_hot, len(cold_idx))
    pick = np.concatenate([rng.choice(hot_idx, n_hot, replace=False),
                           rng.choice(cold_idx, n_cold, replace=False)])
    return np.sort(pick)


def amr_boxes(seed=0, n_boxes=400, levels=3, edges=(8, 16, 32, 64), target_cells=8_000_000):
    """Box table of an uneven 3-level AMR hierarchy: list of dicts (nx, ny, nz, level, origin).

    Edges are drawn per axis from `edges`; boxes are drawn level by level (more boxes on finer
    levels), then edges of the largest boxes are halved until the total is near target_cells."""
    rng = np.random.default_rng(seed)
    lv = np.sort(rng.integers(0, levels, size=n_boxes))
    dims = rng.choice(edges, size=(n_boxes, 3))
    total = int(np.prod(dims, axis=1).sum())
    # trim: halve the largest edge of the largest box until the total is within 2% of the target
    while total > target_cells * 1.02:
        b = int(np.argmax(np.prod(dims, axis=1)))
        a = int(np.argmax(dims[b]))
        if dims[b, a] <= min(edges):
            break
        dims[b, a] //= 2
        total = int(np.prod(dims, axis=1).sum())
    origins = rng.uniform(0.0, 1.0, size=(n_boxes, 3))
    return [dict(nx=int(d[0]), ny=int(d[1]), nz=int(d[2]), level=int(l), origin=o)
            for d, l, o in zip(dims, lv, origins)]


def helix_box_fields(mech, boxes, seed=0, stiff_frac=0.03, alpha=0.5):
    """Reacting shear layer on a seeded helix, sampled in each AMR box.

    Each box spans a cube of side 0.25 / 2^level placed at its origin in the unit domain.
    Cells within a thickness chosen so that `stiff_frac` of all cells lie in the layer get
    mixture fraction Z ~ U[0, 1] between fuel and air, T ~ U[1500, 3000] K and radicals from
    a Dirichlet(alpha); the rest are cold air (above the helix axis) or cold fuel (below).
    Returns a list of (T, p, Y, hot) per box."""
    rng = np.random.default_rng(seed + 104729)
    Rh, c, phase = rng.uniform(0.2, 0.35), rng.uniform(0.08, 0.15), rng.uniform(0, 2 * np.pi)
    ns = mech["ns"]
    pm = premix_mass_fractions(mech)
    air = np.zeros(ns)
    air[mech["oxidizer"]], air[mech["inert"]] = 1.0, 3.76
    air *= mech["W"]
    air /= air.sum()
    fuel = np.zeros(ns)
    fuel[mech["fuel"]] = 1.0
    dists, coords = [], []
    for bx in boxes:
        side = 0.25 / 2 ** bx["level"]
        n = bx["nx"] * bx["ny"] * bx["nz"]
        i = np.arange(n)
        ix, iy, iz = i % bx["nx"], (i // bx["nx"]) % bx["ny"], i // (bx["nx"] * bx["ny"])
        h = side / max(bx["nx"], bx["ny"], bx["nz"])
        px = bx["origin"][0] * 0.75 + (ix + 0.5) * h
        py = bx["origin"][1] * 0.75 + (iy + 0.5) * h
        pz = bx["origin"][2] * 0.75 + (iz + 0.5) * h
        # distance to the helix (R cos s, R sin s, c s) around the domain centre, sampled in s
        s = (pz - 0.5) / c + phase
        dx, dy = px - 0.5 - Rh * np.cos(s), py - 0.5 - Rh * np.sin(s)
        dists.append(np.hypot(dx, dy))
        coords.append(py)
    alld = np.concatenate(dists)
    delta = np.quantile(alld, stiff_frac) if stiff_frac > 0 else -1.0
    out = []
    for d, py in zip(dists, coords):
        n = len(d)
        hot = d <= delta
        T = rng.uniform(300.0, 400.0, size=n)
        p = np.full(n, P_ATM)
        Y = np.where((py > 0.5)[None, :], air[:, None], fuel[:, None]).astype(np.float64)
        nh = int(hot.sum())
        if nh:
            Z = rng.uniform(0.0, 1.0, size=nh)
            mix = Z[None, :] * fuel[:, None] + (1 - Z[None, :]) * air[:, None]
            rad = rng.dirichlet(np.full(ns, alpha), size=nh).T
            w = rng.uniform(0.1, 0.5, size=nh)
            Y[:, hot] = (1 - w) * mix + w * rad
            T[hot] = rng.uniform(1500.0, 3000.0, size=nh)
            p[hot] = rng.uniform(1.0, 20.0, size=nh) * P_ATM
        out.append((T, p, Y, hot))
    return out


def surrogate_samples(mech, n, seed=0, alpha=0.5, T_range=(300.0, 3200.0), p_atm=(1.0, 50.0),
                      log_dt=(np.log(1e-9), np.log(1e-6)), premix_frac=0.0, kappa=200.0, alpha_trace=1e-3,
                      mixing_frac=0.0):
    """Inputs of surrogate training samples: T, p, Y ~ Dirichlet, dt log-uniform.

    A fraction `premix_frac` of the samples draws Y from a Dirichlet concentrated on the
    stoichiometric premix (concentrations kappa * Y_premix + alpha_trace): near-premix states with
    trace radicals, the cold part of the reacting-front fields.  A fraction `mixing_frac` draws Y
    from a Dirichlet concentrated on the fuel / air mixing line, Z Y_fuel + (1 - Z) Y_air with
    Z ~ U[0, 1] and each end (pure fuel, pure air) taken exactly for a tenth of them: the cold part
    of the shear-layer fields.  The rest draws from Dirichlet(alpha)."""
    rng = np.random.default_rng(seed + 15485863)
    T = rng.uniform(*T_range, size=n)
    p = rng.uniform(*p_atm, size=n) * P_ATM
    Y = rng.dirichlet(np.full(mech["ns"], alpha), size=n).T
    dt = np.exp(rng.uniform(*log_dt, size=n))
    u = rng.random(n)
    if premix_frac > 0:
        pick = u < premix_frac
        conc = kappa * premix_mass_fractions(mech) + alpha_trace
        Y[:, pick] = rng.dirichlet(conc, size=int(pick.sum())).T
    if mixing_frac > 0:
        pick = np.nonzero((u >= premix_frac) & (u < premix_frac + mixing_frac))[0]
        air = np.zeros(mech["ns"])
        air[mech["oxidizer"]], air[mech["inert"]] = 1.0, 3.76
        air *= mech["W"]
        air /= air.sum()
        fuel = np.zeros(mech["ns"])
        fuel[mech["fuel"]] = 1.0
        Z = rng.uniform(0.0, 1.0, size=pick.size)
        end = rng.random(pick.size)
        Z[end < 0.1], Z[(end >= 0.1) & (end < 0.2)] = 0.0, 1.0
        base = Z[None, :] * fuel[:, None] + (1 - Z[None, :]) * air[:, None]
        exact = (Z == 0.0) | (Z == 1.0)
        draw = np.array([rng.dirichlet(kappa * base[:, j] + alpha_trace) for j in range(pick.size)]).T \
            if pick.size else np.zeros((mech["ns"], 0))
        Y[:, pick] = np.where(exact[None, :], base, draw)
    return T, p, Y, dt
