"""The roofline arithmetic of bench.py (no GPU): the algorithmic FP64 flop counts per unit of
stiff-integrator work, pinned to the operation counts of the method on the 9-species mechanism's
8-species active block, and the stiff-phase flop total assembled from the kernel's counters."""
import numpy as np

import bench
import synth


def _lu_flops_by_hand(na):
    # partial-pivoting LU of an na x na block: at column k, one reciprocal of the pivot, na-k-1
    # multipliers and an (na-k-1)^2 rank-1 update (a multiply and an add each)
    total = 0
    for k in range(na):
        m = na - k - 1
        total += 1 + m + 2 * m * m
    return total


def test_active_block_of_the_9_species_mechanism():
    mech = synth.h2_air_mechanism(0)
    assert mech["ns"] == 9
    d = np.asarray(mech["nu_r"], int) - np.asarray(mech["nu_f"], int)
    na = bench.active_species(mech)
    assert na == 8
    assert not d[:, na:].any() and d[:, na - 1].any()   # only the trailing inert species is left out


def test_per_unit_flop_counts():
    ns, na = 9, 8
    # I - g h J: na^2 products and na^2 additions (the identity on the diagonal)
    assert bench.f_factor(ns, na) == 2 * na * na + _lu_flops_by_hand(na) == 444
    # error estimate (5 per species), its filter (one solve: 2 na^2) and its norm (2 per species)
    assert bench.f_attempt(ns, na) == 444 + 5 * na + 2 * na * na + 2 * na == 628
    # T(e): six mixture sums of ns products (12 ns) and two Newton iterations of 21 flops
    assert bench.f_te(ns) == 6 * 2 * ns + 2 * 21 == 150
    # a Newton iteration: T(e) of the iterate, the residual (3 per species), a solve, the update
    assert bench.f_newton(ns, na) == 150 + 3 * na + 2 * na * na + 2 * na == 318
    assert bench.f_accept(ns, na) == 150


def test_stiff_flops_from_counters():
    ns, na = 9, 8
    st = {"attempts": 1000, "newton": 4000, "substeps": 990}
    # every attempt factors (no reuse counter); the first Newton iterate of each attempt is the
    # step's initial state, whose temperature is known: one T(e) fewer per attempt
    want = 1000 * 628 + 4000 * 318 - 1000 * 150 + 990 * 150
    assert bench._stiff_flops(st, ns, na) == want
    # with reuse (the 53-species kernel) only the factorisations done are counted
    st2 = dict(st, factorizations=250)
    assert bench._stiff_flops(st2, ns, na) == want - 750 * bench.f_factor(ns, na)
