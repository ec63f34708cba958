"""Training pairs for the chemistry surrogate, made by this library's own plain integrator.

A training pair is (T, p, dt, Y) -> (Y1, T1): a cell's state after dt at constant density and
internal energy (the new state rather than its difference, which FP32 would round away when a
species falls from O(1) to its equilibrium trace level).  The pairs are produced on the GPU by chem_advance_boxes at a
tight tolerance, one box of cells per dt value, so that a data set of millions of samples costs
seconds; the surrogate is then trained on them by Context.surrogate_train.
"""
import numpy as np
import torch

from . import CHEM_FLAG_FP64_RATES, ChemError


def make_pairs(ctx, T, p, Y, dt_box, rtol=1e-6, atol=1e-11, fp64_rates=True, rho=None, e=None, stream=None):
    """Pairs for n cells in nbox = len(dt_box) equal boxes (n divisible by nbox, nbox <= 4096).

    T, p: [n] float32 CUDA tensors, Y: [ns][n] float32 CUDA tensor (inputs, not modified);
    dt_box: step of each box (host sequence); rho, e: the cells' density and internal energy, computed
    from (T, p, Y) by chem_state_from_TpY when not given.  rtol and atol are the integrator's
    tolerances for the pairs (tighter than the 1e-4 / 1e-10 the pairs are judged by); fp64_rates
    evaluates the stiff cells' rates in FP64 (CHEM_FLAG_FP64_RATES), which the 1e-10 bar on
    near-equilibrium minor species needs.  Returns (X [m][ns + 3], Yt [m][ns + 1], keep [n] bool) with
    X rows (T, p, dt, Y) and Yt rows (Y1, T1) for the m cells the integrator finished.  The
    context's box table is replaced and its parameters are restored afterwards."""
    n, nbox = T.shape[0], len(dt_box)
    if n % nbox:
        raise ValueError("cell count must be a multiple of the box count")
    m = n // nbox
    dev = T.device
    if rho is None or e is None:
        rho, e = torch.empty_like(T), torch.empty_like(T)
        ctx.state_from_TpY(T, p, Y, rho, e, stream)
    T1, p1, Y1 = T.clone(), p.clone(), Y.clone()
    sub = torch.zeros(n, dtype=torch.int32, device=dev)
    boxes = [dict(T=T1[b * m:(b + 1) * m], p=p1[b * m:(b + 1) * m], Y=Y1[:, b * m:(b + 1) * m],
                  rho=rho[b * m:(b + 1) * m], e=e[b * m:(b + 1) * m], substeps=sub[b * m:(b + 1) * m],
                  dt=float(dt_box[b]), level=0) for b in range(nbox)]
    old = (ctx.params.rtol, ctx.params.atol, ctx.params.flags)
    try:
        flags = old[2] | CHEM_FLAG_FP64_RATES if fp64_rates else old[2] & ~CHEM_FLAG_FP64_RATES
        ctx.set_params(rtol=rtol, atol=atol, flags=flags)
        ctx.set_boxes(boxes)
        ctx.advance_boxes(stream)
        st = ctx.status(stream)
    finally:
        ctx.set_params(rtol=old[0], atol=old[1], flags=old[2])
    if st["status"] not in (0, -3, -4):   # cells that hit k_max or collapsed are dropped below
        raise ChemError(st["status"], "training-pair integration")
    keep = (sub >= 0) & torch.isfinite(T1)
    dtc = torch.from_numpy(np.repeat(np.asarray(dt_box, np.float32), m)).to(dev)
    X = torch.cat([T[:, None], p[:, None], dtc[:, None], Y.t()], dim=1)[keep].contiguous()
    Yt = torch.cat([Y1.t(), T1[:, None]], dim=1)[keep].contiguous()
    return X, Yt, keep
