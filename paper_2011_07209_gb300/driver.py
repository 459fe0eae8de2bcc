"""Convenience layer over the C ABI: run one cell (or a batch) from numpy inputs.

Device memory comes from PyTorch; the computation is entirely the CUDA
library's.  ``mem="host"`` passes numpy buffers and lets the library do the
host<->device copies itself (the end-to-end path).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import exx


@dataclasses.dataclass
class CellRun:
    """Device-resident inputs and outputs of one cell."""
    ws: object
    params: exx.Params
    plan: exx.Plan
    phi: object
    centres: object
    box_lo: object
    dxx: object
    dbox: np.ndarray
    dbox_lo_np: np.ndarray
    dbox_lo: object
    pair_e: object
    pair_sig: object
    pair_iter: object
    pair_cap: int

    def orbitals(self):
        return exx.make_orbitals(self.ws.n_orb, self.ws.box, self.centres, self.box_lo, self.phi, exx.MEM_DEVICE)

    def result(self, pair_outputs=True):
        return exx.make_result(self.dxx, self.dbox, self.dbox_lo, exx.MEM_DEVICE,
                               self.pair_cap if pair_outputs else 0,
                               self.pair_e if pair_outputs else None,
                               self.pair_sig if pair_outputs else None,
                               self.pair_iter if pair_outputs else None)


def prepare(ctx: exx.Context, ws, params: exx.Params, *, device=0, want_d=True, plan=None, max_orb=None,
            dxx=None) -> CellRun:
    """Device inputs and outputs of one cell.  dxx: an existing D buffer
    [n_orb][dbox...] to write into (shared between cells solved one after the
    other); otherwise one is allocated when want_d."""
    import torch
    dev = torch.device("cuda", device)
    if plan is None:
        plan = exx.Plan(ctx, ws.lattice, ws.n, params, max_orb or max(ws.n_orb, 1), ws.box)
    phi = torch.as_tensor(np.ascontiguousarray(ws.phi), device=dev)
    centres = torch.as_tensor(np.ascontiguousarray(ws.centres, np.float64), device=dev)
    box_lo = torch.as_tensor(np.ascontiguousarray(ws.box_lo, np.int32), device=dev)
    dbox, dbox_lo_np = exx.dbox_layout(ws.lattice, ws.n, ws.centres, params,
                                       dbox=None if dxx is None else tuple(dxx.shape[1:]))
    if dxx is not None or want_d:
        if dxx is None:
            dxx = torch.zeros((ws.n_orb,) + tuple(int(x) for x in dbox), dtype=torch.float64, device=dev)
        dbox_lo = torch.as_tensor(dbox_lo_np, device=dev)
    else:
        dxx = None
        dbox_lo = None
    pair_cap = max(1, ws.n_orb * (ws.n_orb + 1) // 2)
    pair_e = torch.zeros(pair_cap, dtype=torch.float64, device=dev)
    pair_sig = torch.zeros((pair_cap, 3, 3), dtype=torch.float64, device=dev)
    pair_iter = torch.zeros(pair_cap, dtype=torch.int32, device=dev)
    return CellRun(ws, params, plan, phi, centres, box_lo, dxx, dbox, dbox_lo_np, dbox_lo, pair_e, pair_sig,
                   pair_iter, pair_cap)


def run(ctx: exx.Context, cr: CellRun, *, lattice=None, pair_outputs=True, stream=None, check=True) -> dict:
    """Solve one prepared cell; returns scalars, status and (device) tensors."""
    res = cr.result(pair_outputs)
    lat = cr.ws.lattice if lattice is None else lattice
    code = exx.solve(ctx, cr.plan, lat, cr.ws.n, cr.orbitals(), res, stream=stream, check=check)
    out = exx.result_dict(res)
    out["status"] = code
    if pair_outputs:
        n = out["n_pairs"]
        out["pair_e"] = cr.pair_e[:n].cpu().numpy()
        out["pair_sig"] = cr.pair_sig[:n].cpu().numpy()
        out["pair_iter"] = cr.pair_iter[:n].cpu().numpy()
        out["pairs"] = cr.plan.pair_list()
    return out


def run_host(ctx: exx.Context, plan: exx.Plan, ws, params: exx.Params, *, want_d=True, stream=None) -> dict:
    """End-to-end call with host (numpy) buffers: the library copies in and out."""
    phi = np.ascontiguousarray(ws.phi)
    centres = np.ascontiguousarray(ws.centres, np.float64)
    box_lo = np.ascontiguousarray(ws.box_lo, np.int32)
    orb = exx.make_orbitals(ws.n_orb, ws.box, centres, box_lo, phi, exx.MEM_HOST)
    dbox, dbox_lo = exx.dbox_layout(ws.lattice, ws.n, ws.centres, params)
    dxx = np.zeros((ws.n_orb,) + tuple(int(x) for x in dbox)) if want_d else None
    res = exx.make_result(dxx, dbox, dbox_lo if want_d else None, exx.MEM_HOST)
    code = exx.solve(ctx, plan, ws.lattice, ws.n, orb, res, stream=stream)
    out = exx.result_dict(res)
    out["status"] = code
    out["dxx"] = dxx
    out["dbox"] = dbox
    out["dbox_lo"] = dbox_lo
    return out


def run_batch(ctx: exx.Context, runs, *, pair_outputs=False, stream=None, check=True):
    results = [r.result(pair_outputs) for r in runs]
    code = exx.solve_batch(ctx, [r.plan for r in runs], [(r.ws.lattice, r.ws.n) for r in runs],
                           [r.orbitals() for r in runs], results, stream=stream, check=check)
    outs = [exx.result_dict(r) for r in results]
    for o in outs:
        o["status"] = code
    return outs


def reduce_shards(out: dict, dxx, dist) -> dict:
    """Sum a sharded solve's partial results over the ranks of `dist` (a
    torch.distributed module with an initialised process group): E_xx, dE/dh,
    Pi_xx and p_int (one all-reduce of 20 doubles) and the D_xx boxes (one
    all-reduce of the D buffer, when given).  The sums are the single-rank
    results (Sec. III A, Step V: MPI_SUM of E_xx and sigma, D_ji returned to
    the owner of orbital j).  Returns a copy of `out` with the summed scalars."""
    import torch
    dev = dxx.device if dxx is not None else torch.device("cpu")
    if dev.type == "cpu" or dist.get_backend() == "gloo":
        dev_s = torch.device("cpu")
    else:
        dev_s = dev
    v = torch.tensor([out["e_xx"], *np.asarray(out["dedh"], float).ravel(), *np.asarray(out["stress"], float).ravel(),
                      out["p_int"]], dtype=torch.float64, device=dev_s)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    if dxx is not None:
        dist.all_reduce(dxx, op=dist.ReduceOp.SUM)
    v = v.cpu().numpy()
    red = dict(out)
    red["e_xx"] = float(v[0])
    red["dedh"] = v[1:10].reshape(3, 3)
    red["stress"] = v[10:19].reshape(3, 3)
    red["p_int"] = float(v[19])
    return red

