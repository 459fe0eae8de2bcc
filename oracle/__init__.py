"""Plain FP64 CPU oracle of the exact-exchange pair path (ctypes binding).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the product path never
does.  The C source ``exx_oracle.c`` shares no code with the CUDA library.

Every entry point mirrors one step of the method of arXiv 2011.07209 (see
the header of ``exx_oracle.c`` for the equation each follows).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against printed values, closed forms, identities or brute force; the
``a != 0`` (non-Gaussian) orbitals are checked only through those identities.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "exx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", 1: "bad argument", 2: "singular or left-handed cell", 3: "halo outside ME set",
          4: "no valid Natan-Kronik stencil", 5: "CG did not converge", 6: "capacity too small",
          7: "D box too small", 8: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code, where=""):
        super().__init__(f"oracle error {code} ({ERRORS.get(code, '?')}) {where}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP on)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_LIB)
    return _lib


class Params(C.Structure):
    _fields_ = [("r_pair", C.c_double), ("r_pe_self", C.c_double), ("r_pe_pair", C.c_double),
                ("r_me_self", C.c_double), ("r_me_pair", C.c_double), ("cg_tol", C.c_double),
                ("fd_n", C.c_int), ("lmax", C.c_int), ("cg_max_iter", C.c_int), ("nq", C.c_int),
                ("n_threads", C.c_int), ("frozen", C.c_int), ("lattice0", C.c_double * 9)]


def make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, r_pe_self=None, r_me_self=None, tol=1e-10, fd_n=3, lmax=6,
                max_iter=20000, nq=15, n_threads=0, lattice0=None, freeze_aux=False) -> Params:
    p = Params()
    p.r_pair = r_pair
    p.r_pe_pair = r_pe
    p.r_me_pair = r_me
    p.r_pe_self = r_pe if r_pe_self is None else r_pe_self
    p.r_me_self = r_me if r_me_self is None else r_me_self
    p.cg_tol = tol
    p.fd_n = fd_n
    p.lmax = lmax
    p.cg_max_iter = max_iter
    p.nq = nq
    p.n_threads = n_threads
    if lattice0 is not None:
        # offsets of lattice0; aux directions of the current cell unless freeze_aux
        p.frozen = 2 if freeze_aux else 1
        for k, v in enumerate(np.asarray(lattice0, float).ravel()):
            p.lattice0[k] = float(v)
    return p


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def _check(code, where=""):
    if code != 0:
        raise OracleError(code, where)


def fd2_weights(n: int) -> np.ndarray:
    w, pw = _d(np.zeros(n + 1))
    _check(lib().orc_fd2_weights(C.c_int(n), pw))
    return w


def fd1_weights(n: int) -> np.ndarray:
    w, pw = _d(np.zeros(n + 1))
    _check(lib().orc_fd1_weights(C.c_int(n), pw))
    return w


def metric(lattice, n):
    lat, pl = _d(lattice)
    nn, pn = _i(n)
    h, ph = _d(np.zeros(9)); hi, phi_ = _d(np.zeros(9)); J, pJ = _d(np.zeros(9)); F, pF = _d(np.zeros(9))
    dxi, pdx = _d(np.zeros(3))
    vol = C.c_double()
    _check(lib().orc_metric(pl, pn, ph, phi_, C.byref(vol), pdx, pJ, pF), "metric")
    return dict(h=h.reshape(3, 3), hinv=hi.reshape(3, 3), vol=vol.value, dxi=dxi, J=J.reshape(3, 3), F=F.reshape(3, 3))


def nk_candidates(lattice, n, nq=15):
    lat, pl = _d(lattice)
    nn, pn = _i(n)
    m, pm = _i(np.zeros((nq, 3)))
    ln, plen = _d(np.zeros(nq))
    cnt = C.c_int()
    _check(lib().orc_nk_candidates(pl, pn, C.c_int(nq), pm, plen, C.byref(cnt)), "candidates")
    return m[:cnt.value].copy(), ln[:cnt.value].copy()


def stencil_info(lattice, n, fd_n=3, nq=15, aux=None):
    """Directions (integer steps), coefficients, N_aux, N_off and b of the NK stencil."""
    lat, pl = _d(lattice)
    nn, pn = _i(n)
    dirs, pdirs = _i(np.zeros((6, 3)))
    coef, pcoef = _d(np.zeros(6))
    b, pb = _d(np.zeros(3))
    nd, naux, noff = C.c_int(), C.c_int(), C.c_int()
    if aux is not None:
        ax, pax = _i(np.asarray(aux).reshape(-1, 3))
        nax = ax.shape[0]
    else:
        ax, pax, nax = None, None, 0
    code = lib().orc_stencil_info(pl, pn, C.c_int(fd_n), C.c_int(nq), pax, C.c_int(nax), C.byref(nd), pdirs,
                                  pcoef, C.byref(naux), C.byref(noff), pb)
    _check(code, "stencil")
    return dict(dirs=dirs[:nd.value].copy(), coef=coef[:nd.value].copy(), n_aux=naux.value, n_off=noff.value,
                b=b[:naux.value].copy(), n_stcl=2 * fd_n * nd.value + 1)


def stencil_code(lattice, n, fd_n=3, nq=15, aux=None) -> int:
    """Return code of the stencil build (0 ok, 4 when no definite stencil)."""
    try:
        stencil_info(lattice, n, fd_n, nq, aux)
        return 0
    except OracleError as e:
        return e.code


def apply_lap(lattice, n, f, fd_n=3, nq=15):
    lat, pl = _d(lattice)
    nn, pn = _i(n)
    f, pf = _d(f)
    bx, pbx = _i(f.shape)
    out, po = _d(np.zeros_like(f))
    _check(lib().orc_apply_lap(pl, pn, C.c_int(fd_n), C.c_int(nq), pbx, pf, po), "apply_lap")
    return out


def solid_harmonics(lmax, xyz):
    xyz, px = _d(np.asarray(xyz, float).reshape(-1, 3))
    nlm = (lmax + 1) ** 2
    out, po = _d(np.zeros((xyz.shape[0], nlm)))
    _check(lib().orc_solid_harmonics(C.c_int(lmax), C.c_int(xyz.shape[0]), px, po))
    return out


def multipoles(lmax, xyz, q):
    xyz, px = _d(np.asarray(xyz, float).reshape(-1, 3))
    q, pq = _d(q)
    Q, pQ = _d(np.zeros((lmax + 1) ** 2))
    _check(lib().orc_multipoles(C.c_int(lmax), C.c_int(xyz.shape[0]), px, pq, pQ))
    return Q


def farfield(lmax, Q, xyz):
    xyz, px = _d(np.asarray(xyz, float).reshape(-1, 3))
    Q, pQ = _d(Q)
    v, pv = _d(np.zeros(xyz.shape[0]))
    _check(lib().orc_farfield(C.c_int(lmax), pQ, C.c_int(xyz.shape[0]), px, pv))
    return v


def offsets(lattice, n, r_pe, r_me):
    """(n_pe, m) with m[:n_pe] the PE offsets and m[n_pe:] the shell, lexicographic."""
    lat, pl = _d(lattice)
    nn, pn = _i(n)
    npe, nme = C.c_int(), C.c_int()
    _check(lib().orc_offsets_count(pl, pn, C.c_double(r_pe), C.c_double(r_me), C.byref(npe), C.byref(nme)))
    m, pm = _i(np.zeros((nme.value, 3)))
    _check(lib().orc_offsets_list(pl, pn, C.c_double(r_pe), C.c_double(r_me), C.c_int(nme.value), pm))
    return npe.value, m


def pair_list(lattice, n, centres, r_pair):
    """Rows (i, j, k0, k1, k2, g0, g1, g2) of the unique pair list, i <= j."""
    lat, pl = _d(lattice)
    nn, pn = _i(n)
    cen, pc = _d(np.asarray(centres, float).reshape(-1, 3))
    n_orb = cen.shape[0]
    cap = n_orb * (n_orb + 1) // 2 + 1
    rows, pr = _i(np.zeros((cap, 8)))
    npairs = C.c_int()
    _check(lib().orc_pair_list(pl, pn, C.c_int(n_orb), pc, C.c_double(r_pair), C.c_int(cap), C.byref(npairs), pr))
    return rows[:npairs.value].copy()


def dbox_for(ws, r_pair, r_me):
    """D boxes of half-width ceil((R_pair/2 + R_ME) N |h^-1 row|) + 1 around each centre."""
    lat = np.asarray(ws.lattice, float)
    n = np.asarray(ws.n, np.int64)
    hinv = np.linalg.inv(lat.T)
    hw = np.ceil((0.5 * r_pair + r_me) * n * np.linalg.norm(hinv, axis=1)).astype(np.int64) + 1
    dbox = np.minimum(2 * hw + 1, n)
    frac = ws.centres @ hinv.T
    frac -= np.floor(frac)
    gc = np.floor(frac * n + 0.5).astype(np.int64)
    return dbox.astype(np.int32), (gc - dbox // 2).astype(np.int32)


def exx(ws, params: Params, *, sel=None, want_d=True, dbox=None, dbox_lo=None):
    """Run the whole path on one cell; returns a dict of results and per-pair tables."""
    lat, pl = _d(ws.lattice)
    nn, pn = _i(ws.n)
    cen, pc = _d(ws.centres)
    box, pbox = _i(ws.box)
    blo, pblo = _i(ws.box_lo)
    phi, pphi = _d(ws.phi)
    n_orb = ws.n_orb
    if want_d:
        if dbox is None:
            dbox, dbox_lo = dbox_for(ws, params.r_pair, max(params.r_me_pair, params.r_me_self))
        db, pdb = _i(dbox)
        dlo, pdlo = _i(dbox_lo)
        dxx, pdxx = _d(np.zeros((n_orb,) + tuple(int(x) for x in db)))
    else:
        db = dlo = dxx = None
        pdb = pdlo = pdxx = None
    cap = n_orb * (n_orb + 1) // 2 + 1
    rows, prows = _i(np.zeros((cap, 8)))
    pe, ppe = _d(np.zeros(cap)); ps, pps = _d(np.zeros((cap, 3, 3)))
    pn_cg, pncg = _i(np.zeros(cap)); pres, ppres = _d(np.zeros(cap))
    if sel is not None:
        selv, psel = _i(np.asarray(sel))
        nsel = selv.shape[0]
    else:
        selv, psel, nsel = None, None, 0
    e_xx = C.c_double()
    dedh, pdedh = _d(np.zeros(9)); stress, pstress = _d(np.zeros(9))
    info, pinfo = _i(np.zeros(4))
    npairs = C.c_int()
    code = lib().orc_exx(pl, pn, C.c_int(n_orb), pc, pbox, pblo, pphi, pdb, pdlo, pdxx, C.byref(params),
                         C.c_int(nsel), psel, C.c_int(cap), C.byref(npairs), prows, ppe, pps, pncg, ppres,
                         C.byref(e_xx), pdedh, pstress, pinfo)
    _check(code, "exx")
    npr = npairs.value
    return dict(e_xx=e_xx.value, dedh=dedh.reshape(3, 3), stress=stress.reshape(3, 3), dxx=dxx, dbox=db,
                dbox_lo=dlo, pairs=rows[:npr].copy(), pair_e=pe[:npr].copy(), pair_sig=ps[:npr].copy(),
                pair_ncg=pn_cg[:npr].copy(), pair_res=pres[:npr].copy(), n_aux=int(info[0]),
                n_stcl=int(info[1]), max_cg=int(info[2]))


def pair_potential(ws, i, j, g_ij, params: Params):
    """v of pair (i, j) on its ME offsets (PE first), with the offsets."""
    lat, pl = _d(ws.lattice)
    nn, pn = _i(ws.n)
    box, pbox = _i(ws.box)
    phi = np.ascontiguousarray(ws.phi)
    pi_ = phi[i].ctypes.data_as(C.POINTER(C.c_double))
    pj_ = phi[j].ctypes.data_as(C.POINTER(C.c_double))
    loi, ploi = _i(ws.box_lo[i]); loj, ploj = _i(ws.box_lo[j])
    g, pg = _i(g_ij)
    self_ = int(i == j)
    r_pe = params.r_pe_self if self_ else params.r_pe_pair
    r_me = params.r_me_self if self_ else params.r_me_pair
    lat_ref = np.array(list(params.lattice0)).reshape(3, 3) if params.frozen else ws.lattice
    npe0, m = offsets(lat_ref, ws.n, r_pe, r_me)
    cap = m.shape[0]
    v, pv = _d(np.zeros(cap))
    npe, nme, ncg = C.c_int(), C.c_int(), C.c_int()
    ep = C.c_double()
    code = lib().orc_pair_potential(pl, pn, pbox, pi_, ploi, pj_, ploj, pg, C.c_int(self_), C.byref(params),
                                    C.c_int(cap), pv, C.byref(npe), C.byref(nme), C.byref(ncg), C.byref(ep))
    _check(code, "pair_potential")
    return dict(v=v, n_pe=npe.value, m=m, n_cg=ncg.value, e_pair=ep.value)
