"""Host geometry of a plan (exx_geometry_query: metric, NK stencil of Sec. III C
and Algorithm 1, proto-subdomain offsets of Sec. III B) against the oracle,
without a GPU: the same planner code that exx_plan_create runs before it
uploads anything."""
import numpy as np
import pytest

import oracle
import paper_2011_07209_gb300.synth as synth
from paper_2011_07209_gb300 import build, exx


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    exx.lib()


MONOCLINIC = 14.0 * np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.12, 0.0, 1.0]])   # one off-diagonal metric term


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_benchmark_cells_match_oracle(k):
    c = synth.CONFIGS[k]
    g = exx.geometry(c["lattice"], c["n"], exx.make_params(r_pe=c["r_pe"], r_me=c["r_me"]))
    st = oracle.stencil_info(c["lattice"], c["n"])
    npe, m = oracle.offsets(c["lattice"], c["n"], c["r_pe"], c["r_me"])
    assert g["n_pe_pair"] == g["n_pe_self"] == npe
    assert g["n_me_pair"] == g["n_me_self"] == m.shape[0]
    assert g["n_aux"] == st["n_aux"] and g["n_stcl"] == st["n_stcl"]
    assert np.array_equal(g["dirs"], st["dirs"])
    assert np.allclose(g["coef"], st["coef"], rtol=1e-12)
    assert np.array_equal(g["aux"], st["dirs"][3:])
    assert g["workspace_bytes"] == 0 and g["ctas"] == 0          # no device work
    # the dense CG box holds the PE bounding box plus the stencil reach
    assert all(b > 2 * int(np.ceil(c["r_pe"] / (np.linalg.norm(c["lattice"][a]) / c["n"][a])))
               for a, b in enumerate(g["box_pair"]))


def test_monoclinic_cell_uses_one_bisector_direction():
    n = (56, 56, 56)
    g = exx.geometry(MONOCLINIC, n, exx.make_params(r_pe=5.0, r_me=6.5))
    st = oracle.stencil_info(MONOCLINIC, n)
    assert st["n_off"] == 1 and g["n_aux"] == st["n_aux"] == 1
    assert np.array_equal(g["dirs"], st["dirs"]) and g["n_stcl"] == 25
    assert np.allclose(g["coef"], st["coef"], rtol=1e-12)


def test_separate_self_radii():
    c = synth.CONFIGS[1]
    p = exx.make_params(r_pair=8.0, r_pe=5.0, r_me=7.0, r_pe_self=6.0, r_me_self=10.0)
    g = exx.geometry(c["lattice"], c["n"], p)
    npe_s, ms = oracle.offsets(c["lattice"], c["n"], 6.0, 10.0)
    npe_p, mp = oracle.offsets(c["lattice"], c["n"], 5.0, 7.0)
    assert (g["n_pe_self"], g["n_me_self"]) == (npe_s, ms.shape[0])
    assert (g["n_pe_pair"], g["n_me_pair"]) == (npe_p, mp.shape[0])


def test_errors():
    c = synth.CONFIGS[1]
    flip = np.array(c["lattice"], float).copy()
    flip[0] *= -1.0
    with pytest.raises(exx.ExxError) as e:
        exx.geometry(flip, c["n"], exx.make_params())
    assert e.value.code == exx.ERR_CELL
    with pytest.raises(exx.ExxError) as e:
        exx.geometry(c["lattice"], c["n"], exx.make_params(fd_order=0))
    assert e.value.code == exx.ERR_ARG
    assert exx.lib().exx_geometry_query(None, None, None) == exx.ERR_ARG


def test_dbox_layout_abi():
    """exx_dbox_layout (host only): the smallest extent 2 halfwidth + 1 (clamped
    to n), boxes centred on each centre's nearest grid point, a caller extent
    accepted between that and n and refused outside."""
    from paper_2011_07209_gb300 import exx
    lat = 29.6 * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]])
    n = (150, 150, 150)
    p = exx.make_params()
    rng = np.random.default_rng(4)
    cen = (rng.random((40, 3)) * 1.4 - 0.2) @ lat      # some centres outside the cell
    dbox, lo = exx.dbox_layout(lat, n, cen, p)
    hw = exx.dbox_halfwidth(lat, n, p)
    assert np.array_equal(dbox, np.minimum(2 * hw + 1, n))
    frac = cen @ np.linalg.inv(lat.T).T
    frac -= np.floor(frac)
    gc = np.floor(frac * np.asarray(n) + 0.5).astype(np.int64)
    assert np.array_equal(lo, gc - dbox // 2)
    big, lo2 = exx.dbox_layout(lat, n, cen, p, dbox=dbox + 2)
    assert np.array_equal(big, dbox + 2) and np.array_equal(lo2, gc - (dbox + 2) // 2)
    import pytest
    with pytest.raises(ValueError):
        exx.dbox_layout(lat, n, cen, p, dbox=dbox - 1)
    with pytest.raises(ValueError):
        exx.dbox_layout(lat, n, cen, p, dbox=(151, 151, 151))
