"""The allocation-free pair-list entry point (for callers that cannot call
cudaMalloc when they need the list) against the pair list of a regular solve:
identical rows and count, bit for bit, on two calls in a row.  Collected last
so that a failure here stops a -x run only after every other test ran."""
import numpy as np
import pytest

import paper_2011_07209_gb300.synth as synth

pytestmark = pytest.mark.gpu


def _cases():
    tri = 14.0 * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]])
    return [("cubic_config1", synth.make_config(1), 8.0, 6.0, 8.0),
            ("triclinic", synth.water_cell(tri, (56, 56, 56), 4, 3), 7.0, 5.0, 6.5)]


@pytest.mark.parametrize("case", range(2))
def test_noalloc_pair_list_matches_solve(case):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_07209_gb300 import driver, exx
    name, ws, r_pair, r_pe, r_me = _cases()[case]
    ctx = exx.Context(0)
    try:
        p = exx.make_params(r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=1e-8, precision=exx.MIXED)
        cr = driver.prepare(ctx, ws, p, want_d=False)
        out = driver.run(ctx, cr, pair_outputs=False)
        ref = cr.plan.pair_list()
        assert ref.shape[0] == out["n_pairs"] > 0
        cen = torch.as_tensor(np.ascontiguousarray(ws.centres), device="cuda")
        cap = ws.n_orb * (ws.n_orb + 1) // 2
        for call in range(2):
            rows = torch.full((cap, 8), -7, dtype=torch.int32, device="cuda")
            n = torch.zeros(1, dtype=torch.int32, device="cuda")
            code = exx.pair_list_noalloc(ws.lattice, ws.n, cen, ws.n_orb, r_pair, rows, n)
            assert code == exx.OK, (name, call, code)
            torch.cuda.synchronize()
            k = int(n.item())
            assert k == ref.shape[0], (name, call)
            assert np.array_equal(rows[:k].cpu().numpy(), ref), (name, call)
            assert np.all(rows[k:].cpu().numpy() == -7)
        # a capacity below the pair count: the first cap rows are written, the
        # rest of the buffer is untouched and the count is still the full one
        cap2 = max(1, k // 3)
        rows = torch.full((cap2 + 5, 8), -7, dtype=torch.int32, device="cuda")
        n.fill_(-1)
        assert exx.pair_list_noalloc(ws.lattice, ws.n, cen, ws.n_orb, r_pair, rows[:cap2], n) == exx.OK
        torch.cuda.synchronize()
        assert int(n.item()) == k
        assert np.array_equal(rows[:cap2].cpu().numpy(), ref[:cap2])
        assert np.all(rows[cap2:].cpu().numpy() == -7)
        # no orbitals: zero pairs, nothing written
        rows = torch.full((cap2 + 5, 8), -7, dtype=torch.int32, device="cuda")
        n.fill_(-1)
        assert exx.pair_list_noalloc(ws.lattice, ws.n, cen, 0, r_pair, rows, n) == exx.OK
        torch.cuda.synchronize()
        assert int(n.item()) == 0
        assert np.all(rows.cpu().numpy() == -7)
        # sizes beyond the static scratch are refused
        big = torch.zeros((16385, 3), dtype=torch.float64, device="cuda")
        assert exx.pair_list_noalloc(ws.lattice, ws.n, big, 16385, r_pair, rows, n) == exx.ERR_CAPACITY
    finally:
        ctx.close()
