"""The boundary's graph handle and host outputs (ABI of include/fgbd.h).

fgbd_graph_export makes a standalone CSR copy of the context's graph
(Section 2.2); fgbd_graph_csr lends its device arrays.  They must equal the
oracle's adjacency bit for bit (and the copy made by fgbd_graph_csr_copy),
carry the Eq. 4 weights and sigma_g, and outlive the context.  The host
outputs of fgbd_estimate_noise and fgbd_select_filter must equal the values
the device received.
"""
import numpy as np
import pytest
import torch

from oracle import fgbd_oracle as orc
from paper_2401_09721_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fgbd():
    build.build()
    from paper_2401_09721_gb300 import fgbd as F
    return F


def _oracle_graph(xyz, bits):
    codes = orc.scan_line_codes(xyz, bits)
    e = orc.slg_edges(orc.scan_orders(codes), 1)
    rp, col = orc.adjacency_csr(e, xyz.shape[0])
    return rp, col, orc.sigma_g(xyz, rp, col)


@pytest.mark.parametrize("n", [0, 1, 2, 7, 5000])
def test_exported_graph_equals_the_oracle_and_outlives_the_context(fgbd, n):
    rng = np.random.default_rng(n)
    xyz = rng.integers(0, 64, size=(n, 3)).astype(np.int32)
    ctx = fgbd.Context(max(n, 1), bits=6)
    ctx.build_graph(torch.from_numpy(xyz).cuda())
    rp_c, col_c, w_c = ctx.graph_csr()
    g = ctx.export_graph()
    ctx.close()
    rp, col, sg = _oracle_graph(xyz, 6)
    assert g.n == n and g.nnz == col.size
    if n == 0:
        return
    assert np.array_equal(g.row_ptr.cpu().numpy(), rp)
    assert np.array_equal(g.col.cpu().numpy(), col)
    assert torch.equal(g.row_ptr, rp_c) and torch.equal(g.col, col_c) and torch.equal(g.w, w_c)
    assert abs(g.sigma_g - sg) <= 1e-6 * max(sg, 1.0)
    if col.size:
        # Eq. 4 weights in the log, as the other parity tests compare them
        w_ref = orc.edge_weights(xyz, rp, col, sg)
        ok = w_ref > 1e-30
        lw_or = np.log(np.maximum(w_ref, 1e-300))
        lw = np.log(np.maximum(g.w.cpu().numpy().astype(np.float64), 1e-300))
        assert (np.abs(lw - lw_or)[ok] <= 1e-6 * np.maximum(1.0, np.abs(lw_or[ok])) + 1e-6).all()


def test_exported_graph_of_the_small_frame(fgbd):
    fr = synth.sphere_frame(20500, 9, 20.0, 0)
    ctx = fgbd.Context(fr.n, bits=9)
    ctx.build_graph(torch.from_numpy(fr.xyz).cuda())
    g1 = ctx.export_graph()
    g2 = ctx.export_graph()          # two handles of one graph are independent copies
    rp, col, sg = _oracle_graph(fr.xyz, 9)
    del g1
    torch.cuda.synchronize()
    assert np.array_equal(g2.row_ptr.cpu().numpy(), rp) and np.array_equal(g2.col.cpu().numpy(), col)
    assert g2.row_ptr.data_ptr() != 0
    ctx.close()


def test_host_outputs_of_the_estimate_and_the_selection(fgbd):
    fr = synth.sphere_frame(20500, 9, 20.0, 0)
    ctx = fgbd.Context(fr.n, bits=9)
    c = torch.from_numpy(fr.noisy).cuda()
    ctx.build_graph(torch.from_numpy(fr.xyz).cuda())
    sig_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    sig_host = ctx.estimate_noise(c, sigma_out=sig_dev, host=True)
    q_dev = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    q_host = ctx.select_filter(c, q_out=q_dev, host=True)
    st = ctx.stats()
    assert sig_host == st["sigma_est"] == float(sig_dev.item())
    assert q_host == st["q"] == int(q_dev.item())
    ref = orc.fgbd(fr.xyz, fr.noisy, orc.Params(bits=9))
    assert abs(sig_host - ref.noise["sigma_est"]) <= 1e-5 * ref.noise["sigma_est"]
    assert q_host == ref.q
    ctx.close()
