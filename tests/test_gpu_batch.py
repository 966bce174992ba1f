"""Batched solves (blockcg_batch_*): many independent problems, one stream
each, iterations replayed from one captured CUDA graph.  Each problem's
result must be bit-identical to blockcg_solve on the same handle (the same
kernels in the same order, with deterministic reductions), and its true
residual, recomputed by the CPU oracle, must meet the tolerance."""
import ctypes as ct

import numpy as np
import pytest

import hisq_inputs as hi
from oracle import hisq

from gpu_helpers import ensure_built, to_np

pytestmark = pytest.mark.gpu

TOL = 1e-10
# the oracle recomputes b - A x in FP64: rounding adds up to ~8 u |A| |x| / |b|
# <= 8 * 2^-53 * 4.4 / m^2 relative, 4% of TOL at m = 0.01
RES_SLACK = 1.05

SMALL = [
    {"dims": (4, 4, 4, 4), "mass": 0.1, "n_rhs": 4, "link_seed": 501, "source_seed": 601},
    {"dims": (4, 4, 4, 6), "mass": 0.05, "n_rhs": 3, "link_seed": 502, "source_seed": 602},
    {"dims": (6, 6, 6, 6), "mass": 0.02, "n_rhs": 8, "link_seed": 503, "source_seed": 603},
    {"dims": (8, 8, 8, 8), "mass": 0.2, "n_rhs": 2, "link_seed": 504, "source_seed": 604},
    {"dims": (4, 6, 4, 8), "mass": 0.15, "n_rhs": 5, "link_seed": 505, "source_seed": 605},
]


def _make(spec, prec, **kw):
    import torch
    from paper_1710_09745_gb300 import BlockCG
    fat, lng = hi.random_links_torch(spec["dims"], spec["link_seed"], torch.device("cuda"))
    kw.setdefault("max_iter", 20000)
    s = BlockCG(spec["dims"], fat, lng, spec["mass"], prec=prec, max_rhs=spec["n_rhs"], **kw)
    b = hi.gaussian_sources(spec["dims"], spec["n_rhs"], spec["source_seed"])
    return s, to_np(fat), to_np(lng), b


def _true_res(spec, fat, lng, b, X):
    r = b - hisq.apply_A(spec["dims"], fat, lng, spec["mass"], X)
    n = b.shape[0]
    return np.linalg.norm(r.reshape(n, -1), axis=1) / np.linalg.norm(b.reshape(n, -1), axis=1)


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("prec", ["mixed_f32", "f64"])
def test_batch_equals_individual_solves(prec, graph):
    import torch
    from paper_1710_09745_gb300 import BlockCGBatch
    ensure_built()
    probs = [_make(sp, prec) for sp in SMALL]
    batch = BlockCGBatch([p[0] for p in probs])
    Xs, infos, binfo = batch.solve([p[3] for p in probs], tol=TOL, graph=graph)
    assert binfo["status"] == 0, (binfo, infos)
    assert binfo["launches"] > 0 and binfo["ms_total"] > 0
    if graph:
        assert binfo["graph_replays"] >= 1 and binfo["graph_captures"] >= 1
        assert binfo["graph_nodes"] > 0
    else:
        assert binfo["graph_replays"] == 0
    for sp, (s, fat, lng, b), X, info in zip(SMALL, probs, Xs, infos):
        assert info["status"] == 0 and info["true_rel_res_max"] <= TOL
        Xi, ii = s.solve(b, tol=TOL)
        assert ii["iters"] == info["iters"]
        assert ii["reliable_updates"] == info["reliable_updates"]
        assert torch.equal(Xi, X)
        # per-right-hand-side true residuals: the same as the single solve's
        assert info["true_rel_res"] == ii["true_rel_res"]
        assert max(info["true_rel_res"]) == info["true_rel_res_max"]
        assert _true_res(sp, fat, lng, b, to_np(X)).max() <= TOL * RES_SLACK
    batch.close()


def test_batch_many_lattices_masses_and_widths():
    """64 problems: L^4 with L in {8, 12, 16}, m uniform in [0.01, 0.2], N in
    2..16, FP32 iterations with FP64 Grams and reliable updates, one CUDA
    graph per chunk.  Graph and plain launches agree bit for bit."""
    import torch
    from paper_1710_09745_gb300 import BlockCGBatch
    ensure_built()
    specs = hi.batch_problems(64, seed=4000)
    probs = [_make(sp, "mixed_f32") for sp in specs]
    batch = BlockCGBatch([p[0] for p in probs])
    Bs = [p[3] for p in probs]
    Xg, ig, bg = batch.solve(Bs, tol=TOL, graph=True)
    assert bg["status"] == 0, bg
    Xp, ip, bp = batch.solve(Bs, tol=TOL, graph=False)
    assert bp["status"] == 0, bp
    for sp, (s, fat, lng, b), a, c, inf in zip(specs, probs, Xg, Xp, ig):
        assert inf["status"] == 0 and inf["true_rel_res_max"] <= TOL, (sp, inf)
        assert torch.equal(a, c)
        assert _true_res(sp, fat, lng, b, to_np(a)).max() <= TOL * RES_SLACK, sp
    print(f"\n64 problems, {sum(sp['n_rhs'] for sp in specs)} RHS: graph {bg['ms_total']:.1f} ms "
          f"({bg['graph_replays']} replays, {bg['graph_captures']} captures, chunk {bg['chunk']}), "
          f"plain streams {bp['ms_total']:.1f} ms")
    batch.close()


def test_batch_reports_per_problem_outcome():
    """A problem that reaches max_iter fails alone: the batch returns
    NOT_CONVERGED, that problem's status says so, the others converge."""
    from paper_1710_09745_gb300 import BlockCGBatch
    ensure_built()
    good = _make(SMALL[0], "mixed_f32")
    bad = _make(SMALL[2], "mixed_f32", max_iter=3)
    batch = BlockCGBatch([good[0], bad[0]])
    Xs, infos, binfo = batch.solve([good[3], bad[3]], tol=TOL, graph=True)
    assert binfo["status"] == 6
    assert infos[0]["status"] == 0 and infos[1]["status"] == 6
    assert _true_res(SMALL[0], good[1], good[2], good[3], to_np(Xs[0])).max() <= TOL * RES_SLACK
    msg = batch.lib.blockcg_batch_last_error(batch.b).decode()
    assert msg.startswith("problem 1")
    batch.close()


def test_batch_rejects_width_beyond_workspace():
    """n_rhs above a handle's workspace is refused before any work, naming the problem."""
    import torch
    from paper_1710_09745_gb300 import BlockCGBatch
    ensure_built()
    a = _make(SMALL[0], "mixed_f32")
    c = _make(SMALL[3], "mixed_f32")
    batch = BlockCGBatch([a[0], c[0]])
    B0 = torch.as_tensor(a[3]).cuda()
    B1 = torch.zeros((8, c[0].Vh, 3), dtype=torch.complex128, device="cuda")  # max_rhs is 2
    X0, X1 = torch.zeros_like(B0), torch.zeros_like(B1)
    Bp = (ct.c_void_p * 2)(B0.data_ptr(), B1.data_ptr())
    Xp = (ct.c_void_p * 2)(X0.data_ptr(), X1.data_ptr())
    Np = (ct.c_int * 2)(B0.shape[0], 8)
    rc = batch.lib.blockcg_batch_solve(batch.b, Bp, Xp, Np, TOL, 1, None, None, None)
    assert rc == 3
    assert batch.lib.blockcg_batch_last_error(batch.b).decode().startswith("problem 1")
    assert torch.count_nonzero(X0) == 0
    batch.close()
