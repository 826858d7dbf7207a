"""GPU tests of the mixed-size request runtime (include/tat_service.h) and the
launch-shape autotuner: results (A, A*, A^-1 and the pair A* A) match the FP64
oracle at every size served (n = 1024 included) and equal the direct batched
calls, graphs are reused, admission under a tight memory budget evicts and shrinks batches and
reports out-of-memory for a request that fits at no batch size.
"""
import numpy as np
import pytest

from tat_inputs import ellipse_phantom, random_sinogram

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_24687_gb300 as p
    return p


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return t


SIZES = [(64, 128, 128), (96, 192, 160), (128, 256, 256)]


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _requests(torch, count=12):
    reqs = []
    for i in range(count):
        n, nd, nt = SIZES[i % len(SIZES)]
        op = ("forward", "adjoint", "inverse", "pair")[(i // len(SIZES)) % 4]
        if op in ("forward", "pair"):
            x = torch.tensor(ellipse_phantom(n, i).astype(np.float32), device="cuda:0")
            out = torch.empty((nd, nt) if op == "forward" else (n, n), device="cuda:0")
        else:
            x = torch.tensor(random_sinogram(nd, nt, i).astype(np.float32), device="cuda:0")
            out = torch.empty((n, n), device="cuda:0")
        reqs.append((n, nd, nt, op, x, out))
    return reqs


def _direct(pkg, torch, n, nd, nt, op, x):
    o = pkg.TatOperator(n, nd, nt, device="cuda:0", support_radius=0.9)
    if op == "pair":
        return o.adjoint(o.forward(x)).cpu().numpy()
    return getattr(o, op)(x).cpu().numpy()


def _oracle(n, nd, nt, op, x):
    """The FP64 oracle's answer to one request (the pair's intermediate A f kept in FP64)."""
    from oracle import tat_oracle as O
    P = O.OraclePlan(n, nd, nt, support_radius=0.9)
    xd = x.cpu().numpy().astype(np.float64)
    if op == "pair":
        return O.adjoint(P, O.forward(P, xd))
    return getattr(O, op)(P, xd)


@pytest.mark.parametrize("one_graph", [True, False], ids=["one-graph-flush", "graph-per-slot"])
def test_service_matches_oracle_and_direct_calls_and_reuses_graphs(pkg, torch, one_graph):
    """Every request of the mixed batch (three sizes, among them 96 x 96 with 192 x 160 data,
    times A, A*, A^-1 and the pair A* A) against the FP64 oracle at the parity bar 1e-5, and
    against the direct calls: the forward bit for bit, the rest to 1e-6 (A^-1 and the pair
    run with the service's batch, whose launch shapes may differ); with the whole flush as one
    graph launch (every size a parallel branch) and with one graph per slot."""
    svc = pkg.TatService(memory_budget=2 << 30, max_batch=4, one_graph=one_graph)
    reqs = _requests(torch)
    for rnd in range(2):
        ids = [svc.submit(svc.desc(n, nd, nt, support_radius=0.9), op, x, out) for n, nd, nt, op, x, out in reqs]
        svc.flush()
        svc.synchronize()
        for rid, (n, nd, nt, op, x, out) in zip(ids, reqs):
            ms, status = svc.latency(rid)
            assert status == 0 and ms > 0
            got = out.cpu().numpy()
            if rnd == 0:
                assert rel(got, _oracle(n, nd, nt, op, x)) <= 1e-5, (n, op)
            ref = _direct(pkg, torch, n, nd, nt, op, x)
            if op == "forward":
                assert np.array_equal(got, ref)
            else:
                assert rel(got, ref) <= 1e-6
    st = svc.stats()
    assert st["requests"] == st["completed"] == 2 * len(reqs)
    assert st["plans"] == len(SIZES) and st["evictions"] == 0
    if one_graph:
        # the composition's first flush runs per slot; from its second on, one graph launch covers
        # every size and operation
        assert st["flush_graphs"] == 1
    else:
        assert st["graph_launches"] > 0 and st["flush_graphs"] == 0
    svc.close()


def test_service_n1024_member_matches_oracle(pkg, torch):
    """The largest member of the mixed-size workload: n = 1024 with 2048 detectors x 2048
    samples (N = 8192, the 32-point four-step transforms), one A and one A* request through
    the service against the FP64 oracle at 1e-5."""
    n, nd, nt = 1024, 2048, 2048
    svc = pkg.TatService(memory_budget=8 << 30, max_batch=2)
    f = torch.tensor(ellipse_phantom(n, 7).astype(np.float32), device="cuda:0")
    g = torch.tensor(random_sinogram(nd, nt, 8).astype(np.float32), device="cuda:0")
    out_g = torch.empty((nd, nt), device="cuda:0")
    out_f = torch.empty((n, n), device="cuda:0")
    d = svc.desc(n, nd, nt, support_radius=0.9)
    ids = [svc.submit(d, "forward", f, out_g), svc.submit(d, "adjoint", g, out_f)]
    svc.flush()
    svc.synchronize()
    assert all(svc.latency(i)[1] == 0 for i in ids)
    assert rel(out_g.cpu().numpy(), _oracle(n, nd, nt, "forward", f)) <= 1e-5
    assert rel(out_f.cpu().numpy(), _oracle(n, nd, nt, "adjoint", g)) <= 1e-5
    svc.close()


def test_pinned_host_buffers(pkg, torch):
    """Requests with page-locked host inputs and outputs: the service uploads, runs and
    downloads them on the slot streams, with the results of the device-pointer path."""
    reqs = _requests(torch)
    svc = pkg.TatService(memory_budget=2 << 30, max_batch=4)
    hreqs = []
    for n, nd, nt, op, x, out in reqs:
        hx = x.cpu().pin_memory()
        hout = torch.empty(out.shape, dtype=torch.float32).pin_memory()
        hreqs.append((n, nd, nt, op, hx, hout))
    ids_h = [svc.submit(svc.desc(n, nd, nt, support_radius=0.9), op, hx, ho) for n, nd, nt, op, hx, ho in hreqs]
    ids_d = [svc.submit(svc.desc(n, nd, nt, support_radius=0.9), op, x, out) for n, nd, nt, op, x, out in reqs]
    svc.flush()
    svc.synchronize()
    for (n, nd, nt, op, hx, ho), (_, _, _, _, x, out), ih in zip(hreqs, reqs, ids_h):
        assert svc.latency(ih)[1] == 0
        if op == "forward":
            assert torch.equal(ho, out.cpu())
        else:
            assert rel(ho.numpy(), out.cpu().numpy()) <= 1e-6
    svc.close()


def test_admission_evicts_and_shrinks_batches(pkg, torch):
    """A budget that holds one (n = 128, batch 2) slot at a time: slots are evicted between sizes and
    the batch cap is halved; results stay exact."""
    info = pkg.tat_plan_query(pkg.tat_plan_desc_default(128, 256, 256))
    plan = pkg.tat_plan_create(128, 256, 256)
    ws1 = pkg.tat_workspace_size(plan, 1)
    pkg.tat_plan_destroy(plan)
    per_image = ws1 + 4 * (128 * 128 + 256 * 256) + 1024
    svc = pkg.TatService(memory_budget=int(2.5 * per_image), max_batch=8)
    reqs = [r for r in _requests(torch, 9) if r[3] == "forward"] + \
           [r for r in _requests(torch, 9) if r[3] == "adjoint"]
    ids = [svc.submit(svc.desc(n, nd, nt, support_radius=0.9), op, x, out) for n, nd, nt, op, x, out in reqs]
    svc.flush()
    svc.synchronize()
    for rid, (n, nd, nt, op, x, out) in zip(ids, reqs):
        assert svc.latency(rid)[1] == 0
        ref = _direct(pkg, torch, n, nd, nt, op, x)
        assert rel(out.cpu().numpy(), ref) <= 1e-6
    st = svc.stats()
    assert st["evictions"] > 0 and st["peak_bytes"] <= st["arena_bytes"]
    assert info["N"] == 1024
    svc.close()


def test_request_too_large_reports_oom(pkg, torch):
    svc = pkg.TatService(memory_budget=1 << 20, max_batch=2)
    x = torch.zeros((128, 128), device="cuda:0")
    out = torch.empty((256, 256), device="cuda:0")
    rid = svc.submit(svc.desc(128, 256, 256), "forward", x, out)
    with pytest.raises(pkg.TatError):
        svc.flush()
    svc.synchronize()
    assert svc.latency(rid)[1] == 3      # TAT_ERR_OOM
    svc.close()


def test_autotune_keeps_results(pkg, torch):
    n, nd, nt, B = 128, 256, 256, 4
    op = pkg.TatOperator(n, nd, nt, device="cuda:0", support_radius=0.9)
    f = torch.tensor(np.stack([ellipse_phantom(n, 30 + b) for b in range(B)]).astype(np.float32), device="cuda:0")
    g0 = op.forward(f).cpu().numpy()
    a0 = op.adjoint(op.forward(f)).cpu().numpy()
    g = torch.empty((B, nd, nt), device="cuda:0")
    f2 = torch.empty_like(f)
    ws = op.workspace(B)
    s = torch.cuda.current_stream().cuda_stream
    ms, strip, rp, ct, rt = pkg.tat_plan_autotune(op.plan, B, f.data_ptr(), g.data_ptr(), f2.data_ptr(), ws.data_ptr(), s)
    assert ms > 0 and strip in (2, 4, 8, 16, 32) and rp in (1, 2, 4, 8, 16) and ct in (64, 128, 256, 384)
    assert rt in (64, 128, 256)
    order = pkg.tat_plan_get_fft_order(op.plan)
    assert order in (0, 1)
    split = pkg.tat_plan_get_column_split(op.plan)
    assert split in (0, 1, 2, 3)
    g1 = op.forward(f).cpu().numpy()
    if order == 0 and split & 1:
        assert np.array_equal(g1, g0)     # launch shapes only regroup work
    else:
        assert rel(g1, g0) <= 1e-6        # another FFT pass order or column transform rounds differently
    assert rel(op.adjoint(op.forward(f)).cpu().numpy(), a0) <= 1e-6
    # at a fixed pass order A* does not depend on the launch shapes, bit for bit
    gfix = torch.tensor(g0, device="cuda:0")
    a_t = op.adjoint(gfix).cpu().numpy()
    pkg.tat_plan_set_launch_shape(op.plan, 8, 4, 256, 256)
    assert np.array_equal(op.adjoint(gfix).cpu().numpy(), a_t)
