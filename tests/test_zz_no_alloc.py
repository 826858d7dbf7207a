"""tat_forward_noalloc: the forward operator with the library's static scratch.

For callers that cannot allocate device memory when they need A (their GPU
memory is all handed to their own pool, or cudaMalloc's implicit device
synchronisation is not acceptable in their loop).  This file sorts last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from tat_inputs import ellipse_phantom

pytestmark = pytest.mark.gpu


def test_noalloc_forward_matches_workspace_forward():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_24687_gb300 as pkg

    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    for n, nd, nt in ((64, 128, 128), (512, 1024, 1024)):
        op = pkg.TatOperator(n, nd, nt, support_radius=0.9, device="cuda:0")
        ws = op.workspace(1)
        g_ref = torch.empty((nd, nt), dtype=torch.float32, device="cuda:0")
        g_na = torch.empty((nd, nt), dtype=torch.float32, device="cuda:0")
        for seed in (0, 1):                      # two calls in a row, different inputs
            f = torch.tensor(ellipse_phantom(n, seed), dtype=torch.float32, device="cuda:0")
            g_na.fill_(float("nan"))
            pkg.tat_forward(op.plan, f.data_ptr(), g_ref.data_ptr(), ws.data_ptr(), st)
            pkg.tat_forward_noalloc(op.plan, f.data_ptr(), g_na.data_ptr(), st)
            torch.cuda.synchronize()
            a, b = g_na.cpu().numpy(), g_ref.cpu().numpy()
            assert np.isfinite(a).all()
            # the same five kernels in the same launch shapes: the forward is bit-deterministic
            assert np.array_equal(a, b)
        op.close()


def test_noalloc_rejects_plans_beyond_the_static_buffer():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_24687_gb300 as pkg

    torch.cuda.set_device(0)
    op = pkg.TatOperator(768, 1536, 1536, support_radius=0.9, device="cuda:0")
    assert pkg.tat_workspace_size(op.plan, 1) > 16 << 20
    f = torch.zeros((768, 768), dtype=torch.float32, device="cuda:0")
    g = torch.zeros((1536, 1536), dtype=torch.float32, device="cuda:0")
    with pytest.raises(pkg.TatError) as e:
        pkg.tat_forward_noalloc(op.plan, f.data_ptr(), g.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 2
    op.close()


def test_noalloc_rejects_misaligned_pointers_on_the_host():
    """A pointer that is not 4-byte aligned is refused before any launch, as by tat_forward."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_24687_gb300 as pkg

    torch.cuda.set_device(0)
    op = pkg.TatOperator(64, 128, 128, support_radius=0.9, device="cuda:0")
    f = torch.zeros(64 * 64 + 4, dtype=torch.float32, device="cuda:0")
    g = torch.zeros(128 * 128 + 4, dtype=torch.float32, device="cuda:0")
    st = torch.cuda.current_stream().cuda_stream
    for fp, gp in ((f.data_ptr() + 2, g.data_ptr()), (f.data_ptr(), g.data_ptr() + 2)):
        with pytest.raises(pkg.TatError) as e:
            pkg.tat_forward_noalloc(op.plan, fp, gp, st)
        assert e.value.status == 1
    torch.cuda.synchronize()
    op.close()
