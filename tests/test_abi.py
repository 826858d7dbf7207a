"""The C ABI library builds, loads and exports every function include/*.h declares.

Host-only calls are exercised here; nothing launches GPU work.
"""
import math

import pytest


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_24687_gb300 as p
    return p


def test_exports_every_declared_symbol(pkg):
    lib = pkg.load()
    names = pkg.header_symbols()
    assert "tat_plan_create" in names and "tat_forward_batched" in names
    missing = [s for s in names if not hasattr(lib, s)]
    assert not missing, missing


def test_package_binds_every_declared_function(pkg):
    """The Python binding offers each C entry point under its own name (argument marshalling only)."""
    missing = [s for s in pkg.header_symbols() if not callable(getattr(pkg, s, None))]
    assert not missing, missing


def test_status_strings(pkg):
    assert pkg.tat_status_string(0) == "ok"
    assert pkg.tat_status_string(1) == "invalid argument"
    assert pkg.tat_status_string(4) == "CUDA error"
    assert pkg.tat_status_string(99) == "unknown status"


@pytest.mark.parametrize("bad", [
    dict(n=4), dict(n_det=7), dict(n_det=130, n_phi=130), dict(n_t=3), dict(c=0.0), dict(R=-1.0),
    dict(T=0.0), dict(n_phi=64), dict(support_radius=0.0), dict(pad_L=-1.0),
])
def test_query_rejects_invalid_descriptors(pkg, bad):
    d = pkg.tat_plan_desc_default(64, 128, 128)
    for k, v in bad.items():
        setattr(d, k, v)
    with pytest.raises(pkg.TatError) as e:
        pkg.tat_plan_query(d)
    assert e.value.status == 1


def test_unsupported_sizes(pkg):
    d = pkg.tat_plan_desc_default(4000, 8000, 8000)     # padded grid beyond 16384
    with pytest.raises(pkg.TatError) as e:
        pkg.tat_plan_query(d)
    assert e.value.status == 2


def test_null_handles_are_rejected(pkg):
    lib = pkg.load()
    assert lib.tat_forward(None, None, None, None, None) == 1
    assert lib.tat_adjoint_batched(None, 1, None, 0, None, 0, None, None) == 1
    assert lib.tat_plan_destroy(None) == 1
    assert lib.tat_workspace_size(None, 1) == 0
    assert lib.tat_plan_set_launch_shape(None, 8, 1, 256, 0) == 1
    assert lib.tat_plan_set_fft_order(None, 0) == 1
    assert lib.tat_plan_get_fft_order(None, None) == 1
    assert lib.tat_plan_set_column_split(None, 1) == 1
    assert lib.tat_plan_get_column_split(None, None) == 1


def test_plan_create_without_device_fails_cleanly(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(pkg.TatError) as e:
        pkg.tat_plan_create(64, 128, 128)
    assert e.value.status == 4
    # argument errors are reported before any CUDA call
    with pytest.raises(pkg.TatError) as e:
        pkg.tat_plan_create(64, 127, 128)
    assert e.value.status == 1


def test_default_descriptor_is_the_papers(pkg):
    d = pkg.tat_plan_desc_default(257, 360, 513, 1.0, 1.0, 4.0)
    assert d.support_radius == 0.98 and d.low_mode_quadrature == 1
    assert d.arc_begin == 0.0 and abs(d.arc_len - 2 * math.pi) < 1e-15
    info = pkg.tat_plan_query(d)
    assert info["n_phi"] == 360 and info["K"] == 180


def test_lpd_layers_reject_bad_arguments_before_any_device_work(pkg):
    """Argument checks of the convolution layers return before touching memory: misaligned
    activation pointers (the TMA-staged layers need 16 bytes), a missing weight pointer for
    data gradients, a scratch buffer that is too small."""
    bad = pkg.TatError
    fake, odd = 1 << 20, (1 << 20) + 2           # never dereferenced
    with pytest.raises(bad):
        pkg.tat_conv_out_fwd(1, 8, 16, odd, fake, fake, fake, fake)
    with pytest.raises(bad):
        pkg.tat_conv_mid_fwd(1, 8, 16, odd, fake, fake, fake)
    with pytest.raises(bad):
        pkg.tat_conv_in_bwd(1, 8, 16, 3, fake, fake, fake, odd, fake, fake, fake, 0, 0, 0, 0, 0, 0, 0)
    with pytest.raises(bad):
        pkg.tat_conv_in_bwd(1, 8, 16, 3, fake, fake, fake, fake, fake, 0, fake, 0, 0, 0, 0, 0, 0, 0)
    with pytest.raises(bad):
        pkg.tat_conv_out_bwd(1, 8, 16, fake, fake, fake, 0, fake, fake, 1, fake, fake)
    with pytest.raises(bad):
        pkg.tat_conv_in_fwd(1, 8, 16, 4, fake, fake, fake, fake, fake, fake)
    with pytest.raises(bad):                     # 2^32 pixels: tile indices are 32-bit
        pkg.tat_conv_out_fwd(1 << 16, 1 << 8, 1 << 8, fake, fake, fake, fake, fake)
    for tries in (0, (1 << 20) + 1):
        with pytest.raises(bad):
            pkg.tat_lpd_timeout_probe(tries, fake)
    with pytest.raises(bad):
        pkg.tat_lpd_timeout_probe(16, 0)
