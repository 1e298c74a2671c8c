"""GPU parity of the 7-point diffusion step (the reduced weather application's
kernel, Sec. 4) in both storage orders (Sec. 1.3): each against the FP64
oracle (FP64 within 1e-12, FP32 within 2e-5 relative L2 and max), and the
two orders against each other bit for bit (same arithmetic per cell)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def asuca():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_08616_gb300 as a
    torch.cuda.set_device(0)
    return a


def _run(asuca, f, c, layout, dtype):
    import torch
    x = torch.tensor(f if layout == asuca.LAYOUT_IJK else np.transpose(f, (1, 2, 0)), dtype=dtype,
                     device="cuda").contiguous()
    y = torch.empty_like(x)
    asuca.stencil7(x, y, c, layout)
    torch.cuda.synchronize()
    out = y.double().cpu().numpy()
    return out if layout == asuca.LAYOUT_IJK else np.transpose(out, (2, 0, 1))


@pytest.mark.parametrize("shape", [(58, 37, 70), (3, 4, 5), (16, 33, 32), (58, 256, 256)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stencil7_both_layouts_against_oracle(asuca, shape, prec):
    import torch
    rng = np.random.default_rng(sum(shape))
    f = rng.standard_normal(shape) + 2.0
    c = 0.11
    ref = oracle.stencil7(f, c)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 2e-5
    outs = []
    for layout in (asuca.LAYOUT_IJK, asuca.LAYOUT_KIJ):
        got = _run(asuca, f, c, layout, dtype)
        l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        mx = np.abs(got - ref).max() / np.abs(ref).max()
        assert l2 <= tol and mx <= tol, (layout, l2, mx)
        outs.append(got)
    assert np.array_equal(outs[0], outs[1])


def test_stencil7_rejects_bad_arguments(asuca):
    import torch
    x = torch.zeros((4, 5, 6), device="cuda")
    with pytest.raises(asuca.AsucaError):
        asuca.stencil7(x, x, 0.1)
    with pytest.raises(asuca.AsucaError):
        asuca.stencil7(x, torch.empty_like(x), 0.1, 7)
