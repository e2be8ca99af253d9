"""srp_force_noalloc: the variant of srp_force for callers that cannot
allocate GPU memory (its partial sums live in a fixed array inside the
library instead of context-owned scratch).  Checked through the C ABI
against srp_force on the same inputs, on two calls in a row (the second call
reuses the array the first one left filled).  This file is collected last."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_srp_force_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    ctx = srp.Context(0)
    m, rho, _, com = W.config2(4)
    sun = W.fibonacci_directions(6)
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    r_t = torch.from_numpy(rho[None].copy()).to(dev)
    s_t = torch.from_numpy(sun.copy()).to(dev)
    c_t = torch.from_numpy(com[None].copy()).to(dev)
    kw = dict(rays_x=300, rays_y=200, max_bounces=3, seed=5)
    ref = srp.srp_force(ctx, [b], r_t, s_t, c_t, out_sigma=True, **kw)
    torch.cuda.synchronize()
    for call in range(2):
        out = torch.full((1, 6, 6), float("nan"), dtype=torch.float64, device=dev)
        sig = torch.full((1, 6, 6), float("nan"), dtype=torch.float64, device=dev)
        st = torch.full((1,), -1, dtype=torch.int32, device=dev)
        srp.srp_force_noalloc([b], r_t, s_t, c_t, out, out_sigma=sig, status=st, **kw)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        # same chunking as srp_force here, so the tolerance of the suite's
        # FP32-partial comparisons is ample (results are in fact identical)
        assert np.allclose(out.cpu().numpy(), ref[0].cpu().numpy(), rtol=1e-6, atol=1e-12), call
        assert np.allclose(sig.cpu().numpy(), ref[1].cpu().numpy(), rtol=1e-6, atol=1e-12), call


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    dev = torch.device("cuda:0")
    ctx = srp.Context(0)
    m, rho, _, com = W.config1()
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    r_t = torch.from_numpy(rho[None].copy()).to(dev)
    c_t = torch.from_numpy(com[None].copy()).to(dev)
    big = torch.from_numpy(W.fibonacci_directions(90000)).to(dev)
    out = torch.empty((1, 90000, 6), dtype=torch.float64, device=dev)
    with pytest.raises(srp.SRPError) as e:
        srp.srp_force_noalloc([b], r_t, big, c_t, out, rays_x=64)
    assert e.value.code == srp.SRP_EINVAL and "capacity" in str(e.value)
