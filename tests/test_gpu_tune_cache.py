"""The autotune cache on the GPU: the first Chain.autotune tunes and stores its choice, a new
handle for the same workload applies it without tuning, and the integration gives the same
bits as an untuned run (every tiling computes the same operations)."""
import numpy as np
import pytest

import chain_inputs as ci

pytestmark = pytest.mark.gpu


def test_cached_choice_is_reused(tmp_path):
    import torch
    import paper_1412_0544_gb300 as rk
    assert torch.cuda.is_available()
    path = str(tmp_path / "tune.json")
    n = (1 << 18) + 17
    y0 = ci.uniform_state(n, 3, seed=980).astype(np.float32)
    a = rk.Chain(n, precision=rk.RK4_FP32_KAHAN)
    st = a.new_state(y0)
    first = a.autotune(st, a.new_comp(), 8, cache=path)
    assert first["cached"] is False
    b = rk.Chain(n, precision=rk.RK4_FP32_KAHAN)
    second = b.autotune(b.new_state(y0), b.new_comp(), 8, cache=path)
    assert second["cached"] is True
    assert (second["block"], second["v"], second["k"]) == (first["block"], first["v"], first["k"])
    assert b.tiling["block"] == first["block"] and b.tiling["k"] == first["k"]
    sb, cb = b.new_state(y0), b.new_comp()
    b.integrate(sb, cb, 40)
    c = rk.Chain(n, precision=rk.RK4_FP32_KAHAN, kernel=rk.RK4_KERNEL_STAGED)
    sc, cc = c.new_state(y0), c.new_comp()
    c.integrate(sc, cc, 40)
    torch.cuda.synchronize()
    assert torch.equal(sb, sc) and torch.equal(cb, cc)
    for ch in (a, b, c):
        ch.close()
