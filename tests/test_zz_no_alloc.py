"""The allocation-free head-correction entry point agrees with the value
bse_create computes (the existing path), on two calls in a row.

Callers that cannot allocate device memory where they need W^div (a
framework owning the memory budget through its own pool, a latency-critical
loop, a plug-in given only pre-allocated buffers) use
bse_head_correction_noalloc, whose scratch is a fixed array inside the
library.  This file is collected last so that a run stopping at the first
failure has run every other test before it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.mark.parametrize("name", ["si4", "mos2_331", "mos2_331_uni", "si8"])
def test_noalloc_matches_create_twice(name):
    import torch
    from paper_2603_24860_gb300 import bse
    from synth import generate
    d = generate(name)
    stream = torch.cuda.current_stream()
    ctx = bse.bse_create(d, stream=stream)
    ref = bse.bse_tables(ctx)["w_div"]
    bse.bse_destroy(ctx)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for i in range(2):
        bse.bse_head_correction_noalloc(d["lattice"], d["mesh"], d["eps_inf"], out[i:], stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.abs(got - ref) <= TOL * abs(ref)), (got, ref)


def test_noalloc_rejects_meshes_beyond_the_fixed_scratch():
    import torch
    from paper_2603_24860_gb300 import bse
    from synth import generate
    d = generate("si4")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(bse.BseError) as e:
        bse.bse_head_correction_noalloc(d["lattice"], [64, 64, 64], d["eps_inf"], out)
    assert e.value.code == bse.BSE_EINVAL
    assert "fixed scratch" in str(e.value)
    # a mesh whose point count overflows 32 bits, and one whose lattice columns
    # (third axis) are too long for one thread, are rejected before any launch
    for mesh in ([2, 1, 1 << 30], [1, 1, 1 << 20]):
        with pytest.raises(bse.BseError) as e:
            bse.bse_head_correction_noalloc(d["lattice"], mesh, d["eps_inf"], out)
        assert e.value.code == bse.BSE_EINVAL
