"""Full-size checks for the LiF-like rocksalt 10x10x10 mesh (Nv = 3, Nc = 6,
N = 18000): the blocks of all ten irreps of Oh from one build (one direct
pass shared by every block), in FP64, FP32 and both split precisions.  Their dimensions add up to
N; sampled star-pair sub-blocks of every irrep are compared with the oracle
(its canonical basis restricted to the two stars, U_a^dagger H_ab U_b); the
FP32 exciton energies of every block agree with the FP64 ones within
0.1 meV."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "wdiv.json")))
HA_MEV = 27211.386245988


@pytest.fixture(scope="module")
def lif10():
    import torch
    from paper_2603_24860_gb300 import bse
    from synth import generate
    from oracle.hamiltonian import Inputs
    from oracle.tables import Group, MeshTables, orbits
    d = generate("lif10")
    ctx = bse.bse_create(d, stream=torch.cuda.current_stream())
    t = bse.bse_tables(ctx)
    h64 = bse.blocks(ctx, prec=bse.BSE_FP64)
    h32 = bse.blocks(ctx, prec=bse.BSE_FP32)
    cols = [bse.bse_block_star_columns(ctx, mu) for mu in range(int(t["n_irreps"]))]
    inp = Inputs(d)
    grp = Group(d["rot"], d["tau"], d["lattice"])
    mt = MeshTables(grp, d["mesh"])
    orb = orbits(mt, inp.eps, inp.nv, inp.nc)
    yield bse, torch, ctx, t, h64, h32, cols, d, inp, grp, mt, orb
    bse.bse_destroy(ctx)


def test_dimensions(lif10):
    bse, torch, ctx, t, h64, h32, cols, d, inp, *_ = lif10
    assert sum(h.shape[0] for h in h64) == inp.N == 18000
    for mu, h in enumerate(h64):
        assert h.shape[0] == t["block_dim"][mu] == cols[mu][-1]
        if h.shape[0]:
            assert float(torch.max(torch.abs(h - h.conj().T)).item()) <= 1e-14 * float(torch.max(torch.abs(h)).item())


def test_head_correction(lif10):
    t = lif10[3]
    assert abs(t["w_div"] - GOLD["lif10"]) <= 1e-10 * GOLD["lif10"]


def test_sampled_sub_blocks_every_irrep(lif10):
    from oracle.hamiltonian import hamiltonian_block
    from oracle.projection import star_basis
    bse, torch, ctx, t, h64, h32, cols, d, inp, grp, mt, orb = lif10
    chi, dims, cls = grp.characters()
    sizes = np.array([len(s) for s in mt.stars])
    big = int(np.nonzero(sizes == 48)[0][0])
    mid = int(np.nonzero(sizes == 12)[0][0])
    small = int(np.nonzero(sizes == 6)[0][0])
    pairs = [(0, big), (small, mid), (mid, big), (big, big)]
    cache = {}
    checked = 0
    for a, b in pairs:
        if (a, b) not in cache:
            cache[(a, b)] = hamiltonian_block(inp, mt, [int(k) for k in mt.stars[a]],
                                              [int(k) for k in mt.stars[b]], GOLD["lif10"])
        Hab = cache[(a, b)]
        for mu in range(len(dims)):
            w = int(dims[mu]) / grp.n * np.conj(chi[mu])
            ra, Ua = star_basis(inp, grp, mt, orb, a, w)
            rb, Ub = star_basis(inp, grp, mt, orb, b, w)
            c = cols[mu]
            assert Ua.shape[1] == c[a + 1] - c[a] and Ub.shape[1] == c[b + 1] - c[b]
            if Ua.shape[1] == 0 or Ub.shape[1] == 0:
                continue
            ref = Ua.conj().T @ Hab @ Ub
            scale = float(torch.max(torch.abs(h64[mu])).item())
            sub = lambda h: h[c[a]:c[a + 1], c[b]:c[b + 1]].cpu().numpy()
            assert np.abs(sub(h64[mu]) - ref).max() <= 1e-10 * scale, (mu, a, b)
            assert np.abs(sub(h32[mu]) - ref).max() <= 2e-6 * scale, (mu, a, b)
            checked += 1
    assert checked >= 20


def test_fp32_levels_within_0p1_mev(lif10):
    bse, torch, ctx, t, h64, h32, *_ = lif10
    for mu in range(len(h64)):
        if h64[mu].shape[0] == 0:
            continue
        e64 = torch.linalg.eigvalsh(h64[mu]).cpu().numpy()
        e32 = torch.linalg.eigvalsh(h32[mu]).cpu().numpy()
        assert np.abs(e32 - e64).max() * HA_MEV <= 0.1, mu


@pytest.mark.parametrize("split", ["BSE_FP16_SPLIT", "BSE_BF16_SPLIT"])
def test_split_blocks_within_0p1_mev(lif10, split):
    """All ten blocks from one split-precision build (tensor-core direct
    term): elements within the split mode's tolerance of the FP64 blocks and
    exciton energies within 0.1 meV."""
    bse, torch, ctx, t, h64, *_ = lif10
    tol = {"BSE_FP16_SPLIT": 4e-6, "BSE_BF16_SPLIT": 2e-5}[split]
    hs = bse.blocks(ctx, prec=getattr(bse, split))
    for mu in range(len(h64)):
        if h64[mu].shape[0] == 0:
            continue
        err = (hs[mu] - h64[mu]).abs().max().item() / h64[mu].abs().max().item()
        assert err <= tol, (mu, err)
        e64 = torch.linalg.eigvalsh(h64[mu]).cpu().numpy()
        es = torch.linalg.eigvalsh(hs[mu]).cpu().numpy()
        assert np.abs(es - e64).max() * HA_MEV <= 0.1, mu
    del hs


def test_levels_of_every_block(lif10):
    """AUTO solves the nine dark blocks through the tridiagonal path (levels
    only) and the T1u block densely; all levels agree with cuSOLVER's
    eigenvalues of the same blocks."""
    bse, torch, ctx, t, h64, *_ = lif10
    import numpy as np
    d = lif10[7]
    omega = torch.tensor(d["omega"], device="cuda")
    for mu, h in enumerate(h64):
        if h.shape[0] == 0:
            continue
        om, osc, im = (x.cpu().numpy() for x in bse.spectrum(ctx, mu, h, omega, d["eta"]))
        ref = torch.linalg.eigvalsh(h).cpu().numpy()
        assert np.abs(om - ref).max() <= 1e-10 * np.abs(ref).max(), mu
        if not t["bright"][mu]:
            assert bse.bse_get_stats(ctx)["solver"] == bse.BSE_SOLVER_TRIDIAG
            assert np.all(osc == 0.0)
