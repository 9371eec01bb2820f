"""Lanczos-Haydock spectrum on the GPU (bse_block_spectrum_lanczos) against
the oracle's recurrence and continued fraction (oracle/haydock.py), and
against the exact spectrum of the block."""
import numpy as np
import pytest

from conftest import oracle_case, oracle_h
from synth import generate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_2603_24860_gb300 import bse
    assert torch.cuda.is_available()
    ctxs = {}

    def get(name):
        if name not in ctxs:
            ctxs[name] = bse.bse_create(generate(name), stream=torch.cuda.current_stream())
        return ctxs[name]
    yield bse, torch, get
    for c in ctxs.values():
        bse.bse_destroy(c)


def _oracle_block(name, mu):
    from oracle import projection as pj
    from oracle import spectrum as spc
    d, inp, grp, mt, b = oracle_case(name)
    U, _ = b.basis(mu)
    Hm = pj.project(U, oracle_h(name))
    c = np.conj(U.T @ spc.dipoles(inp, mt))
    return d, inp, Hm, c


@pytest.mark.parametrize("name,steps", [("si4", 24), ("mos2_331", 3), ("lif4", 16)])
def test_ritz_pairs_and_spectrum_match_the_oracle(gpu, name, steps):
    """On the oracle's own block: the GPU's Ritz values and Gauss weights are
    those of the oracle's Lanczos tridiagonal, and its Im eps (Lorentzian sum
    over the Ritz pairs) is the oracle's continued fraction."""
    from oracle import haydock as hk
    bse, torch, get = gpu
    ctx = get(name)
    t = bse.bse_tables(ctx)
    # the polar-vector irrep that carries the dipole weight for this qhat
    cands = [_oracle_block(name, int(m)) for m in np.nonzero(t["bright"])[0]]
    k = int(np.argmax([np.vdot(x[3], x[3]).real for x in cands]))
    mu = int(np.nonzero(t["bright"])[0][k])
    d, inp, Hm, c = cands[k]
    h = torch.tensor(Hm, device="cuda").T.contiguous().T      # column-major on the device
    omega = torch.tensor(d["omega"], device="cuda")
    rz, wt, im = (x.cpu().numpy() for x in bse.lanczos_spectrum(ctx, mu, h, omega, d["eta"], steps))
    a, bb, n2 = hk.lanczos(Hm, c, steps)
    th, w = hk.ritz(a, bb, n2)
    assert len(rz) == len(th)
    assert np.abs(rz - th).max() <= 1e-10 * max(np.abs(th).max(), 1.0)
    assert np.abs(wt - w).max() <= 1e-10 * n2
    ref = hk.haydock_spectrum(inp, a, bb, n2, d["omega"], d["eta"])
    assert np.linalg.norm(im - ref) <= 1e-9 * np.linalg.norm(ref)


def test_fraction_alone_equals_the_ritz_pole_sum(gpu):
    """Without Ritz pairs Im eps comes from the continued fraction alone; it
    equals the call with Ritz pairs and the oracle's fraction.  20 steps: two
    recurrences without reorthogonalisation, summed in different orders,
    stay within rounding of each other only until a Ritz value converges."""
    from oracle import haydock as hk
    bse, torch, get = gpu
    ctx = get("si4")
    t = bse.bse_tables(ctx)
    mu = int(np.nonzero(t["bright"])[0][0])
    d, inp, Hm, c = _oracle_block("si4", mu)
    h = torch.tensor(Hm, device="cuda").T.contiguous().T
    omega = torch.tensor(d["omega"], device="cuda")
    _, _, im_r = bse.lanczos_spectrum(ctx, mu, h, omega, d["eta"], 20)
    rz, wt, im_f = bse.lanczos_spectrum(ctx, mu, h, omega, d["eta"], 20, ritz=False)
    assert rz is None and wt is None
    im_r, im_f = im_r.cpu().numpy(), im_f.cpu().numpy()
    a, bb, n2 = hk.lanczos(Hm, c, 20)
    ref = hk.haydock_spectrum(inp, a, bb, n2, d["omega"], d["eta"])
    assert np.linalg.norm(im_f - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.linalg.norm(im_f - im_r) <= 1e-9 * np.linalg.norm(ref)


def test_partner_block_gives_the_same_recurrence(gpu):
    """The dipole measure of the whole T1u block equals that of its partner
    block (summed over partners), so both recurrences give the same Ritz
    pairs."""
    bse, torch, get = gpu
    ctx = get("si4")
    t = bse.bse_tables(ctx)
    mu = int(np.nonzero(t["bright"])[0][0])
    d = generate("si4")
    omega = torch.tensor(d["omega"], device="cuda")
    hb = bse.block(ctx, mu)
    h1 = bse.partner_block(ctx, mu)
    rz, wt, im = (x.cpu().numpy() for x in bse.lanczos_spectrum(ctx, mu, hb, omega, d["eta"], 20))
    rz1, wt1, im1 = (x.cpu().numpy() for x in bse.lanczos_spectrum(ctx, mu, h1, omega, d["eta"], 20, partner=True))
    assert np.abs(rz - rz1).max() <= 1e-9 * np.abs(rz).max()
    assert np.abs(wt - wt1).max() <= 1e-9 * wt.sum()
    assert np.linalg.norm(im - im1) <= 1e-8 * np.linalg.norm(im)


def test_full_length_is_exact_on_a_small_block(gpu):
    """As many steps as the block has rows: the recurrence spans the whole
    Krylov space (or stops early on an invariant subspace) and the spectrum
    is the exact one."""
    bse, torch, get = gpu
    ctx = get("si2")
    t = bse.bse_tables(ctx)
    mu = int(np.nonzero(t["bright"])[0][0])
    d = generate("si2")
    omega = torch.tensor(d["omega"], device="cuda")
    h1 = bse.partner_block(ctx, mu)
    n = h1.shape[0]
    rz, wt, im = (x.cpu().numpy() for x in bse.lanczos_spectrum(ctx, mu, h1, omega, d["eta"], n, partner=True))
    om, osc, ime = (x.cpu().numpy() for x in bse.partner_spectrum(ctx, mu, h1, omega, d["eta"]))
    assert len(rz) <= n
    assert abs(wt.sum() - osc.sum()) <= 1e-10 * osc.sum()
    assert np.linalg.norm(im - ime) <= 1e-7 * np.linalg.norm(ime)


@pytest.mark.parametrize("block", ["partner", "whole"])
def test_converges_to_the_exact_spectrum_si8(gpu, block):
    """The 806-dim partner block (and the 2418-dim whole block) of the Si-like
    8x8x8 mesh: 150 steps give Im eps within 1e-3 relative L2 of the exact
    spectrum of the same block, and the Gauss weights sum to |U^T B|^2."""
    bse, torch, get = gpu
    ctx = get("si8")
    t = bse.bse_tables(ctx)
    mu = int(np.nonzero(t["bright"])[0][0])
    d = generate("si8")
    omega = torch.tensor(d["omega"], device="cuda")
    partner = block == "partner"
    h = bse.partner_block(ctx, mu) if partner else bse.block(ctx, mu)
    _, osc, ref = (x.cpu().numpy() for x in (bse.partner_spectrum if partner else bse.spectrum)(
        ctx, mu, h, omega, d["eta"]))
    rz, wt, im = (x.cpu().numpy() for x in bse.lanczos_spectrum(ctx, mu, h, omega, d["eta"], 150, partner=partner))
    assert len(rz) == 150
    assert abs(wt.sum() - osc.sum()) <= 1e-9 * osc.sum()
    assert np.linalg.norm(im - ref) <= 1e-3 * np.linalg.norm(ref)


def test_dark_irrep_and_arguments(gpu):
    bse, torch, get = gpu
    ctx = get("si4")
    t = bse.bse_tables(ctx)
    dark = int(np.nonzero(t["bright"] == 0)[0][0])
    mu = int(np.nonzero(t["bright"])[0][0])
    d = generate("si4")
    omega = torch.tensor(d["omega"], device="cuda")
    hd = bse.block(ctx, dark)
    rz, wt, im = bse.lanczos_spectrum(ctx, dark, hd, omega, d["eta"], 5)
    assert rz.numel() == 0 and float(im.abs().max()) == 0.0
    h = bse.block(ctx, mu)
    n = h.shape[0]
    for steps in (0, n + 1):
        with pytest.raises(bse.BseError) as e:
            bse.lanczos_spectrum(ctx, mu, h, omega, d["eta"], steps)
        assert e.value.code == bse.BSE_EINVAL
