"""Full-size parity for the Si-like 8x8x8 mesh (Nv = 4, Nc = 6, N = 12288) in
the launch configuration the benchmark times: the whole T1u block is built
by bse_build_block and sampled star-pair sub-blocks are compared with the
oracle, which computes each one from its definition (U_a^dagger H_ab U_b)."""
import json
import os

import numpy as np
import pytest

from conftest import oracle_case

pytestmark = pytest.mark.gpu

TOL = 1e-10
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "wdiv.json")))


@pytest.fixture(scope="module")
def built():
    import torch
    from paper_2603_24860_gb300 import bse
    from synth import generate
    d = generate("si8")
    ctx = bse.bse_create(d, stream=torch.cuda.current_stream())
    t = bse.bse_tables(ctx)
    mu = int(np.nonzero(t["bright"])[0][0])
    h = bse.block(ctx, mu).cpu().numpy()
    yield bse, torch, ctx, t, mu, h
    bse.bse_destroy(ctx)


def test_block_dimension(built):
    bse, torch, ctx, t, mu, h = built
    d, inp, grp, mt, b = oracle_case("si8")
    assert mu == b.bright()[0]
    assert h.shape[0] == b.basis(mu)[0].shape[1] == t["block_dim"][mu]
    assert np.abs(h - h.conj().T).max() <= 1e-14 * np.abs(h).max()


def _star_cols(b, mt, mu):
    U, owner = b.basis(mu)
    star_of_orbit = np.array([mt.star_of[m[0] // (b.inp.nv * b.inp.nc)] for m in b.orbits])
    return U, star_of_orbit[owner]


@pytest.mark.parametrize("pair", ["gamma", "small-large", "large-large", "mid-mid"])
def test_sampled_star_pair_blocks(built, pair):
    from oracle.hamiltonian import hamiltonian_block
    bse, torch, ctx, t, mu, h = built
    d, inp, grp, mt, b = oracle_case("si8")
    sizes = np.array([len(s) for s in mt.stars])
    big = int(np.nonzero(sizes == 48)[0][0])
    mid = int(np.nonzero(sizes == 12)[0][0])
    small = int(np.nonzero(sizes == 6)[0][0])
    a, c = {"gamma": (0, 0), "small-large": (small, big), "large-large": (big, big), "mid-mid": (mid, mid)}[pair]
    U, col_star = _star_cols(b, mt, mu)
    ca, cb = np.nonzero(col_star == a)[0], np.nonzero(col_star == c)[0]
    if len(ca) == 0 or len(cb) == 0:
        pytest.skip("star carries no T1u vectors")
    B = inp.nv * inp.nc
    rows = np.concatenate([np.arange(k * B, (k + 1) * B) for k in mt.stars[a]])
    cols = np.concatenate([np.arange(k * B, (k + 1) * B) for k in mt.stars[c]])
    Hab = hamiltonian_block(inp, mt, list(mt.stars[a]), list(mt.stars[c]), GOLD["si8"])
    ref = U[np.ix_(rows, ca)].conj().T @ Hab @ U[np.ix_(cols, cb)]
    got = h[np.ix_(ca, cb)]
    assert np.abs(got - ref).max() <= TOL * np.abs(h).max()


def test_spectrum_sum_rule(built):
    """sum_lambda |B_lambda|^2 = |U_mu^T B|^2 and the spectrum is positive."""
    from oracle.spectrum import dipoles
    bse, torch, ctx, t, mu, h = built
    d, inp, grp, mt, b = oracle_case("si8")
    U, _ = b.basis(mu)
    bmu = U.T @ dipoles(inp, mt)
    hd = torch.tensor(h, device="cuda").T.contiguous().T
    omega = torch.tensor(d["omega"], device="cuda")
    om, osc, im = (x.cpu().numpy() for x in bse.spectrum(ctx, mu, hd, omega, d["eta"]))
    assert abs(osc.sum() - np.linalg.norm(bmu) ** 2) <= 1e-10 * np.linalg.norm(bmu) ** 2
    assert np.all(np.diff(om) >= -1e-14)
    assert np.all(im[d["omega"] > 0] > 0)


def test_fp32_build_within_0p1_mev(built):
    """FP32 direct term vs the FP64 build (itself pinned to the oracle above):
    exciton energies within 0.1 meV, spectra within 1e-3 relative L2."""
    bse, torch, ctx, t, mu, h = built
    d, inp, grp, mt, b = oracle_case("si8")
    h32 = bse.block(ctx, mu, prec=bse.BSE_FP32)
    h64 = torch.tensor(h, device="cuda").T.contiguous().T
    omega = torch.tensor(d["omega"], device="cuda")
    om64, osc64, im64 = (x.cpu().numpy() for x in bse.spectrum(ctx, mu, h64, omega, d["eta"]))
    om32, osc32, im32 = (x.cpu().numpy() for x in bse.spectrum(ctx, mu, h32, omega, d["eta"]))
    assert np.abs(om32 - om64).max() * 27211.386245988 <= 0.1
    assert np.linalg.norm(im32 - im64) <= 1e-3 * np.linalg.norm(im64)
    assert np.abs(h32.cpu().numpy() - h).max() <= 2e-6 * np.abs(h).max()


def test_partner_block_levels(built):
    """The T1u block is three copies of the partner block: levels and the
    spectrum agree with the whole block (built above in FP64)."""
    bse, torch, ctx, t, mu, h = built
    d, inp, grp, mt, b = oracle_case("si8")
    assert t["partner_dim"][mu] * 3 == t["block_dim"][mu]
    h1 = bse.partner_block(ctx, mu)
    omega = torch.tensor(d["omega"], device="cuda")
    om1, osc1, im1 = (x.cpu().numpy() for x in bse.partner_spectrum(ctx, mu, h1, omega, d["eta"]))
    hd = torch.tensor(h, device="cuda").T.contiguous().T
    om, osc, im = (x.cpu().numpy() for x in bse.spectrum(ctx, mu, hd, omega, d["eta"]))
    assert np.abs(np.repeat(om1, 3) - om).max() <= TOL
    assert abs(osc1.sum() - osc.sum()) <= 1e-10 * osc.sum()
    assert np.linalg.norm(im1 - im) <= 1e-9 * np.linalg.norm(im)


@pytest.mark.parametrize("split", ["BSE_BF16_SPLIT", "BSE_FP16_SPLIT"])
def test_split_build_within_0p1_mev(built, split):
    """Tensor-core split-precision direct term vs the FP64 build."""
    bse, torch, ctx, t, mu, h = built
    d, inp, grp, mt, b = oracle_case("si8")
    hb = bse.block(ctx, mu, prec=getattr(bse, split))
    h64 = torch.tensor(h, device="cuda").T.contiguous().T
    omega = torch.tensor(d["omega"], device="cuda")
    om64, osc64, im64 = (x.cpu().numpy() for x in bse.spectrum(ctx, mu, h64, omega, d["eta"]))
    omb, oscb, imb = (x.cpu().numpy() for x in bse.spectrum(ctx, mu, hb, omega, d["eta"]))
    assert np.abs(omb - om64).max() * 27211.386245988 <= 0.1
    assert np.linalg.norm(imb - im64) <= 1e-3 * np.linalg.norm(im64)


def test_partner_solvers_agree(built):
    """Levels and strengths of the partner block without eigenvectors
    (tridiagonal reduction held in shared memory across all SMs) against the
    dense eigensolver."""
    bse, torch, ctx, t, mu, h = built
    d, inp, grp, mt, b = oracle_case("si8")
    h1 = bse.partner_block(ctx, mu)
    omega = torch.tensor(d["omega"], device="cuda")
    out = {}
    kinds = {}
    for solver in (bse.BSE_SOLVER_DENSE, bse.BSE_SOLVER_TRIDIAG, bse.BSE_SOLVER_TRIDIAG_BLOCKED,
                   bse.BSE_SOLVER_TRIDIAG_BLOCKED_DF, bse.BSE_SOLVER_TRIDIAG_TWOSTAGE):
        bse.bse_set_solver(ctx, solver)
        out[solver] = [x.cpu().numpy() for x in bse.partner_spectrum(ctx, mu, h1, omega, d["eta"])]
        kinds[solver] = bse.bse_get_stats(ctx)["reduce_kind"]
    bse.bse_set_solver(ctx, bse.BSE_SOLVER_AUTO)
    assert kinds[bse.BSE_SOLVER_TRIDIAG_BLOCKED] == 1 and kinds[bse.BSE_SOLVER_TRIDIAG_BLOCKED_DF] == 2
    assert kinds[bse.BSE_SOLVER_TRIDIAG_TWOSTAGE] == 3
    # the reduction in shared memory, the blocked one (26 panels of 32 reflectors) with the
    # panel-end update from exact digit GEMMs on the tensor cores and in double-float, and the
    # two-stage one (band of half-bandwidth 32, then bulge chasing)
    for other in (bse.BSE_SOLVER_TRIDIAG, bse.BSE_SOLVER_TRIDIAG_BLOCKED, bse.BSE_SOLVER_TRIDIAG_BLOCKED_DF,
                  bse.BSE_SOLVER_TRIDIAG_TWOSTAGE):
        (om, osc, im), (om2, osc2, im2) = out[bse.BSE_SOLVER_DENSE], out[other]
        assert np.abs(om - om2).max() <= TOL * np.abs(om).max()
        assert np.abs(osc - osc2).max() <= 1e-9 * osc.sum()
        assert np.linalg.norm(im - im2) <= 1e-9 * np.linalg.norm(im)
        # the reduction and the bisection compute in double-float (48-bit
        # significand): backward error of order n 2^-47, far inside the tolerance
        assert np.abs(om - om2).max() <= len(om) * 2.0 ** -47 * np.abs(om).max()


def test_loss_levels_against_dense(built):
    """The secular-equation levels of H + alpha B* B^T on the 806-dim partner
    block against a dense eigensolution of that matrix (torch, FP64)."""
    import math
    bse, torch, ctx, t, mu, h = built
    d, inp, grp, mt, b = oracle_case("si8")
    h1 = bse.partner_block(ctx, mu)
    omega = torch.tensor(d["omega"], device="cuda")
    om, osc, _ = bse.partner_spectrum(ctx, mu, h1, omega, d["eta"])
    lv, lw, ls = bse.loss_spectrum(ctx, om, osc, omega, d["eta"])
    alpha = 4.0 * math.pi * 2 / inp.nk
    # the partner block's dipole projections are parallel: c = conj(U_1^T B) carries all the strength
    ev, vec = torch.linalg.eigh(h1)
    w = osc                                    # |a_l^T b|^2 in the eigenbasis (levels ascending)
    hp = torch.diag(ev) + alpha * torch.sqrt(w)[:, None] * torch.sqrt(w)[None, :]
    ref = torch.linalg.eigvalsh(hp).cpu().numpy()
    assert np.abs(lv.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    assert abs(lw.sum().item() - osc.sum().item()) <= 1e-9 * osc.sum().item()
