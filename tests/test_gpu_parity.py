"""Parity of the CUDA library (through the C ABI) with the CPU oracle.

Tolerances: integer tables bit-exact; FP64 floating point within 1e-10
relative to the largest element (H, H_mu, U_mu), eigenvalues within 1e-10 Ha,
spectra within 1e-9 relative L2."""
import json
import os

import numpy as np
import pytest

from conftest import oracle_case, oracle_h

pytestmark = pytest.mark.gpu

TOL = 1e-10
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "wdiv.json")))
SMALL = ["si2", "si4", "lif4", "mos2_331"]


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_2603_24860_gb300 import bse
    assert torch.cuda.is_available()
    ctxs = {}

    def get(name):
        if name not in ctxs:
            from synth import generate
            ctxs[name] = bse.bse_create(generate(name), stream=torch.cuda.current_stream())
        return ctxs[name]
    yield bse, torch, get
    for c in ctxs.values():
        bse.bse_destroy(c)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("name", SMALL)
def test_tables_bit_exact(gpu, name):
    bse, torch, get = gpu
    t = bse.bse_tables(get(name))
    d, inp, grp, mt, b = oracle_case(name)
    chi, dims, cls = grp.characters()
    assert np.array_equal(t["rotk"], mt.rotk)
    assert np.array_equal(t["star_of_k"], mt.star_of)
    assert np.array_equal(t["star_rep"], mt.star_rep)
    assert np.array_equal(t["s_k"], mt.s_k)
    assert np.array_equal(t["class_of_op"], cls)
    assert np.array_equal(t["chi"], chi)
    assert np.array_equal(t["irrep_dim"], dims)
    vec = grp.vector_character()
    assert np.array_equal(t["bright"], np.rint(chi @ vec / grp.n).astype(int))
    assert np.array_equal(t["block_dim"], [b.basis(mu)[0].shape[1] for mu in range(len(dims))])
    orb = np.zeros(inp.N, dtype=np.int64)
    for o, mem in enumerate(b.orbits):
        orb[mem] = o
    assert np.array_equal(t["orbit_of"], orb)
    assert t["n_orbits"] == len(b.orbits)
    # folds of the rotated mesh points (Eq. sk) and the coset spheres S_k, S_q
    assert np.array_equal(t["fold"], mt.fold)
    assert np.array_equal(t["npw"], d["nk_count"]) and np.array_equal(t["ng"], d["ng_count"])
    for k in range(inp.nk):
        assert np.array_equal(t["gk"][k, :t["npw"][k]], np.asarray(d["gk"])[k, :d["nk_count"][k]])
        assert np.array_equal(t["gq"][k, :t["ng"][k]], np.asarray(d["gq"])[k, :d["ng_count"][k]])


@pytest.mark.parametrize("name", ["si2", "si4", "lif4", "mos2_331", "mos2_331_uni", "si8", "lif10"])
def test_head_correction(gpu, name):
    bse, torch, get = gpu
    w = bse.bse_tables(get(name))["w_div"]
    assert abs(w - GOLD[name]) <= TOL * abs(GOLD[name])


@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("bands", [0, 1, 2])
def test_pair_densities(gpu, name, bands):
    bse, torch, get = gpu
    from oracle.hamiltonian import pair_density
    d, inp, grp, mt, b = oracle_case(name)
    rng = np.random.default_rng(11)
    k = np.concatenate([[0, inp.nk - 1, 1], rng.integers(0, inp.nk, 13)]).astype(np.int32)
    kp = np.concatenate([[0, 0, inp.nk - 1], rng.integers(0, inp.nk, 13)]).astype(np.int32)
    nv, nc = inp.nv, inp.nc
    sets = {0: (range(nv, nv + nc), range(nv, nv + nc)), 1: (range(nv), range(nv)), 2: (range(nv, nv + nc), range(nv))}
    n, npr = (len(x) for x in sets[bands])
    ngmax = inp.gq.shape[1]
    out = torch.zeros((len(k), n, npr, ngmax), dtype=torch.complex128, device="cuda")
    bse.bse_pairdens(get(name), k, kp, bands, out)
    got = out.cpu().numpy()
    for i in range(len(k)):
        ref, q = pair_density(inp, mt, int(k[i]), int(kp[i]), *sets[bands])
        ng = ref.shape[2]
        assert np.abs(got[i, :, :, :ng] - ref).max() < 1e-13
        assert np.all(got[i, :, :, ng:] == 0)
    # the FP32 densities of the mixed builds (FP32 coefficients, FP32 sums of about 50 terms)
    for prec in (bse.BSE_FP32, bse.BSE_FP16_SPLIT):
        out32 = torch.zeros((len(k), n, npr, ngmax), dtype=torch.complex64, device="cuda")
        bse.bse_pairdens(get(name), k, kp, bands, out32, prec=prec)
        got32 = out32.cpu().numpy()
        for i in range(len(k)):
            ref, q = pair_density(inp, mt, int(k[i]), int(kp[i]), *sets[bands])
            ng = ref.shape[2]
            assert np.abs(got32[i, :, :, :ng] - ref).max() < 2e-6
            assert np.all(got32[i, :, :, ng:] == 0)


@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("terms", [1, 2, 4, 7])
def test_full_hamiltonian(gpu, name, terms):
    bse, torch, get = gpu
    code = "".join(c for bit, c in ((1, "d"), (2, "x"), (4, "w")) if terms & bit)
    ref = oracle_h(name, code)
    got = bse.full(get(name), terms).cpu().numpy()
    assert _rel(got, ref) <= TOL


@pytest.mark.parametrize("name", SMALL)
def test_basis(gpu, name):
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    mus = range(len(b.dims)) if name != "si4" else b.bright() + [0, 4]
    for mu in mus:
        U, _ = b.basis(mu)
        if U.shape[1] == 0:
            continue
        got = bse.basis(get(name), mu).cpu().numpy()
        assert got.shape == U.shape
        assert _rel(got, U) <= TOL


@pytest.mark.parametrize("name", SMALL)
def test_blocks(gpu, name):
    """H_mu = U_mu^dagger H U_mu for every irrep (si4: bright and two others)."""
    from oracle.projection import project
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    H = oracle_h(name)
    mus = range(len(b.dims)) if name != "si4" else b.bright() + [0, 4]
    for mu in mus:
        U, _ = b.basis(mu)
        ref = project(U, H)
        got = bse.block(get(name), mu).cpu().numpy()
        assert got.shape == ref.shape
        if ref.size:
            assert _rel(got, ref) <= TOL, (name, mu)


@pytest.mark.parametrize("terms", [1, 2, 4])
def test_block_terms(gpu, terms):
    from oracle.projection import project
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case("si4")
    code = "".join(c for bit, c in ((1, "d"), (2, "x"), (4, "w")) if terms & bit)
    mu = b.bright()[0]
    ref = project(b.basis(mu)[0], oracle_h("si4", code))
    got = bse.block(get("si4"), mu, terms=terms).cpu().numpy()
    assert _rel(got, ref) <= TOL


@pytest.mark.parametrize("name", SMALL)
def test_dipoles(gpu, name):
    from oracle.spectrum import dipoles
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    out = torch.empty(inp.N, dtype=torch.complex128, device="cuda")
    bse.bse_dipoles(get(name), out)
    assert _rel(out.cpu().numpy(), dipoles(inp, mt)) <= 1e-12


def _clusters(om, tol=1e-8):
    """Group indices of (sorted) eigenvalues closer than tol."""
    out, cur = [], [0]
    for i in range(1, len(om)):
        if om[i] - om[cur[-1]] <= tol:
            cur.append(i)
        else:
            out.append(cur)
            cur = [i]
    out.append(cur)
    return out


@pytest.mark.parametrize("name", SMALL)
def test_block_spectrum(gpu, name):
    from oracle.projection import project
    from oracle.spectrum import block_spectrum, dipoles
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    B = dipoles(inp, mt)
    omega = torch.tensor(d["omega"], device="cuda")
    ref, got = [], []
    for mu in b.bright():
        U, _ = b.basis(mu)
        if U.shape[1] == 0:
            continue
        ref.append(block_spectrum(inp, project(U, oracle_h(name)), U, B, d["omega"], d["eta"]))
        h = bse.block(get(name), mu)
        got.append([x.cpu().numpy() for x in bse.spectrum(get(name), mu, h, omega, d["eta"])])
    # a block can be dark for this polarisation; scale by the whole spectrum
    scale_osc = np.linalg.norm(B) ** 2
    scale_im = max(np.linalg.norm(r[2]) for r in ref)
    for (rom, rosc, rim), (om, osc, im) in zip(ref, got):
        assert np.abs(om - rom).max() <= TOL
        # oscillator strengths are basis independent only summed over degenerate levels
        for cl in _clusters(rom):
            assert abs(osc[cl].sum() - rosc[cl].sum()) <= 1e-9 * scale_osc
        assert np.linalg.norm(im - rim) <= 1e-9 * scale_im


def test_empty_block(gpu):
    """An irrep whose block is empty builds and solves to nothing."""
    bse, torch, get = gpu
    for name in SMALL:
        t = bse.bse_tables(get(name))
        empty = [mu for mu in range(t["n_irreps"]) if t["block_dim"][mu] == 0]
        if empty:
            h = bse.block(get(name), empty[0])
            assert h.shape == (0, 0)
            return
    pytest.skip("no empty irrep block among the small cases")


# --- FP32 direct term (CUDA cores); diagonal FP64, projection and exchange in
#     double-float (48-bit significand) ---
HA_MEV = 27211.386245988
TOL32 = 2e-6          # H_mu elements relative to the largest element


@pytest.mark.parametrize("name", SMALL)
def test_blocks_fp32(gpu, name):
    from oracle.projection import project
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    H = oracle_h(name)
    for mu in b.bright():
        U, _ = b.basis(mu)
        if U.shape[1] == 0:
            continue
        ref = project(U, H)
        got = bse.block(get(name), mu, prec=bse.BSE_FP32).cpu().numpy()
        assert _rel(got, ref) <= TOL32, (name, mu, _rel(got, ref))
        # exciton energies within 0.1 meV of the oracle
        assert np.abs(np.linalg.eigvalsh(got) - np.linalg.eigvalsh(ref)).max() * HA_MEV <= 0.1


@pytest.mark.parametrize("terms", [2, 4])
def test_block_terms_fp32(gpu, terms):
    """The FP32 mode changes the direct term; the exchange, projected in
    double-float (products exact, 48-bit sums), keeps the FP64 tolerance."""
    from oracle.projection import project
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case("si4")
    code = {2: "x", 4: "w"}[terms]
    mu = b.bright()[0]
    ref = project(b.basis(mu)[0], oracle_h("si4", code))
    got = bse.block(get("si4"), mu, prec=bse.BSE_FP32, terms=terms).cpu().numpy()
    assert _rel(got, ref) <= (TOL * 10 if terms == 2 else 1e-5)


# --- partner (row) blocks of every irrep ---

@pytest.mark.parametrize("name", SMALL)
def test_partner_blocks(gpu, name):
    """Partner blocks of every irrep (Cartesian irrep matrices for the
    polar-vector irreps, the regular-representation copy for the others)
    against the oracle's U_1^dagger H U_1 with the same canonical matrices;
    levels d-fold equal to the whole block's; dark irreps carry no strength."""
    from oracle.projection import PartnerBasis, partner_spectrum
    from oracle.spectrum import dipoles
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    t = bse.bse_tables(get(name))
    H = oracle_h(name)
    B = dipoles(inp, mt)
    omega = torch.tensor(d["omega"], device="cuda")
    for mu in range(len(b.dims)):
        pb = PartnerBasis(b, mu)
        assert t["partner_dim"][mu] == pb.U[0].shape[1]
        if pb.U[0].shape[1] == 0:
            continue
        ref = pb.U[0].conj().T @ H @ pb.U[0]
        for prec, tol in ((bse.BSE_FP64, TOL), (bse.BSE_FP32, TOL32)):
            got = bse.partner_block(get(name), mu, prec=prec).cpu().numpy()
            assert _rel(got, ref) <= tol, (name, mu, prec)
        h1 = bse.partner_block(get(name), mu)
        om, osc, im = (x.cpu().numpy() for x in bse.partner_spectrum(get(name), mu, h1, omega, d["eta"]))
        rom, rosc, rim = partner_spectrum(inp, ref, pb.U, B, d["omega"], d["eta"])
        assert np.abs(om - rom).max() <= TOL
        for cl in _clusters(rom):
            assert abs(osc[cl].sum() - rosc[cl].sum()) <= 1e-9 * np.linalg.norm(B) ** 2
        if not t["bright"][mu]:
            assert np.all(osc == 0.0)
        # the same spectrum as the whole irrep block
        hb = bse.block(get(name), mu)
        bom, bosc, bim = (x.cpu().numpy() for x in bse.spectrum(get(name), mu, hb, omega, d["eta"]))
        assert np.abs(np.repeat(om, pb.d) - bom).max() <= TOL
        scale = max(np.linalg.norm(bim), np.linalg.norm(B) ** 2 * 1e-3)
        assert np.linalg.norm(im - bim) <= 1e-9 * scale


@pytest.mark.parametrize("name", SMALL)
def test_partner_dims_every_irrep(gpu, name):
    """Every irrep has a partner block: d_mu partner_dim = block_dim."""
    bse, torch, get = gpu
    t = bse.bse_tables(get(name))
    assert np.all(t["partner_dim"] * t["irrep_dim"] == t["block_dim"])


# --- split-precision tensor-core direct term (tcgen05), FP32 accumulation ---
# H_mu elements relative to the largest element: bf16 hi + lo keeps about 16
# significant bits of every operand, fp16 hi + lo about 22 (the pair densities
# themselves are FP32), so fp16 split sits near the FP32 path.
SPLIT = {"bf16": ("BSE_BF16_SPLIT", 2e-5, 2e-4), "fp16": ("BSE_FP16_SPLIT", 4e-6, 2e-5)}


@pytest.mark.parametrize("split", ["bf16", "fp16"])
@pytest.mark.parametrize("name", ["si2", "si4", "lif4", "mos2_331"])
def test_blocks_split(gpu, name, split):
    """Split-precision blocks against the oracle; mos2_331 (NG = 102) takes
    the two-pairs-per-CTA plan of the tensor-core kernel, the others four."""
    from oracle.projection import PartnerBasis, project
    bse, torch, get = gpu
    prec, tol, _ = SPLIT[split]
    prec = getattr(bse, prec)
    d, inp, grp, mt, b = oracle_case(name)
    H = oracle_h(name)
    for mu in b.bright():
        U, _ = b.basis(mu)
        if U.shape[1] == 0:
            continue
        ref = project(U, H)
        got = bse.block(get(name), mu, prec=prec).cpu().numpy()
        assert _rel(got, ref) <= tol, (name, mu, _rel(got, ref))
        assert np.abs(np.linalg.eigvalsh(got) - np.linalg.eigvalsh(ref)).max() * HA_MEV <= 0.1
        pb = PartnerBasis(b, mu)
        ref1 = pb.U[0].conj().T @ H @ pb.U[0]
        got1 = bse.partner_block(get(name), mu, prec=prec).cpu().numpy()
        assert _rel(got1, ref1) <= tol


@pytest.mark.parametrize("split", ["bf16", "fp16"])
def test_split_direct_term_only(gpu, split):
    """The split modes change only the direct term."""
    from oracle.projection import project
    bse, torch, get = gpu
    prec, _, tol = SPLIT[split]
    d, inp, grp, mt, b = oracle_case("si4")
    mu = b.bright()[0]
    ref = project(b.basis(mu)[0], oracle_h("si4", "w"))
    got = bse.block(get("si4"), mu, prec=getattr(bse, prec), terms=4).cpu().numpy()
    assert _rel(got, ref) <= tol      # relative to the largest element of K^d alone


def test_fp16_split_more_accurate_than_bf16(gpu):
    """fp16 hi + lo carries 22 significant bits against bf16's 16, so its
    K^d is closer to the oracle's."""
    from oracle.projection import project
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case("lif4")
    mu = b.bright()[0]
    ref = project(b.basis(mu)[0], oracle_h("lif4", "w"))
    e16 = _rel(bse.block(get("lif4"), mu, prec=bse.BSE_FP16_SPLIT, terms=4).cpu().numpy(), ref)
    ebf = _rel(bse.block(get("lif4"), mu, prec=bse.BSE_BF16_SPLIT, terms=4).cpu().numpy(), ref)
    assert e16 < 0.25 * ebf, (e16, ebf)


def test_split_scales_are_exact(gpu):
    """The fp16 operands are scaled by powers of two: W(q) multiplied by 2^20
    (far outside fp16's range before scaling) gives K^d multiplied by 2^20
    to rounding, and the build stays finite."""
    from synth import generate
    bse, torch, get = gpu
    d = dict(generate("si2"))
    t = bse.bse_tables(get("si2"))
    mu = int(np.nonzero(t["bright"])[0][0])
    ref = bse.block(get("si2"), mu, prec=bse.BSE_FP64, terms=4).cpu().numpy()
    d["w"] = np.asarray(d["w"]) * 2.0 ** 20
    ctx = bse.bse_create(d, stream=torch.cuda.current_stream())
    try:
        got = bse.block(ctx, mu, prec=bse.BSE_FP16_SPLIT, terms=4).cpu().numpy()
    finally:
        bse.bse_destroy(ctx)
    assert np.all(np.isfinite(got))
    assert _rel(got * 2.0 ** -20, ref) <= 2e-5


@pytest.mark.parametrize("split", ["BSE_BF16_SPLIT", "BSE_FP16_SPLIT"])
def test_split_rejects_large_spheres(gpu, split):
    """W(q) with more than 128 plane waves does not fit one M = 128 MMA tile:
    EUNSUPPORTED, and the context stays usable."""
    from fractions import Fraction
    from synth import generate
    from synth.generate import CONFIGS, Config
    bse, torch, get = gpu
    base = CONFIGS["si4"]
    cfg = Config("si2_r52", "Si", (2, 2, 2), 4, 4, Fraction(26, 5), base.gap_ev, base.eps_inf, base.seed + 100)
    d = generate(cfg)
    assert np.asarray(d["gq"]).shape[1] > 128
    ctx = bse.bse_create(d, stream=torch.cuda.current_stream())
    try:
        t = bse.bse_tables(ctx)
        mu = int(np.nonzero(t["bright"])[0][0])
        n = max(int(t["block_dim"][mu]), 1)
        buf = torch.empty(n * n, dtype=torch.complex128, device="cuda")
        with pytest.raises(bse.BseError) as e:
            bse.bse_build_block(ctx, mu, getattr(bse, split), bse.BSE_TERM_ALL, buf, n)
        assert e.value.code == bse.BSE_EUNSUPPORTED
        bse.bse_build_block(ctx, mu, bse.BSE_FP32, bse.BSE_TERM_ALL, buf, n)
    finally:
        bse.bse_destroy(ctx)


@pytest.mark.parametrize("name", ["si4", "lif4", "mos2_331"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_all_blocks_one_build(gpu, name, prec):
    """Every irrep block and every partner block from one bse_build_blocks
    call: each equals the oracle's U^dagger H U and the single-target build
    of the same block."""
    from oracle.projection import PartnerBasis, project
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    H = oracle_h(name)
    p = bse.BSE_FP64 if prec == "fp64" else bse.BSE_FP32
    tol = TOL if prec == "fp64" else TOL32
    ctx = get(name)
    t = bse.bse_tables(ctx)
    n_ir = len(b.dims)
    targets = [(mu, 0) for mu in range(n_ir)] + [(mu, 1) for mu in range(n_ir)]
    dims = [int(t["partner_dim" if pt else "block_dim"][mu]) for mu, pt in targets]
    bufs = [torch.empty(max(n * n, 1), dtype=torch.complex128, device="cuda") for n in dims]
    bse.bse_build_blocks(ctx, [mu for mu, _ in targets], [pt for _, pt in targets], p, bse.BSE_TERM_ALL,
                         bufs, [max(n, 1) for n in dims])
    for (mu, pt), buf, n in zip(targets, bufs, dims):
        got = bse.colmajor(buf, n, n, max(n, 1)).cpu().numpy()
        U = PartnerBasis(b, mu).U[0] if pt else b.basis(mu)[0]
        assert got.shape == (U.shape[1],) * 2
        if n == 0:
            continue
        ref = project(U, H)
        assert _rel(got, ref) <= tol, (name, mu, pt, _rel(got, ref))
        single = (bse.partner_block if pt else bse.block)(ctx, mu, prec=p).cpu().numpy()
        assert np.abs(got - single).max() <= 1e-13 * np.abs(single).max(), (name, mu, pt)


def test_build_blocks_arguments(gpu):
    bse, torch, get = gpu
    ctx = get("si4")
    bse.bse_build_blocks(ctx, [], None, bse.BSE_FP64, bse.BSE_TERM_ALL, [], [])
    with pytest.raises(RuntimeError):
        bse.bse_build_blocks(ctx, [99], None, bse.BSE_FP64, bse.BSE_TERM_ALL, [None], [1])
    mu = int(np.nonzero(bse.bse_tables(ctx)["bright"])[0][0])
    n = int(bse.bse_tables(ctx)["block_dim"][mu])
    buf = torch.empty(n * n, dtype=torch.complex128, device="cuda")
    with pytest.raises(RuntimeError):
        bse.bse_build_blocks(ctx, [mu], None, bse.BSE_FP64, bse.BSE_TERM_ALL, [buf], [n - 1])
    with pytest.raises(RuntimeError):
        bse.bse_build_blocks(ctx, [mu], None, bse.BSE_FP64, bse.BSE_TERM_ALL, [None], [n])


@pytest.mark.parametrize("name", SMALL)
def test_solver_choice_and_agreement(gpu, name):
    """AUTO solves partner blocks without eigenvectors (tridiagonal
    reduction from the dipole direction) and whole blocks of bright
    multi-dimensional irreps with the dense solver; forcing either solver
    on a partner block gives the same levels, strengths and spectrum."""
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    ctx = get(name)
    t = bse.bse_tables(ctx)
    omega = torch.tensor(d["omega"], device="cuda")
    for mu in b.bright():
        if t["partner_dim"][mu] == 0:
            continue
        h1 = bse.partner_block(ctx, mu)
        out = {}
        for solver in (bse.BSE_SOLVER_AUTO, bse.BSE_SOLVER_DENSE, bse.BSE_SOLVER_TRIDIAG,
                       bse.BSE_SOLVER_TRIDIAG_BLOCKED, bse.BSE_SOLVER_TRIDIAG_BLOCKED_DF,
                       bse.BSE_SOLVER_TRIDIAG_TWOSTAGE):
            bse.bse_set_solver(ctx, solver)
            out[solver] = [x.cpu().numpy() for x in bse.partner_spectrum(ctx, mu, h1, omega, d["eta"])]
            used = bse.bse_get_stats(ctx)["solver"]
            assert used == (bse.BSE_SOLVER_DENSE if solver == bse.BSE_SOLVER_DENSE else bse.BSE_SOLVER_TRIDIAG)
        bse.bse_set_solver(ctx, bse.BSE_SOLVER_AUTO)
        # the reduction in shared memory and the blocked (panel) reduction with its tensor-core
        # and its double-float panel update, all against zheevd
        for other in (bse.BSE_SOLVER_TRIDIAG, bse.BSE_SOLVER_TRIDIAG_BLOCKED, bse.BSE_SOLVER_TRIDIAG_BLOCKED_DF,
                      bse.BSE_SOLVER_TRIDIAG_TWOSTAGE):
            (om, osc, im), (om2, osc2, im2) = out[bse.BSE_SOLVER_DENSE], out[other]
            assert np.abs(om - om2).max() <= TOL
            for cl in _clusters(om):
                assert abs(osc[cl].sum() - osc2[cl].sum()) <= 1e-10 * max(osc.sum(), 1e-300)
            assert np.linalg.norm(im - im2) <= 1e-9 * max(np.linalg.norm(im), 1e-300)
        if t["irrep_dim"][mu] > 1:
            hb = bse.block(ctx, mu)
            bse.spectrum(ctx, mu, hb, omega, d["eta"])
            assert bse.bse_get_stats(ctx)["solver"] == bse.BSE_SOLVER_DENSE


@pytest.mark.parametrize("name", SMALL)
def test_dark_blocks_levels_only(gpu, name):
    """Irreps outside the polar-vector representation: levels from the
    tridiagonal path equal the oracle's eigenvalues, strengths are 0."""
    from oracle.projection import project
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    ctx = get(name)
    H = oracle_h(name)
    omega = torch.tensor(d["omega"], device="cuda")
    bright = set(b.bright())
    for mu in range(len(b.dims)):
        U, _ = b.basis(mu)
        if mu in bright or U.shape[1] == 0:
            continue
        ref = np.linalg.eigvalsh(project(U, H))
        h = bse.block(ctx, mu)
        om, osc, im = (x.cpu().numpy() for x in bse.spectrum(ctx, mu, h, omega, d["eta"]))
        assert bse.bse_get_stats(ctx)["solver"] == bse.BSE_SOLVER_TRIDIAG
        assert np.abs(om - ref).max() <= TOL * max(np.abs(ref).max(), 1.0), (name, mu)
        assert np.all(osc == 0.0) and np.all(im == 0.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp16"])
def test_batched_build_small(gpu, prec):
    """Blocks of several contexts (Oh and D6h cells, whole and partner
    blocks) from one graph launch equal the single-context builds, and in
    FP64 and the split modes the oracle; a second launch of the same graph
    gives the same."""
    from oracle.projection import PartnerBasis, project
    bse, torch, get = gpu
    p = {"fp64": bse.BSE_FP64, "fp32": bse.BSE_FP32, "bf16": bse.BSE_BF16_SPLIT, "fp16": bse.BSE_FP16_SPLIT}[prec]
    tol_oracle = {"fp64": TOL, "fp32": None, "bf16": SPLIT["bf16"][1], "fp16": SPLIT["fp16"][1]}[prec]
    names = ["si2", "si4", "lif4", "mos2_331", "si4"]
    ctxs = [get(nm) for nm in names]
    targets = []
    for i, (nm, c) in enumerate(zip(names, ctxs)):
        t = bse.bse_tables(c)
        mu = int(np.nonzero(t["bright"])[0][0])
        pt = int(i % 2 == 1 and t["partner_dim"][mu] > 0)
        targets.append((mu, pt, int(t["partner_dim" if pt else "block_dim"][mu])))
    bufs = [torch.full((max(n * n, 1),), float("nan"), dtype=torch.complex128, device="cuda") for _, _, n in targets]
    lds = [max(n, 1) for _, _, n in targets]
    batch = bse.bse_batch_create(ctxs, [m for m, _, _ in targets], [pt for _, pt, _ in targets], p,
                                 bse.BSE_TERM_ALL, bufs, lds)
    try:
        assert bse.bse_batch_kernels(batch) >= 1 + 2 * len(names)
        bse.bse_batch_run(batch)
        torch.cuda.synchronize()
        first = [b.clone() for b in bufs]
        bse.bse_batch_run(batch)
        torch.cuda.synchronize()
    finally:
        bse.bse_batch_destroy(batch)
    for (mu, pt, n), b, f, nm, c in zip(targets, bufs, first, names, ctxs):
        got = bse.colmajor(b, n, n, max(n, 1)).cpu().numpy()
        assert torch.equal(b, f)
        single = (bse.partner_block if pt else bse.block)(c, mu, prec=p).cpu().numpy()
        assert np.abs(got - single).max() <= 1e-13 * np.abs(single).max(), (nm, mu, pt)
        if tol_oracle is not None:
            d, inp, grp, mt, bb = oracle_case(nm)
            U = PartnerBasis(bb, mu).U[0] if pt else bb.basis(mu)[0]
            assert _rel(got, project(U, oracle_h(nm))) <= tol_oracle, (nm, mu, pt)


def test_batched_build_arguments(gpu):
    bse, torch, get = gpu
    ctxs = [get("si2"), get("si4")]
    mus = [int(np.nonzero(bse.bse_tables(c)["bright"])[0][0]) for c in ctxs]
    dims = [int(bse.bse_tables(c)["block_dim"][m]) for c, m in zip(ctxs, mus)]
    bufs = [torch.empty(n * n, dtype=torch.complex128, device="cuda") for n in dims]
    with pytest.raises(bse.BseError) as e:
        bse.bse_build_blocks_batched(ctxs, mus, None, 7, bse.BSE_TERM_ALL, bufs, dims)
    assert e.value.code == bse.BSE_EUNSUPPORTED
    with pytest.raises(bse.BseError) as e:
        bse.bse_build_blocks_batched(ctxs, mus, None, bse.BSE_FP64, bse.BSE_TERM_ALL, bufs, [dims[0] - 1, dims[1]])
    assert e.value.code == bse.BSE_EINVAL
    # the one-shot form equals the single builds
    bse.bse_build_blocks_batched(ctxs, mus, None, bse.BSE_FP64, bse.BSE_TERM_ALL, bufs, dims)
    for c, m, b, n in zip(ctxs, mus, bufs, dims):
        single = bse.block(c, m).cpu().numpy()
        assert np.abs(bse.colmajor(b, n, n, n).cpu().numpy() - single).max() <= 1e-13 * np.abs(single).max()


@pytest.mark.parametrize("name", ["si4", "lif4", "mos2_331"])
def test_all_blocks_packed(gpu, name):
    """bse_build_block(BSE_IRREP_ALL) packs every block in irrep order; each
    equals the oracle's projection."""
    from oracle.projection import project
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    ctx = get(name)
    assert bse.bse_block_dim(ctx, bse.BSE_IRREP_ALL) == inp.N
    dims = [bse.bse_block_dim(ctx, mu) for mu in range(len(b.dims))]
    assert sum(dims) == inp.N
    buf = torch.empty(sum(n * n for n in dims), dtype=torch.complex128, device="cuda")
    bse.bse_build_block(ctx, bse.BSE_IRREP_ALL, bse.BSE_FP64, bse.BSE_TERM_ALL, buf, 0)
    H = oracle_h(name)
    off = 0
    for mu, n in enumerate(dims):
        if n:
            got = buf[off:off + n * n].view(n, n).transpose(0, 1).cpu().numpy()
            assert _rel(got, project(b.basis(mu)[0], H)) <= TOL, (name, mu)
        off += n * n


@pytest.mark.parametrize("name", SMALL)
def test_seeds_match_all_pairs(gpu, name):
    """Eq. Wtrafo: blocks from one k pair per symmetry orbit plus rotated
    blocks equal the pair-by-pair build (FP64 and FP32), and the seeds are a
    fraction of the pairs."""
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    ctx = get(name)
    t = bse.bse_tables(ctx)
    for mu in b.bright():
        if t["block_dim"][mu] == 0:
            continue
        w_on = bse.bse_build_work(ctx, mu)
        bse.bse_set_seeds(ctx, False)
        try:
            w_off = bse.bse_build_work(ctx, mu)
            off = {p: bse.block(ctx, mu, prec=p).cpu().numpy() for p in (bse.BSE_FP64, bse.BSE_FP32)}
        finally:
            bse.bse_set_seeds(ctx, True)
        on = {p: bse.block(ctx, mu, prec=p).cpu().numpy() for p in (bse.BSE_FP64, bse.BSE_FP32)}
        assert w_on["k_pairs"] == w_off["k_pairs"] == w_on["seeds"] + w_on["rotated"]
        assert w_off["rotated"] == 0 and w_off["seeds"] == w_off["k_pairs"]
        if grp.n > 1 and inp.nk > 1:
            assert w_on["seeds"] < w_on["k_pairs"]
        assert _rel(on[bse.BSE_FP64], off[bse.BSE_FP64]) <= 1e-12, (name, mu)
        assert _rel(on[bse.BSE_FP32], off[bse.BSE_FP32]) <= 2e-6, (name, mu)


@pytest.mark.parametrize("name", SMALL)
def test_loss_spectrum(gpu, name):
    """Longitudinal levels (Eq. secular), strengths (Eq. eigenvec_xi) and the
    loss spectrum from the partner-block levels against the oracle."""
    from oracle import loss
    from oracle.projection import PartnerBasis, project
    from oracle.spectrum import dipoles
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case(name)
    ctx = get(name)
    t = bse.bse_tables(ctx)
    H = oracle_h(name)
    B = dipoles(inp, mt)
    scale = np.linalg.norm(B) ** 2
    omega = torch.tensor(d["omega"], device="cuda")
    checked = 0
    for mu in b.bright():
        if t["partner_dim"][mu] == 0:
            continue
        pb = PartnerBasis(b, mu)
        Hm = project(pb.U[0], H)
        Om, a = np.linalg.eigh(Hm)
        osc = sum(np.abs(a.T @ (U.T @ B)) ** 2 for U in pb.U)
        ref_l, ref_w = loss.secular_levels(Om, osc, loss.loss_alpha(inp))
        ref_s = loss.loss_spectrum(inp, ref_l, ref_w, d["omega"], d["eta"])
        h1 = bse.partner_block(ctx, mu)
        om, os_, _ = bse.partner_spectrum(ctx, mu, h1, omega, d["eta"])
        gl, gw, gs = (x.cpu().numpy() for x in bse.loss_spectrum(ctx, om, os_, omega, d["eta"]))
        assert np.abs(gl - ref_l).max() <= TOL * max(np.abs(ref_l).max(), 1.0), (name, mu)
        assert np.abs(gw - ref_w).max() <= 1e-9 * scale, (name, mu)
        assert np.linalg.norm(gs - ref_s) <= 1e-9 * max(np.linalg.norm(ref_s), scale * 1e-3), (name, mu)
        assert abs(gw.sum() - os_.cpu().numpy().sum()) <= 1e-9 * scale
        checked += 1
    assert checked >= 1


def test_blocks_uniaxial_head_correction(gpu):
    """The MoS2-like cell with a uniaxial dielectric tensor diag(15, 15, 6):
    the library's H00 (Gauss-Legendre quadrature of Eq. hinv0) and orbit sum
    enter the diagonal of every block exactly as the oracle's W^div does."""
    from oracle.projection import project
    bse, torch, get = gpu
    d, inp, grp, mt, b = oracle_case("mos2_331_uni")
    assert abs(bse.bse_tables(get("mos2_331_uni"))["w_div"] - GOLD["mos2_331_uni"]) <= TOL * GOLD["mos2_331_uni"]
    H = oracle_h("mos2_331_uni")
    for mu in range(len(b.dims)):
        U, _ = b.basis(mu)
        if U.shape[1] == 0:
            continue
        got = bse.block(get("mos2_331_uni"), mu).cpu().numpy()
        assert _rel(got, project(U, H)) <= TOL, mu
