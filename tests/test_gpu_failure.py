"""Failure handling through the C ABI, made on the host or by a wait limit
that runs out; nothing here faults, traps or hangs the GPU.

* Bounded device waits: bse_set_wait_limit(ctx, 0) makes every bounded wait
  give up at once (the grid barriers of the tridiagonal reduction and of the
  Lanczos recurrence, the mbarrier waits of the tensor-core direct kernel and
  of the tensor-core panel update).
  The call reports ETIMEOUT, and once the default limit is back the same
  context gives the oracle's results.
* Inputs that break the symmetry the method relies on (Sec. III.C): a cut
  multiplet, a band rescaled so that the band rotations are not unitary,
  energies that vary over a star, a set of operations that is not a group,
  and a q = 0 sphere without G = 0, each rejected by bse_create."""
import numpy as np
import pytest

from conftest import oracle_case, oracle_h

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2603_24860_gb300 import bse
    assert torch.cuda.is_available()
    return bse, torch


def _code(bse, fn, *args):
    try:
        fn(*args)
    except bse.BseError as e:
        return e.code
    return bse.BSE_OK


@pytest.mark.parametrize("solver,kind", [("BSE_SOLVER_TRIDIAG", 0), ("BSE_SOLVER_TRIDIAG_BLOCKED", 1),
                                         ("BSE_SOLVER_TRIDIAG_TWOSTAGE", 3)])
def test_tridiagonal_wait_gives_up_and_context_recovers(lib, solver, kind):
    """The 69-dim partner block of si4: the reduction in shared memory; the
    blocked one, whose tensor-core panel updates (after steps 30 and 62)
    give up at their first mbarrier wait, let their bulk copies land, free
    their tensor memory and return; and the two-stage one, whose tensor-core
    kernels do the same and whose bulge-chasing sweeps give up at their first
    wait for the sweep before."""
    from oracle.projection import PartnerBasis
    bse, torch = lib
    from synth import generate
    d, inp, grp, mt, b = oracle_case("si4")
    ctx = bse.bse_create(generate("si4"), stream=torch.cuda.current_stream())
    mu = b.bright()[0]
    bse.bse_set_solver(ctx, getattr(bse, solver))
    h = bse.partner_block(ctx, mu)
    omega = torch.tensor(d["omega"], device="cuda")
    bse.bse_set_wait_limit(ctx, 0)
    assert _code(bse, bse.partner_spectrum, ctx, mu, h, omega, d["eta"]) == bse.BSE_ETIMEOUT
    bse.bse_set_wait_limit(ctx, -1)
    om = bse.partner_spectrum(ctx, mu, h, omega, d["eta"])[0].cpu().numpy()
    pb = PartnerBasis(b, mu)
    ref = pb.U[0].conj().T @ oracle_h("si4") @ pb.U[0]
    assert np.abs(om - np.linalg.eigvalsh(ref)).max() <= TOL
    assert bse.bse_get_stats(ctx)["reduce_kind"] == kind
    bse.bse_destroy(ctx)


def test_lanczos_wait_gives_up_and_context_recovers(lib):
    bse, torch = lib
    from synth import generate
    d, inp, grp, mt, b = oracle_case("si4")
    ctx = bse.bse_create(generate("si4"), stream=torch.cuda.current_stream())
    mu = b.bright()[0]
    h = bse.partner_block(ctx, mu)
    n = h.shape[0]
    omega = torch.tensor(d["omega"], device="cuda")
    im = torch.empty(omega.numel(), dtype=torch.float64, device="cuda")
    bse.bse_set_wait_limit(ctx, 0)
    assert _code(bse, bse.bse_block_spectrum_lanczos, ctx, mu, 1, h, n, 20, omega, d["eta"], None, None,
                 im) == bse.BSE_ETIMEOUT
    bse.bse_set_wait_limit(ctx, -1)
    assert bse.bse_block_spectrum_lanczos(ctx, mu, 1, h, n, 20, omega, d["eta"], None, None, im) > 0
    assert np.all(np.isfinite(im.cpu().numpy()))
    bse.bse_destroy(ctx)


@pytest.mark.parametrize("split", ["BSE_BF16_SPLIT", "BSE_FP16_SPLIT"])
def test_tensor_core_wait_gives_up_and_context_recovers(lib, split):
    """The split-precision kernel gives up at its first mbarrier wait, lets
    the bulk copy it issued land, frees its tensor memory and returns; the
    build reports ETIMEOUT and the next build matches the oracle."""
    from oracle.projection import project
    bse, torch = lib
    from synth import generate
    d, inp, grp, mt, b = oracle_case("si4")
    ctx = bse.bse_create(generate("si4"), stream=torch.cuda.current_stream())
    mu = b.bright()[0]
    prec = getattr(bse, split)
    bse.bse_set_wait_limit(ctx, 0)
    assert _code(bse, bse.block, ctx, mu, prec) == bse.BSE_ETIMEOUT
    bse.bse_set_wait_limit(ctx, -1)
    got = bse.block(ctx, mu, prec=prec).cpu().numpy()
    ref = project(b.basis(mu)[0], oracle_h("si4"))
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
    bse.bse_destroy(ctx)


def test_wait_limit_arguments(lib):
    bse, torch = lib
    from synth import generate
    ctx = bse.bse_create(generate("si2"), stream=torch.cuda.current_stream())
    for polls in (-5, 0, 1, 1 << 50):
        bse.bse_set_wait_limit(ctx, polls)
    bse.bse_destroy(ctx)
    assert bse.lib().bse_set_wait_limit(None, 0) == bse.BSE_EINVAL


# --- inputs that break the symmetry (rejected at bse_create) ---

def _create_code(bse, torch, d):
    return _code(bse, bse.bse_create, d, torch.cuda.current_stream())


def test_cut_multiplet_is_rejected(lib):
    """Dropping the last conduction band cuts the threefold multiplet at
    Gamma: the band rotations restricted to the kept bands are not unitary."""
    bse, torch = lib
    from synth import generate
    d = dict(generate("si2"))
    e0 = np.asarray(d["eps"])[0]
    nb = d["nv"] + d["nc"]
    assert abs(e0[nb - 1] - e0[nb - 2]) < 1e-9   # the top band belongs to a multiplet
    d["coef"] = np.ascontiguousarray(np.asarray(d["coef"])[:, :nb - 1])
    d["eps"] = np.ascontiguousarray(np.asarray(d["eps"])[:, :nb - 1])
    d["nc"] = d["nc"] - 1
    assert _create_code(bse, torch, d) == bse.BSE_ESYMM


def test_non_unitary_band_rotation_is_rejected(lib):
    """One band at one k rescaled: <phi_sk|s phi_k> is no longer unitary."""
    bse, torch = lib
    from synth import generate
    d = dict(generate("si2"))
    coef = np.array(d["coef"])
    coef[1, 0] *= 1.1
    d["coef"] = coef
    assert _create_code(bse, torch, d) == bse.BSE_ESYMM


def test_energies_varying_in_a_star_are_rejected(lib):
    bse, torch = lib
    from synth import generate
    from oracle.tables import Group, MeshTables
    d = dict(generate("si4"))
    mt = MeshTables(Group(d["rot"], d["tau"], d["lattice"]), d["mesh"])
    star = next(s for s in mt.stars if len(s) > 1)
    eps = np.array(d["eps"])
    eps[int(star[-1]), 0] += 1e-4
    d["eps"] = eps
    assert _create_code(bse, torch, d) == bse.BSE_ESYMM


def test_operations_not_a_group_are_rejected(lib):
    """Removing one operation of Oh leaves a set that does not close."""
    bse, torch = lib
    from synth import generate
    d = dict(generate("si2"))
    d["rot"] = np.ascontiguousarray(np.asarray(d["rot"])[1:])
    d["tau"] = np.ascontiguousarray(np.asarray(d["tau"])[1:])
    assert _create_code(bse, torch, d) == bse.BSE_ESYMM


def test_sphere_without_g0_is_rejected(lib):
    """The q = 0 sphere of W must contain G = 0 (its head is replaced by
    W^div, Sec. III.B)."""
    bse, torch = lib
    from synth import generate
    d = dict(generate("si2"))
    gq = np.array(d["gq"])
    ng = np.array(d["ng_count"])
    g0 = int(np.nonzero(np.all(gq[0, :ng[0]] == 0, axis=1))[0][0])
    gq[0, g0] = gq[0, ng[0] - 1]
    ng[0] -= 1
    d["gq"], d["ng_count"] = gq, ng
    assert _create_code(bse, torch, d) == bse.BSE_EINVAL


def test_truncated_sizes_are_rejected(lib):
    """A plane-wave count beyond the capacity of the coefficient array."""
    bse, torch = lib
    from synth import generate
    d = dict(generate("si2"))
    npw = np.array(d["nk_count"])
    npw[3] = np.asarray(d["gk"]).shape[1] + 1
    d["nk_count"] = npw
    assert _create_code(bse, torch, d) == bse.BSE_EINVAL
