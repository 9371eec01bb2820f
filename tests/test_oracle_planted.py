"""Each plausible mistake planted in the oracle (on the CPU) is caught by one
of the pins of the other test files."""
import numpy as np

from conftest import oracle_case
from oracle import hamiltonian as hm
from oracle import projection as pj
from oracle import spectrum as spc
from test_oracle_hamiltonian import rho_fft


def _comm(b, K):
    return max(np.abs(r @ K - (r.T @ K.T).T).max() for r in b.reps) / np.abs(K).max()


def test_transposed_w_breaks_symmetry(monkeypatch):
    d, inp, grp, mt, b = oracle_case("si2")
    assert _comm(b, hm.direct_matrix(inp, mt)) < 1e-12
    orig = hm.w_of_q
    monkeypatch.setattr(hm, "w_of_q", lambda i, q: orig(i, q).T)
    assert _comm(b, hm.direct_matrix(inp, mt)) > 1e-6


def test_dropped_conjugate_breaks_hermiticity(monkeypatch):
    d, inp, grp, mt, b = oracle_case("si2")
    def bad(inp, mt, k, kp):
        nv, nc = inp.nv, inp.nc
        rc, q = hm.pair_density(inp, mt, k, kp, range(nv, nv + nc), range(nv, nv + nc))
        rv, _ = hm.pair_density(inp, mt, k, kp, range(nv), range(nv))
        blk = np.einsum("cdQ,QR,vwR->vcwd", rc, hm.w_of_q(inp, q), rv) / inp.volume
        return blk.reshape(nv * nc, nv * nc)
    monkeypatch.setattr(hm, "direct_block", bad)
    K = hm.direct_matrix(inp, mt)
    assert np.abs(K - K.conj().T).max() > 1e-6 * np.abs(K).max() or _comm(b, K) > 1e-6


def test_wrong_fold_fails_fft_route(monkeypatch):
    d, inp, grp, mt, b = oracle_case("si2")
    orig = mt.minus
    monkeypatch.setattr(mt, "minus", lambda k, kp: (orig(k, kp)[0], 0 * orig(k, kp)[1]))
    bad = [hm.pair_density(inp, mt, k, kp, range(inp.nb), range(inp.nb))[0]
           for k, kp in ((1, 0), (0, 1), (3, 5))]
    monkeypatch.setattr(mt, "minus", orig)
    ref = [rho_fft(d, k, kp, range(inp.nb), range(inp.nb)) for k, kp in ((1, 0), (0, 1), (3, 5))]
    assert max(np.abs(x - y).max() for x, y in zip(bad, ref)) > 1e-3


def test_wrong_phase_sign_breaks_unitarity(monkeypatch):
    d, inp, grp, mt, b = oracle_case("si2")
    tau = grp.tau.copy()
    monkeypatch.setattr(grp, "tau", -tau)
    worst = 0.0
    for s in range(grp.n):
        for k in range(inp.nk):
            g = pj.band_rotation(inp, grp, mt, s, k)
            worst = max(worst, np.abs(g.conj().T @ g - np.eye(inp.nb)).max())
    assert worst > 1e-3


def test_unconjugated_dipole_leaks_out_of_bright_block(monkeypatch):
    d, inp, grp, mt, b = oracle_case("si2")
    orig = np.conj
    B_good = spc.dipoles(inp, mt)
    monkeypatch.setattr(spc.np, "conj", lambda x: x)
    B_bad = spc.dipoles(inp, mt)
    monkeypatch.setattr(spc.np, "conj", orig)
    br = b.bright()
    leak = max(np.linalg.norm(b.basis(mu)[0].T @ B_bad)
               for mu in range(len(b.dims)) if mu not in br)
    assert leak > 1e-6 * np.linalg.norm(B_good)


def test_head_and_wings_ignored_at_q0():
    """A nonzero head/wing of W(q=0) in the input must not change H."""
    d, inp, grp, mt, b = oracle_case("si2")
    K0 = hm.direct_matrix(inp, mt)
    w = np.array(inp.w)
    g0 = int(np.nonzero(np.all(inp.gq[0, :inp.ngc[0]] == 0, axis=1))[0][0])
    w[0, g0, :inp.ngc[0]] = 5.0
    w[0, :inp.ngc[0], g0] = 5.0
    saved = inp.w
    inp.w = w
    try:
        K1 = hm.direct_matrix(inp, mt)
    finally:
        inp.w = saved
    assert np.abs(K1 - K0).max() == 0.0


def test_dropped_head_correction_in_sub_block_is_caught():
    """A sub-block builder that forgets -W^div on the diagonal (or takes the
    exchange vectors of the rows for the columns) fails the restriction pin of
    test_oracle_hamiltonian."""
    from conftest import oracle_h
    from test_oracle_hamiltonian import _block_cases, _sub_index, _wdiv_of
    d, inp, grp, mt, b = oracle_case("si4")
    H = oracle_h("si4")
    wd = _wdiv_of("si4")
    scale = np.abs(H).max()

    def no_head(rows, cols):
        same = _sub_index(inp, rows)[:, None] == _sub_index(inp, cols)[None, :]
        return hm.hamiltonian_block(inp, mt, rows, cols, wd) + wd * same

    def rows_for_cols(rows, cols):
        P, vbar = hm.exchange_vectors_for(inp, mt, rows)
        Pr, _ = hm.exchange_vectors_for(inp, mt, rows[:1] * len(cols))
        return (hm.hamiltonian_block(inp, mt, rows, cols, wd)
                - inp.spin * (P * vbar) @ hm.exchange_vectors_for(inp, mt, cols)[0].conj().T / inp.volume
                + inp.spin * (P * vbar) @ Pr.conj().T / inp.volume)

    rows, cols = _block_cases(mt)[0]
    ref = H[np.ix_(_sub_index(inp, rows), _sub_index(inp, cols))]
    assert np.abs(hm.hamiltonian_block(inp, mt, rows, cols, wd) - ref).max() <= 1e-14 * scale
    assert np.abs(no_head(rows, cols) - ref).max() > 1e-3 * abs(wd)
    rows, cols = _block_cases(mt)[1]
    ref = H[np.ix_(_sub_index(inp, rows), _sub_index(inp, cols))]
    assert np.abs(rows_for_cols(rows, cols) - ref).max() > 1e-8 * scale
