"""Seeded synthetic inputs shaped like the paper's Si, LiF and MoS2 workloads.

This module writes inputs only.  It holds none of the Bethe-Salpeter
arithmetic (pair densities, exchange and direct kernels, projection,
spectrum): the CPU oracle and the CUDA library both consume the dictionary
returned by :func:`generate`.

What it models (a plane-wave stand-in for the paper's FLAPW inputs, Sec. IV):
  * band coefficients c_kn(p) on coset spheres S_k = {p = f_k + m : |p| <= R}
    (full wave vectors, reciprocal fractional coordinates).  At each star
    representative a seeded random Hermitian matrix is averaged over the
    little group (action of Eq. sphi: (s phi)(r) = phi(s^{-1} r), i.e.
    c'(R^{-T} p) = exp(-2 pi i R^{-T}p . t) c(p)) and diagonalised; its
    eigenvector multiplets are never split.  Star members receive the rotated
    coefficients, so every symmetry holds to rounding;
  * band energies that are constant on each (star, multiplet) with a direct
    gap E_g at Gamma;
  * a model static screened interaction W_{QQ'}(q) = v^1/2(Q) eps^-1_{QQ'} v^1/2(Q')
    on coset spheres S_q, with head and wings zero at q = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction as Fr
from functools import lru_cache, reduce

import numpy as np

from .crystal import (Crystal, Mesh, coset_sphere, int_inv3, lif_rocksalt,
                      mos2_2h, norm2_cart, si_diamond, space_group)

HA_EV = 27.211386245988   # CODATA 2018
SEED_BASE = 20260324


@dataclass(frozen=True)
class Config:
    name: str
    material: str            # "Si", "LiF", "MoS2"
    mesh: tuple
    nv: int
    nc: int
    rho: Fr                  # cutoff radius in units of 2 pi / a (wavefunctions and W)
    gap_ev: float
    eps_inf: float
    seed: int
    eta_ev: float = 0.1
    qhat: tuple = (1.0, 0.0, 0.0)
    wv_ev: float = 1.5       # valence band width parameter
    wc_ev: float = 1.5       # conduction band width parameter
    kappa: float = 1.0       # bohr^-1, decay of the diagonal screening
    sigma: float = 1.0       # bohr^-1, decay of local-field terms
    gamma: float = 0.1       # strength of local-field terms
    n_omega: int = 4001
    a: float | None = None   # lattice constant override (bohr)
    eps_inf_z: float | None = None   # zz element of the dielectric tensor of the head correction, if uniaxial


CONFIGS = {
    # Si-like diamond, 4x4x4, Nv = Nc = 4, |G| <= 3.2 (2 pi / a): full dim 1024
    "si4": Config("si4", "Si", (4, 4, 4), 4, 4, Fr(16, 5), 1.1, 12.0, SEED_BASE + 1),
    # Si-like 8x8x8, Nv = 4, Nc = 6: full dim 12288
    "si8": Config("si8", "Si", (8, 8, 8), 4, 6, Fr(16, 5), 1.1, 12.0, SEED_BASE + 2),
    # Si-like 12x12x12, Nv = 4, Nc = 8, |G| <= 4.0 (2 pi / a): full dim 55296
    "si12": Config("si12", "Si", (12, 12, 12), 4, 8, Fr(4), 1.1, 12.0, SEED_BASE + 3),
    # LiF-like rocksalt 10x10x10, Nv = 3, Nc = 6
    "lif10": Config("lif10", "LiF", (10, 10, 10), 3, 6, Fr(16, 5), 14.0, 1.9, SEED_BASE + 4,
                    eta_ev=0.18),
    # small cases used by tests
    "si2": Config("si2", "Si", (2, 2, 2), 4, 4, Fr(16, 5), 1.1, 12.0, SEED_BASE + 11),
    "si3": Config("si3", "Si", (3, 3, 3), 2, 3, Fr(16, 5), 1.1, 12.0, SEED_BASE + 12),
    "lif4": Config("lif4", "LiF", (4, 4, 4), 3, 3, Fr(16, 5), 14.0, 1.9, SEED_BASE + 13,
                   eta_ev=0.18),
    "mos2_331": Config("mos2_331", "MoS2", (3, 3, 1), 2, 2, Fr(93, 50), 1.9, 15.0,
                       SEED_BASE + 14, eta_ev=0.05),
    # the same cell with a uniaxial dielectric tensor diag(15, 15, 6) in the head correction
    "mos2_331_uni": Config("mos2_331_uni", "MoS2", (3, 3, 1), 2, 2, Fr(93, 50), 1.9, 15.0,
                           SEED_BASE + 14, eta_ev=0.05, eps_inf_z=6.0),
}


# Meshes of the mixed batch: MoS2-like hexagonal cells from 9x9x1 to 18x18x3 and
# Si-like cells from 4^3 to 8^3.
BATCH_MOS2_MESHES = [(9, 9, 1), (12, 12, 1), (9, 9, 3), (12, 12, 2), (15, 15, 1), (18, 18, 1), (18, 18, 2),
                     (18, 18, 3)]
BATCH_SI_MESHES = [(4, 4, 4), (5, 5, 5), (6, 6, 6), (7, 7, 7), (8, 8, 8)]


def batch_configs(count: int = 32, seed: int = SEED_BASE + 5, n_si: int = 10) -> list:
    """A seeded batch of independent instances: count - n_si MoS2-like D6h cells
    (a = 5.97 bohr, c/a = 39/10) and n_si Si-like Oh cells, meshes from the
    lists above, N_v and N_c drawn from {2..6} (Si valence from {2, 4}).  A
    draw whose band counts would split a degenerate multiplet is replaced by
    the next draw, so the list generates (each instance is generated once to
    check; generate() caches it)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        si = i >= count - n_si
        while True:
            if si:
                mesh = BATCH_SI_MESHES[int(rng.integers(len(BATCH_SI_MESHES)))]
                nv, nc = int(rng.choice([2, 4])), int(rng.integers(2, 7))
                cfg = Config("b%02d_si_%d%d%d_%d%d" % (i, *mesh, nv, nc), "Si", mesh, nv, nc, Fr(16, 5), 1.1, 12.0,
                             seed + 1000 + i)
            else:
                mesh = BATCH_MOS2_MESHES[int(rng.integers(len(BATCH_MOS2_MESHES)))]
                nv, nc = int(rng.integers(2, 7)), int(rng.integers(2, 7))
                cfg = Config("b%02d_mos2_%d%d%d_%d%d" % (i, *mesh, nv, nc), "MoS2", mesh, nv, nc, Fr(93, 50), 1.9,
                             15.0, seed + 1000 + i, eta_ev=0.05)
            try:
                generate(cfg)
            except RuntimeError:
                continue
            out.append(cfg)
            break
    return out


def crystal_of(cfg: Config) -> Crystal:
    if cfg.material == "Si":
        return si_diamond(cfg.a or 10.26)
    if cfg.material == "LiF":
        return lif_rocksalt(cfg.a or 7.6)
    if cfg.material == "MoS2":
        return mos2_2h(cfg.a or 5.97)
    raise ValueError(cfg.material)


def _tau_int(taus):
    den = reduce(lambda a, b: a * b // math.gcd(a, b),
                 [x.denominator for t in taus for x in t], 1)
    return np.array([[int(x * den) for x in t] for t in taus], dtype=np.int64), den


def _phase(Xp: np.ndarray, t_int: np.ndarray, tden: int, N: int) -> np.ndarray:
    """exp(-2 pi i y'.t) for y' = Xp / N and t = t_int / tden, exact angle."""
    num = (Xp @ t_int) % (N * tden)
    return np.exp(-2j * math.pi * num / (N * tden))


def _nn_shell(crys: Crystal) -> np.ndarray:
    gi = crys.metric_int()
    cand = np.array([(i, j, l) for i in range(-2, 3) for j in range(-2, 3)
                     for l in range(-2, 3) if (i, j, l) != (0, 0, 0)], dtype=np.int64)
    nrm = np.einsum("ni,ij,nj->n", cand, gi, cand)
    return cand[nrm == nrm.min()]


def _pick(mults, nwant):
    """First multiplets (in order) whose sizes add up to nwant, skipping any
    multiplet that would overshoot."""
    got, tot = [], 0
    for mi, m in enumerate(mults):
        if tot + len(m) <= nwant:
            got.append(mi)
            tot += len(m)
        if tot == nwant:
            return got
    raise RuntimeError("cannot fill %d bands without splitting a multiplet" % nwant)


def generate(cfg: Config | str) -> dict:
    """Build the seeded input set of a configuration (cached per name)."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    return _generate(cfg)


@lru_cache(maxsize=40)
def _generate(cfg: Config) -> dict:
    rng = np.random.default_rng(cfg.seed)
    crys = crystal_of(cfg)
    rot, taus = space_group(crys)
    nops = len(rot)
    t_int, tden = _tau_int(taus)
    rk = np.array([int_inv3(r).T for r in rot])          # action on reciprocal coords
    mesh = Mesh(cfg.mesh)
    nk, N = mesh.nk, mesh.N
    nb = cfg.nv + cfg.nc

    # mesh rotations
    rotk = np.zeros((nops, nk), dtype=np.int64)
    for s in range(nops):
        for k in range(nk):
            rotk[s, k] = mesh.rotate(rk[s], k)[0]

    # coset spheres (same radius for wavefunctions and W)
    spheres = [coset_sphere(crys, mesh, k, cfg.rho) for k in range(nk)]
    lookup = [{tuple(m): i for i, m in enumerate(sp)} for sp in spheres]
    nkmax = max(len(sp) for sp in spheres)

    # stars: representative = lowest index; s_k = lowest op index reaching k
    star_of = -np.ones(nk, dtype=np.int64)
    reps = []
    for k in range(nk):
        if star_of[k] >= 0:
            continue
        star_of[rotk[:, k]] = len(reps)
        reps.append(k)

    shell = _nn_shell(crys)
    wv, wc, eg = cfg.wv_ev / HA_EV, cfg.wc_ev / HA_EV, cfg.gap_ev / HA_EV

    coef = np.zeros((nk, nb, nkmax), dtype=np.complex128)
    eps = np.zeros((nk, nb), dtype=np.float64)
    gk = np.zeros((nk, nkmax, 3), dtype=np.int32)
    nkc = np.array([len(sp) for sp in spheres], dtype=np.int32)
    for k in range(nk):
        gk[k, :nkc[k]] = spheres[k]

    for a, p in enumerate(reps):
        sp = spheres[p]
        npw = len(sp)
        Xp = sp * N + mesh.X[p]
        little = [s for s in range(nops) if rotk[s, p] == p]
        h = rng.standard_normal((npw, npw)) + 1j * rng.standard_normal((npw, npw))
        h = 0.5 * (h + h.conj().T)
        hs = np.zeros_like(h)
        for s in little:
            Xr = Xp @ rk[s].T
            mr = Xr - mesh.X[p]
            assert np.all(mr % N == 0)
            mr //= N
            j = np.array([lookup[p][tuple(m)] for m in mr])
            d = np.zeros((npw, npw), dtype=np.complex128)
            d[j, np.arange(npw)] = _phase(Xr, t_int[s], tden, N)
            hs += d @ h @ d.conj().T
        hs /= len(little)
        lam, vec = np.linalg.eigh(hs)
        tol = 1e-8 * np.abs(lam).max()
        mults, cur = [], [0]
        for i in range(1, npw):
            if lam[i] - lam[cur[-1]] <= tol:
                cur.append(i)
            else:
                mults.append(cur)
                cur = [i]
        mults.append(cur)
        vsel = _pick(mults, cfg.nv)
        rest = [m for i, m in enumerate(mults) if i not in set(vsel)]
        csel = _pick(rest, cfg.nc)
        vm = [mults[i] for i in vsel]
        cm = [rest[i] for i in csel]
        # energies: constant on (star, multiplet), direct gap eg at Gamma
        dv = np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.5, len(vm) - 1))]) / HA_EV
        dc = np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.5, len(cm) - 1))]) / HA_EV
        phi = float(np.mean(np.cos(2.0 * math.pi * (shell @ mesh.f(p)))))
        cp = np.zeros((nb, npw), dtype=np.complex128)
        ep = np.zeros(nb)
        b = 0
        for i, m in enumerate(vm):
            for col in m:
                cp[b] = vec[:, col]
                ep[b] = -wv * (1.0 - phi) - dv[i]
                b += 1
        for i, m in enumerate(cm):
            for col in m:
                cp[b] = vec[:, col]
                ep[b] = eg + wc * (1.0 - phi) + dc[i]
                b += 1
        # rotate to every star member with its lowest-index operation
        members = np.nonzero(star_of == a)[0]
        for k in members:
            s = int(np.nonzero(rotk[:, p] == k)[0][0])
            Xr = Xp @ rk[s].T
            mr = Xr - mesh.X[k]
            assert np.all(mr % N == 0)
            mr //= N
            j = np.array([lookup[k][tuple(m)] for m in mr])
            assert len(set(j.tolist())) == npw == nkc[k]
            ph = _phase(Xr, t_int[s], tden, N)
            coef[k][:, j] = cp * ph[None, :]
            eps[k] = ep

    # model W(q) on the same coset spheres
    ng = nkc.copy()
    ngmax = nkmax
    w = np.zeros((nk, ngmax, ngmax), dtype=np.complex128)
    atoms_num = []
    wsum = sum(crys.weight_of(sp) for sp, _ in crys.atoms)
    for sp, x in crys.atoms:
        den = reduce(lambda u, v: u * v // math.gcd(u, v), [c.denominator for c in x], 1)
        atoms_num.append((crys.weight_of(sp) / wsum, np.array([int(c * den) for c in x]), den))
    ei = 1.0 / cfg.eps_inf
    for q in range(nk):
        m = spheres[q]
        X = m * N + mesh.X[q]
        q2 = norm2_cart(crys, mesh, X)
        dG = m[:, None, :] - m[None, :, :]
        d2 = norm2_cart(crys, mesh, dG * N)
        sfac = np.zeros(d2.shape, dtype=np.complex128)
        for wt, num, den in atoms_num:
            ang = (dG @ num) % den
            sfac += wt * np.exp(-2j * math.pi * ang / den)
        einv = (cfg.gamma * (1.0 - ei) * sfac
                * np.exp(-(q2[:, None] + q2[None, :]) / (4.0 * cfg.kappa ** 2))
                * np.exp(-d2 / (2.0 * cfg.sigma ** 2)))
        np.fill_diagonal(einv, 1.0 - (1.0 - ei) * np.exp(-q2 / (2.0 * cfg.kappa ** 2)))
        with np.errstate(divide="ignore"):
            vh = np.where(q2 > 0, math.sqrt(4.0 * math.pi) / np.sqrt(np.where(q2 > 0, q2, 1.0)), 0.0)
        wq = vh[:, None] * einv * vh[None, :]
        w[q, :len(m), :len(m)] = wq

    omega_max = eg + 2.0 * (wv + wc) + 2.0 / HA_EV
    out = dict(
        name=cfg.name,
        lattice=crys.lattice(),
        volume=crys.volume(),
        rot=rot.astype(np.int32),
        tau=np.array([[float(x) for x in t] for t in taus]),
        mesh=np.array(cfg.mesh, dtype=np.int32),
        nv=cfg.nv,
        nc=cfg.nc,
        nk_count=nkc,
        gk=gk,
        coef=coef,
        eps=eps,
        ng_count=ng.astype(np.int32),
        gq=gk.copy(),
        w=w,
        eps_inf=np.diag([cfg.eps_inf, cfg.eps_inf, cfg.eps_inf if cfg.eps_inf_z is None else cfg.eps_inf_z]),
        qhat=np.array(cfg.qhat, dtype=np.float64),
        scissor=0.0,
        spin_factor=2,
        eta=cfg.eta_ev / HA_EV,
        omega=np.linspace(0.0, omega_max, cfg.n_omega),
    )
    for v in out.values():
        if isinstance(v, np.ndarray):
            v.setflags(write=False)
    return out


def subset_pairs(inp: dict, n: int, seed: int = 7):
    """A seeded sample of (k, k') pairs of an input set, for sampled checks."""
    nk = int(np.prod(inp["mesh"]))
    rng = np.random.default_rng(seed)
    k = rng.integers(0, nk, n)
    kp = rng.integers(0, nk, n)
    return k.astype(np.int32), kp.astype(np.int32)
