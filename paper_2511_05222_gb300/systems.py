"""Seeded synthetic inputs: geometries, contracted-Gaussian bases, frozen orbitals, walkers.

This module is input preparation only. It is shared by the CUDA path, the CPU oracle, the
tests and the benchmark, and it holds none of the VMC arithmetic (no AO evaluation, no
determinants, no Jastrow, no local energy, no estimators). Primitive and contraction
normalisation is left to each consumer: the basis is handed out with RAW contraction
coefficients (coefficients of normalised primitives, before renormalisation of the
contraction).

The one integral computed here is the AO overlap matrix S. The method takes S as an input
from the mean-field code (Eq. Q_projector); the generator needs it to orthonormalise the
random occupied-orbital columns (C^T S C = I) and hands it out for the optional
virtual-space projection. It is built from Cartesian Gaussian-product overlaps, so that it
is an independent check on the normalisation both consumers apply.

Workload recipe (all sizes follow the basis rule "heavy atom 3s2p1d, H 2s1p", three
primitives per shell):
  * water (10 e-): O-H 1.81 bohr, 104.5 deg, each coordinate jittered U(-0.05, 0.05);
  * C2OH6 (26 e-) and C9O4H8 (94 e-): covalent-walk placement, bond lengths U(1.9, 2.9),
    every pair at least 1.7 bohr apart;
  * exponents log-uniform in [0.1, 5000] for O s shells and [0.1, 30] otherwise, sorted
    descending within a shell; raw contraction coefficients U(0.2, 1);
  * orbitals: independent Gaussian M x n matrices per spin, Loewdin-orthonormalised in S;
  * walkers: electron e (up block first) at nucleus e mod K plus N(0, 1) per coordinate.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MAXPRIM = 3
GEN_SEED_BASE = 52220

# Real solid harmonics r^l Y_lm as Cartesian monomials (coefficient, (a, b, c)).
# Order: s; p = (x, y, z); d = (xy, yz, 3z^2 - r^2, xz, x^2 - y^2).  The angular
# normalisation makes the integral of Y^2 over the unit sphere equal to one.
_SQ = math.sqrt
_PI = math.pi
CART_TERMS = {
    0: [[(_SQ(1.0 / (4 * _PI)), (0, 0, 0))]],
    1: [[(_SQ(3.0 / (4 * _PI)), (1, 0, 0))],
        [(_SQ(3.0 / (4 * _PI)), (0, 1, 0))],
        [(_SQ(3.0 / (4 * _PI)), (0, 0, 1))]],
    2: [[(_SQ(15.0 / (4 * _PI)), (1, 1, 0))],
        [(_SQ(15.0 / (4 * _PI)), (0, 1, 1))],
        [(2 * _SQ(5.0 / (16 * _PI)), (0, 0, 2)),
         (-_SQ(5.0 / (16 * _PI)), (2, 0, 0)),
         (-_SQ(5.0 / (16 * _PI)), (0, 2, 0))],
        [(_SQ(15.0 / (4 * _PI)), (1, 0, 1))],
        [(_SQ(15.0 / (16 * _PI)), (2, 0, 0)),
         (-_SQ(15.0 / (16 * _PI)), (0, 2, 0))]],
}
NCOMP = {0: 1, 1: 3, 2: 5}


@dataclass
class JastrowBasis:
    """Jastrow basis of the AO-expanded Jastrow terms: shells on the system's nuclei (same
    conventions as the determinant basis: real solid harmonics, raw coefficients of normalised
    primitives), one-body coefficients xi (MJ,) and symmetric pair coefficients Xi (MJ, MJ)."""
    shell_center: np.ndarray  # (nshell,) int32
    shell_l: np.ndarray       # (nshell,) int32, 0..2
    shell_nprim: np.ndarray   # (nshell,) int32
    shell_exp: np.ndarray     # (nshell, MAXPRIM) float64
    shell_coef: np.ndarray    # (nshell, MAXPRIM) float64, RAW coefficients
    xi: np.ndarray            # (MJ,) float64
    Xi: np.ndarray            # (MJ, MJ) float64, symmetric

    @property
    def MJ(self) -> int:
        return int(sum(NCOMP[int(l)] for l in self.shell_l))

    @property
    def nshell(self) -> int:
        return int(self.shell_l.shape[0])


@dataclass
class Jastrow:
    """One-body e-n cusp term chi_I(r) = -Z_I r / (1 + b_en r) and spin-dependent two-body
    term with cusp a (1/2 antiparallel, 1/4 parallel): Pade u(r) = a r / (1 + F r), or with
    two_body_exp the exponential form u(r) = (a / F) (1 - exp(-F r)); optionally the AO-expanded
    one-body and pair terms over a Jastrow basis (basis, None for none)."""
    F_anti: float = 0.8
    F_par: float = 0.8
    a_anti: float = 0.5
    a_par: float = 0.25
    b_en: float = 1.5
    enable_J1: bool = True
    enable_J2: bool = True
    two_body_exp: bool = False
    basis: JastrowBasis | None = None


@dataclass
class System:
    name: str
    Z: np.ndarray            # (K,) int32 nuclear charges
    R: np.ndarray            # (K, 3) float64, bohr
    shell_center: np.ndarray  # (nshell,) int32
    shell_l: np.ndarray       # (nshell,) int32, 0..2
    shell_nprim: np.ndarray   # (nshell,) int32, 1..MAXPRIM
    shell_exp: np.ndarray     # (nshell, MAXPRIM) float64
    shell_coef: np.ndarray    # (nshell, MAXPRIM) float64, RAW coefficients
    n_up: int
    n_dn: int
    C_up: np.ndarray          # (M, n_up) float64, row-major [mu][i]
    C_dn: np.ndarray          # (M, n_dn)
    jastrow: Jastrow = field(default_factory=Jastrow)
    S: np.ndarray | None = None  # (M, M) AO overlap, when computed

    @property
    def K(self) -> int:
        return int(self.Z.shape[0])

    @property
    def M(self) -> int:
        return int(sum(NCOMP[int(l)] for l in self.shell_l))

    @property
    def Ne(self) -> int:
        return self.n_up + self.n_dn

    @property
    def nshell(self) -> int:
        return int(self.shell_l.shape[0])


# --------------------------------------------------------------------------- geometry
def water_geometry(rng: np.random.Generator) -> tuple[np.ndarray, np.ndarray]:
    d, ang = 1.81, math.radians(104.5)
    R = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0], [d * math.cos(ang), d * math.sin(ang), 0.0]])
    R = R + rng.uniform(-0.05, 0.05, size=R.shape)
    return np.array([8, 1, 1], dtype=np.int32), R


def covalent_walk(Z: list[int], rng: np.random.Generator, bond=(1.9, 2.9), dmin=1.7) -> np.ndarray:
    """Heavy atoms first; every new atom bonds to a uniformly chosen, already placed heavy
    atom along a uniform direction; a placement closer than dmin to any atom is redrawn."""
    heavy = [i for i, z in enumerate(Z) if z > 1]
    light = [i for i, z in enumerate(Z) if z == 1]
    if not heavy:
        raise ValueError("covalent walk needs at least one heavy atom")
    order = heavy + light
    R = np.zeros((len(Z), 3))
    placed: list[int] = []
    placed_heavy: list[int] = []
    for idx in order:
        if not placed:
            R[idx] = 0.0
        else:
            for _ in range(100000):
                anchor = placed_heavy[rng.integers(len(placed_heavy))]
                v = rng.standard_normal(3)
                v /= np.linalg.norm(v)
                cand = R[anchor] + rng.uniform(*bond) * v
                if np.min(np.linalg.norm(R[placed] - cand, axis=1)) >= dmin:
                    R[idx] = cand
                    break
            else:  # pragma: no cover
                raise RuntimeError("covalent walk failed to place an atom")
        placed.append(idx)
        if Z[idx] > 1:
            placed_heavy.append(idx)
    return R


# --------------------------------------------------------------------------- basis
def basis_rule(Z: np.ndarray, rng: np.random.Generator):
    """Heavy atom 3s2p1d (6 shells, 14 AOs); H 2s1p (3 shells, 5 AOs); 3 primitives each."""
    centers, ls, exps, coefs = [], [], [], []
    for I, z in enumerate(Z):
        shells = [0, 0, 0, 1, 1, 2] if z > 1 else [0, 0, 1]
        for l in shells:
            hi = 5000.0 if (z == 8 and l == 0) else 30.0
            e = np.exp(rng.uniform(math.log(0.1), math.log(hi), size=MAXPRIM))
            centers.append(I)
            ls.append(l)
            exps.append(np.sort(e)[::-1])
            coefs.append(rng.uniform(0.2, 1.0, size=MAXPRIM))
    n = len(ls)
    return (np.array(centers, np.int32), np.array(ls, np.int32), np.full(n, MAXPRIM, np.int32),
            np.array(exps, np.float64), np.array(coefs, np.float64))


# --------------------------------------------------------------------------- overlap (input prep)
def _moment(k: int, p: np.ndarray) -> np.ndarray:
    """Integral over t of t^k exp(-p t^2)."""
    if k % 2:
        return np.zeros_like(p)
    return math.gamma((k + 1) / 2.0) / p ** ((k + 1) / 2.0)


def _overlap_1d(a: int, b: int, A: float, B: float, al: np.ndarray, be: np.ndarray) -> np.ndarray:
    """Integral of (x-A)^a (x-B)^b exp(-al (x-A)^2 - be (x-B)^2), vectorised over (al, be),
    by the Gaussian product theorem and a binomial expansion about the product centre."""
    p = al + be
    P = (al * A + be * B) / p
    PA, PB = P - A, P - B
    pref = np.exp(-al * be / p * (A - B) ** 2)
    acc = np.zeros_like(p)
    for i in range(a + 1):
        for j in range(b + 1):
            acc = acc + math.comb(a, i) * math.comb(b, j) * PA ** (a - i) * PB ** (b - j) * _moment(i + j, p)
    return pref * acc


def _cart_overlap(terms1, terms2, A, B, al, be) -> np.ndarray:
    tot = np.zeros_like(al)
    for c1, (a1, b1, z1) in terms1:
        for c2, (a2, b2, z2) in terms2:
            tot = tot + c1 * c2 * (_overlap_1d(a1, a2, A[0], B[0], al, be)
                                   * _overlap_1d(b1, b2, A[1], B[1], al, be)
                                   * _overlap_1d(z1, z2, A[2], B[2], al, be))
    return tot


def generator_ao_coefficients(sys: System) -> np.ndarray:
    """Coefficients (per shell, per primitive) of the normalised contracted AO, found by
    normalising each primitive and then the contraction through the Cartesian overlap
    integrals above (no closed-form normalisation constant is used)."""
    out = np.zeros_like(sys.shell_coef)
    for s in range(sys.nshell):
        l, npr = int(sys.shell_l[s]), int(sys.shell_nprim[s])
        t = CART_TERMS[l][0]
        a = sys.shell_exp[s, :npr]
        zero = np.zeros(3)
        selfov = _cart_overlap(t, t, zero, zero, a, a)
        nrm = 1.0 / np.sqrt(selfov)
        d = sys.shell_coef[s, :npr] * nrm
        al, be = np.meshgrid(a, a, indexing="ij")
        Spp = _cart_overlap(t, t, zero, zero, al.ravel(), be.ravel()).reshape(npr, npr)
        out[s, :npr] = d / math.sqrt(float(d @ Spp @ d))
    return out


def overlap_matrix(sys: System) -> np.ndarray:
    coef = generator_ao_coefficients(sys)
    ao0 = np.concatenate([[0], np.cumsum([NCOMP[int(l)] for l in sys.shell_l])])
    S = np.zeros((sys.M, sys.M))
    for s1 in range(sys.nshell):
        l1, n1 = int(sys.shell_l[s1]), int(sys.shell_nprim[s1])
        A = sys.R[sys.shell_center[s1]]
        for s2 in range(s1, sys.nshell):
            l2, n2 = int(sys.shell_l[s2]), int(sys.shell_nprim[s2])
            B = sys.R[sys.shell_center[s2]]
            al, be = np.meshgrid(sys.shell_exp[s1, :n1], sys.shell_exp[s2, :n2], indexing="ij")
            al, be = al.ravel(), be.ravel()
            w = np.outer(coef[s1, :n1], coef[s2, :n2]).ravel()
            # 1-D overlaps for every pair of powers on each axis, shared by all Cartesian terms
            tab = [[[_overlap_1d(a, b, A[ax], B[ax], al, be) for b in range(l2 + 1)] for a in range(l1 + 1)]
                   for ax in range(3)]
            for m1, t1 in enumerate(CART_TERMS[l1]):
                for m2, t2 in enumerate(CART_TERMS[l2]):
                    tot = np.zeros_like(al)
                    for c1, (a1, b1, z1) in t1:
                        for c2, (a2, b2, z2) in t2:
                            tot = tot + c1 * c2 * (tab[0][a1][a2] * tab[1][b1][b2] * tab[2][z1][z2])
                    v = float(w @ tot)
                    S[ao0[s1] + m1, ao0[s2] + m2] = v
                    S[ao0[s2] + m2, ao0[s1] + m1] = v
    return S


def orthonormal_orbitals(S: np.ndarray, n: int, rng: np.random.Generator) -> np.ndarray:
    """Random Gaussian M x n columns, Loewdin-orthonormalised so that C^T S C = I."""
    M = S.shape[0]
    C0 = rng.standard_normal((M, n))
    if n == 0:
        return C0
    w, V = np.linalg.eigh(C0.T @ S @ C0)
    return np.ascontiguousarray(C0 @ (V * (1.0 / np.sqrt(w))) @ V.T)


# --------------------------------------------------------------------------- systems
_CFG_COMPOSITION = {
    1: ("C2OH6", [6, 6, 8, 1, 1, 1, 1, 1, 1]),
    4: ("C9O4H8", [6] * 9 + [8] * 4 + [1] * 8),
}


def _rng(cfg: int, purpose: int) -> np.random.Generator:
    return np.random.default_rng([GEN_SEED_BASE + cfg, purpose])


def make_molecule(name: str, Z, R, rng_basis, rng_orb, jastrow: Jastrow | None = None,
                  with_S: bool = True) -> System:
    Z = np.asarray(Z, np.int32)
    c, l, npr, e, co = basis_rule(Z, rng_basis)
    ne = int(Z.sum())
    if ne % 2:
        raise ValueError("closed-shell systems only")
    n = ne // 2
    sys = System(name, Z, np.ascontiguousarray(R, dtype=np.float64), c, l, npr, e, co, n, n,
                 np.zeros((0, 0)), np.zeros((0, 0)), jastrow or Jastrow())
    S = overlap_matrix(sys)
    sys.C_up = orthonormal_orbitals(S, n, rng_orb)
    sys.C_dn = orthonormal_orbitals(S, n, rng_orb)
    sys.S = S if with_S else None
    return sys


def make_system(cfg: int) -> System:
    """The fixed workloads: 0 = water (10 e-), 1 and 2 = C2OH6 (26 e-), 4 = C9O4H8 (94 e-)."""
    if cfg == 0:
        Z, R = water_geometry(_rng(0, 0))
        return make_molecule("H2O", Z, R, _rng(0, 1), _rng(0, 2))
    base = 1 if cfg == 2 else cfg
    if base not in _CFG_COMPOSITION:
        raise ValueError(f"no single-system workload {cfg}")
    name, Z = _CFG_COMPOSITION[base]
    R = covalent_walk(Z, _rng(base, 0))
    return make_molecule(name, Z, R, _rng(base, 1), _rng(base, 2))


def ragged_batch_plan(n_geom: int = 64, seed: int = 3) -> list[tuple[list[int], int]]:
    """Compositions and walker counts of the ragged batch, without building the molecules:
    n_geom lists of 3..21 H/C/O nuclear charges (a C or O first) with an even electron count
    in [10, 94], and 512..4096 walkers each (multiple of 128)."""
    rng = np.random.default_rng([GEN_SEED_BASE + seed, 0])
    out = []
    while len(out) < n_geom:
        K = int(rng.integers(3, 22))
        Z = [int(rng.choice([6, 8]))] + [int(rng.choice([1, 6, 8])) for _ in range(K - 1)]
        ne = sum(Z)
        if ne % 2 or not (10 <= ne <= 94):
            continue
        W = int(rng.integers(512, 4097)) // 128 * 128
        out.append((Z, max(W, 512)))
    return out


def make_ragged_batch(n_geom: int = 64, seed: int = 3, only=None):
    """Ragged batch: n_geom covalent-walk molecules of 3..21 H/C/O nuclei, an even electron
    count in [10, 94], and 512..4096 walkers each (multiple of 128). Returns (System, W) per
    geometry; with `only` (indices), just those geometries, in index order."""
    plan = ragged_batch_plan(n_geom, seed)
    out = []
    for g, (Z, W) in enumerate(plan):
        if only is not None and g not in only:
            continue
        R = covalent_walk(Z, np.random.default_rng([GEN_SEED_BASE + seed, 1, g]))
        sys = make_molecule(f"ragged{g}", Z, R, np.random.default_rng([GEN_SEED_BASE + seed, 2, g]),
                            np.random.default_rng([GEN_SEED_BASE + seed, 3, g]))
        out.append((sys, W))
    return out


def jastrow_basis(sys: System, seed: int = 0, xi_scale: float = 0.1, same_scale: float = 0.03,
                  pair_scale: float = 0.01) -> JastrowBasis:
    """Seeded Jastrow basis and coefficients for the AO-expanded Jastrow terms: uncontracted
    primitives, H [3s1p] and heavy atoms [4s2p1d] (the medium Jastrow basis); exponents log-uniform
    in [0.1, 3] for s, [0.2, 2] for p, [0.3, 1.5] for d, sorted descending per l; xi_mu uniform in
    +-xi_scale; Xi symmetric with Gaussian entries of standard deviation same_scale between functions
    of one nucleus and pair_scale between nuclei (the inter-nuclear entries are kept)."""
    rng = np.random.default_rng([GEN_SEED_BASE + 2000, seed])
    centers, ls, exps = [], [], []
    ranges = {0: (0.1, 3.0), 1: (0.2, 2.0), 2: (0.3, 1.5)}
    for I, z in enumerate(sys.Z):
        counts = {0: 3, 1: 1} if z == 1 else {0: 4, 1: 2, 2: 1}
        for l, cnt in counts.items():
            lo, hi = ranges[l]
            for a in np.sort(np.exp(rng.uniform(math.log(lo), math.log(hi), size=cnt)))[::-1]:
                centers.append(I)
                ls.append(l)
                exps.append(a)
    ns = len(ls)
    ex = np.zeros((ns, MAXPRIM))
    co = np.zeros((ns, MAXPRIM))
    ex[:, 0] = exps
    co[:, 0] = 1.0
    cen = np.array(centers, np.int32)
    lv = np.array(ls, np.int32)
    fcen = np.concatenate([[c] * NCOMP[int(l)] for c, l in zip(cen, lv)]).astype(np.int32)
    MJ = fcen.shape[0]
    xi = rng.uniform(-xi_scale, xi_scale, size=MJ)
    same = fcen[:, None] == fcen[None, :]
    G = rng.standard_normal((MJ, MJ)) * np.where(same, same_scale, pair_scale)
    Xi = np.triu(G) + np.triu(G, 1).T
    return JastrowBasis(cen, lv, np.ones(ns, np.int32), ex, co, xi, np.ascontiguousarray(Xi))


def with_jastrow_basis(sys: System, jb: JastrowBasis | None = None, seed: int = 0) -> System:
    """A copy of the system whose Jastrow also holds the AO-expanded terms (jb, or a seeded
    jastrow_basis of the system)."""
    import copy
    out = copy.copy(sys)
    out.jastrow = copy.copy(sys.jastrow)
    out.jastrow.basis = jb if jb is not None else jastrow_basis(sys, seed)
    return out


def initial_walkers(sys: System, W: int, seed: int = 0) -> np.ndarray:
    """(W, Ne, 3) float64: electron e (up block first) at nucleus e mod K plus N(0, 1)."""
    rng = np.random.default_rng([GEN_SEED_BASE + 1000, seed])
    pos = np.empty((W, sys.Ne, 3))
    for e in range(sys.Ne):
        pos[:, e, :] = sys.R[e % sys.K] + rng.standard_normal((W, 3))
    return pos


def custom_system(name: str, Z, R, shells, n_up: int, n_dn: int, C_up, C_dn,
                  jastrow: Jastrow | None = None) -> System:
    """Hand-built system for pins: shells = [(center, l, [exps], [raw coefs]), ...]."""
    ns = len(shells)
    M = sum(NCOMP[int(s[1])] for s in shells)

    def _mat(C, n):
        return np.zeros((M, 0)) if n == 0 else np.ascontiguousarray(np.asarray(C, np.float64).reshape(M, n))

    ex = np.zeros((ns, MAXPRIM))
    co = np.zeros((ns, MAXPRIM))
    for s, (_, _, e, c) in enumerate(shells):
        ex[s, :len(e)] = e
        co[s, :len(c)] = c
    return System(name, np.asarray(Z, np.int32), np.asarray(R, np.float64).reshape(-1, 3),
                  np.array([s[0] for s in shells], np.int32), np.array([s[1] for s in shells], np.int32),
                  np.array([len(s[2]) for s in shells], np.int32), ex, co, n_up, n_dn,
                  _mat(C_up, n_up), _mat(C_dn, n_dn),
                  jastrow or Jastrow())
