"""Seeded synthetic workloads shaped like the paper's molecules.

This module only draws random numbers and lays out geometry; it holds none of
the method's arithmetic (no normalisation, no integrals, no densities).  It is
shared by the tests, the benchmark and the oracle-side checks so that both
sides of every parity test see the same inputs.

Recipe (one ``numpy.random.default_rng(seed)`` per workload; draw order fixed):
  1. basis per element kind, in the order heavy, central heavy, H; per shell
     (s shells, then p, then d) 3 exponents log-uniform in [0.1, 5e3] sorted
     descending and 3 coefficients 1 - U[0,1) (so in (0, 1]);
  2. MO coefficients C ~ N(0,1), [N, N] (first o columns occupied);
  3. eps_o ~ U[-1.5, -0.3] sorted, then eps_v ~ U[0.1, 3.0] sorted;
  4. transition amplitudes X ~ N(0,1), [npair, o, v];
  5. (gradient workloads) P_r, Q_r = (A + A^T)/2 with A ~ N(0,1).

Basis sets: heavy atom 3s2p1d (15 Cartesian AO), central heavy atom 4s3p2d
(25 AO), H 2s1p (5 AO).  Electron counts use Z = 6 for heavy atoms, 12 for the
central atom and 1 for H; o = electrons / 2.

f-shell (triple-zeta-shaped) workloads stand in for the paper's f-shell
systems (def2-TZVP / cc-pVTZ-class bases): heavy atom 4s3p2d1f (35 Cartesian
AO), H 3s2p1d (15 AO), drawn by ``draw_tz_bases`` with the same per-shell
recipe (step 1) for the kinds heavy_tz then H_tz, in place of step 1, except
that f exponents are log-uniform in [0.2, 5] (f shells are polarization
functions: def2-TZVP-class f exponents lie near 0.5-2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KIND_SHELLS = {
    "heavy": (0, 0, 0, 1, 1, 2),
    "central": (0, 0, 0, 0, 1, 1, 1, 2, 2),
    "H": (0, 0, 1),
}
KIND_Z = {"heavy": 6, "central": 12, "H": 1, "heavy_tz": 6, "H_tz": 1}
TZ_KIND_SHELLS = {
    "heavy_tz": (0, 0, 0, 0, 1, 1, 1, 2, 2, 3),
    "H_tz": (0, 0, 0, 1, 1, 2),
}
NPRIM = 3
EXP_RANGE = (0.1, 5.0e3)
EXP_RANGE_F = (0.2, 5.0)


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


@dataclasses.dataclass
class Molecule:
    """Atoms, Cartesian shells and raw contraction coefficients (host arrays)."""
    coords: np.ndarray        # [natoms, 3] float64, bohr
    kinds: list               # element kind per atom
    shell_atom: np.ndarray    # [nshells] int32
    shell_l: np.ndarray       # [nshells] int32
    shell_nprim: np.ndarray   # [nshells] int32
    exps: np.ndarray          # [nprim_total] float64
    coefs: np.ndarray         # [nprim_total] float64, w.r.t. normalised primitives

    @property
    def natoms(self) -> int:
        return self.coords.shape[0]

    @property
    def nshells(self) -> int:
        return self.shell_l.shape[0]

    @property
    def nao(self) -> int:
        return int(sum(ncart(int(l)) for l in self.shell_l))

    @property
    def nelec(self) -> int:
        return int(sum(KIND_Z[k] for k in self.kinds))

    def with_coords(self, coords: np.ndarray) -> "Molecule":
        return dataclasses.replace(self, coords=np.ascontiguousarray(coords, dtype=np.float64))


def draw_kind_bases(rng: np.random.Generator, kind_shells: dict | None = None) -> dict:
    """Per element kind: list of (l, exps[3], coefs[3])."""
    out = {}
    kind_shells = KIND_SHELLS if kind_shells is None else kind_shells
    for kind in kind_shells:
        shells = []
        for l in kind_shells[kind]:
            lo, hi = (math.log(v) for v in (EXP_RANGE_F if l == 3 else EXP_RANGE))
            e = np.sort(np.exp(rng.uniform(lo, hi, NPRIM)))[::-1].copy()
            c = 1.0 - rng.random(NPRIM)
            shells.append((l, e, c))
        out[kind] = shells
    return out


def draw_tz_bases(rng: np.random.Generator) -> dict:
    """The f-shell kinds: heavy_tz 4s3p2d1f, H_tz 3s2p1d."""
    return draw_kind_bases(rng, TZ_KIND_SHELLS)


def tz_kinds(kinds):
    """The f-shell counterpart of every atom kind of a geometry."""
    return [{"heavy": "heavy_tz", "central": "heavy_tz", "H": "H_tz"}[k] for k in kinds]


def build_molecule(coords, kinds, bases) -> Molecule:
    sh_atom, sh_l, sh_np, exps, coefs = [], [], [], [], []
    for ia, kind in enumerate(kinds):
        for (l, e, c) in bases[kind]:
            sh_atom.append(ia)
            sh_l.append(l)
            sh_np.append(len(e))
            exps.extend(e)
            coefs.extend(c)
    return Molecule(
        coords=np.ascontiguousarray(np.asarray(coords, dtype=np.float64).reshape(-1, 3)),
        kinds=list(kinds),
        shell_atom=np.asarray(sh_atom, dtype=np.int32),
        shell_l=np.asarray(sh_l, dtype=np.int32),
        shell_nprim=np.asarray(sh_np, dtype=np.int32),
        exps=np.asarray(exps, dtype=np.float64),
        coefs=np.asarray(coefs, dtype=np.float64),
    )


# ------------------------------------------------------------------ geometries
def water_like():
    """O-like heavy atom at the origin, two H at 1.81 bohr with a 104.5 degree angle."""
    h = math.radians(104.5 / 2)
    r = 1.81
    coords = [(0.0, 0.0, 0.0), (r * math.sin(h), 0.0, r * math.cos(h)),
              (-r * math.sin(h), 0.0, r * math.cos(h))]
    return coords, ["heavy", "H", "H"]


def chain(n_heavy: int, n_h: int | None = None):
    """Zig-zag heavy-atom chain in the xy plane, 1.4 bohr between neighbours,
    with one H per heavy atom (first n_h of them) 2.05 bohr out of the chain."""
    if n_h is None:
        n_h = n_heavy
    coords, kinds = [], []
    step = 1.4 * math.sqrt(3.0) / 2.0
    for k in range(n_heavy):
        coords.append((k * step, (k % 2) * 0.7, 0.0))
        kinds.append("heavy")
    for k in range(n_h):
        x, y, z = coords[k]
        sgn = -1.0 if k % 2 == 0 else 1.0
        coords.append((x, y + 2.05 * sgn, z))
        kinds.append("H")
    return coords, kinds


def macrocycle():
    """Porphine-shaped planar D4h-like layout: central heavy atom, 4 N-like,
    8 alpha, 8 beta, 4 meso heavy atoms, 8 beta-H and 4 meso-H (37 atoms)."""
    coords, kinds = [(0.0, 0.0, 0.0)], ["central"]

    def put(r, deg, kind):
        t = math.radians(deg)
        coords.append((r * math.cos(t), r * math.sin(t), 0.0))
        kinds.append(kind)

    for k in range(4):
        put(3.85, 90.0 * k, "heavy")
    for k in range(4):
        for s in (-22.0, 22.0):
            put(5.2, 90.0 * k + s, "heavy")
    for k in range(4):
        for s in (-13.0, 13.0):
            put(6.5, 90.0 * k + s, "heavy")
    for k in range(4):
        put(6.4, 45.0 + 90.0 * k, "heavy")
    for k in range(4):
        for s in (-12.0, 12.0):
            put(8.5, 90.0 * k + s, "H")
    for k in range(4):
        put(8.45, 45.0 + 90.0 * k, "H")
    return coords, kinds


# ------------------------------------------------------------------ workloads
@dataclasses.dataclass
class JKWorkload:
    name: str
    mol: Molecule
    nocc: int
    nvir: int
    C: np.ndarray        # [N, N]; columns 0..o-1 occupied, o..N-1 virtual
    eps_occ: np.ndarray  # [o]
    eps_vir: np.ndarray  # [v]
    X: np.ndarray        # [npair, o, v]
    nlap: int
    schwarz_tau: float
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def C_occ(self):
        return np.ascontiguousarray(self.C[:, : self.nocc])

    @property
    def C_vir(self):
        return np.ascontiguousarray(self.C[:, self.nocc: self.nocc + self.nvir])

    @property
    def ndens(self):
        return self.nlap * self.X.shape[0]


def _mo_part(rng, mol: Molecule, nocc: int, npair: int):
    N = mol.nao
    nvir = N - nocc
    C = rng.standard_normal((N, N))
    eps_o = np.sort(rng.uniform(-1.5, -0.3, nocc))
    eps_v = np.sort(rng.uniform(0.1, 3.0, nvir))
    X = rng.standard_normal((npair, nocc, nvir))
    return nvir, C, eps_o, eps_v, X


def jk_workload(name: str, coords, kinds, seed: int, npair: int, nlap: int,
                nocc: int | None = None, tau: float = 1e-12, tz: bool = False) -> JKWorkload:
    rng = np.random.default_rng(seed)
    bases = draw_tz_bases(rng) if tz else draw_kind_bases(rng)
    if tz:
        kinds = tz_kinds(kinds)
    mol = build_molecule(coords, kinds, bases)
    if nocc is None:
        nocc = mol.nelec // 2
    nvir, C, eo, ev, X = _mo_part(rng, mol, nocc, npair)
    return JKWorkload(name, mol, nocc, nvir, C, eo, ev, X, nlap, tau)


def config1() -> JKWorkload:
    """25-AO water-like molecule, 5 occupied / 20 virtual, 1 pair x 8 Laplace points."""
    c, k = water_like()
    return jk_workload("water-like 25 AO, 8 densities", c, k, seed=1, npair=1, nlap=8,
                       nocc=5, tau=1e-12)


def config2() -> JKWorkload:
    """200-AO chain: 10 heavy 3s2p1d + 10 H 2s1p, 35 occupied, 3 pairs x 16 points."""
    c, k = chain(10)
    return jk_workload("chain 200 AO, 48 densities", c, k, seed=2, npair=3, nlap=16,
                       nocc=35, tau=1e-12)


def config3() -> JKWorkload:
    """445-AO porphine-shaped macrocycle, 86 occupied, 8 pairs x 16 points."""
    c, k = macrocycle()
    return jk_workload("macrocycle 445 AO, 128 densities", c, k, seed=3, npair=8, nlap=16,
                       nocc=86, tau=1e-12)


def small_chain(n_heavy: int, n_h: int, seed: int, npair: int = 1, nlap: int = 4,
                tau: float = 0.0) -> JKWorkload:
    """Small chain for parity tests the oracle finishes in seconds."""
    c, k = chain(n_heavy, n_h)
    rng_seed = 1000 + seed
    w = jk_workload(f"chain {n_heavy}+{n_h}", c, k, seed=rng_seed, npair=npair, nlap=nlap,
                    tau=tau)
    return w


def water_tz(seed: int = 11, npair: int = 1, nlap: int = 4, tau: float = 0.0) -> JKWorkload:
    """65-AO water-like molecule in the f-shell basis (O-like 4s3p2d1f, two H 3s2p1d)."""
    c, k = water_like()
    return jk_workload("water-like f-shell 65 AO", c, k, seed=seed, npair=npair, nlap=nlap, tau=tau,
                       tz=True)


def small_chain_tz(n_heavy: int, n_h: int, seed: int, npair: int = 1, nlap: int = 4,
                   tau: float = 0.0) -> JKWorkload:
    """Small f-shell chain for parity tests."""
    c, k = chain(n_heavy, n_h)
    return jk_workload(f"f-shell chain {n_heavy}+{n_h}", c, k, seed=2000 + seed, npair=npair, nlap=nlap,
                       tau=tau, tz=True)


def config_fshell() -> JKWorkload:
    """200-AO f-shell chain: 4 heavy 4s3p2d1f + 4 H 3s2p1d, 3 pairs x 16 points."""
    c, k = chain(4)
    return jk_workload("f-shell chain 200 AO, 48 densities", c, k, seed=6, npair=3, nlap=16,
                       tau=1e-12, tz=True)


@dataclasses.dataclass
class GradWorkload:
    name: str
    mol: Molecule
    P: np.ndarray   # [R, N, N]
    Q: np.ndarray   # [R, N, N]
    cJ: float
    cK: float
    schwarz_tau: float


def _sym_terms(rng, R, N):
    A = rng.standard_normal((R, N, N))
    B = rng.standard_normal((R, N, N))
    return 0.5 * (A + A.transpose(0, 2, 1)), 0.5 * (B + B.transpose(0, 2, 1))


def grad_workload(name, coords, kinds, seed, R, cJ=1.0, cK=0.0, tau=1e-12,
                  symmetric=True, tz=False) -> GradWorkload:
    rng = np.random.default_rng(seed)
    bases = draw_tz_bases(rng) if tz else draw_kind_bases(rng)
    if tz:
        kinds = tz_kinds(kinds)
    mol = build_molecule(coords, kinds, bases)
    N = mol.nao
    # same draw order as the J/K workloads up to X, so the geometry/basis agree
    _mo_part(rng, mol, mol.nelec // 2, 1)
    if symmetric:
        P, Q = _sym_terms(rng, R, N)
    else:
        P = rng.standard_normal((R, N, N))
        Q = rng.standard_normal((R, N, N))
    return GradWorkload(name, mol, P, Q, cJ, cK, tau)


def config4(R: int = 16) -> GradWorkload:
    """Gradient on the 200-AO chain geometry, Gamma = sum_r P_r (x) Q_r, symmetric N(0,1)."""
    c, k = chain(10)
    return grad_workload("chain 200 AO gradient, 16 terms", c, k, seed=4, R=R, cJ=1.0, cK=0.0)


def grad_water_tz(seed: int = 12) -> GradWorkload:
    """Gradient on the 65-AO f-shell water (O-like 4s3p2d1f, two H 3s2p1d),
    two non-symmetric N(0,1) terms, cJ = 1, cK = -1/2."""
    c, k = water_like()
    return grad_workload("water-like f-shell 65 AO gradient, 2 terms", c, k, seed=seed, R=2,
                         cJ=1.0, cK=-0.5, tau=0.0, symmetric=False, tz=True)


def serving_requests(n_req: int = 256, seed: int = 5, nao_lo: int = 25, nao_hi: int = 730,
                     rate_hz: float = 50.0):
    """Request stream: AO target log-uniform in [nao_lo, nao_hi], chain molecules with
    ceil(N/20) heavy atoms and the H count chosen to land near N, 8..16 Laplace points,
    1..3 pairs, 70% J/K and 30% gradient (R = 8), Poisson arrivals at rate_hz."""
    rng = np.random.default_rng(seed)
    bases = draw_kind_bases(rng)
    t = 0.0
    reqs = []
    for i in range(n_req):
        t += rng.exponential(1.0 / rate_hz)
        target = math.exp(rng.uniform(math.log(nao_lo), math.log(nao_hi)))
        n_heavy = max(1, math.ceil(target / 20.0))
        n_h = int(min(n_heavy, max(0, round((target - 15 * n_heavy) / 5.0))))
        coords, kinds = chain(n_heavy, n_h)
        mol = build_molecule(coords, kinds, bases)
        kind = "jk" if rng.random() < 0.7 else "grad"
        nlap = int(rng.integers(8, 17))
        npair = int(rng.integers(1, 4))
        reqs.append(dict(index=i, arrival=t, mol=mol, kind=kind, nlap=nlap, npair=npair,
                         seed=int(rng.integers(0, 2**31 - 1))))
    return reqs


def request_inputs(req) -> dict:
    """Draw the per-request arrays (MO data or gradient terms) from the request's seed."""
    rng = np.random.default_rng(req["seed"])
    mol = req["mol"]
    N = mol.nao
    nocc = max(1, min(N - 1, mol.nelec // 2))
    nvir, C, eo, ev, X = _mo_part(rng, mol, nocc, req["npair"])
    out = dict(nocc=nocc, nvir=nvir, C=C, eps_occ=eo, eps_vir=ev, X=X)
    if req["kind"] == "grad":
        P, Q = _sym_terms(rng, 8, N)
        out.update(P=P, Q=Q)
    return out
