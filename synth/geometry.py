"""Seeded synthetic geometries (Angstrom) for the five workloads.

Nothing here computes anything of the method: atoms are placed by rejection
sampling with distance constraints only.

* ``c4h6(seed)``            -- C4H6: random bonded C tree + 6 H (10 atoms, 22 sp orbitals)
* ``carbon_packing(seed)``  -- 840 C by random sequential addition at 2.2 g/cc, open box
* ``organic_molecule``      -- C/N/O heavy-atom tree filled with H (batch workload)
* ``molecule_batch(seed)``  -- 128 molecules with 12..200 atoms
* ``carbon_fragments(seed)``-- 400 C as chains plus graphene-like sheet fragments
* ``fullerene_c60(...)``    -- truncated-icosahedron C60 cages (closed, no dangling bonds)
* ``serving_requests``      -- Poisson arrival times, sizes and step counts
"""
from dataclasses import dataclass
import numpy as np

VALENCE = {1: 1, 6: 4, 7: 3, 8: 2}
ZCORE = {1: 1, 6: 4, 7: 5, 8: 6}


@dataclass
class Molecule:
    Z: np.ndarray        # (N,) int32 atomic numbers
    R: np.ndarray        # (N, 3) float64 positions, Angstrom
    charge: int = 0

    @property
    def natoms(self):
        return len(self.Z)

    @property
    def norb(self):
        return int(sum(1 if z == 1 else 4 for z in self.Z))

    @property
    def nelec(self):
        return int(sum(ZCORE[int(z)] for z in self.Z)) - self.charge


def _rng(tag, seed):
    return np.random.default_rng(np.random.SeedSequence([tag, seed]))


def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _grow_tree(rng, Zheavy, bond=(1.30, 1.55), nonbond=2.0, tries=20000):
    """Place heavy atoms one by one, each bonded to a random earlier atom."""
    pos = [np.zeros(3)]
    nbr = [0]
    for i in range(1, len(Zheavy)):
        for _ in range(tries):
            j = int(rng.integers(0, i))
            if nbr[j] >= VALENCE[int(Zheavy[j])] or nbr[j] >= 3:
                continue
            p = pos[j] + rng.uniform(*bond) * _unit(rng)
            d = np.linalg.norm(np.array(pos) - p, axis=1)
            d[j] = np.inf
            if d.min() >= nonbond:
                pos.append(p)
                nbr[j] += 1
                nbr.append(1)
                break
        else:
            raise RuntimeError("tree growth failed")
    return np.array(pos), nbr


def _add_hydrogens(rng, Zheavy, pos, nbr, nH, dist=1.09, tries=20000):
    """Attach nH hydrogens at 1.09 A to heavy atoms with free valence."""
    allpos = [p for p in pos]
    free = [VALENCE[int(z)] - k for z, k in zip(Zheavy, nbr)]
    Hs = []
    for _ in range(nH):
        cand = [i for i, f in enumerate(free) if f > 0]
        if not cand:
            cand = list(range(len(Zheavy)))
        for _ in range(tries):
            j = int(cand[rng.integers(0, len(cand))])
            p = pos[j] + dist * _unit(rng)
            d = np.linalg.norm(np.array(allpos) - p, axis=1)
            d[j] = np.inf
            if d.min() >= 1.6:
                allpos.append(p)
                Hs.append(p)
                free[j] -= 1
                break
        else:
            raise RuntimeError("hydrogen placement failed")
    return np.array(Hs).reshape(-1, 3)


def c4h6(seed=1):
    """C4H6 with a random bonded carbon backbone (10 atoms, n = 22)."""
    rng = _rng(101, seed)
    Zc = np.full(4, 6)
    pos, nbr = _grow_tree(rng, Zc)
    H = _add_hydrogens(rng, Zc, pos, nbr, 6)
    Z = np.array([6] * 4 + [1] * 6, dtype=np.int32)
    R = np.vstack([pos, H])
    return Molecule(Z, R - R.mean(axis=0))


def carbon_packing(seed=2, natoms=840, density=2.2, dmin=1.3):
    """Random sequential addition of carbon atoms in an open cubic box."""
    rng = _rng(202, seed)
    side = (natoms * 12.011 * 1.66054 / density) ** (1.0 / 3.0)
    pos = np.empty((0, 3))
    while len(pos) < natoms:
        p = rng.uniform(0.0, side, size=3)
        if len(pos) == 0 or np.min(np.sum((pos - p) ** 2, axis=1)) >= dmin * dmin:
            pos = np.vstack([pos, p])
    Z = np.full(natoms, 6, dtype=np.int32)
    return Molecule(Z, pos - pos.mean(axis=0))


def organic_molecule(rng, natoms):
    """C/N/O tree (60/20/20 %) covering ~55 % of atoms, the rest hydrogen."""
    nheavy = max(1, int(round(0.55 * natoms)))
    nH = natoms - nheavy
    Zh = rng.choice([6, 7, 8], size=nheavy, p=[0.6, 0.2, 0.2]).astype(np.int32)
    Zh[0] = 6
    pos, nbr = _grow_tree(rng, Zh)
    H = _add_hydrogens(rng, Zh, pos, nbr, nH)
    Z = np.concatenate([Zh, np.ones(len(H), dtype=np.int32)])
    R = np.vstack([pos, H])
    if sum(ZCORE[int(z)] for z in Z) % 2:        # closed shell: even electron count
        if nH > 0:
            Z, R = Z[:-1], R[:-1]
        else:
            Z = np.concatenate([Z, [1]]).astype(np.int32)
            R = np.vstack([R, R[-1] + np.array([1.09, 0.0, 0.0])])
    return Molecule(Z.astype(np.int32), R - R.mean(axis=0))


def molecule_batch(seed=3, count=128, nmin=12, nmax=200):
    rng = _rng(303, seed)
    return [organic_molecule(rng, int(rng.integers(nmin, nmax + 1))) for _ in range(count)]


def carbon_fragments(seed=5, natoms=400, spacing=6.0):
    """Carbon chains and graphene-like sheet fragments (C-C 1.40 A, no H)."""
    rng = _rng(505, seed)
    pieces = []
    left = natoms
    while left > 0:
        if rng.random() < 0.5:
            k = int(min(left, rng.integers(8, 30)))
            pts = [np.zeros(3)]
            d = _unit(rng)
            for _ in range(k - 1):
                d = d + 0.35 * _unit(rng)
                d /= np.linalg.norm(d)
                pts.append(pts[-1] + 1.40 * d)
            piece = np.array(pts)
        else:
            # hexagonal lattice patch: a = 1.40 * sqrt(3)
            nx, ny = int(rng.integers(3, 7)), int(rng.integers(3, 7))
            a1 = np.array([1.40 * np.sqrt(3.0), 0.0, 0.0])
            a2 = np.array([0.5 * 1.40 * np.sqrt(3.0), 1.5 * 1.40, 0.0])
            basis = [np.zeros(3), np.array([0.0, 1.40, 0.0])]
            pts = [i * a1 + j * a2 + b for i in range(nx) for j in range(ny) for b in basis]
            piece = np.array(pts)[: int(min(left, 2 * nx * ny))]
        pieces.append(piece)
        left -= len(piece)
    # place pieces on a loose grid with random rotations, keeping them apart
    allpos = []
    g = int(np.ceil(len(pieces) ** (1.0 / 3.0)))
    for idx, piece in enumerate(pieces):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
        c = np.array([idx % g, (idx // g) % g, idx // (g * g)], dtype=float)
        p = (piece - piece.mean(axis=0)) @ rot.T
        allpos.append(p + c * (spacing + np.ptp(p, axis=0).max()))
    R = np.vstack(allpos)[:natoms]
    Z = np.full(len(R), 6, dtype=np.int32)
    return Molecule(Z, R - R.mean(axis=0))


def _c60_unit():
    """Vertices of the truncated icosahedron with edge length 1, centred at 0.

    With edge length 2 the vertices are the even (cyclic) permutations of
    (0, +-1, +-3p), (+-1, +-(2 + p), +-2p) and (+-p, +-2, +-(2p + 1)), p the
    golden ratio."""
    p = (1.0 + 5.0 ** 0.5) / 2.0
    base = [(0.0, 1.0, 3 * p), (1.0, 2.0 + p, 2 * p), (p, 2.0, 2 * p + 1.0)]
    pts = set()
    for a, b, c in base:
        for sa in (-1, 1):
            for sb in (-1, 1):
                for sc in (-1, 1):
                    v = (sa * a, sb * b, sc * c)
                    for k in range(3):                       # cyclic permutations
                        pts.add(tuple(round(x, 12) + 0.0 for x in (v[k], v[(k + 1) % 3], v[(k + 2) % 3])))
    P = np.array(sorted(pts)) / 2.0
    assert P.shape == (60, 3)
    return P


def fullerene_c60(seed=5, copies=1, bond=1.42, spacing=12.0, charge=0):
    """``copies`` C60 cages (C-C ``bond`` Angstrom), each randomly rotated and
    jittered by 0.02 A, on a line ``spacing`` Angstrom apart."""
    rng = _rng(606, seed)
    unit = _c60_unit() * bond
    out = []
    for c in range(copies):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        Rm = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                       [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                       [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
        out.append(unit @ Rm.T + rng.normal(size=unit.shape) * 0.02 + np.array([c * spacing, 0.0, 0.0]))
    R = np.concatenate(out)
    return Molecule(np.full(len(R), 6, dtype=np.int32), R, charge=charge)


def serving_requests(seed=4, count=64, rate_per_s=1.0, nmin=20, nmax=600, smin=10, smax=100, kind="organic"):
    """Poisson arrivals of MD requests: (arrival_s, Molecule, nsteps) tuples.

    kind "organic": C/N/O/H trees of nmin..nmax atoms.  kind "fullerene":
    1..nmax/60 C60 cages (60..600 atoms) at a 1.60 A bond length."""
    rng = _rng(404, seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        if kind == "fullerene":
            k = int(rng.integers(max(1, nmin // 60), max(1, nmax // 60) + 1))
            mol = fullerene_c60(seed=int(rng.integers(1 << 30)), copies=k, bond=1.60)
        else:
            mol = organic_molecule(rng, int(rng.integers(nmin, nmax + 1)))
        out.append((t, mol, int(rng.integers(smin, smax + 1))))
    return out
