"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA library.

This module holds no arithmetic of the method itself (no basis functions, no
quadrature, no Hamiltonian): only counter-based random numbers and the
analytic model functions (Gaussian wells, Gaussian projectors) that stand in
for the paper's pseudopotential data, evaluated at points that the caller
supplies from its own mesh.

Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used two ways:
  * counter mode  u(seed, idx) = mix(seed + (idx + 1) * GAMMA) -> [-1/2, 1/2)
    for the initial block X0 (element (i, j) uses idx = i * ncol + j) and the
    Lanczos start vector;
  * stream mode   state += GAMMA; next = mix(state), seeded with
    seed ^ 0xA5A5A5A5A5A5A5A5, for atom positions, jitter and projector
    couplings, drawn in the order: atoms (x, y, z each), then couplings
    (atom-major, projector-minor).
"""
import math
import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1
STREAM_XOR = 0xA5A5A5A5A5A5A5A5


def _mix_u64(z):
    """SplitMix64 finaliser on a numpy uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _mix_int(z):
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def counter_uniform(seed, count, offset=0):
    """u(seed, idx) for idx in [offset, offset+count): values in [-1/2, 1/2)."""
    idx = np.arange(offset, offset + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK) + (idx + np.uint64(1)) * np.uint64(GAMMA)
    z = _mix_u64(z)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 0.5


def random_block(seed, nrow, ncol):
    """Initial block X0 (nrow x ncol, row-major): X0[i, j] = u(seed, i*ncol + j)."""
    out = np.empty((nrow, ncol), dtype=np.float64)
    chunk = max(1, (1 << 24) // max(ncol, 1))
    for r0 in range(0, nrow, chunk):
        r1 = min(nrow, r0 + chunk)
        out[r0:r1] = counter_uniform(seed, (r1 - r0) * ncol, r0 * ncol).reshape(r1 - r0, ncol)
    return out


def random_rows(seed, rows, ncol):
    """Rows `rows` of the block random_block(seed, nrow, ncol), without forming the rest."""
    rows = np.asarray(rows, dtype=np.uint64)
    idx = (rows[:, None] * np.uint64(ncol) + np.arange(ncol, dtype=np.uint64)[None, :]).ravel()
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK) + (idx + np.uint64(1)) * np.uint64(GAMMA)
    z = _mix_u64(z)
    return ((z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 0.5).reshape(len(rows), ncol)


class Stream:
    """Sequential SplitMix64 stream; uniform() returns values in [0, 1)."""

    def __init__(self, seed):
        self.state = (seed ^ STREAM_XOR) & MASK

    def next_u64(self):
        self.state = (self.state + GAMMA) & MASK
        return _mix_int(self.state)

    def uniform(self):
        return (self.next_u64() >> 11) * (2.0 ** -53)


# --------------------------------------------------------------------------
# Workload recipes (the synthetic stand-ins for the paper's Mo/Al systems)
# --------------------------------------------------------------------------

class Workload:
    """A periodic cube with Gaussian wells and (optionally) Gaussian projectors."""

    def __init__(self, name, L, ncell, degree, depth, width, centres,
                 nstates, block, cheb_degree, passes, seed,
                 proj_width=None, proj_cutoff=None, couplings=None):
        self.name = name
        self.L = float(L)
        self.ncell = int(ncell)
        self.degree = int(degree)
        self.depth = float(depth)
        self.width = float(width)
        self.centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
        self.nstates = nstates
        self.block = block
        self.cheb_degree = cheb_degree
        self.passes = passes
        self.seed = seed
        self.proj_width = proj_width
        self.proj_cutoff = proj_cutoff
        self.couplings = None if couplings is None else np.asarray(couplings, np.float64)

    @property
    def ndofs(self):
        return (self.ncell * self.degree) ** 3

    @property
    def nproj(self):
        return 0 if self.couplings is None else self.couplings.size


def small_wells(seed=0, ncell=6, degree=4, nstates=32, block=32, cheb_degree=20, passes=10):
    """Plain FP64 system: 10 bohr cube, 6^3 cells, p=4 (13,824 DoFs), 8 wells of
    depth 2 Ha and width 1 bohr at centres uniform in the box; no projectors."""
    s = Stream(seed)
    L = 10.0
    centres = [[L * s.uniform() for _ in range(3)] for _ in range(8)]
    return Workload("wells8-L10-6c-p4", L, ncell, degree, 2.0, 1.0, centres,
                    nstates, block, cheb_degree, passes, seed)


def lattice_atoms(seed=0, ncell=24, degree=6, nstates=512, block=128, cheb_degree=40, passes=5,
                  L=30.0, nside=4):
    """FP64 system at scale: 30 bohr cube, 24^3 cells, p=6 (2,985,984 DoFs),
    64 wells (depth 3 Ha, width 0.8 bohr) at (i+1/2)*7.5 bohr lattice sites
    jittered by U[-1/2, 1/2] bohr per coordinate, 4 projectors per atom
    (s and three p, Gaussian radial width 1 bohr, cutoff 3 bohr) with
    couplings U[0.5, 2] Ha."""
    s = Stream(seed)
    a = L / nside
    centres = []
    for k in range(nside):
        for j in range(nside):
            for i in range(nside):
                base = ((i + 0.5) * a, (j + 0.5) * a, (k + 0.5) * a)
                centres.append([base[d] + (s.uniform() - 0.5) for d in range(3)])
    couplings = np.array([[0.5 + 1.5 * s.uniform() for _ in range(4)]
                          for _ in range(len(centres))])
    return Workload(f"wells{len(centres)}-L{L:g}-{ncell}c-p{degree}-nl", L, ncell, degree, 3.0, 0.8,
                    centres, nstates, block, cheb_degree, passes, seed,
                    proj_width=1.0, proj_cutoff=3.0, couplings=couplings.ravel())


def _wrap(d, L):
    return d - L * np.round(d / L)


def gaussian_wells(points, centres, depth, width, L):
    """V(x) = -depth * sum_atoms sum_images exp(-|x - R - L n|^2 / (2 width^2)),
    images with |x - R - L n| < 8 width; points is (n, 3)."""
    pts = np.asarray(points, dtype=np.float64)
    v = np.zeros(pts.shape[0])
    rcut = 8.0 * width
    # after the minimum-image wrap every other image is at least L/2 away (L: scalar or
    # one length per axis)
    Lv = np.broadcast_to(np.asarray(L, np.float64), (3,))
    k = [0 if rcut <= 0.5 * Ld else int(math.ceil((rcut + 0.5 * Ld) / Ld)) for Ld in Lv]
    shifts = [(i, j, l) for i in range(-k[0], k[0] + 1) for j in range(-k[1], k[1] + 1)
              for l in range(-k[2], k[2] + 1)]
    L = np.asarray(L, np.float64)
    for R in centres:
        d0 = _wrap(pts - R, L)
        for sh in shifts:
            d = d0 - L * np.asarray(sh, dtype=np.float64)
            r2 = np.einsum("ij,ij->i", d, d)
            m = r2 < rcut * rcut
            v[m] -= depth * np.exp(-r2[m] / (2.0 * width * width))
    return v


def harmonic(points, centre, omega, L):
    """V(x) = omega^2 |x - c|^2 / 2 with the minimum-image distance."""
    d = _wrap(np.asarray(points, np.float64) - np.asarray(centre, np.float64), L)
    return 0.5 * omega * omega * np.einsum("ij,ij->i", d, d)


def projector_csr(node_xyz, centres, width, cutoff, L):
    """Projector values at mesh nodes, CSR by projector.

    Per atom, four projectors in the order s, p_x, p_y, p_z:
      chi_s  = g(r) / (pi w^2)^(3/4),
      chi_pm = (x_m / w) g(r) / sqrt((pi w^2)^(3/2) / 2),   g = exp(-r^2 / (2 w^2)),
    each normalised analytically over R^3 and cut off hard at r < cutoff
    (minimum-image displacement; L a scalar or one length per axis).
    Returns (rowptr int64, node int64, chi f64).
    """
    xyz = np.asarray(node_xyz, np.float64)
    n_s = (math.pi * width * width) ** 0.75
    n_p = math.sqrt(0.5 * (math.pi * width * width) ** 1.5)
    rowptr = [0]
    nodes, vals = [], []
    L = np.asarray(L, np.float64)
    for R in centres:
        d = _wrap(xyz - np.asarray(R), L)
        r2 = np.einsum("ij,ij->i", d, d)
        idx = np.nonzero(r2 < cutoff * cutoff)[0]
        g = np.exp(-r2[idx] / (2.0 * width * width))
        comps = [g / n_s] + [(d[idx, m] / width) * g / n_p for m in range(3)]
        for c in comps:
            nodes.append(idx.astype(np.int64))
            vals.append(c)
            rowptr.append(rowptr[-1] + idx.size)
    if not nodes:
        return np.zeros(1, np.int64), np.zeros(0, np.int64), np.zeros(0)
    return (np.asarray(rowptr, np.int64), np.concatenate(nodes), np.concatenate(vals))


def projector_disp(node_xyz, centres, cutoff, L):
    """Minimum-image displacement x_node - R_atom (nnz x 3) of every entry of
    projector_csr(node_xyz, centres, ..., cutoff, L), in the same order."""
    xyz = np.asarray(node_xyz, np.float64)
    L = np.asarray(L, np.float64)
    out = []
    for R in centres:
        d = _wrap(xyz - np.asarray(R), L)
        idx = np.nonzero(np.einsum("ij,ij->i", d, d) < cutoff * cutoff)[0]
        out.extend([d[idx]] * 4)
    return np.concatenate(out) if out else np.zeros((0, 3))


def atom_walk(seed, centres, steps, step_len=0.05):
    """Positions of an SCF-like sequence: at every step each atom moves by `step_len` bohr in a
    direction drawn uniformly on the sphere (seeded stream); returns steps + 1 arrays (the
    first is `centres`).  Input generation only: the caller mixes the potentials."""
    s = Stream(seed)
    pos = [np.asarray(centres, dtype=np.float64).copy()]
    for _ in range(steps):
        nxt = pos[-1].copy()
        for a in range(nxt.shape[0]):
            z = 2.0 * s.uniform() - 1.0
            phi = 2.0 * math.pi * s.uniform()
            r = math.sqrt(max(0.0, 1.0 - z * z))
            nxt[a] += step_len * np.array([r * math.cos(phi), r * math.sin(phi), z])
        pos.append(nxt)
    return pos


# (cells per axis, FE degree, states, atoms, Chebyshev degree) of the sixteen systems of the
# batched k-point workload: meshes of 8^3 to 20^3 cells, p = 4 to 6, 64 to 768 states,
# 8 to 48 atoms, degrees 20 to 40 (the larger state counts on the smaller meshes, so that
# every system's 8 k-points fit on one device together)
KPOINT_BATCH = [(8, 6, 768, 8, 40), (8, 5, 512, 10, 36), (8, 4, 640, 12, 32), (9, 6, 384, 14, 40),
                (10, 6, 192, 16, 36), (10, 5, 320, 12, 32), (10, 4, 448, 18, 28), (11, 5, 160, 20, 30),
                (12, 4, 256, 22, 26), (12, 5, 96, 24, 28), (13, 4, 160, 28, 24), (14, 4, 128, 32, 22),
                (15, 4, 96, 36, 22), (16, 4, 80, 40, 20), (18, 4, 64, 44, 20), (20, 4, 64, 48, 20)]
# cell edge by FE degree: about 0.21 bohr between nodes at every degree
KPOINT_BATCH_CELL = {4: 0.85, 5: 1.05, 6: 1.25}


def kpoint_batch(seed=0, systems=None):
    """The batched k-point workload: one Workload per system (atoms of depth 3 Ha and width
    0.8 bohr at centres uniform in the box, 4 projectors per atom of width 1 bohr and cutoff
    2.5 bohr with couplings U[0.5, 2] Ha, complex block 64) with its 8 k-points, the 2 x 2 x 2
    Monkhorst-Pack grid (2 pi / L)(+-1/4, +-1/4, +-1/4) in bohr^-1.  Returns a list of
    (Workload, kpoints)."""
    out = []
    for i, (n, p, N, natoms, deg) in enumerate(KPOINT_BATCH if systems is None else systems):
        s = Stream(seed * 1000 + i)
        L = n * KPOINT_BATCH_CELL[p]
        centres = [[L * s.uniform() for _ in range(3)] for _ in range(natoms)]
        couplings = np.array([0.5 + 1.5 * s.uniform() for _ in range(4 * natoms)])
        wl = Workload(f"kbatch{i}-{n}c-p{p}-N{N}", L, n, p, 3.0, 0.8, centres, N, 64, deg, 1, seed * 1000 + i,
                      proj_width=1.0, proj_cutoff=2.5, couplings=couplings)
        g = 2.0 * math.pi / L
        kpts = [(g * a / 4.0, g * b / 4.0, g * c / 4.0) for a in (-1, 1) for b in (-1, 1) for c in (-1, 1)]
        out.append((wl, kpts))
    return out
