"""Seeded synthetic inputs shared by the CPU oracle tests and the CUDA path.

This module holds workload parameters and random numbers only.  It contains no
discretization arithmetic (no quadrature, no basis functions, no mass matrix,
no Hamiltonian): both sides compute those themselves from the parameters here.

The workloads are synthetic stand-ins for the molecules of the paper's results
section (Sec. VII): hexahedral meshes, spectral elements of degree 4-8,
doubly occupied orbitals, a weak delta kick (Sec. VII.A) and Krylov tolerances
in the range the paper uses (Table "simulation parameters").
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class SystemConfig:
    """One TDKS workload: mesh, basis degree, nuclei and propagation settings."""

    name: str
    X: np.ndarray              # element breakpoints along x (nx+1)
    Y: np.ndarray              # element breakpoints along y (ny+1)
    Z: np.ndarray              # element breakpoints along z (nz+1)
    p: int                     # polynomial degree of the spectral elements
    n_orb: int                 # number of orbitals
    occ: np.ndarray            # occupation per orbital (2.0: spin-unpolarized)
    atom_R: np.ndarray         # (n_atoms, 3) positions in bohr
    atom_Z: np.ndarray         # (n_atoms,) charges
    nuc_kind: str              # 'soft' | 'erf' | 'bare' | 'harmonic' | 'none'
    nuc_param: float           # soft: a^2; erf: r_c; harmonic: omega
    hartree: bool = True
    xc: bool = True
    kick: float = 0.0          # delta-kick strength kappa
    kick_dir: tuple = (0.0, 0.0, 1.0)
    dt: float = 0.05
    n_steps: int = 100
    tol: float = 1e-10
    k_max: int = 64
    nq: int = 0                # Gauss points per direction; 0 -> p+1
    seed: Optional[int] = None

    @property
    def nx(self) -> int:
        return len(self.X) - 1

    @property
    def ny(self) -> int:
        return len(self.Y) - 1

    @property
    def nz(self) -> int:
        return len(self.Z) - 1

    @property
    def n_elem(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_int_axes(self) -> tuple:
        """Interior (Dirichlet-free) node counts per axis, x first."""
        p = self.p
        return (self.nx * p - 1, self.ny * p - 1, self.nz * p - 1)

    @property
    def n_int(self) -> int:
        a, b, c = self.n_int_axes
        return a * b * c

    @property
    def nq_eff(self) -> int:
        return self.nq if self.nq > 0 else self.p + 1


def uniform_breaks(lo: float, hi: float, n: int) -> np.ndarray:
    return np.linspace(lo, hi, n + 1)


def graded_breaks(half_width: float, n_side: int, ratio: float) -> np.ndarray:
    """Breakpoints symmetric about 0: n_side intervals per side, sizes growing by
    `ratio` outward from the origin and summing to `half_width`."""
    h0 = half_width * (ratio - 1.0) / (ratio ** n_side - 1.0)
    sizes = h0 * ratio ** np.arange(n_side)
    right = np.concatenate([[0.0], np.cumsum(sizes)])
    right[-1] = half_width
    return np.concatenate([-right[::-1], right[1:]])


def seeded_atoms(n_atoms: int, radius: float, min_sep: float, seed: int) -> np.ndarray:
    """Positions drawn uniformly in a ball by rejection, with a minimum separation."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n_atoms:
        c = rng.uniform(-radius, radius, size=3)
        if np.dot(c, c) > radius * radius:
            continue
        if all(np.linalg.norm(c - q) >= min_sep for q in pts):
            pts.append(c)
    return np.array(pts)


def config1() -> SystemConfig:
    """2-electron atom-like system, soft-Coulomb Z=2, 6^3 elements, p=4."""
    b = uniform_breaks(-10.0, 10.0, 6)
    return SystemConfig(
        name="atom_soft_Z2_6x6x6_p4", X=b, Y=b.copy(), Z=b.copy(), p=4, n_orb=1,
        occ=np.array([2.0]), atom_R=np.zeros((1, 3)), atom_Z=np.array([2.0]),
        nuc_kind="soft", nuc_param=0.5, kick=1e-3, kick_dir=(0.0, 0.0, 1.0),
        dt=0.05, n_steps=100, tol=1e-10, k_max=64)


CONFIG2_SEED = 18101302


def config2() -> SystemConfig:
    """8-atom pseudopotential-like molecule, 16^3 elements, p=6, 16 orbitals."""
    b = uniform_breaks(-16.0, 16.0, 16)
    R = seeded_atoms(8, 6.0, 1.5, CONFIG2_SEED)
    return SystemConfig(
        name="molecule_erf8_16x16x16_p6", X=b, Y=b.copy(), Z=b.copy(), p=6, n_orb=16,
        occ=np.full(16, 2.0), atom_R=R, atom_Z=np.full(8, 4.0),
        nuc_kind="erf", nuc_param=0.8, kick=1e-3, kick_dir=(1.0, 0.0, 0.0),
        dt=0.1, n_steps=500, tol=1e-10, k_max=64, seed=CONFIG2_SEED)


MID_SEED = 18101306


def config_mid() -> SystemConfig:
    """Mid-size multi-orbital molecule: the structure of config2 (erf pseudopotential
    atoms with Z_v = 4, 2-bohr hexahedra, p = 6, Hartree + LDA, kick along x, dt 0.1)
    on [-8,8]^3 with 8^3 elements (103,823 DoF), 4 atoms in a 3-bohr ball and 8
    orbitals (16 electrons, neutral).  The oracle can propagate it for tens of steps."""
    b = uniform_breaks(-8.0, 8.0, 8)
    R = seeded_atoms(4, 3.0, 1.5, MID_SEED)
    return SystemConfig(
        name="molecule_erf4_8x8x8_p6", X=b, Y=b.copy(), Z=b.copy(), p=6, n_orb=8,
        occ=np.full(8, 2.0), atom_R=R, atom_Z=np.full(4, 4.0),
        nuc_kind="erf", nuc_param=0.8, kick=1e-3, kick_dir=(1.0, 0.0, 0.0),
        dt=0.1, n_steps=50, tol=1e-10, k_max=64, seed=MID_SEED)


def config3() -> SystemConfig:
    """All-electron-like CH4 stand-in on a geometrically graded 24^3 mesh, p=8."""
    b = graded_breaks(20.0, 12, 1.25)
    d = 2.05 / math.sqrt(3.0)
    R = np.array([[0, 0, 0], [d, d, d], [d, -d, -d], [-d, d, -d], [-d, -d, d]], float)
    return SystemConfig(
        name="ch4_bare_graded24_p8", X=b, Y=b.copy(), Z=b.copy(), p=8, n_orb=5,
        occ=np.full(5, 2.0), atom_R=R, atom_Z=np.array([6.0, 1, 1, 1, 1]),
        nuc_kind="bare", nuc_param=0.0, kick=1e-3, kick_dir=(1.0, 0.0, 0.0),
        dt=0.01, n_steps=1000, tol=1e-10, k_max=64)


@dataclasses.dataclass
class PulseConfig:
    """A train of Gaussian-envelope laser pulses along `direction`:
    E(t) = sum_j a_j exp(-(t - t_j)^2 / (2 sigma^2)) sin(omega t + phi_j)."""
    omega: float
    sigma: float
    centers: np.ndarray
    a: np.ndarray
    phi: np.ndarray
    direction: tuple
    n_steps: int
    dt: float
    ckpt_every: int
    fd_h: float

    @property
    def params(self) -> np.ndarray:
        """The 2 n_pulses parameters (a_1.., phi_1..)."""
        return np.concatenate([self.a, self.phi])

    def objective_weights(self) -> np.ndarray:
        """Trapezoid weights of int d(t)^2 dt over the n_steps + 1 dipole samples."""
        w = np.full(self.n_steps + 1, self.dt)
        w[0] = w[-1] = 0.5 * self.dt
        return w


PULSE_SEED = 18101304


def config4():
    """The atom of config1 driven by four seeded Gaussian pulses (no kick), 200 steps."""
    sc = config1()
    sc.name = "atom_soft_Z2_6x6x6_p4_pulses"
    sc.kick = 0.0
    sc.dt = 0.1
    sc.n_steps = 200
    rng = np.random.default_rng(PULSE_SEED)
    pc = PulseConfig(omega=0.3, sigma=5.0, centers=np.array([4.0, 8.0, 12.0, 16.0]),
                     a=rng.uniform(0.5e-3, 1.5e-3, size=4), phi=rng.uniform(0.0, 2 * math.pi, size=4),
                     direction=(0.0, 0.0, 1.0), n_steps=200, dt=0.1, ckpt_every=20, fd_h=1e-5)
    return sc, pc


def pulse_samples(params, pc: PulseConfig):
    """Field samples of the predictor-corrector steps, [n_steps, 6]: E at t_n + dt/4
    then at t_n + dt/2 (t_n = n dt).  params = (a_1.., phi_1..) as a numpy array or a
    float64 torch tensor (differentiable)."""
    n_p = len(pc.centers)
    t = np.arange(pc.n_steps) * pc.dt
    tt = np.stack([t + 0.25 * pc.dt, t + 0.5 * pc.dt], axis=1)          # [n, 2]
    d = np.asarray(pc.direction, float)
    try:
        import torch
        is_t = isinstance(params, torch.Tensor)
    except ImportError:
        is_t = False
    if is_t:
        a, ph = params[:n_p], params[n_p:]
        T = torch.as_tensor(tt, dtype=params.dtype, device=params.device)[..., None]
        c = torch.as_tensor(pc.centers, dtype=params.dtype, device=params.device)
        env = torch.exp(-(T - c) ** 2 / (2 * pc.sigma ** 2))
        e = (a * env * torch.sin(pc.omega * T + ph)).sum(-1)            # [n, 2]
        D = torch.as_tensor(d, dtype=params.dtype, device=params.device)
        return (e[..., None] * D).reshape(pc.n_steps, 6)
    params = np.asarray(params, float)
    a, ph = params[:n_p], params[n_p:]
    T = tt[..., None]
    env = np.exp(-(T - pc.centers) ** 2 / (2 * pc.sigma ** 2))
    e = (a * env * np.sin(pc.omega * T + ph)).sum(-1)
    return (e[..., None] * d).reshape(pc.n_steps, 6)


@dataclasses.dataclass
class KBParams:
    """Synthetic Kleinman-Bylander projectors (stand-ins for tabulated pseudopotential
    data) on every atom of a system: u_lm = exp(-d^2/(2 a^2)) Y_lm(d), Y_00 = 1,
    Y_1m = d_x, d_y, d_z; dV_l = c_l exp(-d^2/(2 b^2)); l = 0..lmax."""
    a: float = 1.0
    b: float = 0.8
    c: tuple = (-2.0, -1.0)
    lmax: int = 1


BATCH_SEED = 18101305


def config5(n_sys: int = 64, seed: int = BATCH_SEED):
    """Batch of independent systems of uneven size: n^3 elements (n in 4..12, 2 bohr
    wide), p in 4..8, 1-8 doubly occupied orbitals, 1-4 soft-Coulomb nuclei (Z in
    1..4) inside a third of the box, own kick direction, dt in {0.02, 0.05, 0.1}.
    Returns (configs, dts, kick directions)."""
    rng = np.random.default_rng(seed)
    cfgs, dts, dirs = [], [], []
    for k in range(n_sys):
        n = int(rng.integers(4, 13))
        p = int(rng.integers(4, 9))
        n_orb = int(rng.integers(1, 9))
        n_nuc = int(rng.integers(1, 5))
        L = float(n)
        b = uniform_breaks(-L, L, n)
        R = rng.uniform(-L / 3, L / 3, size=(n_nuc, 3))
        Z = rng.integers(1, 5, size=n_nuc).astype(float)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        cfgs.append(SystemConfig(
            name=f"batch{k}_{n}^3_p{p}_o{n_orb}", X=b, Y=b.copy(), Z=b.copy(), p=p, n_orb=n_orb,
            occ=np.full(n_orb, 2.0), atom_R=R, atom_Z=Z, nuc_kind="soft", nuc_param=0.5,
            kick=1e-3, kick_dir=tuple(d), dt=float(rng.choice([0.02, 0.05, 0.1])), n_steps=200,
            tol=1e-10, k_max=64, seed=seed + k))
        dts.append(cfgs[-1].dt)
        dirs.append(d)
    return cfgs, np.array(dts), np.array(dirs)


def small_batch(seed: int = 11):
    """A few small uneven systems (degrees 2-5, 1-3 orbitals, own time steps) for
    parity tests of the batched path."""
    rng = np.random.default_rng(seed)
    specs = [((3, 2, 2), 3, 2, 0.05), ((2, 2, 2), 2, 1, 0.1), ((2, 3, 2), 4, 3, 0.02),
             ((2, 2, 3), 5, 1, 0.05), ((3, 3, 2), 3, 2, 0.1)]
    cfgs = []
    for k, (n, p, no, dt) in enumerate(specs):
        c = small_config(*n, p=p, n_orb=no, seed=seed + k)
        c.dt = dt
        d = rng.standard_normal(3)
        c.kick_dir = tuple(d / np.linalg.norm(d))
        cfgs.append(c)
    return cfgs


def small_config(nx=3, ny=2, nz=2, p=3, n_orb=2, L=6.0, seed=7, nuc_kind="soft",
                 hartree=True, xc=True, graded=False) -> SystemConfig:
    """A small test system with uneven element counts and (optionally) uneven sizes."""
    rng = np.random.default_rng(seed)

    def axis(n):
        if not graded:
            return uniform_breaks(-L, L, n)
        w = rng.uniform(0.6, 1.4, size=n)
        return np.concatenate([[-L], -L + 2 * L * np.cumsum(w) / w.sum()])

    return SystemConfig(
        name=f"small_{nx}x{ny}x{nz}_p{p}", X=axis(nx), Y=axis(ny), Z=axis(nz), p=p,
        n_orb=n_orb, occ=np.full(n_orb, 2.0), atom_R=np.array([[0.3, -0.2, 0.1]]),
        atom_Z=np.array([1.0 * n_orb]), nuc_kind=nuc_kind, nuc_param=0.5,
        hartree=hartree, xc=xc, kick=1e-3, kick_dir=(0.0, 0.0, 1.0), dt=0.05,
        n_steps=4, tol=1e-10, k_max=64, seed=seed)


# ----------------------------------------------------------------------------
# Random and smooth input vectors
# ----------------------------------------------------------------------------

def random_psi(n_orb: int, n: int, seed: int) -> np.ndarray:
    """Complex Gaussian random orbitals, each scaled to unit Euclidean norm."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n_orb, n)) + 1j * rng.standard_normal((n_orb, n))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    return a


def random_potential(n: int, seed: int, lo: float = -3.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n)


def smooth_orbitals(n_int_axes: tuple, n_orb: int, seed: int) -> np.ndarray:
    """Orthonormal orbitals that are smooth functions of the interior node index.

    Each orbital is a seeded combination of Gaussians in normalized index
    coordinates s_d = (i_d+1)/(n_d+1) in (0, 1), times low-order polynomials,
    vanishing towards the boundary.  The block is orthonormalized with a
    Householder QR (plain linear algebra on the input vectors).
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = n_int_axes
    sx = (np.arange(nx) + 1.0) / (nx + 1.0)
    sy = (np.arange(ny) + 1.0) / (ny + 1.0)
    sz = (np.arange(nz) + 1.0) / (nz + 1.0)
    S = np.meshgrid(sx, sy, sz, indexing="ij")
    cols = []
    for a in range(n_orb):
        c = rng.uniform(0.4, 0.6, size=3)
        w = rng.uniform(0.07, 0.12)
        r2 = sum((S[d] - c[d]) ** 2 for d in range(3))
        poly = 1.0 + sum(rng.uniform(-3, 3) * (S[d] - c[d]) for d in range(3))
        phase = np.exp(1j * rng.uniform(-2, 2) * (S[0] - c[0]))
        f = np.exp(-r2 / (2 * w * w)) * poly * phase
        # x fastest in memory: transpose (x, y, z) -> (z, y, x) before ravel
        cols.append(np.transpose(f, (2, 1, 0)).ravel())
    A = np.array(cols).T
    Q, _ = np.linalg.qr(A)
    return np.ascontiguousarray(Q.T)
